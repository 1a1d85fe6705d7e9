"""GPU pivoted incomplete Cholesky (dsrg_cholesky) against the oracle
(oracle.cholesky): the same operations in the same order, so the pivots must
agree exactly and the vectors bit for bit.  Covers integral supermatrices
with several CTAs and a ragged tail, a full-rank matrix factorised to the
end, the threshold and capacity stops, ties in the pivot search, and a
threshold above every diagonal (no vectors)."""
import numpy as np
import pytest

from oracle import cholesky

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1701_02011_gb300 import build
    build.build()
    import paper_1701_02011_gb300 as g
    g.load_library()
    return g


def _supermatrix(n, rank, seed):
    rng = np.random.default_rng(seed)
    B0 = rng.standard_normal((rank, n, n))
    B0 = 0.3 * (B0 + np.transpose(B0, (0, 2, 1)))
    return cholesky.supermatrix(np.einsum("Qpq,Qrs->pqrs", B0, B0))


def _compare(lib, V, tau, max_vecs):
    import torch
    B_ref, piv_ref = cholesky.pivoted_cholesky(V, tau, max_vecs)
    B, piv = lib.dsrg_cholesky(torch.from_numpy(V).cuda(), tau, max_vecs)
    assert piv.tolist() == piv_ref.tolist()
    assert np.array_equal(B.cpu().numpy(), B_ref)
    return len(piv)


@pytest.mark.parametrize("n,rank,tau", [(7, 20, 1e-6), (23, 60, 1e-8), (20, 40, 1e-10)])
def test_integral_supermatrix_bit_exact(lib, n, rank, tau):
    # N = n^2 = 49 (one CTA), 529 (three CTAs, ragged), 400
    nv = _compare(lib, _supermatrix(n, rank, seed=n + rank), tau, 3 * n * n)
    assert 0 < nv <= rank


def test_full_rank_and_capacity_stop(lib):
    rng = np.random.default_rng(3)
    X = rng.standard_normal((300, 300))
    V = X @ X.T + 300 * np.eye(300)
    assert _compare(lib, V, 0.0, 300) == 300   # to the end
    assert _compare(lib, V, 0.0, 37) == 37     # capacity stop


def test_ties_and_empty_result(lib):
    V = np.diag([1.0, 3.0, 2.0, 3.0, 0.5])
    assert _compare(lib, V, 0.0, 5) == 5
    assert _compare(lib, V, 5.0, 5) == 0
