"""Pins of the oracle's pivoted incomplete Cholesky (oracle.cholesky), the
factorisation of Eq. int_fact used for the paper's Cholesky integrals.

Fixed by: numpy's Cholesky of the pivot-permuted matrix (a full-rank matrix
factorised to the end is the textbook factor), the residual bound that
defines the threshold (every remaining diagonal <= tau, hence every residual
element <= tau for a PSD residual), exact rank recovery, the zero pattern at
earlier pivots, the tie rule, and the energies of the method from the factor
against four-index integrals.
"""
import numpy as np
import pytest

import synth
from oracle import cholesky, dsrg


def _psd(n, rank, seed, scale=0.3):
    rng = np.random.default_rng(seed)
    B0 = rng.standard_normal((rank, n, n))
    B0 = scale * (B0 + np.transpose(B0, (0, 2, 1)))
    eri = np.einsum("Qpq,Qrs->pqrs", B0, B0)
    return B0, eri


def test_full_rank_equals_numpy_cholesky_of_permuted_matrix():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((40, 40))
    V = X @ X.T + 40 * np.eye(40)
    B, piv = cholesky.pivoted_cholesky(V, 0.0)
    assert sorted(piv.tolist()) == list(range(40))
    L = np.linalg.cholesky(V[np.ix_(piv, piv)])
    np.testing.assert_allclose(B[:, piv].T, L, rtol=0, atol=1e-12 * np.abs(L).max())
    # the pivot is the largest remaining diagonal: first pivot = largest diagonal
    assert piv[0] == int(np.argmax(np.diag(V)))


@pytest.mark.parametrize("tau", [1e-6, 1e-8])
def test_threshold_bounds_the_residual(tau):
    B0, eri = _psd(6, 20, seed=4)
    V = cholesky.supermatrix(eri)
    B, piv = cholesky.pivoted_cholesky(V, tau)
    R = V - B.T @ B
    assert np.diag(R).max() <= tau * (1 + 1e-6)
    assert np.abs(R).max() <= tau * (1 + 1e-6) + 1e-13
    # earlier pivots are (to rounding) zero in later vectors
    for q in range(1, len(piv)):
        assert np.abs(B[q, piv[:q]]).max() <= 1e-12 * np.abs(B).max()


def test_exact_rank_recovery():
    B0, eri = _psd(5, 7, seed=6)
    V = cholesky.supermatrix(eri)
    B, piv = cholesky.pivoted_cholesky(V, 1e-10)
    assert len(piv) == 7
    np.testing.assert_allclose(B.T @ B, V, rtol=0, atol=1e-10 * np.abs(V).max())


def test_ties_go_to_the_smallest_index():
    V = np.diag([1.0, 3.0, 2.0, 3.0, 0.5])
    B, piv = cholesky.pivoted_cholesky(V, 0.0)
    assert piv.tolist() == [1, 3, 2, 0, 4]


def test_energies_from_the_factor_equal_four_index_energies():
    """Eq. int_fact with the factor of a tight threshold reproduces the energies
    of the four-index integrals."""
    base = synth.make_instance(1, 2, 2, 3, 8, 0.5, seed=17)
    n = base["nc"] + base["na"] + base["nv"]
    B0, eri = _psd(n, 9, seed=8)
    B, piv = cholesky.pivoted_cholesky(cholesky.supermatrix(eri), 1e-12)
    Bc = B.reshape(len(piv), n, n)
    a = dsrg.dsrg_pt3(dict(base, B=Bc, naux=len(piv)))
    b = dsrg.dsrg_pt3(dict(base, B=B0, naux=9), eri=eri)
    for k in ("e2", "e3a", "e3b"):
        assert abs(a[k] - b[k]) <= 1e-11 * abs(b[k]) + 1e-14, k
