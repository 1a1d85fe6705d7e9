"""Split-precision tensor-core product (dsrg_split_gemm) against exact and
FP64 references."""
import numpy as np
import pytest

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


def test_one_slice_is_exact_on_small_integers(lib):
    """|a|, |b| <= 63: one balanced 7-bit digit (|d| <= 64 on the grid of
    the row/column exponent, 2^6 for a maximum of 63) holds every element
    exactly, so the product must be exact (ragged M, N, K across tiles)."""
    import torch
    rng = np.random.default_rng(1)
    M, N, K = 200, 150, 300
    A = rng.integers(-63, 64, (M, K)).astype(np.float64)
    B = rng.integers(-63, 64, (K, N)).astype(np.float64)
    ref = (A.astype(np.int64) @ B.astype(np.int64)).astype(np.float64)
    C = torch.zeros((M, N), dtype=torch.float64, device="cuda")
    lib.dsrg_split_gemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), C, 1.0, 1)
    assert np.array_equal(C.cpu().numpy(), ref)


@pytest.mark.parametrize("slices,tol", [(3, 1e-5), (6, 1e-11), (7, 1e-13), (8, 1e-14)])
def test_many_slices_match_fp64(lib, slices, tol):
    import torch
    rng = np.random.default_rng(2)
    M, N, K = 257, 131, 700
    A = rng.standard_normal((M, K)) * np.exp(rng.uniform(-6, 6, (M, 1)))
    B = rng.standard_normal((K, N)) * np.exp(rng.uniform(-6, 6, (1, N)))
    ref = A @ B
    bound = np.abs(A).max(axis=1)[:, None] * np.abs(B).max(axis=0)[None, :] * K
    C0 = rng.standard_normal((M, N))
    C = torch.from_numpy(C0.copy()).cuda()
    lib.dsrg_split_gemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), C, -0.5, slices)
    err = np.abs(C.cpu().numpy() - (C0 - 0.5 * ref)) / bound
    assert err.max() < tol


@pytest.mark.parametrize("M,N,K", [(300, 20, 500), (60, 700, 130), (100, 40, 20000), (129, 129, 65)])
def test_tile_shapes_orientation_and_k_split(lib, M, N, K):
    """Narrow N tiles (32/64), the transposed orientation (M < N), a long K
    split over CTAs, and ragged edges; exact on small integers with one slice."""
    import torch
    rng = np.random.default_rng(M + N + K)
    A = rng.integers(-63, 64, (M, K)).astype(np.float64)
    B = rng.integers(-63, 64, (K, N)).astype(np.float64)
    ref = (A.astype(np.int64) @ B.astype(np.int64)).astype(np.float64)
    C = torch.zeros((M, N), dtype=torch.float64, device="cuda")
    lib.dsrg_split_gemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), C, 1.0, 1)
    assert np.array_equal(C.cpu().numpy(), ref)


@pytest.mark.parametrize("slices,lo,hi", [(2, 1e-10, 2.0 ** -10), (3, 1e-12, 2.0 ** -17)])
def test_few_slices_truncate_visibly(lib, slices, lo, hi):
    """With 2 or 3 digit slices the product carries about 7 S bits relative to
    the row/column maxima (each operand rounded to a 2^(7 S - 1) grid): its error against FP64 must exceed FP64 rounding by
    orders of magnitude (so an FP64 fallback would fail here) and stay within
    the digit-rounding bound."""
    import torch
    rng = np.random.default_rng(5)
    M, N, K = 300, 200, 500
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((K, N))
    ref = A @ B
    bound = np.abs(A).max(axis=1)[:, None] * np.abs(B).max(axis=0)[None, :] * K
    C = torch.zeros((M, N), dtype=torch.float64, device="cuda")
    lib.dsrg_split_gemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), C, 1.0, slices)
    err = (np.abs(C.cpu().numpy() - ref) / bound).max()
    assert lo < err < hi, err
