"""dsrg_df_ladder_noalloc: the ladder for callers that cannot allocate.

Frameworks whose caching allocator owns all device memory, and runtimes that
forbid allocation after start-up, cannot let a library call cudaMalloc.  The
no-allocation entry point keeps its scratch in a fixed device array; its
result must equal the allocating entry point's, including on a later call
that finds the previous call's data still in that array, when the rows are
formed in several batches that reuse the array, and at the largest size the
array accepts.  This file is collected last so a failure here cannot stop the
rest of a run that stops at the first failure.
"""
import ctypes

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
    L = g.load_library()
    L.dsrg_df_ladder_noalloc.argtypes = [ctypes.c_int] * 5 + [ctypes.c_void_p] * 4
    L.dsrg_df_ladder_noalloc.restype = ctypes.c_int
    return g, L


def _call(fn, B, t, out, p0):
    naux, n, _ = B.shape
    npart, _, nh, _ = t.shape
    return fn(n, naux, p0, npart, nh, ctypes.c_void_p(B.data_ptr()), ctypes.c_void_p(t.data_ptr()),
              ctypes.c_void_p(out.data_ptr()), None)


def _compare(L, n, naux, p0, npart, nh, seed):
    import torch
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((naux, n, n))
    B = torch.from_numpy(0.5 * (B + np.transpose(B, (0, 2, 1)))).cuda()
    t = torch.from_numpy(rng.standard_normal((npart, npart, nh, nh))).cuda()
    ref = torch.zeros((npart, npart, nh, nh), dtype=torch.float64, device="cuda")
    got = torch.full((npart, npart, nh, nh), 3.0, dtype=torch.float64, device="cuda")
    assert _call(L.dsrg_df_ladder, B, t, ref, p0) == 0, L.dsrg_last_error()
    assert _call(L.dsrg_df_ladder_noalloc, B, t, got, p0) == 0, L.dsrg_last_error()
    r, q = ref.cpu().numpy(), got.cpu().numpy()
    assert np.abs(q - r).max() < 1e-11 * max(1.0, np.abs(r).max())


def test_noalloc_matches_allocating_ladder_twice(lib):
    g, L = lib
    # the second call is smaller and finds the first call's data in the array
    for k, shape in enumerate([(50, 40, 6, 41, 7), (30, 25, 2, 27, 5)]):
        _compare(L, *shape, seed=100 + k)


def test_noalloc_several_batches_and_largest_size(lib):
    """np = 60 forms (pr|qs) in four batches of at most 19 rows that reuse the
    array (each at its own row offset r0 of L); np = 161 is the largest size
    the array holds, one row per batch."""
    g, L = lib
    _compare(L, 66, 30, 4, 60, 4, seed=7)
    _compare(L, 163, 12, 1, 161, 2, seed=8)


def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    import torch
    g, L = lib
    B = torch.zeros((1, 170, 170), dtype=torch.float64, device="cuda")
    t = torch.zeros((170, 170, 1, 1), dtype=torch.float64, device="cuda")
    out = torch.zeros((170, 170, 1, 1), dtype=torch.float64, device="cuda")
    assert _call(L.dsrg_df_ladder_noalloc, B, t, out, 0) == -1
    assert b"np <= 161" in L.dsrg_last_error()
