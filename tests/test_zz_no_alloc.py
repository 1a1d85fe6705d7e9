"""dsrg_df_ladder_noalloc: the ladder for callers that cannot allocate.

Callers inside CUDA graph capture, or that hand all device memory to their
own pool, cannot let a library call cudaMalloc.  The no-allocation entry
point keeps its scratch in a fixed device array; its result must equal the
allocating entry point's, including on a second call that finds the
previous call's data still in that array.  This file is collected last so a
failure here cannot stop the rest of a run that stops at the first failure.
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


def test_noalloc_matches_allocating_ladder_twice(lib):
    import torch
    g, L = lib
    shapes = [(50, 40, 6, 41, 7), (30, 25, 2, 27, 5)]  # second call: smaller, finds stale scratch
    for k, (n, naux, p0, npart, nh) in enumerate(shapes):
        rng = np.random.default_rng(100 + k)
        B = rng.standard_normal((naux, n, n))
        B = torch.from_numpy(0.5 * (B + np.transpose(B, (0, 2, 1)))).cuda()
        t = torch.from_numpy(rng.standard_normal((npart, npart, nh, nh))).cuda()
        ref = torch.zeros((npart, npart, nh, nh), dtype=torch.float64, device="cuda")
        got = torch.full((npart, npart, nh, nh), 3.0, dtype=torch.float64, device="cuda")
        assert _call(L.dsrg_df_ladder, B, t, ref, p0) == 0
        assert _call(L.dsrg_df_ladder_noalloc, B, t, got, p0) == 0, L.dsrg_last_error()
        r, q = ref.cpu().numpy(), got.cpu().numpy()
        assert np.abs(q - r).max() < 1e-11 * max(1.0, np.abs(r).max())


def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    import torch
    g, L = lib
    B = torch.zeros((1, 170, 170), dtype=torch.float64, device="cuda")
    t = torch.zeros((170, 170, 1, 1), dtype=torch.float64, device="cuda")
    out = torch.zeros((170, 170, 1, 1), dtype=torch.float64, device="cuda")
    assert _call(L.dsrg_df_ladder_noalloc, B, t, out, 0) == -1
    assert b"np <= 161" in L.dsrg_last_error()
