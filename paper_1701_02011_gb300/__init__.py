"""Python binding of the GB300 DSRG-MRPT2/PT3 energy library (include/dsrg.h).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of ``libdsrg.so``.  Importing works without a GPU; the first call
that needs the library loads it and raises if it has not been built.

Inputs are a dict with the keys of ``dsrg_inputs``: nc, na, nv, naux, s,
eps, B, g1a, g1b, l2aa, l2ab, l2bb, l3aaa, l3aab, l3abb, l3bbb and optional
f1.  Arrays may be numpy (host memory) or CUDA torch tensors (device memory,
float64, contiguous); all arrays of one call must live in the same place.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(HERE, "libdsrg.so")

DSRG_MEM_HOST = 0
DSRG_MEM_DEVICE = 1
DSRG_PREC_FP64 = 0
DSRG_PREC_SPLIT = 1
DSRG_ERR_ARG, DSRG_ERR_OOM, DSRG_ERR_CUDA, DSRG_ERR_STATE, DSRG_ERR_INTERNAL, DSRG_ERR_TIMEOUT = -1, -2, -3, -4, -5, -6

_P = ctypes.POINTER(ctypes.c_double)


class dsrg_inputs(ctypes.Structure):
    _fields_ = [("nc", ctypes.c_int), ("na", ctypes.c_int), ("nv", ctypes.c_int), ("naux", ctypes.c_int),
                ("s", ctypes.c_double), ("eps", _P), ("B", _P), ("g1a", _P), ("g1b", _P),
                ("l2aa", _P), ("l2ab", _P), ("l2bb", _P), ("l3aaa", _P), ("l3aab", _P), ("l3abb", _P),
                ("l3bbb", _P), ("f1", _P), ("memory", ctypes.c_int)]


class dsrg_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("stream", ctypes.c_void_p), ("slices", ctypes.c_int),
                ("tune", ctypes.c_int), ("wait_limit", ctypes.c_longlong)]


class dsrg_energies(ctypes.Structure):
    _fields_ = [("e2", ctypes.c_double), ("e3a", ctypes.c_double), ("e3b", ctypes.c_double),
                ("e3", ctypes.c_double)]


class dsrg_relaxed_energies(ctypes.Structure):
    _fields_ = [("e2", ctypes.c_double), ("e3a", ctypes.c_double), ("e3b", ctypes.c_double),
                ("e3", ctypes.c_double), ("e_relaxed2", ctypes.c_double), ("e_relaxed3", ctypes.c_double),
                ("residual2", ctypes.c_double), ("residual3", ctypes.c_double), ("ndet", ctypes.c_longlong),
                ("steps2", ctypes.c_int), ("steps3", ctypes.c_int)]


class dsrg_dyall_result(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int), ("max_residual", ctypes.c_double),
                ("max_source", ctypes.c_double), ("min_shifted_denominator", ctypes.c_double),
                ("pairs_not_converged", ctypes.c_longlong), ("small_denominators", ctypes.c_longlong)]


EXPORTS = ("dsrg_init", "dsrg_load", "dsrg_pt2", "dsrg_pt3", "dsrg_pt3_batch", "dsrg_free", "dsrg_last_error",
           "dsrg_last_launch_count", "dsrg_peak_bytes", "dsrg_fetch", "dsrg_profile", "dsrg_profile_stats",
           "dsrg_profile_step",
           "dsrg_last_d2h_bytes", "dsrg_df_ladder", "dsrg_df_ladder_noalloc", "dsrg_split_gemm", "dsrg_cholesky",
           "dsrg_relaxed", "dsrg_dyall_aavv")

_lib = None


def load_library(path: str = LIBPATH) -> ctypes.CDLL:
    """Load libdsrg.so; raises if it is missing (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1701_02011_gb300.build.build()")
    L = ctypes.CDLL(path)
    L.dsrg_init.argtypes = [ctypes.POINTER(dsrg_inputs), ctypes.POINTER(dsrg_options), ctypes.POINTER(ctypes.c_void_p)]
    L.dsrg_init.restype = ctypes.c_int
    L.dsrg_load.argtypes = [ctypes.c_void_p, ctypes.POINTER(dsrg_inputs)]
    L.dsrg_load.restype = ctypes.c_int
    for f in ("dsrg_pt2", "dsrg_pt3"):
        getattr(L, f).argtypes = [ctypes.c_void_p, ctypes.POINTER(dsrg_energies)]
        getattr(L, f).restype = ctypes.c_int
    L.dsrg_relaxed.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(dsrg_relaxed_energies)]
    L.dsrg_relaxed.restype = ctypes.c_int
    L.dsrg_dyall_aavv.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.POINTER(dsrg_dyall_result)]
    L.dsrg_dyall_aavv.restype = ctypes.c_int
    L.dsrg_pt3_batch.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.POINTER(dsrg_energies)]
    L.dsrg_pt3_batch.restype = ctypes.c_int
    L.dsrg_free.argtypes = [ctypes.c_void_p]
    L.dsrg_free.restype = None
    L.dsrg_last_error.argtypes = []
    L.dsrg_last_error.restype = ctypes.c_char_p
    L.dsrg_last_launch_count.argtypes = [ctypes.c_void_p]
    L.dsrg_last_launch_count.restype = ctypes.c_longlong
    L.dsrg_last_d2h_bytes.argtypes = [ctypes.c_void_p]
    L.dsrg_last_d2h_bytes.restype = ctypes.c_longlong
    L.dsrg_peak_bytes.argtypes = [ctypes.c_void_p]
    L.dsrg_peak_bytes.restype = ctypes.c_longlong
    L.dsrg_fetch.argtypes = [ctypes.c_void_p, ctypes.c_char_p, _P, ctypes.c_longlong]
    L.dsrg_fetch.restype = ctypes.c_int
    L.dsrg_profile.argtypes = [ctypes.c_void_p, ctypes.c_int]
    L.dsrg_profile.restype = ctypes.c_int
    L.dsrg_profile_stats.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_char_p),
                                     ctypes.POINTER(ctypes.c_longlong), _P, _P, _P, _P]
    L.dsrg_profile_stats.restype = ctypes.c_int
    L.dsrg_profile_step.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_char_p),
                                    ctypes.POINTER(ctypes.c_longlong), _P, _P]
    L.dsrg_profile_step.restype = ctypes.c_int
    L.dsrg_df_ladder.argtypes = [ctypes.c_int] * 5 + [ctypes.c_void_p] * 4
    L.dsrg_df_ladder.restype = ctypes.c_int
    L.dsrg_df_ladder_noalloc.argtypes = [ctypes.c_int] * 5 + [ctypes.c_void_p] * 4
    L.dsrg_df_ladder_noalloc.restype = ctypes.c_int
    L.dsrg_split_gemm.argtypes = [ctypes.c_longlong] * 3 + [ctypes.c_void_p, ctypes.c_longlong,
                                                            ctypes.c_void_p, ctypes.c_longlong,
                                                            ctypes.c_void_p, ctypes.c_longlong,
                                                            ctypes.c_double, ctypes.c_int, ctypes.c_void_p]
    L.dsrg_split_gemm.restype = ctypes.c_int
    L.dsrg_cholesky.argtypes = [ctypes.c_longlong, ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_void_p,
                                ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_longlong), ctypes.c_void_p]
    L.dsrg_cholesky.restype = ctypes.c_int
    _lib = L
    return L


class DsrgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"dsrg error {code}: {msg}")
        self.code = code


def _check(rc):
    if rc != 0:
        raise DsrgError(rc, load_library().dsrg_last_error().decode())


_ARRAYS = ("eps", "B", "g1a", "g1b", "l2aa", "l2ab", "l2bb", "l3aaa", "l3aab", "l3abb", "l3bbb", "f1")


def _pointer(x, keep, device):
    if x is None:
        return None
    if device:
        if not (x.is_cuda and x.dtype.is_floating_point and x.element_size() == 8 and x.is_contiguous()):
            raise ValueError("device inputs must be contiguous float64 CUDA tensors")
        keep.append(x)
        return ctypes.cast(ctypes.c_void_p(x.data_ptr()), _P)
    a = np.ascontiguousarray(x, dtype=np.float64)
    keep.append(a)
    return a.ctypes.data_as(_P)


def _is_device(inst):
    for k in _ARRAYS:
        x = inst.get(k)
        if x is not None and hasattr(x, "is_cuda"):
            return bool(x.is_cuda)
    return False


def make_inputs(inst: dict):
    """Return (dsrg_inputs, keepalive list)."""
    device = _is_device(inst)
    keep = []
    s = dsrg_inputs()
    s.nc, s.na, s.nv, s.naux = int(inst["nc"]), int(inst["na"]), int(inst["nv"]), int(inst["naux"])
    s.s = float(inst["s"])
    for k in _ARRAYS:
        p = _pointer(inst.get(k), keep, device)
        setattr(s, k, p)
    s.memory = DSRG_MEM_DEVICE if device else DSRG_MEM_HOST
    return s, keep


def dsrg_init(inst: dict, stream=None, precision=DSRG_PREC_FP64, slices: int = 0,
              tune: bool = False, wait_limit: int = 0) -> ctypes.c_void_p:
    L = load_library()
    s, keep = make_inputs(inst)
    opt = dsrg_options(precision, ctypes.c_void_p(stream) if stream else None, int(slices), int(bool(tune)),
                       int(wait_limit))
    h = ctypes.c_void_p()
    _check(L.dsrg_init(ctypes.byref(s), ctypes.byref(opt), ctypes.byref(h)))
    return h


def dsrg_load(h, inst: dict) -> None:
    s, keep = make_inputs(inst)
    _check(load_library().dsrg_load(h, ctypes.byref(s)))


def _energies(fn, h):
    e = dsrg_energies()
    _check(fn(h, ctypes.byref(e)))
    return {"e2": e.e2, "e3a": e.e3a, "e3b": e.e3b, "e3": e.e3}


def dsrg_pt2(h) -> dict:
    return _energies(load_library().dsrg_pt2, h)


def dsrg_pt3(h) -> dict:
    return _energies(load_library().dsrg_pt3, h)


def dsrg_relaxed(h, n_alpha: int, n_beta: int) -> dict:
    """Unrelaxed components and the one-step relaxed DSRG-MRPT2/PT3 energies
    (relative to E0) over the determinants with n_alpha, n_beta active electrons."""
    out = dsrg_relaxed_energies()
    _check(load_library().dsrg_relaxed(h, int(n_alpha), int(n_beta), ctypes.byref(out)))
    return {k: getattr(out, k) for k, _ in dsrg_relaxed_energies._fields_}


def dsrg_dyall_aavv(h, tol: float = 1e-10, max_iter: int = 200) -> dict:
    """First-order aavv amplitudes with Dyall's H(0) at s -> infinity (App. B);
    the amplitudes are fetched as "Taavv"."""
    out = dsrg_dyall_result()
    _check(load_library().dsrg_dyall_aavv(h, float(tol), int(max_iter), ctypes.byref(out)))
    return {k: getattr(out, k) for k, _ in dsrg_dyall_result._fields_}


def dsrg_pt3_batch(handles) -> list:
    """PT3 energies of several handles at once (graph-captured after the first
    call per handle); handles are raw handles or Dsrg objects."""
    hs = [x.h if isinstance(x, Dsrg) else x for x in handles]
    n = len(hs)
    arr = (ctypes.c_void_p * max(n, 1))(*hs)
    out = (dsrg_energies * max(n, 1))()
    _check(load_library().dsrg_pt3_batch(arr, n, out))
    return [{"e2": e.e2, "e3a": e.e3a, "e3b": e.e3b, "e3": e.e3} for e in list(out)[:n]]


def dsrg_free(h) -> None:
    if h:
        load_library().dsrg_free(h)


def dsrg_last_launch_count(h) -> int:
    return int(load_library().dsrg_last_launch_count(h))


def dsrg_last_d2h_bytes(h) -> int:
    return int(load_library().dsrg_last_d2h_bytes(h))


def dsrg_peak_bytes(h) -> int:
    return int(load_library().dsrg_peak_bytes(h))


def dsrg_profile(h, enable: bool) -> None:
    _check(load_library().dsrg_profile(h, 1 if enable else 0))


def dsrg_profile_stats(h) -> dict:
    """{kernel name: dict(launches, ms, flops, exec_flops, bytes)} accumulated since dsrg_profile."""
    L = load_library()
    out = {}
    k = 0
    while True:
        name = ctypes.c_char_p()
        n = ctypes.c_longlong()
        ms, fl, xf, by = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        rc = L.dsrg_profile_stats(h, k, ctypes.byref(name), ctypes.byref(n), ctypes.byref(ms), ctypes.byref(fl),
                                  ctypes.byref(xf), ctypes.byref(by))
        if rc != 0:
            break
        out[name.value.decode()] = dict(launches=n.value, ms=ms.value, flops=fl.value, exec_flops=xf.value,
                                        bytes=by.value)
        k += 1
    return out


def dsrg_profile_steps(h) -> dict:
    """{step name: dict(launches, ms, flops)} accumulated since dsrg_profile, in order of first use."""
    L = load_library()
    out = {}
    k = 0
    while True:
        name = ctypes.c_char_p()
        n = ctypes.c_longlong()
        ms, fl = ctypes.c_double(), ctypes.c_double()
        if L.dsrg_profile_step(h, k, ctypes.byref(name), ctypes.byref(n), ctypes.byref(ms), ctypes.byref(fl)) != 0:
            break
        out[name.value.decode() or "other"] = dict(launches=n.value, ms=ms.value, flops=fl.value)
        k += 1
    return out


def tensor_shape(name: str, nc: int, na: int, nv: int):
    h, p = 2 * (nc + na), 2 * (na + nv)
    if name in ("T1", "T1b", "O1"):
        return (p, h)
    if name in ("T2", "T2b", "O2"):
        return (p, p, h, h)
    if name in ("Hbar1_2", "Hbar1_3"):
        return (2 * na, 2 * na)
    if name in ("Hbar2_2", "Hbar2_3"):
        return (2 * na,) * 4
    if name == "Taavv":
        return (2 * nv, 2 * nv, 2 * na, 2 * na)
    raise KeyError(name)


def dsrg_fetch(h, name: str, nc: int, na: int, nv: int) -> np.ndarray:
    shape = tensor_shape(name, nc, na, nv)
    out = np.empty(shape, dtype=np.float64)
    _check(load_library().dsrg_fetch(h, name.encode(), out.ctypes.data_as(_P), int(out.size)))
    return out


def _dev_ptr(x):
    if not (hasattr(x, "is_cuda") and x.is_cuda and x.element_size() == 8 and x.is_contiguous()):
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(x.data_ptr())


def dsrg_df_ladder(B, t, L, p0: int, stream=None) -> None:
    """L[p,q,i,j] = sum_rs (sum_Q B[Q,p0+p,p0+r] B[Q,p0+q,p0+s]) t[r,s,i,j] on CUDA tensors."""
    naux, n, _ = B.shape
    np_, _, nh, _ = t.shape
    _check(load_library().dsrg_df_ladder(n, naux, p0, np_, nh, _dev_ptr(B), _dev_ptr(t), _dev_ptr(L),
                                         ctypes.c_void_p(stream) if stream else None))


def dsrg_df_ladder_noalloc(B, t, L, p0: int, stream=None) -> None:
    """dsrg_df_ladder without device allocation (fixed 32 MiB scratch, np <= 161),
    for callers whose device memory is owned by their own allocator or that may
    not allocate after start-up; overlapping calls must be serialised."""
    naux, n, _ = B.shape
    np_, _, nh, _ = t.shape
    _check(load_library().dsrg_df_ladder_noalloc(n, naux, p0, np_, nh, _dev_ptr(B), _dev_ptr(t), _dev_ptr(L),
                                                 ctypes.c_void_p(stream) if stream else None))


def dsrg_split_gemm(A, B, C, alpha: float = 1.0, slices: int = 6, stream=None) -> None:
    """C += alpha A B (2-D CUDA float64 tensors, row-major, unit column stride) on the tensor cores."""
    M, K = A.shape
    K2, N = B.shape
    assert K == K2 and tuple(C.shape) == (M, N)
    for x in (A, B, C):
        if not (x.is_cuda and x.element_size() == 8 and x.stride(1) == 1):
            raise ValueError("expected CUDA float64 matrices with unit column stride")
    _check(load_library().dsrg_split_gemm(M, N, K, ctypes.c_void_p(A.data_ptr()), A.stride(0),
                                          ctypes.c_void_p(B.data_ptr()), B.stride(0),
                                          ctypes.c_void_p(C.data_ptr()), C.stride(0), float(alpha), int(slices),
                                          ctypes.c_void_p(stream) if stream else None))


def dsrg_cholesky(V, tau: float, max_vecs: int, stream=None):
    """Pivoted incomplete Cholesky of the PSD CUDA float64 matrix V [N][N]:
    returns (B [nvecs][N] CUDA tensor, pivots numpy int64 array)."""
    import torch
    N = V.shape[0]
    if not (V.is_cuda and V.dtype == torch.float64 and V.is_contiguous() and tuple(V.shape) == (N, N)):
        raise ValueError("expected a contiguous square CUDA float64 matrix")
    B = torch.empty((max(max_vecs, 1), N), dtype=torch.float64, device=V.device)
    n = ctypes.c_int(0)
    piv = np.zeros(max(max_vecs, 1), dtype=np.int64)
    _check(load_library().dsrg_cholesky(N, ctypes.c_void_p(V.data_ptr()), float(tau), int(max_vecs),
                                        ctypes.c_void_p(B.data_ptr()), ctypes.byref(n),
                                        piv.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)),
                                        ctypes.c_void_p(stream) if stream else None))
    return B[: n.value], piv[: n.value]


class Dsrg:
    """Convenience owner of one handle."""

    def __init__(self, inst: dict, stream=None, precision=DSRG_PREC_FP64, slices: int = 0, tune: bool = False,
                 wait_limit: int = 0):
        self.sizes = (int(inst["nc"]), int(inst["na"]), int(inst["nv"]))
        self.h = None
        self.h = dsrg_init(inst, stream, precision, slices, tune, wait_limit)

    def load(self, inst):
        dsrg_load(self.h, inst)

    def pt2(self):
        return dsrg_pt2(self.h)

    def pt3(self):
        return dsrg_pt3(self.h)

    def dyall_aavv(self, tol: float = 1e-10, max_iter: int = 200):
        return dsrg_dyall_aavv(self.h, tol, max_iter)

    def relaxed(self, n_alpha: int, n_beta: int):
        return dsrg_relaxed(self.h, n_alpha, n_beta)

    def fetch(self, name):
        return dsrg_fetch(self.h, name, *self.sizes)

    def profile(self, enable=True):
        dsrg_profile(self.h, enable)

    def profile_stats(self):
        return dsrg_profile_stats(self.h)

    def profile_steps(self):
        return dsrg_profile_steps(self.h)

    @property
    def launches(self):
        return dsrg_last_launch_count(self.h)

    def close(self):
        if self.h:
            dsrg_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
