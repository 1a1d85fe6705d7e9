"""GPU parity: the CUDA path through the C interface against the FP64 oracle.

Energies must agree to 1e-9 Eh (the plain FP64 path's tolerance); the
amplitudes and the excitation blocks of 1/2 [Htilde(1), A(1)]_{1,2} are
compared element by element after mapping the oracle's spin-orbital order
(sigma * n + p) onto the library's interval layout.
"""
import numpy as np
import pytest

import synth
from oracle import dsrg

pytestmark = pytest.mark.gpu

TOL_E = 1e-9


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


def _so_index(n, lo, hi):
    return np.array([s * n + x for s in (0, 1) for x in range(lo, hi)])


def _to_gpu_layout(full, n, ivs):
    return full[np.ix_(*[_so_index(n, a, b) for a, b in ivs])]


SHAPES = [
    # (nc, na, nel, nv, naux)
    (1, 3, 2, 2, 5),
    (2, 2, 2, 3, 6),
    (0, 3, 2, 2, 5),   # no core
    (2, 0, 0, 3, 6),   # no active space: single reference
    (1, 2, 2, 0, 4),   # no virtuals
    (2, 4, 4, 12, 60),  # the small CAS(4,4) workload
    (3, 4, 4, 21, 50),  # several 64-wide tiles with ragged tails
]


def _check_against_oracle(lib, inst):
    """Energies within TOL_E; T1, T2, second-order T1, T2 and the excitation
    blocks of 1/2 [Htilde(1), A(1)]_{1,2} element by element."""
    nc, na = inst["nc"], inst["na"]
    ref = dsrg.dsrg_pt3(inst, return_intermediates=True)
    P, I = ref["_problem"], ref["_inter"]
    h = lib.Dsrg(inst)
    try:
        e = h.pt3()
        for k in ("e2", "e3a", "e3b", "e3"):
            assert abs(e[k] - ref[k]) < TOL_E, (k, e[k], ref[k])
        n = P.n
        Hiv, Piv = (0, nc + na), (nc, n)
        cmp = {"T1": (I["T1"], [Piv, Hiv]), "T2": (I["T2"], [Piv, Piv, Hiv, Hiv]),
               "T1b": (I["T1b"], [Piv, Hiv]), "T2b": (I["T2b"], [Piv, Piv, Hiv, Hiv])}
        for name, (full, ivs) in cmp.items():
            want = _to_gpu_layout(full, n, ivs)
            got = h.fetch(name)
            scale = max(1.0, np.abs(want).max())
            assert np.abs(got - want).max() < 1e-11 * scale, name
        # non-diagonal blocks of 1/2 [Htilde(1), A(1)] (internal elements excluded)
        O = I["O"]
        w1 = _to_gpu_layout(np.where(P.mask1, O.z[1], 0.0), n, [Piv, Hiv])
        g1 = h.fetch("O1")
        m1 = _to_gpu_layout(P.mask1, n, [Piv, Hiv])
        assert np.abs((g1 - w1)[m1]).max(initial=0.0) < 1e-11 * max(1.0, np.abs(w1).max())
        w2 = _to_gpu_layout(O.z[2], n, [Piv, Piv, Hiv, Hiv])
        m2 = _to_gpu_layout(P.mask2, n, [Piv, Piv, Hiv, Hiv])
        g2 = h.fetch("O2")
        assert np.abs((g2 - w2)[m2]).max(initial=0.0) < 1e-11 * max(1.0, np.abs(w2).max())
    finally:
        h.close()
    return ref


@pytest.mark.parametrize("shape", SHAPES, ids=[str(s) for s in SHAPES])
def test_energies_and_intermediates(lib, shape):
    nc, na, nel, nv, naux = shape
    _check_against_oracle(lib, synth.make_instance(nc, na, nel, nv, naux, 0.5, seed=sum(shape) + 7))


def test_degenerate_and_near_degenerate_denominators(lib):
    """Orbital energies with exact and near degeneracies across blocks, so that
    many denominators D of Eqs. T1_1st, T2_1st, T1_2nd and T2_2nd are exactly
    0 (regulariser limit 0) or 1e-9 .. 1e-6 (the series branch and the switch
    point s D^2 = 1e-12), on both sides."""
    inst = synth.make_instance(2, 4, 4, 6, 24, 0.5, seed=41)
    eps = inst["eps"].copy()
    nc, na = 2, 4
    a0, v0 = nc, nc + na
    eps[0], eps[1] = -3.0, -2.5            # exactly representable sums
    eps[v0 + 0] = eps[a0 + 0]               # D = 0: T1[v0, u0], T2[v0, x, u0, x], ...
    eps[v0 + 1] = eps[a0 + 1] + 1e-8        # |D| ~ 1e-8: series branch
    eps[v0 + 2] = eps[a0 + 2] - 3e-9
    eps[v0 + 3] = eps[a0 + 3] + 1e-6 / np.sqrt(0.5)   # s D^2 at the 1e-12 switch
    eps[v0 + 4], eps[v0 + 5] = -6.75, 1.25  # eps_c0 + eps_c1 = eps_v4 + eps_v5: D = 0 for T2[v4, v5, c0, c1]
    inst["eps"] = eps
    ref = _check_against_oracle(lib, inst)
    D2 = ref["_problem"].D2
    assert (np.abs(D2) == 0.0).sum() > 0 and ((np.abs(D2) > 0) & (np.abs(D2) < 1e-7)).sum() > 0


def test_pt2_call_matches_pt3_e2(lib):
    inst = synth.make_instance(1, 3, 2, 4, 10, 0.5, seed=3)
    h = lib.Dsrg(inst)
    try:
        a = h.pt2()
        b = h.pt3()
        assert a["e3"] == 0.0
        assert abs(a["e2"] - b["e2"]) < 1e-13
    finally:
        h.close()


def test_off_diagonal_fock_input(lib):
    inst = synth.make_instance(1, 3, 2, 3, 8, 0.5, seed=19)
    n = 7
    f1 = np.random.default_rng(4).standard_normal((n, n)) * 0.05
    inst["f1"] = f1 + f1.T
    ref = dsrg.dsrg_pt3(inst)
    h = lib.Dsrg(inst)
    try:
        e = h.pt3()
    finally:
        h.close()
    for k in ("e2", "e3a", "e3b"):
        assert abs(e[k] - ref[k]) < TOL_E


def test_device_inputs_and_reload(lib):
    import torch
    inst = synth.make_instance(2, 2, 2, 5, 12, 0.5, seed=23)
    ref = dsrg.dsrg_pt3(inst)
    dev = {k: (torch.from_numpy(np.ascontiguousarray(v)).cuda() if isinstance(v, np.ndarray) else v)
           for k, v in inst.items()}
    h = lib.Dsrg(dev)
    try:
        e = h.pt3()
        assert abs(e["e3"] - ref["e3"]) < TOL_E and abs(e["e2"] - ref["e2"]) < TOL_E
        # reload a second problem of the same sizes into the same handle
        inst2 = synth.make_instance(2, 2, 2, 5, 12, 0.7, seed=29)
        ref2 = dsrg.dsrg_pt3(inst2)
        h.load(inst2)
        e2 = h.pt3()
        assert abs(e2["e3"] - ref2["e3"]) < TOL_E and abs(e2["e2"] - ref2["e2"]) < TOL_E
        assert h.launches > 0
    finally:
        h.close()


def test_argument_errors(lib):
    inst = synth.make_instance(1, 2, 2, 2, 4, 0.5, seed=1)
    bad = dict(inst, s=-1.0)
    with pytest.raises(lib.DsrgError) as ex:
        lib.Dsrg(bad)
    assert ex.value.code == -1
    bad = dict(inst, naux=0)
    with pytest.raises(lib.DsrgError):
        lib.Dsrg(bad)
