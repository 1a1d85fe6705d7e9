"""GPU first-order aavv amplitudes with Dyall's H(0) (dsrg_dyall_aavv; App. B,
Eq. t2_aavv) against the oracle (oracle.dyall).

* Small instances: the amplitudes element by element against the oracle's
  direct solution (FP64 path 1e-10 of the largest amplitude, split path
  1e-8), convergence, the smallest shifted denominator and the count below
  1e-2 (an instance whose virtual band overlaps the active one has small
  shifted denominators).
* The CAS(6,6)/10 core/100 virtual/400 aux workload (too large for the dense
  oracle): the residual of Eq. t2_aavv recomputed on the host from B, the
  active densities and the GPU's amplitudes on sampled virtual pairs.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1701_02011_gb300 import build
    build.build()
    import paper_1701_02011_gb300 as g
    g.load_library()
    return g


def _device(inst):
    import torch
    return {k: (torch.from_numpy(np.ascontiguousarray(v)).cuda() if isinstance(v, np.ndarray) else v)
            for k, v in inst.items() if k not in ("ci", "dets", "g1_so", "l2_so", "l3_so")}


CASES = [
    ("c1a3v2", dict(nc=1, na=3, nel=2, nv=2, naux=6, seed=7)),
    ("c2a4v12", dict(nc=2, na=4, nel=4, nv=12, naux=60, seed=8)),
    ("overlap", dict(nc=1, na=3, nel=2, nv=3, naux=8, seed=5, eps_vir=(0.05, 0.4))),
]


@pytest.mark.parametrize("name,kw", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_aavv_amplitudes_match_oracle(lib, name, kw, precision):
    from oracle import dyall
    kw = dict(kw)
    nc, na, nel, nv, naux, seed = (kw.pop(k) for k in ("nc", "na", "nel", "nv", "naux", "seed"))
    inst = synth.make_instance(nc, na, nel, nv, naux, 0.5, seed=seed, **kw)
    Vs, Va, g, D = dyall.blocks(inst)
    want = dyall.solve(Vs, Va, g, D)
    Ds = dyall.shifted_denominators(Va, g, D)
    off = ~np.eye(Va.shape[0], dtype=bool)[None, None]
    opts = dict(precision=lib.DSRG_PREC_SPLIT, slices=7) if precision == "split" else {}
    h = lib.Dsrg(_device(inst), **opts)
    try:
        r = h.dyall_aavv(tol=1e-12, max_iter=300)
        t = h.fetch("Taavv")
    finally:
        h.close()
    tol = 1e-10 if precision == "fp64" else 1e-8
    assert np.abs(t - want).max() <= tol * np.abs(want).max()
    assert r["converged"] == 1 and r["pairs_not_converged"] == 0
    assert r["max_source"] == pytest.approx(np.abs(np.where(off, Vs, 0)).max(), rel=1e-12)
    assert r["min_shifted_denominator"] == pytest.approx(np.abs(Ds[np.broadcast_to(off, Ds.shape)]).min(), rel=1e-9)
    assert r["small_denominators"] == int((np.abs(Ds[np.broadcast_to(off, Ds.shape)]) < 1e-2).sum())
    if name == "overlap":
        assert r["small_denominators"] > 0


def _so_integrals(B, P, Q, R, S):
    """<pq||rs> for spin-orbital index lists (spatial, spin) of the four slots."""
    def J(a, b, c, d):  # (ab|cd) over spatial lists
        return np.einsum("Xab,Xcd->abcd", B[:, a][:, :, b], B[:, c][:, :, d], optimize=True)
    out = np.zeros((len(P), len(Q), len(R), len(S)))
    sp = lambda L: (np.array([x[0] for x in L]), np.array([x[1] for x in L]))
    (p, sp_), (q, sq), (r, sr), (s, ss) = sp(P), sp(Q), sp(R), sp(S)
    direct = J(p, r, q, s).transpose(0, 2, 1, 3)       # (pr|qs) at [p,q,r,s]
    exch = J(p, s, q, r).transpose(0, 2, 3, 1)         # (ps|qr) at [p,q,r,s]
    d1 = (sp_[:, None, None, None] == sr[None, None, :, None]) & (sq[None, :, None, None] == ss[None, None, None, :])
    d2 = (sp_[:, None, None, None] == ss[None, None, None, :]) & (sq[None, :, None, None] == sr[None, None, :, None])
    return np.where(d1, direct, 0.0) - np.where(d2, exch, 0.0)


def test_full_size_residual_on_sampled_pairs(lib):
    from oracle import dyall
    inst = synth.config_instance("cas66_c10_v100_q400")
    h = lib.Dsrg(_device(inst), precision=lib.DSRG_PREC_SPLIT, slices=6)
    try:
        r = h.dyall_aavv(tol=1e-10, max_iter=300)
        t = h.fetch("Taavv")
    finally:
        h.close()
    assert r["converged"] == 1
    nc, na, nv = inst["nc"], inst["na"], inst["nv"]
    B = np.asarray(inst["B"])
    act = [(nc + u, 0) for u in range(na)] + [(nc + u, 1) for u in range(na)]
    vir = [(nc + na + e, 0) for e in range(nv)] + [(nc + na + e, 1) for e in range(nv)]
    Va = _so_integrals(B, act, act, act, act)
    g = np.zeros((2 * na, 2 * na))
    g[:na, :na] = np.asarray(inst["g1a"]).reshape(na, na)
    g[na:, na:] = np.asarray(inst["g1b"]).reshape(na, na)
    eps = np.asarray(inst["eps"])
    ea = np.concatenate([eps[nc:nc + na]] * 2)
    ev = np.concatenate([eps[nc + na:]] * 2)
    rng = np.random.default_rng(0)
    es = rng.choice(2 * nv, 6, replace=False)
    fs = rng.choice(2 * nv, 6, replace=False)
    Vs = _so_integrals(B, [vir[e] for e in es], [vir[f] for f in fs], act, act)
    tt = t[np.ix_(es, fs)]
    D = ea[None, None, :, None] + ea[None, None, None, :] - ev[es][:, None, None, None] - ev[fs][None, :, None, None]
    R = dyall.residual(tt, Vs, Va, g, D)
    off = ~np.eye(2 * na, dtype=bool)[None, None]
    assert np.abs(np.where(off, R, 0)).max() <= 1e-8 * r["max_source"]
