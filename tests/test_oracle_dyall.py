"""Pins of the Dyall-H(0) aavv amplitude equation of the oracle (oracle.dyall,
Eq. t2_aavv, App. B).

Fixed by: the generic Mukherjee-Kutzelnigg commutator (oracle.mkgno, itself
pinned against explicit Fock-space commutators) of H(0) = F(0) + the
all-active part of V with an aavv T2, whose aavv block must equal the
printed terms; the Moller-Plesset limit (no active two-body part: t = V/D);
the shifted denominator as the diagonal of the linear system found by
probing it with unit amplitudes, and its natural-orbital form; the direct
solution's residual and antisymmetry, and the diagonally preconditioned
iteration converging to it.
"""
import numpy as np
import pytest

import synth
from oracle import dsrg, dyall
from oracle.mkgno import Op, commutator


def _random_aavv(rng, nv, m):
    t = rng.standard_normal((nv, nv, m, m))
    t = t - t.transpose(1, 0, 2, 3)
    return t - t.transpose(0, 1, 3, 2)


@pytest.mark.parametrize("shape", [(1, 3, 2, 2, 6), (0, 2, 2, 3, 6)], ids=["c1a3v2", "c0a2v3"])
def test_printed_terms_equal_the_generic_commutator(shape):
    inst = synth.make_instance(*shape, 0.5, seed=31 + sum(shape))
    P = dsrg.SpinOrbitalProblem(inst)
    act = np.where(P.actm)[0]
    vir = np.where(P.vir)[0]
    Vact = np.zeros_like(P.V)
    Vact[np.ix_(act, act, act, act)] = P.V[np.ix_(act, act, act, act)]
    t = _random_aavv(np.random.default_rng(2), len(vir), len(act))
    T2 = np.zeros_like(P.V)
    T2[np.ix_(vir, vir, act, act)] = t
    H0 = Op(P.nso, 0.0, {1: np.diag(P.eps), 2: Vact})
    C = commutator(H0, Op(P.nso, 0.0, {2: T2}), P.ref, out_max=2).z[2][np.ix_(vir, vir, act, act)]
    Vs, Va, g, D = dyall.blocks(inst)
    want = -D * t + dyall.coupling(t, Va, g)
    assert np.abs(C - want).max() <= 1e-13 * np.abs(want).max()


def test_moller_plesset_limit():
    inst = synth.make_instance(1, 3, 2, 3, 8, 0.5, seed=4)
    Vs, Va, g, D = dyall.blocks(inst)
    t = dyall.solve(Vs, np.zeros_like(Va), g, D)
    m = Va.shape[0]
    off = ~np.eye(m, dtype=bool)
    want = np.where(off[None, None], Vs / np.where(off[None, None], D, 1.0), 0.0)
    assert np.abs(t - want).max() <= 1e-13 * np.abs(want).max()


def test_shifted_denominator_is_the_diagonal():
    inst = synth.make_instance(1, 3, 2, 2, 6, 0.5, seed=9)
    Vs, Va, g, D = dyall.blocks(inst)
    Ds = dyall.shifted_denominators(Va, g, D)
    nv, _, m, _ = Vs.shape
    for (a, b, u, v) in [(0, 1, 0, 1), (1, 2, 1, 4), (3, 0, 5, 2), (2, 2, 3, 0)]:
        t = np.zeros_like(Vs)
        t[a, b, u, v], t[a, b, v, u] = 1.0, -1.0
        coef = -(dyall.residual(t, np.zeros_like(Vs), Va, g, D)[a, b, u, v])
        assert abs(coef - Ds[a, b, u, v]) <= 1e-13 * max(1.0, abs(coef))
    # natural orbitals (diagonal gamma): D + v^{uv}_{uv} (1 - n_u - n_v)
    n = np.linspace(0.1, 0.9, m)
    Dn = dyall.shifted_denominators(Va, np.diag(n), D)
    i = np.arange(m)
    vuv = Va[i[:, None], i[None, :], i[:, None], i[None, :]]
    want = D + (vuv * (1.0 - n[:, None] - n[None, :]))[None, None]
    assert np.abs(Dn - want).max() <= 1e-13 * np.abs(want).max()


def test_direct_solution_and_preconditioned_iteration():
    inst = synth.config_instance("cas44_c2_v12_q60")
    Vs, Va, g, D = dyall.blocks(inst)
    t = dyall.solve(Vs, Va, g, D)
    assert np.abs(dyall.residual(t, Vs, Va, g, D)).max() <= 1e-12 * np.abs(Vs).max()
    assert np.abs(t + t.transpose(1, 0, 2, 3)).max() <= 1e-12 and np.abs(t + t.transpose(0, 1, 3, 2)).max() <= 1e-12
    Ds = dyall.shifted_denominators(Va, g, D)
    m = Va.shape[0]
    off = ~np.eye(m, dtype=bool)[None, None]
    x = np.zeros_like(Vs)
    for _ in range(40):
        x = x + np.where(off, dyall.residual(x, Vs, Va, g, D) / np.where(off, Ds, 1.0), 0.0)
    assert np.abs(x - t).max() <= 1e-12 * np.abs(t).max()
