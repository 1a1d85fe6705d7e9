"""Pins of the generalized-normal-order commutator engine against brute force.

For random one- and two-body operators X, Y and a genuinely multireference
state, the engine's [X, Y] = C0 + C1 + C2 + C3 (all ranks kept) must equal
the matrix commutator in an explicit Fock space.  This fixes every
contraction pattern, sign and multiplicity the engine generates, and
therefore the meaning of the 1,2-body truncation used in the paper
(after Eq. exactBCH; Eq. E(3) approximation).
"""
import numpy as np
import pytest

import synth
from oracle import fockspace as fsm
from oracle import mkgno


def _reference(nso, core, act, nel_act, seed):
    rng = np.random.default_rng(seed)
    nact = len(act)
    adets = fsm._bits(nact, nel_act)
    ci = rng.standard_normal(len(adets))
    ci /= np.linalg.norm(ci)
    cbits = 0
    for c in core:
        cbits |= 1 << c
    full = []
    for d in adets:
        b = cbits
        for k in range(nact):
            if d >> k & 1:
                b |= 1 << int(act[k])
        full.append(b)
    fs = fsm.FockSpace(nso, len(core) + nel_act, kmax=3)
    psi = fs.state(full, ci)
    g = fs.rdm(psi, 1)
    G2 = fs.rdm(psi, 2)
    G3 = fs.rdm(psi, 3)
    l2, l3 = synth.cumulants(g[np.ix_(act, act)], G2[np.ix_(*[act] * 4)], G3[np.ix_(*[act] * 6)])
    lam = {2: l2, 3: l3}
    ref = mkgno.Reference(gamma=g, eta=np.eye(nso) - g, act=np.asarray(act), lam=lam)
    return fs, psi, g, lam, ref


CASES = [
    # (nso, core spin orbitals, active spin orbitals, active electrons)
    (8, [0, 1], np.array([2, 3, 4, 5]), 2),
    (10, [0, 1], np.array([2, 3, 4, 5, 6, 7]), 3),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_normal_ordered_operators_have_zero_expectation(case):
    nso, core, act, ne = CASES[case]
    fs, psi, g, lam, ref = _reference(nso, core, act, ne, seed=10 + case)
    rng = np.random.default_rng(1)
    for k in (1, 2, 3):
        Z = fsm.random_antisym(rng, nso, k)
        M = fsm.normal_ordered(fs, Z, k, g, act, lam)
        assert abs(psi @ M @ psi) < 1e-12 * max(1.0, np.abs(Z).max())


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("kx,ky", [(1, 1), (1, 2), (2, 1), (2, 2)])
def test_commutator_matches_fock_space(case, kx, ky):
    nso, core, act, ne = CASES[case]
    fs, psi, g, lam, ref = _reference(nso, core, act, ne, seed=20 + case)
    rng = np.random.default_rng(100 * kx + ky)
    X = fsm.random_antisym(rng, nso, kx)
    Y = fsm.random_antisym(rng, nso, ky)
    C = mkgno.commutator(mkgno.Op(nso, 0.0, {kx: X}), mkgno.Op(nso, 0.0, {ky: Y}), ref, out_max=3)
    MX = fsm.normal_ordered(fs, X, kx, g, act, lam)
    MY = fsm.normal_ordered(fs, Y, ky, g, act, lam)
    exact = MX @ MY - MY @ MX
    M = fsm.operator_matrix(fs, C.c0, C.z, g, act, lam)
    assert np.abs(M - exact).max() < 1e-11 * np.abs(exact).max()
    # the scalar part is the reference expectation value
    assert abs(C.c0 - psi @ exact @ psi) < 1e-11 * np.abs(exact).max()


def test_single_determinant_normal_order_is_particle_hole_order():
    """With one determinant, MK normal order is ordinary quasi-particle order,
    built here by reordering operators with no contractions at all."""
    rng = np.random.default_rng(3)
    occ = [0, 1, 2, 3]
    fs = fsm.FockSpace(8, 4, kmax=3)
    g = np.zeros((8, 8))
    g[occ, occ] = 1.0
    empty = np.array([], dtype=int)
    lam = {2: np.zeros((0,) * 4), 3: np.zeros((0,) * 6)}
    for k in (1, 2):
        Z = fsm.random_antisym(rng, 8, k)
        a = fsm.normal_ordered(fs, Z, k, g, empty, lam)
        b = fsm.quasiparticle_normal_ordered(fs, Z, k, occ)
        assert np.abs(a - b).max() < 1e-12 * np.abs(Z).max()


def test_pattern_multiplicities_count_all_contractions():
    """Sum of multiplicities equals a direct count of contraction sets for
    [2,2] with pairs only (ladders, rings and their partial versions)."""
    pats = mkgno.enumerate_patterns(2, 2, lam_max=1, out_max=4, commutator=False)
    # direct count: choose k gamma pairs (L cre x R ann) and m eta pairs
    from math import comb, factorial
    direct = 0
    for k in range(3):
        for m in range(3):
            if k + m == 0:
                continue
            direct += comb(2, k) ** 2 * factorial(k) * comb(2, m) ** 2 * factorial(m)
    assert sum(mult for _, mult in pats) == direct
