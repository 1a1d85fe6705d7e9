"""Pins of the one-step relaxed energies of the oracle (oracle.relaxed,
Eq. E_relaxed with App. A).

Fixed by:
* Fock-space brute force: the full operator Hbar^[k]_{1,2} (every block, core
  and virtual included) in Mukherjee-Kutzelnigg normal order relative to the
  reference, built as an explicit matrix on the whole N-electron space and
  restricted to the reference's determinant space (Eq. energy_relaxed taken
  literally), must equal the matrix the oracle builds from the all-active
  elements alone through Eq. Hbar_DNO and the core folding of Eq. c0_cas;
* the CI builder against plain second quantisation in an explicit Fock space
  for random one- and two-body coefficients;
* the expectation value over the reference, which must be the unrelaxed
  energy (the scalar of Hbar^[k]), and the variational bound;
* no active space: one determinant, relaxed = unrelaxed.
"""
import numpy as np
import pytest

import synth
from oracle import fockspace as fsm
from oracle import relaxed
from _fock_helpers import mr_fock_instance


def _cas_projection(M, fs, nc, na, n, dets_active):
    """Rows/columns of the full-space matrix M at the determinants with the
    core filled, virtuals empty and the given active occupations."""
    idx = []
    for d in dets_active:
        full = 0
        for m in range(nc):
            full |= 1 << m
            full |= 1 << (n + m)
        for u in range(na):
            if d >> u & 1:
                full |= 1 << (nc + u)
            if d >> (na + u) & 1:
                full |= 1 << (n + nc + u)
        idx.append(fs.sec[0].index[full])
    return M[np.ix_(idx, idx)]


@pytest.mark.parametrize("shape", [(1, 2, 2, 2), (2, 2, 2, 1), (0, 3, 2, 2), (1, 3, 4, 1)],
                         ids=["c1a2v2", "c2a2v1", "c0a3v2", "c1a3v1-4e"])
@pytest.mark.parametrize("order", [2, 3])
def test_ci_matrix_equals_fock_space_projection(shape, order):
    nc, na, nel, nv = shape
    inst, fs, psi, g, act, lam = mr_fock_instance(nc, na, nel, nv, 6, 0.5, seed=40 + sum(shape) + order)
    n = nc + na + nv
    hb, P, _ = relaxed.hbar_operator(inst, order=order)
    M = fsm.operator_matrix(fs, hb.c0, {k: hb.z[k] for k in (1, 2) if k in hb.z}, g, act, lam)
    out = relaxed.relaxed_energies(inst, nel // 2, nel // 2, orders=(order,))
    p = out[f"_pieces{order}"]
    Mp = _cas_projection(M, fs, nc, na, n, p["dets"])
    scale = np.abs(Mp).max()
    assert np.abs(Mp - p["H"]).max() <= 1e-12 * scale
    # and the reference state has the unrelaxed energy in both pictures
    assert abs(psi @ M @ psi - hb.c0) <= 1e-12 * scale


def test_ci_builder_against_plain_second_quantisation():
    rng = np.random.default_rng(3)
    na = 3
    m = 2 * na
    c = rng.standard_normal((m, m))
    w = fsm.random_antisym(rng, m, 2)
    fs = fsm.FockSpace(m, 3, kmax=2)
    M = 0.7 * np.eye(fs.dim) + fs.plain(c, 1) + fs.plain(w, 2)
    for nalpha, nbeta in [(2, 1), (1, 2), (3, 0)]:
        dets = relaxed.determinants(na, nalpha, nbeta)
        H = relaxed.ci_matrix(0.7, c, w, dets)
        idx = [fs.sec[0].index[d] for d in dets]
        assert np.abs(H - M[np.ix_(idx, idx)]).max() <= 1e-13 * np.abs(M).max()


@pytest.mark.parametrize("order", [2, 3])
def test_reference_expectation_is_the_unrelaxed_energy(order):
    inst = synth.make_instance(2, 4, 4, 3, 12, 0.5, seed=21, with_so=True)
    out = relaxed.relaxed_energies(inst, 2, 2, orders=(order,))
    p = out[f"_pieces{order}"]
    idx = {d: k for k, d in enumerate(p["dets"])}
    v = np.zeros(len(p["dets"]))
    for d, x in zip(inst["dets"], inst["ci"]):
        v[idx[d]] = x
    want = out["e2"] + (out["e3"] if order == 3 else 0.0)
    assert abs(p["h0"] - want) <= 1e-12 * abs(want)
    assert abs(v @ p["H"] @ v - want) <= 1e-11 * np.abs(p["H"]).max()
    assert out[f"e_relaxed{order}"] <= want + 1e-12


def test_no_active_space_relaxed_equals_unrelaxed():
    inst = synth.make_instance(2, 0, 0, 3, 10, 0.5, seed=8)
    out = relaxed.relaxed_energies(inst, 0, 0)
    assert len(out["_pieces3"]["dets"]) == 1
    assert out["e_relaxed2"] == pytest.approx(out["e2"], rel=1e-13, abs=1e-15)
    assert out["e_relaxed3"] == pytest.approx(out["e2"] + out["e3"], rel=1e-13, abs=1e-15)
