"""Pins of the input generator: density cumulants of the CAS reference.

The method takes the reference only through gamma1, lambda2 and lambda3
(Sec. II.A; Conclusions: at most the three-body cumulant is needed).  These
checks fix the cumulant construction by properties that hold exactly.
"""
import numpy as np
import pytest

import synth
from oracle import fockspace as fsm

from _fock_helpers import product_dets_signs


def test_single_determinant_has_no_cumulants():
    dets = synth.ms0_determinants(3, 4)
    ci = np.zeros(len(dets))
    ci[4] = 1.0
    ref = synth.reference_from_ci(3, 4, ci=ci, dets=dets)
    assert np.abs(ref["l2_so"]).max() < 1e-14
    assert np.abs(ref["l3_so"]).max() < 1e-14
    g = ref["g1_so"]
    assert np.allclose(g @ g, g)  # idempotent


def test_trace_and_partial_trace_identities():
    rng = np.random.default_rng(4)
    ref = synth.reference_from_ci(3, 4, rng=rng)
    g, l2 = ref["g1_so"], ref["l2_so"]
    assert abs(np.trace(g) - 4.0) < 1e-12
    # sum_q G2[p,q,r,q] = (N-1) g[p,r]  =>  sum_q l2[p,q,r,q] = (g^2 - g)[p,r]
    pt = np.einsum("pqrq->pr", l2)
    assert np.allclose(pt, g @ g - g, atol=1e-13)
    # Ms = 0: no alpha-beta block in gamma
    na = 3
    assert np.abs(g[:na, na:]).max() == 0.0


def test_rdms_match_fock_space():
    """Two independent constructions of the RDMs of the same state."""
    rng = np.random.default_rng(9)
    na, nel = 3, 2
    dets = synth.ms0_determinants(na, nel)
    ci = rng.standard_normal(len(dets))
    ci /= np.linalg.norm(ci)
    g1, G2, G3 = synth.rdms(2 * na, dets, ci, 3)
    fs = fsm.FockSpace(2 * na, nel, kmax=3)
    psi = fs.state(dets, ci)
    assert np.allclose(fs.rdm(psi, 1), g1, atol=1e-14)
    assert np.allclose(fs.rdm(psi, 2), G2, atol=1e-14)
    assert np.allclose(fs.rdm(psi, 3), G3, atol=1e-14)


def test_cumulants_are_additively_separable():
    """A fermionic product of two states has no cumulant across the parts."""
    rng = np.random.default_rng(2)
    da = synth.ms0_determinants(2, 2)
    db = synth.ms0_determinants(2, 2)
    ca = rng.standard_normal(len(da))
    cb = rng.standard_normal(len(db))
    dets, signs = product_dets_signs(da, 2, db, 2)
    ci = np.array([x * y for x in ca for y in cb]) * signs
    ref = synth.reference_from_ci(4, 4, ci=ci, dets=dets)
    l2, l3 = ref["l2_so"], ref["l3_so"]
    # spin orbitals of part a: alpha 0,1 and beta 4,5; of part b: 2,3,6,7
    A = [0, 1, 4, 5]
    Bp = [2, 3, 6, 7]
    mixed2 = 0.0
    for idx in np.ndindex(*l2.shape):
        parts = {x in A for x in idx}
        if len(parts) > 1:
            mixed2 = max(mixed2, abs(l2[idx]))
    assert mixed2 < 1e-13
    sub = np.ix_(*[A] * 6)
    l3_mixed = l3.copy()
    l3_mixed[sub] = 0.0
    l3_mixed[np.ix_(*[Bp] * 6)] = 0.0
    assert np.abs(l3_mixed).max() < 1e-13
    # and within a part the cumulants are those of the part alone
    ra = synth.reference_from_ci(2, 2, ci=ca, dets=da)
    assert np.allclose(l3[np.ix_(*[A] * 6)], ra["l3_so"], atol=1e-13)
    assert np.abs(ra["l3_so"]).max() > 1e-6 or np.abs(ra["l2_so"]).max() > 1e-3


def test_instances_are_deterministic():
    a = synth.config_instance("cas44_c2_v12_q60")
    b = synth.config_instance("cas44_c2_v12_q60")
    for k in ("eps", "B", "l3aab"):
        assert np.array_equal(a[k], b[k])
    assert np.allclose(a["B"], np.transpose(a["B"], (0, 2, 1)))


def test_scan_recipe():
    """The 32-point scan: core 4..12, CAS(4,4) or CAS(6,6), virtual 60..200,
    aux = 4 x virtual, and the virtual band's lower edge falling linearly
    from 0.6 to 0.05 Eh along the scan (shrinking gaps, as in dissociation)."""
    sizes = [synth.scan_sizes(j) for j in range(32)]
    for j, z in enumerate(sizes):
        assert 4 <= z["nc"] <= 12 and z["na"] in (4, 6) and 60 <= z["nv"] <= 200
        assert z["naux"] == 4 * z["nv"]
        assert abs(z["vlo"] - (0.6 - 0.55 * j / 31)) < 1e-12
    assert len({(z["nc"], z["nv"]) for z in sizes}) > 20  # uneven sizes
    for j in (0, 31):  # two full instances: sizes and the virtual band
        inst = synth.scan_instance(j)
        z = sizes[j]
        assert (inst["nc"], inst["na"], inst["nv"], inst["naux"]) == (z["nc"], z["na"], z["nv"], z["naux"])
        eps_v = np.asarray(inst["eps"])[z["nc"] + z["na"]:]
        assert eps_v.min() >= z["vlo"] - 1e-12 and eps_v.max() <= 5.0


def test_synthetic_reference_has_cumulant_symmetries():
    """Synthetic references for large active spaces: gamma1 symmetric with
    eigenvalues in [0, 1]; lambda2, lambda3 assembled from the spin blocks
    are antisymmetric in creators and in annihilators and Hermitian."""
    from oracle.dsrg import _spin_tensor
    na = 4
    d = synth.synthetic_reference(na, np.random.default_rng(7))
    for k in ("g1a", "g1b"):
        g = d[k]
        assert np.allclose(g, g.T)
        w = np.linalg.eigvalsh(g)
        assert w.min() >= -1e-12 and w.max() <= 1 + 1e-12
    l2 = _spin_tensor({0: d["l2aa"], 1: d["l2ab"], 2: d["l2bb"]}, na, 2)
    l3 = _spin_tensor({0: d["l3aaa"], 1: d["l3aab"], 2: d["l3abb"], 3: d["l3bbb"]}, na, 3)
    assert np.abs(l2 + l2.transpose(1, 0, 2, 3)).max() < 1e-15
    assert np.abs(l2 + l2.transpose(0, 1, 3, 2)).max() < 1e-15
    assert np.abs(l2 - l2.transpose(2, 3, 0, 1)).max() < 1e-15
    for perm in ((1, 0, 2, 3, 4, 5), (0, 2, 1, 3, 4, 5), (0, 1, 2, 4, 3, 5), (0, 1, 2, 3, 5, 4)):
        assert np.abs(l3 + l3.transpose(perm)).max() < 1e-15
    assert np.abs(l3 - l3.transpose(3, 4, 5, 0, 1, 2)).max() < 1e-15


def test_block_oracle_matches_dense_oracle_on_a_synthetic_cas88():
    """The large-active regime (lambda3 terms of order N_A^6 N_V): the two
    oracles agree on a synthetic 8-orbital active space."""
    from oracle import dsrg, dsrg_df
    inst = synth.make_synthetic_instance(1, 8, 3, 12, seed=8)
    a, b = dsrg.dsrg_pt3(inst), dsrg_df.dsrg_pt3(inst)
    for k in ("e2", "e3a", "e3b"):
        assert abs(a[k] - b[k]) <= 1e-12 * abs(a[k]) + 1e-15, k
