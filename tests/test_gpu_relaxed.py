"""GPU one-step relaxed energies (dsrg_relaxed; Eq. E_relaxed, App. A) against
the oracle (oracle.relaxed).

* Small instances (the oracle's dense engine): the all-active blocks of
  Hbar^[2] and of the third-order additions element by element (1e-10 of
  their largest element), and the relaxed energies within 1e-9 Eh, on the
  FP64 path; the split path within 1e-6 Eh.
* The CAS(6,6)/10 core/100 virtual/400 aux workload (400 determinants, too
  large for the dense oracle): the oracle's App. A reduction and CI matrix
  built from the GPU's active blocks must give the GPU's relaxed energies
  (1e-9 Eh) and, over the reference CI vector, the unrelaxed energy; the
  relaxed energy lies below the unrelaxed one and its eigenvector residual
  is small.
* No active space: one determinant, relaxed = unrelaxed; electron counts
  outside [0, na] are rejected.
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


SMALL = [((1, 3, 2, 2, 6), 1, 1, 7), ((2, 4, 4, 3, 12), 2, 2, 21), ((1, 2, 2, 8, 20), 1, 1, 5)]


@pytest.mark.parametrize("case", SMALL, ids=["c1a3v2", "c2a4v3", "c1a2v8"])
def test_relaxed_matches_oracle(lib, case):
    from oracle import relaxed
    (nc, na, nel, nv, naux), nalpha, nbeta, seed = case
    inst = synth.make_instance(nc, na, nel, nv, naux, 0.5, seed=seed)
    ref = relaxed.relaxed_energies(inst, nalpha, nbeta)
    h = lib.Dsrg(_device(inst))
    try:
        got = h.relaxed(nalpha, nbeta)
        b12, b22 = h.fetch("Hbar1_2"), h.fetch("Hbar2_2")
        b13, b23 = h.fetch("Hbar1_3"), h.fetch("Hbar2_3")
    finally:
        h.close()
    p2, p3 = ref["_pieces2"], ref["_pieces3"]
    for got_b, want in [(b12, p2["h1"]), (b22, p2["h2"]), (b13, p3["h1"] - p2["h1"]), (b23, p3["h2"] - p2["h2"])]:
        assert np.abs(got_b - want).max() <= 1e-10 * max(1.0, np.abs(want).max())
    for k in ("e2", "e3a", "e3b", "e3", "e_relaxed2", "e_relaxed3"):
        assert abs(got[k] - ref[k]) < 1e-9, (k, got[k], ref[k])
    assert got["ndet"] == len(p3["dets"])
    assert got["residual3"] < 1e-8


def test_relaxed_split_path(lib):
    from oracle import relaxed
    inst = synth.config_instance("cas44_c2_v12_q60")
    ref = relaxed.relaxed_energies(inst, 2, 2)
    h = lib.Dsrg(_device(inst), precision=lib.DSRG_PREC_SPLIT, slices=6)
    try:
        got = h.relaxed(2, 2)
    finally:
        h.close()
    for k in ("e_relaxed2", "e_relaxed3"):
        assert abs(got[k] - ref[k]) < 1e-6, (k, got[k], ref[k])


def test_relaxed_full_size_cas66(lib):
    from oracle import relaxed
    inst = synth.config_instance("cas66_c10_v100_q400", with_so=True)
    h = lib.Dsrg(_device(inst))
    try:
        got = h.relaxed(3, 3)
        b = {k: h.fetch(k) for k in ("Hbar1_2", "Hbar2_2", "Hbar1_3", "Hbar2_3")}
    finally:
        h.close()
    na = inst["na"]
    assert got["ndet"] == 400
    # the reference densities on active spin orbitals
    g1 = np.asarray(inst["g1_so"])
    l2 = np.asarray(inst["l2_so"])
    g2 = relaxed.two_rdm(g1, l2)
    dets = relaxed.determinants(na, 3, 3)
    idx = {d: k for k, d in enumerate(dets)}
    v = np.zeros(len(dets))
    for d, x in zip(inst["dets"], inst["ci"]):
        v[idx[d]] = x
    for order, h0 in ((2, got["e2"]), (3, got["e2"] + got["e3"])):
        h1 = b["Hbar1_2"] + (b["Hbar1_3"] if order == 3 else 0.0)
        h2 = b["Hbar2_2"] + (b["Hbar2_3"] if order == 3 else 0.0)
        Es, c, w = relaxed.dno_active(h0, h1, h2, g1, g2)
        H = relaxed.ci_matrix(Es, c, w, dets)
        scale = np.abs(H).max()
        assert abs(v @ H @ v - h0) <= 1e-11 * scale
        e_min = np.linalg.eigvalsh(H)[0]
        assert abs(got[f"e_relaxed{order}"] - e_min) < 1e-9
        assert got[f"e_relaxed{order}"] <= h0 + 1e-9
        assert got[f"residual{order}"] < 1e-8 * max(1.0, abs(e_min))


def test_no_active_space_and_bad_counts(lib):
    inst = synth.make_instance(2, 0, 0, 3, 10, 0.5, seed=8)
    h = lib.Dsrg(_device(inst))
    try:
        got = h.relaxed(0, 0)
        assert got["ndet"] == 1
        assert abs(got["e_relaxed2"] - got["e2"]) < 1e-12
        assert abs(got["e_relaxed3"] - (got["e2"] + got["e3"])) < 1e-12
    finally:
        h.close()
    inst = synth.make_instance(1, 2, 2, 3, 8, 0.5, seed=9)
    h = lib.Dsrg(_device(inst))
    try:
        for na_, nb_ in [(3, 1), (-1, 1), (1, 5)]:
            with pytest.raises(lib.DsrgError):
                h.relaxed(na_, nb_)
    finally:
        h.close()
