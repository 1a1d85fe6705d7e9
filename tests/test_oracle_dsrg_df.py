"""Pins of the block-restricted, density-fitted oracle (oracle.dsrg_df).

It evaluates the same steps as oracle.dsrg (itself pinned by Fock-space brute
force, MP2/MP3 limits and invariances) on orbital blocks only, with the
two-electron integrals built from B^Q_pq and the particle-particle ladder
formed from B slab by slab.  Here it must reproduce the dense oracle's
energies and intermediates to rounding on shapes that cover empty core,
active or virtual spaces, ragged sizes, the CAS(4,4) workload and the
off-diagonal Fock source term, and its closed form of W = [H(0), A(1)] must
equal the dense oracle's generic commutator.
"""
import numpy as np
import pytest

import synth
from oracle import dsrg, dsrg_df

SHAPES = [
    (1, 3, 2, 2, 5),
    (2, 2, 2, 3, 6),
    (0, 3, 2, 2, 5),    # no core
    (2, 0, 0, 3, 6),    # no active space
    (1, 2, 2, 0, 4),    # no virtuals
    (2, 4, 4, 12, 60),  # the CAS(4,4) workload's sizes
]


def _close(a, b, rel=1e-12, floor=1e-15):
    return abs(a - b) <= rel * abs(a) + floor


@pytest.mark.parametrize("shape", SHAPES, ids=[str(s) for s in SHAPES])
def test_block_oracle_matches_dense_oracle(shape):
    inst = synth.make_instance(*shape, 0.5, seed=sum(shape) + 11)
    a = dsrg.dsrg_pt3(inst)
    b = dsrg_df.dsrg_pt3(inst)
    for k in ("e2", "e3a", "e3b", "e3"):
        assert _close(a[k], b[k]), (k, a[k], b[k])


def test_block_oracle_with_offdiagonal_fock():
    inst = synth.make_instance(1, 3, 2, 3, 8, 0.5, seed=19)
    f1 = np.random.default_rng(4).standard_normal((7, 7)) * 0.05
    inst["f1"] = f1 + f1.T
    a = dsrg.dsrg_pt3(inst)
    b = dsrg_df.dsrg_pt3(inst)
    for k in ("e2", "e3a", "e3b"):
        assert _close(a[k], b[k]), (k, a[k], b[k])


def _dense_block(full, sp, spaces):
    return full[np.ix_(*[sp[s] for s in spaces])]


def test_block_intermediates_and_closed_form_w():
    """T1, T2, W (closed form vs the dense oracle's generic [H(0), A(1)]),
    the excitation blocks of O, and the second-order amplitudes."""
    inst = synth.make_instance(2, 3, 2, 4, 14, 0.7, seed=5)
    a = dsrg.dsrg_pt3(inst, return_intermediates=True)
    b = dsrg_df.dsrg_pt3(inst, return_intermediates=True)
    A, Bi, sp = a["_inter"], b["_inter"], b["_problem"].sp
    pairs = [("T1", A["T1"], ("P", "H")), ("T2", A["T2"], ("P", "P", "H", "H")),
             ("W1", A["W"].z[1], ("P", "H")), ("W2", A["W"].z[2], ("P", "P", "H", "H")),
             ("T1b", A["T1b"], ("P", "H")), ("T2b", A["T2b"], ("P", "P", "H", "H"))]
    for name, full, spaces in pairs:
        want = _dense_block(full, sp, spaces)
        got = Bi[name]
        assert np.abs(got - want).max() <= 1e-13 * max(1.0, np.abs(want).max()), name
    # O's excitation blocks outside the internal (all-active) elements
    P = b["_problem"]
    w1 = _dense_block(A["O"].z[1], sp, ("P", "H"))
    w2 = _dense_block(A["O"].z[2], sp, ("P", "P", "H", "H"))
    assert np.abs((Bi["O1"] - w1)[P.mask1]).max() <= 1e-13 * max(1.0, np.abs(w1).max())
    assert np.abs((Bi["O2"] - w2)[P.mask2]).max() <= 1e-13 * max(1.0, np.abs(w2).max())
    # W has no internal part and is the full generic commutator outside its
    # two excitation blocks and their images (all other blocks vanish)
    W = A["W"]
    H_, P_ = sp["H"], sp["P"]
    rest = W.z[2].copy()
    rest[np.ix_(P_, P_, H_, H_)] = 0.0
    rest[np.ix_(H_, H_, P_, P_)] = 0.0
    assert np.abs(rest).max() < 1e-13


def test_ladder_slabs_cover_all_rows():
    """The all-particle block enters only through the slab-wise ladder: a
    particle space longer than one slab (8 rows) with a ragged last slab."""
    inst = synth.make_instance(1, 2, 2, 8, 20, 0.5, seed=9)   # 2 x 10 = 20 particle spin orbitals
    a = dsrg.dsrg_pt3(inst)
    b = dsrg_df.dsrg_pt3(inst)
    for k in ("e3a", "e3b"):
        assert _close(a[k], b[k]), (k, a[k], b[k])


def test_ladder_sample_rows_match_dense_ladder():
    """LadderSample (the oracle's ladder on a few rows, used as the timed CPU
    sample) against sum_rs <pq||rs> (eta eta T2)[r,s,i,j] from the dense
    oracle's integrals and amplitudes."""
    inst = synth.make_instance(1, 2, 2, 4, 10, 0.5, seed=13)
    a = dsrg.dsrg_pt3(inst, pt2_only=True, return_intermediates=True)
    P = a["_problem"]
    part = np.where(P.part)[0]
    eta = P.ref.eta[np.ix_(part, part)]
    T2 = a["_inter"]["T2"][np.ix_(part, part, np.where(P.hole)[0], np.where(P.hole)[0])]
    M = np.einsum("ce,df,efij->cdij", eta, eta, T2)
    want = np.einsum("pqrs,rsij->pqij", P.V[np.ix_(part, part, part, part)], M)
    s = dsrg_df.LadderSample(inst)
    got = np.concatenate([s.rows(0, 5), s.rows(5, s.nrows)])
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()
