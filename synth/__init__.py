"""Seeded synthetic inputs for the DSRG-MRPT2/PT3 energy path.

This module only *makes inputs*: orbital energies, a symmetric three-index
factor B^Q_pq and a complete-active-space reference (a random CI vector) with
its exact one-particle density and two-/three-body density cumulants.  It holds
none of the perturbation theory itself; both the CPU oracle and the GPU path
read the arrays produced here.

Conventions (spin orbitals of the active space are ordered alpha block first,
then beta block; a determinant is the product of creators in ascending
spin-orbital order acting on the vacuum):

* ``g1[p,q]   = <a+_p a_q>``
* ``G2[p,q,r,s] = <a+_p a+_q a_s a_r>``
* ``G3[p,q,r,s,t,u] = <a+_p a+_q a+_r a_u a_t a_s>``
* ``l2 = G2 - g1^g1`` and ``l3 = G3 - A(g1 g1 g1) - A(g1 l2)`` (density
  cumulants, Sec. II of the paper: the reference enters only through them).

The workloads mirror the configurations the paper's method is timed on: a
CAS(n,n) reference with core, active and virtual blocks, DF auxiliary index
of a few times the orbital count (Eq. int_fact, M ~ 3N).
"""
from __future__ import annotations

import math
from itertools import combinations, permutations

import numpy as np

SEED0 = 170102011

# name -> sizes; (nc, na, nel, nv, naux, s)
CONFIGS = {
    "cas44_c2_v12_q60": dict(nc=2, na=4, nel=4, nv=12, naux=60, s=0.5, seed=SEED0 + 0),
    "cas66_c10_v100_q400": dict(nc=10, na=6, nel=6, nv=100, naux=400, s=0.5, seed=SEED0 + 1),
    "cas88_c30_v300_q1200": dict(nc=30, na=8, nel=8, nv=300, naux=1200, s=0.5, seed=SEED0 + 2),
    "cas44_c40_v500_q1800": dict(nc=40, na=4, nel=4, nv=500, naux=1800, s=0.5, seed=SEED0 + 4),
}

EPS_CORE = (-20.0, -0.5)
EPS_ACT = (-0.3, 0.3)
EPS_VIR = (0.2, 5.0)


# ----------------------------------------------------------------------------
# determinant strings and the active-space state
# ----------------------------------------------------------------------------

def _strings(norb: int, nel: int) -> list[int]:
    """Occupation bitstrings of ``nel`` electrons in ``norb`` orbitals, ascending."""
    out = []
    for occ in combinations(range(norb), nel):
        b = 0
        for o in occ:
            b |= 1 << o
        out.append(b)
    return sorted(out)


def ms0_determinants(na: int, nel: int) -> list[int]:
    """Ms=0 determinants of CAS(nel, na) as 2*na-bit strings (alpha bits low)."""
    if nel % 2:
        raise ValueError("Ms=0 needs an even electron count")
    sa = _strings(na, nel // 2)
    return [a | (b << na) for a in sa for b in sa]


class FockVector:
    """A state in one particle-number sector of a small Fock space."""

    def __init__(self, nso: int, dets: list[int], coef: np.ndarray):
        self.nso = nso
        self.dets = list(dets)
        self.coef = np.asarray(coef, dtype=np.float64)


def _annihilate_all(nso, dets, coefs_rows):
    """Apply a_s for every spin orbital s to each row-state.

    ``coefs_rows`` has shape (nrow, len(dets)).  Returns (new_dets,
    new_rows[s]) where new_rows[s] has shape (nrow, len(new_dets)).
    """
    nel = bin(dets[0]).count("1") if dets else 0
    new_dets = _sector(nso, nel - 1)
    index = {d: k for k, d in enumerate(new_dets)}
    out = np.zeros((nso, coefs_rows.shape[0], len(new_dets)))
    for k, d in enumerate(dets):
        for s in range(nso):
            if d >> s & 1:
                sign = -1.0 if bin(d & ((1 << s) - 1)).count("1") % 2 else 1.0
                out[s, :, index[d ^ (1 << s)]] += sign * coefs_rows[:, k]
    return new_dets, out


def _sector(nso, nel):
    return _strings(nso, nel) if nel >= 0 else []


def rdms(nso: int, dets: list[int], coef: np.ndarray, kmax: int = 3):
    """Exact spin-orbital reduced density matrices G1..G_kmax of a state.

    G_k[p1..pk, q1..qk] = <a+_p1 .. a+_pk a_qk .. a_q1>, computed as overlaps
    of the vectors a_qk..a_q1|Psi> for ordered tuples, then antisymmetrised.
    """
    out = []
    rows = coef[None, :].copy()
    cur_dets = list(dets)
    # phi[tuple] for ascending tuples built incrementally: a_{qk} acts last
    tuples = [()]
    vecs = rows  # (ntuple, ndet)
    for k in range(1, kmax + 1):
        new_dets, ann = _annihilate_all(nso, cur_dets, vecs)
        new_tuples, new_rows = [], []
        for t_idx, t in enumerate(tuples):
            last = t[-1] if t else -1
            for s in range(last + 1, nso):
                new_tuples.append(t + (s,))
                new_rows.append(ann[s, t_idx])
        tuples = new_tuples
        vecs = np.array(new_rows) if new_rows else np.zeros((0, len(new_dets)))
        cur_dets = new_dets
        ov = vecs @ vecs.T  # <phi_P|phi_S>
        G = np.zeros((nso,) * (2 * k))
        perms = list(permutations(range(k)))
        psign = [_perm_sign(p) for p in perms]
        for a, P in enumerate(tuples):
            for b, S in enumerate(tuples):
                v = ov[a, b]
                if v == 0.0:
                    continue
                for p1, s1 in zip(perms, psign):
                    PP = tuple(P[i] for i in p1)
                    for p2, s2 in zip(perms, psign):
                        SS = tuple(S[i] for i in p2)
                        G[PP + SS] = s1 * s2 * v
        out.append(G)
    return out


def _perm_sign(p) -> int:
    p = list(p)
    s = 1
    for i in range(len(p)):
        for j in range(i + 1, len(p)):
            if p[i] > p[j]:
                s = -s
    return s


def cumulants(g1: np.ndarray, G2: np.ndarray, G3: np.ndarray | None = None):
    """Density cumulants l2 (and l3) from the RDMs."""
    l2 = G2 - np.einsum("pr,qs->pqrs", g1, g1) + np.einsum("ps,qr->pqrs", g1, g1)
    if G3 is None:
        return l2, None
    n = g1.shape[0]
    ggg = np.zeros((n,) * 6)
    for perm in permutations(range(3)):
        sg = _perm_sign(perm)
        lows = "stu"
        sub = "".join(lows[i] for i in perm)
        ggg += sg * np.einsum(f"p{sub[0]},q{sub[1]},r{sub[2]}->pqrstu", g1, g1, g1)
    gl = np.zeros((n,) * 6)
    ups, lows = "pqr", "stu"
    for i in range(3):
        for j in range(3):
            rest_u = "".join(ups[k] for k in range(3) if k != i)
            rest_l = "".join(lows[k] for k in range(3) if k != j)
            sg = -1.0 if (i + j) % 2 else 1.0
            gl += sg * np.einsum(f"{ups[i]}{lows[j]},{rest_u}{rest_l}->pqrstu", g1, l2)
    l3 = G3 - ggg - gl
    return l2, l3


def spin_blocks(na: int, g1, l2, l3):
    """Cut spin-orbital active tensors (alpha block first) into the spin blocks
    the library takes: g1a, g1b, l2aa, l2ab, l2bb, l3aaa, l3aab, l3abb, l3bbb."""
    A = slice(0, na)
    Bb = slice(na, 2 * na)
    return dict(
        g1a=np.ascontiguousarray(g1[A, A]),
        g1b=np.ascontiguousarray(g1[Bb, Bb]),
        l2aa=np.ascontiguousarray(l2[A, A, A, A]),
        l2ab=np.ascontiguousarray(l2[A, Bb, A, Bb]),
        l2bb=np.ascontiguousarray(l2[Bb, Bb, Bb, Bb]),
        l3aaa=np.ascontiguousarray(l3[A, A, A, A, A, A]),
        l3aab=np.ascontiguousarray(l3[A, A, Bb, A, A, Bb]),
        l3abb=np.ascontiguousarray(l3[A, Bb, Bb, A, Bb, Bb]),
        l3bbb=np.ascontiguousarray(l3[Bb, Bb, Bb, Bb, Bb, Bb]),
    )


def reference_from_ci(na: int, nel: int, ci: np.ndarray | None = None, rng=None, dets=None):
    """Active-space RDMs and cumulants of a CI vector over Ms=0 determinants
    (or over ``dets`` if given).  Returns the spin-block dict plus the full
    spin-orbital active tensors under keys g1_so, l2_so, l3_so."""
    nso = 2 * na
    if na == 0 or nel == 0:
        ci = np.ones(1)
        dets = [0]
        z2 = np.zeros((nso,) * 4)
        z3 = np.zeros((nso,) * 6)
        g1 = np.zeros((nso, nso))
        d = spin_blocks(na, g1, z2, z3)
        d.update(g1_so=g1, l2_so=z2, l3_so=z3, ci=ci, dets=dets)
        return d
    if dets is None:
        dets = ms0_determinants(na, nel)
    if ci is None:
        ci = rng.standard_normal(len(dets))
    ci = np.asarray(ci, dtype=np.float64).ravel()
    ci = ci / np.linalg.norm(ci)
    g1, G2, G3 = rdms(nso, dets, ci, 3)
    l2, l3 = cumulants(g1, G2, G3)
    d = spin_blocks(na, g1, l2, l3)
    d.update(g1_so=g1, l2_so=l2, l3_so=l3, ci=ci, dets=dets)
    return d


# ----------------------------------------------------------------------------
# three-index factor, orbital energies, full instances
# ----------------------------------------------------------------------------

def df_factor(rng, n: int, naux: int, scale: float = 0.1) -> np.ndarray:
    """B[Q,p,q]: Gaussian, symmetric in pq, row Q scaled by scale*exp(-3Q/naux)."""
    B = np.empty((naux, n, n))
    iu = np.triu_indices(n)
    for Q in range(naux):
        z = np.empty((n, n))
        z[iu] = rng.standard_normal(len(iu[0]))
        z.T[iu] = z[iu]
        B[Q] = z * (scale * math.exp(-3.0 * Q / naux))
    return B


def make_instance(nc: int, na: int, nel: int, nv: int, naux: int, s: float = 0.5,
                  seed: int = SEED0, eps_vir=EPS_VIR, eps_core=EPS_CORE, eps_act=EPS_ACT,
                  with_so: bool = False) -> dict:
    """One synthetic DSRG problem.  Draw order: core, active, virtual energies,
    CI vector, then B row by row in Q."""
    rng = np.random.default_rng(seed)
    eps = np.concatenate([
        rng.uniform(*eps_core, nc),
        rng.uniform(*eps_act, na),
        rng.uniform(*eps_vir, nv),
    ])
    ref = reference_from_ci(na, nel, rng=rng) if na > 0 else reference_from_ci(0, 0)
    n = nc + na + nv
    B = df_factor(rng, n, naux)
    inst = dict(nc=nc, na=na, nv=nv, naux=naux, s=float(s), eps=eps, B=B)
    for k in ("g1a", "g1b", "l2aa", "l2ab", "l2bb", "l3aaa", "l3aab", "l3abb", "l3bbb"):
        inst[k] = ref[k]
    if with_so:
        inst["g1_so"], inst["l2_so"], inst["l3_so"] = ref["g1_so"], ref["l2_so"], ref["l3_so"]
        inst["ci"], inst["dets"] = ref["ci"], ref["dets"]
    return inst


# large active spaces with synthetic references (make_synthetic_instance)
SYNTHETIC_CONFIGS = {
    "cas1616_c10_v100_q400": dict(nc=10, na=16, nv=100, naux=400, s=0.5, seed=SEED0 + 5),
}


def config_instance(name: str, **kw) -> dict:
    if name in SYNTHETIC_CONFIGS:
        c = dict(SYNTHETIC_CONFIGS[name])
        c.update(kw)
        return make_synthetic_instance(**c)
    c = dict(CONFIGS[name])
    c.update(kw)
    return make_instance(**c)


def config_seed(name: str) -> int:
    return (SYNTHETIC_CONFIGS.get(name) or CONFIGS[name])["seed"]


def scan_sizes(j: int, nscan: int = 32) -> dict:
    """Sizes of point j of the 32-point scan (drawn first, from their own
    seed): core uniform {4..12}, CAS(4,4) or CAS(6,6), virtual uniform
    {60..200}, aux 4 x virtual, virtual lower edge 0.6 -> 0.05 Eh."""
    rng = np.random.default_rng(SEED0 + 100 + j)
    nc = int(rng.integers(4, 13))
    cas = 4 if rng.random() < 0.5 else 6
    nv = int(rng.integers(60, 201))
    vlo = 0.6 - 0.55 * j / (nscan - 1)
    return {"nc": nc, "na": cas, "nv": nv, "naux": 4 * nv, "vlo": vlo}


def scan_instance(j: int, nscan: int = 32) -> dict:
    """Instance j of a 32-point dissociation-like scan: uneven sizes, the
    virtual band's lower edge falls linearly from 0.6 to 0.05 Eh."""
    z = scan_sizes(j, nscan)
    return make_instance(z["nc"], z["na"], z["na"], z["nv"], z["naux"], 0.5, seed=SEED0 + 1000 + j,
                         eps_vir=(z["vlo"], 5.0))


def random_small(nc, na, nel, nv, naux, s=0.5, seed=1):
    return make_instance(nc, na, nel, nv, naux, s, seed=seed)


# ----------------------------------------------------------------------------
# synthetic references for large active spaces
# ----------------------------------------------------------------------------

def _symmetrised_block(rng, na, rank, groups, scale):
    """Random block X[p1..pk, q1..qk] (each index over the na active orbitals
    of one spin), Hermitian (X[p.., q..] = X[q.., p..]) and antisymmetric
    under exchanges within each group of same-spin creator slots and the same
    groups of annihilator slots (`groups`: tuples of slot positions 0..k-1)."""
    from itertools import permutations as _perms
    X = rng.standard_normal((na,) * (2 * rank))
    X = X + np.transpose(X, list(range(rank, 2 * rank)) + list(range(rank)))
    for grp in groups:
        if len(grp) < 2:
            continue
        # antisymmetry: one group permutation on creators and one, independent, on annihilators
        acc = np.zeros_like(X)
        for pc in _perms(range(len(grp))):
            for pa in _perms(range(len(grp))):
                axes = list(range(2 * rank))
                for i, j in zip(grp, pc):
                    axes[i] = grp[j]
                for i, j in zip(grp, pa):
                    axes[rank + i] = rank + grp[j]
                acc += _perm_sign(pc) * _perm_sign(pa) * np.transpose(X, axes)
        X = acc
    return X * scale


def synthetic_reference(na: int, rng, l2_scale: float = 0.02, l3_scale: float = 0.002) -> dict:
    """Spin blocks of a synthetic active-space reference for active spaces too
    large for an exact CI (CAS(12,12) has 853776 Ms=0 determinants): gamma1
    per spin a random symmetric matrix with eigenvalues in [0, 1] (natural
    occupations); lambda2 and lambda3 blocks random with the symmetries of
    density cumulants (Hermitian, antisymmetric under exchanges of same-spin
    creators and of same-spin annihilators), small in magnitude.  They are
    not the cumulants of any one state; the energy expressions take them as
    given.  Blocks as spin_blocks returns them (alpha slots first)."""
    out = {}
    for k in ("g1a", "g1b"):
        U, _ = np.linalg.qr(rng.standard_normal((na, na)))
        occ = rng.uniform(0.0, 1.0, na)
        out[k] = (U * occ) @ U.T
    out["l2aa"] = _symmetrised_block(rng, na, 2, [(0, 1)], l2_scale)
    out["l2ab"] = _symmetrised_block(rng, na, 2, [], l2_scale)
    out["l2bb"] = _symmetrised_block(rng, na, 2, [(0, 1)], l2_scale)
    out["l3aaa"] = _symmetrised_block(rng, na, 3, [(0, 1, 2)], l3_scale)
    out["l3aab"] = _symmetrised_block(rng, na, 3, [(0, 1)], l3_scale)
    out["l3abb"] = _symmetrised_block(rng, na, 3, [(1, 2)], l3_scale)
    out["l3bbb"] = _symmetrised_block(rng, na, 3, [(0, 1, 2)], l3_scale)
    return {k: np.ascontiguousarray(v) for k, v in out.items()}


def make_synthetic_instance(nc: int, na: int, nv: int, naux: int, s: float = 0.5, seed: int = SEED0) -> dict:
    """A problem with the orbital-energy and B^Q recipe of make_instance and a
    synthetic reference (synthetic_reference) in place of the CI vector.
    Draw order: core, active, virtual energies, gamma1 / lambda2 / lambda3,
    then B row by row."""
    rng = np.random.default_rng(seed)
    eps = np.concatenate([rng.uniform(*EPS_CORE, nc), rng.uniform(*EPS_ACT, na), rng.uniform(*EPS_VIR, nv)])
    ref = synthetic_reference(na, rng)
    B = df_factor(rng, nc + na + nv, naux)
    inst = dict(nc=nc, na=na, nv=nv, naux=naux, s=float(s), eps=eps, B=B)
    for k in ("g1a", "g1b", "l2aa", "l2ab", "l2bb", "l3aaa", "l3aab", "l3abb", "l3bbb"):
        inst[k] = ref[k]
    return inst
