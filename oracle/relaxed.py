"""One-step relaxed DSRG-MRPT2 and DSRG-MRPT3 energies (Eq. E_relaxed, App. A).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The relaxed energy of order k is the lowest eigenvalue of the summed
transformed Hamiltonian Hbar^[k]_{1,2} = sum_{n <= k} Hbar^(n)_{1,2} within
the determinant space of the reference (Eq. energy_relaxed, used once with
Eq. E_relaxed).  Steps, in the paper's order:

1. Hbar^[k]_{1,2} as an operator (Eqs. Hbar_0th to Hbar_3rd), with
   Htilde^(1) and Htilde^(2) as in ``oracle.dsrg``:
     Hbar^(0) = H^(0),  Hbar^(1) = [H^(0), A^(1)] + H^(1),
     Hbar^(2) = [H^(0), A^(2)] + 1/2 [Htilde^(1), A^(1)],
     Hbar^(3) = [H^(0), A^(3)] + 1/2 [Htilde^(1), A^(2)] + 1/2 [Htilde^(2), A^(1)],
   each commutator truncated to one- and two-body terms.  E0 needs the bare
   integrals, which are not inputs, so every scalar is taken relative to it:
   the scalar of Hbar^[k] is E(2) (k = 2) or E(2) + E(3) (k = 3).  A^(3) is
   not formed: it has no all-active amplitudes and [H^(0), A] has the blocks
   of A, so [H^(0), A^(3)] has no all-active block, and only that block
   enters the relaxed energy (step 2).
2. App. A: with the core folded, only the all-active elements Hbar^u_v and
   Hbar^{uv}_{xy} enter.  In true-vacuum order (Eq. Hbar_DNO) the operator
   on the active space is
     E_s + sum_uv c^u_v a+_u a_v + 1/4 sum_uvxy w^{uv}_{xy} a+_u a+_v a_y a_x,
     E_s = Hbar_0 - sum_uv Hbar^u_v gamma^u_v
           - sum_uvxy Hbar^{uv}_{xy} (1/4 gamma^{uv}_{xy} - gamma^u_x gamma^v_y),
     c^u_v = Hbar^u_v - sum_xy Hbar^{ux}_{vy} gamma^x_y,   w = Hbar^{uv}_{xy},
   with gamma^{uv}_{xy} = <a+_u a+_v a_y a_x> of the reference (the core
   terms of Eq. Hbar_DNO cancel against Eq. c0_cas).
3. The matrix of that operator over the determinants with the reference's
   numbers of alpha and beta active electrons (alpha orbitals on the low
   bits, determinants ordered alpha string first, strings ascending), built
   by applying the creation and annihilation strings to each determinant.
4. Its lowest eigenvalue.

Active spin orbitals are numbered alpha 0..na-1, then beta na..2na-1.
"""
from __future__ import annotations

from itertools import combinations

import numpy as np

from . import dsrg
from .mkgno import Op, commutator


def hbar_operator(inst: dict, order: int = 3):
    """Hbar^[order]_{1,2} relative to E0 on all spin orbitals, and the
    problem (``oracle.dsrg.SpinOrbitalProblem``) it lives on."""
    if order not in (2, 3):
        raise ValueError("order is 2 or 3")
    r = dsrg.dsrg_pt3(inst, return_intermediates=True)
    P, I = r["_problem"], r["_inter"]
    n, ref = P.nso, P.ref
    H0 = Op(n, 0.0, {1: np.diag(P.eps)})           # H^(0) - E0
    H1 = Op(n, 0.0, {1: P.f1, 2: P.V})
    T = Op(n, 0.0, {1: I["T1"], 2: I["T2"]})
    A = T - T.adjoint()
    Tb = Op(n, 0.0, {1: I["T1b"], 2: I["T2b"]})
    Ab = Tb - Tb.adjoint()
    W = I["W"]                                       # [H^(0), A^(1)]
    Ht1 = H1.scale(2.0) + W                          # Htilde^(1)
    O = I["O"].truncate(2)                           # 1/2 [Htilde^(1), A^(1)]_{1,2}, scalar E(2)
    hb = H0 + H1 + W + commutator(H0, Ab, ref) + O
    if order == 3:
        Ht2 = I["Ht2"]                               # Htilde^(2)_{1,2}
        hb = hb + commutator(Ht1, Ab, ref, out_max=2).scale(0.5) \
                + commutator(Ht2, A, ref, out_max=2).scale(0.5)
    return hb.truncate(2), P, r


def active_blocks(hb: Op, P):
    """(Hbar_0, Hbar^u_v [2na,2na], Hbar^{uv}_{xy} [2na]^4)."""
    a = P.act
    z1 = hb.z.get(1)
    z2 = hb.z.get(2)
    h1 = z1[np.ix_(a, a)].copy() if z1 is not None else np.zeros((a.size, a.size))
    h2 = z2[np.ix_(a, a, a, a)].copy() if z2 is not None else np.zeros((a.size,) * 4)
    return float(hb.c0), h1, h2


def two_rdm(g1: np.ndarray, l2: np.ndarray) -> np.ndarray:
    """gamma^{uv}_{xy} = <a+_u a+_v a_y a_x> = lambda^{uv}_{xy} + g^u_x g^v_y - g^u_y g^v_x."""
    return l2 + np.einsum("ux,vy->uvxy", g1, g1) - np.einsum("uy,vx->uvxy", g1, g1)


def dno_active(h0: float, h1: np.ndarray, h2: np.ndarray, g1: np.ndarray, g2: np.ndarray):
    """App. A: (E_s, c, w) of the active-space operator in true-vacuum order."""
    Es = (h0 - np.einsum("uv,uv->", h1, g1)
          - np.einsum("uvxy,uvxy->", h2, 0.25 * g2 - np.einsum("ux,vy->uvxy", g1, g1)))
    c = h1 - np.einsum("uxvy,xy->uv", h2, g1)
    return float(Es), c, h2.copy()


def determinants(na: int, nalpha: int, nbeta: int) -> list[int]:
    """2na-bit occupation strings, alpha bits low, alpha string major."""
    def strings(k):
        out = []
        for occ in combinations(range(na), k):
            b = 0
            for o in occ:
                b |= 1 << o
            out.append(b)
        return sorted(out)
    return [a | (b << na) for a in strings(nalpha) for b in strings(nbeta)]


def _apply(det: int, ops):
    """Apply a string of elementary operators (rightmost first) to a
    determinant; returns (sign, new determinant) or (0, None)."""
    sign = 1
    for kind, x in reversed(ops):
        occ = (det >> x) & 1
        if kind == "a":
            if not occ:
                return 0, None
        elif occ:
            return 0, None
        if bin(det & ((1 << x) - 1)).count("1") % 2:
            sign = -sign
        det ^= 1 << x
    return sign, det


def ci_matrix(Es: float, c: np.ndarray, w: np.ndarray, dets: list[int]) -> np.ndarray:
    """<D_I| Es + sum c a+_u a_v + 1/4 sum w a+_u a+_v a_y a_x |D_J>."""
    m = c.shape[0]
    index = {d: k for k, d in enumerate(dets)}
    H = np.zeros((len(dets), len(dets)))
    H[np.diag_indices(len(dets))] = Es
    for J, d in enumerate(dets):
        for u in range(m):
            for v in range(m):
                if c[u, v] == 0.0:
                    continue
                sg, e = _apply(d, [("c", u), ("a", v)])
                if sg and e in index:
                    H[index[e], J] += sg * c[u, v]
        # 1/4 sum over all ordered quadruples = sum over u < v, x < y
        for u, v in combinations(range(m), 2):
            for x, y in combinations(range(m), 2):
                val = w[u, v, x, y]
                if val == 0.0:
                    continue
                sg, e = _apply(d, [("c", u), ("c", v), ("a", y), ("a", x)])
                if sg and e in index:
                    H[index[e], J] += sg * val
    return H


def relaxed_energies(inst: dict, nalpha: int, nbeta: int, orders=(2, 3)) -> dict:
    """Unrelaxed E(2), E(3) and the one-step relaxed energies of the given
    orders (all relative to E0), with the intermediate pieces."""
    out = {}
    na = int(inst["na"])
    for k in orders:
        hb, P, r = hbar_operator(inst, order=k)
        h0, h1, h2 = active_blocks(hb, P)
        a = P.act
        g1 = P.gamma[np.ix_(a, a)]
        l2 = P.ref.lam[2] if na > 0 else np.zeros((0,) * 4)
        g2 = two_rdm(g1, l2)
        Es, c, w = dno_active(h0, h1, h2, g1, g2)
        dets = determinants(na, nalpha, nbeta)
        H = ci_matrix(Es, c, w, dets)
        out[f"e_relaxed{k}"] = float(np.linalg.eigvalsh(H)[0]) if len(dets) else float("nan")
        out[f"unrelaxed{k}"] = h0
        out[f"_pieces{k}"] = dict(h0=h0, h1=h1, h2=h2, Es=Es, c=c, w=w, H=H, dets=dets)
        out.update(e2=r["e2"], e3a=r["e3a"], e3b=r["e3b"], e3=r["e3"])
    return out
