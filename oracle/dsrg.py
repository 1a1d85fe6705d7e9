"""DSRG-MRPT2 / MRPT3 unrelaxed energies, plain FP64 on dense spin orbitals.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Follows Sec. II.B of the paper step by step:

* H^(0) = E0 + sum_p eps_p {a+_p a_p}  (Eq. F0th, semicanonical orbitals)
* H^(1) = off-diagonal Fock + the full two-electron operator V, with the
  integrals from the factorisation (pq|rs) = sum_Q B^Q_pq B^Q_rs
  (Eq. int_fact)
* first-order amplitudes, Eqs. T1_1st and T2_1st, regulariser
  (1 - exp(-s D^2)) / D, internal (all-active) amplitudes zero
* Htilde^(1) = H^(1) + Hbar^(1) = 2 H^(1) + [H^(0), A^(1)]  (Eq. Hbar_1st)
* E^(2) = <[Htilde^(1), T^(1)]>  (Eq. E(2))
* second-order amplitudes from the non-diagonal one- and two-body parts of
  1/2 [Htilde^(1), A^(1)], Eqs. T1_2nd and T2_2nd
* Htilde^(2)_{1,2} = [H^(0), A^(2)] + 1/2 [Htilde^(1), A^(1)]_{1,2}
  - 1/6 [[H^(0), A^(1)], A^(1)]_{1,2}  (Eq. Hbar_2nd and the definition of
  Htilde^(2), truncated to one- and two-body terms as in Eq. E(3)'s
  approximation)
* E^(3) = <[Htilde^(1), T^(2)]> + <[Htilde^(2)_{1,2}, T^(1)]>  (Eq. E(3))

Spin orbitals are ordered (all alpha, then all beta); orbital p of spin
sigma has index sigma * n + p.
"""
from __future__ import annotations

import itertools

import numpy as np

from .mkgno import Op, Reference, commutator, parity


# ----------------------------------------------------------------------------
# regulariser (Eqs. T1_1st, T2_1st)
# ----------------------------------------------------------------------------

def regulariser(s: float, D: np.ndarray) -> np.ndarray:
    """(1 - exp(-s D^2)) / D with its limit 0 at D = 0.

    Evaluated as -expm1(-s D^2) / D; below s D^2 = 1e-12 the two-term series
    s D (1 - s D^2 / 2) is used, which is exact to rounding there.
    """
    D = np.asarray(D, dtype=np.float64)
    x = s * D * D
    small = x < 1e-12
    safe = np.where(small, 1.0, D)
    out = -np.expm1(-x) / safe
    return np.where(small, s * D * (1.0 - 0.5 * x), out)


# ----------------------------------------------------------------------------
# spin-orbital problem
# ----------------------------------------------------------------------------

def _spin_tensor(blocks: dict, na: int, rank: int) -> np.ndarray:
    """Full spin-orbital active cumulant from its spin blocks.

    ``blocks[m]`` holds the block whose first ``rank-m`` creators and
    annihilators are alpha and the last ``m`` beta.  Other spin orderings
    follow from antisymmetry under creator and annihilator permutations.
    """
    out = np.zeros((2 * na,) * (2 * rank))
    for sc in itertools.product((0, 1), repeat=rank):
        for sa in itertools.product((0, 1), repeat=rank):
            if sum(sc) != sum(sa):
                continue
            pc = sorted(range(rank), key=lambda i: (sc[i], i))
            pa = sorted(range(rank), key=lambda i: (sa[i], i))
            sign = parity(pc) * parity(pa)
            blk = blocks[sum(sc)]
            # blk axis j is creator pc[j]; move it to axis pc[j]
            axes = [0] * (2 * rank)
            for j in range(rank):
                axes[pc[j]] = j
                axes[rank + pa[j]] = rank + j
            view = tuple(slice(s * na, (s + 1) * na) for s in sc) + \
                tuple(slice(s * na, (s + 1) * na) for s in sa)
            out[view] = sign * np.transpose(blk, axes)
    return out


class SpinOrbitalProblem:
    def __init__(self, inst: dict, eri=None):
        nc, na, nv = inst["nc"], inst["na"], inst["nv"]
        n = nc + na + nv
        self.nc, self.na, self.nv, self.n = nc, na, nv, n
        self.s = float(inst["s"])
        nso = 2 * n
        self.nso = nso
        eps = np.asarray(inst["eps"], dtype=np.float64)
        self.eps = np.concatenate([eps, eps])
        # (pr|qs) stored at J[p,q,r,s]  (Eq. int_fact)
        if eri is None:
            B = np.asarray(inst["B"], dtype=np.float64)
            J = np.einsum("Qpr,Qqs->pqrs", B, B, optimize=True)
        else:
            J = np.transpose(np.asarray(eri, dtype=np.float64), (0, 2, 1, 3))  # (pr|qs) from (pq|rs)
        V = np.zeros((nso,) * 4)
        sp = [slice(0, n), slice(n, 2 * n)]
        for a in range(2):
            for b in range(2):
                V[sp[a], sp[b], sp[a], sp[b]] += J
                V[sp[a], sp[b], sp[b], sp[a]] -= np.transpose(J, (0, 1, 3, 2))
        self.V = V
        f1 = inst.get("f1")
        F = np.zeros((nso, nso))
        if f1 is not None:
            f1 = np.array(f1, dtype=np.float64)
            blocks = [range(0, nc), range(nc, nc + na), range(nc + na, n)]
            for blk in blocks:
                idx = np.array(list(blk), dtype=int)
                if idx.size:
                    f1[np.ix_(idx, idx)] = 0.0
            F[:n, :n] = f1
            F[n:, n:] = f1
        self.f1 = F
        # index classes
        core = np.zeros(nso, bool)
        act = np.zeros(nso, bool)
        vir = np.zeros(nso, bool)
        for s in range(2):
            core[s * n: s * n + nc] = True
            act[s * n + nc: s * n + nc + na] = True
            vir[s * n + nc + na: (s + 1) * n] = True
        self.core, self.actm, self.vir = core, act, vir
        self.hole = core | act
        self.part = act | vir
        self.act = np.concatenate([np.arange(nc, nc + na), np.arange(n + nc, n + nc + na)])
        # reference quantities (Sec. II.A: gamma, eta and cumulants)
        g = np.zeros((nso, nso))
        g[core, core] = 0.0
        for s in range(2):
            for m in range(nc):
                g[s * n + m, s * n + m] = 1.0
        ga = np.asarray(inst["g1a"]).reshape(na, na)
        gb = np.asarray(inst["g1b"]).reshape(na, na)
        g[nc:nc + na, nc:nc + na] = ga
        g[n + nc:n + nc + na, n + nc:n + nc + na] = gb
        self.gamma = g
        self.eta = np.eye(nso) - g
        lam = {}
        if na > 0:
            sh2 = (na,) * 4
            sh3 = (na,) * 6
            lam[2] = _spin_tensor({0: np.reshape(inst["l2aa"], sh2), 1: np.reshape(inst["l2ab"], sh2),
                                   2: np.reshape(inst["l2bb"], sh2)}, na, 2)
            lam[3] = _spin_tensor({0: np.reshape(inst["l3aaa"], sh3), 1: np.reshape(inst["l3aab"], sh3),
                                   2: np.reshape(inst["l3abb"], sh3), 3: np.reshape(inst["l3bbb"], sh3)}, na, 3)
        else:
            lam[2] = np.zeros((0,) * 4)
            lam[3] = np.zeros((0,) * 6)
        self.ref = Reference(gamma=self.gamma, eta=self.eta, act=self.act, lam=lam)
        # excitation masks (internal amplitudes are zero, Sec. II.A)
        P, H, A = self.part, self.hole, self.actm
        self.mask1 = P[:, None] & H[None, :] & ~(A[:, None] & A[None, :])
        m2 = P[:, None, None, None] & P[None, :, None, None] & H[None, None, :, None] & H[None, None, None, :]
        allact = A[:, None, None, None] & A[None, :, None, None] & A[None, None, :, None] & A[None, None, None, :]
        self.mask2 = m2 & ~allact
        e = self.eps
        self.D1 = e[None, :] - e[:, None]                            # D^i_a at [a,i]
        self.D2 = (e[None, None, :, None] + e[None, None, None, :]
                   - e[:, None, None, None] - e[None, :, None, None])  # D^{ij}_{ab} at [a,b,i,j]

    # Eqs. T1_1st / T1_2nd: t^i_a = [f^i_a + sum_ux D^u_x t^{iu}_{ax} gamma^x_u] R(D^i_a).
    # The paper's denominators put particle-type labels first:
    # D^{ab..}_{ij..} = eps_i + eps_j + .. - eps_a - eps_b - .., so D^u_x = eps_x - eps_u.
    def amplitudes(self, f1_like, v_like):
        s = self.s
        T2 = np.where(self.mask2, v_like * regulariser(s, self.D2), 0.0)
        a = self.act
        e = self.eps
        Dux = e[a][None, :] - e[a][:, None]             # D^u_x = eps_x - eps_u at [u, x]
        g = self.gamma[np.ix_(a, a)]                    # gamma[x, u]
        T2ax = T2[:, :, :, a][:, a, :, :]               # T2[a, x, i, u] with x,u active
        src = np.einsum("axiu,ux,xu->ai", T2ax, Dux, g, optimize=True) if a.size else 0.0
        T1 = np.where(self.mask1, (f1_like + src) * regulariser(s, self.D1), 0.0)
        return T1, T2


def _excitation(T1, T2, n):
    return Op(n, 0.0, {1: T1, 2: T2})


def dsrg_pt3(inst: dict, pt2_only: bool = False, eri=None, return_intermediates=False) -> dict:
    """E(2), E(3)a, E(3)b and E(3) of Eqs. E(2)/E(3)."""
    P = SpinOrbitalProblem(inst, eri=eri)
    n, ref = P.nso, P.ref
    H0 = Op(n, 0.0, {1: np.diag(P.eps)})
    H1 = Op(n, 0.0, {1: P.f1, 2: P.V})
    T1, T2 = P.amplitudes(P.f1, P.V)
    T = _excitation(T1, T2, n)
    A = T - T.adjoint()
    W = commutator(H0, A, ref)                 # [H^(0), A^(1)]
    Ht1 = H1.scale(2.0) + W                    # Htilde^(1)
    E2 = commutator(Ht1, T, ref, out_max=0).c0
    out = {"e2": E2}
    inter = {"T1": T1, "T2": T2, "W": W}
    if not pt2_only:
        O = commutator(Ht1, A, ref, out_max=2).scale(0.5)   # 1/2 [Htilde^(1), A^(1)]_{1,2}
        U1, U2 = P.amplitudes(O.z[1], O.z[2])                # second-order amplitudes
        Tb = _excitation(U1, U2, n)
        Ab = Tb - Tb.adjoint()
        Ht2 = commutator(H0, Ab, ref) + O.truncate(2) - commutator(W, A, ref, out_max=2).scale(1.0 / 6.0)
        E3a = commutator(Ht1, Tb, ref, out_max=0).c0
        E3b = commutator(Ht2, T, ref, out_max=0).c0
        out.update(e3a=E3a, e3b=E3b, e3=E3a + E3b)
        inter.update(O=O, T1b=U1, T2b=U2, Ht2=Ht2)
    if return_intermediates:
        out["_inter"] = inter
        out["_problem"] = P
    return out


def df_ladder(B: np.ndarray, t: np.ndarray, p0: int) -> np.ndarray:
    """Spatial particle-particle ladder of Eq. scaling_problem with the
    integrals of Eq. int_fact: L[p,q,i,j] = sum_rs (p r|q s) t[r,s,i,j],
    (p r|q s) = sum_Q B[Q,p0+p,p0+r] B[Q,p0+q,p0+s]."""
    npart = t.shape[0]
    Bp = B[:, p0:p0 + npart, p0:p0 + npart]
    J = np.einsum("Qpr,Qqs->pqrs", Bp, Bp)
    return np.einsum("pqrs,rsij->pqij", J, t)
