"""First-order aavv amplitudes with Dyall's zeroth-order Hamiltonian (App. B).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

With H(0) = E0 + F(0) + 1/4 sum_uvxy v(0)^{uv}_{xy} {a+_u a+_v a_y a_x} (the
Fock diagonal plus the all-active part of V), the first-order amplitudes
that promote two active electrons into the virtuals satisfy, at s -> infinity
(Eq. t2_aavv), for virtual e, f and active u, v:

  0 = V[e,f,u,v] - D[e,f,u,v] t[e,f,u,v] - 1/2 sum_xy Va[x,y,u,v] t[e,f,x,y]
                                         + sum_xyz Va[x,y,u,v] t[e,f,x,z] gamma[y,z]

with D[e,f,u,v] = eps_u + eps_v - eps_e - eps_f, Va the all-active block of
V, gamma the active 1-RDM (spin orbitals; X2[p,q,r,s] multiplies
{a+_p a+_q a_s a_r}).  The block is closed: for every virtual pair (e, f)
the amplitudes t[e,f,:,:] solve one linear system on the active pairs, the
same matrix shifted by eps_e + eps_f.

The shifted denominator is taken as the exact diagonal of that system (the
coefficient of t[e,f,u,v] in the residual, up to sign):

  Ds[e,f,u,v] = D[e,f,u,v] + Va[u,v,u,v]
                - sum_y (Va[u,y,u,v] gamma[y,v] - Va[v,y,u,v] gamma[y,u]),

which in natural orbitals is D + v^{uv}_{uv} (1 - n_u - n_v).  (The paper's
Eq. full_preconditioner and Eq. no_preconditioner differ from each other in
the sign of the two-body term and from the amplitude equation by a factor of
two; the diagonal of Eq. t2_aavv decides here.)
"""
from __future__ import annotations

import numpy as np

from .dsrg import SpinOrbitalProblem


def blocks(inst: dict):
    """Spin-orbital V[vir,vir,act,act], Va[act]^4, gamma[act,act], D and the
    orbital energies of a problem."""
    P = SpinOrbitalProblem(inst)
    act = np.where(P.actm)[0]
    vir = np.where(P.vir)[0]
    e = P.eps
    Vs = P.V[np.ix_(vir, vir, act, act)].copy()
    Va = P.V[np.ix_(act, act, act, act)].copy()
    g = P.gamma[np.ix_(act, act)].copy()
    D = (e[act][None, None, :, None] + e[act][None, None, None, :]
         - e[vir][:, None, None, None] - e[vir][None, :, None, None])
    return Vs, Va, g, D


def coupling(t, Va, g):
    """-1/2 sum_xy Va[x,y,u,v] t[e,f,x,y] + sum_xyz Va[x,y,u,v] t[e,f,x,z] gamma[y,z]."""
    return (-0.5 * np.einsum("xyuv,efxy->efuv", Va, t, optimize=True)
            + np.einsum("xyuv,efxz,yz->efuv", Va, t, g, optimize=True))


def residual(t, Vs, Va, g, D):
    """Eq. t2_aavv: V - D t + coupling(t)."""
    return Vs - D * t + coupling(t, Va, g)


def shifted_denominators(Va, g, D):
    """The exact diagonal Ds (see the module docstring)."""
    m = Va.shape[0]
    i = np.arange(m)
    diag = Va[i[:, None], i[None, :], i[:, None], i[None, :]]           # Va[u,v,u,v]
    diag = diag - np.einsum("uyuv,yv->uv", Va, g) + np.einsum("vyuv,yu->uv", Va, g)
    return D + diag[None, None]


def solve(Vs, Va, g, D):
    """Direct solution of Eq. t2_aavv for every virtual pair (numpy solve on
    the active pairs; the u = v components are zero by antisymmetry)."""
    nv, _, m, _ = Vs.shape
    # residual = Vs - t G with t a row vector over (x, y) and G the same for
    # every pair but for the shift eps_e + eps_f carried by D
    G0 = np.zeros((m * m, m * m))
    for k in range(m * m):
        unit = np.zeros((1, 1, m, m))
        unit.reshape(-1)[k] = 1.0
        G0[k] = -coupling(unit, Va, g).reshape(-1)
    t = np.zeros_like(Vs)
    off = ~np.eye(m, dtype=bool).reshape(-1)
    for a in range(nv):
        for b in range(nv):
            G = G0 + np.diag(D[a, b].reshape(-1))
            sub = G[np.ix_(off, off)]
            x = np.linalg.solve(sub.T, Vs[a, b].reshape(-1)[off])
            row = np.zeros(m * m)
            row[off] = x
            t[a, b] = row.reshape(m, m)
    return t
