"""Shared test helpers: small multireference problems built in an explicit
Fock space, so that the reference's densities come from the state itself."""
import numpy as np

import synth
from oracle import fockspace as fsm


def product_dets_signs(dets_a, na_a, dets_b, na_b):
    """Fermionic product of two active-space states (alpha bits low in each).

    Subsystem a owns orbitals 0..na_a-1, b owns na_a..na_a+na_b-1 of the
    combined active space.  Returns (combined determinant bitstrings, signs)
    where sign reorders (a creators)(b creators) into ascending order."""
    na = na_a + na_b
    out, signs = [], []
    for da in dets_a:
        for db in dets_b:
            so = []
            for u in range(na_a):
                if da >> u & 1:
                    so.append(u)
            for u in range(na_a):
                if da >> (na_a + u) & 1:
                    so.append(na + u)
            for u in range(na_b):
                if db >> u & 1:
                    so.append(na_a + u)
            for u in range(na_b):
                if db >> (na_b + u) & 1:
                    so.append(na + na_a + u)
            d = 0
            for x in so:
                d |= 1 << x
            out.append(d)
            signs.append(synth._perm_sign(so))
    return out, np.array(signs, dtype=float)


def mr_fock_instance(nc, na, nel, nv, naux, s, seed, eps_ranges=((-0.8, -0.3), (-0.3, 0.3), (0.2, 0.9)),
                     bscale=1.0):
    """Instance whose reference is a random Ms=0 CAS state in an explicit
    Fock space ordered as the oracle's spin orbitals (sigma*n + p)."""
    rng = np.random.default_rng(seed)
    n = nc + na + nv
    eps = np.concatenate([rng.uniform(*eps_ranges[0], nc), rng.uniform(*eps_ranges[1], na),
                          rng.uniform(*eps_ranges[2], nv)])
    B = synth.df_factor(rng, n, naux, scale=bscale)
    nso = 2 * n
    sa = synth._strings(na, nel // 2)
    dets = []
    for a in sa:
        for b in sa:
            d = 0
            for m in range(nc):
                d |= 1 << m
                d |= 1 << (n + m)
            for u in range(na):
                if a >> u & 1:
                    d |= 1 << (nc + u)
                if b >> u & 1:
                    d |= 1 << (n + nc + u)
            dets.append(d)
    ci = rng.standard_normal(len(dets))
    ci /= np.linalg.norm(ci)
    fs = fsm.FockSpace(nso, 2 * nc + nel, kmax=3)
    psi = fs.state(dets, ci)
    act = np.concatenate([np.arange(nc, nc + na), np.arange(n + nc, n + nc + na)])
    g = fs.rdm(psi, 1)
    G2 = fs.rdm(psi, 2)
    G3 = fs.rdm(psi, 3)
    l2, l3 = synth.cumulants(g[np.ix_(act, act)], G2[np.ix_(*[act] * 4)], G3[np.ix_(*[act] * 6)])
    blk = synth.spin_blocks(na, g[np.ix_(act, act)], l2, l3)
    inst = dict(nc=nc, na=na, nv=nv, naux=naux, s=s, eps=eps, B=B, **blk)
    return inst, fs, psi, g, act, {2: l2, 3: l3}
