"""Block-restricted, density-fitted DSRG-MRPT2/PT3 energies (plain FP64 numpy).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The same steps as ``oracle.dsrg``, in the paper's order (Sec. II.B: Eqs.
T2_1st, T1_1st, Hbar_1st, E(2), T1_2nd, T2_2nd, Hbar_2nd, E(3)), but sized
for workloads whose dense spin-orbital tensors do not fit in memory:

* Every operator is kept only on the orbital blocks where it can be
  non-zero: amplitudes and the excitation part of W on [P,P,H,H] and [P,H]
  (P = active + virtual, H = core + active, internal all-active elements
  zero), the two-electron operator built from B^Q_pq on the blocks a term
  asks for (Eq. int_fact), never as a full four-index array.
* Each commutator is the sum of the generalized Wick contraction patterns of
  ``oracle.mkgno`` (the enumeration pinned against explicit Fock-space
  commutators), each evaluated on the index ranges its contractions allow:
  a gamma contraction (creator of the left operator with an annihilator of
  the right one) runs over H, an eta contraction over P, a cumulant leg over
  the active orbitals, and an open leg over the output block requested.
  gamma is the identity on core and zero outside H, eta the identity on
  virtual and zero outside P, so nothing is dropped.
* Only the output blocks the energy needs are formed: the scalar part for
  E(2) and E(3), and the excitation blocks [P,H], [P,P,H,H] of
  1/2 [Htilde(1), A(1)] and of [W, A(1)] (their de-excitation blocks follow
  by hermiticity and are the only ones <[X, T]> reads besides them).
* The one contraction that needs the all-particle block of V, the
  particle-particle ladder (Eq. scaling_problem), builds <pq||rs> from B a
  slab of rows p at a time and uses each slab at once.
* W = [H(0), A(1)] in closed form: W2 = -D^{ij}_{ab} T2, W1 = -D^i_a T1 +
  sum_{ux} (eps_x - eps_u) T2[a,x,i,u] gamma[x,u] (Eqs. T1_1st, T2_1st with
  the commutator of a diagonal H(0)), excitation block plus its transpose.

Spin orbitals are ordered as in ``oracle.dsrg`` (orbital p of spin sigma at
sigma * n + p); spin blocks that vanish are carried as zeros (the alpha/beta
structure is not exploited beyond that).
"""
from __future__ import annotations

import math

import numpy as np

from . import mkgno
from .dsrg import _spin_tensor, regulariser


# ----------------------------------------------------------------------------
# orbital spaces (spin-orbital index arrays)
# ----------------------------------------------------------------------------

class Spaces:
    def __init__(self, nc, na, nv):
        n = nc + na + nv
        self.n, self.nso = n, 2 * n

        def so(lo, hi):
            return np.concatenate([np.arange(lo, hi), np.arange(n + lo, n + hi)]).astype(np.int64)

        self.r = {"C": so(0, nc), "A": so(nc, nc + na), "V": so(nc + na, n), "H": so(0, nc + na),
                  "P": so(nc, n), "G": so(0, n)}
        # position of every spin orbital inside each space (-1 outside)
        self.pos = {}
        for k, idx in self.r.items():
            p = -np.ones(self.nso, dtype=np.int64)
            p[idx] = np.arange(idx.size)
            self.pos[k] = p

    def __getitem__(self, k):
        return self.r[k]


def _embed(X, slots, req, sp: Spaces):
    """X stored over spaces `slots`, returned over spaces `req` (zero where a
    requested orbital lies outside the stored space)."""
    sel_out, sel_in = [], []
    for s, r in zip(slots, req):
        p = sp.pos[s][sp[r]]
        m = p >= 0
        sel_out.append(np.nonzero(m)[0])
        sel_in.append(p[m])
    out = np.zeros([sp[r].size for r in req])
    if all(a.size for a in sel_out):
        out[np.ix_(*sel_out)] = X[np.ix_(*sel_in)]
    return out


# ----------------------------------------------------------------------------
# operator pieces
# ----------------------------------------------------------------------------

class Stored:
    """A tensor stored on given spaces, optionally with its Hermitian image
    (creator and annihilator slots exchanged) added."""

    def __init__(self, X, slots, herm=False):
        self.X, self.slots, self.herm = X, tuple(slots), herm
        self.cache = {}

    def block(self, req, sp):
        req = tuple(req)
        if req == self.slots and not self.herm:
            return self.X
        if req in self.cache:
            return self.cache[req]
        out = _embed(self.X, self.slots, req, sp)
        if self.herm:
            k = len(self.slots) // 2
            Xt = np.transpose(self.X, list(range(k, 2 * k)) + list(range(k)))
            out += _embed(Xt, self.slots[k:] + self.slots[:k], req, sp)
        if out.nbytes <= CACHE_BYTES:
            self.cache[req] = out
        return out


class DFTwoBody:
    """<pq||rs> = (pr|qs) d(s_p s_r) d(s_q s_s) - (ps|qr) d(s_p s_s) d(s_q s_r)
    with (pr|qs) = sum_Q B^Q_pr B^Q_qs (Eq. int_fact), built on the blocks a
    term asks for.  The all-particle block [P,P,P,P] is returned as a lazy
    marker: it is only contracted slab by slab (``_lazy_contract``)."""

    def __init__(self, B, sp: Spaces):
        self.B, self.sp = B, sp
        self.cache = {}

    def rows(self, idx0, r1, r2, r3):
        """Explicit <pq||rs> for spin orbitals idx0 (array) x spaces r1, r2, r3,
        assembled spin block by spin block from spatial integrals."""
        sp, n, B = self.sp, self.sp.n, self.B
        I = [idx0, sp[r1], sp[r2], sp[r3]]
        pos = [[np.nonzero(i // n == s_)[0] for s_ in (0, 1)] for i in I]   # positions of each spin
        X = [i % n for i in I]                                            # spatial orbitals
        out = np.zeros([i.size for i in I])

        def spatial(a, b, c, d, sa, sb, sc, sd):
            # (ac|bd) over the spatial orbitals of slots a, b, c, d restricted to spins sa..sd
            return np.einsum("Qac,Qbd->abcd", B[:, X[a][pos[a][sa]]][:, :, X[c][pos[c][sc]]],
                             B[:, X[b][pos[b][sb]]][:, :, X[d][pos[d][sd]]], optimize=True)

        for s0 in (0, 1):
            for s1 in (0, 1):
                # (pr|qs): spin of r = spin of p, spin of s = spin of q
                ix = np.ix_(pos[0][s0], pos[1][s1], pos[2][s0], pos[3][s1])
                out[ix] += spatial(0, 1, 2, 3, s0, s1, s0, s1)
                # -(ps|qr): spin of s = spin of p, spin of r = spin of q
                ix = np.ix_(pos[0][s0], pos[1][s1], pos[2][s1], pos[3][s0])
                out[ix] -= np.transpose(spatial(0, 1, 3, 2, s0, s1, s0, s1), (0, 1, 3, 2))
        return out

    def block(self, req, sp):
        req = tuple(req)
        if req == ("P", "P", "P", "P"):
            return LAZY_V
        if req in self.cache:
            return self.cache[req]
        out = self.rows(sp[req[0]], *req[1:])
        if out.nbytes <= CACHE_BYTES:
            self.cache[req] = out
        return out


# blocks up to this size are kept for reuse; larger ones are rebuilt on request
CACHE_BYTES = 256 << 20

LAZY_V = object()


class BOp:
    """c0 + sum_k Z_k with Z_k a sum of weighted pieces (Stored / DFTwoBody)."""

    def __init__(self, c0=0.0, parts=None):
        self.c0 = c0
        self.parts = parts or {}

    def __add__(self, o):
        parts = {k: list(v) for k, v in self.parts.items()}
        for k, v in o.parts.items():
            parts.setdefault(k, []).extend(v)
        return BOp(self.c0 + o.c0, parts)

    def scale(self, a):
        return BOp(a * self.c0, {k: [(a * c, p) for c, p in v] for k, v in self.parts.items()})

    def block(self, k, req, sp):
        """(explicit sum or None, [(coef, lazy piece)])"""
        out, lazy = None, []
        for c, p in self.parts.get(k, []):
            b = p.block(req, sp)
            if b is LAZY_V:
                lazy.append((c, p))
                continue
            out = c * b if out is None else out + c * b
        return out, lazy


# ----------------------------------------------------------------------------
# commutator on blocks
# ----------------------------------------------------------------------------

_RANGE_G, _RANGE_E, _RANGE_L = "H", "P", "A"


class Ref:
    def __init__(self, gamma_HH, eta_PP, lam):
        self.gamma, self.eta, self.lam = gamma_HH, eta_PP, lam


def _ladder_slab(piece, rows, V_sub, M, m_letters, out_sub):
    """sum over V's contracted letters of <pq||rs> M for the spin-orbital
    rows p of V's first slot, <pq||rs> built from B for those rows."""
    Vs = piece.rows(rows, "P", "P", "P")
    return np.einsum(V_sub + "," + m_letters + "->" + out_sub, Vs, M, optimize="greedy")


def _lazy_contract(piece, coef, V_sub, others, out_sub, dims, sp, slab=8):
    """sum over V's contracted letters of <pq||rs> M, with M the product of
    every other operand, <pq||rs> on [P,P,P,P] built a slab of rows p at a
    time (the first V letter must be an output letter)."""
    subs, ops = zip(*others)
    o0 = V_sub[0]
    if o0 not in out_sub:
        raise NotImplementedError("lazy two-body block: first slot must be open")
    m_letters = "".join(c for c in V_sub if any(c in s for s in subs)) + \
        "".join(c for c in out_sub if c not in V_sub)
    M = np.einsum(",".join(subs) + "->" + m_letters, *ops, optimize="greedy")
    K = np.zeros([dims[c] for c in out_sub])
    ax = out_sub.index(o0)
    P = sp["P"]
    for lo in range(0, P.size, slab):
        rows = P[lo:lo + slab]
        idx = [slice(None)] * K.ndim
        idx[ax] = slice(lo, lo + rows.size)
        K[tuple(idx)] += coef * _ladder_slab(piece, rows, V_sub, M, m_letters, out_sub)
    return K


class LadderSample:
    """The oracle's particle-particle ladder of 1/2 [Htilde(1), A(1)]
    (Eq. scaling_problem), out[p,q,i,j] = sum_{r,s in P} <pq||rs> M[r,s,i,j]
    with M = eta eta T2(1), evaluated a few spin-orbital rows p at a time by
    the same slab routine the energy uses.  Construction forms the
    first-order amplitudes and M; ``rows(lo, hi)`` evaluates rows [lo, hi) of
    the particle space.  Used to time the oracle on a bounded part of a
    workload too large for a whole energy on the host."""

    def __init__(self, inst: dict):
        Pb = BlockProblem(inst)
        self.sp, self.V = Pb.sp, Pb.V
        T1, T2, _ = Pb.amplitudes(Pb.F1[np.ix_(Pb.sp["P"], Pb.sp["H"])], Pb.V.block(EXC2, Pb.sp))
        del T1
        eta = Pb.ref.eta
        self.M = np.einsum("ce,df,efij->cdij", eta, eta, T2, optimize="greedy")
        self.nrows = Pb.sp["P"].size

    def rows(self, lo, hi):
        return _ladder_slab(self.V, self.sp["P"][lo:hi], "abcd", self.M, "cdij", "abij")


def _product_blocks(L: BOp, kL, R: BOp, kR, ref: Ref, want, sp: Spaces):
    """sum over pattern-containing contractions of {L_kL}{R_kR} on the wanted
    output blocks; want: {rank: [ranges, ...]} (rank 0: [()])."""
    out = {}
    ranks = sorted(want)
    patterns = mkgno.enumerate_patterns(kL, kR, lam_max=3, out_max=max(ranks))
    pref0 = 1.0 / (math.factorial(kL) ** 2 * math.factorial(kR) ** 2)
    for groups, mult in patterns:
        assigned, open_legs = mkgno._representative(groups, kL, kR)
        r = len(open_legs) // 2
        if r not in want:
            continue
        letter = {}
        li = iter(mkgno._LETTERS)
        for legs in assigned:
            for l in legs:
                letter[l] = next(li)
        for l in open_legs:
            letter[l] = next(li)
        target = []
        rng = {}
        for g, legs in zip(groups, assigned):
            cre, ann = mkgno._canonical(legs, kL, kR)
            target += (ann + cre) if g == mkgno._GROUP_PAIR_E else (cre + ann)
            R_ = _RANGE_G if g == mkgno._GROUP_PAIR_G else _RANGE_E if g == mkgno._GROUP_PAIR_E else _RANGE_L
            for l in legs:
                rng[l] = R_
        ocre, oann = mkgno._canonical(open_legs, kL, kR)
        target += ocre + oann
        sign = mkgno.parity([mkgno._position(*l, kL, kR) for l in target])
        out_legs = list(ocre) + list(reversed(oann))
        out_sub = "".join(letter[l] for l in out_legs)
        for blk in want[r]:
            for l, R_ in zip(out_legs, blk):
                rng[l] = R_
            dims = {letter[l]: sp[rng[l]].size for l in letter}
            others = []
            for g, legs in zip(groups, assigned):
                cre, ann = mkgno._canonical(legs, kL, kR)
                if g == mkgno._GROUP_PAIR_G:
                    others.append((letter[cre[0]] + letter[ann[0]], ref.gamma))
                elif g == mkgno._GROUP_PAIR_E:
                    others.append((letter[ann[0]] + letter[cre[0]], ref.eta))
                else:
                    others.append(("".join(letter[l] for l in cre) + "".join(letter[l] for l in reversed(ann)),
                                   ref.lam[len(cre)]))
            blocks = []
            for side, Op, k in ((0, L, kL), (1, R, kR)):
                legs = [(side, "c", i) for i in range(k)] + [(side, "a", i) for i in range(k)]
                blocks.append(("".join(letter[l] for l in legs), Op.block(k, tuple(rng[l] for l in legs), sp)))
            (subL, (ZL, lazyL)), (subR, (ZR, lazyR)) = blocks
            if lazyR:
                raise NotImplementedError("lazy block on the right operand")
            K = np.zeros([dims[c] for c in out_sub])
            if ZR is not None:
                if ZL is not None:
                    K = K + np.einsum(",".join([s for s, _ in others] + [subL, subR]) + "->" + out_sub,
                                      *([o for _, o in others] + [ZL, ZR]), optimize="greedy")
                for c, piece in lazyL:
                    K = K + _lazy_contract(piece, c, subL, others + [(subR, ZR)], out_sub, dims, sp)
            val = (sign * mult * pref0) * mkgno.antisymmetrize(np.asarray(K), r)
            key = (r, blk)
            out[key] = out[key] + val if key in out else val
    return out


def bcommutator(L: BOp, R: BOp, ref: Ref, want, sp: Spaces):
    """Wanted blocks of [L, R] (generalized normal order, cumulants to rank 3):
    {(rank, ranges): array}, the scalar under (0, ())."""
    res = {}
    for kL in L.parts:
        for kR in R.parts:
            lr = _product_blocks(L, kL, R, kR, ref, want, sp)
            rl = _product_blocks(R, kR, L, kL, ref, want, sp)
            for key in set(lr) | set(rl):
                v = lr.get(key, 0.0) - rl.get(key, 0.0)
                res[key] = res[key] + v if key in res else np.asarray(v, dtype=np.float64)
    return res


# ----------------------------------------------------------------------------
# the DSRG problem on blocks
# ----------------------------------------------------------------------------

EXC1 = ("P", "H")
EXC2 = ("P", "P", "H", "H")


class BlockProblem:
    def __init__(self, inst: dict):
        nc, na, nv = inst["nc"], inst["na"], inst["nv"]
        self.nc, self.na, self.nv = nc, na, nv
        sp = self.sp = Spaces(nc, na, nv)
        n = sp.n
        self.s = float(inst["s"])
        eps = np.asarray(inst["eps"], dtype=np.float64)
        self.eps = np.concatenate([eps, eps])
        self.B = np.asarray(inst["B"], dtype=np.float64)
        self.V = DFTwoBody(self.B, sp)
        # off-diagonal Fock part f^(1) on all spin orbitals (its diagonal blocks removed)
        F = np.zeros((sp.nso, sp.nso))
        if inst.get("f1") is not None:
            f1 = np.array(inst["f1"], dtype=np.float64)
            for lo, hi in ((0, nc), (nc, nc + na), (nc + na, n)):
                f1[lo:hi, lo:hi] = 0.0
            F[:n, :n] = f1
            F[n:, n:] = f1
        self.F1 = F
        # gamma on H (identity on core), eta on P (identity on virtual), cumulants on A
        g = np.zeros((sp.nso, sp.nso))
        for s_ in range(2):
            for m in range(nc):
                g[s_ * n + m, s_ * n + m] = 1.0
        if na:
            g[nc:nc + na, nc:nc + na] = np.asarray(inst["g1a"]).reshape(na, na)
            g[n + nc:n + nc + na, n + nc:n + nc + na] = np.asarray(inst["g1b"]).reshape(na, na)
        self.gamma = g
        H, P = sp["H"], sp["P"]
        lam = {}
        if na:
            sh2, sh3 = (na,) * 4, (na,) * 6
            lam[2] = _spin_tensor({0: np.reshape(inst["l2aa"], sh2), 1: np.reshape(inst["l2ab"], sh2),
                                   2: np.reshape(inst["l2bb"], sh2)}, na, 2)
            lam[3] = _spin_tensor({0: np.reshape(inst["l3aaa"], sh3), 1: np.reshape(inst["l3aab"], sh3),
                                   2: np.reshape(inst["l3abb"], sh3), 3: np.reshape(inst["l3bbb"], sh3)}, na, 3)
        else:
            lam[2], lam[3] = np.zeros((0,) * 4), np.zeros((0,) * 6)
        self.ref = Ref(g[np.ix_(H, H)], np.eye(sp.nso)[np.ix_(P, P)] - g[np.ix_(P, P)], lam)
        e = self.eps
        eP, eH = e[P], e[H]
        self.D1 = eH[None, :] - eP[:, None]                                   # D^i_a at [a,i]
        self.D2 = (eH[None, None, :, None] + eH[None, None, None, :]
                   - eP[:, None, None, None] - eP[None, :, None, None])      # D^{ij}_{ab} at [a,b,i,j]
        isA = lambda idx: sp.pos["A"][idx] >= 0
        aP, aH = isA(P), isA(H)
        self.mask1 = ~(aP[:, None] & aH[None, :])
        self.mask2 = ~(aP[:, None, None, None] & aP[None, :, None, None] & aH[None, None, :, None]
                       & aH[None, None, None, :])
        # active-active pieces for the gamma source term of Eqs. T1_1st / T1_2nd
        A = sp["A"]
        self.Dux = e[A][None, :] - e[A][:, None]   # D^u_x = eps_x - eps_u at [u, x]
        self.gA = g[np.ix_(A, A)]                  # gamma[x, u]
        self.posP_A = sp.pos["P"][A]
        self.posH_A = sp.pos["H"][A]

    # Eqs. T1_1st / T2_1st (and T1_2nd / T2_2nd with O in place of H(1)):
    # t^{ij}_{ab} = o^{ij}_{ab} R(D^{ij}_{ab}), t^i_a = [o^i_a + sum_ux D^u_x t^{iu}_{ax} gamma^x_u] R(D^i_a)
    def amplitudes(self, o1, o2):
        s = self.s
        T2 = np.empty(self.D2.shape)
        for lo in range(0, T2.shape[0], 8):   # element-wise; in slabs to bound temporaries
            sl = slice(lo, lo + 8)
            T2[sl] = np.where(self.mask2[sl], o2[sl] * regulariser(s, self.D2[sl]), 0.0)
        src = self.gamma_source(T2)
        T1 = np.where(self.mask1, (o1 + src) * regulariser(s, self.D1), 0.0)
        return T1, T2, src

    def gamma_source(self, T2):
        if self.na == 0:
            return np.zeros(self.D1.shape)
        T2ax = T2[:, self.posP_A][:, :, :, self.posH_A]        # T2[a, x, i, u], x, u active
        return np.einsum("axiu,ux,xu->ai", T2ax, self.Dux, self.gA, optimize=True)

    def w_closed_form(self, T1, T2, src):
        """Excitation blocks of W = [H(0), A(1)]."""
        return -self.D1 * T1 + src, -self.D2 * T2

    def excitation_op(self, X1, X2, herm):
        """X1 on [P,H], X2 on [P,P,H,H]; herm adds the Hermitian image.  With
        herm the internal (all-active) elements are left out: the image would
        count them twice, and no scalar <[X, T]> reads them (T's internal
        elements vanish)."""
        if herm:
            X1 = None if X1 is None else np.where(self.mask1, X1, 0.0)
            X2 = None if X2 is None else np.where(self.mask2, X2, 0.0)
        parts = {}
        if X1 is not None:
            parts[1] = [(1.0, Stored(X1, EXC1, herm))]
        if X2 is not None:
            parts[2] = [(1.0, Stored(X2, EXC2, herm))]
        return BOp(0.0, parts)

    def v_op(self, coef):
        """coef (f^(1) + V)"""
        parts = {2: [(coef, self.V)]}
        if np.any(self.F1):
            parts[1] = [(coef, Stored(self.F1, ("G", "G")))]
        return BOp(0.0, parts)


def _blocks(res, rank, ranges, shape):
    return res.get((rank, ranges), np.zeros(shape))


def dsrg_pt3(inst: dict, pt2_only: bool = False, return_intermediates: bool = False) -> dict:
    """E(2), E(3)a, E(3)b and E(3) of Eqs. E(2) and E(3)."""
    Pb = BlockProblem(inst)
    sp, ref = Pb.sp, Pb.ref
    scalar = {0: [()]}
    exc = {1: [EXC1], 2: [EXC2]}
    # first-order amplitudes from H(1) = f^(1) + V (Eqs. T1_1st, T2_1st)
    f1_PH = Pb.F1[np.ix_(sp["P"], sp["H"])]
    v_PPHH = Pb.V.block(EXC2, sp)
    T1, T2, src = Pb.amplitudes(f1_PH, v_PPHH)
    W1, W2 = Pb.w_closed_form(T1, T2, src)
    T = Pb.excitation_op(T1, T2, herm=False)
    # A(1) = T(1) - T(1)^+ (the de-excitation part stored on [H,P], [H,H,P,P])
    A = T + BOp(0.0, {1: [(-1.0, Stored(np.ascontiguousarray(T1.T), ("H", "P")))],
                      2: [(-1.0, Stored(np.ascontiguousarray(np.transpose(T2, (2, 3, 0, 1))), ("H", "H", "P", "P")))]})
    W = Pb.excitation_op(W1, W2, herm=True)
    # Htilde(1) = 2 H(1) + [H(0), A(1)]  (Eq. Hbar_1st)
    Ht1 = Pb.v_op(2.0) + W
    E2 = float(bcommutator(Ht1, T, ref, scalar, sp).get((0, ()), 0.0))
    out = {"e2": E2}
    inter = {"T1": T1, "T2": T2, "W1": W1, "W2": W2}
    if not pt2_only:
        # O = 1/2 [Htilde(1), A(1)]_{1,2} on its excitation blocks
        Ob = bcommutator(Ht1, A, ref, exc, sp)
        O1 = 0.5 * _blocks(Ob, 1, EXC1, T1.shape)
        O2 = 0.5 * _blocks(Ob, 2, EXC2, T2.shape)
        # second-order amplitudes (Eqs. T1_2nd, T2_2nd)
        U1, U2, src2 = Pb.amplitudes(O1, O2)
        Tb = Pb.excitation_op(U1, U2, herm=False)
        # Htilde(2)_{1,2} = [H(0), A(2)] + O - 1/6 [W, A(1)]_{1,2}, excitation blocks
        Z1, Z2 = Pb.w_closed_form(U1, U2, src2)
        Qb = bcommutator(W, A, ref, exc, sp)
        Z1 = Z1 + O1 - _blocks(Qb, 1, EXC1, T1.shape) / 6.0
        Z2 = Z2 + O2 - _blocks(Qb, 2, EXC2, T2.shape) / 6.0
        Ht2 = Pb.excitation_op(Z1, Z2, herm=True)
        E3a = float(bcommutator(Ht1, Tb, ref, scalar, sp).get((0, ()), 0.0))
        E3b = float(bcommutator(Ht2, T, ref, scalar, sp).get((0, ()), 0.0))
        out.update(e3a=E3a, e3b=E3b, e3=E3a + E3b)
        inter.update(O1=O1, O2=O2, T1b=U1, T2b=U2, Z1=Z1, Z2=Z2)
    if return_intermediates:
        out["_inter"] = inter
        out["_problem"] = Pb
    return out
