"""Brute-force second quantisation in one particle-number sector.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  Used to pin the
generalized-normal-order engine and the energy expressions on spaces of
at most a dozen spin orbitals: operators become explicit matrices, so a
commutator is a matrix commutator and an expectation value a quadratic form.

Normal order is that of Mukherjee and Kutzelnigg relative to a reference
|Psi> (Sec. II.A): the plain operator string minus all of its internal
contractions, where a creator followed by an annihilator contracts to
gamma[c,a] = <Psi|a+_c a_a|Psi> and k creators with k annihilators to the
k-body density cumulant.  The decomposition below is written independently
of the engine in ``mkgno``: it enumerates concrete contractions of one string.
"""
from __future__ import annotations

import itertools
import math
from functools import lru_cache

import numpy as np


def _bits(nso, nel):
    out = []
    for occ in itertools.combinations(range(nso), nel):
        b = 0
        for o in occ:
            b |= 1 << o
        out.append(b)
    return out


class Sector:
    """Basis of all determinants with ``nel`` electrons in ``nso`` spin orbitals."""

    def __init__(self, nso, nel):
        self.nso, self.nel = nso, nel
        self.dets = _bits(nso, nel) if 0 <= nel <= nso else []
        self.index = {d: k for k, d in enumerate(self.dets)}

    @property
    def dim(self):
        return len(self.dets)


class FockSpace:
    """Annihilation matrices between the sectors N, N-1, ..., N-kmax."""

    def __init__(self, nso, nel, kmax=3):
        self.nso, self.nel = nso, nel
        self.sec = {k: Sector(nso, nel - k) for k in range(0, kmax + 1)}
        self.ann = {}  # (k, s) -> matrix from sector N-k to N-k-1
        for k in range(0, kmax):
            src, dst = self.sec[k], self.sec[k + 1]
            for s in range(nso):
                M = np.zeros((dst.dim, src.dim))
                for j, d in enumerate(src.dets):
                    if d >> s & 1:
                        sign = -1.0 if bin(d & ((1 << s) - 1)).count("1") % 2 else 1.0
                        M[dst.index[d ^ (1 << s)], j] = sign
                self.ann[(k, s)] = M
        self._tuples = {}
        self._stack = {}

    @property
    def dim(self):
        return self.sec[0].dim

    def tuples(self, k):
        if k not in self._tuples:
            self._tuples[k] = list(itertools.combinations(range(self.nso), k))
        return self._tuples[k]

    def stack(self, k):
        """an[t] = a_{tk} ... a_{t1} (acting on sector N) for ascending tuples t."""
        if k not in self._stack:
            mats = []
            for t in self.tuples(k):
                M = np.eye(self.dim)
                for lvl, s in enumerate(t):
                    M = self.ann[(lvl, s)] @ M
                mats.append(M)
            self._stack[k] = np.array(mats)
        return self._stack[k]

    def plain(self, Z, k):
        """(1/(k!)^2) sum Z[c..,a..] a+_c1..a+_ck a_ak..a_a1 on sector N."""
        if k == 0:
            return float(Z) * np.eye(self.dim)
        tup = self.tuples(k)
        # sorted-tuple block of Z: Zs[C, A]
        cidx = np.array(tup)
        Zs = Z[tuple(cidx[:, i][:, None] for i in range(k)) + tuple(cidx[:, i][None, :] for i in range(k))]
        S = self.stack(k)
        W = np.tensordot(Zs, S, axes=(1, 0))          # [C, m, N]
        return np.tensordot(S, W, axes=((0, 1), (0, 1)))  # sum_C S[C]^T W[C]

    def state(self, dets_full, coef):
        v = np.zeros(self.dim)
        for d, c in zip(dets_full, coef):
            v[self.sec[0].index[d]] += c
        return v

    def rdm(self, psi, k):
        """Gamma_k[p..,q..] = <psi| a+_p1..a+_pk a_qk..a_q1 |psi> (antisymmetrised)."""
        S = self.stack(k)
        phi = S @ psi  # [T, m]
        ov = phi @ phi.T
        G = np.zeros((self.nso,) * (2 * k))
        tup = self.tuples(k)
        perms = list(itertools.permutations(range(k)))
        for a, P in enumerate(tup):
            for b, Q in enumerate(tup):
                v = ov[a, b]
                if v == 0.0:
                    continue
                for p1 in perms:
                    s1 = _parity(p1)
                    for p2 in perms:
                        G[tuple(P[i] for i in p1) + tuple(Q[i] for i in p2)] = s1 * _parity(p2) * v
        return G


def _parity(seq):
    seq = list(seq)
    s = 1
    for i in range(len(seq)):
        for j in range(i + 1, len(seq)):
            if seq[i] > seq[j]:
                s = -s
    return s


def _antisym(K, r):
    if r <= 1:
        return np.array(K, copy=True)
    out = np.zeros_like(K)
    for pc in itertools.permutations(range(r)):
        for pa in itertools.permutations(range(r)):
            out += _parity(pc) * _parity(pa) * np.transpose(K, list(pc) + [r + i for i in pa])
    return out


@lru_cache(maxsize=None)
def _string_patterns(k):
    """All sets of internal contractions of c0+..c(k-1)+ a(k-1)..a0.

    A pattern is a tuple of groups (creators, annihilators) with equal sizes;
    size 1 is a gamma contraction, size m >= 2 a lambda_m contraction.
    """
    out = []

    def rec(free_c, free_a, groups):
        if not free_c:
            out.append(tuple(groups))
            return
        c = free_c[0]
        rest_c = free_c[1:]
        # leave creator c open
        rec(rest_c, free_a, groups)
        # put c into a group of size m with m-1 larger free creators
        for m in range(1, len(free_c) + 1):
            for others in itertools.combinations(rest_c, m - 1):
                for anns in itertools.combinations(free_a, m):
                    rc = tuple(x for x in rest_c if x not in others)
                    ra = tuple(x for x in free_a if x not in anns)
                    rec(rc, ra, groups + [((c,) + others, anns)])

    rec(tuple(range(k)), tuple(range(k)), [])
    return [p for p in out if p]  # drop the empty pattern


def normal_ordered(fs: FockSpace, Z, k, gamma, act, lam):
    """Matrix of (1/(k!)^2) sum Z {a+..a..} in MK normal order on sector N."""
    if k == 0:
        return float(Z) * np.eye(fs.dim)
    M = fs.plain(Z, k)
    pos_c = lambda i: i
    pos_a = lambda i: k + (k - 1 - i)
    letters = "abcdefghijklmnop"
    for pattern in _string_patterns(k):
        used_c = set(x for g in pattern for x in g[0])
        used_a = set(x for g in pattern for x in g[1])
        open_c = [i for i in range(k) if i not in used_c]
        open_a = sorted([i for i in range(k) if i not in used_a], key=pos_a)
        seq = []
        for cs, as_ in pattern:
            seq += [pos_c(i) for i in sorted(cs)] + sorted(pos_a(i) for i in as_)
        seq += [pos_c(i) for i in open_c] + [pos_a(i) for i in open_a]
        sign = _parity(seq)
        L = {("c", i): letters[i] for i in range(k)}
        L.update({("a", i): letters[k + i] for i in range(k)})
        ops, subs = [], []
        Zt = Z
        for cs, as_ in pattern:
            if len(cs) == 1:
                ops.append(gamma)
                subs.append(L[("c", cs[0])] + L[("a", as_[0])])
            else:
                m = len(cs)
                ann_string = sorted(as_, key=pos_a)          # string order
                ops.append(lam[m])
                subs.append("".join(L[("c", i)] for i in sorted(cs)) +
                            "".join(L[("a", i)] for i in reversed(ann_string)))
                for i in cs:
                    Zt = np.take(Zt, act, axis=i)
                for i in as_:
                    Zt = np.take(Zt, act, axis=k + i)
        ops.append(Zt)
        subs.append("".join(L[("c", i)] for i in range(k)) + "".join(L[("a", i)] for i in range(k)))
        # open annihilators: output slot 1 is the last in string order
        out = "".join(L[("c", i)] for i in open_c) + "".join(L[("a", i)] for i in reversed(open_a))
        K = np.einsum(",".join(subs) + "->" + out, *ops, optimize="greedy")
        r = len(open_c)
        Y = _antisym(np.asarray(K), r) * (sign / math.factorial(k) ** 2)
        M = M - normal_ordered(fs, Y, r, gamma, act, lam)
    return M


def operator_matrix(fs, c0, zs: dict, gamma, act, lam):
    M = c0 * np.eye(fs.dim)
    for k, Z in zs.items():
        M = M + normal_ordered(fs, Z, k, gamma, act, lam)
    return M


def random_antisym(rng, n, k, scale=1.0):
    Z = rng.standard_normal((n,) * (2 * k)) * scale
    return _antisym(Z, k) if k > 1 else Z


def quasiparticle_normal_ordered(fs: FockSpace, Z, k, occ):
    """Single-determinant normal order, built without any contraction:
    for each string the occupied-orbital annihilators-of-holes (a+_i with i
    occupied) are moved to the right of the particle operators by plain
    reordering with the permutation sign."""
    if k == 0:
        return float(Z) * np.eye(fs.dim)
    occ = set(int(i) for i in occ)
    n = fs.nso
    full = np.eye(fs.dim)
    # elementary matrices on sector N for creators/annihilators: use the
    # Fock-space product through intermediate sectors computed on the fly
    M = np.zeros((fs.dim, fs.dim))
    rng_idx = range(n)
    for c in itertools.product(rng_idx, repeat=k):
        if len(set(c)) < k:
            continue
        for a in itertools.product(rng_idx, repeat=k):
            if len(set(a)) < k:
                continue
            z = Z[c + a]
            if z == 0.0:
                continue
            # string: c0+ .. c(k-1)+ a(k-1) .. a0 ; quasi-annihilators are
            # a+_i (i occupied) and a_e (e unoccupied); move them right
            ops = [("c", x) for x in c] + [("a", x) for x in reversed(a)]
            is_qann = [(t == "c" and x in occ) or (t == "a" and x not in occ) for t, x in ops]
            order = [i for i in range(len(ops)) if not is_qann[i]] + [i for i in range(len(ops)) if is_qann[i]]
            sign = _parity(order)
            M += (z * sign / math.factorial(k) ** 2) * _string_matrix(fs, [ops[i] for i in order])
    return M


def _string_matrix(fs, ops):
    """Matrix on sector N of a number-conserving product of elementary operators
    (applied right to left), by direct action on determinants."""
    dim = fs.dim
    M = np.zeros((dim, dim))
    sec = fs.sec[0]
    for j, d in enumerate(sec.dets):
        det, sign = d, 1.0
        ok = True
        for t, x in reversed(ops):
            occ_x = det >> x & 1
            below = bin(det & ((1 << x) - 1)).count("1")
            if t == "a":
                if not occ_x:
                    ok = False
                    break
                det ^= 1 << x
            else:
                if occ_x:
                    ok = False
                    break
                det |= 1 << x
            if below % 2:
                sign = -sign
        if ok:
            M[sec.index[det], j] += sign
    return M
