"""Generic commutator engine in Mukherjee-Kutzelnigg generalized normal order.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper evaluates every commutator of Eqs. Hbar_1st-Hbar_3rd with the
generalized Wick theorem of Mukherjee and Kutzelnigg (Sec. II.A) and keeps at
most two-body terms (the "1,2" truncation after Eq. exactBCH).  It prints no
term list (Sec. III defers it), so this module enumerates the contractions
itself, on dense spin-orbital tensors:

* An operator is ``c0 + sum Z1[p,q] {a+_p a_q} + 1/4 sum Z2[p,q,r,s]
  {a+_p a+_q a_s a_r} + 1/36 sum Z3[...] {...}``; Z_k is antisymmetric among
  its creator indices and among its annihilator indices.
* In a product {L}{R} the contractions are: an L-creator with an
  R-annihilator -> gamma[c,a] = <a+_c a_a>; an L-annihilator with an
  R-creator -> eta[a,c] = <a_a a+_c>; and k-body density cumulants
  lambda_k (k = 2, 3) joining k creators and k annihilators taken from both
  operators.  The sign is the parity of the permutation that brings each
  contracted group and then the open legs into canonical order.
* Contraction patterns that use cumulants only cancel between LR and RL,
  so the commutator keeps patterns with at least one single contraction.

Patterns equivalent under relabelling of the legs of one class (L creators,
L annihilators, R creators, R annihilators) give the same contribution; one
representative is evaluated and multiplied by the number of such patterns.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np


# ----------------------------------------------------------------------------
# operators
# ----------------------------------------------------------------------------

@dataclass
class Op:
    n: int
    c0: float = 0.0
    z: dict = field(default_factory=dict)  # rank -> dense tensor

    def get(self, k):
        return self.z.get(k)

    def copy(self):
        return Op(self.n, self.c0, {k: v.copy() for k, v in self.z.items()})

    def __add__(self, o):
        out = self.copy()
        out.c0 += o.c0
        for k, v in o.z.items():
            out.z[k] = out.z[k] + v if k in out.z else v.copy()
        return out

    def __sub__(self, o):
        return self + o.scale(-1.0)

    def scale(self, a):
        return Op(self.n, a * self.c0, {k: a * v for k, v in self.z.items()})

    def truncate(self, kmax=2):
        return Op(self.n, self.c0, {k: v for k, v in self.z.items() if k <= kmax})

    def adjoint(self):
        """Hermitian conjugate of a real operator: swap creator/annihilator slots."""
        out = {}
        for k, v in self.z.items():
            out[k] = np.ascontiguousarray(np.transpose(v, list(range(k, 2 * k)) + list(range(k))))
        return Op(self.n, self.c0, out)


@dataclass
class Reference:
    """gamma, eta on all spin orbitals; cumulants on the active spin orbitals."""
    gamma: np.ndarray
    eta: np.ndarray
    act: np.ndarray               # active spin-orbital indices
    lam: dict                     # rank -> tensor over len(act)


# ----------------------------------------------------------------------------
# permutations
# ----------------------------------------------------------------------------

def parity(seq) -> int:
    seq = list(seq)
    s = 1
    for i in range(len(seq)):
        for j in range(i + 1, len(seq)):
            if seq[i] > seq[j]:
                s = -s
    return s


def antisymmetrize(K: np.ndarray, r: int) -> np.ndarray:
    """Signed sum over all permutations of the r creator and r annihilator axes."""
    if r <= 1:
        return K.copy()
    out = np.zeros_like(K)
    perms = list(itertools.permutations(range(r)))
    for pc in perms:
        sc = parity(pc)
        for pa in perms:
            sa = parity(pa)
            axes = list(pc) + [r + i for i in pa]
            out += (sc * sa) * np.transpose(K, axes)
    return out


# ----------------------------------------------------------------------------
# contraction patterns
# ----------------------------------------------------------------------------
# A leg is (side, kind, i): side 0 = left operator, 1 = right; kind 'c'/'a';
# i = slot in the tensor.  The string of an operator of rank k is
#   c0+ c1+ .. c(k-1)+ a(k-1) .. a1 a0
# so annihilator slot i sits at position k + (k-1-i).

def _position(side, kind, i, kL, kR):
    base = 0 if side == 0 else 2 * kL
    k = kL if side == 0 else kR
    return base + (i if kind == "c" else k + (k - 1 - i))


_GROUP_PAIR_G = (1, 0, 0, 1)   # L creator with R annihilator -> gamma
_GROUP_PAIR_E = (0, 1, 1, 0)   # L annihilator with R creator -> eta


def _group_types(kL, kR, lam_max):
    """All admissible group types (nLc, nLa, nRc, nRa)."""
    types = [_GROUP_PAIR_G, _GROUP_PAIR_E]
    for m in range(2, lam_max + 1):
        for nLc in range(0, min(kL, m) + 1):
            nRc = m - nLc
            if nRc > kR:
                continue
            for nLa in range(0, min(kL, m) + 1):
                nRa = m - nLa
                if nRa > kR:
                    continue
                if nLc + nLa == 0 or nRc + nRa == 0:
                    continue  # all legs from one operator: vanishes in normal order
                types.append((nLc, nLa, nRc, nRa))
    return types


def enumerate_patterns(kL, kR, lam_max=3, out_max=3, commutator=True):
    """Yield (groups, multiplicity) where groups is a tuple of group types."""
    types = _group_types(kL, kR, lam_max)
    caps = (kL, kL, kR, kR)
    results = []

    def rec(start, chosen, used):
        if chosen:
            open_legs = sum(caps) - sum(used)
            r = open_legs // 2
            ok = r <= out_max
            if commutator and not any(g in (_GROUP_PAIR_G, _GROUP_PAIR_E) for g in chosen):
                ok = False
            # open creators must equal open annihilators (always true: each group balanced)
            if ok:
                results.append(tuple(chosen))
        for t in range(start, len(types)):
            g = types[t]
            nu = tuple(u + x for u, x in zip(used, g))
            if any(a > b for a, b in zip(nu, caps)):
                continue
            rec(t, chosen + [g], nu)

    rec(0, [], (0, 0, 0, 0))
    out = []
    for groups in results:
        used = [sum(g[c] for g in groups) for c in range(4)]
        mult = 1
        for c in range(4):
            k = caps[c]
            m = math.factorial(k)
            for g in groups:
                m //= math.factorial(g[c])
            m //= math.factorial(k - used[c])
            mult *= m
        for g in set(groups):
            mult //= math.factorial(groups.count(g))
        out.append((groups, mult))
    return out


def _representative(groups, kL, kR):
    """Assign concrete legs to each group (lowest free slots first)."""
    nxt = {(0, "c"): 0, (0, "a"): 0, (1, "c"): 0, (1, "a"): 0}
    assigned = []
    for g in groups:
        nLc, nLa, nRc, nRa = g
        legs = []
        for side, kind, cnt in ((0, "c", nLc), (0, "a", nLa), (1, "c", nRc), (1, "a", nRa)):
            for _ in range(cnt):
                legs.append((side, kind, nxt[(side, kind)]))
                nxt[(side, kind)] += 1
        assigned.append(legs)
    open_legs = []
    for side, k in ((0, kL), (1, kR)):
        for kind in ("c", "a"):
            for i in range(nxt[(side, kind)], k):
                open_legs.append((side, kind, i))
    return assigned, open_legs


def _canonical(legs, kL, kR):
    """Creators then annihilators, each in string order."""
    pos = lambda l: _position(*l, kL, kR)
    cre = sorted([l for l in legs if l[1] == "c"], key=pos)
    ann = sorted([l for l in legs if l[1] == "a"], key=pos)
    return cre, ann


# ----------------------------------------------------------------------------
# evaluation
# ----------------------------------------------------------------------------

_LETTERS = "abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ"


def product_terms(ZL, kL, ZR, kR, ref: Reference, lam_max=3, out_max=3):
    """Sum over pair-containing contraction patterns of {L}{R}.

    Returns dict rank -> tensor (rank 0 as a 0-d array) in the Z convention.
    """
    out = {}
    patterns = enumerate_patterns(kL, kR, lam_max=lam_max, out_max=out_max)
    pref0 = 1.0 / (math.factorial(kL) ** 2 * math.factorial(kR) ** 2)
    for groups, mult in patterns:
        assigned, open_legs = _representative(groups, kL, kR)
        letter = {}
        li = iter(_LETTERS)
        for legs in assigned:
            for l in legs:
                letter[l] = next(li)
        for l in open_legs:
            letter[l] = next(li)
        # permutation sign: string order -> [groups canonical][open canonical]
        target = []
        for g, legs in zip(groups, assigned):
            cre, ann = _canonical(legs, kL, kR)
            if g == _GROUP_PAIR_E:
                target += ann + cre          # <a_a a+_c>
            else:
                target += cre + ann          # gamma: <a+_c a_a>;  lambda: c.. then a..
        ocre, oann = _canonical(open_legs, kL, kR)
        target += ocre + oann
        sign = parity([_position(*l, kL, kR) for l in target])
        # operands
        act_axes = {}
        operands, subs = [], []
        lam_legs = set()
        for g, legs in zip(groups, assigned):
            cre, ann = _canonical(legs, kL, kR)
            if g == _GROUP_PAIR_G:
                operands.append(ref.gamma)
                subs.append(letter[cre[0]] + letter[ann[0]])
            elif g == _GROUP_PAIR_E:
                operands.append(ref.eta)
                subs.append(letter[ann[0]] + letter[cre[0]])
            else:
                m = len(cre)
                if m not in ref.lam:
                    raise KeyError(f"cumulant of rank {m} not supplied")
                # lambda[x1..xm, y1..ym] <-> a+x1..a+xm a_ym..a_y1
                operands.append(ref.lam[m])
                subs.append("".join(letter[l] for l in cre) + "".join(letter[l] for l in reversed(ann)))
                lam_legs.update(legs)
        for side, Z, k in ((0, ZL, kL), (1, ZR, kR)):
            legs = [(side, "c", i) for i in range(k)] + [(side, "a", i) for i in range(k)]
            T = Z
            for ax, l in enumerate(legs):
                if l in lam_legs:
                    T = np.take(T, ref.act, axis=ax)
            operands.append(T)
            subs.append("".join(letter[l] for l in legs))
        out_sub = "".join(letter[l] for l in ocre) + "".join(letter[l] for l in reversed(oann))
        K = np.einsum(",".join(subs) + "->" + out_sub, *operands, optimize="greedy")
        r = len(ocre)
        val = (sign * mult * pref0) * antisymmetrize(np.asarray(K), r)
        out[r] = out[r] + val if r in out else val
    return out


def commutator(L: Op, R: Op, ref: Reference, out_max=2, lam_max=3) -> Op:
    """[L, R] in generalized normal order, keeping outputs of rank <= out_max."""
    res = Op(L.n)
    for kL, ZL in L.z.items():
        for kR, ZR in R.z.items():
            lr = product_terms(ZL, kL, ZR, kR, ref, lam_max=lam_max, out_max=out_max)
            rl = product_terms(ZR, kR, ZL, kL, ref, lam_max=lam_max, out_max=out_max)
            for r in set(lr) | set(rl):
                v = lr.get(r, 0.0) - rl.get(r, 0.0)
                if r == 0:
                    res.c0 += float(v)
                else:
                    res.z[r] = res.z[r] + v if r in res.z else np.asarray(v)
    return res
