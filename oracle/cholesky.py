"""Pivoted incomplete Cholesky factorisation of a two-electron supermatrix.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper factorises the two-electron integrals as (pq|rs) ~ sum_Q B^Q_pq
B^Q_rs (Eq. int_fact) and, for its larger applications, obtains B by
Cholesky decomposition with a threshold of 1e-6 or 1e-8 a.u. (Sec. IV).
This is the pivoted incomplete Cholesky algorithm of Beebe and Linderberg
(Int. J. Quantum Chem. 12, 683 (1977)) as described by Koch, Sanchez de
Meras and Pedersen (J. Chem. Phys. 118, 9481 (2003)), on the supermatrix
V[(pq), (rs)] = (pq|rs) with compound indices (pq) = p n + q:

  D = diag(V)
  for Q = 0, 1, ...:
      J = the compound index of the largest D (the smallest such index on ties)
      stop if D[J] <= tau (or after max_vecs vectors)
      L[:] = (V[:, J] - sum_{Q' < Q} B[Q'][:] B[Q'][J]) / sqrt(D[J])
      B[Q] = L;  D -= L * L

Every correction is summed over Q' in increasing order with a separate
rounding of each product and each sum, so that another implementation doing
the same operations in the same order reproduces the pivots and vectors bit
for bit.
"""
from __future__ import annotations

import numpy as np


def pivoted_cholesky(V: np.ndarray, tau: float, max_vecs: int | None = None):
    """Returns (B [nvec][N], pivots [nvec]) for the N x N PSD matrix V."""
    V = np.asarray(V, dtype=np.float64)
    N = V.shape[0]
    if max_vecs is None:
        max_vecs = N
    D = np.diag(V).copy()
    vecs, piv = [], []
    for _ in range(max_vecs):
        J = int(np.argmax(D))          # first occurrence of the maximum
        dJ = D[J]
        if not dJ > tau:
            break
        acc = np.zeros(N)
        for Bq in vecs:                # increasing Q', one product and one sum rounding each
            acc = acc + Bq * Bq[J]
        L = (V[J, :] - acc) / np.sqrt(dJ)   # row J = column J (V symmetric)
        vecs.append(L)
        piv.append(J)
        D = D - L * L
    return (np.array(vecs) if vecs else np.zeros((0, N))), np.array(piv, dtype=np.int64)


def supermatrix(eri: np.ndarray) -> np.ndarray:
    """(pq|rs) as the (n^2 x n^2) matrix V[(pq), (rs)]."""
    n = eri.shape[0]
    return np.ascontiguousarray(eri.reshape(n * n, n * n))
