"""Brute-force exact k-NN in a prefix P_{1:m}: the definition the method reaches.

Theorem 1 (Sec. 4.1) is stated for N_k(q), the k nearest sites of q in P;
the prefix-subset reading (Sec. 4.2, "Prefix-Subset and Multiresolution
Queries") restricts the candidate set to P_{1:m}. The order among equal
distances follows Eq. (2), whose "<=" keeps the earlier site: the key of
rank r is (D(r), r), smaller first.

D(r) is the squared Euclidean distance evaluated in float64 from the
float32 inputs promoted to double, in the fixed order
    D = ((qx - px)^2 + (qy - py)^2) + (qz - pz)^2,
no fused multiply-add. Ranks are 0-based (the paper's p_i is rank i-1).

Test infrastructure only; see the package docstring.
"""
from __future__ import annotations

import numpy as np


def sq_dist64(P: np.ndarray, q) -> np.ndarray:
    """float64 squared distances from q to every row of P (float32 (n,3))."""
    P64 = np.asarray(P, dtype=np.float32).astype(np.float64)
    q64 = np.asarray(q, dtype=np.float32).astype(np.float64)
    dx = q64[0] - P64[:, 0]
    dy = q64[1] - P64[:, 1]
    dz = q64[2] - P64[:, 2]
    return (dx * dx + dy * dy) + dz * dz


def knn_one(P: np.ndarray, q, k: int, m: int):
    """The min(k, m) smallest keys (D(r), r) over ranks r < m.

    Returns (ranks int64, D float64), ascending by key.
    """
    m = int(m)
    kk = min(int(k), m)
    D = sq_dist64(P[:m], q)
    thresh = np.partition(D, kk - 1)[kk - 1]
    cand = np.nonzero(D <= thresh)[0]
    order = np.lexsort((cand, D[cand]))[:kk]
    r = cand[order]
    return r.astype(np.int64), D[r]


def knn(P: np.ndarray, Q: np.ndarray, k: int, m=0):
    """Brute-force k-NN for every query row of Q.

    P: float32 (n,3) in rank order; Q: float32 (nq,3); m: 0 (= n), an int,
    or an int array (nq,) of per-query prefix bounds.
    Returns idx int32 (nq,k), d2 float32 (nq,k), D64 float64 (nq,k);
    positions past min(k, m) hold (-1, +inf, +inf).
    """
    n = P.shape[0]
    nq = Q.shape[0]
    if np.ndim(m) == 0:
        ms = np.full(nq, n if int(m) == 0 else int(m), dtype=np.int64)
    else:
        ms = np.asarray(m, dtype=np.int64).reshape(nq)
    idx = np.full((nq, k), -1, dtype=np.int32)
    D64 = np.full((nq, k), np.inf, dtype=np.float64)
    for i in range(nq):
        r, D = knn_one(P, Q[i], k, ms[i])
        idx[i, :r.size] = r
        D64[i, :r.size] = D
    return idx, D64.astype(np.float32), D64


def keys_upto(P: np.ndarray, q, m: int, dmax: float):
    """Every key (D(r), r) with r < m and D(r) <= dmax, ascending.

    Used to list the whole group of near-equal distances around the k-th
    neighbour when results are compared.
    """
    D = sq_dist64(P[: int(m)], q)
    cand = np.nonzero(D <= dmax)[0]
    order = np.lexsort((cand, D[cand]))
    r = cand[order]
    return r.astype(np.int64), D[r]
