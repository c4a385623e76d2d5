"""Algorithm 1 and Algorithm 2 (Sec. 4), step by step, in float64.

The successor table is given in CSR form: the successors of rank i are
succ[rowp[i]:rowp[i+1]], ascending (insertion order, Sec. 3).

Readings of the paper used here (each also listed in the design notes):
  * Alg. 1 replaces the list being scanned when it moves to a closer site;
    the scan of the new list starts at its head (the rest of the old list is
    abandoned: every later transition is in the new site's list by Eqs. 3-4).
  * The site moved to is the first entry, in list order, that is strictly
    closer (Alg. 1's "<"); with ascending lists this is the next prefix
    nearest neighbour of Eq. (2).
  * Every site the descent moves to is a transition site and is inserted
    into N, as the "more robust implementation" of Sec. 4.2 does.
  * Alg. 2's loop "p <- N[i] for i = 1..k-1" is run as: repeatedly expand
    the nearest not-yet-expanded entry among the first k-1 of N until none
    is left. In exact arithmetic this visits the same entries in the same
    order (an insertion never lands before the entry being expanded).
  * "p_successor not in N" tests membership in the current N only.
  * Prefix bound m (Sec. 4.2): entries with rank >= m are ignored; lists are
    ascending, so a scan stops at the first such entry.
  * N is kept sorted by the key (D, rank) with D the float64 squared
    distance; capacity min(k, m); insertion sort as in Sec. 5.5.

Counters (per query) used for the algorithmic byte count:
  rows     successor rows opened (each scan start, descent or expansion)
  entries  successor entries read (including the one >= m that stops a scan)
  coords   site coordinates read (p_1 plus every entry < m that is read)

Test infrastructure only; see the package docstring.
"""
from __future__ import annotations

import numpy as np


class _Dist:
    """Squared distance to a fixed query in float64, same order as oracle.knn."""

    def __init__(self, P: np.ndarray, q):
        self.P = np.asarray(P, dtype=np.float32).astype(np.float64)
        self.q = np.asarray(q, dtype=np.float32).astype(np.float64)

    def __call__(self, r: int) -> float:
        p = self.P[r]
        dx = self.q[0] - p[0]
        dy = self.q[1] - p[1]
        dz = self.q[2] - p[2]
        return (dx * dx + dy * dy) + dz * dz


def strict_prefix_minima(P: np.ndarray, q, m: int):
    """Ranks r < m whose D(r) is strictly below every D(r') with r' < r.

    By Eq. (2) these are exactly the sites with Phi_{1:r}(q) = p_r, the
    transition sites of Sec. 4.2; the last one is the 1-NN in P_{1:m}.
    A linear scan, independent of any successor table.
    """
    dist = _Dist(P, q)
    out = []
    best = None
    for r in range(int(m)):
        d = dist(r)
        if best is None or d < best:
            best = d
            out.append(r)
    return out


class Counters:
    __slots__ = ("rows", "entries", "coords")

    def __init__(self):
        self.rows = 0
        self.entries = 0
        self.coords = 0

    def as_tuple(self):
        return (self.rows, self.entries, self.coords)


def descent(P, rowp, succ, q, m: int, cnt: Counters | None = None):
    """Algorithm 1: the 1-NN descent from p_1, returning the transition sites
    in the order they are reached (the last is the 1-NN in P_{1:m})."""
    cnt = cnt if cnt is not None else Counters()
    dist = _Dist(P, q)
    curr = 0
    dcurr = dist(0)
    cnt.coords += 1
    sites = [(dcurr, 0)]
    while True:
        cnt.rows += 1
        moved = False
        for e in range(int(rowp[curr]), int(rowp[curr + 1])):
            s = int(succ[e])
            cnt.entries += 1
            if s >= m:
                break
            d = dist(s)
            cnt.coords += 1
            if d < dcurr:
                curr, dcurr = s, d
                sites.append((d, s))
                moved = True
                break
        if not moved:
            return sites


def _insert(N, key, cap):
    """Insert key=(D, r) into the sorted list N (entries [D, r, expanded]),
    keeping at most cap entries; a key already present is not inserted."""
    d, r = key
    if len(N) == cap and (d, r) >= (N[-1][0], N[-1][1]):
        return
    pos = len(N)
    for i, e in enumerate(N):
        if e[0] == d and e[1] == r:
            return
        if (d, r) < (e[0], e[1]):
            pos = i
            break
    N.insert(pos, [d, r, False])
    if len(N) > cap:
        N.pop()


def knn_dp(P, rowp, succ, q, k: int, m: int = 0, cnt: Counters | None = None):
    """Algorithm 2 initialised by Algorithm 1. Returns (ranks, D) ascending."""
    n = int(len(rowp) - 1)
    m = n if int(m) == 0 else int(m)
    cnt = cnt if cnt is not None else Counters()
    dist = _Dist(P, q)
    cap = min(int(k), m)
    N: list = []
    for d, s in descent(P, rowp, succ, q, m, cnt):
        _insert(N, (d, s), cap)
    while True:
        lim = min(len(N), int(k) - 1)
        i = next((j for j in range(lim) if not N[j][2]), None)
        if i is None:
            break
        N[i][2] = True
        p = N[i][1]
        cnt.rows += 1
        for e in range(int(rowp[p]), int(rowp[p + 1])):
            s = int(succ[e])
            cnt.entries += 1
            if s >= m:
                break
            d = dist(s)
            cnt.coords += 1
            _insert(N, (d, s), cap)
    return (np.array([e[1] for e in N], dtype=np.int64),
            np.array([e[0] for e in N], dtype=np.float64))


def complete_table(n: int):
    """L_i = {i+1, ..., n-1}: a superset of every successor list, so the
    methods above stay exact on it (extra entries are extra candidates)."""
    rowp = np.zeros(n + 1, dtype=np.int64)
    rowp[1:] = np.cumsum(np.arange(n - 1, -1, -1))
    succ = np.concatenate([np.arange(i + 1, n) for i in range(n)] or [np.zeros(0)]).astype(np.int32)
    return rowp, succ
