"""Element-by-element comparison of query results with the oracle.

Rule (float32 path against the float64 definition):
  * squared distances: |d_gpu - D(idx_gpu)| <= 1e-6 * D, or both 0, where D
    is the oracle's float64 distance of the returned rank;
  * returned ranks are distinct and in [0, m); positions past min(k, m)
    hold (-1, +inf);
  * the sorted float64 distances of the returned ranks equal the oracle's
    k smallest within 1e-6 relative;
  * ranks are identical position by position, except inside groups of
    consecutive oracle positions whose distances differ by less than 1e-6
    relative ("near-ties"): there the sets must match, and a group that
    reaches past the k-th position (its distance within 1e-6 of the
    (k+1)-th) may hold any members of the full group;
  * equal float32 distances in a returned row appear in ascending rank
    (the tie rule of Eq. 2 in the path's own arithmetic).
"""
from __future__ import annotations

import numpy as np

import oracle.knn as ok

REL = 1e-6


def _rel_close(a, b):
    return np.abs(a - b) <= REL * np.maximum(np.abs(a), np.abs(b))


def check_query(P, q, k, m, gi, gd, where=""):
    """Raises AssertionError with a description if the row (gi, gd) breaks
    the rule for query q with prefix m. Returns the number of near-tie
    positions (for reporting)."""
    m = int(m)
    kk = min(k, m)
    gi = np.asarray(gi)
    gd = np.asarray(gd, dtype=np.float32)
    assert np.all(gi[kk:] == -1) and np.all(np.isinf(gd[kk:])), f"{where}: padding {gi} {gd}"
    g = gi[:kk].astype(np.int64)
    assert np.all((g >= 0) & (g < m)), f"{where}: rank out of [0,{m}): {g}"
    assert np.unique(g).size == kk, f"{where}: repeated rank {g}"
    Dg = ok.sq_dist64(P[g], q)
    dg = gd[:kk].astype(np.float64)
    ok_d = (np.abs(dg - Dg) <= REL * Dg) | ((dg == 0) & (Dg == 0))
    assert np.all(ok_d), f"{where}: distance mismatch {dg[~ok_d]} vs {Dg[~ok_d]}"
    # equal float32 distances -> ascending ranks
    same = gd[:kk][1:] == gd[:kk][:-1]
    assert np.all(~same | (g[1:] > g[:-1])), f"{where}: tie order {g} {gd}"
    # oracle, with one extra to see the boundary
    r_or, D_or = ok.knn_one(P, q, kk + 1, m)
    D_next = D_or[kk] if r_or.size > kk else None
    r_or, D_or = r_or[:kk], D_or[:kk]
    assert np.all(_rel_close(np.sort(Dg), D_or) | ((np.sort(Dg) == 0) & (D_or == 0))), \
        f"{where}: distance multiset {np.sort(Dg)} vs {D_or}"
    # near-tie runs over oracle positions
    link = np.zeros(kk, dtype=bool)          # link[p]: p and p+1 near-tied
    if kk > 1:
        link[:-1] = _rel_close(D_or[1:], D_or[:-1])
    boundary_tie = D_next is not None and bool(_rel_close(np.array([D_next]), D_or[-1:])[0])
    ties = 0
    p = 0
    while p < kk:
        e = p
        while e < kk - 1 and link[e]:
            e += 1
        run = slice(p, e + 1)
        at_boundary = (e == kk - 1) and boundary_tie
        if e == p and not at_boundary:
            assert g[p] == r_or[p], f"{where}: position {p}: {g} vs oracle {r_or}"
        elif not at_boundary:
            ties += e - p + 1
            assert set(g[run]) == set(r_or[run]), f"{where}: tie group {p}..{e}: {g} vs {r_or}"
        else:
            ties += e - p + 1
            dmax = D_or[p] * (1 + 4 * REL) + 1e-300
            allowed, _ = ok.keys_upto(P, q, m, dmax)
            assert set(g[run]) <= set(allowed.tolist()), f"{where}: boundary group {g[run]}"
        p = e + 1
    return ties


def check_rows(P, Q, k, m, idx, d2, rows=None):
    """Checks the given query rows (all if rows is None). m: scalar or array."""
    nq = Q.shape[0]
    rows = range(nq) if rows is None else rows
    ties = 0
    for i in rows:
        mi = (m[i] if np.ndim(m) else (m or P.shape[0]))
        ties += check_query(P, Q[i], k, mi, idx[i], d2[i], where=f"query {i}")
    return ties


def check_row_properties(idx, d2, k, m_vec, n):
    """Size-independent properties of every row (for full-size runs):
    sorted by (d, rank), valid distinct ranks, padding exactly past min(k, m)."""
    idx = np.asarray(idx)
    d2 = np.asarray(d2)
    kk = np.minimum(k, m_vec)
    pos = np.arange(k)[None, :]
    real = pos < kk[:, None]
    assert np.all((idx >= 0) == real), "padding layout"
    assert np.all(np.isinf(d2[~real])), "padding distances"
    assert np.all(idx < np.where(real, m_vec[:, None], 1)), "rank >= m"
    dd = np.where(real, d2, np.inf)
    assert np.all(np.diff(dd, axis=1)[real[:, 1:]] >= 0), "rows not sorted by distance"
    srt = np.sort(np.where(real, idx, -1 - pos), axis=1)
    assert np.all(np.diff(srt, axis=1) != 0), "repeated rank in a row"
