"""The oracle against facts that do not come from the oracle (CPU only)."""
from __future__ import annotations

import itertools
from fractions import Fraction

import numpy as np
import pytest

import oracle.dpknn as dp
import oracle.knn as ok
import oracle.successors as osucc
import workloads as W
from tests import oracle_pins as pins


# --------------------------------------------------------------- brute force

@pytest.mark.parametrize("pin", pins.ALL_KNN_PINS, ids=lambda f: f.__name__)
def test_knn_pins(pin):
    pin(ok.knn_one)


def test_knn_batch_matches_one():
    wl = W.small_sphere(nq=50)
    P = wl.ranked_points()
    idx, d2, D = ok.knn(P, wl.queries, 8, 0)
    for i in range(50):
        r, Di = ok.knn_one(P, wl.queries[i], 8, P.shape[0])
        assert list(idx[i]) == list(r)
        assert np.array_equal(D[i], Di)
    m = np.full(50, 3, np.int32)
    idx, d2, D = ok.knn(P, wl.queries, 8, m)
    assert np.all(idx[:, 3:] == -1) and np.all(np.isinf(d2[:, 3:]))


# A plausible mistake planted in a copy of the oracle must fail a pin.

def _planted(kind):
    def sq(P, q):
        P64 = np.asarray(P, np.float32).astype(np.float64)
        q64 = np.asarray(q, np.float32).astype(np.float64)
        dx, dy, dz = q64[0] - P64[:, 0], q64[1] - P64[:, 1], q64[2] - P64[:, 2]
        if kind == "dropped_z":
            return dx * dx + dy * dy
        if kind == "wrong_axis":
            return (dx * dx + dy * dy) + dy * dy
        if kind == "sign":
            return (dx * dx + dy * dy) - dz * dz
        return (dx * dx + dy * dy) + dz * dz

    def knn_one(P, q, k, m):
        m_eff = m + 1 if kind == "prefix_off_by_one" and m < P.shape[0] else m
        kk = min(k, m_eff)
        if kind == "k_minus_one":
            kk = max(1, kk - 1) if kk > 1 else kk
        D = sq(P[:m_eff], q)
        r = np.arange(m_eff)
        if kind == "tie_high_rank_first":
            order = np.lexsort((-r, D))[:kk]
        elif kind == "float32_keys":
            order = np.lexsort((r, D.astype(np.float32)))[:kk]
        else:
            order = np.lexsort((r, D))[:kk]
        return r[order].astype(np.int64), D[order]
    return knn_one


@pytest.mark.parametrize("kind", ["dropped_z", "wrong_axis", "sign", "prefix_off_by_one",
                                  "k_minus_one", "tie_high_rank_first"])
def test_planted_mistakes_fail_a_pin(kind):
    bad = _planted(kind)
    failed = []
    for pin in pins.ALL_KNN_PINS:
        try:
            pin(bad)
        except AssertionError:
            failed.append(pin.__name__)
    assert failed, f"planted mistake {kind} passed every pin"


def test_unplanted_copy_passes():
    pins.run_knn_pins(_planted("none"))


# ------------------------------------------------------- Algorithms 1 and 2

def _random_cloud(n, seed, kind="cube"):
    if kind == "cube":
        P, _ = W.uniform_cube(n, seed)
    else:
        P, _ = W.surface(kind, n, seed)
    return P[W.permutation(n, seed + 1)]


def test_hand_example_descent():
    h = pins.read_hand()
    P, q = pins.hand_points()
    rowp, succ = dp.complete_table(6)
    assert [s for _, s in dp.descent(P, rowp, succ, q, 6)] == h["transitions"]
    assert [s for _, s in dp.descent(P, rowp, succ, q, 4)] == h["prefix4_transitions"]
    assert dp.strict_prefix_minima(P, q, 6) == h["transitions"]
    r, _ = dp.knn_dp(P, rowp, succ, q, 3)
    assert list(r) == h["knn3"]


@pytest.mark.parametrize("n,seed,kind", [(30, 1, "cube"), (40, 2, "sphere"), (35, 3, "torus")])
def test_descent_is_prefix_minima_complete_table(n, seed, kind):
    P = _random_cloud(n, seed, kind)
    rowp, succ = dp.complete_table(n)
    Q = W.box_queries(40, seed + 7, [-1.5] * 3, [1.5] * 3)
    for q in Q:
        for m in (1, 2, n // 3, n):
            got = [s for _, s in dp.descent(P, rowp, succ, q, m)]
            assert got == dp.strict_prefix_minima(P, q, m)


@pytest.mark.parametrize("n,seed", [(24, 11), (40, 12)])
def test_dp_knn_equals_bruteforce_complete_table(n, seed):
    P = _random_cloud(n, seed)
    rowp, succ = dp.complete_table(n)
    Q = W.box_queries(25, seed, [-1.5] * 3, [1.5] * 3)
    for q in Q:
        for m in (1, 5, n):
            for k in range(1, n + 1, 3):
                r, D = dp.knn_dp(P, rowp, succ, q, k, m)
                rb, Db = ok.knn_one(P, q, k, m)
                assert list(r) == list(rb)
                assert np.array_equal(D, Db)


@pytest.mark.parametrize("n,seed", [(120, 21), (200, 22)])
def test_dp_knn_equals_bruteforce_definition_table(n, seed):
    P = _random_cloud(n, seed)
    L = osucc.successor_lists(P)
    rowp, succ = osucc.to_csr(L)
    Q = W.box_queries(60, seed, [-1.5] * 3, [1.5] * 3)
    for q in Q:
        assert [s for _, s in dp.descent(P, rowp, succ, q, n)] == dp.strict_prefix_minima(P, q, n)
        for m in (7, n // 2, n):
            for k in (1, 2, 5, 16, 33):
                r, D = dp.knn_dp(P, rowp, succ, q, k, m)
                rb, Db = ok.knn_one(P, q, k, m)
                assert list(r) == list(rb), (k, m)


def test_dp_counters_monotone_in_k():
    P = _random_cloud(150, 31)
    rowp, succ = osucc.to_csr(osucc.successor_lists(P))
    q = np.array([0.1, -0.2, 0.3], np.float32)
    prev = (0, 0, 0)
    for k in (1, 2, 4, 8, 16):
        c = dp.Counters()
        dp.knn_dp(P, rowp, succ, q, k, 0, c)
        assert c.as_tuple() >= prev
        prev = c.as_tuple()
    c = dp.Counters()
    dp.knn_dp(P, rowp, succ, q, 1, 0, c)
    # k = 1 is the descent alone: rows = transitions, coords = 1 + entries read below m
    assert c.rows == len(dp.descent(P, rowp, succ, q, 150))


def test_dp_knn_lattice_rings_complete_table():
    """Maximally degenerate input (every cube's corners are cospherical) on
    a table that does not depend on any triangulation."""
    P, rank_of = pins.lattice_setup(L=5, seed=8)
    rowp, succ = dp.complete_table(P.shape[0])
    q = np.array([2, 2, 2], np.float32)
    for k in (1, 7, 19, 27, 33):
        r, D = dp.knn_dp(P, rowp, succ, q, k)
        rb, Db = ok.knn_one(P, q, k, P.shape[0])
        assert list(r) == list(rb)


# ------------------------------------------------------- successor lists

def _exact_insphere_inside(a, b, c, d, e):
    """True iff e is strictly inside the sphere through a, b, c, d (exact)."""
    rows = []
    for p in (a, b, c, d):
        v = [Fraction(float(p[i])) - Fraction(float(e[i])) for i in range(3)]
        rows.append(v + [v[0] ** 2 + v[1] ** 2 + v[2] ** 2])

    def det3(m):
        return (m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1])
                - m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0])
                + m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]))

    def det4(m):
        s = 0
        for j in range(4):
            minor = [r[:j] + r[j + 1:] for r in m[1:]]
            s += (-1) ** j * m[0][j] * det3(minor)
        return s

    o = det3([[Fraction(float(p[i])) - Fraction(float(a[i])) for i in range(3)] for p in (b, c, d)])
    return o != 0 and (det4(rows) * (1 if o > 0 else -1)) < 0


@pytest.mark.parametrize("seed", [41, 42])
def test_successor_definition_against_empty_spheres(seed):
    """Library-triangulation successor lists equal the empty-sphere
    enumeration over all tetrahedra of each prefix (exact arithmetic)."""
    n = 9
    P = _random_cloud(n, seed)
    L = osucc.successor_lists(P)
    for j in range(4, n):
        nb = set()
        pts = list(range(j))
        for a, b, c in itertools.combinations(pts, 3):
            tet = (a, b, c, j)
            vol = np.linalg.det(np.array([P[b] - P[a], P[c] - P[a], P[j] - P[a]], np.float64))
            if vol == 0:
                continue
            if not any(_exact_insphere_inside(P[a], P[b], P[c], P[j], P[o])
                       for o in range(j + 1) if o not in tet):
                nb.update((a, b, c))
        got = {i for i in range(j) if j in L[i]}
        assert got == nb, (j, sorted(got), sorted(nb))


# ------------------------------------------------------- keys_upto

@pytest.mark.parametrize("pin", pins.ALL_UPTO_PINS, ids=lambda f: f.__name__)
def test_keys_upto_pins(pin):
    pin(ok.keys_upto)


def _planted_upto(kind):
    def keys_upto(P, q, m, dmax):
        mm = P.shape[0] if kind == "ignores_m" else int(m)
        D = ok.sq_dist64(P[:mm], q)
        cand = np.nonzero(D < dmax)[0] if kind == "strict" else np.nonzero(D <= dmax)[0]
        if kind == "rank_order":
            order = np.argsort(cand, kind="stable")
        elif kind == "tie_high_rank_first":
            order = np.lexsort((-cand, D[cand]))
        else:
            order = np.lexsort((cand, D[cand]))
        r = cand[order]
        return r.astype(np.int64), D[r]
    return keys_upto


@pytest.mark.parametrize("kind", ["strict", "ignores_m", "rank_order", "tie_high_rank_first"])
def test_keys_upto_planted_mistakes_fail_a_pin(kind):
    bad = _planted_upto(kind)
    failed = []
    for pin in pins.ALL_UPTO_PINS:
        try:
            pin(bad)
        except AssertionError:
            failed.append(pin.__name__)
    assert failed, f"planted mistake {kind} passed every keys_upto pin"


def test_keys_upto_unplanted_copy_passes():
    for pin in pins.ALL_UPTO_PINS:
        pin(_planted_upto("none"))
