"""Checks that pin the oracle to facts outside itself.

Each check returns None when it holds and raises AssertionError otherwise,
so the same checks run on the real oracle (tests/test_oracle.py) and on
copies of it with a planted mistake (they must then fail).
"""
from __future__ import annotations

import itertools
import os
from fractions import Fraction

import numpy as np

import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_r3():
    out = {}
    with open(os.path.join(GOLDEN, "r3_sum_of_three_squares.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            s, c = line.split()
            out[int(s)] = int(c)
    return out


def read_hand():
    out = {}
    with open(os.path.join(GOLDEN, "hand_line.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            key, *vals = line.split()
            out[key] = [int(v) for v in vals]
    return out


HAND_X = [0.0, 8.0, 4.0, 6.0, 2.0, 5.0]
HAND_Q = 5.25


def hand_points():
    P = np.zeros((6, 3), np.float32)
    P[:, 0] = HAND_X
    q = np.array([HAND_Q, 0.0, 0.0], np.float32)
    return P, q


# ---------------------------------------------------------------- knn pins

def pin_hand_example(knn_one):
    h = read_hand()
    P, q = hand_points()
    assert list(knn_one(P, q, 3, 6)[0]) == h["knn3"]
    assert list(knn_one(P, q, 6, 6)[0]) == h["knn6"]
    assert list(knn_one(P, q, 2, 4)[0]) == h["prefix4_knn2"]
    assert list(knn_one(P, q, 1, 2)[0]) == h["prefix2_knn1"]
    D = knn_one(P, q, 6, 6)[1]
    exact = sorted((HAND_Q - x) ** 2 for x in HAND_X)
    assert np.array_equal(D, np.array(exact))


def lattice_setup(L=16, seed=5):
    P_in, _ = W.lattice(L)
    order = W.permutation(P_in.shape[0], seed)
    P = P_in[order]                       # rank order
    rank_of = np.empty(P.shape[0], np.int64)
    rank_of[order] = np.arange(P.shape[0])
    return P, rank_of


def _lattice_rank(rank_of, L, x, y, z):
    return int(rank_of[int(x) + L * (int(y) + L * int(z))])


def pin_lattice_rings(knn_one, L=16, seed=5):
    """Integer-lattice query: k equal to a cumulative ring size returns
    exactly the rings, ranks ascending within each ring."""
    r3 = read_r3()
    P, rank_of = lattice_setup(L, seed)
    # the ring table itself, re-derived by enumerating offsets
    for s in range(13):
        cnt = sum(1 for a, b, c in itertools.product(range(-4, 5), repeat=3) if a * a + b * b + c * c == s)
        assert cnt == r3[s], (s, cnt, r3[s])
    cum = np.cumsum([r3[s] for s in range(13)])
    rng = np.random.default_rng(0)
    for _ in range(6):
        cx, cy, cz = rng.integers(5, L - 5, size=3)
        q = np.array([cx, cy, cz], np.float32)
        for k in (1, 7, 19, 27, 33):
            assert k in cum
            r, D = knn_one(P, q, k, P.shape[0])
            smax = int(np.searchsorted(cum, k))
            want = []
            for a, b, c in itertools.product(range(-4, 5), repeat=3):
                s = a * a + b * b + c * c
                if s <= smax:
                    want.append((float(s), _lattice_rank(rank_of, L, cx + a, cy + b, cz + c)))
            want.sort()
            assert len(want) == k
            assert [w[1] for w in want] == list(r), (k, want[:5], list(r)[:5])
            assert np.array_equal(D, np.array([w[0] for w in want]))


def pin_lattice_cell_centres(knn_one, L=16, seed=6):
    """Query at a cell centre (+0.5)^3: rings of half-integer offsets."""
    P, rank_of = lattice_setup(L, seed)
    cx, cy, cz = 7, 8, 6
    q = np.array([cx + 0.5, cy + 0.5, cz + 0.5], np.float32)
    rings = {}
    for a, b, c in itertools.product(range(-4, 4), repeat=3):
        s = (a + 0.5) ** 2 + (b + 0.5) ** 2 + (c + 0.5) ** 2
        rings.setdefault(s, []).append(_lattice_rank(rank_of, L, cx + a + 1, cy + b + 1, cz + c + 1))
    svals = sorted(rings)[:4]           # 0.75, 2.75, 4.75, 6.75
    assert [len(rings[s]) for s in svals[:3]] == [8, 24, 24]
    k = sum(len(rings[s]) for s in svals)
    r, D = knn_one(P, q, k, P.shape[0])
    want = sorted((s, rr) for s in svals for rr in rings[s])
    assert list(r) == [w[1] for w in want]
    assert np.array_equal(D, np.array([w[0] for w in want]))


def pin_sphere_centre(knn_one, n=2000):
    """Origin against points normalised onto the unit sphere: every squared
    distance is 1 up to float32 normalisation error, all ranks returned."""
    P, _ = W.sphere(n, seed=1)
    r, D = knn_one(P, np.zeros(3, np.float32), n, n)
    assert sorted(r.tolist()) == list(range(n))
    assert np.all(np.abs(D - 1.0) <= 1e-6)
    assert np.all(np.diff(D) >= 0)


def _exact_sq(P, q, r):
    p = [Fraction(float(v)) for v in P[r]]
    qq = [Fraction(float(v)) for v in q]
    return sum((a - b) ** 2 for a, b in zip(qq, p))


def pin_exact_rational(knn_one, trials=30, n=40, seed=9):
    """Tiny random inputs against exact rational distances: same ranks in
    the same order (no near-ties at this size), D within 1e-15 relative."""
    rng = np.random.default_rng(seed)
    for t in range(trials):
        P = rng.uniform(-1, 1, size=(n, 3)).astype(np.float32)
        q = rng.uniform(-1.5, 1.5, size=3).astype(np.float32)
        m = int(rng.integers(1, n + 1))
        k = int(rng.integers(1, n + 1))
        ex = sorted((_exact_sq(P, q, r), r) for r in range(m))[: min(k, m)]
        r, D = knn_one(P, q, k, m)
        assert list(r) == [e[1] for e in ex]
        for d, e in zip(D, ex):
            assert abs(Fraction(float(d)) - e[0]) <= Fraction(1, 10 ** 15) * e[0]


def pin_special_cases(knn_one):
    rng = np.random.default_rng(3)
    P = rng.uniform(-1, 1, size=(50, 3)).astype(np.float32)
    q = rng.uniform(-1, 1, size=3).astype(np.float32)
    # m = 1 -> rank 0
    r, _ = knn_one(P, q, 5, 1)
    assert list(r) == [0]
    # n = 1
    r, _ = knn_one(P[:1], q, 3, 1)
    assert list(r) == [0]
    # k >= m -> all m ranks
    r, _ = knn_one(P, q, 64, 20)
    assert sorted(r.tolist()) == list(range(20))
    # duplicates of an earlier site tie with it; the lower rank comes first
    P2 = P.copy()
    P2[30] = P2[4]
    P2[31] = P2[4]
    q2 = (P2[4] + np.float32(1e-3)).astype(np.float32)
    r, _ = knn_one(P2, q2, 3, 50)
    assert list(r) == [4, 30, 31]


# ---------------------------------------------------------- keys_upto pins

def pin_upto_hand_example(keys_upto):
    """The hand example: dmax exactly on a site's distance includes it, a
    prefix bound m drops later ranks, keys come out ascending."""
    h = read_hand()
    P, q = hand_points()
    for key, vals in h.items():
        if not key.startswith("upto_"):
            continue
        _, ms, ds = key.split("_")
        r, D = keys_upto(P, q, int(ms[1:]), float(ds[1:]))
        assert list(r) == vals, (key, list(r), vals)
        assert np.array_equal(D, np.array([(HAND_Q - HAND_X[v]) ** 2 for v in vals]))


def pin_upto_lattice_ring(keys_upto, L=16, seed=5):
    """Integer lattice, dmax exactly on a ring value: every lattice point of
    squared distance <= s among ranks < m, enumerated from offsets, ordered
    by (distance, rank); m is chosen to cut the outer ring."""
    P, rank_of = lattice_setup(L, seed)
    n = P.shape[0]
    cx, cy, cz = 8, 7, 9
    q = np.array([cx, cy, cz], np.float32)
    for s in (0, 1, 2, 3, 5):
        ring = []
        for a, b, c in itertools.product(range(-3, 4), repeat=3):
            d = a * a + b * b + c * c
            if d <= s:
                ring.append((float(d), _lattice_rank(rank_of, L, cx + a, cy + b, cz + c)))
        outer = sorted(r for d, r in ring if d == s)
        cut = outer[len(outer) // 2] if len(outer) > 1 else n   # drops the later half of ring s
        for m in (n, cut):
            want = sorted((d, r) for d, r in ring if r < m)
            r, D = keys_upto(P, q, m, float(s))
            assert list(r) == [w[1] for w in want], (s, m)
            assert np.array_equal(D, np.array([w[0] for w in want]))
            if m == cut and len(outer) > 1:
                assert len(want) < len(ring)


ALL_UPTO_PINS = [pin_upto_hand_example, pin_upto_lattice_ring]


ALL_KNN_PINS = [pin_hand_example, pin_lattice_rings, pin_lattice_cell_centres,
                pin_sphere_centre, pin_exact_rational, pin_special_cases]


def run_knn_pins(knn_one):
    for pin in ALL_KNN_PINS:
        pin(knn_one)
