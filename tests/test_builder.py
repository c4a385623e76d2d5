"""Host builder and exact predicates (CPU only; the library is loaded, no
GPU call is made)."""
from __future__ import annotations

import os
import re
from fractions import Fraction

import numpy as np
import pytest

import oracle.dpknn as dp
import oracle.knn as ok
import oracle.successors as osucc
import workloads as W
from paper_2605_02224_gb300 import mknn as M

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


# ------------------------------------------------------------- the library

def test_library_exports_every_declared_symbol():
    hdr = open(os.path.join(ROOT, "include", "mknn.h")).read()
    names = set(re.findall(r"\b(mknn_[a-z0-9_]+)\s*\(", hdr))
    assert len(names) > 20
    lib = M.lib()
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


# ------------------------------------------------------------- predicates

def _frac(p):
    return [Fraction(float(v)) for v in p]


def _orient_exact(a, b, c, d):
    a, b, c, d = map(_frac, (a, b, c, d))
    u = [b[i] - a[i] for i in range(3)]
    v = [c[i] - a[i] for i in range(3)]
    w = [d[i] - a[i] for i in range(3)]
    det = (u[0] * (v[1] * w[2] - v[2] * w[1]) - u[1] * (v[0] * w[2] - v[2] * w[0])
           + u[2] * (v[0] * w[1] - v[1] * w[0]))
    return (det > 0) - (det < 0)


def _insphere_exact(a, b, c, d, e):
    """+1 inside for positive orientation, from the circumcentre (exact)."""
    A, B, Cc, D, E = map(_frac, (a, b, c, d, e))
    # solve for the centre x: 2 (p - A) . x = |p|^2 - |A|^2 for p in B, C, D
    rows = []
    for p in (B, Cc, D):
        rows.append([2 * (p[i] - A[i]) for i in range(3)]
                    + [sum(p[i] ** 2 - A[i] ** 2 for i in range(3))])
    # Cramer's rule
    def det3(m):
        return (m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1])
                - m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0])
                + m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]))
    M3 = [r[:3] for r in rows]
    dd = det3(M3)
    assert dd != 0
    x = []
    for j in range(3):
        mj = [r[:3] for r in rows]
        for i in range(3):
            mj[i][j] = rows[i][3]
        x.append(det3(mj) / dd)
    r2 = sum((A[i] - x[i]) ** 2 for i in range(3))
    e2 = sum((E[i] - x[i]) ** 2 for i in range(3))
    s = (e2 < r2) - (e2 > r2)
    return s * _orient_exact(a, b, c, d)


def _random_cases(rng, count):
    out = []
    for _ in range(count):
        kind = rng.integers(0, 4)
        if kind == 0:       # generic
            pts = rng.uniform(-1, 1, size=(5, 3))
        elif kind == 1:     # near-cospherical: on a sphere plus tiny noise
            d = rng.normal(size=(5, 3))
            pts = d / np.linalg.norm(d, axis=1, keepdims=True) * 0.7 + 0.1
            pts += rng.normal(scale=1e-7, size=pts.shape)
        elif kind == 2:     # integer lattice (exact degeneracies)
            pts = rng.integers(-3, 4, size=(5, 3)).astype(np.float64)
        else:               # near-coplanar
            pts = rng.uniform(-1, 1, size=(5, 3))
            pts[:, 2] = 0.3 * pts[:, 0] - 0.2 * pts[:, 1] + rng.normal(scale=1e-8, size=5)
        out.append(pts.astype(np.float32))
    return out


def test_orient3d_matches_exact_rationals():
    rng = np.random.default_rng(1)
    for pts in _random_cases(rng, 600):
        want = _orient_exact(*pts[:4])
        assert M.mknn_orient3d(*pts[:4]) == want
        assert M.mknn_orient3d(*pts[:4], exact=True) == want


def test_insphere_matches_exact_rationals():
    rng = np.random.default_rng(2)
    checked = 0
    for pts in _random_cases(rng, 800):
        if _orient_exact(*pts[:4]) == 0:
            continue
        want = _insphere_exact(*pts)
        assert M.mknn_insphere(*pts) == want
        assert M.mknn_insphere(*pts, exact=True) == want
        checked += 1
    assert checked > 500


def test_insphere_degenerate_zero_and_sign_flip():
    a, b, c, d = ([0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1])
    assert M.mknn_orient3d(a, b, c, d) == 1
    assert M.mknn_insphere(a, b, c, d, [1, 1, 1]) == 0          # cube corner: cospherical
    assert M.mknn_insphere(a, b, c, d, [0.25, 0.25, 0.25]) == 1
    assert M.mknn_insphere(a, b, c, d, [2, 2, 2]) == -1
    assert M.mknn_insphere(b, a, c, d, [0.25, 0.25, 0.25]) == -1  # negative orientation flips


def test_predicates_extreme_exponents():
    tiny = np.float32(1e-30)
    big = np.float32(1e30)
    a = np.array([0, 0, 0], np.float32)
    b = np.array([big, 0, 0], np.float32)
    c = np.array([0, tiny, 0], np.float32)
    d = np.array([0, 0, tiny], np.float32)
    assert M.mknn_orient3d(a, b, c, d) == _orient_exact(a, b, c, d)
    e = np.array([tiny, tiny, tiny], np.float32)
    assert M.mknn_insphere(a, b, c, d, e) == _insphere_exact(a, b, c, d, e)


# ------------------------------------------------------------- builder

@pytest.mark.parametrize("n,seed", [(60, 1), (150, 2), (300, 3), (400, 4)])
def test_successor_lists_equal_definition(n, seed):
    P, _ = W.uniform_cube(n, seed)
    order = W.permutation(n, seed + 1)
    h = M.mknn_build(P, order)
    try:
        xyz, rowp, succ = M.mknn_cloud_table(h)
        assert np.array_equal(xyz, P[order])
        L = osucc.successor_lists(P[order])
        r2, s2 = osucc.to_csr(L)
        assert np.array_equal(rowp, r2)
        assert np.array_equal(succ, s2)
        assert np.array_equal(M.mknn_cloud_order(h), order)
    finally:
        M.mknn_cloud_free(h)


def _table_checks(h, n):
    xyz, rowp, succ = M.mknn_cloud_table(h)
    assert rowp[0] == 0 and rowp[-1] == succ.size
    for i in range(n):
        row = succ[rowp[i]:rowp[i + 1]]
        assert np.all(np.diff(row) > 0) and (row.size == 0 or (row[0] > i and row[-1] < n))
    return xyz, rowp, succ


def _degenerate_inputs():
    P, _ = W.lattice(6)                        # 216 points, every cube cospherical
    yield "lattice6", P, W.permutation(P.shape[0], 3)
    P, _ = W.sphere(400, 9)                    # every point on the hull
    yield "sphere400", P, W.permutation(400, 10)
    P, _ = W.patches4(400, 11)                 # four near-planar patches
    yield "patches400", P, W.permutation(400, 12)
    P, _ = W.uniform_cube(300, 13)
    P = P.copy()
    P[100:140] = P[0:40]                       # exact duplicates of earlier points
    yield "duplicates", P, W.permutation(300, 14)
    P, _ = W.lattice(5)
    P = P.copy()
    P[:, 2] = 0.0                              # many coplanar points, then off-plane
    P[-3:, 2] = [1.0, 2.0, 3.0]
    yield "mostly_coplanar", P, np.arange(P.shape[0])


@pytest.mark.parametrize("name,P,order", list(_degenerate_inputs()), ids=lambda x: x if isinstance(x, str) else "")
def test_degenerate_inputs_give_valid_delaunay_and_exact_queries(name, P, order):
    n = P.shape[0]
    h = M.mknn_build(P, order, keep_tets=True)
    try:
        xyz, rowp, succ = _table_checks(h, n)
        bad_o, bad_s = M.mknn_cloud_validate(h)
        assert bad_o == 0 and bad_s == 0, (bad_o, bad_s)
        st = M.mknn_cloud_stats(h)
        if name == "duplicates":
            assert st["duplicates"] >= 1
        Pr = P[order]
        rng = np.random.default_rng(5)
        lo, hi = Pr.min(0) - 0.5, Pr.max(0) + 0.5
        Q = rng.uniform(lo, hi, size=(40, 3)).astype(np.float32)
        Q = np.concatenate([Q, Pr[rng.integers(0, n, 10)]])   # queries on sites
        for q in Q:
            assert [s for _, s in dp.descent(Pr, rowp, succ, q, n)] == dp.strict_prefix_minima(Pr, q, n)
            for k, m in ((1, n), (8, n), (27, n), (8, n // 3)):
                r, _ = dp.knn_dp(Pr, rowp, succ, q, k, m)
                rb, _ = ok.knn_one(Pr, q, k, m)
                assert list(r) == list(rb), (name, k, m)
    finally:
        M.mknn_cloud_free(h)


def test_all_coplanar_small_gives_complete_table_large_is_rejected():
    rng = np.random.default_rng(7)
    P = rng.uniform(-1, 1, size=(50, 3)).astype(np.float32)
    P[:, 2] = 0.5
    h = M.mknn_build(P)
    _, rowp, succ = M.mknn_cloud_table(h)
    assert succ.size == 50 * 49 // 2
    M.mknn_cloud_free(h)
    P = rng.uniform(-1, 1, size=(5000, 3)).astype(np.float32)
    P[:, 2] = 0.5
    with pytest.raises(M.MknnError) as ei:
        M.mknn_build(P)
    assert ei.value.status == 6


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_tiny_clouds(n):
    P, _ = W.uniform_cube(n, 17)
    h = M.mknn_build(P)
    _, rowp, succ = _table_checks(h, n)
    assert succ.size == n * (n - 1) // 2 or n == 5
    M.mknn_cloud_free(h)


def test_bad_inputs_are_rejected():
    P, _ = W.uniform_cube(20, 1)
    bad = P.copy()
    bad[3, 1] = np.nan
    with pytest.raises(M.MknnError) as ei:
        M.mknn_build(bad)
    assert ei.value.status == 1
    with pytest.raises(M.MknnError):
        M.mknn_build(P, np.zeros(20, np.int64))
    with pytest.raises(M.MknnError):
        M.mknn_cloud_from_table(P, np.zeros(21, np.int64) + 1, np.zeros(0, np.int32))
    rowp = np.array([0, 1] + [1] * 19, np.int64)
    with pytest.raises(M.MknnError):   # entry not greater than its row
        M.mknn_cloud_from_table(P, rowp, np.array([0], np.int32))


def test_save_load_roundtrip(tmp_path):
    P, _ = W.torus(2000, 3)
    order = W.permutation(2000, 4)
    h = M.mknn_build(P, order)
    path = str(tmp_path / "c.mknn")
    M.mknn_cloud_save(h, path)
    h2 = M.mknn_cloud_load(path)
    for a, b in zip(M.mknn_cloud_table(h), M.mknn_cloud_table(h2)):
        assert np.array_equal(a, b)
    assert np.array_equal(M.mknn_cloud_order(h), M.mknn_cloud_order(h2))
    with open(path, "r+b") as f:
        f.truncate(100)
    with pytest.raises(M.MknnError) as ei:
        M.mknn_cloud_load(path)
    assert ei.value.status == 7
    M.mknn_cloud_free(h)
    M.mknn_cloud_free(h2)


def test_sphere_small_workload_queries_exact():
    """The 2,000-point sphere with its own seeds: Alg. 1 + 2 on the built
    table equal brute force for a sample of the workload's queries."""
    wl = W.small_sphere(nq=300)
    h = M.mknn_build(wl.points, wl.order)
    _, rowp, succ = M.mknn_cloud_table(h)
    Pr = wl.ranked_points()
    for q in wl.queries:
        r, _ = dp.knn_dp(Pr, rowp, succ, q, wl.k)
        rb, _ = ok.knn_one(Pr, q, wl.k, Pr.shape[0])
        assert list(r) == list(rb)
    M.mknn_cloud_free(h)


# ------------------------------------------------------------- appends

def _ranked(P, order):
    return np.ascontiguousarray(P[order], np.float32)


@pytest.mark.parametrize("kind,n,n0", [("sphere", 3000, 500), ("patches", 2500, 40),
                                       ("torus", 4000, 3999)])
def test_appends_equal_one_build(kind, n, n0):
    """Build the first n0 ranks with the dynamic option, append the rest in
    chunks of 1, 7, 100 and the remainder: the table equals one build over
    all the points in the same order, entry for entry."""
    from paper_2605_02224_gb300 import Cloud
    P, _ = W.surface(kind, n, 71)
    Pr = _ranked(P, W.permutation(n, 72))
    ref = Cloud.build(Pr)
    c = Cloud.build(Pr[:n0], dynamic=True)
    at = n0
    for step in (1, 7, 100, n):
        if at >= n:
            break
        c.append(Pr[at:at + step])
        at = min(n, at + step)
    x1, r1, s1 = c.table()
    x2, r2, s2 = ref.table()
    assert np.array_equal(x1, x2) and np.array_equal(r1, r2) and np.array_equal(s1, s2)
    assert np.array_equal(c.order(), np.arange(n))
    st = c.stats()
    assert st["n"] == n and st["entries"] == s2.size
    c.close()
    ref.close()


def test_appends_with_duplicates_match_the_definition():
    """Appended points that repeat earlier ones (and each other): the table
    equals one build, and every row holds the definition's list (Delaunay
    neighbours at insertion, computed by the oracle)."""
    from paper_2605_02224_gb300 import Cloud
    P, _ = W.uniform_cube(60, 81)
    extra = np.concatenate([P[:5], P[:2], W.uniform_cube(20, 82)[0]]).astype(np.float32)
    allp = np.concatenate([P, extra]).astype(np.float32)
    c = Cloud.build(P, dynamic=True)
    c.append(extra[:3])
    c.append(extra[3:])
    ref = Cloud.build(allp)
    t1, t2 = c.table(), ref.table()
    assert all(np.array_equal(a, b) for a, b in zip(t1, t2))
    rowp, succ = t1[1], t1[2]
    # coincident points: either twin may stand for both in the library's
    # triangulation, so read its neighbours through the earlier twin
    first = {}
    twin = [first.setdefault(tuple(p), r) for r, p in enumerate(allp.tolist())]
    defn = osucc.successor_lists(allp)
    for i, lst in enumerate(defn):
        row = set(succ[rowp[twin[i]]:rowp[twin[i] + 1]].tolist())
        assert set(lst) <= row, i
    c.close()
    ref.close()


def test_append_errors_leave_the_cloud_unchanged():
    from paper_2605_02224_gb300 import Cloud
    P, _ = W.sphere(500, 91)
    static = Cloud.build(P)
    with pytest.raises(M.MknnError) as ei:
        static.append(P[:3])
    assert ei.value.status == 1                        # EINVAL: not dynamic
    with pytest.raises(M.MknnError):
        static.compact()
    c = Cloud.build(P, dynamic=True)
    bad = np.array([[0.1, 0.2, np.nan]], np.float32)
    with pytest.raises(M.MknnError):
        c.append(bad)
    assert M.mknn_cloud_info(c.handle)[0] == 500
    c.append(np.zeros((0, 3), np.float32))              # nothing to do
    assert M.mknn_cloud_info(c.handle)[0] == 500
    flat = np.stack([W.uniform(92, 1, 50), W.uniform(92, 2, 50),
                     np.zeros(50)], 1).astype(np.float32)
    with pytest.raises(M.MknnError) as ei:
        Cloud.build(flat, dynamic=True)
    assert ei.value.status == 6                        # EDEGENERATE: coplanar
    static.close()
    c.close()
