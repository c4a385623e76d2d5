"""The CPU baselines (kd-tree with prefix support, Algorithms 1-2 on the
host) against the oracle: both compute the exact k-NN definition in
float64, so ranks and float32 distances must be identical."""
from __future__ import annotations

import numpy as np
import pytest

import cpu
import oracle.dpknn as dp
import oracle.knn as ok
import oracle.successors as osucc
import workloads as W
from tests import oracle_pins as pins


@pytest.fixture(scope="module", autouse=True)
def built():
    cpu.build()


def _oracle(P, Q, k, m):
    idx, d2, _ = ok.knn(P, Q, k, m)
    return idx, d2


@pytest.mark.parametrize("n,seed,kind", [(40, 1, "cube"), (300, 2, "sphere"), (1000, 3, "torus")])
def test_kdtree_equals_oracle(n, seed, kind):
    P, _ = (W.uniform_cube(n, seed) if kind == "cube" else W.surface(kind, n, seed))
    P = P[W.permutation(n, seed + 1)]
    Q = W.box_queries(80, seed + 2, [-1.6] * 3, [1.6] * 3)
    t = cpu.KDTree(P, leaf=4)
    for k in (1, 3, 8, 16, 33):
        for m in (0, 1, 7, n // 2):
            gi, gd = t.knn(Q, k, m)
            ri, rd = _oracle(P, Q, k, m)
            assert np.array_equal(gi, ri), (k, m)
            assert np.array_equal(gd, rd), (k, m)
    mq = (1 + (W.rand_u64(seed, 9, 80) % np.uint64(n))).astype(np.int32)
    gi, gd = t.knn(Q, 5, mq)
    ri, rd = _oracle(P, Q, 5, mq)
    assert np.array_equal(gi, ri) and np.array_equal(gd, rd)
    t.close()


def test_kdtree_lattice_rings_and_sphere_centre():
    """Maximal ties: lattice rings come out whole, in rank order, and the
    sphere's centre returns every point at distance ~1."""
    P, rank_of = pins.lattice_setup(L=12, seed=5)
    t = cpu.KDTree(P, leaf=8)
    q = np.array([[6, 5, 6]], np.float32)
    for k in (1, 7, 19, 27, 33):
        gi, gd = t.knn(q, k)
        ri, rd = _oracle(P, q, k, 0)
        assert np.array_equal(gi, ri) and np.array_equal(gd, rd)
    S, _ = W.sphere(2000, seed=1)
    t2 = cpu.KDTree(S)
    gi, gd = t2.knn(np.zeros((1, 3), np.float32), 128)
    ri, rd = _oracle(S, np.zeros((1, 3), np.float32), 128, 0)
    assert np.array_equal(gi, ri) and np.all(np.abs(gd - 1) <= 1e-6)


def test_kdtree_threads_agree():
    P, _ = W.surface("bumpy", 5000, 11)
    Q = W.box_queries(3000, 12, [-1.3] * 3, [1.3] * 3)
    t = cpu.KDTree(P)
    a = t.knn(Q, 10, threads=1, sort=False)
    b = t.knn(Q, 10, threads=0, sort=True)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("n,seed", [(150, 21), (250, 22)])
def test_dpknn_equals_oracle_on_definition_table(n, seed):
    P, _ = W.uniform_cube(n, seed)
    P = P[W.permutation(n, seed + 1)]
    rowp, succ = osucc.to_csr(osucc.successor_lists(P))
    Q = W.box_queries(60, seed, [-1.5] * 3, [1.5] * 3)
    for k in (1, 2, 5, 16, 33):
        for m in (0, 7, n // 2):
            gi, gd, cnt = cpu.dpknn(P, rowp, succ, Q, k, m, counters=True)
            ri, rd = _oracle(P, Q, k, m)
            assert np.array_equal(gi, ri) and np.array_equal(gd, rd), (k, m)
            # rows, entries and coordinates read equal the step-by-step oracle
            for i in range(0, 60, 7):
                c = dp.Counters()
                dp.knn_dp(P, rowp, succ, Q[i], k, m, c)
                assert tuple(cnt[i, :3]) == c.as_tuple()


def test_dpknn_on_built_tables_and_prefix_vectors():
    from paper_2605_02224_gb300 import Cloud
    for kind, n, seed in (("torus", 3000, 31), ("patches", 3000, 32)):
        P, _ = W.surface(kind, n, seed)
        order = W.permutation(n, seed + 1)
        c = Cloud.build(P, order)
        Pr, rowp, succ = c.table()
        lo, hi = W.padded_box(P)
        Q = W.box_queries(400, seed + 2, lo, hi)
        mq = (1 + (W.rand_u64(seed, 3, 400) % np.uint64(n))).astype(np.int32)
        for k, m in ((16, 0), (7, mq), (100, 0)):
            gi, gd = cpu.dpknn(Pr, rowp, succ, Q, k, m, threads=3, sort=(k != 7))
            ri, rd = _oracle(Pr, Q, k, m)
            assert np.array_equal(gi, ri) and np.array_equal(gd, rd), (kind, k)
        c.close()


def test_invalid_arguments_raise():
    P, _ = W.uniform_cube(20, 1)
    t = cpu.KDTree(P)
    with pytest.raises(ValueError):
        t.knn(np.zeros((2, 3), np.float32), 0)
    with pytest.raises(ValueError):
        t.knn(np.zeros((2, 3), np.float32), 4, 21)
