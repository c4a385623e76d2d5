"""Insertion orders (CPU only): the Hilbert curve, the BRIO rounds, the
farthest-point property, and builds in each order against the definition."""
from __future__ import annotations

import numpy as np
import pytest

import oracle.successors as osucc
import workloads as W
from paper_2605_02224_gb300 import Cloud
from paper_2605_02224_gb300 import mknn as M


@pytest.mark.parametrize("bits", [1, 2, 3, 4])
def test_hilbert_curve_visits_every_cell_once_through_neighbours(bits):
    """A Hilbert curve on a 2^bits grid: the index is a bijection onto
    0 .. 8^bits - 1 and cells at consecutive indices share a face."""
    side = 1 << bits
    cells = {}
    for x in range(side):
        for y in range(side):
            for z in range(side):
                cells[M.mknn_hilbert_index3(x, y, z, bits)] = (x, y, z)
    assert sorted(cells) == list(range(side ** 3))
    for h in range(side ** 3 - 1):
        a, b = np.array(cells[h]), np.array(cells[h + 1])
        assert np.abs(a - b).sum() == 1, (h, cells[h], cells[h + 1])
    assert M.mknn_hilbert_index3(0, 0, 0, 0) == 0 and M.mknn_hilbert_index3(0, 0, 0, 22) == 0


def _keys16(P):
    lo = P.min(axis=0).astype(np.float64)
    span = float((P.max(axis=0).astype(np.float64) - lo).max())
    c = np.minimum(np.floor((P.astype(np.float64) - lo) * ((2 ** 16 - 1) / span)), 2 ** 16 - 1)
    return [M.mknn_hilbert_index3(int(a), int(b), int(d), 16) for a, b, d in c.astype(np.int64)]


def test_brio_rounds_are_hilbert_sorted_and_double():
    P, _ = W.bumpy_sphere(5000, 3)
    o = M.mknn_insertion_order(P, M.ORDER_BRIO_HILBERT, 11)
    assert np.array_equal(np.sort(o), np.arange(5000))
    cuts = [5000]
    while cuts[-1] > 64:
        cuts.append(cuts[-1] // 2)
    cuts = [0] + cuts[::-1]
    keys = np.array(_keys16(P[o]), dtype=np.uint64)
    for a, b in zip(cuts[:-1], cuts[1:]):
        assert np.all(np.diff(keys[a:b].astype(np.float64)) >= 0), (a, b)
    assert not np.array_equal(o, M.mknn_insertion_order(P, M.ORDER_BRIO_HILBERT, 12))


def test_farthest_point_order_property():
    """Each point taken is at the largest distance from those taken before
    it (float64, ties to the lower index), starting from index 0."""
    P, _ = W.uniform_cube(1500, 4)
    P = np.concatenate([P, P[:10]])                  # duplicates: distance 0 at the end
    o = M.mknn_insertion_order(P, M.ORDER_FARTHEST_POINT)
    assert o[0] == 0 and np.array_equal(np.sort(o), np.arange(P.shape[0]))
    X = P.astype(np.float64)
    mind = np.full(P.shape[0], np.inf)
    taken = np.zeros(P.shape[0], bool)
    for t, i in enumerate(o):
        if t > 0:
            cand = np.where(~taken, mind, -1.0)
            best = cand.max()
            assert mind[i] == best and i == np.flatnonzero(cand == best)[0], t
        taken[i] = True
        mind = np.minimum(mind, ((X - X[i]) ** 2).sum(axis=1))


@pytest.mark.parametrize("kind", [M.ORDER_RANDOM, M.ORDER_BRIO_HILBERT, M.ORDER_FARTHEST_POINT])
def test_builds_in_each_order_match_the_definition(kind):
    P, _ = W.sphere(250, 21)
    o = M.mknn_insertion_order(P, kind, 5)
    c = Cloud.build(P, o)
    _, rowp, succ = c.table()
    defn = osucc.successor_lists(P[o])
    for i, lst in enumerate(defn):
        assert set(lst) <= set(succ[rowp[i]:rowp[i + 1]].tolist()), i
    c.close()


def test_order_errors():
    with pytest.raises(M.MknnError):
        M.mknn_insertion_order(np.zeros((3, 3), np.float32), 7)
    with pytest.raises(M.MknnError):
        M.mknn_insertion_order(np.array([[0, 0, np.inf]], np.float32), M.ORDER_RANDOM)
    assert M.mknn_insertion_order(np.zeros((0, 3), np.float32), M.ORDER_FARTHEST_POINT).size == 0
