"""The comparison rule itself, on the CPU: the oracle's own rows pass,
rows with a plausible mistake fail."""
from __future__ import annotations

import numpy as np
import pytest

import oracle.knn as ok
import workloads as W
from tests import parity


def _setup():
    wl = W.small_sphere(nq=60)
    P = wl.ranked_points()
    idx, d2, D = ok.knn(P, wl.queries, 8, 0)
    return P, wl.queries, idx, d2


def test_oracle_rows_pass():
    P, Q, idx, d2 = _setup()
    parity.check_rows(P, Q, 8, 0, idx, d2)
    parity.check_row_properties(idx, d2, 8, np.full(Q.shape[0], P.shape[0]), P.shape[0])


@pytest.mark.parametrize("mistake", ["swap_far", "drop_last", "wrong_distance", "repeat",
                                     "out_of_prefix", "unsorted", "bad_padding"])
def test_mistakes_fail(mistake):
    P, Q, idx, d2 = _setup()
    idx = idx.copy()
    d2 = d2.copy()
    m = 0
    if mistake == "swap_far":
        r, D = ok.knn_one(P, Q[0], 40, P.shape[0])
        idx[0, 3] = r[30]
        d2[0, 3] = np.float32(D[30])
        d2[0] = np.sort(d2[0])
    elif mistake == "drop_last":
        r, D = ok.knn_one(P, Q[0], 40, P.shape[0])
        idx[0, 7] = r[9]
        d2[0, 7] = np.float32(D[9])
    elif mistake == "wrong_distance":
        d2[0, 2] *= np.float32(1.00001)
    elif mistake == "repeat":
        idx[0, 5] = idx[0, 4]
    elif mistake == "out_of_prefix":
        m = np.full(Q.shape[0], 100)
        idx, d2, _ = ok.knn(P, Q, 8, 0)
    elif mistake == "unsorted":
        idx[0, [1, 2]] = idx[0, [2, 1]]
        d2[0, [1, 2]] = d2[0, [2, 1]]
    elif mistake == "bad_padding":
        idx, d2, _ = ok.knn(P, Q, 8, 5)
        idx = idx.copy()
        idx[0, 6] = 7
        m = 5
    with pytest.raises(AssertionError):
        parity.check_rows(P, Q, 8, m, idx, d2)
