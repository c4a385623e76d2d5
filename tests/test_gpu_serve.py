"""The serving loop: continuous batching, admission by memory, results equal
alone and in the mix, bounded waits."""
from __future__ import annotations

import threading
import time

import numpy as np
import pytest

import workloads as W
from paper_2605_02224_gb300 import Cloud
from paper_2605_02224_gb300 import mknn as M
from tests import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.fixture(scope="module")
def resident(torch):
    wls = W.serve_clouds(n_clouds=4, lo=5000, hi=80000, seed=41)
    cl = [Cloud.build(w.points, w.order).upload() for w in wls]
    yield wls, cl
    for c in cl:
        c.close()


def _requests(wls, n_req, seed=42, max_q=5000, rate=5000.0):
    return W.serve_requests(wls, n_req, rate, seed=seed, max_q=max_q)


def _alone(clouds, r):
    c = clouds[r.cloud]
    return c.knn_host(r.queries, r.k, r.m)


def _check_against_oracle(wls, r, oi, od, every=50):
    """Rows 0, every, 2*every, ... of a served request against the float64
    brute-force oracle on P_{1:m} of its cloud (at least one row per request)."""
    P = wls[r.cloud].ranked_points()
    nq = r.queries.shape[0]
    rows = range(0, nq, every)
    parity.check_rows(P, r.queries, r.k, np.full(nq, r.m, np.int64), np.asarray(oi),
                      np.asarray(od), rows=rows)
    return len(rows)


def _pinned(torch, shape, dtype):
    return torch.empty(shape, dtype=dtype).pin_memory()


@pytest.mark.parametrize("plain", [0, 1])
def test_each_result_equal_alone_and_in_the_mix(torch, resident, plain):
    wls, cl = resident
    reqs = _requests(wls, 120)
    srv = M.mknn_server_create(slots=3, plain=plain, mem_budget=256 << 20)
    ids = [M.mknn_server_add_cloud(srv, c.handle) for c in cl]
    outs, tickets = [], []
    for r in reqs:
        oi = np.empty((r.queries.shape[0], r.k), np.int32)     # pageable on purpose
        od = np.empty((r.queries.shape[0], r.k), np.float32)
        tickets.append(M.mknn_server_submit(srv, ids[r.cloud], r.queries, r.k, r.m, oi, od))
        outs.append((oi, od))
    M.mknn_server_drain(srv, 120.0)
    st = M.mknn_server_stats(srv)
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["p99_ms"] >= st["p50_ms"] > 0
    assert st["h2d_ms"] > 0 and st["kernel_ms"] > 0 and st["d2h_ms"] > 0
    if not plain:
        assert st["mean_requests_per_launch"] > 1.0     # requests really were batched
    checked = 0
    for r, (oi, od), t in zip(reqs, outs, tickets):
        assert M.mknn_server_poll(srv, t) == 1
        ai, ad = _alone(cl, r)
        assert np.array_equal(oi, ai) and np.array_equal(od, ad)
        checked += _check_against_oracle(wls, r, oi, od)
    assert checked >= len(reqs)
    M.mknn_server_destroy(srv, 60.0)


def test_poisson_arrivals_pinned_buffers_overlap(torch, resident):
    """Requests arrive while others run (Poisson, from a client thread);
    all complete with results equal to running each alone."""
    wls, cl = resident
    reqs = _requests(wls, 80, seed=7, rate=400.0)
    srv = M.mknn_server_create(slots=3, mem_budget=512 << 20)
    ids = [M.mknn_server_add_cloud(srv, c.handle) for c in cl]
    bufs = []
    for r in reqs:
        q = _pinned(torch, r.queries.shape, torch.float32)
        q.copy_(torch.from_numpy(r.queries))
        bufs.append((q, _pinned(torch, (r.queries.shape[0], r.k), torch.int32),
                     _pinned(torch, (r.queries.shape[0], r.k), torch.float32)))
    t0 = time.perf_counter()

    def client():
        for r, (q, oi, od) in zip(reqs, bufs):
            delay = r.arrival_s - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            M.mknn_server_submit(srv, ids[r.cloud], q, r.k, r.m, oi, od)

    th = threading.Thread(target=client)
    th.start()
    th.join()
    M.mknn_server_drain(srv, 120.0)
    st = M.mknn_server_stats(srv)
    assert st["completed"] == len(reqs)
    for r, (q, oi, od) in zip(reqs, bufs):
        ai, ad = _alone(cl, r)
        assert np.array_equal(oi.numpy(), ai) and np.array_equal(od.numpy(), ad)
        _check_against_oracle(wls, r, oi.numpy(), od.numpy())
    lat = M.mknn_server_latencies(srv, len(reqs))
    assert lat.shape[0] == len(reqs) and np.all(lat > 0)
    M.mknn_server_destroy(srv, 60.0)


def test_admission_by_memory_queues_and_rejects(torch, resident):
    wls, cl = resident
    srv = M.mknn_server_create(slots=2, mem_budget=24 << 20)
    cid = M.mknn_server_add_cloud(srv, cl[0].handle)
    lo, hi = W.padded_box(wls[0].points)
    big = W.box_queries(200_000, 5, lo, hi)                 # ~ 30 MB in flight: too big
    oi = np.empty((200_000, 16), np.int32)
    od = np.empty((200_000, 16), np.float32)
    with pytest.raises(M.MknnError) as ei:
        M.mknn_server_submit(srv, cid, big, 16, 0, oi, od)
    assert ei.value.status == 2
    # many requests that fit one or two at a time: all complete, in order of budget
    qs = [W.box_queries(30_000, 100 + i, lo, hi) for i in range(12)]
    outs = [(np.empty((30_000, 8), np.int32), np.empty((30_000, 8), np.float32)) for _ in qs]
    for q, (a, b) in zip(qs, outs):
        M.mknn_server_submit(srv, cid, q, 8, 0, a, b)
    M.mknn_server_drain(srv, 120.0)
    st = M.mknn_server_stats(srv)
    assert st["completed"] == 12
    for q, (a, b) in zip(qs, outs):
        ai, _ = cl[0].knn_host(q, 8)
        assert np.array_equal(a, ai)
    M.mknn_server_destroy(srv, 60.0)


def test_held_cloud_cannot_be_freed_and_bad_requests(torch, resident):
    wls, cl = resident
    extra = Cloud.build(wls[1].points, wls[1].order)
    srv = M.mknn_server_create()
    cid = M.mknn_server_add_cloud(srv, extra.handle)
    with pytest.raises(M.MknnError) as ei:
        M.mknn_cloud_free(extra.handle)
    assert ei.value.status == 4
    q = np.zeros((4, 3), np.float32)
    oi = np.empty((4, 8), np.int32)
    od = np.empty((4, 8), np.float32)
    with pytest.raises(M.MknnError):
        M.mknn_server_submit(srv, cid + 5, q, 8, 0, oi, od)     # unknown cloud
    with pytest.raises(M.MknnError):
        M.mknn_server_submit(srv, cid, q, 0, 0, oi, od)          # k = 0
    with pytest.raises(M.MknnError):
        M.mknn_server_submit(srv, cid, q, 8, extra.n + 1, oi, od)  # m > n
    M.mknn_server_destroy(srv, 30.0)
    extra.close()                                                # released: frees fine


def test_drain_times_out_then_completes(torch, resident):
    wls, cl = resident
    srv = M.mknn_server_create(slots=1)
    cid = M.mknn_server_add_cloud(srv, cl[3].handle)
    lo, hi = W.padded_box(wls[3].points)
    q = W.box_queries(1_000_000, 9, lo, hi)
    oi = np.empty((1_000_000, 32), np.int32)
    od = np.empty((1_000_000, 32), np.float32)
    t = M.mknn_server_submit(srv, cid, q, 32, 0, oi, od)
    with pytest.raises(M.MknnError) as ei:
        M.mknn_server_drain(srv, 0.0)
    assert ei.value.status == 5
    M.mknn_server_drain(srv, 120.0)
    assert M.mknn_server_poll(srv, t) == 1
    M.mknn_server_destroy(srv, 30.0)


def test_served_rows_on_a_cloud_with_box_trees(torch):
    """A resident cloud with box trees (400k-site planar patches, lists of up
    to ~33k entries) beside one without: the batched server's packs hand the
    one-lane queries that meet a list with a tree over to the one-warp kernel
    and walk the trees for one-warp requests; every served row equals the
    same request run alone through mknn_knn."""
    from tests.gpu_util import built_cloud
    n = 400_000
    P, _ = W.patches4(n, 21200)
    c = built_cloud(P, W.permutation(n, 21201), "patches400k")
    c.upload()
    assert c.trees()[0] > 0
    S, _ = W.sphere(20000, 75)
    cs = built_cloud(S, W.permutation(20000, 76), "sphere20k")
    cs.upload()
    Pr = P[W.permutation(n, 21201)]
    _, rowp, _ = c.table()
    hubs = np.argsort(-np.diff(rowp), kind="stable")[:200]
    # packs of up to 2^20 queries, so that k <= 8 requests stay one lane wide
    # (smaller packs widen them to 32 lanes)
    srv = M.mknn_server_create(slots=3, plain=0, mem_budget=1 << 30, max_batch_queries=1 << 20)
    ids = [M.mknn_server_add_cloud(srv, h.handle) for h in (c, cs)]
    jobs = []
    for j, (k, m) in enumerate([(1, 0), (4, 0), (8, n // 3), (16, 0), (48, 0), (100, n // 2),
                                (4, 0), (32, 0)]):
        nq = 30000 + 1000 * j
        near = Pr[hubs[np.arange(nq) % len(hubs)]] + \
            1e-3 * W.normal(80 + j, 1, 3 * nq).reshape(-1, 3)
        Q = np.concatenate([near[: nq // 2],
                            W.box_queries(nq - nq // 2, 90 + j, [0.0] * 3, [1.0] * 3)])
        Q = np.ascontiguousarray(Q, np.float32)
        which = 0 if j % 4 else 1
        oi = np.empty((nq, k), np.int32)
        od = np.empty((nq, k), np.float32)
        mm = m if which == 0 else 0
        t = M.mknn_server_submit(srv, ids[which], Q, k, mm, oi, od)
        jobs.append(((c, cs)[which], Q, k, mm, oi, od, t))
    M.mknn_server_drain(srv, 120.0)
    st = M.mknn_server_stats(srv)
    assert st["completed"] == len(jobs) and st["failed"] == 0
    for cl, Q, k, mm, oi, od, _ in jobs:
        ri, rd = cl.knn(torch.from_numpy(Q).cuda(), k, mm or None)
        torch.cuda.synchronize()
        assert np.array_equal(oi, ri.cpu().numpy()) and np.array_equal(od, rd.cpu().numpy()), k
    M.mknn_server_destroy(srv, 10.0)
    cs.close()
    c.close()
