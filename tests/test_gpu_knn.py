"""Parity of the CUDA query path (through the C ABI) with the oracle."""
from __future__ import annotations

import numpy as np
import pytest

import oracle.dpknn as dp
import oracle.knn as ok
import workloads as W
from paper_2605_02224_gb300 import Cloud
from paper_2605_02224_gb300 import mknn as M
from tests import parity
from tests.gpu_util import built_cloud, run_knn

pytestmark = pytest.mark.gpu

LANES = (1, 4, 8, 16, 32)
# lanes per query; candidate-list placement for 1 and 32 lanes (1 = registers,
# 2 = shared memory: a list per thread, or one per warp)
VARIANTS = (dict(lanes=1, placement=1), dict(lanes=1, placement=2),
            dict(lanes=4, placement=1), dict(lanes=8, placement=1), dict(lanes=16, placement=1),
            dict(lanes=32, placement=1), dict(lanes=32, placement=2))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()


# ------------------------------------------------------------ tiny, exhaustive

@pytest.mark.parametrize("n", [1, 2, 5, 17, 64, 150, 4200])
@pytest.mark.parametrize("table", ["complete", "built"])
def test_tiny_exhaustive(n, table):
    P, _ = W.uniform_cube(n, 100 + n)
    order = W.permutation(n, 200 + n)
    Pr = P[order]
    if table == "complete":
        rowp, succ = dp.complete_table(n)
        c = Cloud.from_table(Pr, rowp, succ).upload()
    else:
        c = Cloud.build(P, order).upload()
    Q = W.box_queries(60, 7, [-1.5] * 3, [1.5] * 3)
    Q = np.concatenate([Q, Pr[: min(n, 20)]])          # queries exactly on sites
    ks = sorted({1, 2, min(n, 8), min(n + 1, 64), 33, 64, 100, 128})
    for v in VARIANTS:
        for k in ks:
            small = v["lanes"] in (4, 8) or (v["lanes"] == 1 and v["placement"] == 1)
            if k > 64 and small:                       # these variants hold k <= 64
                with pytest.raises(M.MknnError):
                    run_knn(c, Q, k, **v)
                continue
            for m in sorted({1, max(1, n // 2), n}):
                idx, d2 = run_knn(c, Q, k, m, **v, sort=1 if k % 2 else -1)
                parity.check_rows(Pr, Q, k, m, idx, d2)
    c.close()


def test_small_sphere_workload_all_queries():
    """2,000 points on the unit sphere, 10,000 queries, k = 8: every row."""
    wl = W.small_sphere()
    c = Cloud.build(wl.points, wl.order).upload()
    Pr = wl.ranked_points()
    for v in VARIANTS:
        idx, d2 = run_knn(c, wl.queries, wl.k, **v)
        parity.check_rows(Pr, wl.queries, wl.k, 0, idx, d2)
    idx0, d20 = run_knn(c, wl.queries, wl.k)
    assert c.check() == 0
    c.close()


def test_sphere_centre_closed_form():
    """Origin against the 2,000-point sphere: every squared distance is 1 up
    to float32 normalisation; the 64 returned ranks are distinct."""
    wl = W.small_sphere(nq=1)
    c = Cloud.build(wl.points, wl.order).upload()
    Q = np.zeros((4, 3), np.float32)
    for v in VARIANTS:
        idx, d2 = run_knn(c, Q, 64, **v)
        assert np.all(np.abs(d2 - 1.0) <= 1e-6)
        assert all(np.unique(r).size == 64 for r in idx)
        assert np.all(idx >= 0) and np.all(idx < 2000)
    c.close()


def test_lattice_rings_closed_form():
    """Integer lattice (all cubes cospherical): k equal to cumulative ring
    sizes returns whole rings, exact squared distances, ranks ascending
    inside each ring."""
    from tests import oracle_pins as pins
    L = 16
    P_in, _ = W.lattice(L)
    order = W.permutation(P_in.shape[0], 5)
    c = Cloud.build(P_in, order).upload()
    P, rank_of = pins.lattice_setup(L, 5)
    r3 = pins.read_r3()
    rng = np.random.default_rng(0)
    centres = rng.integers(5, L - 5, size=(50, 3)).astype(np.float32)
    for k in (1, 7, 19, 27, 33):
        for v in VARIANTS:
            idx, d2 = run_knn(c, centres, k, **v)
            parity.check_rows(P, centres, k, 0, idx, d2)
            cum = np.cumsum([r3[s] for s in range(13)])
            smax = int(np.searchsorted(cum, k))
            want = np.concatenate([np.full(r3[s], float(s)) for s in range(smax + 1)])
            assert np.all(d2 == want[None, :])
    c.close()


def test_prefix_bound_per_query_and_padding():
    P, _ = W.bumpy_sphere(20000, 31)
    order = W.permutation(20000, 32)
    c = built_cloud(P, order, "bumpy20k")
    c.upload()
    Pr = P[order]
    nq = 3000
    Q = np.concatenate([W.box_queries(nq // 2, 33, [-1.3] * 3, [1.3] * 3),
                        W.near_surface_queries("bumpy", nq - nq // 2, 34)])
    u = W.uniform(35, 1, nq)
    m = np.floor(np.exp(u * np.log(20000))).astype(np.int32)
    m = np.clip(m, 1, 20000)
    m[:50] = np.arange(1, 51)                       # m < k: padded rows
    for k in (1, 10, 64):
        for v in VARIANTS:
            idx, d2 = run_knn(c, Q, k, m, **v)
            parity.check_row_properties(idx, d2, k, m.astype(np.int64), 20000)
            parity.check_rows(Pr, Q, k, m, idx, d2, rows=range(0, nq, 7))
    assert c.check() == 0
    c.close()


def test_persistent_grid_equals_one_block_per_256_queries():
    """The one-lane kernel's persistent grid (blocks_per_sm > 0: each thread
    loops over many queries) gives the same rows, bit for bit, as the
    default grid of one block per 256 queries, with per-query prefix bounds
    (some outside [1, n]) and k in every block-size class."""
    P, _ = W.bumpy_sphere(20000, 31)
    order = W.permutation(20000, 32)
    c = built_cloud(P, order, "bumpy20k")
    c.upload()
    Pr = P[order]
    nq = 120_001                                    # a ragged last block
    Q = np.concatenate([W.box_queries(nq // 2, 36, [-1.3] * 3, [1.3] * 3),
                        W.near_surface_queries("bumpy", nq - nq // 2, 37)])
    m = np.clip(np.floor(np.exp(W.uniform(38, 1, nq) * np.log(20000))), 1, 20000)
    m = m.astype(np.int32)
    m[7::5000] = 0                                  # invalid bounds: padded rows, flag set
    for k in (1, 16, 40, 100):
        base_i, base_d = run_knn(c, Q, k, m, lanes=1, placement=2)
        for bps in (1, 2):
            i2, d2 = run_knn(c, Q, k, m, lanes=1, placement=2, blocks_per_sm=bps)
            assert np.array_equal(i2, base_i) and np.array_equal(d2, base_d), (k, bps)
        ok_rows = np.flatnonzero(m > 0)
        parity.check_rows(Pr, Q, k, m, base_i, base_d, rows=ok_rows[::997])
        bad = np.flatnonzero(m == 0)
        assert np.all(base_i[bad] == -1) and np.all(np.isinf(base_d[bad]))
    assert c.check() & 1
    c.close()


def test_hub_rows_all_variants():
    """Four nearly planar patches: a few successor lists hold hundreds to
    thousands of entries (hubs). Every row against the oracle, per-query m
    included, for every kernel variant; all variants give the same bits."""
    P, _ = W.patches4(30000, 61)
    order = W.permutation(30000, 62)
    c = built_cloud(P, order, "patches30k")
    c.upload()
    Pr = P[order]
    _, rowp, _ = c.table()
    assert np.diff(rowp).max() > 500                   # the workload has hubs
    nq = 1500
    Q = np.concatenate([W.box_queries(nq // 3, 63, [0.0] * 3, [1.0] * 3),
                        Pr[W.permutation(30000, 64)[: nq // 3]]
                        + 1e-3 * W.normal(65, 1, nq // 3 * 3).reshape(-1, 3).astype(np.float32),
                        Pr[: nq - 2 * (nq // 3)]]).astype(np.float32)
    m = np.clip(np.floor(np.exp(W.uniform(66, 1, nq) * np.log(30000))), 1, 30000).astype(np.int32)
    for k in (1, 8, 33, 64):
        mk = m if k != 8 else None
        base = None
        for v in VARIANTS:
            if v["lanes"] == 4 and k > 16:
                continue
            idx, d2 = run_knn(c, Q, k, mk, **v)
            if base is None:
                parity.check_rows(Pr, Q, k, mk if mk is not None else 0, idx, d2)
                base = (idx, d2)
            else:
                assert np.array_equal(idx, base[0]) and np.array_equal(d2, base[1]), (k, v)
    c.close()


def test_box_trees_give_the_scans_rows():
    """Successor lists of 256 entries or more get box trees, which only the
    one-warp kernel walks (descent: the lowest-rank strictly closer entry;
    expansion: the entries below the k-th key); one lane per query hands
    the queries that would read such a list through over to it. The
    400k-site patch cloud has lists of up to ~33k entries (a tree of three
    levels). Queries exactly on and next to the sites with the longest
    lists, next to those lists' entries, and in the box; for every k and
    prefix bound the tree walk and the hand-over give the same bits as the
    scanning kernels (register groups; one lane whose workspace is too
    small for the hand-over), sampled rows against the oracle."""
    import torch
    n = 400_000
    P, _ = W.patches4(n, 21200)
    order = W.permutation(n, 21201)
    c = built_cloud(P, order, "patches400k")
    c.upload()
    Pr = P[order]
    _, rowp, succ = c.table()
    L = np.diff(rowp)
    assert L.max() > 32 * 1024 and (L >= 256).sum() > 100
    trees, covered = c.trees()
    assert trees == (L >= 256).sum() and covered == L[L >= 256].sum()
    hubs = np.argsort(-L, kind="stable")[:64]
    near = np.concatenate([succ[rowp[h]:rowp[h + 1]][::41] for h in hubs[:8]])[:2000]
    Q = np.concatenate([
        Pr[hubs],
        Pr[hubs] + 1e-4 * W.normal(71, 1, 3 * len(hubs)).reshape(-1, 3),
        Pr[near] + 2e-3 * W.normal(72, 1, 3 * len(near)).reshape(-1, 3),
        W.box_queries(1500, 73, [0.0] * 3, [1.0] * 3)]).astype(np.float32)
    nq = len(Q)
    m = np.clip(np.floor(np.exp(W.uniform(74, 1, nq) * np.log(n))), 1, n).astype(np.int32)
    order = torch.arange(nq, dtype=torch.int32, device="cuda")
    tiny_ws = torch.zeros(64, dtype=torch.uint8, device="cuda")
    for k in (1, 4, 32, 100):
        for mk in (None, m):
            tree = run_knn(c, Q, k, mk, lanes=32, placement=2)
            handed = run_knn(c, Q, k, mk, lanes=1, placement=2)
            scan1 = run_knn(c, Q, k, mk, lanes=1, placement=2, order=order, workspace=tiny_ws,
                            workspace_bytes=64)
            group = run_knn(c, Q, k, mk, lanes=32 if k <= 64 else 16, placement=1)
            for other in (handed, scan1, group):
                assert np.array_equal(tree[0], other[0]) and np.array_equal(tree[1], other[1]), k
            parity.check_rows(Pr, Q, k, mk if mk is not None else 0, *tree,
                              rows=range(0, nq, 37))
    # the persistent kernels' tree forms in one plan with a sphere (no list
    # reaches 4096 entries: no trees): one warp per query (the tree walk) and
    # one lane per query (the hand-over to the one-warp kernel, k = 4 and 48
    # in the first class, 100 in the last)
    S, _ = W.sphere(20000, 75)
    so = W.permutation(20000, 76)
    cs = built_cloud(S, so, "sphere20k")
    cs.upload()
    assert cs.trees() == (0, 0)
    QS = W.box_queries(3000, 77, [-1.2] * 3, [1.2] * 3)
    for k, lanes in ((4, 32), (48, 32), (4, 1), (48, 1), (100, 1)):
        outs, reqs = [], []
        for cl, qq in ((c, Q), (cs, QS)):
            qt = torch.from_numpy(qq).cuda()
            oi = torch.full((len(qq), k), -9, dtype=torch.int32, device="cuda")
            od = torch.full((len(qq), k), -9.0, dtype=torch.float32, device="cuda")
            reqs.append(dict(cloud=cl.handle, q=qt, nq=len(qq), q_stride=3, k=k, m=None,
                             m_scalar=0, out_idx=oi, out_d2=od))
            outs.append((cl, qq, oi, od))
        M.mknn_knn_batch(reqs, torch.cuda.current_stream().cuda_stream, lanes=lanes, placement=2)
        torch.cuda.synchronize()
        for cl, qq, oi, od in outs:
            ri, rd = run_knn(cl, qq, k, None, lanes=1, placement=2)
            assert np.array_equal(oi.cpu().numpy(), ri) and np.array_equal(od.cpu().numpy(), rd)
    cs.close()
    c.close()


def test_large_k_with_prefix_bounds():
    """k above 64 (the temporal-defect setting of Sec. 5 uses k = 100):
    near-surface and volume queries with per-query m on a 20,000-site bumpy
    sphere, one lane (shared-memory list), 16 and 32 lanes and the default
    bit-identical, rows against the oracle."""
    P, _ = W.bumpy_sphere(20000, 31)
    order = W.permutation(20000, 32)
    c = built_cloud(P, order, "bumpy20k")
    c.upload()
    Pr = P[order]
    nq = 1200
    Q = np.concatenate([W.box_queries(nq // 2, 41, [-1.3] * 3, [1.3] * 3),
                        W.near_surface_queries("bumpy", nq - nq // 2, 42)])
    m = np.clip(np.floor(np.exp(W.uniform(43, 1, nq) * np.log(20000))), 1, 20000).astype(np.int32)
    for k in (65, 100, 128):
        base = None
        for lanes, placement in ((0, 0), (1, 2), (16, 1), (32, 1), (32, 2)):
            idx, d2 = run_knn(c, Q, k, m, lanes=lanes, placement=placement)
            if base is None:
                parity.check_row_properties(idx, d2, k, m.astype(np.int64), 20000)
                parity.check_rows(Pr, Q, k, m, idx, d2, rows=range(0, nq, 3))
                base = (idx, d2)
            else:
                assert np.array_equal(idx, base[0]) and np.array_equal(d2, base[1]), (k, lanes)
    c.close()


@pytest.mark.parametrize("ratio", [0.003, 0.03, 0.1, "uniform"])
def test_degraded_manifold_and_uniform_volume(ratio):
    """The sensitivity study's inputs at 20,000 sites: a bumpy sphere with
    every point displaced by up to a fraction of its bbox diagonal, and
    points uniform in a cube with queries in the same cube. Every row
    against the oracle for the default kernel; other variants identical."""
    if ratio == "uniform":
        wl = W.uniform_volume(20000, 2000, 16)
    else:
        wl = W.degraded_bumpy(ratio, 20000, 2000, 16)
    c = Cloud.build(wl.points, wl.order).upload()
    Pr = wl.ranked_points()
    idx, d2 = run_knn(c, wl.queries, 16)
    parity.check_rows(Pr, wl.queries, 16, 0, idx, d2)
    for v in (dict(lanes=1, placement=1), dict(lanes=32, placement=1),
              dict(lanes=32, placement=2)):
        i2, d22 = run_knn(c, wl.queries, 16, **v)
        assert np.array_equal(i2, idx) and np.array_equal(d22, d2)
    c.close()


@pytest.mark.parametrize("kind", [M.ORDER_BRIO_HILBERT, M.ORDER_FARTHEST_POINT])
def test_other_insertion_orders(kind):
    """Clouds built in a BRIO/Hilbert or farthest-point order: every row
    against the oracle, per-query m included (the prefix follows the order)."""
    P, _ = W.bumpy_sphere(20000, 31)
    order = M.mknn_insertion_order(P, kind, 9)
    c = Cloud.build(P, order).upload()
    Pr = P[order]
    Q = np.concatenate([W.box_queries(1000, 33, [-1.3] * 3, [1.3] * 3),
                        W.near_surface_queries("bumpy", 1000, 34)])
    m = np.clip(np.floor(np.exp(W.uniform(35, 1, 2000) * np.log(20000))), 1, 20000).astype(np.int32)
    for k, mm in ((16, None), (8, m)):
        idx, d2 = run_knn(c, Q, k, mm)
        parity.check_rows(Pr, Q, k, mm if mm is not None else 0, idx, d2)
    c.close()


def test_invalid_per_query_m_sets_flag_and_pads():
    import torch
    wl = W.small_sphere(nq=64)
    c = Cloud.build(wl.points, wl.order).upload()
    m = np.full(64, 2000, np.int32)
    m[5] = 0
    m[9] = 2001
    idx, d2 = run_knn(c, wl.queries, 8, m)
    assert np.all(idx[5] == -1) and np.all(np.isinf(d2[5]))
    assert np.all(idx[9] == -1)
    assert c.check() & 1
    assert c.check() == 0
    parity.check_rows(wl.ranked_points(), wl.queries, 8, m, idx, d2,
                      rows=[i for i in range(64) if i not in (5, 9)])
    with pytest.raises(M.MknnError):
        c.knn(torch.zeros((4, 3), device="cuda"), 129)
    with pytest.raises(M.MknnError):
        c.knn(torch.zeros((4, 3), device="cuda"), 8, 2001)
    idx, d2 = c.knn(torch.zeros((0, 3), device="cuda"), 8)
    assert idx.shape == (0, 8)
    c.close()


def test_duplicates_and_degenerate_clouds():
    P, _ = W.lattice(8)
    P = np.concatenate([P, P[:100]])                 # exact duplicates, later ranks
    n = P.shape[0]
    order = W.permutation(n, 77)
    c = Cloud.build(P, order).upload()
    Pr = P[order]
    Q = np.concatenate([W.box_queries(500, 78, [-1] * 3, [8] * 3), Pr[:100]]).astype(np.float32)
    for k in (1, 2, 9, 27, 64):
        for v in VARIANTS:
            idx, d2 = run_knn(c, Q, k, **v)
            parity.check_rows(Pr, Q, k, 0, idx, d2)
    c.close()


def test_host_buffer_entry_point_matches_device():
    wl = W.small_sphere()
    c = Cloud.build(wl.points, wl.order).upload()
    idx, d2 = run_knn(c, wl.queries, 8)
    hi, hd = c.knn_host(wl.queries, 8)
    assert np.array_equal(hi, idx) and np.array_equal(hd, d2)
    m = np.full(wl.nq, 777, np.int32)
    hi, hd = c.knn_host(wl.queries, 8, m)
    idx, d2 = run_knn(c, wl.queries, 8, m)
    assert np.array_equal(hi, idx) and np.array_equal(hd, d2)
    c.close()


def test_counters_match_algorithm_restatement():
    """Per-query rows opened / entries read / coordinates read / transition
    sites counted by the kernel equal those of the step-by-step Alg. 1 + 2
    (float64) for all but near-tie queries."""
    import torch
    P, _ = W.torus(30000, 11)
    order = W.permutation(30000, 12)
    c = built_cloud(P, order, "torus30k")
    c.upload()
    Pr = P[order]
    _, rowp, succ = c.table()
    Q = W.box_queries(400, 13, [-1.5, -1.5, -0.5], [1.5, 1.5, 0.5])
    for k, lanes in ((1, 8), (16, 8), (16, 32), (5, 4), (16, 1), (1, 1)):
        cnt = torch.zeros((Q.shape[0], 4), dtype=torch.int32, device="cuda")
        idx, d2 = run_knn(c, Q, k, lanes=lanes, counters=cnt)
        cnt = cnt.cpu().numpy()
        same = 0
        for i in range(Q.shape[0]):
            cc = dp.Counters()
            dp.knn_dp(Pr, rowp, succ, Q[i], k, 0, cc)
            trans = len(dp.descent(Pr, rowp, succ, Q[i], 30000))
            if tuple(cnt[i]) == (cc.rows, cc.entries, cc.coords, trans):
                same += 1
        assert same >= 0.99 * Q.shape[0], (k, lanes, same)
    c.close()


@pytest.mark.slow
def test_prefix_workload_full_size_sampled():
    """The 4M-site bumpy sphere with 8M queries, each with its own m
    (log-uniform in [1000, n]), k = 10: every row's properties, a sample
    of rows against brute force restricted to P_{1:m}."""
    wl = W.prefix_bumpy()
    c = built_cloud(wl.points, wl.order, "bumpy4m")
    c.upload()
    idx, d2 = run_knn(c, wl.queries, wl.k, wl.m)
    parity.check_row_properties(idx, d2, wl.k, wl.m.astype(np.int64), wl.n)
    Pr = wl.ranked_points()
    rows = np.linspace(0, wl.nq - 1, 120).astype(np.int64)
    parity.check_rows(Pr, wl.queries, wl.k, wl.m, idx, d2, rows=rows)
    assert c.check() == 0
    c.close()


@pytest.mark.slow
def test_large_torus_full_size_sampled():
    """The 1M-point torus with 4M queries, k = 16, launched as the benchmark
    launches it: every row's properties, and a sample of rows against the
    oracle one by one."""
    wl = W.large_torus()
    c = built_cloud(wl.points, wl.order, "torus1m")
    c.upload()
    idx, d2 = run_knn(c, wl.queries, wl.k)
    parity.check_row_properties(idx, d2, wl.k, np.full(wl.nq, wl.n, np.int64), wl.n)
    for v in (dict(lanes=1, placement=1), dict(lanes=16, placement=1)):
        i2, d22 = run_knn(c, wl.queries, wl.k, **v)      # other variants: the same rows
        assert np.array_equal(i2, idx) and np.array_equal(d22, d2)
    Pr = wl.ranked_points()
    rows = np.linspace(0, wl.nq - 1, 400).astype(np.int64)
    parity.check_rows(Pr, wl.queries, wl.k, 0, idx, d2, rows=rows)
    hi, hd = c.knn_host(wl.queries[:300000], wl.k)
    assert np.array_equal(hi, idx[:300000]) and np.array_equal(hd, d2[:300000])
    c.close()


def test_output_rows_unaligned_and_k_not_multiple_of_4():
    """Rows are written four values per 16-byte store only when k is a
    multiple of 4 and both output arrays are 16-byte aligned; outputs that
    start 4 bytes into an allocation, and k = 10, take one value per store.
    Every combination gives the same rows."""
    import torch
    wl = W.small_sphere(nq=3000)
    c = Cloud.build(wl.points, wl.order).upload()
    q = torch.from_numpy(wl.queries).cuda()
    nq = wl.nq
    for k in (16, 10, 8, 4):
        ref_i, ref_d = c.knn(q, k)
        base_i = torch.full((nq * k + 1,), -7, dtype=torch.int32, device="cuda")
        base_d = torch.full((nq * k + 1,), -7.0, dtype=torch.float32, device="cuda")
        oi, od = base_i[1:], base_d[1:]          # 4 bytes past a 256-byte boundary
        s = torch.cuda.current_stream().cuda_stream
        M.mknn_knn(c.handle, q, nq, 3, k, None, 0, oi, od, s)
        torch.cuda.synchronize()
        assert torch.equal(oi.view(nq, k), ref_i) and torch.equal(od.view(nq, k), ref_d), k
        assert int(base_i[0]) == -7 and float(base_d[0]) == -7.0   # nothing written before
    c.close()
