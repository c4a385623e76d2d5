"""The persistent multi-cloud kernel, its plan, graph replay and tuner."""
from __future__ import annotations

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
def clouds(torch):
    """Eight clouds of the batching workload's recipe, scaled down."""
    wls = W.batch_clouds(n_clouds=8, lo=2000, hi=60000, seed=21)
    out = []
    for wl in wls:
        c = Cloud.build(wl.points, wl.order).upload()
        out.append((wl, c))
    yield out
    for _, c in out:
        c.close()


def _requests(torch, clouds, m_mode="scalar"):
    reqs, keep = [], []
    for i, (wl, c) in enumerate(clouds):
        q = torch.from_numpy(wl.queries).cuda()
        nq = wl.nq
        idx = torch.full((nq, wl.k), -9, dtype=torch.int32, device="cuda")
        d2 = torch.full((nq, wl.k), -9.0, dtype=torch.float32, device="cuda")
        m = None
        ms = 0
        if m_mode == "array" and i % 2 == 0:
            mv = np.clip(np.floor(np.exp(W.uniform(70 + i, 1, nq) * np.log(wl.n))), 1, wl.n)
            m = torch.from_numpy(mv.astype(np.int32)).cuda()
        elif m_mode == "array":
            ms = max(1, wl.n // 3)
        reqs.append(dict(cloud=c.handle, q=q, nq=nq, q_stride=3, k=wl.k, m=m, m_scalar=ms,
                         out_idx=idx, out_d2=d2))
        keep.append((wl, c, q, m, ms, idx, d2))
    return reqs, keep


def _plain(torch, c, q, k, m, ms):
    idx, d2 = c.knn(q, k, m if m is not None else (ms or None))
    torch.cuda.synchronize()
    return idx.cpu().numpy(), d2.cpu().numpy()


@pytest.mark.parametrize("lanes,placement", [(0, 0), (1, 0), (4, 0), (8, 0), (16, 0), (32, 1),
                                             (32, 2)])
def test_batch_equals_plain_per_request(torch, clouds, lanes, placement):
    reqs, keep = _requests(torch, clouds, "array")
    kmax = {4: 16}.get(lanes, 64)     # variants compiled into the persistent kernel
    if any(r["k"] > kmax for r in reqs):
        bad = [dict(r) for r in reqs]
        with pytest.raises(M.MknnError) as ei:
            M.mknn_knn_batch(bad, torch.cuda.current_stream().cuda_stream, lanes=lanes,
                             placement=placement)
        assert ei.value.status == 1
        reqs = [r for r in reqs if r["k"] <= kmax]
        keep = [kp for kp in keep if kp[0].k <= kmax]
    M.mknn_knn_batch(reqs, torch.cuda.current_stream().cuda_stream, lanes=lanes,
                     placement=placement)
    torch.cuda.synchronize()
    for wl, c, q, m, ms, idx, d2 in keep:
        pi, pd = _plain(torch, c, q, wl.k, m, ms)
        assert np.array_equal(idx.cpu().numpy(), pi), wl.name
        assert np.array_equal(d2.cpu().numpy(), pd), wl.name


def test_plan_with_many_variants_equals_plain(torch, clouds, tmp_path):
    """A tuning table that gives the eight requests different lane widths:
    the plan runs one persistent launch per variant (one-lane kernel and
    group kernels on two streams), and every row equals a plain launch."""
    reqs, keep = _requests(torch, clouds, "array")
    widths = (1, 32, 8, 16, 1, 32, 16, 8)
    lines = []
    for (wl, c, *_), w in zip(keep, widths):
        longest = int(np.diff(c.table()[1]).max())
        lines.append(f"{wl.k} {int(np.floor(np.log2(wl.n)))} "
                     f"{int(np.floor(np.log2(1 + longest)))} {w}\n")
    path = tmp_path / "table.txt"
    path.write_text("# k log2n hub lanes\n" + "".join(lines))
    M.mknn_tune_clear()
    M.mknn_tune_load(str(path))
    try:
        plan = M.mknn_batch_create(reqs)
        lanes, items, grid = M.mknn_batch_info(plan, len(reqs))
        assert len(set(lanes.tolist())) >= 3, lanes
        s = torch.cuda.current_stream().cuda_stream
        for _ in range(2):                           # graph replay twice
            M.mknn_batch_run(plan, s)
        torch.cuda.synchronize()
        for wl, c, q, m, ms, idx, d2 in keep:
            pi, pd = _plain(torch, c, q, wl.k, m, ms)
            assert np.array_equal(idx.cpu().numpy(), pi), wl.name
            assert np.array_equal(d2.cpu().numpy(), pd), wl.name
        M.mknn_batch_free(plan)
    finally:
        M.mknn_tune_clear()


def test_tuning_table_with_both_placements(torch, clouds, tmp_path):
    """Table lines with a placement column: the same k on 32 lanes in
    registers for some requests and one list per warp in shared memory for
    others; the plan runs both kernels and every row equals a plain launch."""
    reqs, keep = _requests(torch, clouds, "array")
    modes = ((32, 1), (32, 2), (1, 2), (32, 2), (32, 1), (8, 1), (32, 2), (16, 1))
    lines = []
    for (wl, c, *_), (w, p) in zip(keep, modes):
        longest = int(np.diff(c.table()[1]).max())
        lines.append(f"{wl.k} {int(np.floor(np.log2(wl.n)))} "
                     f"{int(np.floor(np.log2(1 + longest)))} {w} {p}\n")
    path = tmp_path / "table.txt"
    path.write_text("# k log2n hub lanes placement\n" + "".join(lines))
    M.mknn_tune_clear()
    M.mknn_tune_load(str(path))
    try:
        plan = M.mknn_batch_create(reqs)
        lanes, _, _ = M.mknn_batch_info(plan, len(reqs))
        pl = M.mknn_batch_placement(plan, len(reqs))
        got = set(zip(lanes.tolist(), pl.tolist()))
        assert (32, 1) in got and (32, 2) in got, got
        M.mknn_batch_run(plan, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        for wl, c, q, m, ms, idx, d2 in keep:
            pi, pd = _plain(torch, c, q, wl.k, m, ms)
            assert np.array_equal(idx.cpu().numpy(), pi), wl.name
            assert np.array_equal(d2.cpu().numpy(), pd), wl.name
        M.mknn_batch_free(plan)
        saved = tmp_path / "saved.txt"
        M.mknn_tune_save(str(saved))
        rows = [l.split() for l in saved.read_text().splitlines() if not l.startswith("#")]
        assert rows and all(len(r) == 5 for r in rows)
    finally:
        M.mknn_tune_clear()


def test_large_k_requests_in_a_plan(torch, clouds):
    """Requests with k = 65, 100 and 128 (the one-lane kernel with 128-slot
    lists, or 16 and 32 lanes) mixed with the workload's own: the plan equals
    plain launches, and a sample equals the oracle."""
    reqs, keep = _requests(torch, clouds[:3], "array")
    for (wl, c), k in zip(clouds[3:6], (65, 100, 128)):
        q = torch.from_numpy(wl.queries).cuda()
        idx = torch.full((wl.nq, k), -9, dtype=torch.int32, device="cuda")
        d2 = torch.full((wl.nq, k), -9.0, dtype=torch.float32, device="cuda")
        reqs.append(dict(cloud=c.handle, q=q, nq=wl.nq, q_stride=3, k=k, m=None, m_scalar=0,
                         out_idx=idx, out_d2=d2))
        keep.append((wl, c, q, None, 0, idx, d2, k))
    for forced, placement in ((0, 0), (32, 2), (32, 1), (16, 0)):
        plan = M.mknn_batch_create(reqs, lanes=forced, placement=placement)
        lanes, _, _ = M.mknn_batch_info(plan, len(reqs))
        assert all(l in (1, 16, 32) for l in lanes[3:])
        M.mknn_batch_run(plan, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        M.mknn_batch_free(plan)
        _check_large_k(torch, keep)


def _check_large_k(torch, keep):
    for item in keep:
        wl, c, q, m, ms, idx, d2 = item[:7]
        k = item[7] if len(item) > 7 else wl.k
        pi, pd = _plain(torch, c, q, k, m, ms)
        assert np.array_equal(idx.cpu().numpy(), pi), wl.name
        assert np.array_equal(d2.cpu().numpy(), pd), wl.name
        if k > 64:
            parity.check_rows(wl.ranked_points(), wl.queries, k, 0, idx.cpu().numpy(),
                              d2.cpu().numpy(), rows=range(0, wl.nq, max(1, wl.nq // 60)))
        idx.fill_(-9)
        d2.fill_(-9.0)


def test_batch_against_oracle_sample(torch, clouds):
    reqs, keep = _requests(torch, clouds, "array")
    plan = M.mknn_batch_create(reqs)
    M.mknn_batch_run(plan, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    for wl, c, q, m, ms, idx, d2 in keep:
        mh = m.cpu().numpy() if m is not None else (ms or wl.n)
        I, D = idx.cpu().numpy(), d2.cpu().numpy()
        mv = mh if np.ndim(mh) else np.full(wl.nq, mh)
        parity.check_row_properties(I, D, wl.k, np.asarray(mv, np.int64), wl.n)
        parity.check_rows(wl.ranked_points(), wl.queries, wl.k, mh, I, D,
                          rows=range(0, wl.nq, max(1, wl.nq // 150)))
    lanes, items, grid = M.mknn_batch_info(plan, len(reqs))
    assert items > 0 and grid > 0 and all(l in (1, 4, 8, 16, 32) for l in lanes)
    M.mknn_batch_free(plan)


def test_graph_replay_sees_new_query_contents(torch, clouds):
    reqs, keep = _requests(torch, clouds[:3])
    plan = M.mknn_batch_create(reqs, graph=0)
    s = torch.cuda.current_stream().cuda_stream
    M.mknn_batch_run(plan, s)
    torch.cuda.synchronize()
    first = [k[5].clone() for k in keep]
    for wl, c, q, m, ms, idx, d2 in keep:         # move the queries, same buffers
        q.mul_(0.5)
    M.mknn_batch_run(plan, s)
    M.mknn_batch_run(plan, s)                      # replay twice in a row
    torch.cuda.synchronize()
    for (wl, c, q, m, ms, idx, d2), f in zip(keep, first):
        pi, pd = _plain(torch, c, q, wl.k, m, ms)
        assert np.array_equal(idx.cpu().numpy(), pi)
        assert not np.array_equal(f.cpu().numpy(), pi) or wl.nq < 10
    M.mknn_batch_free(plan)


def test_tuner_fills_table_and_plan_uses_it(torch, clouds, tmp_path):
    reqs, keep = _requests(torch, clouds)
    s = torch.cuda.current_stream().cuda_stream
    M.mknn_batch_tune(reqs, 4096, s)
    path = str(tmp_path / "tune.txt")
    M.mknn_tune_save(path)
    lines = [l for l in open(path) if not l.startswith("#")]
    assert len(lines) >= 1
    M.mknn_tune_load(path)
    plan = M.mknn_batch_create(reqs)
    lanes, _, _ = M.mknn_batch_info(plan, len(reqs))
    placement = M.mknn_batch_placement(plan, len(reqs))
    table = {(int(a), int(b), int(h)): (int(c), int(p))
             for a, b, h, c, p in (l.split() for l in lines)}
    for (wl, c, *_), l, p in zip(keep, lanes, placement):
        longest = int(np.diff(c.table()[1]).max())
        key = (wl.k, int(np.floor(np.log2(wl.n))), int(np.floor(np.log2(1 + longest))))
        assert key in table
        assert table[key][0] == l or l > table[key][0]   # widened only to fill the GPU
        if table[key][0] == l:
            assert table[key][1] == p                     # the tuned placement is kept
    M.mknn_batch_run(plan, s)
    torch.cuda.synchronize()
    for wl, c, q, m, ms, idx, d2 in keep:
        pi, _ = _plain(torch, c, q, wl.k, m, ms)
        assert np.array_equal(idx.cpu().numpy(), pi)
    M.mknn_batch_free(plan)


def test_batch_rejects_bad_requests(torch, clouds):
    reqs, _ = _requests(torch, clouds[:2])
    reqs[1]["k"] = 0
    with pytest.raises(M.MknnError) as ei:
        M.mknn_batch_create(reqs)
    assert ei.value.status == 1
    reqs[1]["k"] = 129
    with pytest.raises(M.MknnError):
        M.mknn_batch_create(reqs)
    reqs[1]["k"] = 8
    reqs[1]["nq"] = 2 ** 31 - 256          # a lane's index + 32 must stay in int32
    with pytest.raises(M.MknnError) as ei:
        M.mknn_batch_create(reqs)
    assert ei.value.status == 1
