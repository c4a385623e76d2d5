"""mknn_knn_noalloc, the query entry point that allocates nothing during a
call, checked against mknn_knn on the same inputs.

It exists for callers that cannot allocate device memory while serving
queries (a memory pool that already owns the device memory they may use, or
a latency-bound loop that cannot take cudaMalloc's synchronisation). Its
scratch is a fixed array inside the library shared by every call, so the
test makes two calls in a row, with different batches, to check that the
second call does not see the first call's leftovers.

The file name makes pytest collect it last.
"""
from __future__ import annotations

import numpy as np
import pytest

import workloads as W
from paper_2605_02224_gb300 import Cloud
from paper_2605_02224_gb300 import mknn as M

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _run(torch, fn, cloud, Q, k, m):
    nq = Q.shape[0]
    q = torch.from_numpy(np.ascontiguousarray(Q, np.float32)).cuda()
    mt = None if m is None else torch.from_numpy(np.ascontiguousarray(m, np.int32)).cuda()
    idx = torch.full((nq, k), -7, dtype=torch.int32, device="cuda")
    d2 = torch.full((nq, k), -7.0, dtype=torch.float32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    fn(cloud.handle, q, nq, 3, k, mt, 0, idx, d2, s)
    torch.cuda.synchronize()
    return idx.cpu().numpy(), d2.cpu().numpy()


def test_noalloc_matches_knn_on_two_calls_in_a_row(torch_cuda):
    torch = torch_cuda
    P, _ = W.torus(50_000, 61)
    order = W.permutation(50_000, 62)
    cloud = Cloud.build(P, order).upload()
    lo, hi = W.padded_box(P)
    batches = [
        (W.box_queries(200_000, 63, lo, hi), 16, None),
        (W.box_queries(70_001, 64, lo, hi), 9,
         np.clip(np.floor(np.exp(W.uniform(65, 1, 70_001) * np.log(50_000))), 1, 50_000)),
    ]
    for Q, k, m in batches:
        ref_i, ref_d = _run(torch, M.mknn_knn, cloud, Q, k, m)
        got_i, got_d = _run(torch, M.mknn_knn_noalloc, cloud, Q, k, m)
        assert np.array_equal(got_i, ref_i)
        real = ref_i >= 0
        assert np.all(np.abs(got_d[real] - ref_d[real]) <= 1e-6 * ref_d[real])
        assert np.all(np.isinf(got_d[~real]))
    assert cloud.check() == 0
    cloud.close()


def test_noalloc_at_its_limit_and_on_small_batches(torch_cuda):
    """A batch of exactly the limit fills the whole scratch array; tiny
    batches on a cloud with long successor lists take the wide lane
    variant and skip the locality sort, as mknn_knn does."""
    torch = torch_cuda
    P, _ = W.torus(50_000, 71)
    cloud = Cloud.build(P, W.permutation(50_000, 72)).upload()
    lo, hi = W.padded_box(P)
    limit = M.mknn_knn_noalloc_max_queries()
    Q = W.box_queries(limit, 73, lo, hi)
    ref_i, ref_d = _run(torch, M.mknn_knn, cloud, Q, 8, None)
    got_i, got_d = _run(torch, M.mknn_knn_noalloc, cloud, Q, 8, None)
    assert np.array_equal(got_i, ref_i) and np.array_equal(got_d, ref_d)
    cloud.close()
    Ph, _ = W.patches4(30_000, 61)
    hub = Cloud.build(Ph, W.permutation(30_000, 62)).upload()
    lo, hi = W.padded_box(Ph)
    for nq, k in ((1, 16), (100, 33), (4095, 5)):
        Q = W.box_queries(nq, 74 + nq, lo, hi)
        ref_i, ref_d = _run(torch, M.mknn_knn, hub, Q, k, None)
        got_i, got_d = _run(torch, M.mknn_knn_noalloc, hub, Q, k, None)
        assert np.array_equal(got_i, ref_i) and np.array_equal(got_d, ref_d)
    assert hub.check() == 0
    hub.close()


def test_noalloc_on_a_cloud_with_box_trees(torch_cuda):
    """On a cloud with box trees the call takes the one-warp kernel, which
    walks them (it has no scratch for the one-lane hand-over); rows equal
    mknn_knn's, for small and large batches."""
    torch = torch_cuda
    from tests.gpu_util import built_cloud
    n = 400_000
    P, _ = W.patches4(n, 21200)
    c = built_cloud(P, W.permutation(n, 21201), "patches400k")
    c.upload()
    assert c.trees()[0] > 0
    lo, hi = W.padded_box(P)
    for nq, k in ((100, 4), (5000, 8), (300_000, 4), (20_000, 48)):
        Q = W.box_queries(nq, 80 + nq % 97, lo, hi)
        ref_i, ref_d = _run(torch, M.mknn_knn, c, Q, k, None)
        got_i, got_d = _run(torch, M.mknn_knn_noalloc, c, Q, k, None)
        assert np.array_equal(got_i, ref_i) and np.array_equal(got_d, ref_d), (nq, k)
    assert c.check() == 0
    c.close()


def test_noalloc_rejects_batches_above_its_limit(torch_cuda):
    torch = torch_cuda
    wl = W.small_sphere(nq=1)
    cloud = Cloud.build(wl.points, wl.order).upload()
    limit = M.mknn_knn_noalloc_max_queries()
    assert limit == 1 << 20
    nq = limit + 1
    q = torch.zeros((nq, 3), dtype=torch.float32, device="cuda")
    idx = torch.empty((nq, 4), dtype=torch.int32, device="cuda")
    d2 = torch.empty((nq, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(M.MknnError) as ei:
        M.mknn_knn_noalloc(cloud.handle, q, nq, 3, 4, None, 0, idx, d2)
    assert ei.value.status == 1 and str(limit) in str(ei.value)
    cloud.close()
