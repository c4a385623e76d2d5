"""Dynamic clouds on the device: queries after appends equal queries on a
cloud built once over the same points, old prefixes are unchanged, the
device arrays grow, and plans and servers see the change safely."""
from __future__ import annotations

import numpy as np
import pytest

import workloads as W
from paper_2605_02224_gb300 import Cloud
from paper_2605_02224_gb300 import mknn as M
from tests import parity
from tests.gpu_util import run_knn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def _points(n, seed=5):
    P, _ = W.torus(n, seed)
    return np.ascontiguousarray(P[W.permutation(n, seed + 1)], np.float32)


def test_appends_equal_one_build_on_the_device(torch):
    """2,000 sites uploaded, then 100, 1,900 and 16,000 more appended (the
    site and entry arrays outgrow their headroom and move): after every
    append the rows equal those of a cloud built once over the same points,
    and queries bounded by the old n return exactly what they did before."""
    Pr = _points(20000)
    Q = W.box_queries(3000, 7, [-1.5, -1.5, -0.5], [1.5, 1.5, 0.5])
    c = Cloud.build(Pr[:2000], dynamic=True).upload()
    bytes0 = c.device_bytes()
    before = run_knn(c, Q, 16)
    at = 2000
    for step in (100, 1900, 16000):
        c.append(Pr[at:at + step])
        at += step
        ref = Cloud.build(Pr[:at]).upload()
        for k in (1, 16, 100):
            a = run_knn(c, Q, k)
            b = run_knn(ref, Q, k)
            assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]), (at, k)
        old = run_knn(c, Q, 16, 2000)                 # m = the first upload's n
        assert np.array_equal(old[0], before[0]) and np.array_equal(old[1], before[1])
        ref.close()
    assert c.device_bytes() > bytes0
    a = run_knn(c, Q, 16)
    c.compact()
    b = run_knn(c, Q, 16)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    c.append(Pr[:0])
    idx, d2 = run_knn(c, Q, 16)
    parity.check_rows(Pr, Q, 16, 0, idx, d2, rows=range(0, 3000, 10))
    m = np.clip(np.floor(np.exp(W.uniform(8, 1, 3000) * np.log(20000))), 1, 20000)
    idx, d2 = run_knn(c, Q, 8, m.astype(np.int32))
    parity.check_rows(Pr, Q, 8, m.astype(np.int32), idx, d2, rows=range(0, 3000, 10))
    assert c.check() == 0
    c.close()


def test_site_queries_reach_appended_sites(torch):
    Pr = _points(6000, 11)
    c = Cloud.build(Pr[:3000], dynamic=True).upload()
    c.append(Pr[3000:])
    sites = np.arange(2900, 3100, dtype=np.int32)
    st = torch.from_numpy(sites).cuda()
    idx, d2 = c.knn_sites(st, 12)
    torch.cuda.synchronize()
    idx, d2 = idx.cpu().numpy(), d2.cpu().numpy()
    assert np.array_equal(idx[:, 0], sites)
    parity.check_rows(Pr, Pr[sites], 12, 0, idx, d2)
    c.close()


def test_plans_refuse_a_changed_cloud_and_servers_block_appends(torch):
    Pr = _points(8000, 21)
    c = Cloud.build(Pr[:6000], dynamic=True).upload()
    q = torch.from_numpy(W.box_queries(500, 3, [-1.2] * 3, [1.2] * 3)).cuda()
    out_i = torch.empty((500, 8), dtype=torch.int32, device="cuda")
    out_d = torch.empty((500, 8), dtype=torch.float32, device="cuda")
    req = dict(cloud=c.handle, q=q, nq=500, q_stride=3, k=8, m=None, m_scalar=0,
               out_idx=out_i, out_d2=out_d)
    plan = M.mknn_batch_create([req])
    s = torch.cuda.current_stream().cuda_stream
    M.mknn_batch_run(plan, s)
    c.append(Pr[6000:7000])
    with pytest.raises(M.MknnError) as ei:
        M.mknn_batch_run(plan, s)
    assert ei.value.status == 1
    M.mknn_batch_free(plan)
    plan = M.mknn_batch_create([req])
    M.mknn_batch_run(plan, s)
    torch.cuda.synchronize()
    ri, rd = c.knn(q, 8)
    torch.cuda.synchronize()
    assert torch.equal(ri, out_i) and torch.equal(rd, out_d)
    M.mknn_batch_free(plan)
    srv = M.mknn_server_create(slots=1)
    M.mknn_server_add_cloud(srv, c.handle)
    with pytest.raises(M.MknnError) as ei:
        c.append(Pr[7000:])
    assert ei.value.status == 4                        # EBUSY
    M.mknn_server_destroy(srv, 30.0)
    c.append(Pr[7000:])
    assert M.mknn_cloud_info(c.handle)[0] == 8000
    c.close()
