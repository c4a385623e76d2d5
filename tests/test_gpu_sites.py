"""Same-manifold queries (each query one of the cloud's own sites) through
the C ABI, against the oracle and against mknn_knn on the same coordinates."""
from __future__ import annotations

import numpy as np
import pytest

import workloads as W
from paper_2605_02224_gb300 import Cloud
from paper_2605_02224_gb300 import mknn as M
from tests import parity
from tests.gpu_util import built_cloud, run_knn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def _sites(torch, c, sites, k, m=None, **opt):
    st = torch.from_numpy(np.ascontiguousarray(sites, np.int32)).cuda()
    mt = m
    if m is not None and not isinstance(m, int):
        mt = torch.from_numpy(np.ascontiguousarray(m, np.int32)).cuda()
    idx, d2 = c.knn_sites(st, k, mt, **opt)
    torch.cuda.synchronize()
    return idx.cpu().numpy(), d2.cpu().numpy()


def test_every_site_of_the_small_sphere(torch):
    """All 2,000 sites as queries (normal-estimation style), k = 8 and 16:
    rows equal the oracle's for the sites' coordinates, the first neighbour
    is the site itself at distance 0, and the rows equal mknn_knn on the
    same coordinates bit for bit."""
    wl = W.small_sphere(nq=10)
    c = Cloud.build(wl.points, wl.order).upload()
    Pr = wl.ranked_points()
    sites = W.permutation(2000, 9).astype(np.int32)      # every rank, shuffled
    for k in (8, 16):
        idx, d2 = _sites(torch, c, sites, k)
        parity.check_rows(Pr, Pr[sites], k, 0, idx, d2)
        assert np.array_equal(idx[:, 0], sites) and np.all(d2[:, 0] == 0.0)
        ri, rd = run_knn(c, Pr[sites], k)
        assert np.array_equal(idx, ri) and np.array_equal(d2, rd)
    assert c.check() == 0
    c.close()


def test_sites_with_prefix_bounds_and_large_k(torch):
    """Sites probed across prefixes (the temporal setting of Sec. 5): per
    query m log-uniform in [1, n], k in {10, 100}; rows against the oracle.
    A site at or above its m is not a candidate of its own query."""
    P, _ = W.bumpy_sphere(20000, 31)
    order = W.permutation(20000, 32)
    c = built_cloud(P, order, "bumpy20k")
    c.upload()
    Pr = P[order]
    nq = 900
    sites = (W.uniform(51, 1, nq) * 20000).astype(np.int32)
    m = np.clip(np.floor(np.exp(W.uniform(52, 1, nq) * np.log(20000))), 1, 20000).astype(np.int32)
    for k in (10, 100):
        idx, d2 = _sites(torch, c, sites, k, m)
        parity.check_row_properties(idx, d2, k, m.astype(np.int64), 20000)
        parity.check_rows(Pr, Pr[sites], k, m, idx, d2, rows=range(0, nq, 2))
        inside = sites < m
        assert np.array_equal(idx[inside, 0], sites[inside])
        assert not np.any(idx[~inside] == sites[~inside, None])
    c.close()


def test_duplicate_sites_tie_to_the_earlier_twin(torch):
    """Exact duplicates: the query at a later twin finds the earlier twin
    first (distance 0, lower rank), then itself."""
    P, _ = W.lattice(8)
    P = np.concatenate([P, P[:100]])
    n = P.shape[0]
    order = W.permutation(n, 77)
    c = Cloud.build(P, order).upload()
    Pr = P[order]
    sites = np.arange(n, dtype=np.int32)
    for k in (1, 2, 9, 27):
        idx, d2 = _sites(torch, c, sites, k)
        parity.check_rows(Pr, Pr[sites], k, 0, idx, d2)
    # ranks of the duplicated coordinates: the lower one comes first
    idx, d2 = _sites(torch, c, sites, 2)
    key = {tuple(p): [] for p in Pr.tolist()}
    for r, p in enumerate(Pr.tolist()):
        key[tuple(p)].append(r)
    twins = [v for v in key.values() if len(v) == 2]
    assert len(twins) == 100
    for a, b in twins:
        assert list(idx[b]) == [a, b] and list(d2[b]) == [0.0, 0.0]
    c.close()


def test_bad_site_ranks_pad_and_flag(torch):
    wl = W.small_sphere(nq=10)
    c = Cloud.build(wl.points, wl.order).upload()
    sites = np.array([0, 5, -1, 1999, 2000, 7], np.int32)
    idx, d2 = _sites(torch, c, sites, 4)
    for bad in (2, 4):
        assert np.all(idx[bad] == -1) and np.all(np.isinf(d2[bad]))
    assert c.check() & 1
    assert c.check() == 0
    parity.check_rows(wl.ranked_points(), wl.ranked_points()[sites[[0, 1, 3, 5]]], 4, 0,
                      idx[[0, 1, 3, 5]], d2[[0, 1, 3, 5]])
    with pytest.raises(M.MknnError):
        _sites(torch, c, sites, 129)
    c.close()


def test_caller_workspace_and_sort_options(torch):
    wl = W.small_sphere(nq=10)
    c = Cloud.build(wl.points, wl.order).upload()
    sites = np.tile(np.arange(2000, dtype=np.int32), 4)         # 8,000 queries: sorted
    need = M.mknn_knn_sites_workspace_size(sites.size)
    assert need >= 20 * sites.size
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    a = _sites(torch, c, sites, 8, workspace=ws, workspace_bytes=need)
    b = _sites(torch, c, sites, 8, sort=-1)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    with pytest.raises(M.MknnError):
        _sites(torch, c, sites, 8, workspace=ws, workspace_bytes=need - 256)
    c.close()
