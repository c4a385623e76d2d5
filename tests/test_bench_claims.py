"""What bench.py claims about a run, checked against the sources it
describes (CPU only): the metric's name, the query kernel's name, the
launches per step and per plan replay, and the traffic record's hash check."""
from __future__ import annotations

import json
import os
import re

import numpy as np
import pytest

import bench

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_2605_02224_gb300", "csrc")


def _read(name):
    with open(os.path.join(CSRC, name)) as f:
        return f.read()


def test_metric_name_follows_k_and_n():
    assert bench.metric_name(16, 1_000_000) == bench.METRIC
    assert "k=4," in bench.metric_name(4, 1_000_000)
    assert "0.25M-pt" in bench.metric_name(16, 250_000)


def test_query_kernel_name_matches_the_dispatch():
    """The one-lane dispatch picks 256/128/64-thread blocks with 1/2/4 flag
    words for k up to 32/64/128, and the list kind: 8 slots (k <= 8), the
    permutation list (k <= 16), k slots above."""
    src = _read("knn_plain.cu")
    assert "if (L.k <= 8) return run_smem<256, 32, 8, false>" in src
    assert "if (L.k <= 16) return run_smem<256, 32, 16, false>" in src
    assert "if (L.k <= 32) return run_smem<256, 32, 0, false>" in src
    assert "if (L.k <= 64) return run_smem<128, 64, 0, false>" in src
    assert "return run_smem<64, 128, 0, false>" in src
    assert "constexpr int W = KMAX / 32;" in src
    assert bench._query_kernel_name(0, 16, 0) == "knn_plain_smem_kernel<256, 1, 16, false>"
    assert bench._query_kernel_name(0, 4, 0) == "knn_plain_smem_kernel<256, 1, 8, false>"
    assert bench._query_kernel_name(0, 20, 0) == "knn_plain_smem_kernel<256, 1, 0, false>"
    assert bench._query_kernel_name(0, 33, 0) == "knn_plain_smem_kernel<128, 2, 0, false>"
    assert bench._query_kernel_name(1, 128, 2) == "knn_plain_smem_kernel<64, 4, 0, false>"
    # one warp per query from k = 48 by default, and for 32 lanes in shared memory
    hdr = _read("knn_kernels.h")
    assert f"constexpr int kWarpMinK = {bench.WARP_MIN_K};" in hdr
    assert "int default_lanes(int k) { return k >= kWarpMinK ? 32 : 1; }" in _read("knn_plain.cu")
    assert bench._query_kernel_name(0, 100, 0) == "knn_plain_warp_kernel<128, false>"
    assert bench._query_kernel_name(0, 48, 0) == "knn_plain_warp_kernel<64, false>"
    assert bench._query_kernel_name(32, 16, 2) == "knn_plain_warp_kernel<32, false>"
    assert bench._query_kernel_name(32, 16, 2, True) == "knn_plain_warp_kernel<32, true>"
    assert bench._query_kernel_name(0, 47, 0) == "knn_plain_smem_kernel<128, 2, 0, false>"
    # on a cloud with box trees the one-lane kernel hands queries over
    assert bench._query_kernel_name(1, 4, 2, True) == "knn_plain_smem_kernel<256, 1, 8, true>"
    assert bench._query_kernel_name(1, 16, 1) == "knn_plain_thread_kernel"
    assert bench._query_kernel_name(8, 16, 0).startswith("knn_plain_kernel<8")


def test_sort_launches_five_kernels():
    """A sorted step is the sort's five kernels plus the query kernel."""
    src = _read("query_sort.cu")
    body = src[src.index("cudaError_t launch_query_sort_split("):]
    assert len(re.findall(r"<<<", body)) == 5


def test_plan_variant_table_matches_the_library():
    src = _read("batch.cu")
    init = src[src.index("constexpr VariantDesc kVariants[] = {"):]
    init = init[:init.index("};")]
    table = [(int(a), int(b), int(c))
             for a, b, c in re.findall(r"\{(\d+),\s*(\d+),\s*(\d+)\}", init)]
    assert table == bench._PLAN_VARIANTS
    assert "reqs[r].nq < (o.sort > 0 ? 1 : 4096)" in src
    h = open(os.path.join(CSRC, "batch.h")).read()
    assert "constexpr int kWarpVariant32 = 16;" in h
    assert "constexpr int kTreeVariant32 = 19;" in h and bench._TREE_VARIANT32 == 19
    assert table[16:19] == [(32, 1, 2), (32, 2, 2), (32, 4, 2)]
    assert table[19:22] == table[16:19]
    assert "constexpr int kHandoverVariant = 22;" in h and bench._HANDOVER_VARIANT == 22
    assert table[22:24] == [table[12], table[15]] and len(table) == 24


def test_plan_launch_count():
    reqs = [dict(k=k, nq=nq) for k, nq in [(16, 20000), (32, 5000), (1, 100), (8, 3_000_000),
                                          (100, 9000)]]
    lanes = np.array([1, 32, 1, 1, 32])
    # one-lane segments of 16 slots (k = 16) and 8 slots (k = 1, 8), and the
    # warp kernels (32, 1), (32, 4) in shared memory; four requests of >= 4096
    # queries
    assert bench._plan_launches(lanes, reqs) == 4 + 5 * 4
    # registers for the 32-lane requests: (32, 1) and (32, 4) register groups
    assert bench._plan_launches(lanes, reqs, np.array([2, 1, 2, 2, 1])) == 4 + 5 * 4
    # one lane on clouds with box trees: the hand-over form and a one-warp
    # launch per hand-over class (k <= 32 here)
    reqs3 = [dict(k=4, nq=10), dict(k=16, nq=10), dict(k=4, nq=10)]
    assert bench._plan_launches(np.array([1, 1, 1]), reqs3, None, [True, True, False]) == 3 + 1
    # both placements at k = 32: two 32-lane variants
    lanes2 = np.array([32, 32])
    reqs2 = [dict(k=32, nq=10), dict(k=32, nq=10)]
    assert bench._plan_launches(lanes2, reqs2, np.array([1, 2])) == 2
    # one-warp lists on a cloud with box trees and on one without: two kernels
    assert bench._plan_launches(lanes2, reqs2, np.array([2, 2]), [True, False]) == 2
    assert bench._plan_launches(lanes2, reqs2, np.array([2, 2]), [True, True]) == 1


def test_traffic_record_is_used_only_for_its_own_sources():
    assert bench._profiled_traffic("not-a-hash", 1_000_000, 4_000_000) is None
    path = os.path.join(os.path.dirname(CSRC), "..", "profiles", "knn_plain_torus1m_traffic.json")
    with open(path) as f:
        rec = json.load(f)
    if rec["kernel_hash"] != bench._kernel_hash():
        pytest.skip("kernel sources changed since the record was taken")
    got = bench._profiled_traffic(rec["kernel_hash"], 1_000_000, 4_000_000)
    assert got == pytest.approx(rec["dram_bytes_per_query"] * 4_000_000)
    assert got == pytest.approx(rec["dram_bytes_read_per_launch"] +
                                rec["dram_bytes_write_per_launch"], rel=1e-3)


def _cache_worker(seed):
    import bench as b
    import workloads as W
    P, _ = W.sphere(3000, seed)
    c, _ = b._cloud_cache(P, np.arange(3000), "race")
    return int(c.stats()["entries"])


def test_cloud_cache_survives_concurrent_writers():
    """Processes that build the same cloud at once leave one complete cache
    file that loads back to the same table, and no temporary files."""
    import multiprocessing as mp
    import workloads as W
    P, _ = W.sphere(3000, 77)
    h = bench.hashlib.sha1(np.ascontiguousarray(P).tobytes() +
                           np.ascontiguousarray(np.arange(3000)).tobytes()).hexdigest()[:16]
    path = os.path.join("/tmp", "mknn_clouds", f"{h}.mknn")
    if os.path.exists(path):
        os.remove(path)
    with mp.get_context("spawn").Pool(3) as pool:
        entries = pool.map(_cache_worker, [77, 77, 77])
    assert len(set(entries)) == 1
    c, secs = bench._cloud_cache(P, np.arange(3000), "race")
    assert secs is None and int(c.stats()["entries"]) == entries[0]
    assert not [f for f in os.listdir(os.path.dirname(path)) if f.startswith(h) and
                f.endswith(".tmp")]


def test_algorithmic_bytes_and_roofline_fields():
    """The byte count per query is 12 (xyz) + 8 per row + 4 per entry + 12
    per coordinate + 8 k (output); the roofline reports the effective
    fraction against HBM and the fraction against the L2 probe."""
    assert bench._alg_bytes(3, 10, 11, 1, 4) == 12 + 24 + 40 + 132 + 32
    assert bench._alg_bytes(0, 0, 0, 2, 1, extra_per_query=4) == 2 * 16 + 16
    r = bench._roofline(1e9, 1.0, 1000, l2={"l2_read_gbs": 20000.0})
    assert r["achieved"] == pytest.approx(1000.0)
    assert r["frac"] == pytest.approx(1000.0 / r["peak"])
    assert r["frac_l2"] == pytest.approx(0.05)
    assert r["bound"] == "latency/divergence"
    assert bench._roofline(1e9, 1.0, 1000)["frac_l2"] is None


def test_oracle_pool_rate_on_a_tiny_sample():
    """The multi-process oracle timing runs the oracle as it stands on a
    spawn pool and counts the queries it answered."""
    import workloads as W
    P, _ = W.sphere(500, 3)
    Q = W.box_queries(200, 4, [-1.5] * 3, [1.5] * 3)
    rate, s, dt, cores = bench.oracle_rate(P, Q, 4, 0.2, cores=2)
    assert cores == 2 and 4 <= s <= 196 and rate > 0 and dt > 0
