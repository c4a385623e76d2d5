#!/usr/bin/env python3
"""Exact k-NN queries/sec on the 1M-point torus (4M volume queries, k = 16).

One step = one pass of the query path over the whole batch: the locality
order of the 4M queries (five small kernels) and the k-NN kernel
(Algorithm 1 descent + Algorithm 2 expansion), inputs resident in HBM.
L2 is flushed (a 256 MB write) before every timed step, outside the timed
events. Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Beside the headline the default single-GPU run reports, each with its own
clock samples: the same step without the locality sort, a k sweep
(k = 4, 32, 100), the prefix workload (4M-point bumpy sphere, 8M queries,
per-query m), the batching workload (64 clouds, one persistent plan against
one plain launch per cloud), the serving loop (16 resident clouds, Poisson
arrivals), an L2 read-bandwidth probe for the roofline, and the CPU
baselines on the host cores (the float64 oracle on a sample, the kd-tree
and Algorithms 1-2 on the host).

--impl reference times the float64 brute-force oracle on all host cores
on a bounded sample of the same workload (the slow reference arm).
Under torchrun each rank runs the same independent batch on its own GPU
(weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "k-NN queries/sec (k=16, 1M-pt surface, volume queries) + served p50/p99 vs plain"


def metric_name(k: int, n: int) -> str:
    """The headline metric's name for the k and cloud size actually run."""
    return METRIC.replace("k=16", f"k={k}").replace("1M-pt", f"{n / 1e6:g}M-pt")
UNIT = "queries/s"
KERNEL_SOURCES = ["paper_2605_02224_gb300/csrc/knn_device.cuh",
                  "paper_2605_02224_gb300/csrc/knn_plain.cu"]


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--lanes", type=int, default=0)
    ap.add_argument("--nq", type=int, default=4_000_000)
    ap.add_argument("--k", type=int, default=16)
    ap.add_argument("--blocks-per-sm", type=int, default=0,
                    help="resident query blocks per SM (0 = as many as fit)")
    ap.add_argument("--placement", type=int, default=0,
                    help="one-lane candidate lists: 0 default, 1 registers, 2 shared memory")
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sort", action="store_true", help="process queries in input order")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving section")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--scale", type=float, default=1.0,
                    help="size factor of the prefix, batching and serving workloads (1 = as "
                         "specified; smaller only for trying the benchmark out)")
    ap.add_argument("--quick", action="store_true",
                    help="headline only: no sort ablation, k sweep, prefix, batching or CPU baselines")
    ap.add_argument("--workload", default="torus",
                    choices=["torus", "batch", "prefix", "sites", "dynamic", "sweep", "orders"])
    ap.add_argument("--append-batch", type=int, default=10000,
                    help="dynamic workload: points per append call")
    return ap.parse_args()


def _dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


WARP_MIN_K = 48   # from this k the library's default is one warp per query


def _query_kernel_name(lanes: int, k: int, placement: int, trees: bool = False) -> str:
    """The query kernel a plain launch with these options runs (its default:
    one lane per query with the list in shared memory, one warp per query
    with the warp's list in shared memory from k = 48; the one-warp kernel's
    second form walks the box trees of a cloud that has them)."""
    if (lanes == 0 and k >= WARP_MIN_K) or (lanes == 32 and placement in (0, 2)):
        kc = 32 if k <= 32 else (64 if k <= 64 else 128)
        return f"knn_plain_warp_kernel<{kc}, {'true' if trees else 'false'}>"
    if lanes in (0, 1) and placement in (0, 2):
        threads, words = (256, 1) if k <= 32 else ((128, 2) if k <= 64 else (64, 4))
        kind = 8 if k <= 8 else (16 if k <= 16 else 0)
        return f"knn_plain_smem_kernel<{threads}, {words}, {kind}, {'true' if trees else 'false'}>"
    if lanes in (0, 1):
        return "knn_plain_thread_kernel"
    return f"knn_plain_kernel<{lanes}, S>"


def _kernel_hash():
    h = hashlib.sha1()
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:12]


def _profiled_traffic(khash: str, n: int, nq: int):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source (same hash) and scales to this launch."""
    path = os.path.join(ROOT, "profiles", "knn_plain_torus1m_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except Exception:
        return None
    if rec.get("kernel_hash") != khash:
        return None
    per_q = rec.get("dram_bytes_per_query")
    if per_q is None:
        return None
    return float(per_q) * nq


class Clocks:
    """nvidia-smi samples every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            if len(r) < 9:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def _profile_record(khash: str):
    """The committed ncu record of the headline kernel (launch-list traffic
    and the section-set figures), if taken on the current kernel sources."""
    path = os.path.join(ROOT, "profiles", "knn_plain_torus1m_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except Exception:
        return None
    return rec if rec.get("kernel_hash") == khash else None


def _clocked(local: int, fn):
    """Runs fn() with nvidia-smi clock samples taken around it."""
    ck = Clocks(local)
    ck.start()
    time.sleep(0.3)
    try:
        out = fn()
    finally:
        time.sleep(0.2)
        clk = ck.stop()
    return out, clk


def _timed_ms(torch, stream, fn, steps: int, warmup: int, flush):
    """CUDA-event times (ms) of `steps` calls of fn on `stream`, each after
    an L2 flush outside the events, after max(3, warmup) untimed calls."""
    for _ in range(max(3, warmup)):
        fn()
    torch.cuda.synchronize()
    ms = []
    for i in range(steps):
        flush.fill_(float(i))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    return ms


def l2_probe(M, torch, dev, stream):
    """L2 read bandwidth: buffers of a quarter and half of the L2 size
    (two allocations each, since the placement across the L2 partitions
    varies) read 50 times per launch with 16-byte loads through L2
    (mknn_read_probe), best of 5 launches each; the best overall."""
    l2 = int(getattr(torch.cuda.get_device_properties(dev), "L2_cache_size", 0) or 0)
    if l2 <= 0:
        return None
    s = stream.cuda_stream
    passes = 50
    sink = torch.zeros(1, dtype=torch.int32, device=dev)
    best, per = 0.0, []
    for frac in (4, 2, 4, 2):
        nbytes = (l2 // frac) // 16 * 16
        buf = torch.ones(nbytes // 4, dtype=torch.int32, device=dev)
        M.mknn_read_probe(buf, nbytes, 2, sink, s)          # bring the buffer into L2
        b = 0.0
        for _ in range(5):
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            M.mknn_read_probe(buf, nbytes, passes, sink, s)
            ev1.record(stream)
            torch.cuda.synchronize()
            b = max(b, nbytes * passes / (ev0.elapsed_time(ev1) / 1e3) / 1e9)
        per.append({"buffer_bytes": nbytes, "gbs": b})
        best = max(best, b)
        del buf
    return {"l2_read_gbs": best, "l2_bytes": l2, "passes": passes, "runs": per,
            "how": "mknn_read_probe: 16-byte loads through L2 over buffers of 1/4 and 1/2 of "
                   "the L2 size (two allocations each), 50 passes per launch, best of 5 "
                   "launches each (CUDA events); the best overall"}


def _alg_bytes(rows, entries, coords, nq, k, extra_per_query=0):
    """Algorithmic bytes of a launch: 12 B per query (xyz) + 8 per row
    opened (row bounds) + 4 per successor entry + 12 per site coordinate
    read + 8 k per query (output), plus extra_per_query (e.g. a prefix
    bound)."""
    return (12 + extra_per_query) * nq + 8 * rows + 4 * entries + 12 * coords + 8 * k * nq


def _roofline(alg_bytes, kern_ms, nq, l2=None, rec=None, kernel=None, counts=None):
    peak, kind = _peaks()
    achieved = alg_bytes / (kern_ms / 1e3) / 1e9
    out = {"bound": "latency/divergence", "achieved": achieved, "peak": peak, "unit": "GB/s",
           "frac": achieved / peak,
           "frac_kind": "effective: algorithmic bytes / kernel time, against the measured HBM "
                        "copy bandwidth (most of the bytes are served by L1/L2, not DRAM)",
           "peak_source": f"{kind} hbm_gbs (MEASURED_PEAKS.json)",
           "l2_peak_gbs": (l2 or {}).get("l2_read_gbs"),
           "frac_l2": achieved / l2["l2_read_gbs"] if l2 else None,
           "kernel": kernel, "kernel_ms": kern_ms, "alg_bytes_per_launch": alg_bytes,
           "alg_bytes_per_query": alg_bytes / nq}
    if counts is not None:
        out["counts_per_query"] = counts
    if rec is not None:
        out["threads_per_inst"] = rec.get("threads_per_inst")
        out["issue_active"] = rec.get("issue_active_pct")
        out["profile_kernel_hash"] = rec.get("kernel_hash")
    return out


def _counts(M, torch, cloud, q, nq, k, m, stream, order=None, sort_flag=0, sites=None):
    """Per-launch totals of rows opened, entries read, coordinates read and
    transition sites, from the counting kernel (untimed)."""
    dev = q.device if sites is None else sites.device
    idx = torch.empty((nq, k), dtype=torch.int32, device=dev)
    d2 = torch.empty((nq, k), dtype=torch.float32, device=dev)
    cnt = torch.zeros((nq, 4), dtype=torch.int32, device=dev)
    lanes = 32 if k > 64 else 1
    if sites is not None:
        M.mknn_knn_sites(cloud.handle, sites, nq, k, m, 0, idx, d2, stream, counters=cnt,
                         lanes=lanes)
    else:
        M.mknn_knn_ex(cloud.handle, q, nq, 3, k, m, 0, idx, d2, stream, order=order,
                      sort=sort_flag, counters=cnt, lanes=lanes)
    torch.cuda.synchronize()
    rows, entries, coords, trans = (int(x) for x in cnt.to(torch.int64).sum(dim=0).cpu().numpy())
    del idx, d2, cnt
    return rows, entries, coords, trans


def _cloud_cache(points, order, tag):
    from paper_2605_02224_gb300 import Cloud
    d = os.path.join("/tmp", "mknn_clouds")
    os.makedirs(d, exist_ok=True)
    h = hashlib.sha1(np.ascontiguousarray(points).tobytes() +
                     np.ascontiguousarray(order).tobytes()).hexdigest()[:16]
    path = os.path.join(d, f"{h}.mknn")
    if os.path.exists(path):
        try:
            return Cloud.load(path), None
        except Exception:
            os.remove(path)
    t0 = time.perf_counter()
    c = Cloud.build(points, order)
    secs = time.perf_counter() - t0
    # written under a name of this process's own, then renamed into place: ranks
    # that build the same cloud at once never see (or leave) a half-written file
    tmp = f"{path}.{os.getpid()}.tmp"
    c.save(tmp)
    os.replace(tmp, path)
    return c, secs


_ORACLE_P = None


def _oracle_init(P):
    global _ORACLE_P
    _ORACLE_P = P


def _oracle_noop(_):
    import oracle.knn  # noqa: F401  (imported once per worker before timing)
    return 0


def _oracle_chunk(args):
    import oracle.knn as ok
    Q, k = args
    for q in Q:
        ok.knn_one(_ORACLE_P, q, k, _ORACLE_P.shape[0])
    return int(Q.shape[0])


class OraclePool:
    """Host processes that run the float64 brute-force oracle, as it
    stands, on the points P (a spawn pool, so it is safe after CUDA is
    initialised; workers are started and have imported the oracle before
    any timing)."""

    def __init__(self, P, cores: int | None = None):
        import multiprocessing as mp
        self.cores = cores or os.cpu_count() or 1
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_oracle_init,
                                                 initargs=(P,))
        self.pool.map(_oracle_noop, range(self.cores))

    def rate(self, Q, k, seconds: float):
        """Queries/s over a bounded sample of Q: the first queries, sized
        from a short probe to about `seconds` of work on all workers.
        Returns (rate, queries, seconds)."""
        probe = 4
        t0 = time.perf_counter()
        self.pool.apply(_oracle_chunk, ((Q[:probe], k),))
        per_q = (time.perf_counter() - t0) / probe
        s = int(max(2 * self.cores,
                    min(Q.shape[0] - probe, seconds * self.cores / max(per_q, 1e-6))))
        chunks = np.array_split(Q[probe:probe + s], 4 * self.cores)
        t0 = time.perf_counter()
        done = sum(self.pool.map(_oracle_chunk, [(c, k) for c in chunks if c.shape[0]]))
        return done / (time.perf_counter() - t0), done, time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()


def oracle_rate(P, Q, k, seconds: float, cores: int | None = None):
    """OraclePool(P).rate(...) in one call. Returns (rate, queries, seconds, cores)."""
    op = OraclePool(P, cores)
    try:
        r, s, dt = op.rate(Q, k, seconds)
    finally:
        op.close()
    return r, s, dt, op.cores


def _cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baselines(P, rowp, succ, Q, k, oracle_seconds: float, single_sample: int = 100_000):
    """The CPU baselines on this host's cores, in this run: the float64
    oracle (all cores, a sample), the project's kd-tree and Algorithms 1-2
    on the host (all cores on every query; one core on a sample). The
    kd-tree and the host restatement both process the queries in Morton
    order (the sort is inside the timing) and compute in float64."""
    import cpu
    cpu.build()
    model = _cpu_model()
    nq = Q.shape[0]
    rate, s, dt, cores = oracle_rate(P, Q, k, oracle_seconds)
    threads = cpu.threads()
    out = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"first {s} queries of the workload, float64 brute force over all "
                     f"{P.shape[0]} sites, {cores} host processes, {dt:.1f} s",
           "cpu_model": model, "others": []}
    t0 = time.perf_counter()
    tree = cpu.KDTree(P)
    kd_build = time.perf_counter() - t0
    ref = None
    for name, fn in (("kd-tree (exact, prefix-aware, float64)",
                      lambda QQ, th: tree.knn(QQ, k, threads=th)),
                     ("Algorithms 1-2 on the host (float64, successor table)",
                      lambda QQ, th: cpu.dpknn(P, rowp, succ, QQ, k, threads=th))):
        for th, QQ, label in ((0, Q, f"all {nq} queries"),
                              (1, Q[:single_sample], f"first {min(nq, single_sample)} queries")):
            t0 = time.perf_counter()
            idx, _ = fn(QQ, th)
            dt = time.perf_counter() - t0
            entry = {"kind": name, "value": QQ.shape[0] / dt, "unit": UNIT,
                     "cores": threads if th == 0 else 1,
                     "sample": f"{label}, Morton order, {dt:.2f} s", "cpu_model": model}
            if th == 0:
                if ref is None:
                    ref = idx
                else:
                    entry["same_ranks_as_kd_tree"] = bool(np.array_equal(idx, ref))
            out["others"].append(entry)
    out["kd_tree_build_seconds"] = kd_build
    tree.close()
    return out


def run_reference(args, rank, world):
    """The reference arm: the oracle as it stands on the host cores, each
    step a bounded sample of the headline workload's queries."""
    if rank != 0:
        return
    import workloads as W
    wl = W.large_torus(n=args.n, nq=args.nq, k=args.k)
    P = wl.ranked_points()
    rates = []
    t_all = time.perf_counter()
    total_q = 0
    op = OraclePool(P)
    cores = op.cores
    for step in range(args.warmup + args.steps):
        Q = wl.queries[(step * 9973) % max(1, wl.nq - 100000):]
        r, s, dt = op.rate(Q, wl.k, seconds=args.cpu_seconds / 4)
        if step >= args.warmup:
            rates.append(r)
            total_q += s
    op.close()
    value = float(np.median(rates))
    line = {
        "impl": "reference", "metric": metric_name(args.k, args.n), "value": value,
        "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wl.nq / value,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"torus R=1 r=0.3 sigma=1e-4, n={wl.n}, {wl.nq} box queries, k={wl.k}",
                   "n": wl.n, "nq": wl.nq, "k": wl.k, "m": "n"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{total_q} queries of the workload over {args.steps} steps "
                                   f"(float64 brute force, {cores} host processes); "
                                   f"ms_per_step extrapolated to all {wl.nq} queries",
                         "cpu_model": _cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": time.perf_counter() - t_all,
    }
    print(json.dumps(line), flush=True)


def max_over_ranks(x: float, dist=None, device=None) -> float:
    """The largest x over all ranks (the slowest rank sets the job time);
    x itself with no process group."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(total_ms: float, steps: int, nq_per_rank: int, world: int):
    """(ms per step, whole-job queries/s): every rank answers its own nq
    queries per step (weak scaling), the job takes the slowest rank's time."""
    ms_per_step = total_ms / steps
    return ms_per_step, world * nq_per_rank / (ms_per_step / 1e3)


def _build_many(wls, tag):
    """Builds (or loads cached builds of) several clouds in parallel host threads."""
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as ex:
        res = list(ex.map(lambda w: _cloud_cache(w.points, w.order, f"{tag}-{w.n}"), wls))
    built = [r[1] for r in res if r[1] is not None]
    return [r[0] for r in res], (max(built) if built else None)


def serving_section(args, M, torch, built=None):
    """Serving workload: 16 resident clouds (100k-4M sites, mixed surfaces),
    Poisson arrivals at 0.5 / 0.8 / 0.95 / 1.5 of the plain path's
    saturation rate; each request 1..65536 queries, k in 1..64, m in
    [n/10, n]. The batched server (continuous batching, persistent kernel)
    against the baseline that runs each request alone with the plain
    kernel, in arrival order, on one stream. Same request sequence for
    every run (arrival times scaled). Per load: requests per launch,
    p50/p99 latency, and the GPU time of each launch phase per request."""
    import workloads as W
    wls, clouds, build_s = (built if built is not None
                            else (W.serve_clouds(scale=args.scale), None, None))
    if clouds is None:
        clouds, build_s = _build_many(wls, "serve")
    for c in clouds:
        c.upload()
    n_req = args.serve_requests
    reqs = W.serve_requests(wls, n_req, 1.0, seed=42)
    bufs = []
    for r in reqs:
        q = torch.from_numpy(r.queries).pin_memory()
        bufs.append((q, torch.empty((r.queries.shape[0], r.k), dtype=torch.int32).pin_memory(),
                     torch.empty((r.queries.shape[0], r.k), dtype=torch.float32).pin_memory()))
    total_q = int(sum(r.queries.shape[0] for r in reqs))

    def run(plain: int, rate):
        srv = M.mknn_server_create(slots=1 if plain else 3, plain=plain, mem_budget=4 << 30)
        ids = [M.mknn_server_add_cloud(srv, c.handle) for c in clouds]
        for r, (q, oi, od) in list(zip(reqs, bufs))[:8]:            # warm-up
            M.mknn_server_submit(srv, ids[r.cloud], q, r.k, r.m, oi, od)
        M.mknn_server_drain(srv, 300.0)
        M.mknn_server_reset_stats(srv)
        t0 = time.perf_counter()
        for r, (q, oi, od) in zip(reqs, bufs):
            if rate is not None:
                delay = r.arrival_s / rate - (time.perf_counter() - t0)
                if delay > 0:
                    time.sleep(delay)
            M.mknn_server_submit(srv, ids[r.cloud], q, r.k, r.m, oi, od)
        M.mknn_server_drain(srv, 600.0)
        st = M.mknn_server_stats(srv)
        M.mknn_server_destroy(srv, 60.0)
        done = max(1, st["completed"])
        return {"qps": st["qps"], "rps": st["completed"] / max(st["elapsed_s"], 1e-9),
                "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "mean_ms": st["mean_ms"],
                "launches": st["launches"],
                "requests_per_launch": st["mean_requests_per_launch"],
                "gpu_ms_per_request": {"h2d": st["h2d_ms"] / done,
                                       "kernel": st["kernel_ms"] / done,
                                       "d2h": st["d2h_ms"] / done}}

    def measure():
        sat_plain = run(1, None)
        sat_batched = run(0, None)
        loads = []
        for f in (0.5, 0.8, 0.95, 1.5):
            rate = f * sat_plain["rps"]
            loads.append({"offered": f, "rate_rps": rate, "batched": run(0, rate),
                          "plain": run(1, rate)})
        return sat_plain, sat_batched, loads

    (sat_plain, sat_batched, loads), clk = _clocked(torch.cuda.current_device(), measure)
    del bufs
    return {
        "workload": f"16 resident clouds ({sum(w.n for w in wls)} sites, 100k-4M, mixed "
                    f"surfaces); {n_req} requests, {total_q} queries, Poisson arrivals",
        "build_seconds_max": build_s if build_s is not None else "cached",
        "saturation": {"plain": sat_plain, "batched": sat_batched},
        "loads": loads,
        "phase_times": "GPU time per request of each launch phase (stream time between "
                       "events, summed over launches / requests): host-to-device copies, "
                       "kernels (locality sorts + k-NN), device-to-host copies",
        "clocks": clk,
    }


# (lanes, slots per lane, list placement) of the persistent kernels, as the
# library's plans pick them (placement 2: shared memory, 1: registers)
_PLAN_VARIANTS = [(4, 1, 1), (4, 2, 1), (4, 4, 1), (8, 1, 1), (8, 2, 1), (8, 4, 1), (8, 8, 1),
                  (16, 1, 1), (16, 2, 1), (16, 4, 1), (32, 1, 1), (32, 2, 1), (1, 64, 2),
                  (16, 8, 1), (32, 4, 1), (1, 128, 2), (32, 1, 2), (32, 2, 2), (32, 4, 2),
                  (32, 1, 2), (32, 2, 2), (32, 4, 2), (1, 64, 2), (1, 128, 2)]
# index of the first one-warp variant with box trees, and of the one-lane
# variants that hand queries over to it (plans on clouds with trees)
_TREE_VARIANT32 = 19
_HANDOVER_VARIANT = 22


def _plan_launches(lanes, reqs, placement=None, trees=None) -> int:
    """Kernels one plan replay launches: the locality sort's five per request
    of at least 4096 queries, one persistent kernel per (variant, list class)
    present (the fewest slots per lane that hold the request's k; one-lane
    segments are cut by list class: 8, 16, 32, 64 slots; on clouds with box
    trees, trees[i], a one-warp variant has a tree form and a one-lane
    variant a hand-over form), and one one-warp launch per hand-over class
    (k <= 32, <= 64, <= 128) present."""
    segs, handover = set(), set()
    placement = placement if placement is not None else [2 if g in (1, 32) else 1 for g in lanes]
    trees = trees if trees is not None else [False] * len(reqs)
    for g, p, r, t in zip(lanes.tolist() if hasattr(lanes, "tolist") else lanes,
                          placement.tolist() if hasattr(placement, "tolist") else placement,
                          reqs, trees):
        lst = 2 if g == 1 else (p if g == 32 else 1)
        fits = [i for i, v in enumerate(_PLAN_VARIANTS[:_TREE_VARIANT32])
                if v[0] == g and v[2] == lst and v[0] * v[1] >= r["k"]]
        v = min(fits, key=lambda i: _PLAN_VARIANTS[i][1])
        cls = 0
        if g == 1:
            slots = 8 if r["k"] <= 8 else (16 if r["k"] <= 16 else r["k"])
            cls = 0 if slots <= 8 else (1 if slots <= 16 else (2 if slots <= 32 else 3))
        if t and g == 32 and lst == 2:
            v += _TREE_VARIANT32 - 16
        if t and g == 1:
            v = _HANDOVER_VARIANT + (1 if v == 15 else 0)
            handover.add(0 if r["k"] <= 32 else (1 if r["k"] <= 64 else 2))
        segs.add((v, cls))
    return len(segs) + len(handover) + 5 * sum(1 for r in reqs if r["nq"] >= 4096)


def batch_section(args, M, torch, built=None):
    """Batching workload: 64 clouds (log-uniform 10k-2M sites, mixed
    surfaces), 2n queries per cloud, k from {1,4,8,16,32}; the tuned
    persistent plan (one launch per kernel variant, graph replay) against
    one plain launch per cloud in sequence on one stream. Per-request
    latency: a request of the plan completes with the plan; a plain request
    completes with its own launch (CUDA events after each)."""
    import workloads as W
    wls, clouds, build_s = (built if built is not None
                            else (W.batch_clouds(scale=args.scale), None, None))
    if clouds is None:
        clouds, build_s = _build_many(wls, "batch")
    dev = torch.device("cuda", torch.cuda.current_device())
    reqs = []
    for wl, c in zip(wls, clouds):
        c.upload()
        q = torch.from_numpy(wl.queries).to(dev)
        reqs.append(dict(cloud=c.handle, q=q, nq=wl.nq, q_stride=3, k=wl.k, m=None, m_scalar=0,
                         out_idx=torch.empty((wl.nq, wl.k), dtype=torch.int32, device=dev),
                         out_d2=torch.empty((wl.nq, wl.k), dtype=torch.float32, device=dev)))
    stream = torch.cuda.current_stream(dev)
    s = stream.cuda_stream
    t0 = time.perf_counter()
    M.mknn_batch_tune(reqs, 1 << 16, s)
    tune_s = time.perf_counter() - t0
    plan = M.mknn_batch_create(reqs)
    lanes, items, grid = M.mknn_batch_info(plan, len(reqs))
    placement = M.mknn_batch_placement(plan, len(reqs))
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    nq = int(sum(r["nq"] for r in reqs))
    # algorithmic bytes of one pass over every request (counting kernel, untimed)
    alg = 0
    for wl, c, r in zip(wls, clouds, reqs):
        rows, entries, coords, _ = _counts(M, torch, c, r["q"], r["nq"], r["k"], None, s)
        alg += _alg_bytes(rows, entries, coords, r["nq"], r["k"])

    def plain():
        for r in reqs:
            M.mknn_knn(r["cloud"], r["q"], r["nq"], 3, r["k"], None, 0, r["out_idx"],
                       r["out_d2"], s)

    def measure():
        # an NVTX range around the plan's launches, so that a profiler can
        # select them apart from the tuner's (ncu --nvtx --nvtx-include batch_plan/)
        torch.cuda.nvtx.range_push("batch_plan")
        ms_batch = _timed_ms(torch, stream, lambda: M.mknn_batch_run(plan, s), args.steps,
                             args.warmup, flush)
        torch.cuda.nvtx.range_pop()
        ref = [r["out_idx"].clone() for r in reqs]
        ms_plain = _timed_ms(torch, stream, plain, args.steps, args.warmup, flush)
        same = all(torch.equal(a, r["out_idx"]) for a, r in zip(ref, reqs))
        # per-request completion times of the plain sequence (one timed pass)
        flush.fill_(0.0)
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(len(reqs) + 1)]
        evs[0].record(stream)
        for i, r in enumerate(reqs):
            M.mknn_knn(r["cloud"], r["q"], r["nq"], 3, r["k"], None, 0, r["out_idx"],
                       r["out_d2"], s)
            evs[i + 1].record(stream)
        torch.cuda.synchronize()
        done_plain = np.array([evs[0].elapsed_time(e) for e in evs[1:]])
        return ms_batch, ms_plain, same, done_plain

    (ms_batch, ms_plain, same, done_plain), clk = _clocked(torch.cuda.current_device(), measure)
    M.mknn_batch_free(plan)
    t_b, t_p = float(np.mean(ms_batch)), float(np.mean(ms_plain))
    return {
        "workload": f"64 clouds, {sum(w.n for w in wls)} sites, {nq} queries "
                    f"(half box, half near-surface), k in {{1,4,8,16,32}}",
        "value": nq / (t_b / 1e3), "unit": UNIT, "ms_per_step": t_b, "steps": args.steps,
        "plain_one_launch_per_cloud": {"value": nq / (t_p / 1e3), "ms_per_step": t_p},
        "speedup_vs_plain": t_p / t_b,
        "results_identical": bool(same),
        "latency_ms_per_request": {
            "plan": {"p50": t_b, "p99": t_b, "note": "every request completes with the plan"},
            "plain": {"p50": float(np.percentile(done_plain, 50)),
                      "p99": float(np.percentile(done_plain, 99)),
                      "note": "completion time of each request in the launch sequence"}},
        "roofline": _roofline(alg, t_b, nq, l2=args._l2, kernel="knn_batch_* (persistent)"),
        "config": {"items": items, "grid": grid, "l2": "flushed before every timed step",
                   "lanes_chosen": {str(l): int((lanes == l).sum()) for l in set(lanes.tolist())},
                   "modes_chosen": {f"{l} lanes, {'shared memory' if p == 2 else 'registers'}":
                                    int(((lanes == l) & (placement == p)).sum())
                                    for l, p in set(zip(lanes.tolist(), placement.tolist()))},
                   "tune_seconds": tune_s,
                   "build_seconds_max": build_s if build_s is not None else "cached"},
        "gpu_launches_per_step": _plan_launches(lanes, reqs, placement,
                                                [M.mknn_cloud_trees(r["cloud"])[0] > 0
                                                 for r in reqs]),
        "clocks": clk,
    }


def batch_workload(args, M, torch):
    args._l2 = l2_probe(M, torch, torch.device("cuda", torch.cuda.current_device()),
                        torch.cuda.current_stream())
    out = batch_section(args, M, torch)
    line = {"metric": "batched k-NN queries/sec (64 clouds, one persistent launch, autotuned)",
            "n_gpus": 1, "warmup": args.warmup, "higher_is_better": True, "data": "synthetic",
            "dtype": "f32", **out}
    print(json.dumps(line), flush=True)


def prefix_section(args, M, torch, built=None):
    """Prefix workload: 4M-site bumpy sphere, 8M queries (half volume, half
    near-surface), per-query m log-uniform in [1000, n], k = 10."""
    import workloads as W
    wl, cloud, build_s = (built if built is not None
                          else (W.prefix_bumpy(n=max(2000, int(4_000_000 * args.scale)),
                                               nq=max(1000, int(8_000_000 * args.scale))),
                                None, None))
    if cloud is None:
        cloud, build_s = _cloud_cache(wl.points, wl.order, f"bumpy{wl.n}")
    cloud.upload()
    dev = torch.device("cuda", torch.cuda.current_device())
    q = torch.from_numpy(wl.queries).to(dev)
    m = torch.from_numpy(wl.m).to(dev)
    nq, k = wl.nq, wl.k
    idx = torch.empty((nq, k), dtype=torch.int32, device=dev)
    d2 = torch.empty((nq, k), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    s = stream.cuda_stream
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    rows, entries, coords, trans = _counts(M, torch, cloud, q, nq, k, m, s)
    alg = _alg_bytes(rows, entries, coords, nq, k, extra_per_query=4)
    ms, clk = _clocked(dev.index, lambda: _timed_ms(
        torch, stream, lambda: M.mknn_knn(cloud.handle, q, nq, 3, k, m, 0, idx, d2, s),
        args.steps, args.warmup, flush))
    t = float(np.mean(ms))
    del idx, d2, q, m
    return {
        "workload": f"bumpy sphere n={wl.n}, {nq} queries (half volume, half near-surface), "
                    f"m log-uniform in [1000, n] per query, k={k}",
        "value": nq / (t / 1e3), "unit": UNIT, "ms_per_step": t, "steps": args.steps,
        "roofline": _roofline(alg, t, nq, l2=args._l2, kernel=_query_kernel_name(0, k, 0),
                              counts={"rows": rows / nq, "entries": entries / nq,
                                      "coords": coords / nq, "transitions": trans / nq}),
        "config": {"E": cloud.stats()["entries"], "l2": "flushed before every timed step",
                   "step": "locality sort + k-NN kernel (mknn_knn)",
                   "build_seconds": build_s if build_s is not None else "cached"},
        "clocks": clk,
    }


def prefix_workload(args, M, torch):
    args._l2 = l2_probe(M, torch, torch.device("cuda", torch.cuda.current_device()),
                        torch.cuda.current_stream())
    out = prefix_section(args, M, torch)
    line = {"metric": "prefix k-NN queries/sec (k=10, 4M-pt bumpy sphere, per-query m)",
            "n_gpus": 1, "warmup": args.warmup, "higher_is_better": True, "data": "synthetic",
            "dtype": "f32", **out}
    print(json.dumps(line), flush=True)


def sites_section(args, M, torch, cloud, n):
    """Same-manifold queries: every site of the cloud queried against it
    (normal-estimation style, k = 16), and the same sites probed across
    prefixes with k = 100 (m log-uniform in [1000, n], the temporal setting
    of Sec. 5). Each run with its own clock samples and roofline."""
    import workloads as W
    dev = torch.device("cuda", torch.cuda.current_device())
    sites = torch.from_numpy(W.permutation(n, 61).astype(np.int32)).to(dev)
    stream = torch.cuda.current_stream(dev)
    s = stream.cuda_stream
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    out = {}
    for k, mode in ((16, "all sites, m = n"), (100, "m log-uniform in [1000, n]")):
        m = None
        if k == 100:
            u = W.uniform(62, 1, n)
            mv = np.clip(np.floor(np.exp(np.log(1000) + u * (np.log(n) - np.log(1000)))), 1, n)
            m = torch.from_numpy(mv.astype(np.int32)).to(dev)
        idx = torch.empty((n, k), dtype=torch.int32, device=dev)
        d2 = torch.empty((n, k), dtype=torch.float32, device=dev)
        rows, entries, coords, trans = _counts(M, torch, cloud, None, n, k, m, s, sites=sites)
        alg = _alg_bytes(rows, entries, coords, n, k, extra_per_query=4 + (4 if m is not None
                                                                         else 0))
        ms, clk = _clocked(dev.index, lambda: _timed_ms(
            torch, stream, lambda: M.mknn_knn_sites(cloud.handle, sites, n, k, m, 0, idx, d2, s),
            args.steps, args.warmup, flush))
        t = float(np.mean(ms))
        out[f"k{k}"] = {"workload": f"torus n={n}, {n} site queries ({mode}), k={k}",
                        "value": n / (t / 1e3), "unit": UNIT, "ms_per_step": t,
                        "roofline": _roofline(alg, t, n, l2=args._l2,
                                              kernel=_query_kernel_name(0, k, 0),
                                              counts={"rows": rows / n, "entries": entries / n,
                                                      "coords": coords / n,
                                                      "transitions": trans / n}),
                        "clocks": clk}
        del idx, d2
    return out


def sites_workload(args, M, torch):
    import workloads as W
    wl = W.large_torus(n=args.n, nq=1, k=16)
    cloud, build_s = _cloud_cache(wl.points, wl.order, f"torus{wl.n}")
    cloud.upload()
    args._l2 = l2_probe(M, torch, torch.device("cuda", torch.cuda.current_device()),
                        torch.cuda.current_stream())
    out = sites_section(args, M, torch, cloud, wl.n)
    line = {"metric": "same-manifold k-NN queries/sec (1M-pt torus, every site a query)",
            "value": out["k16"]["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "data": "synthetic",
            "dtype": "f32", "config": {"l2": "flushed before every timed step",
                                        "build_seconds": build_s if build_s is not None
                                        else "cached"},
            "runs": out}
    print(json.dumps(line), flush=True)


def dynamic_workload(args, M, torch):
    """Dynamic insertion: the 1M-point torus built over its first 90% of
    ranks with the dynamic option and uploaded, then the last 10% appended
    in batches (host insertion + device update, timed per call); queries
    afterwards against one static build over all the points (same rows,
    same speed expected)."""
    import workloads as W
    from paper_2605_02224_gb300 import Cloud
    wl = W.large_torus(n=args.n, nq=args.nq, k=args.k)
    Pr = np.ascontiguousarray(wl.ranked_points(), np.float32)
    n = wl.n
    n0 = n - n // 10
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    s = stream.cuda_stream
    t0 = time.perf_counter()
    c = Cloud.build(Pr[:n0], dynamic=True)
    build_s = time.perf_counter() - t0
    c.upload(s)
    ms = []
    B = max(1, args.append_batch)
    for at in range(n0, n, B):
        t1 = time.perf_counter()
        c.append(Pr[at:min(n, at + B)], s)
        ms.append((time.perf_counter() - t1) * 1e3)
    appended = n - n0
    static, _ = _cloud_cache(wl.points, wl.order, f"torus{wl.n}")
    static.upload(s)
    q = torch.from_numpy(wl.queries).to(dev)
    k, nq = wl.k, wl.nq
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)

    def timed(cl):
        idx = torch.empty((nq, k), dtype=torch.int32, device=dev)
        d2 = torch.empty((nq, k), dtype=torch.float32, device=dev)
        for _ in range(max(3, args.warmup)):
            M.mknn_knn(cl.handle, q, nq, 3, k, None, 0, idx, d2, s)
        out = []
        for i in range(args.steps):
            flush.fill_(float(i))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            M.mknn_knn(cl.handle, q, nq, 3, k, None, 0, idx, d2, s)
            b.record(stream)
            torch.cuda.synchronize()
            out.append(a.elapsed_time(b))
        return float(np.mean(out)), idx, d2

    t_dyn, i1, d1 = timed(c)
    t_sta, i2, d2 = timed(static)
    same = bool(torch.equal(i1, i2) and torch.equal(d1, d2))
    t1 = time.perf_counter()
    c.compact(s)
    compact_ms = (time.perf_counter() - t1) * 1e3
    t_cmp, i3, d3 = timed(c)
    same = same and bool(torch.equal(i1, i3) and torch.equal(d1, d3))
    line = {"metric": "appended points/sec (dynamic 1M-pt torus, host insertion + device update)",
            "value": appended / (sum(ms) / 1e3), "unit": "points/s", "n_gpus": 1,
            "higher_is_better": True, "data": "synthetic", "dtype": "f32",
            "config": {"workload": f"torus n={n}: {n0} built (dynamic), {appended} appended in "
                                   f"batches of {B}; {nq} volume queries, k={k}",
                       "build_seconds_dynamic": build_s},
            "append_ms_per_call": {"mean": float(np.mean(ms)), "p50": float(np.median(ms)),
                                   "max": float(np.max(ms)), "calls": len(ms)},
            "queries_after_appends": {"value": nq / (t_dyn / 1e3), "ms_per_step": t_dyn},
            "queries_static_build": {"value": nq / (t_sta / 1e3), "ms_per_step": t_sta},
            "queries_after_compact": {"value": nq / (t_cmp / 1e3), "ms_per_step": t_cmp,
                                      "compact_ms": compact_ms},
            "results_identical": same,
            "device_bytes": {"dynamic": c.device_bytes(), "static": static.device_bytes()}}
    print(json.dumps(line), flush=True)


def sweep_workload(args, M, torch):
    """Sensitivity to manifold structure: the 1M-point bumpy sphere with
    every point displaced by up to a fraction of its bbox diagonal, and
    points uniform in a cube (queries in the same cube), 4M queries, k = 16:
    queries/s, successor-list shape and work per query for each."""
    import workloads as W
    wls = [W.degraded_bumpy(r, args.n, args.nq, args.k)
           for r in (0.0, 0.001, 0.003, 0.01, 0.03, 0.1)]
    wls += [W.uniform_volume(n, args.nq, args.k) for n in (100_000, args.n)]
    clouds, build_s = _build_many(wls, "sweep")
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    s = stream.cuda_stream
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    runs = []
    for wl, c in zip(wls, clouds):
        c.upload(s)
        q = torch.from_numpy(wl.queries).to(dev)
        nq, k = wl.nq, wl.k
        idx = torch.empty((nq, k), dtype=torch.int32, device=dev)
        d2 = torch.empty((nq, k), dtype=torch.float32, device=dev)
        for _ in range(max(3, args.warmup)):
            M.mknn_knn(c.handle, q, nq, 3, k, None, 0, idx, d2, s)
        cnt = torch.zeros((nq, 4), dtype=torch.int32, device=dev)
        M.mknn_knn_ex(c.handle, q, nq, 3, k, None, 0, idx, d2, s, counters=cnt, lanes=1,
                      placement=1)
        torch.cuda.synchronize()
        rows, entries, coords, trans = (int(x) for x in cnt.to(torch.int64).sum(dim=0).cpu())
        ms = []
        for i in range(args.steps):
            flush.fill_(float(i))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            M.mknn_knn(c.handle, q, nq, 3, k, None, 0, idx, d2, s)
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        _, rowp, _ = c.table()
        L = np.diff(rowp)
        runs.append({"workload": wl.name, "displacement_ratio": wl.meta.get("ratio"),
                     "value": nq / (float(np.mean(ms)) / 1e3), "ms_per_step": float(np.mean(ms)),
                     "E_per_site": float(L.mean()), "longest_row": int(L.max()),
                     "per_query": {"rows": rows / nq, "entries": entries / nq,
                                   "transitions": trans / nq}})
        c.close()
    line = {"metric": "k-NN queries/sec vs manifold degradation (1M-pt bumpy sphere, k=16)",
            "value": runs[0]["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "data": "synthetic", "dtype": "f32",
            "config": {"l2": "flushed before every timed step",
                       "build_seconds_max": build_s if build_s is not None else "cached"},
            "runs": runs}
    print(json.dumps(line), flush=True)


def orders_workload(args, M, torch):
    """Insertion orders (Sec. 5): the 1M-point bumpy sphere built in a
    random order, a BRIO round order with Hilbert-sorted rounds, and the
    farthest-point order; the same 4M volume queries, k = 16, against each:
    build time, list shape, work and speed per query."""
    import workloads as W
    from concurrent.futures import ThreadPoolExecutor
    from paper_2605_02224_gb300 import Cloud
    wl = W.degraded_bumpy(0.0, args.n, args.nq, args.k)
    kinds = (("random", M.ORDER_RANDOM), ("brio_hilbert", M.ORDER_BRIO_HILBERT),
             ("farthest_point", M.ORDER_FARTHEST_POINT))

    def make(kind):
        t0 = time.perf_counter()
        o = M.mknn_insertion_order(wl.points, kind, 71)
        t1 = time.perf_counter()
        c = Cloud.build(wl.points, o)
        return c, t1 - t0, time.perf_counter() - t1

    with ThreadPoolExecutor(max_workers=3) as ex:
        built = list(ex.map(lambda kk: make(kk[1]), kinds))
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    s = stream.cuda_stream
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    q = torch.from_numpy(wl.queries).to(dev)
    nq, k = wl.nq, wl.k
    runs = []
    ref = None
    for (name, _), (c, order_s, build_s) in zip(kinds, built):
        c.upload(s)
        idx = torch.empty((nq, k), dtype=torch.int32, device=dev)
        d2 = torch.empty((nq, k), dtype=torch.float32, device=dev)
        for _ in range(max(3, args.warmup)):
            M.mknn_knn(c.handle, q, nq, 3, k, None, 0, idx, d2, s)
        cnt = torch.zeros((nq, 4), dtype=torch.int32, device=dev)
        M.mknn_knn_ex(c.handle, q, nq, 3, k, None, 0, idx, d2, s, counters=cnt, lanes=1,
                      placement=1)
        torch.cuda.synchronize()
        rows, entries, coords, trans = (int(x) for x in cnt.to(torch.int64).sum(dim=0).cpu())
        ms = []
        for i in range(args.steps):
            flush.fill_(float(i))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            M.mknn_knn(c.handle, q, nq, 3, k, None, 0, idx, d2, s)
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        # the same distances whatever the order (equal float32 distances are
        # ordered by rank, which the order changes, so neighbours are
        # compared through their distances)
        same = True if ref is None else bool(torch.equal(d2, ref))
        if ref is None:
            ref = d2.clone()
        _, rowp, _ = c.table()
        L = np.diff(rowp)
        runs.append({"order": name, "order_seconds": order_s, "build_seconds": build_s,
                     "value": nq / (float(np.mean(ms)) / 1e3), "ms_per_step": float(np.mean(ms)),
                     "E_per_site": float(L.mean()), "longest_row": int(L.max()),
                     "per_query": {"rows": rows / nq, "entries": entries / nq,
                                   "transitions": trans / nq},
                     "same_distances_as_random": same})
        c.close()
    line = {"metric": "k-NN queries/sec by insertion order (1M-pt bumpy sphere, k=16)",
            "value": runs[0]["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "data": "synthetic", "dtype": "f32",
            "config": {"l2": "flushed before every timed step"}, "runs": runs}
    print(json.dumps(line), flush=True)


def _start_builds(args):
    """Generates the extra sections' workloads and builds (or loads) their
    clouds in background host threads while the headline runs. Returns
    {section: future of (workloads, clouds, build seconds)}."""
    from concurrent.futures import ThreadPoolExecutor
    import workloads as W
    builders = ThreadPoolExecutor(max_workers=max(1, (os.cpu_count() or 4) - 1))
    sections = ThreadPoolExecutor(max_workers=3)

    def many(make, tag):
        wls = make()
        futs = [builders.submit(_cloud_cache, w.points, w.order, f"{tag}-{w.n}")
                for w in wls]
        res = [f.result() for f in futs]
        built = [r[1] for r in res if r[1] is not None]
        return wls, [r[0] for r in res], (max(built) if built else None)

    def one(make, tag):
        wl = make()
        c, secs = builders.submit(_cloud_cache, wl.points, wl.order, tag).result()
        return wl, c, secs

    sc = args.scale
    jobs = {"prefix": sections.submit(one, lambda: W.prefix_bumpy(
        n=max(2000, int(4_000_000 * sc)), nq=max(1000, int(8_000_000 * sc))), "bumpy")}
    if not args.no_serve:
        jobs["serving"] = sections.submit(many, lambda: W.serve_clouds(scale=sc), "serve")
    jobs["batch"] = sections.submit(many, lambda: W.batch_clouds(scale=sc), "batch")
    return jobs


def main():
    args = _args()
    rank, world, local = _dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch
    import workloads as W
    from paper_2605_02224_gb300 import mknn as M

    torch.cuda.set_device(local)
    if args.workload == "batch":
        batch_workload(args, M, torch)
        return
    if args.workload == "prefix":
        prefix_workload(args, M, torch)
        return
    if args.workload == "sites":
        sites_workload(args, M, torch)
        return
    if args.workload == "dynamic":
        dynamic_workload(args, M, torch)
        return
    if args.workload == "sweep":
        sweep_workload(args, M, torch)
        return
    if args.workload == "orders":
        orders_workload(args, M, torch)
        return
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    extras = rank == 0 and world == 1 and not args.quick
    jobs = _start_builds(args) if extras else {}

    wl = W.large_torus(n=args.n, nq=args.nq, k=args.k)
    cloud, build_s = _cloud_cache(wl.points, wl.order, f"torus{wl.n}")
    cloud.upload()
    st = cloud.stats()
    nq, k = wl.nq, wl.k
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    sptr = stream.cuda_stream
    args._l2 = l2_probe(M, torch, dev, stream)
    q = torch.from_numpy(wl.queries).to(dev)
    idx = torch.empty((nq, k), dtype=torch.int32, device=dev)
    d2 = torch.empty((nq, k), dtype=torch.float32, device=dev)
    perm = torch.empty(nq, dtype=torch.int32, device=dev)
    ws_bytes = M.mknn_query_order_workspace_size(nq)
    ws = torch.empty(max(ws_bytes, 256), dtype=torch.uint8, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2
    lanes = args.lanes or 0

    order = None if args.no_sort else perm
    sort_flag = -1 if args.no_sort else 0

    def step(ev=None, kk=k, oi=idx, od=d2, sorted_=not args.no_sort):
        if ev:
            ev[0].record(stream)
        if sorted_:
            M.mknn_query_order(cloud.handle, q, nq, 3, perm, ws, ws_bytes, sptr)
        if ev:
            ev[1].record(stream)
        M.mknn_knn_ex(cloud.handle, q, nq, 3, kk, None, 0, oi, od, sptr, lanes=lanes,
                      order=perm if sorted_ else None, sort=0 if sorted_ else -1,
                      placement=args.placement, blocks_per_sm=args.blocks_per_sm)
        if ev:
            ev[2].record(stream)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()

    # algorithmic bytes of one launch, from the kernel's own counters (untimed)
    rows, entries, coords, trans = _counts(M, torch, cloud, q, nq, k, None, sptr, order=order,
                                           sort_flag=sort_flag)
    alg_bytes = _alg_bytes(rows, entries, coords, nq, k)

    clocks = Clocks(local)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    for i in range(args.steps):
        flush.fill_(float(i))
        step(evs[i])
    torch.cuda.synchronize()
    time.sleep(0.3)
    clk = clocks.stop()
    step_ms = [e[0].elapsed_time(e[2]) for e in evs]
    kern_ms = [e[1].elapsed_time(e[2]) for e in evs]
    total_ms = max_over_ranks(float(sum(step_ms)), dist, dev)
    if dist:
        dist.barrier()
    ms_per_step, value = job_rate(total_ms, args.steps, nq, world)

    def end_to_end():
        """Queries/s through the host-buffer entry point (pinned host
        memory, copies inside the timed region), mean over calls."""
        qh = torch.from_numpy(wl.queries).pin_memory()
        oh_i = torch.empty((nq, k), dtype=torch.int32).pin_memory()
        oh_d = torch.empty((nq, k), dtype=torch.float32).pin_memory()
        for _ in range(2):
            M.mknn_knn_host(cloud.handle, qh, k, None, 0, oh_i, oh_d)
        if dist:
            dist.barrier()
        e2e_t = []
        for _ in range(max(3, args.steps // 2)):
            t0 = time.perf_counter()
            M.mknn_knn_host(cloud.handle, qh, k, None, 0, oh_i, oh_d)
            e2e_t.append(time.perf_counter() - t0)
        agree = bool(torch.equal(oh_i, idx.cpu()))  # before the copies below overwrite oh_i
        # the call's phases alone, for comparison: the same copies on one
        # stream with nothing to overlap (CUDA events), and the device-path step
        qd = torch.empty((nq, 3), dtype=torch.float32, device=dev)
        od = torch.empty((nq, k), dtype=torch.float32, device=dev)
        strm = torch.cuda.current_stream(dev)

        def timed_copy(fn):
            fn()
            ms = []
            for _ in range(3):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(strm)
                fn()
                b.record(strm)
                torch.cuda.synchronize()
                ms.append(a.elapsed_time(b))
            return float(np.median(ms))
        h2d = timed_copy(lambda: qd.copy_(qh, non_blocking=True))
        d2h = timed_copy(lambda: (oh_i.copy_(idx, non_blocking=True),
                                  oh_d.copy_(od, non_blocking=True)))
        phases = {"h2d_alone_ms": h2d, "device_step_ms": float(np.mean(step_ms)),
                  "d2h_alone_ms": d2h,
                  "note": "the copies timed alone on one stream, and the device-path step; the "
                          "host-buffer call overlaps them over two streams in 2^20-query chunks"}
        return max_over_ranks(float(np.mean(e2e_t)), dist, dev), agree, phases

    kern_s = float(np.mean(kern_ms)) / 1e3
    khash = _kernel_hash()
    rec = _profile_record(khash)
    roof = _roofline(alg_bytes, kern_s * 1e3, nq, l2=args._l2, rec=rec,
                     kernel=_query_kernel_name(lanes, k, args.placement),
                     counts={"rows": rows / nq, "entries": entries / nq, "coords": coords / nq,
                             "transitions": trans / nq})
    roof["traffic"] = _profiled_traffic(khash, wl.n, nq)
    roof["kernel_hash"] = khash

    no_sort = k_sweep = prefix = batch = serving = cpu = sites = None
    if not extras:
        e2e_s, agree, phases = end_to_end()
    else:
        # the same step without the locality sort (queries in input order)
        ms_ns, clk_ns = _clocked(local, lambda: _timed_ms(
            torch, stream, lambda: step(sorted_=False), args.steps, args.warmup, flush))
        t_ns = float(np.mean(ms_ns))
        no_sort = {"value": nq / (t_ns / 1e3), "unit": UNIT, "ms_per_step": t_ns,
                   "speedup_of_sort": t_ns / ms_per_step,
                   "roofline": _roofline(alg_bytes, t_ns, nq, l2=args._l2,
                                         kernel=_query_kernel_name(lanes, k, args.placement)),
                   "clocks": clk_ns}
        # k sweep on the same cloud and queries
        k_sweep = []
        for kk in (4, 32, 100):
            oi = torch.empty((nq, kk), dtype=torch.int32, device=dev)
            od = torch.empty((nq, kk), dtype=torch.float32, device=dev)
            r_, e_, c_, t_ = _counts(M, torch, cloud, q, nq, kk, None, sptr, order=order,
                                     sort_flag=sort_flag)
            ms_k, clk_k = _clocked(local, lambda: _timed_ms(
                torch, stream, lambda: step(kk=kk, oi=oi, od=od), args.steps, args.warmup,
                flush))
            t_k = float(np.mean(ms_k))
            k_sweep.append({"k": kk, "value": nq / (t_k / 1e3), "unit": UNIT, "ms_per_step": t_k,
                            "roofline": _roofline(_alg_bytes(r_, e_, c_, nq, kk), t_k, nq,
                                                  l2=args._l2,
                                                  kernel=_query_kernel_name(lanes, kk, 0),
                                                  counts={"rows": r_ / nq, "entries": e_ / nq,
                                                          "coords": c_ / nq,
                                                          "transitions": t_ / nq}),
                            "clocks": clk_k})
            del oi, od
        sites = sites_section(args, M, torch, cloud, wl.n)
        # the host-buffer path after the background builds are done (host
        # copies and staging are timed, so the host cores should be free)
        for j in jobs.values():
            j.result()
        e2e_s, agree, phases = end_to_end()
        P_ranked, rowp, succ = cloud.table()
        del q, idx, d2, perm, ws
        torch.cuda.empty_cache()
        prefix = prefix_section(args, M, torch, jobs["prefix"].result())
        torch.cuda.empty_cache()
        batch = batch_section(args, M, torch, jobs["batch"].result())
        torch.cuda.empty_cache()
        if "serving" in jobs:
            serving = serving_section(args, M, torch, jobs["serving"].result())
        if not args.no_cpu_baseline:
            cpu = cpu_baselines(P_ranked, rowp, succ, wl.queries, k, args.cpu_seconds)

    if rank == 0:
        line = {
            "metric": metric_name(args.k, args.n), "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {
                "workload": f"torus R=1 r=0.3 sigma=1e-4, n={wl.n}, {nq} queries uniform in the "
                            f"bbox padded by 0.2, k={k}, m=n",
                "n": wl.n, "nq": nq, "k": k, "E": st["entries"],
                "lanes": lanes or 1,  # 0 asks for the library's default: one lane per query
                "query_order": "input order" if args.no_sort else "64^3 Morton cell counting sort",
                "l2": "flushed before every timed step (256 MB write, outside the events)",
                "build_seconds": build_s if build_s is not None else "cached",
                "parallelism": f"replicas x{world}",
            },
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": {"value": world * nq / e2e_s, "unit": UNIT,
                    "h2d_bytes_per_step": nq * 12, "d2h_bytes_per_step": nq * k * 8,
                    "ms_per_step": e2e_s * 1e3, "matches_device_path": agree,
                    "phases": phases},
            # per step: the query kernel, and unless --no-sort the locality sort's five
            # (bounding box, histogram, two scan levels, scatter)
            "gpu_launches": (1 if args.no_sort else 6) * args.steps,
            "clocks": clk,
            "step_ms": step_ms,
            "l2_probe": args._l2,
            "no_sort": no_sort,
            "k_sweep": k_sweep,
            "sites": sites,
            "prefix": prefix,
            "batch": batch,
            "serving": serving,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
