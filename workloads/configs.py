"""The five synthetic workloads, by size and seed.

Each workload is volume-to-surface k-NN: target points on a surface,
queries in the surface's bounding box padded by 0.2 (the paper's Sec. 5.2
setting uses a 2x box; the padded box is the stand-in named by the
workload list) or just off the surface. Sizes can be scaled down for
tests; the seeds stay the same so a scaled workload is a prefix-style
sibling of the full one, not a different distribution.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import gen


@dataclass
class Workload:
    name: str
    points: np.ndarray            # float32 (n, 3), input order
    order: np.ndarray             # int64 (n,), order[r] = input index of rank r
    queries: np.ndarray           # float32 (nq, 3)
    k: int
    m: np.ndarray | int = 0       # scalar (0 = n) or int32 (nq,) per query
    surface: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.points.shape[0])

    @property
    def nq(self) -> int:
        return int(self.queries.shape[0])

    def ranked_points(self) -> np.ndarray:
        """Points in insertion-rank order (rank r = row r)."""
        return np.ascontiguousarray(self.points[self.order])


def padded_box(points: np.ndarray, pad: float = 0.2):
    lo, hi = gen.bbox(points)
    return lo - pad, hi + pad


def small_sphere(nq: int = 10_000) -> Workload:
    """2,000 points on the unit sphere, k = 8, queries in [-1.5, 1.5]^3."""
    p, _ = gen.sphere(2000, seed=1)
    order = gen.permutation(2000, seed=2)
    q = gen.box_queries(nq, 3, [-1.5] * 3, [1.5] * 3)
    return Workload("sphere-2k-k8", p, order, q, k=8, surface="sphere")


def large_torus(n: int = 1_000_000, nq: int = 4_000_000, k: int = 16) -> Workload:
    """Torus R=1, r=0.3 with N(0, 1e-4) normal jitter; queries in the padded bbox."""
    p, _ = gen.torus(n, seed=11)
    order = gen.permutation(n, seed=12)
    lo, hi = padded_box(p)
    q = gen.box_queries(nq, 13, lo, hi)
    return Workload(f"torus-{n}-q{nq}-k{k}", p, order, q, k=k, surface="torus")


def degraded_bumpy(ratio: float, n: int = 1_000_000, nq: int = 4_000_000,
                   k: int = 16) -> Workload:
    """Bumpy sphere with every point displaced by up to `ratio` of the bbox
    diagonal (ratio 0: the surface itself); queries in the padded bbox."""
    p, _ = gen.bumpy_sphere(n, seed=51)
    if ratio > 0:
        p = gen.displace(p, ratio, seed=52)
    order = gen.permutation(n, seed=53)
    lo, hi = padded_box(p)
    q = gen.box_queries(nq, 54, lo, hi)
    return Workload(f"bumpy-displaced{ratio:g}-{n}", p, order, q, k=k, surface="bumpy",
                    meta={"ratio": ratio})


def uniform_volume(n: int = 1_000_000, nq: int = 4_000_000, k: int = 16) -> Workload:
    """Targets and queries uniform in the same cube [-1, 1]^3 (no manifold)."""
    p, _ = gen.uniform_cube(n, seed=61)
    order = gen.permutation(n, seed=62)
    q = gen.box_queries(nq, 63, [-1.0] * 3, [1.0] * 3)
    return Workload(f"uniform-{n}", p, order, q, k=k, surface="uniform")


def _mixed_queries(kind: str, p: np.ndarray, nq: int, seed: int) -> np.ndarray:
    """Half uniform in the padded box, half |N(0, 0.01)| off the surface."""
    lo, hi = padded_box(p)
    nv = nq // 2
    qv = gen.box_queries(nv, seed, lo, hi)
    qs = gen.near_surface_queries(kind, nq - nv, seed + 1)
    return np.concatenate([qv, qs]).astype(np.float32)


def prefix_bumpy(n: int = 4_000_000, nq: int = 8_000_000, k: int = 10) -> Workload:
    """Bumpy sphere with a per-query prefix bound m, log-uniform in [1000, n]."""
    p, _ = gen.bumpy_sphere(n, seed=31)
    order = gen.permutation(n, seed=32)
    q = _mixed_queries("bumpy", p, nq, 33)
    lo_m = min(1000, n)
    u = gen.uniform(34, 1, nq)
    m = np.floor(np.exp(math.log(lo_m) + u * (math.log(n) - math.log(lo_m)))).astype(np.int64)
    m = np.clip(m, 1, n).astype(np.int32)
    return Workload(f"bumpy-{n}-q{nq}-k{k}-prefix", p, order, q, k=k, m=m, surface="bumpy")


def _log_uniform_int(seed: int, stream: int, count: int, lo: float, hi: float) -> np.ndarray:
    u = gen.uniform(seed, stream, count)
    return np.floor(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))).astype(np.int64)


def batch_clouds(n_clouds: int = 64, lo: float = 1e4, hi: float = 2e6, scale: float = 1.0,
                 queries_per_point: int = 2, seed: int = 21) -> list[Workload]:
    """64 clouds of log-uniform size, mixed surfaces, k from {1,4,8,16,32}."""
    sizes = _log_uniform_int(seed, 1, n_clouds, lo, hi)
    kinds = (gen.rand_u64(seed, 2, n_clouds) % np.uint64(4)).astype(np.int64)
    ks_choice = np.array([1, 4, 8, 16, 32])
    ks = ks_choice[(gen.rand_u64(seed, 3, n_clouds) % np.uint64(5)).astype(np.int64)]
    out = []
    for i in range(n_clouds):
        n = max(16, int(sizes[i] * scale))
        kind = gen.SURFACES[int(kinds[i])]
        cs = seed * 1000 + 10 * i
        p, _ = gen.surface(kind, n, cs)
        order = gen.permutation(n, cs + 1)
        q = _mixed_queries(kind, p, queries_per_point * n, cs + 2)
        out.append(Workload(f"batch{i}-{kind}-{n}-k{int(ks[i])}", p, order, q,
                            k=int(ks[i]), surface=kind))
    return out


def serve_clouds(n_clouds: int = 16, lo: float = 1e5, hi: float = 4e6, scale: float = 1.0,
                 seed: int = 41) -> list[Workload]:
    """Resident clouds for the serving loop (queries are drawn per request)."""
    sizes = _log_uniform_int(seed, 1, n_clouds, lo, hi)
    kinds = (gen.rand_u64(seed, 2, n_clouds) % np.uint64(4)).astype(np.int64)
    out = []
    for i in range(n_clouds):
        n = max(16, int(sizes[i] * scale))
        kind = gen.SURFACES[int(kinds[i])]
        cs = seed * 1000 + 10 * i
        p, _ = gen.surface(kind, n, cs)
        order = gen.permutation(n, cs + 1)
        out.append(Workload(f"serve{i}-{kind}-{n}", p, order,
                            np.zeros((0, 3), np.float32), k=1, surface=kind))
    return out


@dataclass
class Request:
    arrival_s: float
    cloud: int
    queries: np.ndarray
    k: int
    m: int


def serve_requests(clouds: list[Workload], n_req: int, rate_hz: float, seed: int = 42,
                   max_q: int = 65536) -> list[Request]:
    """Poisson arrivals; 1..max_q queries (log-uniform), k ~ U{1..64},
    m ~ U{ceil(n/10)..n}; each request names one cloud uniformly."""
    gaps = -np.log(1.0 - gen.uniform(seed, 1, n_req)) / rate_hz
    t = np.cumsum(gaps)
    cl = (gen.rand_u64(seed, 2, n_req) % np.uint64(len(clouds))).astype(np.int64)
    sz = np.floor(np.exp(gen.uniform(seed, 3, n_req) * math.log(max_q))).astype(np.int64)
    sz = np.clip(sz, 1, max_q)
    ks = 1 + (gen.rand_u64(seed, 4, n_req) % np.uint64(64)).astype(np.int64)
    um = gen.uniform(seed, 5, n_req)
    reqs = []
    for i in range(n_req):
        c = clouds[int(cl[i])]
        n = c.n
        lo_m = max(1, math.ceil(n / 10))
        m = int(lo_m + math.floor(um[i] * (n - lo_m + 1)))
        q = _mixed_queries(c.surface, c.points, int(sz[i]), seed * 100000 + 7 * i)
        reqs.append(Request(float(t[i]), int(cl[i]), q, int(ks[i]), min(m, n)))
    return reqs
