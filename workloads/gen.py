"""Counter-based random numbers and surface samplers.

The generator is splitmix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
stream: output i of stream (seed, stream) is mix64(key + (i + 1) * gamma)
with key = mix64(seed * gamma + stream). Any element can be computed
without the ones before it, which keeps every draw vectorised and
independent of chunking.

Surfaces follow the synthetic stand-ins for the paper's manifold datasets
(Sec. 5.2: targets on a surface, queries in a padded box around it).
All coordinates are returned as float32 (the method's input precision);
the intermediate shaping runs in float64.
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_TWO_PI = 2.0 * np.pi


def _mix64(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def rand_u64(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """count uint64 words of stream (seed, stream), starting at element offset."""
    with np.errstate(over="ignore"):
        key = _mix64(np.array([seed], dtype=np.uint64) * _GAMMA
                     + np.array([stream], dtype=np.uint64))
        ctr = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        return _mix64(key + ctr * _GAMMA)


def uniform(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform float64 in [0, 1) with 53 random bits."""
    return (rand_u64(seed, stream, count, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """Standard normal float64 by the Box-Muller transform of two substreams."""
    u1 = 1.0 - uniform(seed, 2 * stream, count, offset)       # (0, 1]
    u2 = uniform(seed, 2 * stream + 1, count, offset)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(_TWO_PI * u2)


def permutation(n: int, seed: int) -> np.ndarray:
    """A uniformly random permutation of 0..n-1 (int64): argsort of random keys.

    order[r] is the input index of the point inserted at rank r.
    """
    keys = rand_u64(seed, 7, n)
    return np.argsort(keys, kind="stable").astype(np.int64)


def _unit(v: np.ndarray) -> np.ndarray:
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


# --------------------------------------------------------------------------
# surfaces: each returns (points float32 (n,3), unit normals float64 (n,3))

def sphere(n: int, seed: int, stream0: int = 100):
    """Unit sphere: normalised N(0, I) directions."""
    g = normal(seed, stream0, 3 * n).reshape(n, 3)
    d = _unit(g)
    return d.astype(np.float32), d


def torus(n: int, seed: int, R: float = 1.0, r: float = 0.3, sigma: float = 1e-4,
          stream0: int = 200):
    """Torus sampled uniformly by area, jittered by N(0, sigma) along the normal.

    The tube angle theta is drawn by rejection with acceptance
    (R + r cos theta) / (R + r), the area density of the torus.
    """
    thetas = []
    have = 0
    offset = 0
    chunk = int(1.5 * n) + 64
    while have < n:
        th = _TWO_PI * uniform(seed, stream0, chunk, offset)
        acc = uniform(seed, stream0 + 1, chunk, offset) * (R + r) < (R + r * np.cos(th))
        thetas.append(th[acc])
        have += int(acc.sum())
        offset += chunk
    th = np.concatenate(thetas)[:n]
    ph = _TWO_PI * uniform(seed, stream0 + 2, n)
    ct, st, cp, sp = np.cos(th), np.sin(th), np.cos(ph), np.sin(ph)
    nrm = np.stack([ct * cp, ct * sp, st], axis=1)
    base = np.stack([(R + r * ct) * cp, (R + r * ct) * sp, r * st], axis=1)
    jitter = sigma * normal(seed, stream0 + 3, n)
    return (base + jitter[:, None] * nrm).astype(np.float32), nrm


def bumpy_sphere(n: int, seed: int, amp: float = 0.1, freq: float = 8.0, stream0: int = 300):
    """Radius 1 + amp sin(freq theta) sin(freq phi) over uniform directions.

    theta is the polar angle, phi the azimuth; the normal is the normalised
    gradient of |x| - rho(theta, phi).
    """
    d = _unit(normal(seed, stream0, 3 * n).reshape(n, 3))
    th = np.arccos(np.clip(d[:, 2], -1.0, 1.0))
    ph = np.arctan2(d[:, 1], d[:, 0])
    rho = 1.0 + amp * np.sin(freq * th) * np.sin(freq * ph)
    p = rho[:, None] * d
    r_th = amp * freq * np.cos(freq * th) * np.sin(freq * ph)
    r_ph = amp * freq * np.sin(freq * th) * np.cos(freq * ph)
    st = np.maximum(np.sin(th), 1e-12)
    e_th = np.stack([np.cos(th) * np.cos(ph), np.cos(th) * np.sin(ph), -np.sin(th)], axis=1)
    e_ph = np.stack([-np.sin(ph), np.cos(ph), np.zeros_like(ph)], axis=1)
    g = d - (r_th / rho)[:, None] * e_th - (r_ph / (rho * st))[:, None] * e_ph
    return p.astype(np.float32), _unit(g)


def patches4(n: int, seed: int, side: float = 0.5, stream0: int = 400):
    """Four planar squares (side 0.5) with random centres in [0.25, 0.75]^3
    and random orientation; points split evenly between them."""
    counts = [n // 4 + (1 if i < n % 4 else 0) for i in range(4)]
    pts, nrms = [], []
    for i, c in enumerate(counts):
        ctr = 0.25 + 0.5 * uniform(seed, stream0 + 10 * i, 3)
        nv = _unit(normal(seed, stream0 + 10 * i + 1, 3))
        axis = np.eye(3)[int(np.argmin(np.abs(nv)))]
        u = _unit(np.cross(nv, axis))
        v = np.cross(nv, u)
        s = side * (uniform(seed, stream0 + 10 * i + 2, c) - 0.5)
        t = side * (uniform(seed, stream0 + 10 * i + 3, c) - 0.5)
        pts.append(ctr[None, :] + s[:, None] * u[None, :] + t[:, None] * v[None, :])
        nrms.append(np.repeat(nv[None, :], c, axis=0))
    return np.concatenate(pts).astype(np.float32), np.concatenate(nrms)


def lattice(L: int):
    """All integer points of {0..L-1}^3 (exact in float32), x fastest."""
    g = np.arange(L, dtype=np.float32)
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    p = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1).astype(np.float32)
    return p, np.zeros_like(p, dtype=np.float64)


def uniform_cube(n: int, seed: int, lo: float = -1.0, hi: float = 1.0, stream0: int = 500):
    p = lo + (hi - lo) * uniform(seed, stream0, 3 * n).reshape(n, 3)
    return p.astype(np.float32), np.zeros((n, 3))


def displace(p: np.ndarray, ratio: float, seed: int, stream0: int = 600) -> np.ndarray:
    """Each point moved by a random vector: uniform direction, length
    uniform in [0, ratio * d) with d the diagonal of the points' bounding
    box (degrading the manifold structure, the sensitivity study of Sec. 5)."""
    n = p.shape[0]
    lo, hi = p.min(axis=0).astype(np.float64), p.max(axis=0).astype(np.float64)
    d = float(np.linalg.norm(hi - lo))
    v = _unit(np.stack([normal(seed, stream0, n), normal(seed, stream0 + 1, n),
                        normal(seed, stream0 + 2, n)], axis=1))
    length = ratio * d * uniform(seed, stream0 + 3, n)
    return (p.astype(np.float64) + v * length[:, None]).astype(np.float32)


SURFACES = ("sphere", "torus", "bumpy", "patches")


def surface(kind: str, n: int, seed: int, stream0: int | None = None):
    fn = {"sphere": sphere, "torus": torus, "bumpy": bumpy_sphere, "patches": patches4}[kind]
    if stream0 is None:
        return fn(n, seed)
    return fn(n, seed, stream0=stream0)


# --------------------------------------------------------------------------
# queries

def bbox(p: np.ndarray):
    return p.min(axis=0).astype(np.float64), p.max(axis=0).astype(np.float64)


def box_queries(nq: int, seed: int, lo, hi, stream0: int = 900) -> np.ndarray:
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    u = uniform(seed, stream0, 3 * nq).reshape(nq, 3)
    return (lo + (hi - lo) * u).astype(np.float32)


def near_surface_queries(kind: str, nq: int, seed: int, sigma: float = 0.01) -> np.ndarray:
    """Fresh samples of the surface pushed off it by |N(0, sigma)| along the normal."""
    p, nrm = surface(kind, nq, seed, stream0=700)
    off = np.abs(sigma * normal(seed, 800, nq))
    return (p.astype(np.float64) + off[:, None] * nrm).astype(np.float32)
