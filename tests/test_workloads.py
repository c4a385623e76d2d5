"""The seeded input generators: determinism and the shapes they promise
(CPU only)."""
from __future__ import annotations

import numpy as np

import workloads as W


def test_streams_are_deterministic_and_chunk_independent():
    a = W.rand_u64(7, 3, 1000)
    b = np.concatenate([W.rand_u64(7, 3, 400), W.rand_u64(7, 3, 600, offset=400)])
    assert np.array_equal(a, b)
    assert not np.array_equal(a, W.rand_u64(7, 4, 1000))
    u = W.uniform(7, 3, 100000)
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.005
    z = W.normal(7, 3, 100000)
    assert abs(z.mean()) < 0.02 and abs(z.std() - 1.0) < 0.02


def test_permutation_is_a_permutation():
    p = W.permutation(10000, 5)
    assert np.array_equal(np.sort(p), np.arange(10000))
    assert not np.array_equal(p, np.arange(10000))


def test_torus_points_lie_on_the_torus():
    p, _ = W.torus(20000, 11)
    rho = np.hypot(p[:, 0].astype(np.float64), p[:, 1].astype(np.float64))
    tube = np.hypot(rho - 1.0, p[:, 2].astype(np.float64))
    assert np.all(np.abs(tube - 0.3) < 1e-3)        # sigma 1e-4 along the normal


def test_displacement_lengths_and_directions():
    """displace: lengths uniform in [0, ratio * diagonal), directions
    isotropic (mean unit vector near 0)."""
    p, _ = W.bumpy_sphere(50000, 51)
    ratio = 0.05
    q = W.displace(p, ratio, 52)
    v = q.astype(np.float64) - p.astype(np.float64)
    d = np.linalg.norm(p.max(0).astype(np.float64) - p.min(0).astype(np.float64))
    length = np.linalg.norm(v, axis=1)
    assert length.max() <= ratio * d * (1 + 1e-6)
    assert abs(length.mean() / (ratio * d) - 0.5) < 0.01
    unit = v / np.maximum(length, 1e-30)[:, None]
    assert np.all(np.abs(unit.mean(axis=0)) < 0.02)
    assert np.array_equal(W.displace(p, 0.0, 52), p)


def test_uniform_volume_and_degraded_workloads():
    w = W.uniform_volume(20000, 5000, 8)
    assert w.points.min() >= -1.0 and w.points.max() < 1.0
    assert w.queries.min() >= -1.0 and w.queries.max() <= 1.0
    s = W.degraded_bumpy(0.0, 2000, 100)
    t = W.degraded_bumpy(0.01, 2000, 100)
    assert not np.array_equal(s.points, t.points)
    assert np.array_equal(s.order, t.order)
