"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package draws random numbers and shapes them into point clouds and
query sets. It holds none of the k-NN method's arithmetic: no distances, no
neighbour search, no successor structure. Everything is a pure function of
its integer seeds (a counter-based generator), so the same call gives the
same arrays on every machine up to the last-ulp behaviour of numpy's
transcendental functions.
"""
from .gen import (  # noqa: F401
    rand_u64, uniform, normal, permutation,
    sphere, torus, bumpy_sphere, patches4, lattice, uniform_cube,
    box_queries, near_surface_queries, bbox, SURFACES, surface, displace,
)
from .configs import (  # noqa: F401
    Workload, small_sphere, large_torus, prefix_bumpy, batch_clouds,
    serve_clouds, serve_requests, padded_box, Request, degraded_bumpy, uniform_volume,
)
