"""Successor lists from their definition (Sec. 3; Fig. 2's caption).

j > i is in L_i iff inserting p_j prunes the Voronoi cell of p_i in the
diagram of P_{1:j}, i.e. iff p_i and p_j are Delaunay neighbours in
DT(P_{1:j}). Computed here the slow way: one library Delaunay
triangulation (scipy.spatial.Delaunay, Qhull) per prefix, read off the
neighbours of the newest vertex. Prefixes of at most four points are
taken complete (every pair adjacent), a superset that keeps the query
exact. Only meaningful for points in general position (no five
cospherical, no four coplanar), where the triangulation is unique.

Test infrastructure only; see the package docstring.
"""
from __future__ import annotations

import numpy as np
from scipy.spatial import Delaunay


def successor_lists(P: np.ndarray) -> list[list[int]]:
    """L[i] = ascending list of successors of rank i, from the definition."""
    P64 = np.asarray(P, dtype=np.float32).astype(np.float64)
    n = P64.shape[0]
    L: list[list[int]] = [[] for _ in range(n)]
    for j in range(1, n):
        if j <= 3:
            nbrs = range(j)
        else:
            tri = Delaunay(P64[: j + 1])
            indptr, indices = tri.vertex_neighbor_vertices
            nbrs = sorted(int(v) for v in indices[indptr[j]:indptr[j + 1]])
        for i in nbrs:
            L[i].append(j)
    return L


def to_csr(L: list[list[int]]):
    rowp = np.zeros(len(L) + 1, dtype=np.int64)
    rowp[1:] = np.cumsum([len(x) for x in L])
    succ = np.array([v for x in L for v in x], dtype=np.int32)
    return rowp, succ
