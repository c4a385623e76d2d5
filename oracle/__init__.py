"""Oracle: plain, slow, obviously correct CPU statements of what the k-NN
query path computes. TEST INFRASTRUCTURE ONLY.

Only the tests, the smoke check of the package entry point and the CPU
baseline leg of the benchmark may import anything from here. The product
library never does, and this package imports nothing from the product.

Contents
--------
knn            The definition (Theorem 1's N_k(q) with the tie rule of
               Eq. (2)): brute-force k nearest ranks in P_{1:m}, squared
               distances evaluated in float64 from the float32 inputs.
dpknn          Algorithm 1 (transition-site collection during the 1-NN
               descent) and Algorithm 2 (k-NN expansion over successor
               lists), step by step in float64, with per-query counters of
               rows opened, successor entries read and coordinates read.
successors     Successor lists from their definition (Sec. 3): j is in L_i
               iff p_j is a Delaunay neighbour of p_i in DT(P_{1:j}), using
               a library Delaunay triangulation of every prefix.

Parity status: every function here is pinned by tests that do not call
it to check itself (closed forms, exhaustive tiny cases, an independent
library triangulation, planted-mistake checks). Nothing is "parity
unpinned".
"""
