// Exact geometric predicates on float32 coordinates, used by the host-side
// incremental Delaunay builder that produces the successor table (Sec. 3).
//
// Method: a float64 evaluation with a forward error bound decides the sign
// when it is clear; otherwise the determinant is evaluated exactly with
// floating-point expansion arithmetic (the adaptive-precision method of
// J. R. Shewchuk, "Adaptive Precision Floating-Point Arithmetic and Fast
// Robust Geometric Predicates", Discrete Comput. Geom. 18, 1997): sums and
// products of float64 values carried as non-overlapping sequences whose
// exact sum is the value. Every product of float32 inputs is exact in that
// representation, so the sign returned is the sign of the exact real
// determinant of the given float32 coordinates.
#pragma once
#include <cstdint>

namespace mknn {

// Sign of det[b-a; c-a; d-a]: +1 when d lies on the side of plane (a,b,c)
// towards which (b-a) x (c-a) points, -1 on the other side, 0 if coplanar.
int orient3d(const float* a, const float* b, const float* c, const float* d);

// For a, b, c, d with orient3d(a,b,c,d) > 0: +1 if e lies strictly inside
// their circumsphere, 0 on it, -1 outside. (For negative orientation the
// sign flips.)
int insphere(const float* a, const float* b, const float* c, const float* d, const float* e);

// Exact test: are a, b, c collinear (or coincident)?
bool collinear3(const float* a, const float* b, const float* c);

struct PredicateCounters {
  uint64_t orient_calls = 0, orient_exact = 0;
  uint64_t insphere_calls = 0, insphere_exact = 0;
};
// Per-thread counters (the builder runs one cloud per thread).
PredicateCounters& predicate_counters();

// The exact stages alone (no filter), for tests of the filter.
int orient3d_exact(const float* a, const float* b, const float* c, const float* d);
int insphere_exact(const float* a, const float* b, const float* c, const float* d, const float* e);

}  // namespace mknn
