// Exact orient3d / insphere on float32 inputs (see predicates.h).
// Compile without -ffast-math and with -ffp-contract=off: the error
// analysis of the filters and the exactness of the expansion steps assume
// IEEE round-to-nearest double arithmetic with no implicit fusion.
#include "predicates.h"

#include <cmath>

namespace mknn {

namespace {

thread_local PredicateCounters g_counters;

// ---------------------------------------------------------------- expansions
// An expansion is an array of doubles, increasing in magnitude and
// non-overlapping, whose exact sum is the value represented. Zero
// components are dropped; the empty sum is stored as a single 0.

inline void two_sum(double a, double b, double& s, double& e) {
  s = a + b;
  double bv = s - a;
  double av = s - bv;
  e = (a - av) + (b - bv);
}

// Requires |a| >= |b| (or a == 0).
inline void fast_two_sum(double a, double b, double& s, double& e) {
  s = a + b;
  e = b - (s - a);
}

inline void two_prod(double a, double b, double& p, double& e) {
  p = a * b;
  e = std::fma(a, b, -p);
}

// h = e + b. h may alias e.
int grow(int elen, const double* e, double b, double* h) {
  double q = b;
  int k = 0;
  for (int i = 0; i < elen; ++i) {
    double s, t;
    two_sum(q, e[i], s, t);
    q = s;
    if (t != 0.0) h[k++] = t;
  }
  if (q != 0.0 || k == 0) h[k++] = q;
  return k;
}

// h = e * b. h must not alias e; capacity 2 * elen.
int scale(int elen, const double* e, double b, double* h) {
  double q, t0;
  int k = 0;
  two_prod(e[0], b, q, t0);
  if (t0 != 0.0) h[k++] = t0;
  for (int i = 1; i < elen; ++i) {
    double hi, lo, s, u;
    two_prod(e[i], b, hi, lo);
    two_sum(q, lo, s, u);
    if (u != 0.0) h[k++] = u;
    fast_two_sum(hi, s, q, u);
    if (u != 0.0) h[k++] = u;
  }
  if (q != 0.0 || k == 0) h[k++] = q;
  return k;
}

// Shortens an expansion without changing its value (two sweeps of
// fast_two_sum, top-down then bottom-up). h may alias e.
int compress(int elen, double* e, double* h) {
  if (elen <= 1) {
    h[0] = e[0];
    return 1;
  }
  double gp[1024];  // callers keep expansions at or below 1024 components
  int bottom = elen - 1;
  double q = e[elen - 1];
  for (int i = elen - 2; i >= 0; --i) {
    double s, t;
    fast_two_sum(q, e[i], s, t);
    if (t != 0.0) {
      gp[bottom--] = s;
      q = t;
    } else {
      q = s;
    }
  }
  gp[bottom] = q;
  int top = 0;
  for (int i = bottom + 1; i < elen; ++i) {
    double s, t;
    fast_two_sum(gp[i], q, s, t);
    if (t != 0.0) h[top++] = t;
    q = s;
  }
  h[top++] = q;
  return top;
}

inline int sign_of(int len, const double* e) {
  double v = e[len - 1];
  return v > 0.0 ? 1 : (v < 0.0 ? -1 : 0);
}

// Accumulates terms exactly; compresses when long.
struct Acc {
  double v[1024];
  int n = 1;
  Acc() { v[0] = 0.0; }
  void add(double x) {
    if (x == 0.0) return;
    n = grow(n, v, x, v);
    if (n > 600) n = compress(n, v, v);
  }
  void add_exp(int len, const double* e) {
    for (int i = 0; i < len; ++i) add(e[i]);
  }
  int finish() {
    n = compress(n, v, v);
    return n;
  }
};

// s * x * y * z exactly (x*y is exact in double for float inputs).
inline void add_triple(Acc& acc, double s, float x, float y, float z) {
  double xy = (double)x * (double)y;
  double p, e;
  two_prod(xy, (double)z, p, e);
  acc.add(s * p);
  acc.add(s * e);
}

// det3 of rows u, v, w (float coordinates) exactly, accumulated with sign s.
inline void add_det3(Acc& acc, double s, const float* u, const float* v, const float* w) {
  add_triple(acc, s, u[0], v[1], w[2]);
  add_triple(acc, -s, u[0], v[2], w[1]);
  add_triple(acc, -s, u[1], v[0], w[2]);
  add_triple(acc, s, u[1], v[2], w[0]);
  add_triple(acc, s, u[2], v[0], w[1]);
  add_triple(acc, -s, u[2], v[1], w[0]);
}

// det4 of rows [p_i, 1] (i = 0..3) exactly, as an expansion in out.
int det4_ones(const float* const* p, double* out) {
  Acc acc;
  // cofactor expansion along the column of ones: sum_i (-1)^(i+3) det3(rows != i)
  add_det3(acc, -1.0, p[1], p[2], p[3]);
  add_det3(acc, 1.0, p[0], p[2], p[3]);
  add_det3(acc, -1.0, p[0], p[1], p[3]);
  add_det3(acc, 1.0, p[0], p[1], p[2]);
  int n = acc.finish();
  for (int i = 0; i < n; ++i) out[i] = acc.v[i];
  return n;
}

}  // namespace

PredicateCounters& predicate_counters() { return g_counters; }

int orient3d_exact(const float* a, const float* b, const float* c, const float* d) {
  const float* p[4] = {a, b, c, d};
  double e[1024];
  int n = det4_ones(p, e);
  // det[b-a; c-a; d-a] = -det[[a,1],[b,1],[c,1],[d,1]]
  return -sign_of(n, e);
}

int insphere_exact(const float* a, const float* b, const float* c, const float* d, const float* e) {
  const float* pts[5] = {a, b, c, d, e};
  Acc total;
  double m4[1024];
  double w[3];
  double prod[2048];
  for (int i = 0; i < 5; ++i) {
    const float* rest[4];
    int r = 0;
    for (int j = 0; j < 5; ++j)
      if (j != i) rest[r++] = pts[j];
    int mlen = det4_ones(rest, m4);
    // w_i = x^2 + y^2 + z^2 exactly (each square is exact in double)
    double wx = (double)pts[i][0] * pts[i][0];
    double wy = (double)pts[i][1] * pts[i][1];
    double wz = (double)pts[i][2] * pts[i][2];
    int wl = 1;
    w[0] = wx;
    wl = grow(wl, w, wy, w);
    wl = grow(wl, w, wz, w);
    // cofactor sign along the lifted column (index 3) of the 5x5 matrix
    double s = ((i + 3) & 1) ? -1.0 : 1.0;
    for (int t = 0; t < wl; ++t) {
      if (w[t] == 0.0) continue;
      int pl = scale(mlen, m4, s * w[t], prod);
      total.add_exp(pl, prod);
    }
  }
  int n = total.finish();
  // det5 of rows [p, |p|^2, 1] is negative when e is inside (positive orientation)
  return -sign_of(n, total.v);
}

bool collinear3(const float* a, const float* b, const float* c) {
  // all three coordinate-plane orientations vanish exactly
  const int ax[3][2] = {{0, 1}, {1, 2}, {2, 0}};
  for (auto& pr : ax) {
    int i = pr[0], j = pr[1];
    Acc acc;
    // (a_i b_j - a_j b_i) + (b_i c_j - b_j c_i) + (c_i a_j - c_j a_i)
    const float* P[3] = {a, b, c};
    for (int t = 0; t < 3; ++t) {
      const float* u = P[t];
      const float* v = P[(t + 1) % 3];
      acc.add((double)u[i] * v[j]);
      acc.add(-(double)u[j] * v[i]);
    }
    int n = acc.finish();
    if (sign_of(n, acc.v) != 0) return false;
  }
  return true;
}

int orient3d(const float* a, const float* b, const float* c, const float* d) {
  g_counters.orient_calls++;
  double bx = (double)b[0] - a[0], by = (double)b[1] - a[1], bz = (double)b[2] - a[2];
  double cx = (double)c[0] - a[0], cy = (double)c[1] - a[1], cz = (double)c[2] - a[2];
  double dx = (double)d[0] - a[0], dy = (double)d[1] - a[1], dz = (double)d[2] - a[2];
  double m1 = cy * dz, m2 = cz * dy;
  double m3 = cx * dz, m4 = cz * dx;
  double m5 = cx * dy, m6 = cy * dx;
  double det = bx * (m1 - m2) - by * (m3 - m4) + bz * (m5 - m6);
  double perm = std::fabs(bx) * (std::fabs(m1) + std::fabs(m2)) +
                std::fabs(by) * (std::fabs(m3) + std::fabs(m4)) +
                std::fabs(bz) * (std::fabs(m5) + std::fabs(m6));
  // The rounding error of this evaluation is below ~8 eps * perm (eps = 2^-53);
  // 1e-13 * perm leaves a wide margin.
  double bound = 1e-13 * perm;
  if (det > bound) return 1;
  if (-det > bound) return -1;
  g_counters.orient_exact++;
  return orient3d_exact(a, b, c, d);
}

int insphere(const float* a, const float* b, const float* c, const float* d, const float* e) {
  g_counters.insphere_calls++;
  const float* p[4] = {a, b, c, d};
  double X[4], Y[4], Z[4], Wt[4];
  for (int i = 0; i < 4; ++i) {
    X[i] = (double)p[i][0] - e[0];
    Y[i] = (double)p[i][1] - e[1];
    Z[i] = (double)p[i][2] - e[2];
    Wt[i] = X[i] * X[i] + Y[i] * Y[i] + Z[i] * Z[i];
  }
  // det4 of translated rows (X, Y, Z, W), expanded along W:
  // sum_i (-1)^(i+3) W_i det3(rows != i)
  double det = 0.0, perm = 0.0;
  for (int i = 0; i < 4; ++i) {
    int r[3], t = 0;
    for (int j = 0; j < 4; ++j)
      if (j != i) r[t++] = j;
    double a1 = Y[r[1]] * Z[r[2]], a2 = Z[r[1]] * Y[r[2]];
    double b1 = X[r[1]] * Z[r[2]], b2 = Z[r[1]] * X[r[2]];
    double c1 = X[r[1]] * Y[r[2]], c2 = Y[r[1]] * X[r[2]];
    double d3 = X[r[0]] * (a1 - a2) - Y[r[0]] * (b1 - b2) + Z[r[0]] * (c1 - c2);
    double p3 = std::fabs(X[r[0]]) * (std::fabs(a1) + std::fabs(a2)) +
                std::fabs(Y[r[0]]) * (std::fabs(b1) + std::fabs(b2)) +
                std::fabs(Z[r[0]]) * (std::fabs(c1) + std::fabs(c2));
    double s = ((i + 3) & 1) ? -1.0 : 1.0;
    det += s * Wt[i] * d3;
    perm += Wt[i] * p3;
  }
  // Error below ~20 eps * perm; 1e-13 * perm leaves a wide margin.
  double bound = 1e-13 * perm;
  if (det > bound) return -1;   // det4 > 0: outside
  if (-det > bound) return 1;   // det4 < 0: inside
  g_counters.insphere_exact++;
  return insphere_exact(a, b, c, d, e);
}

}  // namespace mknn
