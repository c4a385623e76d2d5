// CPU baselines: an exact kd-tree with prefix support, and Algorithms 1-2
// (Sec. 4) run query by query on the host. See mknn_cpu.h.
#include "mknn_cpu.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <limits>
#include <thread>
#include <vector>

namespace {

// Squared distance in float64, ((dx*dx + dy*dy) + dz*dz), no fusion (the
// file is compiled with -ffp-contract=off).
inline double sqd(const float* q, const float* p) {
  const double dx = (double)q[0] - (double)p[0];
  const double dy = (double)q[1] - (double)p[1];
  const double dz = (double)q[2] - (double)p[2];
  return (dx * dx + dy * dy) + dz * dz;
}

inline bool key_lt(double da, int32_t ra, double db, int32_t rb) {
  return da < db || (da == db && ra < rb);
}

// The best min(k, m) keys so far, ascending; insertion sort (Sec. 5.5).
struct Best {
  int cap = 0, cnt = 0;
  double d[128];
  int32_t r[128];
  bool done[128];
  void reset(int c) {
    cap = c;
    cnt = 0;
  }
  bool full() const { return cnt == cap; }
  // would (dd, rr) enter the list?
  bool admits(double dd, int32_t rr) const {
    return cnt < cap || key_lt(dd, rr, d[cnt - 1], r[cnt - 1]);
  }
  // Inserts unless the same key is present. Returns the position, -1 if
  // present, -2 if not admitted.
  int insert(double dd, int32_t rr) {
    if (!admits(dd, rr)) return -2;
    int pos = cnt;
    while (pos > 0 && key_lt(dd, rr, d[pos - 1], r[pos - 1])) --pos;
    if (pos > 0 && d[pos - 1] == dd && r[pos - 1] == rr) return -1;
    const int last = cnt < cap ? cnt : cap - 1;
    for (int i = last; i > pos; --i) {
      d[i] = d[i - 1];
      r[i] = r[i - 1];
      done[i] = done[i - 1];
    }
    d[pos] = dd;
    r[pos] = rr;
    done[pos] = false;
    if (cnt < cap) ++cnt;
    return pos;
  }
  void write(int k, int32_t* oi, float* od) const {
    for (int i = 0; i < k; ++i) {
      if (i < cnt) {
        oi[i] = r[i];
        od[i] = (float)d[i];
      } else {
        oi[i] = -1;
        od[i] = std::numeric_limits<float>::infinity();
      }
    }
  }
};

// Processing order of the queries: input order, or (sorted) the Morton
// order of their cells in a 1024^3 grid over the queries' bounding box, so
// that consecutive queries on a thread touch the same tree nodes or
// successor rows (each result still goes to its own row).
std::vector<int64_t> query_order(const float* q, int64_t nq, int32_t q_stride, bool sorted) {
  std::vector<int64_t> ord(nq);
  for (int64_t i = 0; i < nq; ++i) ord[i] = i;
  if (!sorted || nq < 2) return ord;
  float lo[3], hi[3];
  for (int a = 0; a < 3; ++a) {
    lo[a] = std::numeric_limits<float>::infinity();
    hi[a] = -std::numeric_limits<float>::infinity();
  }
  for (int64_t i = 0; i < nq; ++i)
    for (int a = 0; a < 3; ++a) {
      const float v = q[i * q_stride + a];
      if (v == v) {
        lo[a] = std::min(lo[a], v);
        hi[a] = std::max(hi[a], v);
      }
    }
  auto spread = [](uint64_t v) {
    uint64_t out = 0;
    for (int b = 0; b < 10; ++b) out |= ((v >> b) & 1ull) << (3 * b);
    return out;
  };
  std::vector<std::pair<uint64_t, int64_t>> key(nq);
  for (int64_t i = 0; i < nq; ++i) {
    uint64_t code = 0;
    for (int a = 0; a < 3; ++a) {
      const float ext = hi[a] - lo[a];
      const float v = q[i * q_stride + a];
      int64_t c = (ext > 0 && v == v) ? (int64_t)((v - lo[a]) / ext * 1024.f) : 0;
      c = std::min<int64_t>(1023, std::max<int64_t>(0, c));
      code |= spread((uint64_t)c) << a;
    }
    key[i] = {code, i};
  }
  std::sort(key.begin(), key.end());
  for (int64_t i = 0; i < nq; ++i) ord[i] = key[i].second;
  return ord;
}

template <class F>
void parallel_for(int64_t nq, int threads, F&& body) {
  const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
  int nt = threads > 0 ? threads : hw;
  const int64_t chunk = 256;
  if ((int64_t)nt > (nq + chunk - 1) / chunk) nt = (int)std::max<int64_t>(1, (nq + chunk - 1) / chunk);
  std::atomic<int64_t> next{0};
  auto worker = [&]() {
    for (;;) {
      const int64_t b = next.fetch_add(chunk);
      if (b >= nq) break;
      const int64_t e = std::min(nq, b + chunk);
      for (int64_t i = b; i < e; ++i) body(i);
    }
  };
  if (nt == 1) {
    worker();
    return;
  }
  std::vector<std::thread> pool;
  pool.reserve(nt);
  for (int t = 0; t < nt; ++t) pool.emplace_back(worker);
  for (auto& th : pool) th.join();
}

}  // namespace

// ------------------------------------------------------------------ kd-tree

struct mknn_cpu_kdtree {
  struct Node {
    float lo[3], hi[3];   // bounding box of the node's points
    int64_t begin, end;   // range in pts / rank
    int32_t left, right;  // children, -1 for a leaf
    int32_t min_rank;     // smallest rank below this node
  };
  std::vector<Node> nodes;
  std::vector<float> pts;      // xyz in leaf order
  std::vector<int32_t> rank;   // rank of each point in leaf order
  int64_t n = 0;
};

namespace {

int32_t build_node(mknn_cpu_kdtree* t, std::vector<int32_t>& ids, const float* xyz, int64_t b,
                   int64_t e, int leaf) {
  mknn_cpu_kdtree::Node nd;
  for (int a = 0; a < 3; ++a) {
    nd.lo[a] = std::numeric_limits<float>::infinity();
    nd.hi[a] = -std::numeric_limits<float>::infinity();
  }
  int32_t mr = std::numeric_limits<int32_t>::max();
  for (int64_t i = b; i < e; ++i) {
    const float* p = xyz + 3 * (int64_t)ids[i];
    for (int a = 0; a < 3; ++a) {
      nd.lo[a] = std::min(nd.lo[a], p[a]);
      nd.hi[a] = std::max(nd.hi[a], p[a]);
    }
    mr = std::min(mr, ids[i]);
  }
  nd.begin = b;
  nd.end = e;
  nd.left = nd.right = -1;
  nd.min_rank = mr;
  const int32_t me = (int32_t)t->nodes.size();
  t->nodes.push_back(nd);
  if (e - b > leaf) {
    int ax = 0;
    for (int a = 1; a < 3; ++a)
      if (nd.hi[a] - nd.lo[a] > nd.hi[ax] - nd.lo[ax]) ax = a;
    const int64_t mid = b + (e - b) / 2;
    std::nth_element(ids.begin() + b, ids.begin() + mid, ids.begin() + e,
                     [&](int32_t x, int32_t y) {
                       const float px = xyz[3 * (int64_t)x + ax], py = xyz[3 * (int64_t)y + ax];
                       return px < py || (px == py && x < y);
                     });
    const int32_t l = build_node(t, ids, xyz, b, mid, leaf);
    const int32_t r = build_node(t, ids, xyz, mid, e, leaf);
    t->nodes[me].left = l;
    t->nodes[me].right = r;
  }
  return me;
}

// Lower bound of the float64 distance from q to any point in the box
// (same operations as sqd on the clamped point, so it never exceeds it).
inline double box_dist(const float* q, const mknn_cpu_kdtree::Node& nd) {
  float c[3];
  for (int a = 0; a < 3; ++a) c[a] = std::min(std::max(q[a], nd.lo[a]), nd.hi[a]);
  return sqd(q, c);
}

void kd_search(const mknn_cpu_kdtree* t, int32_t ni, const float* q, int32_t m, Best& B) {
  const auto& nd = t->nodes[ni];
  if (nd.left < 0) {
    for (int64_t i = nd.begin; i < nd.end; ++i) {
      const int32_t r = t->rank[i];
      if (r >= m) continue;
      const double d = sqd(q, &t->pts[3 * i]);
      if (B.admits(d, r)) B.insert(d, r);
    }
    return;
  }
  const auto& L = t->nodes[nd.left];
  const auto& R = t->nodes[nd.right];
  const double dl = L.min_rank < m ? box_dist(q, L) : std::numeric_limits<double>::infinity();
  const double dr = R.min_rank < m ? box_dist(q, R) : std::numeric_limits<double>::infinity();
  const int32_t first = dl <= dr ? nd.left : nd.right;
  const int32_t second = dl <= dr ? nd.right : nd.left;
  const double d1 = dl <= dr ? dl : dr, d2 = dl <= dr ? dr : dl;
  // a box farther than the k-th key cannot hold a better point; a box at
  // exactly that distance may hold an equal distance with a lower rank
  if (d1 != std::numeric_limits<double>::infinity() && (!B.full() || d1 <= B.d[B.cnt - 1]))
    kd_search(t, first, q, m, B);
  if (d2 != std::numeric_limits<double>::infinity() && (!B.full() || d2 <= B.d[B.cnt - 1]))
    kd_search(t, second, q, m, B);
}

bool valid_common(int64_t nq, int32_t q_stride, int32_t k, const int32_t* m, int32_t m_scalar,
                  int64_t n, const float* q, const int32_t* oi, const float* od) {
  if (nq < 0 || q_stride < 3 || k < 1 || k > 128 || n < 1) return false;
  if (!m && (m_scalar < 0 || m_scalar > n)) return false;
  if (nq > 0 && (!q || !oi || !od)) return false;
  return true;
}

}  // namespace

extern "C" int mknn_cpu_kdtree_build(const float* xyz, int64_t n, int32_t leaf,
                                     mknn_cpu_kdtree** out) {
  if (!xyz || !out || n < 1 || n >= (int64_t)std::numeric_limits<int32_t>::max()) return -1;
  if (leaf <= 0) leaf = 8;
  auto* t = new mknn_cpu_kdtree();
  t->n = n;
  std::vector<int32_t> ids(n);
  for (int64_t i = 0; i < n; ++i) ids[i] = (int32_t)i;
  t->nodes.reserve(2 * (size_t)(n / leaf + 1));
  build_node(t, ids, xyz, 0, n, leaf);
  t->pts.resize(3 * (size_t)n);
  t->rank.resize(n);
  for (int64_t i = 0; i < n; ++i) {
    std::memcpy(&t->pts[3 * i], xyz + 3 * (int64_t)ids[i], 3 * sizeof(float));
    t->rank[i] = ids[i];
  }
  *out = t;
  return 0;
}

extern "C" void mknn_cpu_kdtree_free(mknn_cpu_kdtree* t) { delete t; }

extern "C" int mknn_cpu_kdtree_knn(const mknn_cpu_kdtree* t, const float* q, int64_t nq,
                                   int32_t q_stride, int32_t k, const int32_t* m,
                                   int32_t m_scalar, int32_t* out_idx, float* out_d2,
                                   int32_t sorted, int32_t threads) {
  if (!t || !valid_common(nq, q_stride, k, m, m_scalar, t->n, q, out_idx, out_d2)) return -1;
  const int32_t n = (int32_t)t->n;
  const int32_t ms = m_scalar == 0 ? n : m_scalar;
  std::atomic<int> bad{0};
  const std::vector<int64_t> ord = query_order(q, nq, q_stride, sorted != 0);
  parallel_for(nq, threads, [&](int64_t j) {
    const int64_t i = ord[j];
    const int32_t mi = m ? m[i] : ms;
    int32_t* oi = out_idx + i * k;
    float* od = out_d2 + i * k;
    Best B;
    if (mi < 1 || mi > n) {
      B.reset(1);
      B.write(k, oi, od);
      bad.store(1);
      return;
    }
    B.reset(std::min(k, mi));
    kd_search(t, 0, q + i * q_stride, mi, B);
    B.write(k, oi, od);
  });
  return bad.load() ? -2 : 0;
}

// ------------------------------------------------- Algorithms 1 and 2

extern "C" int mknn_cpu_dpknn(const float* xyz, int64_t n, const int64_t* rowp,
                              const int32_t* succ, const float* q, int64_t nq, int32_t q_stride,
                              int32_t k, const int32_t* m, int32_t m_scalar, int32_t* out_idx,
                              float* out_d2, int64_t* counters, int32_t sorted, int32_t threads) {
  if (!xyz || !rowp || !succ || !valid_common(nq, q_stride, k, m, m_scalar, n, q, out_idx, out_d2))
    return -1;
  const int32_t ms = m_scalar == 0 ? (int32_t)n : m_scalar;
  std::atomic<int> bad{0};
  const std::vector<int64_t> ord = query_order(q, nq, q_stride, sorted != 0);
  parallel_for(nq, threads, [&](int64_t j) {
    const int64_t i = ord[j];
    const int32_t mi = m ? m[i] : ms;
    const float* qi = q + i * q_stride;
    int32_t* oi = out_idx + i * k;
    float* od = out_d2 + i * k;
    Best N;
    int64_t c[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (mi < 1 || mi > n) {
      N.reset(1);
      N.write(k, oi, od);
      bad.store(1);
      if (counters) std::memcpy(counters + 8 * i, c, sizeof c);
      return;
    }
    N.reset(std::min(k, mi));
    auto offer = [&](double d, int32_t r) {
      if (!N.admits(d, r)) return;
      ++c[4];
      const int pos = N.insert(d, r);
      if (pos == -1) {
        ++c[5];
      } else if (pos >= 0) {
        ++c[6];
        c[7] += pos;
      }
    };
    // Algorithm 1: from p_1, move to the first strictly closer successor
    // (lists ascending, scan restarted at the head of the new list); every
    // site moved to is a transition site and a candidate
    int32_t cur = 0;
    double dcur = sqd(qi, xyz);
    c[2] = 1;
    c[3] = 1;
    offer(dcur, 0);
    for (bool moved = true; moved;) {
      moved = false;
      ++c[0];
      for (int64_t e = rowp[cur]; e < rowp[cur + 1]; ++e) {
        const int32_t s = succ[e];
        ++c[1];
        if (s >= mi) break;
        const double d = sqd(qi, xyz + 3 * (int64_t)s);
        ++c[2];
        if (d < dcur) {
          cur = s;
          dcur = d;
          ++c[3];
          offer(d, s);
          moved = true;
          break;
        }
      }
    }
    // Algorithm 2: expand the nearest not-yet-expanded entry among the
    // first k-1 until none is left
    for (;;) {
      const int lim = std::min(N.cnt, k - 1);
      int p = 0;
      while (p < lim && N.done[p]) ++p;
      if (p >= lim) break;
      N.done[p] = true;
      const int32_t site = N.r[p];
      ++c[0];
      for (int64_t e = rowp[site]; e < rowp[site + 1]; ++e) {
        const int32_t s = succ[e];
        ++c[1];
        if (s >= mi) break;
        ++c[2];
        offer(sqd(qi, xyz + 3 * (int64_t)s), s);
      }
    }
    N.write(k, oi, od);
    if (counters) std::memcpy(counters + 8 * i, c, sizeof c);
  });
  return bad.load() ? -2 : 0;
}

extern "C" int32_t mknn_cpu_threads(void) {
  return (int32_t)std::max(1u, std::thread::hardware_concurrency());
}
