// Incremental 3D Delaunay (Bowyer-Watson) producing successor lists.
//
// Data structure: tetrahedra with 4 vertex ranks and 4 neighbour links
// (neighbour i lies across the face opposite vertex i). The unbounded side
// is closed by "infinite" tetrahedra that join each hull face to a vertex
// at infinity (INF). Finite tetrahedra are positively oriented
// (orient3d(v0,v1,v2,v3) > 0); an infinite tetrahedron is oriented so
// that putting any point strictly outside its hull face in place of INF
// gives a positive orientation.
//
// Insertion of p_j:
//   1. nearest earlier site by the successor-list descent of Sec. 3 over
//      the lists built so far (exactly the 1-NN in P_{1:j-1});
//   2. a visibility walk from a tetrahedron incident to that site to a
//      tetrahedron in conflict with p_j (the nearest site is always a
//      Delaunay neighbour of p_j, so the walk is short);
//   3. breadth-first growth of the conflict cavity;
//   4. the cavity is replaced by tetrahedra joining p_j to its boundary
//      faces, and j is appended to L_v for every boundary vertex v.
//
// Degeneracies: a point exactly on a circumsphere counts as in conflict,
// and a point in the plane of a hull face conflicts with the infinite
// tetrahedron of that face iff it lies inside or on the face's circumcircle
// (tested as insphere against the finite tetrahedron behind the face,
// whose sphere cuts that plane in exactly this circle). This is the
// symbolic perturbation that lowers each newly inserted point's lifted
// coordinate by an infinitesimal that dominates those of all earlier
// points, so the result is a Delaunay triangulation of the perturbed
// points and hence a valid Delaunay triangulation of the input.
//
// Ranks 0..j0, where j0 is the first rank that makes the prefix
// non-coplanar, get complete lists (every later rank of that prefix);
// this superset keeps queries exact. A rank whose coordinates equal an
// earlier rank's is not inserted into the triangulation; it is appended
// to its twin's list (it ties with the twin, which ranks first).
#include "builder.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <tuple>

#include "predicates.h"

namespace mknn {

namespace build_detail {

constexpr int32_t INF = -1;
constexpr int32_t DEAD = -2;

struct Lists {
  static constexpr int kB = 14;
  struct Block {
    int32_t e[kB];
    int32_t next;
    int32_t cnt;
  };
  std::vector<Block> pool;
  std::vector<int32_t> head, tail, len;
  int64_t total = 0, longest = 0;

  void init(int64_t n) {
    head.assign(n, -1);
    tail.assign(n, -1);
    len.assign(n, 0);
    pool.reserve((size_t)n + 16);
  }
  void pop(int32_t i) {  // removes row i's last entry (undoing an append)
    int32_t t = tail[i];
    if (t < 0) return;
    pool[t].cnt--;
    len[i]--;
    total--;
    if (pool[t].cnt == 0) {  // unlink the emptied block (it stays unused in the pool)
      if (head[i] == t) {
        head[i] = tail[i] = -1;
      } else {
        int32_t b = head[i];
        while (pool[b].next != t) b = pool[b].next;
        pool[b].next = -1;
        tail[i] = b;
      }
    }
  }
  void grow(int64_t n) {  // rows for new ranks, empty
    head.resize(n, -1);
    tail.resize(n, -1);
    len.resize(n, 0);
  }
  void append(int32_t i, int32_t j) {
    int32_t t = tail[i];
    if (t < 0 || pool[t].cnt == kB) {
      int32_t b = (int32_t)pool.size();
      pool.emplace_back();
      pool[b].next = -1;
      pool[b].cnt = 0;
      if (t < 0)
        head[i] = b;
      else
        pool[t].next = b;
      tail[i] = b;
      t = b;
    }
    pool[t].e[pool[t].cnt++] = j;
    len[i]++;
    total++;
    if (len[i] > longest) longest = len[i];
  }
};

inline bool same_point(const float* a, const float* b) {
  return a[0] == b[0] && a[1] == b[1] && a[2] == b[2];
}

inline double dist2(const float* a, const float* b) {
  double dx = (double)a[0] - b[0], dy = (double)a[1] - b[1], dz = (double)a[2] - b[2];
  return dx * dx + dy * dy + dz * dz;
}

class Builder {
 public:
  Builder(const float* xyz, int64_t n) : X_(xyz), n_((int32_t)n) {}

  bool run(bool keep_tets, SuccessorTable* out, std::string* err);
  // Inserts ranks n_ .. n_new-1 of xyz (the same points below n_); each
  // successor entry added is reported as (row, rank) in `added`.
  bool append(const float* xyz, int32_t n_new, std::vector<std::pair<int32_t, int32_t>>* added,
              std::string* err);
  void csr(std::vector<int64_t>* rowp, std::vector<int32_t>* succ) const;
  int32_t size() const { return n_; }
  int64_t row_len(int32_t i) const { return L_.len[i]; }
  int64_t longest_row() const { return L_.longest; }
  void row_tail(int32_t i, int64_t from, std::vector<int32_t>* out) const {
    int64_t at = 0;
    for (int32_t bk = L_.head[i]; bk >= 0; bk = L_.pool[bk].next)
      for (int q = 0; q < L_.pool[bk].cnt; ++q, ++at)
        if (at >= from) out->push_back(L_.pool[bk].e[q]);
  }
  bool has_tetrahedron() const { return tet_made_ && !broken_; }
  const BuildStats& stats() const { return st_; }

 private:
  // One rank after the degenerate prefix: descent to its nearest earlier
  // site over the lists so far, then insertion (or a duplicate's entry).
  // Returns false on a location failure.
  bool insert_rank(int32_t j, std::string* err);
  const float* P(int32_t v) const { return X_ + 3 * (int64_t)v; }
  bool is_inf(int32_t t) const {
    const int32_t* v = &V_[4 * (size_t)t];
    return v[0] == INF || v[1] == INF || v[2] == INF || v[3] == INF;
  }
  int inf_pos(int32_t t) const {
    const int32_t* v = &V_[4 * (size_t)t];
    for (int i = 0; i < 4; ++i)
      if (v[i] == INF) return i;
    return -1;
  }
  uint32_t rnd() {
    rng_ ^= rng_ << 13;
    rng_ ^= rng_ >> 7;
    rng_ ^= rng_ << 17;
    return (uint32_t)rng_;
  }
  int32_t alloc_tet() {
    int32_t t;
    if (!free_.empty()) {
      t = free_.back();
      free_.pop_back();
    } else {
      t = (int32_t)(V_.size() / 4);
      V_.resize(V_.size() + 4);
      N_.resize(N_.size() + 4);
      mark_.push_back(0);
    }
    mark_[t] = 0;
    return t;
  }
  void release_tet(int32_t t) {
    V_[4 * (size_t)t] = DEAD;
    V_[4 * (size_t)t + 1] = DEAD;
    V_[4 * (size_t)t + 2] = DEAD;
    V_[4 * (size_t)t + 3] = DEAD;
    free_.push_back(t);
  }

  bool conflict(int32_t t, const float* p);
  int32_t locate(int32_t start, const float* p);
  int32_t scan_for_conflict(const float* p);
  // Returns: 0 inserted, 1 duplicate (sets twin), -1 failure.
  int insert(int32_t j, int32_t start, bool record);
  void initial_tet(int32_t a, int32_t b, int32_t c, int32_t d);

  const float* X_;
  int32_t n_;
  bool tet_made_ = false;
  bool broken_ = false;  // an append failed: lists rolled back, no more appends
  std::vector<std::pair<int32_t, int32_t>>* added_ = nullptr;
  std::vector<int32_t> V_, N_;
  std::vector<uint32_t> mark_;
  std::vector<int32_t> free_;
  std::vector<int32_t> vtet_, twin_;
  std::vector<uint32_t> vstamp_;
  uint32_t stamp_ = 0;
  uint64_t rng_ = 0x2545F4914F6CDD1DULL;
  Lists L_;
  BuildStats st_;

  // per-insertion scratch
  struct BFace {
    int32_t v[4];
    int32_t face;
    int32_t out;
    int32_t back;
  };
  std::vector<int32_t> cavity_;
  std::vector<BFace> bfaces_;
  struct Slot {
    uint64_t key;
    int32_t tet;
    int32_t face;
    uint32_t stamp;
  };
  std::vector<Slot> table_;
  uint32_t table_stamp_ = 0;
};

bool Builder::conflict(int32_t t, const float* p) {
  st_.conflict_tests++;
  const int32_t* v = &V_[4 * (size_t)t];
  int ip = inf_pos(t);
  if (ip < 0) return insphere(P(v[0]), P(v[1]), P(v[2]), P(v[3]), p) >= 0;
  const float* q[4];
  for (int i = 0; i < 4; ++i) q[i] = (i == ip) ? p : P(v[i]);
  int o = orient3d(q[0], q[1], q[2], q[3]);
  if (o != 0) return o > 0;
  int32_t fn = N_[4 * (size_t)t + ip];
  const int32_t* w = &V_[4 * (size_t)fn];
  return insphere(P(w[0]), P(w[1]), P(w[2]), P(w[3]), p) >= 0;
}

int32_t Builder::locate(int32_t t, const float* p) {
  if (is_inf(t)) t = N_[4 * (size_t)t + inf_pos(t)];
  int32_t prev = -1;
  const int64_t cap = 8 * (int64_t)n_ + 1024;
  for (int64_t it = 0; it < cap; ++it) {
    const int32_t* v = &V_[4 * (size_t)t];
    uint32_t r = rnd() & 3u;
    bool moved = false;
    for (uint32_t s = 0; s < 4; ++s) {
      int i = (int)((r + s) & 3u);
      int32_t nb = N_[4 * (size_t)t + i];
      if (nb == prev) continue;
      const float* q[4] = {P(v[0]), P(v[1]), P(v[2]), P(v[3])};
      q[i] = p;
      if (orient3d(q[0], q[1], q[2], q[3]) < 0) {
        prev = t;
        t = nb;
        moved = true;
        break;
      }
    }
    st_.walk_steps++;
    if (!moved || is_inf(t)) return t;
  }
  return -1;
}

int32_t Builder::scan_for_conflict(const float* p) {
  int32_t nt = (int32_t)(V_.size() / 4);
  for (int32_t t = 0; t < nt; ++t)
    if (V_[4 * (size_t)t] != DEAD && conflict(t, p)) return t;
  return -1;
}

void Builder::initial_tet(int32_t a, int32_t b, int32_t c, int32_t d) {
  int32_t t0 = alloc_tet();
  int32_t v[4] = {a, b, c, d};
  std::memcpy(&V_[4 * (size_t)t0], v, sizeof v);
  int32_t inf[4];
  for (int k = 0; k < 4; ++k) {
    int32_t t = alloc_tet();
    int32_t w[4] = {a, b, c, d};
    w[k] = INF;
    std::swap(w[(k + 1) & 3], w[(k + 2) & 3]);
    std::memcpy(&V_[4 * (size_t)t], w, sizeof w);
    inf[k] = t;
  }
  // link by matching faces (sorted vertex triples)
  std::map<std::tuple<int32_t, int32_t, int32_t>, std::pair<int32_t, int>> open;
  int32_t all[5] = {t0, inf[0], inf[1], inf[2], inf[3]};
  for (int32_t t : all) {
    for (int i = 0; i < 4; ++i) {
      int32_t f[3], m = 0;
      for (int j = 0; j < 4; ++j)
        if (j != i) f[m++] = V_[4 * (size_t)t + j];
      std::sort(f, f + 3);
      auto key = std::make_tuple(f[0], f[1], f[2]);
      auto it = open.find(key);
      if (it == open.end()) {
        open[key] = {t, i};
      } else {
        N_[4 * (size_t)t + i] = it->second.first;
        N_[4 * (size_t)it->second.first + it->second.second] = t;
        open.erase(it);
      }
    }
  }
  vtet_[a] = vtet_[b] = vtet_[c] = vtet_[d] = t0;
}

int Builder::insert(int32_t j, int32_t start, bool record) {
  const float* p = P(j);
  int32_t t0 = locate(start, p);
  if (t0 < 0) t0 = scan_for_conflict(p);
  if (t0 < 0) return -1;
  if (!is_inf(t0)) {
    for (int i = 0; i < 4; ++i) {
      int32_t w = V_[4 * (size_t)t0 + i];
      if (same_point(P(w), p)) {
        twin_[j] = twin_[w];
        return 1;
      }
    }
  }
  stamp_ += 2;
  const uint32_t IN = stamp_, OUT = stamp_ + 1;
  cavity_.clear();
  bfaces_.clear();
  mark_[t0] = IN;
  cavity_.push_back(t0);
  for (size_t ci = 0; ci < cavity_.size(); ++ci) {
    int32_t t = cavity_[ci];
    for (int i = 0; i < 4; ++i) {
      int32_t nb = N_[4 * (size_t)t + i];
      uint32_t mk = mark_[nb];
      if (mk == IN) continue;
      if (mk != OUT) {
        if (conflict(nb, p)) {
          mark_[nb] = IN;
          cavity_.push_back(nb);
          continue;
        }
        mark_[nb] = OUT;
      }
      BFace f;
      std::memcpy(f.v, &V_[4 * (size_t)t], sizeof f.v);
      f.v[i] = j;
      f.face = i;
      f.out = nb;
      f.back = -1;
      for (int k = 0; k < 4; ++k)
        if (N_[4 * (size_t)nb + k] == t) f.back = k;
      bfaces_.push_back(f);
    }
  }
  for (int32_t t : cavity_) release_tet(t);

  size_t want = 16;
  while (want < 4 * bfaces_.size()) want <<= 1;
  if (table_.size() < want) {
    table_.assign(want, Slot{0, 0, 0, 0});
    table_stamp_ = 0;
  }
  const size_t mask = table_.size() - 1;
  ++table_stamp_;
  for (const BFace& f : bfaces_) {
    int32_t nt = alloc_tet();
    std::memcpy(&V_[4 * (size_t)nt], f.v, sizeof f.v);
    N_[4 * (size_t)nt + f.face] = f.out;
    N_[4 * (size_t)f.out + f.back] = nt;
    for (int k = 0; k < 4; ++k) {
      if (k == f.face) continue;
      int32_t e[2], m = 0;
      for (int q = 0; q < 4; ++q)
        if (q != k && q != f.face) e[m++] = f.v[q];
      uint32_t ua = (uint32_t)e[0], ub = (uint32_t)e[1];
      if (ua > ub) std::swap(ua, ub);
      uint64_t key = ((uint64_t)ua << 32) | ub;
      size_t h = (size_t)((key * 0x9E3779B97F4A7C15ULL) >> 40) & mask;
      for (;;) {
        Slot& s = table_[h];
        if (s.stamp != table_stamp_) {
          s.stamp = table_stamp_;
          s.key = key;
          s.tet = nt;
          s.face = k;
          break;
        }
        if (s.key == key) {
          N_[4 * (size_t)nt + k] = s.tet;
          N_[4 * (size_t)s.tet + s.face] = nt;
          s.key = ~0ULL;  // consumed; keeps probing chains intact
          break;
        }
        h = (h + 1) & mask;
      }
    }
    for (int q = 0; q < 4; ++q)
      if (f.v[q] != INF) vtet_[f.v[q]] = nt;
  }
  for (const BFace& f : bfaces_) {
    for (int q = 0; q < 4; ++q) {
      if (q == f.face) continue;
      int32_t v = f.v[q];
      if (v == INF || vstamp_[v] == (uint32_t)j + 1) continue;
      vstamp_[v] = (uint32_t)j + 1;
      if (record) {
        L_.append(v, j);
        if (added_) added_->push_back({v, j});
      }
    }
  }
  return 0;
}

bool Builder::insert_rank(int32_t j, std::string* err) {
  const float* p = P(j);
  int32_t curr = 0;
  double dc = dist2(p, P(0));
restart:
  for (int32_t bk = L_.head[curr]; bk >= 0; bk = L_.pool[bk].next) {
    const Lists::Block& B = L_.pool[bk];
    for (int q = 0; q < B.cnt; ++q) {
      int32_t s = B.e[q];
      double ds = dist2(p, P(s));
      if (ds < dc) {
        curr = s;
        dc = ds;
        goto restart;
      }
    }
  }
  if (dc == 0.0) {
    twin_[j] = twin_[curr];
    L_.append(curr, j);
    if (added_) added_->push_back({curr, j});
    st_.duplicates++;
    return true;
  }
  int32_t start = vtet_[twin_[curr]];
  int rc = insert(j, start, true);
  if (rc < 0) {
    *err = "point location failed at rank " + std::to_string(j);
    return false;
  }
  if (rc == 1) {
    L_.append(twin_[j], j);
    if (added_) added_->push_back({twin_[j], j});
    st_.duplicates++;
  }
  return true;
}

void Builder::csr(std::vector<int64_t>* rowp, std::vector<int32_t>* succ) const {
  const int32_t n = n_;
  rowp->assign((size_t)n + 1, 0);
  for (int32_t i = 0; i < n; ++i) (*rowp)[i + 1] = (*rowp)[i] + L_.len[i];
  succ->resize((size_t)(*rowp)[n]);
  for (int32_t i = 0; i < n; ++i) {
    int64_t o = (*rowp)[i];
    for (int32_t bk = L_.head[i]; bk >= 0; bk = L_.pool[bk].next)
      for (int q = 0; q < L_.pool[bk].cnt; ++q) (*succ)[o++] = L_.pool[bk].e[q];
  }
}

bool Builder::append(const float* xyz, int32_t n_new,
                     std::vector<std::pair<int32_t, int32_t>>* added, std::string* err) {
  if (!tet_made_) {
    *err = "appending needs a cloud whose first points span 3D (not all coplanar)";
    return false;
  }
  if (n_new < n_) {
    *err = "append cannot remove points";
    return false;
  }
  for (int64_t i = 3 * (int64_t)n_; i < 3 * (int64_t)n_new; ++i) {
    if (!std::isfinite(xyz[i])) {
      *err = "non-finite coordinate at rank " + std::to_string(i / 3);
      return false;
    }
  }
  X_ = xyz;
  const int32_t n_old = n_;
  n_ = n_new;
  L_.grow(n_new);
  vtet_.resize(n_new, -1);
  vstamp_.resize(n_new, 0);
  twin_.resize(n_new);
  for (int32_t i = n_old; i < n_new; ++i) twin_[i] = i;
  added_ = added;
  const size_t added0 = added ? added->size() : 0;
  bool ok = true;
  for (int32_t j = n_old; j < n_new && ok; ++j) ok = insert_rank(j, err);
  added_ = nullptr;
  if (!ok) {
    // the triangulation keeps the points inserted so far, but the lists go
    // back to the ranks before this call; no further appends are taken
    if (added) {
      for (size_t a = added->size(); a > added0; --a) L_.pop((*added)[a - 1].first);
      added->resize(added0);
    }
    n_ = n_old;
    L_.longest = 0;
    for (int32_t i = 0; i < n_old; ++i) L_.longest = std::max<int64_t>(L_.longest, L_.len[i]);
    broken_ = true;
  }
  st_.n = n_;
  st_.entries = L_.total;
  return ok;
}

bool Builder::run(bool keep_tets, SuccessorTable* out, std::string* err) {
  auto t_start = std::chrono::steady_clock::now();
  predicate_counters() = PredicateCounters{};
  const int32_t n = n_;
  for (int64_t i = 0; i < 3 * (int64_t)n; ++i) {
    if (!std::isfinite(X_[i])) {
      *err = "non-finite coordinate at rank " + std::to_string(i / 3);
      return false;
    }
  }
  L_.init(n);
  vtet_.assign(n, -1);
  twin_.resize(n);
  for (int32_t i = 0; i < n; ++i) twin_[i] = i;
  vstamp_.assign(n, 0);
  st_ = BuildStats{};
  st_.n = n;

  int32_t a = -1, b = -1, c = -1;
  for (int32_t i = 1; i < n && a < 0; ++i)
    if (!same_point(P(i), P(0))) a = i;
  for (int32_t i = (a < 0 ? n : a + 1); i < n && b < 0; ++i)
    if (!collinear3(P(0), P(a), P(i))) b = i;
  for (int32_t i = (b < 0 ? n : b + 1); i < n && c < 0; ++i)
    if (orient3d(P(0), P(a), P(b), P(i)) != 0) c = i;

  const int32_t j0 = (c < 0) ? n - 1 : c;
  if (c < 0 && (int64_t)n > kMaxCoplanarComplete) {
    *err = "all points are coplanar; n exceeds the complete-table limit " +
           std::to_string(kMaxCoplanarComplete);
    return false;
  }
  st_.degenerate_prefix = (int64_t)j0 + 1;
  for (int32_t i = 0; i <= j0; ++i)
    for (int32_t k = i + 1; k <= j0; ++k) L_.append(i, k);

  if (c >= 0) {
    int32_t ia = a, ib = b;
    if (orient3d(P(0), P(ia), P(ib), P(c)) < 0) std::swap(ia, ib);
    initial_tet(0, ia, ib, c);
    for (int32_t r = 1; r < j0; ++r) {
      if (r == a || r == b) continue;
      int rc = insert(r, vtet_[0], false);
      if (rc < 0) {
        *err = "point location failed at rank " + std::to_string(r);
        return false;
      }
      if (rc == 1) st_.duplicates++;
    }
    tet_made_ = true;
    for (int32_t j = j0 + 1; j < n; ++j)
      if (!insert_rank(j, err)) return false;
  }

  csr(&out->rowp, &out->succ);
  int64_t finite = 0;
  const int32_t ntets = (int32_t)(V_.size() / 4);
  out->tets.clear();
  for (int32_t t = 0; t < ntets; ++t) {
    if (V_[4 * (size_t)t] == DEAD || is_inf(t)) continue;
    ++finite;
    if (keep_tets)
      out->tets.insert(out->tets.end(), &V_[4 * (size_t)t], &V_[4 * (size_t)t] + 4);
  }
  st_.tets_final = finite;
  st_.entries = out->rowp[n];
  const PredicateCounters& pc = predicate_counters();
  st_.orient_calls = (int64_t)pc.orient_calls;
  st_.orient_exact = (int64_t)pc.orient_exact;
  st_.insphere_calls = (int64_t)pc.insphere_calls;
  st_.insphere_exact = (int64_t)pc.insphere_exact;
  st_.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  out->stats = st_;
  return true;
}

}  // namespace build_detail

bool build_successor_table(const float* xyz, int64_t n, bool keep_tets, SuccessorTable* out,
                           std::string* err) {
  if (n < 0 || n > (int64_t)0x7FFFFFF0) {
    *err = "n out of range";
    return false;
  }
  try {
    build_detail::Builder b(xyz, n);
    return b.run(keep_tets, out, err);
  } catch (const std::bad_alloc&) {
    *err = "out of host memory while building";
    return false;
  }
}

IncrementalTable::IncrementalTable() = default;
IncrementalTable::~IncrementalTable() = default;

bool IncrementalTable::build(const float* xyz, int64_t n, bool keep_tets, SuccessorTable* out,
                             std::string* err) {
  if (n < 0 || n > (int64_t)0x7FFFFFF0) {
    *err = "n out of range";
    return false;
  }
  try {
    b_.reset(new build_detail::Builder(xyz, n));
    if (!b_->run(keep_tets, out, err)) {
      b_.reset();
      return false;
    }
    return true;
  } catch (const std::bad_alloc&) {
    b_.reset();
    *err = "out of host memory while building";
    return false;
  }
}

bool IncrementalTable::append(const float* xyz, int64_t n_new,
                              std::vector<std::pair<int32_t, int32_t>>* added, std::string* err) {
  if (!b_) {
    *err = "no triangulation kept";
    return false;
  }
  if (n_new > (int64_t)0x7FFFFFF0) {
    *err = "n out of range";
    return false;
  }
  try {
    return b_->append(xyz, (int32_t)n_new, added, err);
  } catch (const std::bad_alloc&) {
    *err = "out of host memory while appending";
    return false;
  }
}

void IncrementalTable::csr(std::vector<int64_t>* rowp, std::vector<int32_t>* succ) const {
  if (b_) b_->csr(rowp, succ);
}

int64_t IncrementalTable::size() const { return b_ ? b_->size() : 0; }

int64_t IncrementalTable::entries() const { return b_ ? b_->stats().entries : 0; }

int64_t IncrementalTable::row_len(int32_t i) const { return b_ ? b_->row_len(i) : 0; }

int64_t IncrementalTable::longest_row() const { return b_ ? b_->longest_row() : 0; }

void IncrementalTable::row_tail(int32_t i, int64_t from, std::vector<int32_t>* out) const {
  if (b_) b_->row_tail(i, from, out);
}

bool IncrementalTable::can_append() const { return b_ && b_->has_tetrahedron(); }

BuildStats IncrementalTable::stats() const { return b_ ? b_->stats() : BuildStats{}; }

}  // namespace mknn
