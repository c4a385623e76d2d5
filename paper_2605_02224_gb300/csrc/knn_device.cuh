// Device-side body of one k-NN query: Algorithm 1 (successor-list descent
// collecting transition sites) then Algorithm 2 (expansion over the
// successor lists of the nearest sites found so far), Sec. 4.
//
// One query is served by a group of G lanes (G = 4, 8, 16 or 32) of a
// warp. The group reads G consecutive successor entries at a time
// (coalesced), gathers their float4 coordinates through the read-only
// path, and decides with warp votes.
//
// Candidate list N: capacity K = G * S, sorted by the key (d, rank),
// distributed over the group: lane l, slot s holds position s * G + l. An
// insertion counts the keys below the new one with S votes, shifts the
// tail by one position with S shuffles per field and drops position k.
// Bit 31 of a stored rank marks an entry whose list has been expanded.
//
// Readings of the paper (see the design notes for the full list):
//  * descent: the scan of L_curr moves to the FIRST entry (lowest rank) that
//    is strictly closer than p_curr and restarts at the head of the new
//    list; every site moved to is inserted into N (all transition sites are
//    candidates, Sec. 4.2);
//  * "strictly closer" is decided in float32 with a guard band; inside the
//    band both distances are recomputed in float64 in the oracle's order,
//    so the descent follows the exact prefix minima of Eq. (2);
//  * expansion: the nearest not-yet-expanded entry among the first k-1 of
//    N is expanded until none is left (equal to Alg. 2's loop in exact
//    arithmetic, robust to float32 reordering of near-equal distances);
//  * prefix bound m (Sec. 4.2): rows are ascending, so a scan stops at the
//    first entry >= m.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "hub_index.h"

namespace mknn {

constexpr uint32_t kRankMask = 0x7fffffffu;
constexpr uint32_t kDoneBit = 0x80000000u;
constexpr uint32_t kPadRank = 0xffffffffu;
// |d32 - D| <= 5 * 2^-24 * D for the float32 evaluation below; the guard
// band is three times wider than the sum of two such errors.
constexpr float kGuard = 2e-6f;
// Below this the float32 distance may be subnormal; decide in float64.
constexpr float kTiny = 1e-30f;
// Entries of a list with a tree that the descent reads in rank order before
// it turns to the tree: the first strictly closer entry is often among the
// first few (the low ranks are spread over the whole cloud), and a walk
// that must prove its rank the lowest costs more than a chunk. On the patch
// clouds of the batching mix 0 / 32 / 64 / 128 entries took 104 / 98 / 100
// / 102 ms with the hand-over.
constexpr int kHubScanFirst = 32;

struct CloudDev {
  const float4* __restrict__ pts;
  const int2* __restrict__ rows;     // (first, end) of each successor row
  const int32_t* __restrict__ succ;
  int32_t n;
  // succ with each entry's site inlined: (x, y, z, rank bits), one 16-byte
  // load per entry instead of an index load and a dependent point load
  const float4* __restrict__ ent;
  // box trees over the long lists (NULL hub_of: none); read by the one-warp
  // kernel only. hub_of[i]: the tree of site i's list or -1; hub_desc:
  // (first entry, list length, first node, levels); hub_ent: the list's
  // entries along a Morton curve in chunks of 32; hub_node: two float4 per
  // node, (low corner, smallest rank's bits) and (high corner, largest
  // rank's bits), levels stored from the chunks' boxes up
  const int32_t* __restrict__ hub_of = nullptr;
  const int4* __restrict__ hub_desc = nullptr;
  const float4* __restrict__ hub_ent = nullptr;
  const float4* __restrict__ hub_node = nullptr;
};

// Squared distance in float32, fixed operation order (no reassociation).
__device__ __forceinline__ float sqd32(float qx, float qy, float qz, float4 p) {
  const float dx = __fsub_rn(qx, p.x);
  const float dy = __fsub_rn(qy, p.y);
  const float dz = __fsub_rn(qz, p.z);
  float d = __fmul_rn(dx, dx);
  d = __fmaf_rn(dy, dy, d);
  d = __fmaf_rn(dz, dz, d);
  return d;
}

// Squared distance in float64: ((dx*dx + dy*dy) + dz*dz), no fusion.
__device__ __forceinline__ double sqd64(float qx, float qy, float qz, float px, float py,
                                        float pz) {
  const double dx = __dsub_rn((double)qx, (double)px);
  const double dy = __dsub_rn((double)qy, (double)py);
  const double dz = __dsub_rn((double)qz, (double)pz);
  return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

__device__ __forceinline__ bool key_lt(float da, uint32_t ra, float db, uint32_t rb) {
  return da < db || (da == db && ra < rb);
}

template <int G>
struct Grp {
  uint32_t lane, base, mask;
  __device__ __forceinline__ Grp() {
    const uint32_t l = threadIdx.x & 31u;
    lane = l & (G - 1);
    base = l & ~(uint32_t)(G - 1);
    mask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << base);
  }
  __device__ __forceinline__ uint32_t ballot(bool p) const {
    const uint32_t b = __ballot_sync(mask, p);
    return (G == 32) ? b : ((b >> base) & ((1u << G) - 1u));
  }
  template <class T>
  __device__ __forceinline__ T shfl(T v, int src) const {
    return __shfl_sync(mask, v, src, G);
  }
};

template <int G, int S>
struct TopK {
  float d[S];
  uint32_t r[S];
  int cnt;
  float kd;     // key of position k-1 (a pad while fewer than k entries)
  uint32_t kr;
};

template <int G, int S>
__device__ __forceinline__ void topk_init(TopK<G, S>& T) {
#pragma unroll
  for (int s = 0; s < S; ++s) {
    T.d[s] = __int_as_float(0x7f800000);
    T.r[s] = kPadRank;
  }
  T.cnt = 0;
  T.kd = __int_as_float(0x7f800000);
  T.kr = kRankMask;
}

// Inserts (cd, cr) unless an equal key is present; keeps k entries.
template <int G, int S>
__device__ __forceinline__ void topk_insert(TopK<G, S>& T, const Grp<G>& g, float cd, uint32_t cr,
                                            int k) {
  int less = 0;
  bool eq = false;
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const uint32_t rr = T.r[s] & kRankMask;
    less += __popc(g.ballot(key_lt(T.d[s], rr, cd, cr)));
    eq |= (T.d[s] == cd) & (rr == cr);
  }
  if (g.ballot(eq) || less >= k) return;
  const int pos = less;
  const int src = (int)((g.lane + G - 1) & (G - 1));
  float ud[S];
  uint32_t ur[S];
#pragma unroll
  for (int s = 0; s < S; ++s) {
    ud[s] = g.shfl(T.d[s], src);
    ur[s] = g.shfl(T.r[s], src);
  }
#pragma unroll
  for (int s = S - 1; s >= 0; --s) {
    const int p = s * G + (int)g.lane;
    float pd;
    uint32_t pr;
    if (g.lane == 0) {
      pd = (s > 0) ? ud[s > 0 ? s - 1 : 0] : 0.f;
      pr = (s > 0) ? ur[s > 0 ? s - 1 : 0] : 0u;
    } else {
      pd = ud[s];
      pr = ur[s];
    }
    if (p >= k) {
      T.d[s] = __int_as_float(0x7f800000);
      T.r[s] = kPadRank;
    } else if (p > pos) {
      T.d[s] = pd;
      T.r[s] = pr;
    } else if (p == pos) {
      T.d[s] = cd;
      T.r[s] = cr;
    }
  }
  T.cnt = min(T.cnt + 1, k);
  const int kp = k - 1;
  const int ks = kp / G, kl = kp % G;
  float td = T.d[0];
  uint32_t tr = T.r[0];
#pragma unroll
  for (int s = 1; s < S; ++s)
    if (s == ks) {
      td = T.d[s];
      tr = T.r[s];
    }
  T.kd = g.shfl(td, kl);
  T.kr = g.shfl(tr, kl) & kRankMask;
}

struct QueryCounters {
  int rows, entries, coords, trans;
};

// One query by one group. m in [1, n]. Writes k results to oi / od.
template <int G, int S, bool COUNT>
__device__ __forceinline__ void knn_query(const CloudDev& C, const Grp<G>& g, float qx, float qy,
                                          float qz, int k, int m, int32_t* __restrict__ out_idx,
                                          float* __restrict__ out_d2, int32_t row,
                                          QueryCounters& qc) {
  const float INF = __int_as_float(0x7f800000);
  TopK<G, S> T;
  topk_init(T);

  // ---- Algorithm 1: descent from p_1 (rank 0), collecting transition sites
  // (the current site is held as a rank; its coordinates are reloaded only
  // for a float64 recheck)
  int curr = 0;
  float dcur = sqd32(qx, qy, qz, __ldg(C.pts));
  topk_insert(T, g, dcur, 0u, k);
  if (COUNT) {
    qc.coords = 1;
    qc.trans = 1;
  }
  for (;;) {
    const int2 rr = __ldg(C.rows + curr);
    const int beg = rr.x, end = rr.y;
    if (COUNT) qc.rows++;
    bool moved = false;
    for (int base = beg; base < end; base += G) {
      const int e = base + (int)g.lane;
      const bool valid = e < end;
      float4 ps = make_float4(0.f, 0.f, 0.f, 0.f);
      if (valid) ps = __ldg(C.ent + e);  // site and rank of the entry
      const int s = valid ? __float_as_int(ps.w) : 0x7fffffff;
      const bool inr = valid && s < m;
      const float d = inr ? sqd32(qx, qy, qz, ps) : INF;
      bool sure, maybe;
      if (dcur >= kTiny) {
        sure = inr && d < dcur * (1.f - kGuard);
        maybe = inr && !sure && d <= dcur * (1.f + kGuard);
      } else {
        sure = false;
        maybe = inr && d <= 2.f * kTiny;
      }
      uint32_t closer = g.ballot(sure);
      if (g.ballot(maybe)) {
        bool c64 = false;
        if (maybe) {
          const float4 pc = __ldg(C.pts + curr);
          c64 = sqd64(qx, qy, qz, ps.x, ps.y, ps.z) < sqd64(qx, qy, qz, pc.x, pc.y, pc.z);
        }
        closer |= g.ballot(c64);
      }
      const uint32_t stop = g.ballot(valid && !inr);
      if (closer) {
        const int w = __ffs(closer) - 1;
        if (COUNT) {
          qc.entries += w + 1;
          qc.coords += w + 1;
          qc.trans++;
        }
        curr = g.shfl(s, w);
        dcur = g.shfl(d, w);
        topk_insert(T, g, dcur, (uint32_t)curr, k);
        moved = true;
        break;
      }
      if (COUNT) {
        if (stop) {
          const int t = __ffs(stop) - 1;
          qc.entries += t + 1;
          qc.coords += t;
        } else {
          const int nv = min(G, end - base);
          qc.entries += nv;
          qc.coords += nv;
        }
      }
      if (stop) break;
    }
    if (!moved) break;
  }

  // ---- Algorithm 2: expand the nearest unexpanded entry among the first k-1
  for (;;) {
    const int lim = min(T.cnt, k - 1);
    int pos = -1;
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const int p = s * G + (int)g.lane;
      const uint32_t b = g.ballot(p < lim && !(T.r[s] & kDoneBit));
      if (b && pos < 0) pos = s * G + __ffs(b) - 1;
    }
    if (pos < 0) break;
    const int psl = pos / G, pln = pos % G;
    uint32_t rsel = T.r[0];
#pragma unroll
    for (int s = 1; s < S; ++s)
      if (s == psl) rsel = T.r[s];
    const int site = (int)(g.shfl(rsel, pln) & kRankMask);
    if ((int)g.lane == pln) {
#pragma unroll
      for (int s = 0; s < S; ++s)
        if (s == psl) T.r[s] |= kDoneBit;
    }
    const int2 rr = __ldg(C.rows + site);
    const int beg = rr.x, end = rr.y;
    if (COUNT) qc.rows++;
    for (int base = beg; base < end; base += G) {
      const int e = base + (int)g.lane;
      const bool valid = e < end;
      float4 ps = make_float4(0.f, 0.f, 0.f, 0.f);
      if (valid) ps = __ldg(C.ent + e);
      const int s = valid ? __float_as_int(ps.w) : 0x7fffffff;
      const bool inr = valid && s < m;
      const float d = inr ? sqd32(qx, qy, qz, ps) : INF;
      bool pass = inr && key_lt(d, (uint32_t)s, T.kd, T.kr);
      uint32_t b = g.ballot(pass);
      while (b) {
        const int w = __ffs(b) - 1;
        const float cd = g.shfl(d, w);
        const uint32_t cr = g.shfl((uint32_t)s, w);
        topk_insert(T, g, cd, cr, k);
        pass = pass && ((int)g.lane > w) && key_lt(d, (uint32_t)s, T.kd, T.kr);
        b = g.ballot(pass);
      }
      const uint32_t stop = g.ballot(valid && !inr);
      if (COUNT) {
        if (stop) {
          const int t = __ffs(stop) - 1;
          qc.entries += t + 1;
          qc.coords += t;
        } else {
          const int nv = min(G, end - base);
          qc.entries += nv;
          qc.coords += nv;
        }
      }
      if (stop) break;
    }
  }

  // ---- output: sorted (d, rank), padded with (-1, +inf)
  int32_t* oi = out_idx + (int64_t)row * k;
  float* od = out_d2 + (int64_t)row * k;
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int p = s * G + (int)g.lane;
    if (p < k) {
      const uint32_t rr = T.r[s] & kRankMask;
      const bool real = rr != kRankMask;
      __stcs(oi + p, real ? (int32_t)rr : -1);
      __stcs(od + p, real ? T.d[s] : INF);
    }
  }
}

// ---------------------------------------------------------------------------
// One query per thread. The candidate list N is an unsorted array of K
// register slots holding the best min(k, seen) keys, with the worst of them
// tracked as the admission threshold once the list is full. The order the
// algorithm needs is recovered on demand: the nearest not-yet-expanded
// entry among "the first k-1" is the smallest unexpanded key other than the
// worst one (when the list is full). No lane talks to another, so a warp
// serves 32 queries with no votes or shuffles; with locality-sorted
// queries the 32 descents share most of their path.
template <int K>
struct TopT {
  float d[K];
  uint32_t r[K];  // rank, bit 31 = expanded
  int cnt;
  int worst;      // slot of the worst key, valid when cnt == k
  float wd;       // worst key (threshold); (+inf, kRankMask) while cnt < k
  uint32_t wr;
};

template <int K>
__device__ __forceinline__ void topt_init(TopT<K>& T) {
#pragma unroll
  for (int i = 0; i < K; ++i) {
    T.d[i] = __int_as_float(0x7f800000);
    T.r[i] = kPadRank;
  }
  T.cnt = 0;
  T.worst = 0;
  T.wd = __int_as_float(0x7f800000);
  T.wr = kRankMask;
}

// Inserts (cd, cr) unless present. Caller checks key_lt(cd, cr, wd, wr).
template <int K>
__device__ __forceinline__ void topt_insert(TopT<K>& T, float cd, uint32_t cr, int k) {
  bool dup = false;
#pragma unroll
  for (int i = 0; i < K; ++i) dup |= (T.d[i] == cd) & ((T.r[i] & kRankMask) == cr);
  if (dup) return;
  int slot;
  if (T.cnt < k) {
    slot = T.cnt++;
  } else {
    slot = T.worst;
  }
#pragma unroll
  for (int i = 0; i < K; ++i)
    if (i == slot) {
      T.d[i] = cd;
      T.r[i] = cr;
    }
  if (T.cnt == k) {
    float wd = -1.f;
    uint32_t wr = 0;
    int w = 0;
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const uint32_t ri = T.r[i] & kRankMask;
      if (i < k && key_lt(wd, wr, T.d[i], ri)) {
        wd = T.d[i];
        wr = ri;
        w = i;
      }
    }
    T.worst = w;
    T.wd = wd;
    T.wr = wr;
  }
}

template <int K, bool COUNT>
__device__ __forceinline__ void knn_query_thread(const CloudDev& C, float qx, float qy, float qz,
                                                 int k, int m, int32_t* __restrict__ oi,
                                                 float* __restrict__ od, QueryCounters& qc) {
  const float INF = __int_as_float(0x7f800000);
  TopT<K> T;
  topt_init(T);

  // ---- Algorithm 1
  int curr = 0;
  float4 pc = __ldg(C.pts);
  float dcur = sqd32(qx, qy, qz, pc);
  topt_insert(T, dcur, 0u, k);
  if (COUNT) {
    qc.coords = 1;
    qc.trans = 1;
  }
  for (;;) {
    const int2 rr = __ldg(C.rows + curr);
    int e = rr.x;
    const int end = rr.y;
    if (COUNT) qc.rows++;
    bool moved = false;
    for (; e < end; ++e) {
      const int s = __ldg(C.succ + e);
      if (COUNT) qc.entries++;
      if (s >= m) break;
      const float4 ps = __ldg(C.pts + s);
      const float d = sqd32(qx, qy, qz, ps);
      if (COUNT) qc.coords++;
      bool closer;
      if (dcur >= kTiny && d < dcur * (1.f - kGuard)) {
        closer = true;
      } else if ((dcur >= kTiny && d > dcur * (1.f + kGuard)) || (dcur < kTiny && d > 2.f * kTiny)) {
        closer = false;
      } else {
        closer = sqd64(qx, qy, qz, ps.x, ps.y, ps.z) < sqd64(qx, qy, qz, pc.x, pc.y, pc.z);
      }
      if (closer) {
        curr = s;
        dcur = d;
        pc = ps;
        if (key_lt(d, (uint32_t)s, T.wd, T.wr)) topt_insert(T, d, (uint32_t)s, k);
        if (COUNT) qc.trans++;
        moved = true;
        break;
      }
    }
    if (!moved) break;
  }

  // ---- Algorithm 2
  for (;;) {
    float bd = INF;
    uint32_t br = kRankMask;
    int bi = -1;
    const bool full = T.cnt == k;
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const uint32_t ri = T.r[i] & kRankMask;
      const bool ok = (i < T.cnt) && !(T.r[i] & kDoneBit) && !(full && i == T.worst);
      if (ok && key_lt(T.d[i], ri, bd, br)) {
        bd = T.d[i];
        br = ri;
        bi = i;
      }
    }
    if (bi < 0) break;
#pragma unroll
    for (int i = 0; i < K; ++i)
      if (i == bi) T.r[i] |= kDoneBit;
    const int site = (int)br;
    const int2 rr = __ldg(C.rows + site);
    int e = rr.x;
    const int end = rr.y;
    if (COUNT) qc.rows++;
    for (; e < end; ++e) {
      const int s = __ldg(C.succ + e);
      if (COUNT) qc.entries++;
      if (s >= m) break;
      const float d = sqd32(qx, qy, qz, __ldg(C.pts + s));
      if (COUNT) qc.coords++;
      if (key_lt(d, (uint32_t)s, T.wd, T.wr)) topt_insert(T, d, (uint32_t)s, k);
    }
  }

  // ---- output: position of each entry = number of smaller keys
#pragma unroll
  for (int i = 0; i < K; ++i) {
    if (i < T.cnt) {
      const uint32_t ri = T.r[i] & kRankMask;
      int pos = 0;
#pragma unroll
      for (int j = 0; j < K; ++j) pos += key_lt(T.d[j], T.r[j] & kRankMask, T.d[i], ri) ? 1 : 0;
      oi[pos] = (int32_t)ri;
      od[pos] = T.d[i];
    }
  }
  for (int p = T.cnt; p < k; ++p) {
    oi[p] = -1;
    od[p] = INF;
  }
}

// ---------------------------------------------------------------------------
// One query per thread with the candidate list N in shared memory: entry i
// of the lane's list at col[i * 32] (a warp's lists interleaved, so any mix
// of positions across the lanes is bank-conflict free). An entry is one
// 64-bit key, the float bits of the squared distance above the rank:
// distances are never negative, so the integer order of the keys is the
// (distance, rank) order and a comparison, a load or a move is one
// instruction. Slots not yet filled hold a pad key above every real one,
// so the search for an insertion position is a fixed sequence of halving
// steps with no bound to track. The search also finds an equal key, so the
// membership test of Alg. 2 costs nothing extra. The nearest not-yet-
// expanded entry among the first k-1 is one bit scan of the expanded mask;
// the output comes out in order. The list takes no registers, which leaves
// room for more resident warps.
//
// The lanes of a warp run in step, so the warp pays for the insertion code
// whenever any of its lanes inserts (about one entry in five offers a
// candidate below the k-th key, half of them already in N): insertion is
// kept to a short sequence with no data-dependent loop where that pays.
//  * SortedList: keys kept in position order; an insertion shifts the tail
//    by one slot (a loop as long as the longest shift among the lanes
//    inserting). Used where lists are short (k <= 8) or long (k > 16).
//  * PermList16 (9 <= k <= 16): keys stay in the slot they were written to;
//    a 64-bit register holds the slot of each position, four bits each. An
//    insertion writes the new key into the slot of position k-1 (the
//    dropped key, or a pad) and moves that slot's four bits to the
//    insertion position: no key moves, a fixed instruction sequence
//    (measured 1.10x the sorted list at k = 16, 0.97x at k = 8).
__device__ __forceinline__ uint64_t pack_key(float d, uint32_t r) {
  return ((uint64_t)__float_as_uint(d) << 32) | r;
}

// above every real key (real keys have the sign bit of the distance clear)
constexpr uint64_t kPadKey = ~0ull;

// Expanded flags, one bit per list position, in W 32-bit words: W = 1 for
// k <= 32 (one 32-bit register), 2 for k <= 64 (one 64-bit), 4 for k <= 128
// (two 64-bit).
template <int W>
struct Flags {
  uint64_t lo = 0, hi = 0;
};
template <>
struct Flags<1> {
  uint32_t lo = 0;
};

// Opens a clear flag at bit pos of one word: bits at pos and above move up.
template <typename T>
__device__ __forceinline__ T flags_open(T f, int pos) {
  const T low = pos ? (f & (~T(0) >> (8 * sizeof(T) - pos))) : T(0);
  return low | ((f >> pos) << 1 << pos);
}

// Opens a clear flag at list position pos (an insertion there).
template <int W>
__device__ __forceinline__ void flags_insert(Flags<W>& F, int pos) {
  if constexpr (W == 4) {
    if (pos < 64) {
      F.hi = (F.hi << 1) | (F.lo >> 63);
      F.lo = flags_open(F.lo, pos);
    } else {
      F.hi = flags_open(F.hi, pos - 64);
    }
  } else {
    F.lo = flags_open(F.lo, pos);
  }
}

// Position of the first entry among the first lim not yet expanded, or -1.
template <int W>
__device__ __forceinline__ int flags_first_clear(const Flags<W>& F, int lim) {
  if constexpr (W == 1) {
    const uint32_t c = ~F.lo & ((1u << lim) - 1u);  // lim <= 31
    return c ? __ffs((int)c) - 1 : -1;
  } else {
    const int l0 = min(lim, 64);
    const uint64_t c0 = ~F.lo & (l0 == 64 ? ~0ull : ((1ull << l0) - 1ull));
    if (c0) return __ffsll((long long)c0) - 1;
    if constexpr (W == 4) {
      if (lim > 64) {
        const uint64_t c1 = ~F.hi & ((1ull << (lim - 64)) - 1ull);
        if (c1) return 64 + __ffsll((long long)c1) - 1;
      }
    }
    return -1;
  }
}

template <int W>
__device__ __forceinline__ void flags_set(Flags<W>& F, int pos) {
  if constexpr (W == 1) {
    F.lo |= 1u << pos;
  } else if constexpr (W == 2) {
    F.lo |= 1ull << pos;
  } else {
    if (pos < 64)
      F.lo |= 1ull << pos;
    else
      F.hi |= 1ull << (pos - 64);
  }
}

// Keys in position order. KS: the search size (a power of two >= the
// list's capacity cap); positions in [cap, KS) read as pads without a load
// unless EXACT (cap == KS).
template <int KS, int W, bool EXACT>
struct SortedList {
  uint64_t* col;
  int cap;
  int cnt;
  Flags<W> done;   // bit i: entry at position i expanded
  uint64_t worst;  // key of position k-1 (a pad while cnt < k)

  __device__ __forceinline__ void init(uint64_t* c, int capacity) {
    col = c;
    cap = EXACT ? KS : capacity;
    cnt = 0;
    done = Flags<W>{};
    worst = kPadKey;
    for (int i = 0; i < cap; ++i) col[i * 32] = kPadKey;
  }
  __device__ __forceinline__ uint64_t key_at(int pos) const { return col[pos * 32]; }
  __device__ __forceinline__ uint64_t probe(int pos) const {
    return (EXACT || pos < cap) ? col[pos * 32] : kPadKey;
  }
  // Inserts key c unless present; requires c < worst (then the position
  // found is below k <= cap).
  __device__ __forceinline__ void insert(uint64_t c, int k) {
    int pos = 0;
#pragma unroll
    for (int step = KS / 2; step >= 1; step >>= 1)
      if (probe(pos + step - 1) < c) pos += step;
    if (pos >= k || col[pos * 32] == c) return;
    for (int i = min(cnt, k - 1); i > pos; --i) col[i * 32] = col[(i - 1) * 32];
    col[pos * 32] = c;
    flags_insert(done, pos);
    if (cnt < k) cnt++;
    if (cnt == k) worst = col[(k - 1) * 32];
  }
};

// 9 <= k <= 16: sixteen slots, the order held in a register (see above).
struct PermList16 {
  uint64_t* col;
  uint64_t perm;   // bits 4j..4j+3: the slot of position j
  int cnt;
  Flags<1> done;   // by position
  uint64_t worst;  // key of position k-1 (a pad while cnt < k)

  __device__ __forceinline__ void init(uint64_t* c, int) {
    col = c;
    perm = 0xFEDCBA9876543210ull;
    cnt = 0;
    done = Flags<1>{};
    worst = kPadKey;
#pragma unroll
    for (int i = 0; i < 16; ++i) col[i * 32] = kPadKey;
  }
  __device__ __forceinline__ int slot(int pos) const { return (int)((perm >> (4 * pos)) & 15ull); }
  __device__ __forceinline__ uint64_t key_at(int pos) const { return col[slot(pos) * 32]; }
  // Inserts key c unless present; requires c < worst and 9 <= k <= 16.
  __device__ __forceinline__ void insert(uint64_t c, int k) {
    int pos = 0;
#pragma unroll
    for (int step = 8; step >= 1; step >>= 1)
      if (col[slot(pos + step - 1) * 32] < c) pos += step;
    // pos <= k - 1 because c < worst; slot() is below 16 whatever pos is, so
    // no access leaves the thread's sixteen slots
    if (col[slot(pos) * 32] == c) return;
    const int w = slot(k - 1);  // the dropped key's slot (or a pad's)
    col[w * 32] = c;
    // positions pos..k-2 move up by one, w goes to pos, k..15 stay
    const uint64_t below = pos ? (~0ull >> (64 - 4 * pos)) : 0ull;
    const uint64_t live = (k == 16) ? ~0ull : (~0ull >> (64 - 4 * k));
    const uint64_t mid = perm & live & ~below & ~(15ull << (4 * (k - 1)));
    perm = (perm & below) | ((uint64_t)w << (4 * pos)) | (mid << 4) | (perm & ~live);
    flags_insert(done, pos);
    if (cnt < k) cnt++;
    if (cnt == k) worst = (pos == k - 1) ? c : col[slot(k - 1) * 32];
  }
};

// Descent decision: is the candidate at squared distance d (site ps)
// strictly closer than the current site (dcur, pc)? float32 outside the
// guard band, float64 in the oracle's order inside it.
__device__ __forceinline__ bool strictly_closer(float qx, float qy, float qz, float d, float4 ps,
                                                float dcur, float4 pc) {
  if (dcur >= kTiny) {
    if (d < dcur * (1.f - kGuard)) return true;
    if (d > dcur * (1.f + kGuard)) return false;
  } else if (d > 2.f * kTiny) {
    return false;
  }
  return sqd64(qx, qy, qz, ps.x, ps.y, ps.z) < sqd64(qx, qy, qz, pc.x, pc.y, pc.z);
}

// strictly_closer with the current site given by its rank: its coordinates
// are loaded only when the float32 decision is inside the guard band.
__device__ __forceinline__ bool strictly_closer_at(const CloudDev& C, float qx, float qy, float qz,
                                                   float d, float4 ps, float dcur, int cur) {
  if (dcur >= kTiny) {
    if (d < dcur * (1.f - kGuard)) return true;
    if (d > dcur * (1.f + kGuard)) return false;
  } else if (d > 2.f * kTiny) {
    return false;
  }
  const float4 pc = __ldg(C.pts + cur);
  return sqd64(qx, qy, qz, ps.x, ps.y, ps.z) < sqd64(qx, qy, qz, pc.x, pc.y, pc.z);
}

// Algorithms 1 and 2 for one query as one flat loop: each iteration either
// consumes one successor entry (a descent step while descending, an offer
// to N while expanding) or moves to the next row (a descent move, the end
// of the descent, or the nearest list not yet expanded). The threads of a
// warp then advance entry by entry together whatever their row lengths,
// instead of waiting at the end of every row for the longest one (measured
// 1.3x-2x faster than the row-by-row loop nest). Entries come from the
// inlined table (site and rank in one 16-byte load), the next one loaded
// one iteration ahead. L is a SortedList or PermList16 over the thread's
// column col, with `cap` slots.
//
// DEFER (a cloud with box trees over its long lists, hub_of not NULL): the
// query gives up, returning false with nothing written, when it would read
// a list with a tree through - the expansion of such a list, or a descent
// that finds no strictly closer entry among its first kHubScanFirst - so
// that the one-warp kernel, which walks the tree instead, answers it; the
// queries that never meet such a list (most of them) stay on one lane.
template <class L, bool DEFER = false>
__device__ __forceinline__ bool knn_query_smem(const CloudDev& C, float qx, float qy, float qz,
                                               int k, int m, uint64_t* col, int cap,
                                               int32_t* __restrict__ out_idx,
                                               float* __restrict__ out_d2, int32_t row) {
  // an entry past the end of a row: rank bits 0x7fffffff, never < m
  const float4 kNone = make_float4(0.f, 0.f, 0.f, __int_as_float(0x7fffffff));
  L N;
  N.init(col, cap);
  float dcur = sqd32(qx, qy, qz, __ldg(C.pts));
  N.insert(pack_key(dcur, 0u), k);
  // rank of the descent's current site, -1 once the descent is over (its
  // coordinates are reloaded only for a float64 recheck, which is rare)
  int cur = 0;
  int2 rr = __ldg(C.rows);
  // DEFER: the current list has a tree and its scan stops after
  // kHubScanFirst entries
  bool cut = false;
  if constexpr (DEFER) {
    if (__ldg(C.hub_of) >= 0) {
      cut = rr.y > rr.x + kHubScanFirst;
      rr.y = min(rr.y, rr.x + kHubScanFirst);
    }
  }
  int e = rr.x, end = rr.y;
  float4 next = e < end ? __ldg(C.ent + e) : kNone;
  for (;;) {
    const int s = __float_as_int(next.w);
    if (s < m) {  // the row's next entry exists and is in the prefix
      const float4 ps = next;
      ++e;
      next = e < end ? __ldg(C.ent + e) : kNone;
      const float d = sqd32(qx, qy, qz, ps);
      const uint64_t key = pack_key(d, (uint32_t)s);
      if (cur >= 0) {
        if (strictly_closer_at(C, qx, qy, qz, d, ps, dcur, cur)) {
          dcur = d;
          cur = s;
          if (key < N.worst) N.insert(key, k);
          rr = __ldg(C.rows + s);
          if constexpr (DEFER) {
            cut = false;
            if (__ldg(C.hub_of + s) >= 0) {
              cut = rr.y > rr.x + kHubScanFirst;
              rr.y = min(rr.y, rr.x + kHubScanFirst);
            }
          }
          e = rr.x;
          end = rr.y;
          next = e < end ? __ldg(C.ent + e) : kNone;
        }
      } else if (key < N.worst) {
        N.insert(key, k);
      }
      continue;
    }
    // the current row is done: no closer site in it (descent), or fully offered
    if constexpr (DEFER) {
      if (cut && e >= end) return false;  // the descent's scan was cut short
    }
    cur = -1;
    const int pos = flags_first_clear(N.done, min(N.cnt, k - 1));
    if (pos < 0) break;
    flags_set(N.done, pos);
    const int site = (int)(uint32_t)N.key_at(pos);
    if constexpr (DEFER) {
      if (__ldg(C.hub_of + site) >= 0) return false;  // an expansion of a list with a tree
    }
    rr = __ldg(C.rows + site);
    e = rr.x;
    end = rr.y;
    next = e < end ? __ldg(C.ent + e) : kNone;
  }
  // the output row is addressed only now, from its 32-bit index (fewer
  // registers held through the loop); streaming stores, so that the rows
  // written do not push successor entries out of L2; four values per
  // 16-byte store when k is a multiple of 4 and both arrays are 16-byte
  // aligned (then every row is), else one value per store
  int32_t* oi = out_idx + (int64_t)row * k;
  float* od = out_d2 + (int64_t)row * k;
  const bool vec = ((k & 3) == 0) &&
                   ((((uintptr_t)out_idx) | ((uintptr_t)out_d2)) & 15) == 0;
  if (vec) {
    for (int p = 0; p < k; p += 4) {
      int iv[4];
      float dv[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const bool real = p + t < N.cnt;
        const uint64_t key = real ? N.key_at(p + t) : 0ull;
        iv[t] = real ? (int32_t)(uint32_t)key : -1;
        dv[t] = real ? __uint_as_float((uint32_t)(key >> 32)) : __int_as_float(0x7f800000);
      }
      __stcs(reinterpret_cast<int4*>(oi + p), make_int4(iv[0], iv[1], iv[2], iv[3]));
      __stcs(reinterpret_cast<float4*>(od + p), make_float4(dv[0], dv[1], dv[2], dv[3]));
    }
  } else {
    for (int p = 0; p < k; ++p) {
      const bool real = p < N.cnt;
      const uint64_t key = real ? N.key_at(p) : 0ull;
      __stcs(oi + p, real ? (int32_t)(uint32_t)key : -1);
      __stcs(od + p, real ? __uint_as_float((uint32_t)(key >> 32)) : __int_as_float(0x7f800000));
    }
  }
  return true;
}

// Slots of a thread's list column for k: 8 for k <= 8, 16 for k <= 16 (the
// lists search a power-of-two size), k above.
__host__ __device__ __forceinline__ int list_slots(int k) { return k <= 8 ? 8 : (k <= 16 ? 16 : k); }

// ---------------------------------------------------------------------------
// One warp per query with the candidate list N in shared memory (for large
// k, where one list per thread would leave a few warps per SM). The list is
// the warp's KC keys (KC = 32, 64 or 128 >= k), ascending, pads past cnt;
// lane l owns positions l + 32 j. A row is read 32 entries at a time
// (one coalesced 512-byte load of inlined entries); in the descent the
// first strictly closer entry in list order is the lowest lane that votes
// closer. In the expansion each lane whose entry falls below the k-th key
// searches the list for it (a binary search in shared memory, all such
// lanes at once): most of them are already in N (at k = 100, 781 of 948
// per query on the 1M torus), and only the new ones are inserted, one at a
// time by the whole warp: every lane compares its J keys, the votes give
// the position, and the tail moves up by one slot. Expanded flags are kept
// by position, the same in every lane.
template <int KC>
struct WarpList {
  static constexpr int J = KC / 32;
  uint64_t* L;          // the warp's KC keys in shared memory
  int cnt;
  uint32_t done[J];     // bit b of word j: position 32 j + b expanded
  uint64_t worst;       // key of position k-1 (a pad while cnt < k)

  __device__ __forceinline__ void init(uint64_t* list, int lane) {
    L = list;
    cnt = 0;
#pragma unroll
    for (int j = 0; j < J; ++j) {
      done[j] = 0;
      L[lane + 32 * j] = kPadKey;
    }
    worst = kPadKey;
    __syncwarp();
  }
  // bits at position pos and above move up by one (an insertion at pos)
  __device__ __forceinline__ void open_flag(int pos) {
    const int wi = pos >> 5, bi = pos & 31;
#pragma unroll
    for (int j = J - 1; j >= 0; --j) {
      if (j > wi) {
        done[j] = (done[j] << 1) | (j > 0 ? (done[j > 0 ? j - 1 : 0] >> 31) : 0u);
      } else if (j == wi) {
        const uint32_t f = done[j];
        const uint32_t low = bi ? (f & (~0u >> (32 - bi))) : 0u;
        done[j] = low | ((f >> bi) << 1 << bi);
      }
    }
  }
  __device__ __forceinline__ void set_flag(int pos) {
#pragma unroll
    for (int j = 0; j < J; ++j)
      if (j == (pos >> 5)) done[j] |= 1u << (pos & 31);
  }
  // first position below lim not yet expanded, or -1
  __device__ __forceinline__ int first_clear(int lim) const {
    int r = -1;
#pragma unroll
    for (int j = J - 1; j >= 0; --j) {
      const int nb = max(0, min(32, lim - 32 * j));
      const uint32_t c = ~done[j] & (nb == 32 ? ~0u : ((1u << nb) - 1u));
      if (c) r = 32 * j + __ffs((int)c) - 1;
    }
    return r;
  }
  // is key c in the list? pos: the number of keys below c (called by any
  // subset of lanes)
  __device__ __forceinline__ bool contains(uint64_t c, int& pos) const {
    pos = 0;
#pragma unroll
    for (int step = KC / 2; step >= 1; step >>= 1)
      if (L[pos + step - 1] < c) pos += step;
    return L[pos] == c;
  }
  // Inserts key c, not in the list and below the k-th key, at position pos
  // (the number of keys below it; the same in every lane; called by the
  // whole warp).
  __device__ __forceinline__ void insert_at(uint64_t c, int pos, int k, int lane) {
    uint64_t prev[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const int p = lane + 32 * j;
      prev[j] = (p > pos && p < k) ? L[p - 1] : 0ull;
    }
    __syncwarp();  // every lane has read its previous keys
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const int p = lane + 32 * j;
      if (p < k) {
        if (p > pos)
          L[p] = prev[j];
        else if (p == pos)
          L[p] = c;
      }
    }
    __syncwarp();
    open_flag(pos);
    if (cnt < k) cnt++;
    if (cnt == k) worst = L[k - 1];
  }
  // Offers the lanes' keys with `fresh` set (below the k-th key, not in the
  // list; positions from contains) one after another, lowest lane first:
  // each one still below the k-th key goes in at its position, and the
  // positions of the keys after it that are larger move up by one.
  __device__ __forceinline__ void offer(bool fresh, uint64_t key, int pos, int k, int lane) {
    uint32_t b = __ballot_sync(0xffffffffu, fresh);
    while (b) {
      const int j = __ffs((int)b) - 1;
      b &= b - 1;
      const uint64_t c = __shfl_sync(0xffffffffu, key, j);
      const int at = __shfl_sync(0xffffffffu, pos, j);
      if (c < worst) {
        insert_at(c, at, k, lane);
        if (key > c) ++pos;
      }
    }
  }
  // Inserts key c (the same in every lane; called by the whole warp) unless
  // present; keeps k entries.
  __device__ __forceinline__ void insert(uint64_t c, int k, int lane) {
    uint64_t old[J], prev[J];
    int less = 0;
    bool eq = false;
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const int p = lane + 32 * j;
      old[j] = L[p];
      prev[j] = p ? L[p - 1] : 0ull;
      less += __popc(__ballot_sync(0xffffffffu, old[j] < c));
      eq |= old[j] == c;
    }
    if (__any_sync(0xffffffffu, eq) || less >= k) return;
    const int pos = less;
    __syncwarp();  // every lane has read its old and previous keys
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const int p = lane + 32 * j;
      if (p < k) {
        if (p > pos)
          L[p] = prev[j];
        else if (p == pos)
          L[p] = c;
      }
    }
    __syncwarp();
    open_flag(pos);
    if (cnt < k) cnt++;
    if (cnt == k) worst = L[k - 1];
  }
};

// Box trees over long lists (one warp; every lane passes the same arguments).

// Node count of one level of a tree over len entries, and the level's
// offset from the tree's first node (the chunks' level first).
__device__ __forceinline__ void hub_level_of(int len, int level, int& off, int& cnt) {
  int c = (len + 31) >> 5, o = 0;
  for (int l = 0; l < level; ++l) {
    o += c;
    c = (c + 31) >> 5;
  }
  off = o;
  cnt = c;
}

// Squared distance from q to the box [lo, hi] with sqd32's operations,
// applied to per-axis gaps that are never larger in magnitude than the gap
// to any point of the box. Subtraction, product and fused add are monotonic
// under round-to-nearest, so the result is at most sqd32(q, p) for every
// site p in the box: no rounding can make a box look farther than a site
// inside it.
__device__ __forceinline__ float box_sqd32(float qx, float qy, float qz, float4 lo, float4 hi) {
  const float dx = qx < lo.x ? __fsub_rn(qx, lo.x) : (qx > hi.x ? __fsub_rn(qx, hi.x) : 0.f);
  const float dy = qy < lo.y ? __fsub_rn(qy, lo.y) : (qy > hi.y ? __fsub_rn(qy, hi.y) : 0.f);
  const float dz = qz < lo.z ? __fsub_rn(qz, lo.z) : (qz > hi.z ? __fsub_rn(qz, hi.z) : 0.f);
  float d = __fmul_rn(dx, dx);
  d = __fmaf_rn(dy, dy, d);
  d = __fmaf_rn(dz, dz, d);
  return d;
}

// Depth-first walk of tree D. The children of a node are rated one per lane
// with rate(low, high): a priority below 0xffffffff for a child that may
// hold an entry of interest (the smaller, the sooner it is entered), else
// 0xffffffff. The kept children of each level wait in a bit mask, their
// priorities in the warp's shared memory; the one with the smallest
// priority is entered next if still(priority) holds then (the bounds
// tighten as chunks are handled), and a kept chunk (level 0) goes to
// leaf(chunk). Every decision is the same in all lanes, so the warp stays
// converged. stack: kHubStackWords 32-bit words of the warp's shared memory.
template <class Rate, class Still, class Leaf>
__device__ __forceinline__ void hub_walk(const CloudDev& C, int4 D, int lane, uint32_t* stack,
                                         Rate&& rate, Still&& still, Leaf&& leaf) {
  const int len = D.y, node0 = D.z, top = D.w - 1;
  // per level: the children not entered yet (pend), the index of their
  // first (first), and each child's priority (prio, one per lane)
  uint32_t* pend = stack;
  uint32_t* first = stack + kHubMaxLevels;
  uint32_t* prio = stack + 2 * kHubMaxLevels;
  int l = top, off, cnt;
  hub_level_of(len, l, off, cnt);
  uint32_t pr = 0xffffffffu;
  if (lane < cnt) {
    const int j = node0 + off + lane;
    pr = rate(__ldg(C.hub_node + 2 * j), __ldg(C.hub_node + 2 * j + 1));
  }
  prio[32 * l + lane] = pr;
  pend[l] = __ballot_sync(0xffffffffu, pr != 0xffffffffu);
  first[l] = 0;
  __syncwarp();
  for (;;) {
    const uint32_t pm = pend[l];
    if (pm == 0u) {
      if (++l > top) break;
      continue;
    }
    const uint32_t mine = ((pm >> lane) & 1u) ? prio[32 * l + lane] : 0xffffffffu;
    const uint32_t low = __reduce_min_sync(0xffffffffu, mine);
    const int c = __ffs((int)__ballot_sync(0xffffffffu, mine == low)) - 1;
    pend[l] = pm & ~(1u << c);
    const int node = (int)first[l] + c;
    if (!still(low)) continue;
    if (l == 0) {
      leaf(node);
      continue;
    }
    --l;
    hub_level_of(len, l, off, cnt);
    const int ch = 32 * node + lane;
    pr = 0xffffffffu;
    if (ch < cnt) {
      const int jc = node0 + off + ch;
      pr = rate(__ldg(C.hub_node + 2 * jc), __ldg(C.hub_node + 2 * jc + 1));
    }
    __syncwarp();  // every lane has read this level's old priorities
    prio[32 * l + lane] = pr;
    pend[l] = __ballot_sync(0xffffffffu, pr != 0xffffffffu);
    first[l] = (uint32_t)(32 * node);
    __syncwarp();
  }
}

// Algorithm 1's step on a list with a tree: the lowest rank below m whose
// site is strictly closer than the current one (rank cur, squared distance
// dcur) - the first such entry of the list in rank order - or -1; its
// squared distance goes to bd. A box is skipped when its nearest point is
// beyond the float32 distance above which strictly_closer says no, or its
// smallest rank is not below m or below the best found.
__device__ __forceinline__ int hub_first_closer(const CloudDev& C, int hub, float qx, float qy,
                                                float qz, float dcur, int cur, int m, int lane,
                                                uint32_t* stack, float& bd) {
  const int4 D = __ldg(C.hub_desc + hub);
  const float reach = dcur >= kTiny ? dcur * (1.f + kGuard) : 2.f * kTiny;
  int best = 0x7fffffff;
  float bestd = 0.f;
  hub_walk(
      C, D, lane, stack,
      [&](float4 lo, float4 hi) {
        const int r = __float_as_int(lo.w);
        return (r < m && r < best && !(box_sqd32(qx, qy, qz, lo, hi) > reach)) ? (uint32_t)r
                                                                               : 0xffffffffu;
      },
      [&](uint32_t r) { return (int)r < best; },
      [&](int chunk) {
        const float4 ps = __ldg(C.hub_ent + D.x + 32 * chunk + lane);
        const int s = __float_as_int(ps.w);  // pads: 0x7fffffff, never below m
        const float d = sqd32(qx, qy, qz, ps);
        const bool cl = s < m && s < best && strictly_closer_at(C, qx, qy, qz, d, ps, dcur, cur);
        const int low = __reduce_min_sync(0xffffffffu, cl ? s : 0x7fffffff);
        if (low < best) {
          const int w = __ffs((int)__ballot_sync(0xffffffffu, cl && s == low)) - 1;
          best = low;
          bestd = __shfl_sync(0xffffffffu, d, w);
        }
      });
  bd = bestd;
  return best == 0x7fffffff ? -1 : best;
}

// Algorithm 2's offer of a list with a tree: every entry below m whose key
// is below the k-th key of N goes to N. A box is skipped when its nearest
// point is farther than the k-th key's distance (the pad key's distance is
// a NaN, which skips nothing) or its smallest rank is not below m. N ends
// as after the scan in rank order: the k smallest keys of N and the list.
template <int KC>
__device__ __forceinline__ void hub_offer(const CloudDev& C, int hub, float qx, float qy,
                                          float qz, int m, int k, WarpList<KC>& N, int lane,
                                          uint32_t* stack) {
  const int4 D = __ldg(C.hub_desc + hub);
  hub_walk(
      C, D, lane, stack,
      [&](float4 lo, float4 hi) {
        const float wd = __uint_as_float((uint32_t)(N.worst >> 32));
        const float bd = box_sqd32(qx, qy, qz, lo, hi);
        return (__float_as_int(lo.w) < m && !(bd > wd)) ? __float_as_uint(bd) : 0xffffffffu;
      },
      [&](uint32_t d) { return !(__uint_as_float(d) > __uint_as_float((uint32_t)(N.worst >> 32))); },
      [&](int chunk) {
        const float4 ps = __ldg(C.hub_ent + D.x + 32 * chunk + lane);
        const int s = __float_as_int(ps.w);
        const float d = sqd32(qx, qy, qz, ps);
        const uint64_t key = pack_key(d, (uint32_t)s);
        int pos = 0;
        const bool fresh = s < m && key < N.worst && !N.contains(key, pos);
        N.offer(fresh, key, pos, k, lane);
      });
}

// 32-bit words of a warp's tree-walk stack: per level a mask, a first
// index and 32 priorities.
constexpr int kHubStackWords = 34 * kHubMaxLevels;
// 64-bit words of shared memory for one warp of knn_query_warp<KC>.
__host__ __device__ constexpr int kWarpListWords(int kc) { return kc + kHubStackWords / 2; }

// One query by one warp (every lane calls it with the same query). With
// TREES (a cloud whose hub_of is not NULL) a list with a box tree is
// searched through the tree (after kHubScanFirst entries in the descent);
// the result is the same as the scan's. The walk's code costs registers
// and issue slots in the scan loop too, so clouds without trees run the
// instantiation without it. list: the warp's kWarpListWords(KC) words of
// shared memory (KC keys, then the tree walk's stack).
template <int KC, bool TREES>
__device__ __forceinline__ void knn_query_warp(const CloudDev& C, float qx, float qy, float qz,
                                               int k, int m, uint64_t* list,
                                               int32_t* __restrict__ out_idx,
                                               float* __restrict__ out_d2, int32_t row) {
  const int lane = (int)(threadIdx.x & 31u);
  WarpList<KC> N;
  N.init(list, lane);
  float dcur = sqd32(qx, qy, qz, __ldg(C.pts));
  N.insert(pack_key(dcur, 0u), k, lane);
  int cur = 0;  // the descent's current site, -1 once it is over
  int2 rr = __ldg(C.rows);
  int hub = -1;  // the current list's tree, or -1
  if constexpr (TREES) hub = __ldg(C.hub_of);
  int base = rr.x, end = rr.y;
  for (;;) {
    bool via_tree = false;
    if constexpr (TREES) via_tree = hub >= 0 && (cur < 0 || base - rr.x >= kHubScanFirst);
    if (via_tree) {
      if constexpr (TREES) {  // the list through its tree
        if (cur >= 0) {
          float bd;
          const int b = hub_first_closer(C, hub, qx, qy, qz, dcur, cur, m, lane,
                                         (uint32_t*)(list + KC), bd);
          if (b >= 0) {
            cur = b;
            dcur = bd;
            const uint64_t kb = pack_key(bd, (uint32_t)b);
            if (kb < N.worst) N.insert(kb, k, lane);
            rr = __ldg(C.rows + cur);
            base = rr.x;
            end = rr.y;
            hub = __ldg(C.hub_of + cur);
            continue;
          }
          cur = -1;
        } else {
          hub_offer(C, hub, qx, qy, qz, m, k, N, lane, (uint32_t*)(list + KC));
        }
      }
    } else {
      const int e = base + lane;
      const bool valid = e < end;
      float4 ps = make_float4(0.f, 0.f, 0.f, __int_as_float(0x7fffffff));
      if (valid) ps = __ldg(C.ent + e);
      const int s = __float_as_int(ps.w);
      const bool inr = valid && s < m;  // rows ascend: past the first s >= m nothing is
      const float d = sqd32(qx, qy, qz, ps);
      const uint64_t key = pack_key(d, (uint32_t)s);
      const bool row_done = __any_sync(0xffffffffu, valid && !inr) || base + 32 >= end;
      if (cur >= 0) {
        const bool cl = inr && strictly_closer_at(C, qx, qy, qz, d, ps, dcur, cur);
        const uint32_t b = __ballot_sync(0xffffffffu, cl);
        if (b) {
          const int w = __ffs((int)b) - 1;
          cur = __shfl_sync(0xffffffffu, s, w);
          dcur = __shfl_sync(0xffffffffu, d, w);
          const uint64_t kw = __shfl_sync(0xffffffffu, key, w);
          if (kw < N.worst) N.insert(kw, k, lane);
          rr = __ldg(C.rows + cur);
          base = rr.x;
          end = rr.y;
          if constexpr (TREES) hub = __ldg(C.hub_of + cur);
          continue;
        }
        if (row_done) cur = -1;
      } else {
        int pos = 0;
        const bool fresh = inr && key < N.worst && !N.contains(key, pos);
        N.offer(fresh, key, pos, k, lane);
      }
      if (!row_done) {
        base += 32;
        continue;
      }
    }
    const int pos = N.first_clear(min(N.cnt, k - 1));
    if (pos < 0) break;
    N.set_flag(pos);
    const int site = (int)(uint32_t)N.L[pos];
    rr = __ldg(C.rows + site);
    base = rr.x;
    end = rr.y;
    if constexpr (TREES) hub = __ldg(C.hub_of + site);
  }
  int32_t* oi = out_idx + (int64_t)row * k;
  float* od = out_d2 + (int64_t)row * k;
#pragma unroll
  for (int j = 0; j < KC / 32; ++j) {
    const int p = lane + 32 * j;
    if (p < k) {
      const bool real = p < N.cnt;
      const uint64_t key = N.L[p];
      __stcs(oi + p, real ? (int32_t)(uint32_t)key : -1);
      __stcs(od + p, real ? __uint_as_float((uint32_t)(key >> 32)) : __int_as_float(0x7f800000));
    }
  }
  __syncwarp();
}

// Writes a padded row (-1, +inf) for a query that cannot be served.
template <int G>
__device__ __forceinline__ void pad_row(const Grp<G>& g, int k, int32_t* oi, float* od) {
  for (int p = (int)g.lane; p < k; p += G) {
    oi[p] = -1;
    od[p] = __int_as_float(0x7f800000);
  }
}

}  // namespace mknn
