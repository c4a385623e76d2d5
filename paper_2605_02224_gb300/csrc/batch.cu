// Persistent multi-cloud query kernel, its work plan, the autotuner that
// picks the per-request kernel variant, and the CUDA graph that replays a
// plan.
//
// A plan covers many requests, each (cloud, queries, k, m, outputs). Every
// request is served by the kernel variant (lanes per query G, candidate
// slots per lane S) the tuner chose for its (k, cloud size, cloud shape),
// and cut into work items of a few rounds of its group width. The items of
// each variant form one queue, drained by one persistent launch of that
// variant's kernel (SM count x resident blocks): each warp takes the next
// item with one atomic. Items of one request are contiguous in a queue, so
// the warps working at any moment share one cloud's table in L2; requests
// are queued by decreasing estimated cost so that a queue ends with short
// items. The one-lane launch and the group launches run on two streams.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/mknn.h"
#include "batch.h"
#include "cloud.h"
#include "knn_device.cuh"
#include "knn_kernels.h"
#include "per_device.h"

namespace mknn {

namespace {

constexpr int kThreads = 256;

// Variants compiled into the persistent kernels: (G, S, list), list
// capacity G*S. list 2: shared memory (G = 1: a list per thread, any
// k <= 64 or <= 128; G = 32: one list per warp); list 1: the group's
// registers.
struct VariantDesc {
  int g, s, list;
};
constexpr VariantDesc kVariants[] = {{4, 1, 1},  {4, 2, 1},  {4, 4, 1},  {8, 1, 1},
                                     {8, 2, 1},  {8, 4, 1},  {8, 8, 1},  {16, 1, 1},
                                     {16, 2, 1}, {16, 4, 1}, {32, 1, 1}, {32, 2, 1},
                                     {1, 64, 2}, {16, 8, 1}, {32, 4, 1}, {1, 128, 2},
                                     {32, 1, 2}, {32, 2, 2}, {32, 4, 2}, {32, 1, 2},
                                     {32, 2, 2}, {32, 4, 2}, {1, 64, 2},  {1, 128, 2}};
constexpr int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);
static_assert(kVariants[kSmemVariant].g == 1 && kVariants[kSmemVariant128].g == 1,
              "one-lane variant indices");
static_assert(kVariants[kWarpVariant32].g == 32 && kVariants[kWarpVariant32].list == 2 &&
                  kVariants[kWarpVariant32 + 2].s == 4,
              "warp variant indices");
static_assert(kVariants[kTreeVariant32].g == 32 && kVariants[kTreeVariant32].list == 2 &&
                  kVariants[kTreeVariant32 + 2].s == 4 && kTreeVariant32 + 3 == kHandoverVariant,
              "tree variant indices");
static_assert(kVariants[kHandoverVariant].g == 1 && kVariants[kHandoverVariant].s == 64 &&
                  kVariants[kHandoverVariant128].s == 128 && kHandoverVariant128 + 1 == kNumVariants,
              "hand-over variant indices");

}  // namespace

int variant_index(int g, int k, int placement) {
  // one lane always keeps its list in shared memory in a plan; 4, 8 and 16
  // lanes always in registers
  const int list = g == 1 ? 2 : (g == 32 ? (placement == 2 ? 2 : 1) : 1);
  int best = -1;
  for (int i = 0; i < kNumVariants; ++i)
    if (kVariants[i].g == g && kVariants[i].list == list && kVariants[i].g * kVariants[i].s >= k &&
        k >= 1) {
      if (best < 0 || kVariants[i].s < kVariants[best].s) best = i;
    }
  return best;
}

namespace {

// One query by the list kind that suits its k (the thread's column holds
// at least list_slots(k) slots). W: flag words of the kernel's k class.
// DEFER: as knn_query_smem (false when the query was given up).
template <int W, bool DEFER = false>
__device__ __forceinline__ bool knn_query_smem_any(const CloudDev& C, float qx, float qy,
                                                   float qz, int k, int m, uint64_t* col,
                                                   int32_t* __restrict__ out_idx,
                                                   float* __restrict__ out_d2, int32_t row) {
  if constexpr (W == 1) {
    if (k <= 8)
      return knn_query_smem<SortedList<8, 1, true>, DEFER>(C, qx, qy, qz, k, m, col, 8, out_idx,
                                                           out_d2, row);
    else if (k <= 16)
      return knn_query_smem<PermList16, DEFER>(C, qx, qy, qz, k, m, col, 16, out_idx, out_d2,
                                               row);
    else
      return knn_query_smem<SortedList<32, 1, false>, DEFER>(C, qx, qy, qz, k, m, col, k,
                                                             out_idx, out_d2, row);
  } else if constexpr (W == 2) {
    return knn_query_smem<SortedList<64, 2, false>, DEFER>(C, qx, qy, qz, k, m, col, k, out_idx,
                                                           out_d2, row);
  } else {
    return knn_query_smem<SortedList<128, 4, false>, DEFER>(C, qx, qy, qz, k, m, col, k,
                                                            out_idx, out_d2, row);
  }
}

// This thread's column of its warp's shared-memory candidate lists.
__device__ __forceinline__ uint64_t* smem_column(int kcap) {
  extern __shared__ uint64_t batch_lists[];
  const int warp = (int)(threadIdx.x >> 5), lane = (int)(threadIdx.x & 31u);
  return batch_lists + (size_t)warp * kcap * 32 + lane;
}

// DEFER: a query that meets a list with a box tree is handed over
// (appended to the plan's list of its class) instead of answered.
template <int W, bool DEFER>
__device__ __forceinline__ void serve_item_smem(const ReqDev& R, const Item& w, uint64_t* col) {
  const int lane = (int)(threadIdx.x & 31u);
  const CloudDev C{R.pts, R.rows, R.succ, R.n, R.ent, DEFER ? R.hub_of : nullptr};
  for (int i = w.begin + lane; i < w.end; i += 32) {
    const int64_t qi = R.perm ? (int64_t)__ldg(R.perm + i) : (int64_t)i;
    const float* qp = R.q + qi * R.q_stride;
    const float qx = __ldg(qp), qy = __ldg(qp + 1), qz = __ldg(qp + 2);
    const int m = R.m ? __ldg(R.m + qi) : R.m_scalar;
    int32_t* oi = R.out_idx + qi * R.k;
    float* od = R.out_d2 + qi * R.k;
    if (m < 1 || m > C.n) {
      for (int p = 0; p < R.k; ++p) {
        oi[p] = -1;
        od[p] = __int_as_float(0x7f800000);
      }
      atomicOr(R.err, 1);
      continue;
    }
    const bool done =
        knn_query_smem_any<W, DEFER>(C, qx, qy, qz, R.k, m, col, R.out_idx, R.out_d2, (int32_t)qi);
    if constexpr (DEFER) {
      if (!done) {
        const int c = handover_class(R.k);
        R.ho->list[c][atomicAdd(&R.ho->count[c], 1)] = make_int2(w.req, (int)qi);
      }
    }
  }
}

template <int G, int S>
__device__ __forceinline__ void serve_item(const ReqDev& R, const Item& w) {
  const Grp<G> g;
  const int gi = (int)((threadIdx.x & 31u) / G);
  constexpr int kGroups = 32 / G;
  const CloudDev C{R.pts, R.rows, R.succ, R.n, R.ent};
  for (int i = w.begin + gi; i < w.end; i += kGroups) {
    const int64_t qi = R.perm ? (int64_t)__ldg(R.perm + i) : (int64_t)i;
    const float* qp = R.q + qi * R.q_stride;
    const float qx = __ldg(qp), qy = __ldg(qp + 1), qz = __ldg(qp + 2);
    const int m = R.m ? __ldg(R.m + qi) : R.m_scalar;
    if (m < 1 || m > C.n) {
      pad_row(g, R.k, R.out_idx + qi * R.k, R.out_d2 + qi * R.k);
      if (g.lane == 0) atomicOr(R.err, 1);
      continue;
    }
    QueryCounters qc{0, 0, 0, 0};
    knn_query<G, S, false>(C, g, qx, qy, qz, R.k, m, R.out_idx, R.out_d2, (int32_t)qi, qc);
  }
}

// One group variant (lists in registers) per kernel, so that each gets the
// registers it needs and the occupancy that follows (a single kernel holding
// every variant behind a switch was held to the largest one's registers).
// Variants with at most two slots per lane are held to 48 registers (five
// blocks per SM), as their plain counterparts compile to.
template <int G, int S>
__global__ void __launch_bounds__(kThreads, S <= 2 ? 5 : (S <= 4 ? 4 : 3)) knn_batch_group_kernel(const ReqDev* __restrict__ reqs,
                                                                   const Item* __restrict__ items,
                                                                   int nitems,
                                                                   int* __restrict__ next,
                                                                   int kcap) {
  (void)kcap;  // lists in registers
  const uint32_t lane = threadIdx.x & 31u;
  for (;;) {
    int it = 0;
    if (lane == 0) it = atomicAdd(next, 1);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= nitems) return;
    const Item w = items[it];
    serve_item<G, S>(reqs[w.req], w);
    __syncwarp();
  }
}

// The one-lane variant: one query per thread, candidate lists in shared
// memory, 256-thread blocks held to 48 registers as in the plain kernel.
template <int THREADS, int W, bool DEFER>
__global__ void __launch_bounds__(THREADS, THREADS == 256 ? 5 : 1) knn_batch_smem_kernel(const ReqDev* __restrict__ reqs,
                                                                 const Item* __restrict__ items,
                                                                 int nitems,
                                                                 int* __restrict__ next,
                                                                 int kcap) {
  const uint32_t lane = threadIdx.x & 31u;
  uint64_t* col = smem_column(kcap);
  for (;;) {
    int it = 0;
    if (lane == 0) it = atomicAdd(next, 1);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= nitems) return;
    const Item w = items[it];
    serve_item_smem<W, DEFER>(reqs[w.req], w, col);
    __syncwarp();
  }
}

// One warp per query, its candidate list in shared memory (KC keys per
// warp, static): the warp takes an item and answers its queries one after
// another.
template <int KC, bool TREES>
__global__ void __launch_bounds__(kThreads) knn_batch_warp_kernel(const ReqDev* __restrict__ reqs,
                                                                  const Item* __restrict__ items,
                                                                  int nitems,
                                                                  int* __restrict__ next,
                                                                  int kcap) {
  (void)kcap;
  __shared__ uint64_t lists[kThreads / 32][TREES ? kWarpListWords(KC) : KC];
  const int warp = (int)(threadIdx.x >> 5);
  const uint32_t lane = threadIdx.x & 31u;
  for (;;) {
    int it = 0;
    if (lane == 0) it = atomicAdd(next, 1);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= nitems) return;
    const Item w = items[it];
    const ReqDev& R = reqs[w.req];
    const CloudDev C{R.pts,    R.rows,     R.succ,    R.n,       R.ent,
                     R.hub_of, R.hub_desc, R.hub_ent, R.hub_node};
    for (int i = w.begin; i < w.end; ++i) {
      const int64_t qi = R.perm ? (int64_t)__ldg(R.perm + i) : (int64_t)i;
      const float* qp = R.q + qi * R.q_stride;
      const float qx = __ldg(qp), qy = __ldg(qp + 1), qz = __ldg(qp + 2);
      const int m = R.m ? __ldg(R.m + qi) : R.m_scalar;
      if (m < 1 || m > C.n) {
        for (int p = (int)lane; p < R.k; p += 32) {
          R.out_idx[qi * R.k + p] = -1;
          R.out_d2[qi * R.k + p] = __int_as_float(0x7f800000);
        }
        if (lane == 0) atomicOr(R.err, 1);
        continue;
      }
      knn_query_warp<KC, TREES>(C, qx, qy, qz, R.k, m, lists[warp], R.out_idx, R.out_d2,
                                (int32_t)qi);
    }
    __syncwarp();
  }
}

// The queries a plan's one-lane items handed over (class cls, one-warp
// lists of KC keys): one warp per query, the box trees walked; launched
// after every segment, it reads the number handed over from the device.
template <int KC>
__global__ void __launch_bounds__(kThreads) knn_batch_handover_kernel(
    const ReqDev* __restrict__ reqs, Handover* __restrict__ ho, int cls) {
  __shared__ uint64_t lists[kThreads / 32][kWarpListWords(KC)];
  const int warp = (int)(threadIdx.x >> 5);
  const uint32_t lane = threadIdx.x & 31u;
  const int n = ho->count[cls];
  const int2* __restrict__ list = ho->list[cls];
  for (;;) {
    int it = 0;
    if (lane == 0) it = atomicAdd(&ho->taken[cls], 1);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= n) return;
    const int2 pr = list[it];
    const ReqDev& R = reqs[pr.x];
    const CloudDev C{R.pts,    R.rows,     R.succ,    R.n,       R.ent,
                     R.hub_of, R.hub_desc, R.hub_ent, R.hub_node};
    const int64_t qi = pr.y;
    const float* qp = R.q + qi * R.q_stride;
    const float qx = __ldg(qp), qy = __ldg(qp + 1), qz = __ldg(qp + 2);
    const int m = R.m ? __ldg(R.m + qi) : R.m_scalar;  // checked by the one-lane item
    knn_query_warp<KC, true>(C, qx, qy, qz, R.k, m, lists[warp], R.out_idx, R.out_d2,
                             (int32_t)qi);
    __syncwarp();
  }
}

size_t list_bytes(int threads, int kcap) { return (size_t)threads * (size_t)kcap * 8; }

inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// ------------------------------------------------------------------ tuner

struct TuneKey {
  int k, nbucket, hub;
  bool operator<(const TuneKey& o) const {
    if (k != o.k) return k < o.k;
    return nbucket != o.nbucket ? nbucket < o.nbucket : hub < o.hub;
  }
};

std::mutex g_tune_mu;
std::map<TuneKey, Mode> g_tune;  // -> lanes and list placement

int nbucket_of(int64_t n) {
  int b = 0;
  while ((int64_t(1) << (b + 1)) <= n) ++b;
  return b;
}

// Untuned default: one query per thread, except on clouds with hub rows
// (a successor list of 2^12 entries or more, typical of nearly coplanar
// sites), where a whole warp per query scans the long rows 32 entries at a
// time. Timed on 64 mixed clouds, 32 lanes won on 16 of the 17 hub clouds
// (by 1.2x-3.9x) and lost on all but one of the others (by up to 20x).
// With box trees and the hand-over of mknn_knn_ex (one lane per query,
// the queries that meet a list with a tree answered by the one-warp kernel)
// one lane is the default up to k = 8: on the 20 patch clouds of that mix
// with trees it took 119 ms against 124 ms for 32 lanes, winning at k <= 8
// on all but two and losing at k = 16 and 32 by up to 1.7x.
constexpr int kHubBucketWide = 12;
constexpr int kHandoverMaxK = 8;
int heuristic_lanes(int k, int hub, bool handover) {
  if (handover && k <= kHandoverMaxK) return default_lanes(k);
  return hub >= kHubBucketWide ? 32 : default_lanes(k);
}

}  // namespace

int fill_lanes(int64_t nq, int k) {
  // One query per thread fills the GPU with (SMs x resident threads)
  // queries; resident threads of the shared-memory variant are limited by
  // its 48 registers (1280 per SM) and by 8 k bytes of list per thread.
  // Smaller batches give each query a group of lanes so all SMs work.
  const int64_t per_sm = std::min<int64_t>(1280, 233472 / (8 * (int64_t)std::max(k, 8)));
  const int64_t target = (int64_t)num_sms() * per_sm;
  int lanes = 1;
  while (lanes < 32 && nq * lanes < target) lanes <<= 1;
  if (lanes == 2) lanes = 4;  // no two-lane variant
  return lanes;
}

Mode choose_mode(int k, int64_t n, int hub, int64_t nq, bool trees) {
  const Mode t = tuned_mode(k, n, hub);
  const int fill = fill_lanes(nq, k);
  // one lane with the hand-over only where the launch stays one lane wide
  const int base = t.lanes ? t.lanes : heuristic_lanes(k, hub, trees && fill == 1);
  int lanes = std::max(base, fill);
  // widened on a cloud with box trees: the one-warp kernel, which walks them
  // (register groups would read the long lists through)
  if (trees && lanes > base && lanes < 32) lanes = 32;
  while (lanes < 32 && variant_index(lanes, k, 1) < 0) lanes <<= 1;  // e.g. 4 lanes hold k <= 16
  const int placement = (t.lanes && lanes == t.lanes) ? t.placement : default_placement(k, lanes);
  return Mode{lanes, placement};
}

namespace {

// Largest dynamic shared memory each kernel is launched with; set once per
// device (a kernel attribute belongs to one device's context).
PerDevice<int> g_attr_set;

cudaError_t set_smem_attributes() {
  const struct {
    const void* fn;
    size_t bytes;
  } kernels[] = {{(const void*)knn_batch_smem_kernel<256, 1, false>, list_bytes(256, 32)},
                 {(const void*)knn_batch_smem_kernel<128, 2, false>, list_bytes(128, 64)},
                 {(const void*)knn_batch_smem_kernel<64, 4, false>, list_bytes(64, 128)},
                 {(const void*)knn_batch_smem_kernel<256, 1, true>, list_bytes(256, 32)},
                 {(const void*)knn_batch_smem_kernel<128, 2, true>, list_bytes(128, 64)},
                 {(const void*)knn_batch_smem_kernel<64, 4, true>, list_bytes(64, 128)}};
  cudaError_t e = cudaSuccess;
  for (const auto& kn : kernels)
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(kn.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kn.bytes);
  return e;
}

cudaError_t ensure_smem_attributes() {
  return g_attr_set.with(current_device(), cudaErrorInvalidDevice, [](int& done) {
    if (done) return cudaSuccess;
    const cudaError_t e = set_smem_attributes();
    if (e == cudaSuccess) done = 1;
    return e;
  });
}

// The kernel of a variant (the one-lane kernel by its block size).
const void* variant_kernel(int variant, int threads) {
  switch (variant) {
    case 0: return (const void*)knn_batch_group_kernel<4, 1>;
    case 1: return (const void*)knn_batch_group_kernel<4, 2>;
    case 2: return (const void*)knn_batch_group_kernel<4, 4>;
    case 3: return (const void*)knn_batch_group_kernel<8, 1>;
    case 4: return (const void*)knn_batch_group_kernel<8, 2>;
    case 5: return (const void*)knn_batch_group_kernel<8, 4>;
    case 6: return (const void*)knn_batch_group_kernel<8, 8>;
    case 7: return (const void*)knn_batch_group_kernel<16, 1>;
    case 8: return (const void*)knn_batch_group_kernel<16, 2>;
    case 9: return (const void*)knn_batch_group_kernel<16, 4>;
    case 10: return (const void*)knn_batch_group_kernel<32, 1>;
    case 11: return (const void*)knn_batch_group_kernel<32, 2>;
    case 13: return (const void*)knn_batch_group_kernel<16, 8>;
    case 14: return (const void*)knn_batch_group_kernel<32, 4>;
    case kWarpVariant32: return (const void*)knn_batch_warp_kernel<32, false>;
    case kWarpVariant32 + 1: return (const void*)knn_batch_warp_kernel<64, false>;
    case kWarpVariant32 + 2: return (const void*)knn_batch_warp_kernel<128, false>;
    case kTreeVariant32: return (const void*)knn_batch_warp_kernel<32, true>;
    case kTreeVariant32 + 1: return (const void*)knn_batch_warp_kernel<64, true>;
    case kTreeVariant32 + 2: return (const void*)knn_batch_warp_kernel<128, true>;
    case kSmemVariant:
      return threads == 256 ? (const void*)knn_batch_smem_kernel<256, 1, false>
                            : (const void*)knn_batch_smem_kernel<128, 2, false>;
    case kSmemVariant128: return (const void*)knn_batch_smem_kernel<64, 4, false>;
    case kHandoverVariant:
      return threads == 256 ? (const void*)knn_batch_smem_kernel<256, 1, true>
                            : (const void*)knn_batch_smem_kernel<128, 2, true>;
    case kHandoverVariant128: return (const void*)knn_batch_smem_kernel<64, 4, true>;
    default: return nullptr;
  }
}

}  // namespace

BatchLaunch batch_config(int nitems, int blocks_per_sm, int kcap, int variant) {
  ensure_smem_attributes();  // an error shows again at launch
  BatchLaunch b;
  b.variant = variant;
  const bool smem = is_smem_variant(variant);
  b.kcap = smem ? kcap : 0;
  b.threads = is_smem128_variant(variant) ? 64 : smem ? (kcap <= 32 ? 256 : 128) : kThreads;
  b.smem = smem ? list_bytes(b.threads, kcap) : 0;
  int occ = 1;
  const void* fn = variant_kernel(variant, b.threads);
  if (!fn || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, b.threads, b.smem) !=
                 cudaSuccess || occ < 1) {
    cudaGetLastError();
    occ = 1;
  }
  const int per_sm = blocks_per_sm > 0 ? std::min(blocks_per_sm, occ) : occ;
  const int wpb = b.threads / 32;
  const int64_t blocks_needed = ((int64_t)std::max(1, nitems) + wpb - 1) / wpb;
  b.grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)num_sms() * per_sm, blocks_needed));
  return b;
}

cudaError_t launch_batch_kernel(const ReqDev* d_reqs, const Item* d_items, int nitems, int* d_next,
                                const BatchLaunch& b, cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  const cudaError_t ae = ensure_smem_attributes();
  if (ae != cudaSuccess) return ae;
  const void* fn = variant_kernel(b.variant, b.threads);
  if (!fn) return cudaErrorInvalidValue;
  int kcap = b.kcap;
  void* args[] = {(void*)&d_reqs, (void*)&d_items, (void*)&nitems, (void*)&d_next, (void*)&kcap};
  return cudaLaunchKernel(fn, dim3((unsigned)b.grid), dim3((unsigned)b.threads), args, b.smem, s);
}

std::vector<Segment> make_segments(std::vector<Item>& items, int blocks_per_sm,
                                   const std::vector<int>& req_k) {
  // one-lane items by list class (8, 16, 32, 64 slots): a launch's shared
  // memory is sized for its largest list, and a list of 8 slots in a block
  // sized for 32 would cut the resident threads by two fifths (non-hub
  // requests of the batching workload: 99 ms in four one-lane segments
  // against 107 ms in one)
  auto rank = [](int v) { return is_smem_variant(v) ? v - 100 : v; };
  auto cls = [&](const Item& a) {
    if (!is_smem_variant(a.variant)) return 0;
    const int slots = list_slots(req_k[a.req]);
    return slots <= 8 ? 0 : (slots <= 16 ? 1 : (slots <= 32 ? 2 : 3));
  };
  std::stable_sort(items.begin(), items.end(), [&](const Item& a, const Item& c) {
    return rank(a.variant) != rank(c.variant) ? rank(a.variant) < rank(c.variant) : cls(a) < cls(c);
  });
  std::vector<Segment> segs;
  for (int i = 0; i < (int)items.size();) {
    int j = i;
    while (j < (int)items.size() && items[j].variant == items[i].variant &&
           cls(items[j]) == cls(items[i]))
      ++j;
    int kcap = 0;
    for (int t = i; t < j; ++t) kcap = std::max(kcap, list_slots(req_k[items[t].req]));
    Segment g;
    g.begin = i;
    g.count = j - i;
    g.launch = batch_config(g.count, blocks_per_sm, kcap, items[i].variant);
    segs.push_back(g);
    i = j;
  }
  return segs;
}

// The one-warp kernel of hand-over class c and its persistent grid.
static const void* handover_kernel(int c) {
  return c == 0 ? (const void*)knn_batch_handover_kernel<32>
                : (c == 1 ? (const void*)knn_batch_handover_kernel<64>
                          : (const void*)knn_batch_handover_kernel<128>);
}

int handover_grid(int c) {
  int occ = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, handover_kernel(c), kThreads, 0) !=
          cudaSuccess ||
      occ < 1) {
    cudaGetLastError();
    occ = 1;
  }
  return num_sms() * occ;
}

cudaError_t launch_handover(const ReqDev* d_reqs, Handover* d_ho, int c, int grid, cudaStream_t s) {
  void* args[] = {(void*)&d_reqs, (void*)&d_ho, (void*)&c};
  return cudaLaunchKernel(handover_kernel(c), dim3((unsigned)grid), dim3((unsigned)kThreads), args,
                          0, s);
}

cudaError_t launch_segments(const ReqDev* d_reqs, const Item* d_items, int* d_next,
                            const std::vector<Segment>& segs, cudaStream_t s, cudaStream_t aux,
                            cudaEvent_t fork, cudaEvent_t join, int64_t queries) {
  bool one = false, group = false;
  for (const Segment& g : segs) (is_smem_variant(g.launch.variant) ? one : group) = true;
  const bool split = one && group && aux && queries <= kSplitMaxQueries;
  cudaError_t e = cudaSuccess;
  if (split) {
    if ((e = cudaEventRecord(fork, s)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(aux, fork, 0)) != cudaSuccess) return e;
  }
  for (size_t i = 0; i < segs.size() && e == cudaSuccess; ++i) {
    const Segment& g = segs[i];
    cudaStream_t st = (split && !is_smem_variant(g.launch.variant)) ? aux : s;
    e = launch_batch_kernel(d_reqs, d_items + g.begin, g.count, d_next + i, g.launch, st);
  }
  if (e != cudaSuccess || !split) return e;
  if ((e = cudaEventRecord(join, aux)) != cudaSuccess) return e;
  return cudaStreamWaitEvent(s, join, 0);
}

Mode tuned_mode(int k, int64_t n, int hub) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(TuneKey{k, nbucket_of(n), hub});
  return it == g_tune.end() ? Mode{0, 0} : it->second;
}

void set_tuned_mode(int k, int64_t n, int hub, Mode m) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[TuneKey{k, nbucket_of(n), hub}] = m;
}

}  // namespace mknn

using namespace mknn;

struct mknn_batch {
  int device = -1;
  int nreq = 0;
  std::vector<mknn_batch_req> reqs;
  std::vector<uint64_t> gens;    // each request's cloud generation when the plan was made
  std::vector<int> lanes;        // chosen lanes per request
  std::vector<int> placement;    // and list placement (2 shared memory, 1 registers)
  ReqDev* d_reqs = nullptr;
  // work items grouped by kernel variant, one queue counter per segment
  Item* d_items = nullptr;
  int64_t nitems = 0;
  std::vector<Segment> segs;
  int* d_next = nullptr;         // [i] queue of segment i
  void* d_ws = nullptr;          // sort scratch: shared histogram, per-request cells and orders
  size_t ws_bytes = 0;
  std::vector<size_t> cell_off, perm_off;  // per request, 0 if not sorted
  cudaStream_t aux = nullptr;    // second branch: the group segments
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t total_queries = 0;
  // hand-over of one-lane items on clouds with box trees: the lists and
  // counters (device), and which classes a run must drain
  Handover* d_ho = nullptr;
  int2* d_ho_pairs = nullptr;
  bool ho_class[3] = {false, false, false};
  int ho_grid[3] = {0, 0, 0};
};

namespace {

mknn_status bfail(mknn_status s, const std::string& msg) {
  set_error(msg);
  return s;
}

void free_plan(mknn_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  cudaFree(b->d_reqs);
  cudaFree(b->d_items);
  cudaFree(b->d_next);
  cudaFree(b->d_ws);
  cudaFree(b->d_ho);
  cudaFree(b->d_ho_pairs);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->ev_join) cudaEventDestroy(b->ev_join);
  if (b->aux) cudaStreamDestroy(b->aux);
  delete b;
}

// Enqueues the plan's work on stream s: the locality sorts, the persistent
// launch of each segment, then the one-warp launches for the queries the
// one-lane items handed over.
cudaError_t enqueue(mknn_batch* b, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(b->d_next, 0, b->segs.size() * sizeof(int), s);
  if (e != cudaSuccess) return e;
  if (b->d_ho) {
    e = cudaMemsetAsync(&b->d_ho->count[0], 0, sizeof(Handover) - offsetof(Handover, count), s);
    if (e != cudaSuccess) return e;
  }
  for (int r = 0; r < b->nreq; ++r) {
    if (!b->perm_off[r]) continue;
    const mknn_batch_req& R = b->reqs[r];
    const CloudDevHost cd = R.cloud->dev();
    // the histogram at offset 0 is shared: the sorts run one after another
    e = launch_query_sort_split(cd, R.q, R.q_stride, R.nq, b->d_ws,
                                (int32_t*)((char*)b->d_ws + b->cell_off[r]),
                                (int32_t*)((char*)b->d_ws + b->perm_off[r]), s);
    if (e != cudaSuccess) return e;
  }
  e = launch_segments(b->d_reqs, b->d_items, b->d_next, b->segs, s, b->aux, b->ev_fork,
                      b->ev_join, b->total_queries);
  for (int c = 0; c < 3 && e == cudaSuccess; ++c)
    if (b->ho_class[c]) e = launch_handover(b->d_reqs, b->d_ho, c, b->ho_grid[c], s);
  return e;
}

}  // namespace

extern "C" {

size_t mknn_batch_sizeof_req(void) { return sizeof(mknn_batch_req); }

mknn_status mknn_batch_create(const mknn_batch_req* reqs, int32_t nreq,
                              const mknn_batch_opts* opts, mknn_batch** out) {
  if (!out) return bfail(MKNN_EINVAL, "out is NULL");
  *out = nullptr;
  if (nreq < 0 || (nreq > 0 && !reqs)) return bfail(MKNN_EINVAL, "bad request array");
  int dev = 0;
  cudaGetDevice(&dev);
  mknn_batch_opts o{};
  if (opts) o = *opts;
  std::unique_ptr<mknn_batch> b(new mknn_batch());
  b->device = dev;
  b->nreq = nreq;
  b->reqs.assign(reqs, reqs + nreq);
  b->gens.resize(nreq);
  for (int r = 0; r < nreq; ++r) b->gens[r] = reqs[r].cloud ? reqs[r].cloud->generation.load() : 0;
  b->lanes.resize(nreq);
  b->placement.resize(nreq);
  b->cell_off.assign(nreq, 0);
  b->perm_off.assign(nreq, 0);
  std::vector<ReqDev> rd(nreq);
  std::vector<double> cost(nreq);
  int64_t plan_nq = 0;  // all requests run in one launch: widen only if the whole plan is small
  for (int r = 0; r < nreq; ++r) plan_nq += std::max<int64_t>(0, reqs[r].nq);
  for (int r = 0; r < nreq; ++r) {
    const mknn_batch_req& R = reqs[r];
    if (!R.cloud || !R.cloud->d_pts || R.cloud->device != dev)
      return bfail(MKNN_EINVAL, "request " + std::to_string(r) +
                                    ": cloud missing or not uploaded on the current device");
    if (R.nq < 0 || R.nq >= kRequestQueryLimit || R.q_stride < 3 || R.k < 1 ||
        R.k > MKNN_MAX_K)
      return bfail(MKNN_EINVAL, "request " + std::to_string(r) + ": bad nq, q_stride or k");
    int32_t ms = R.m_scalar;
    if (!R.m) {
      if (ms == 0) ms = (int32_t)R.cloud->n;
      if (ms < 1 || ms > R.cloud->n)
        return bfail(MKNN_EINVAL, "request " + std::to_string(r) + ": m_scalar out of [1, n]");
    }
    if (R.nq > 0 && (!R.q || !R.out_idx || !R.out_d2))
      return bfail(MKNN_EINVAL, "request " + std::to_string(r) + ": NULL device pointer");
    const Mode chosen =
        choose_mode(R.k, R.cloud->n, R.cloud->hub_bucket(), plan_nq, R.cloud->d_hub_of != nullptr);
    const int lanes = o.lanes ? o.lanes : chosen.lanes;
    const int placement = o.placement ? o.placement
                                      : (o.lanes ? default_placement(R.k, lanes) : chosen.placement);
    if (variant_index(lanes, R.k, placement) < 0)
      return bfail(MKNN_EINVAL, "request " + std::to_string(r) + ": lanes/k combination");
    b->lanes[r] = lanes;
    b->placement[r] = placement;
    const CloudDevHost cd = R.cloud->dev();
    rd[r] = ReqDev{(const float4*)cd.pts, cd.rows,   cd.succ, cd.n,  R.q_stride,
                   R.q,                   R.m,       nullptr, R.out_idx,
                   R.out_d2,              R.cloud->d_err, R.k, ms, (const float4*)cd.ent,
                   cd.hub_of, (const int4*)cd.hub_desc, (const float4*)cd.hub_ent,
                   (const float4*)cd.hub_node};
    cost[r] = (double)R.k * std::log2((double)R.cloud->n + 2.0);
    b->total_queries += R.nq;
  }
  // sort scratch: one shared histogram, then per request cells and order
  const bool sort_on = o.sort >= 0;
  size_t off = kSortHistBytes;
  for (int r = 0; r < nreq; ++r) {
    if (!sort_on || reqs[r].nq < (o.sort > 0 ? 1 : 4096)) continue;
    b->cell_off[r] = off;
    off += align256((size_t)reqs[r].nq * 4);
    b->perm_off[r] = off;
    off += align256((size_t)reqs[r].nq * 4);
  }
  b->ws_bytes = off;
  // work items, requests by decreasing cost
  std::vector<int> orderq(nreq);
  for (int r = 0; r < nreq; ++r) orderq[r] = r;
  std::stable_sort(orderq.begin(), orderq.end(), [&](int a, int c) { return cost[a] > cost[c]; });
  const int rounds = o.item_rounds > 0 ? o.item_rounds : kItemRounds;
  std::vector<Item> items;
  std::vector<int> req_k(nreq);
  for (int r = 0; r < nreq; ++r) req_k[r] = reqs[r].k;
  int64_t ho_cap[3] = {0, 0, 0};  // queries that may be handed over, per class
  for (int r : orderq) {
    const int v = with_trees(variant_index(b->lanes[r], reqs[r].k, b->placement[r]),
                             reqs[r].cloud->d_hub_of != nullptr, true);
    if (v == kHandoverVariant || v == kHandoverVariant128) {
      ho_cap[handover_class(reqs[r].k)] += reqs[r].nq;
      b->ho_class[handover_class(reqs[r].k)] = true;
    }
    const int per = item_queries(b->lanes[r], rounds);
    for (int64_t s0 = 0; s0 < reqs[r].nq; s0 += per)
      items.push_back(Item{r, (int32_t)s0, (int32_t)std::min<int64_t>(reqs[r].nq, s0 + per), v});
  }
  b->segs = make_segments(items, o.blocks_per_sm, req_k);
  b->nitems = (int64_t)items.size();
  cudaError_t e;
  if ((e = cudaMalloc((void**)&b->d_reqs, sizeof(ReqDev) * std::max(nreq, 1))) != cudaSuccess ||
      (e = cudaMalloc((void**)&b->d_items, sizeof(Item) * std::max<size_t>(items.size(), 1))) !=
          cudaSuccess ||
      (e = cudaMalloc((void**)&b->d_next, 256)) != cudaSuccess ||
      (e = cudaMalloc(&b->d_ws, std::max<size_t>(b->ws_bytes, 256))) != cudaSuccess) {
    cudaGetLastError();
    mknn_batch* raw = b.release();
    free_plan(raw);
    return bfail(MKNN_ENOMEM, "device allocation for the batch plan failed");
  }
  for (int r = 0; r < nreq; ++r)
    if (b->perm_off[r]) rd[r].perm = (const int32_t*)((char*)b->d_ws + b->perm_off[r]);
  if (ho_cap[0] + ho_cap[1] + ho_cap[2] > 0) {
    Handover h{};
    if ((e = cudaMalloc((void**)&b->d_ho, sizeof(Handover))) != cudaSuccess ||
        (e = cudaMalloc((void**)&b->d_ho_pairs,
                        sizeof(int2) * (size_t)(ho_cap[0] + ho_cap[1] + ho_cap[2]))) !=
            cudaSuccess) {
      cudaGetLastError();
      mknn_batch* raw = b.release();
      free_plan(raw);
      return bfail(MKNN_ENOMEM, "device allocation for the batch plan failed");
    }
    int64_t at = 0;
    for (int c = 0; c < 3; ++c) {
      h.list[c] = b->d_ho_pairs + at;
      at += ho_cap[c];
    }
    if ((e = cudaMemcpy(b->d_ho, &h, sizeof(h), cudaMemcpyHostToDevice)) != cudaSuccess) {
      mknn_batch* raw = b.release();
      free_plan(raw);
      return bfail(MKNN_ECUDA, std::string("plan upload: ") + cudaGetErrorString(e));
    }
    for (int r = 0; r < nreq; ++r)
      if (reqs[r].cloud->d_hub_of) rd[r].ho = b->d_ho;
    for (int c = 0; c < 3; ++c)
      if (b->ho_class[c]) b->ho_grid[c] = handover_grid(c);
  }
  if ((e = cudaMemcpy(b->d_reqs, rd.data(), sizeof(ReqDev) * nreq, cudaMemcpyHostToDevice)) !=
          cudaSuccess ||
      (e = cudaMemcpy(b->d_items, items.data(), sizeof(Item) * items.size(),
                      cudaMemcpyHostToDevice)) != cudaSuccess) {
    mknn_batch* raw = b.release();
    free_plan(raw);
    return bfail(MKNN_ECUDA, std::string("plan upload: ") + cudaGetErrorString(e));
  }
  bool one = false, group = false;
  for (const Segment& g : b->segs) (is_smem_variant(g.launch.variant) ? one : group) = true;
  if (one && group) {
    if ((e = cudaStreamCreateWithFlags(&b->aux, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming)) != cudaSuccess) {
      mknn_batch* raw = b.release();
      free_plan(raw);
      return bfail(MKNN_ECUDA, std::string("plan streams: ") + cudaGetErrorString(e));
    }
  }
  if (o.graph >= 0) {
    cudaStream_t cs;
    if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) == cudaSuccess) {
      e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        cudaError_t e2 = enqueue(b.get(), cs);
        e = cudaStreamEndCapture(cs, &b->graph);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
      }
      cudaStreamDestroy(cs);
    }
    if (e != cudaSuccess) {
      cudaGetLastError();
      if (b->exec) cudaGraphExecDestroy(b->exec);
      if (b->graph) cudaGraphDestroy(b->graph);
      b->exec = nullptr;
      b->graph = nullptr;
      mknn_batch* raw = b.release();
      free_plan(raw);
      return bfail(MKNN_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    }
  }
  *out = b.release();
  return MKNN_OK;
}

mknn_status mknn_batch_run(mknn_batch* b, mknn_stream_t stream) {
  if (!b) return bfail(MKNN_EINVAL, "plan is NULL");
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != b->device) return bfail(MKNN_EINVAL, "plan was made on another device");
  for (int r = 0; r < b->nreq; ++r)
    if (b->reqs[r].cloud && b->reqs[r].cloud->generation.load() != b->gens[r])
      return bfail(MKNN_EINVAL, "request " + std::to_string(r) +
                                    ": its cloud changed (append) since the plan was made");
  cudaError_t e = b->exec ? cudaGraphLaunch(b->exec, (cudaStream_t)stream)
                          : enqueue(b, (cudaStream_t)stream);
  if (e != cudaSuccess) return bfail(MKNN_ECUDA, std::string("batch run: ") + cudaGetErrorString(e));
  return MKNN_OK;
}

mknn_status mknn_batch_info(const mknn_batch* b, int32_t* lanes_out, int64_t* items,
                            int32_t* grid) {
  if (!b) return bfail(MKNN_EINVAL, "plan is NULL");
  if (lanes_out)
    for (int r = 0; r < b->nreq; ++r) lanes_out[r] = b->lanes[r];
  if (items) *items = b->nitems;
  if (grid) {
    int g = 0;
    for (const Segment& sg : b->segs) g += sg.launch.grid;
    *grid = g;
  }
  return MKNN_OK;
}

mknn_status mknn_batch_placement(const mknn_batch* b, int32_t* placement_out) {
  if (!b || (!placement_out && b->nreq > 0)) return bfail(MKNN_EINVAL, "NULL argument");
  for (int r = 0; r < b->nreq; ++r) placement_out[r] = b->placement[r];
  return MKNN_OK;
}

mknn_status mknn_batch_free(mknn_batch* b) {
  free_plan(b);
  return MKNN_OK;
}

mknn_status mknn_knn_batch(const mknn_batch_req* reqs, int32_t nreq, const mknn_batch_opts* opts,
                           mknn_stream_t stream) {
  mknn_batch_opts o{};
  if (opts) o = *opts;
  o.graph = -1;
  mknn_batch* b = nullptr;
  mknn_status st = mknn_batch_create(reqs, nreq, &o, &b);
  if (st != MKNN_OK) return st;
  st = mknn_batch_run(b, stream);
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  free_plan(b);
  if (st != MKNN_OK) return st;
  if (e != cudaSuccess) return bfail(MKNN_ECUDA, std::string("batch: ") + cudaGetErrorString(e));
  return MKNN_OK;
}

// Times each candidate (lanes, placement) on a sample of every distinct (k,
// size bucket, hub bucket) among the requests, as the persistent plan
// variant a plan would run, and records the fastest in the tuning table.
mknn_status mknn_batch_tune(const mknn_batch_req* reqs, int32_t nreq, int64_t sample,
                            mknn_stream_t stream) {
  if (nreq < 0 || (nreq > 0 && !reqs)) return bfail(MKNN_EINVAL, "bad request array");
  // The table serves large launches (whole plans), so each candidate is timed
  // on at least twice the queries that fill the GPU one per thread; a
  // request with fewer queries is tiled to that size.
  const int64_t fill = (int64_t)num_sms() * 2048 * 2;
  const int64_t ns = std::max<int64_t>(sample, fill);
  cudaStream_t s = (cudaStream_t)stream;
  std::map<TuneKey, int> seen;
  int32_t* d_idx = nullptr;
  float* d_d2 = nullptr;
  float* d_q = nullptr;
  int32_t* d_m = nullptr;
  size_t cap = 0, cap_q = 0;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  mknn_status st = MKNN_OK;
  static const Mode kCandidates[] = {{1, 2}, {4, 1}, {8, 1}, {16, 1}, {32, 1}, {32, 2}};
  for (int r = 0; r < nreq && st == MKNN_OK; ++r) {
    const mknn_batch_req& R = reqs[r];
    if (!R.cloud || R.nq <= 0) continue;
    const TuneKey key{R.k, nbucket_of(R.cloud->n), R.cloud->hub_bucket()};
    if (seen.count(key)) continue;
    seen[key] = 1;
    const size_t need = (size_t)ns * R.k * 4;
    const size_t need_q = (size_t)ns * R.q_stride * 4;
    if (need > cap || need_q > cap_q) {
      cudaFree(d_idx);
      cudaFree(d_d2);
      cudaFree(d_q);
      cudaFree(d_m);
      d_idx = nullptr;
      d_d2 = nullptr;
      d_q = nullptr;
      d_m = nullptr;
      if (cudaMalloc((void**)&d_idx, need) != cudaSuccess ||
          cudaMalloc((void**)&d_d2, need) != cudaSuccess ||
          cudaMalloc((void**)&d_q, need_q) != cudaSuccess ||
          cudaMalloc((void**)&d_m, (size_t)ns * 4) != cudaSuccess) {
        cudaGetLastError();
        st = bfail(MKNN_ENOMEM, "tuner buffers");
        break;
      }
      cap = need;
      cap_q = need_q;
    }
    for (int64_t off = 0; off < ns; off += R.nq) {
      const int64_t len = std::min<int64_t>(R.nq, ns - off);
      cudaMemcpyAsync(d_q + off * R.q_stride, R.q, (size_t)len * R.q_stride * 4,
                      cudaMemcpyDeviceToDevice, s);
      if (R.m) cudaMemcpyAsync(d_m + off, R.m, (size_t)len * 4, cudaMemcpyDeviceToDevice, s);
    }
    // the sample as one request of a one-request plan
    mknn_batch_req T = R;
    T.q = d_q;
    T.nq = ns;
    T.m = R.m ? d_m : nullptr;
    T.out_idx = d_idx;
    T.out_d2 = d_d2;
    Mode best{0, 0};
    float best_ms = 1e30f;
    for (const Mode& cand : kCandidates) {
      if (variant_index(cand.lanes, R.k, cand.placement) < 0) continue;
      mknn_batch_opts bo{};
      bo.lanes = cand.lanes;
      bo.placement = cand.placement;
      bo.graph = -1;
      mknn_batch* plan = nullptr;
      st = mknn_batch_create(&T, 1, &bo, &plan);
      if (st != MKNN_OK) break;
      float ms_min = 1e30f;
      for (int rep = 0; rep < 3 && st == MKNN_OK; ++rep) {
        cudaEventRecord(e0, s);
        st = mknn_batch_run(plan, stream);
        cudaEventRecord(e1, s);
        if (st != MKNN_OK) break;
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) ms_min = std::min(ms_min, ms);
      }
      free_plan(plan);
      if (st != MKNN_OK) break;
      if (const char* logp = std::getenv("MKNN_TUNE_LOG")) {
        if (FILE* lf = std::fopen(logp, "a")) {
          std::fprintf(lf, "k=%d n=%lld hub=%d sample=%lld lanes=%d placement=%d ms=%.4f\n",
                       R.k, (long long)R.cloud->n, key.hub, (long long)ns, cand.lanes,
                       cand.placement, ms_min);
          std::fclose(lf);
        }
      }
      if (ms_min < best_ms) {
        best_ms = ms_min;
        best = cand;
      }
    }
    if (st == MKNN_OK && best.lanes) set_tuned_mode(R.k, R.cloud->n, key.hub, best);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d_idx);
  cudaFree(d_d2);
  cudaFree(d_q);
  cudaFree(d_m);
  return st;
}

mknn_status mknn_tune_save(const char* path) {
  if (!path) return bfail(MKNN_EINVAL, "NULL path");
  FILE* f = std::fopen(path, "w");
  if (!f) return bfail(MKNN_EIO, std::string("cannot open ") + path);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  std::fprintf(f, "# k log2(n) log2(1+longest list) lanes placement\n");
  for (auto& kv : g_tune)
    std::fprintf(f, "%d %d %d %d %d\n", kv.first.k, kv.first.nbucket, kv.first.hub,
                 kv.second.lanes, kv.second.placement);
  return std::fclose(f) == 0 ? MKNN_OK : bfail(MKNN_EIO, "write failed");
}

mknn_status mknn_tune_clear(void) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune.clear();
  return MKNN_OK;
}

mknn_status mknn_tune_load(const char* path) {
  if (!path) return bfail(MKNN_EINVAL, "NULL path");
  FILE* f = std::fopen(path, "r");
  if (!f) return bfail(MKNN_EIO, std::string("cannot open ") + path);
  char line[256];
  std::map<TuneKey, Mode> t;
  while (std::fgets(line, sizeof line, f)) {
    if (line[0] == '#') continue;
    int k, nb, hub, lanes, placement = 0;
    const int got = std::sscanf(line, "%d %d %d %d %d", &k, &nb, &hub, &lanes, &placement);
    if (got < 4) continue;
    if (got == 4 || placement == 0) placement = default_placement(k, lanes);
    if (variant_index(lanes, k, placement) >= 0) t[TuneKey{k, nb, hub}] = Mode{lanes, placement};
  }
  std::fclose(f);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (auto& kv : t) g_tune[kv.first] = kv.second;
  return MKNN_OK;
}

}  // extern "C"
