// Internal interface of the persistent multi-cloud kernel, its work items
// and the tuning table (shared by the batch plan and the serving loop).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

namespace mknn {

// One request as the persistent kernel sees it (device-side copy).
struct ReqDev {
  const float4* pts;
  const int2* rows;
  const int32_t* succ;
  int32_t n;
  int32_t q_stride;
  const float* q;
  const int32_t* m;
  const int32_t* perm;
  int32_t* out_idx;
  float* out_d2;
  int32_t* err;
  int32_t k;
  int32_t m_scalar;
  const float4* ent;   // the cloud's successor entries with sites inlined
  // the cloud's box trees over its long lists (read by the one-warp variant)
  const int32_t* hub_of;
  const int4* hub_desc;
  const float4* hub_ent;
  const float4* hub_node;
  // the plan's hand-over lists (one-lane items on a cloud with trees), or NULL
  struct Handover* ho;
};

// Queries a plan's one-lane items hand over to the one-warp kernel with
// trees, by the list class of their k (one-warp lists of 32, 64, 128 keys).
struct Handover {
  int2* list[3];      // (request, query index) pairs
  int32_t count[3];   // pairs appended in this run
  int32_t taken[3];   // pairs taken by the one-warp launches
};
__host__ __device__ inline int handover_class(int k) { return k <= 32 ? 0 : (k <= 64 ? 1 : 2); }
// The persistent grid of the one-warp launch that drains hand-over class c,
// and that launch (after the segments whose items hand queries over).
int handover_grid(int c);
cudaError_t launch_handover(const ReqDev* d_reqs, Handover* d_ho, int c, int grid, cudaStream_t s);

// Queries per request below this bound: a lane's query index plus its
// stride within an item (at most 256 queries) then stays below 2^31 - 1.
constexpr int64_t kRequestQueryLimit = (int64_t)0x7FFFFFFF - 256;

// A contiguous range of one request's queries (in processing order),
// served by one warp with kernel variant `variant`.
struct Item {
  int32_t req, begin, end, variant;
};

// Variant index for lanes-per-query G, capacity k and list placement
// (2 = shared memory, 1 = registers; only 32 lanes have both), or -1.
int variant_index(int lanes, int k, int placement);
// Queries per work item for the given lanes and rounds per item.
inline int item_queries(int lanes, int rounds) { return (32 / lanes) * rounds; }
// Rounds per work item (a warp answers its item's queries one round after
// another): one. Longer items hold up the end of a persistent launch and,
// with groups of lanes on clouds with hub rows, let one slow query hold up
// the rest of its item. On the 64-cloud batching workload (57.6M queries)
// the plan took 233 / 240 / 248 ms with items of 1 / 2 / 4 rounds and 276
// ms with the earlier 8 for one lane per query (one plain launch per cloud:
// 240 ms); on a 322k-site planar-patches cloud 32-lane items of 8 queries
// took 9.2 ms, of one query 3.2 ms.
constexpr int kItemRounds = 1;

// Variant indices of the one-lane shared-memory kernels (k <= 64, k <= 128),
// and their forms that hand queries meeting a list with a box tree over to
// the one-warp kernel (a plan's requests on clouds with trees).
constexpr int kSmemVariant = 12;
constexpr int kSmemVariant128 = 15;
constexpr int kHandoverVariant = 22;
constexpr int kHandoverVariant128 = 23;
inline bool is_smem_variant(int v) {
  return v == kSmemVariant || v == kSmemVariant128 || v == kHandoverVariant ||
         v == kHandoverVariant128;
}
inline bool is_smem128_variant(int v) { return v == kSmemVariant128 || v == kHandoverVariant128; }
// Variant indices of the one-warp-per-query kernels with the list in shared
// memory: kWarpVariant32 + 0, 1, 2 for k <= 32, 64, 128.
constexpr int kWarpVariant32 = 16;
// The same three for clouds with box trees over their long lists (the
// walk's code would slow the scan of clouds without them):
// kTreeVariant32 + 0, 1, 2.
constexpr int kTreeVariant32 = 19;
// The variant a request runs: a one-warp variant turns into its tree form
// when the request's cloud has trees, and with `handover` (plans, not the
// server's packs) a one-lane variant into its hand-over form. variant_index
// never returns these forms (it picks the first of equal variants).
inline int with_trees(int v, bool trees, bool handover = false) {
  if (!trees) return v;
  if (v >= kWarpVariant32 && v < kWarpVariant32 + 3) return v + (kTreeVariant32 - kWarpVariant32);
  if (handover && v == kSmemVariant) return kHandoverVariant;
  if (handover && v == kSmemVariant128) return kHandoverVariant128;
  return v;
}

// Lanes per query and where the candidate list lives (2 = shared memory,
// 1 = registers).
struct Mode {
  int lanes = 0, placement = 0;
};

// Shape of one persistent launch: one kernel variant over a queue of items.
struct BatchLaunch {
  int grid = 1, threads = 256;
  size_t smem = 0;    // dynamic shared memory for the one-lane candidate lists
  int kcap = 0;       // list capacity: the largest k among the launch's requests
  int variant = kSmemVariant;
};
// Grid, block and shared memory for `nitems` items of one variant.
BatchLaunch batch_config(int nitems, int blocks_per_sm, int kcap, int variant);
// Launches the persistent kernel of b.variant; *d_next must be zero on entry.
cudaError_t launch_batch_kernel(const ReqDev* d_reqs, const Item* d_items, int nitems, int* d_next,
                                const BatchLaunch& b, cudaStream_t s);

// The items of one variant: a contiguous range of the item array with its
// own queue counter and launch.
struct Segment {
  int begin = 0, count = 0;
  BatchLaunch launch;
};
// Reorders items by variant (the one-lane kernels' first, each variant's
// items in their given order) and returns one segment per variant present;
// req_k[r] is request r's k (a one-lane segment's list capacity is its
// largest k).
std::vector<Segment> make_segments(std::vector<Item>& items, int blocks_per_sm,
                                   const std::vector<int>& req_k);
// Launches every segment, segment i draining the queue counter d_next[i]
// (zero on entry). With one-lane and group segments both present in a
// launch of at most kSplitMaxQueries queries, the group segments run one
// after another on `aux`, forked from s and joined back, concurrently with
// the one-lane segments on s; otherwise all run on s in order. Two
// persistent launches that each size their grid for the whole GPU fill
// each other's tails in a small launch, and share the GPU worse than they
// run in turn in a large one: the 64-cloud batching plan (57.6M queries)
// took 224 ms in turn against 234 ms on two streams, while the serving
// loop (packs of at most 2^17 queries) saturated at 6,510 requests/s on
// two streams against 5,717 in turn.
constexpr int64_t kSplitMaxQueries = int64_t(1) << 21;
cudaError_t launch_segments(const ReqDev* d_reqs, const Item* d_items, int* d_next,
                            const std::vector<Segment>& segs, cudaStream_t s, cudaStream_t aux,
                            cudaEvent_t fork, cudaEvent_t join, int64_t queries);

// Mode recorded by the tuner for (k, n, hub), lanes 0 if none. The tuning
// table is keyed by k, floor(log2 n) and the cloud's hub bucket
// (floor(log2(1 + longest successor list))).
Mode tuned_mode(int k, int64_t n, int hub);
void set_tuned_mode(int k, int64_t n, int hub, Mode m);
// Mode for a launch of nq queries: the tuned (or default) lanes for
// (k, n, hub), widened for batches too small to fill the GPU one query per
// thread, and the tuned placement (or the default for those lanes).
// trees: the cloud has box trees and the launch can use them (the one-warp
// kernel walks them; one lane hands queries that meet them over to it):
// then one lane is the default for small k when the launch stays one lane
// wide, and a launch widened for its size goes to 32 lanes.
Mode choose_mode(int k, int64_t n, int hub, int64_t nq, bool trees = false);
// The smallest lane width that fills the GPU with nq queries of this k.
int fill_lanes(int64_t nq, int k);

}  // namespace mknn
