// Host-side interface of the query kernels (internal to the library).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mknn {

struct CloudDevHost {
  const void* pts;       // float4[n]
  const int2* rows;      // [n]: (first, end) of each successor row in succ / ent
  const int32_t* succ;   // [E]
  int32_t n;
  float lo[3], hi[3];    // bounding box of the sites (query sort)
  const void* ent;       // float4[E]: succ[e]'s (x, y, z) and its rank's bits in w
  // box trees over the long lists (hub_index.h), all NULL when there are none
  const int32_t* hub_of = nullptr;  // [n]: the tree of site i's list, or -1
  const void* hub_desc = nullptr;   // int4 per tree
  const void* hub_ent = nullptr;    // float4 per entry, chunks of 32
  const void* hub_node = nullptr;   // two float4 per node
};

// Same-manifold queries: q[i] = pts[sites[i]] and m_out[i] = the query's
// prefix bound (m[i], or m_scalar when m is NULL), or 0 - which the query
// kernels turn into a padded row and the error flag - when sites[i] is not
// a rank of the cloud.
cudaError_t launch_gather_sites(const CloudDevHost& c, const int32_t* sites, int64_t nq,
                                const int32_t* m, int32_t m_scalar, float4* q, int32_t* m_out,
                                cudaStream_t stream);

// Fills ent[e] = (pts[succ[e]].xyz, rank bits of succ[e]) for e < E.
cudaError_t launch_fill_entries(const void* pts, const int32_t* succ, int64_t E, void* ent,
                                cudaStream_t stream);

struct PlainLaunch {
  const float* q;
  int32_t q_stride;
  int64_t nq;
  int32_t k;
  const int32_t* m;      // per-query or NULL
  int32_t m_scalar;      // used when m is NULL (already resolved: 1..n)
  const int32_t* perm;   // processing order or NULL
  int32_t* out_idx;
  float* out_d2;
  int32_t* counters;     // [4*nq] or NULL
  int32_t* err;          // device error word
  int lanes;             // 1, 4, 8, 16, 32
  int blocks_per_sm;     // 0 = occupancy limit
  // lanes == 1: 1 = registers per thread, 2 = shared-memory list per thread;
  // lanes == 32: 1 = registers spread over the warp, 2 = shared-memory list
  // per warp; ignored for 4, 8, 16 lanes (registers)
  int placement = 1;
  // one lane, shared memory, on a cloud with box trees: device scratch of
  // defer_bytes(nq) for the queries handed to the one-warp kernel (a count,
  // then their indices from kDeferHead on); NULL = no hand-over
  int32_t* defer = nullptr;
  // device count of queries (at most nq) the launch answers, or NULL
  const int32_t* count = nullptr;
};
// The deferred queries' indices start this many int32 into the scratch.
constexpr int kDeferHead = 64;
inline size_t defer_bytes(int64_t nq) {
  return (((size_t)nq + kDeferHead) * 4 + 255) & ~(size_t)255;
}

// Launches the plain (one cloud) query kernel. Returns a CUDA error code.
cudaError_t launch_knn_plain(const CloudDevHost& c, const PlainLaunch& L, cudaStream_t stream);

// Query locality sort: a counting sort of queries by the Morton index of
// their cell in a 64^3 grid over the cloud's bounding box.
constexpr int kSortBits = 6;
constexpr int kSortCells = 1 << (3 * kSortBits);
constexpr int kSortTile = 1024;                       // cells per scan block
constexpr int kSortTiles = kSortCells / kSortTile;    // 256
// histogram + tile totals + the queries' bounding box, each 256-byte aligned
// (the start of a sort workspace)
constexpr size_t kSortHistBytes = (((size_t)kSortCells * 4 + 255) & ~(size_t)255) +
                                  (((size_t)kSortTiles * 4 + 255) & ~(size_t)255) + 256;
// Batches smaller than this skip the locality sort by default (its five
// launches and histogram clear cost more than the order saves).
constexpr int64_t kSortMinQueries = 4096;
// Scratch for the histogram and per-query cells (perm not included).
size_t sort_workspace_bytes(int64_t nq);
// Writes perm[nq] (processing order).
cudaError_t launch_query_sort(const CloudDevHost& c, const float* q, int32_t q_stride, int64_t nq,
                              void* workspace, int32_t* perm, cudaStream_t stream);
// Same, with the histogram (kSortCells int32, cleared here) and the
// per-query cells (nq int32) in separate buffers.
cudaError_t launch_query_sort_split(const CloudDevHost& c, const float* q, int32_t q_stride,
                                    int64_t nq, void* hist, int32_t* cell, int32_t* perm,
                                    cudaStream_t stream);

// From this k up, one warp per query (its list in shared memory) is the
// default instead of one thread per query.
constexpr int kWarpMinK = 48;
int default_lanes(int k);
// 2 (shared memory) for 1 and 32 lanes, 1 (registers) for 4, 8, 16.
int default_placement(int k, int lanes);
// Largest k the plain kernels hold with this many lanes per query.
int plain_max_k(int lanes);
// The current device's ordinal (-1 if it cannot be read) and its SM count
// (cached per device).
int current_device();
int num_sms();

}  // namespace mknn
