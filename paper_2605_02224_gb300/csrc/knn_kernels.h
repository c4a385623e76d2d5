// Host-side interface of the query kernels (internal to the library).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mknn {

struct CloudDevHost {
  const void* pts;       // float4[n]
  const int32_t* rowp;   // [n+1]
  const int32_t* succ;   // [E]
  int32_t n;
  float lo[3], hi[3];    // bounding box of the sites (query sort)
};

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
  int lanes;             // 4, 8, 16, 32
  int blocks_per_sm;     // 0 = occupancy limit
};

// Launches the plain (one cloud) query kernel. Returns a CUDA error code.
cudaError_t launch_knn_plain(const CloudDevHost& c, const PlainLaunch& L, cudaStream_t stream);

// Query locality sort: a counting sort of queries by the Morton index of
// their cell in a 64^3 grid over the cloud's bounding box.
constexpr int kSortBits = 6;
constexpr int kSortCells = 1 << (3 * kSortBits);
// Scratch for the histogram and per-query cells (perm not included).
size_t sort_workspace_bytes(int64_t nq);
// Writes perm[nq] (processing order).
cudaError_t launch_query_sort(const CloudDevHost& c, const float* q, int32_t q_stride, int64_t nq,
                              void* workspace, int32_t* perm, cudaStream_t stream);

int default_lanes(int k);
int num_sms();

}  // namespace mknn
