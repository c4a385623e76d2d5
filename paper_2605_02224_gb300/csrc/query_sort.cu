// Query locality sort (counting sort by cell in a 64^3 grid over the
// queries' own bounding box, cells in Morton order). Queries that land in
// the same or neighbouring cells are then processed by neighbouring lanes,
// warps and blocks, so the successor rows and coordinates they share are
// found in L1 and L2. The sort only changes the processing order: each
// query's result goes to its own row.
#include "knn_kernels.h"

namespace mknn {

namespace {

__device__ __forceinline__ uint32_t spread3(uint32_t v) {  // 6 bits -> every third bit
  uint32_t x = v & 0x3fu;
  x = (x | (x << 8)) & 0x0000f00fu;
  x = (x | (x << 4)) & 0x000c30c3u;
  x = (x | (x << 2)) & 0x00249249u;
  return x;
}

// Float <-> unsigned with the same order (for atomic min / max of floats).
__device__ __forceinline__ uint32_t float_order(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float order_float(uint32_t u) {
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// Bounding box of the queries (NaN coordinates skipped) into box[0..5]:
// minima then maxima in float_order form (set to all-ones / zero first).
__global__ void qsort_bbox(const float* __restrict__ q, int stride, int64_t nq,
                           uint32_t* __restrict__ box) {
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nq; i += step) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const float v = __ldg(q + i * stride + d);
      if (v == v) {
        lo[d] = fminf(lo[d], v);
        hi[d] = fmaxf(hi[d], v);
      }
    }
  }
#pragma unroll
  for (int d = 0; d < 3; ++d)
    for (int o = 16; o > 0; o >>= 1) {
      lo[d] = fminf(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
      hi[d] = fmaxf(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
    }
  // one set of atomics per block, not per warp
  __shared__ float part[32][6];
  const int warp = (int)(threadIdx.x >> 5), nwarps = (int)(blockDim.x >> 5);
  if ((threadIdx.x & 31u) == 0)
    for (int d = 0; d < 3; ++d) {
      part[warp][d] = lo[d];
      part[warp][3 + d] = hi[d];
    }
  __syncthreads();
  if (threadIdx.x < 3) {
    const int d = (int)threadIdx.x;
    float a = part[0][d], b = part[0][3 + d];
    for (int w = 1; w < nwarps; ++w) {
      a = fminf(a, part[w][d]);
      b = fmaxf(b, part[w][3 + d]);
    }
    atomicMin(box + d, float_order(a));
    atomicMax(box + 3 + d, float_order(b));
  }
}

__global__ void qsort_hist(const float* __restrict__ q, int stride, int64_t nq,
                           const uint32_t* __restrict__ box, int32_t* __restrict__ cell,
                           int32_t* __restrict__ hist) {
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  const float cmax = (float)((1 << kSortBits) - 1);
  float lo[3], sc[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    lo[d] = order_float(box[d]);
    const float ext = order_float(box[3 + d]) - lo[d];
    sc[d] = ext > 0.f ? (float)(1 << kSortBits) / ext : 0.f;
  }
  const float lox = lo[0], loy = lo[1], loz = lo[2], sx = sc[0], sy = sc[1], sz = sc[2];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nq; i += step) {
    const float* p = q + i * stride;
    const float fx = fminf(fmaxf((__ldg(p) - lox) * sx, 0.f), cmax);
    const float fy = fminf(fmaxf((__ldg(p + 1) - loy) * sy, 0.f), cmax);
    const float fz = fminf(fmaxf((__ldg(p + 2) - loz) * sz, 0.f), cmax);
    // a NaN coordinate maps to cell 0 (fminf/fmaxf drop NaN operands)
    const uint32_t c = spread3((uint32_t)fx) | (spread3((uint32_t)fy) << 1) |
                       (spread3((uint32_t)fz) << 2);
    cell[i] = (int32_t)c;
    atomicAdd(hist + c, 1);
  }
}

// Exclusive scan of the cell counts, two levels. Level 1: one block per
// tile of kSortTile cells scans its tile in place (coalesced) and writes
// the tile total. Level 2: one block scans the kSortTiles totals in place.
// The scatter adds a cell's in-tile offset to its tile's offset.
__device__ __forceinline__ int32_t block_exclusive_scan(int32_t v, int32_t* warp_sums,
                                                        int32_t* total) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nwarps = blockDim.x >> 5;
  int32_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t u = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += u;
  }
  if (lane == 31) warp_sums[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int32_t w = lane < nwarps ? warp_sums[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t u = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += u;
    }
    if (lane < nwarps) warp_sums[lane] = w;
  }
  __syncthreads();
  *total = warp_sums[nwarps - 1];
  return x - v + (warp > 0 ? warp_sums[warp - 1] : 0);
}

__global__ void __launch_bounds__(kSortTile) qsort_scan_tiles(int32_t* __restrict__ hist,
                                                              int32_t* __restrict__ tiles) {
  __shared__ int32_t warp_sums[32];
  const int64_t i = (int64_t)blockIdx.x * kSortTile + threadIdx.x;
  int32_t total = 0;
  const int32_t ex = block_exclusive_scan(hist[i], warp_sums, &total);
  hist[i] = ex;
  if (threadIdx.x == 0) tiles[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kSortTiles) qsort_scan_top(int32_t* __restrict__ tiles) {
  __shared__ int32_t warp_sums[32];
  int32_t total = 0;
  tiles[threadIdx.x] = block_exclusive_scan(tiles[threadIdx.x], warp_sums, &total);
}

__global__ void qsort_scatter(const int32_t* __restrict__ cell, int64_t nq,
                              int32_t* __restrict__ offs, const int32_t* __restrict__ tiles,
                              int32_t* __restrict__ perm) {
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nq; i += step) {
    const int32_t c = cell[i];
    const int32_t pos = atomicAdd(offs + c, 1) + __ldg(tiles + (c / kSortTile));
    perm[pos] = (int32_t)i;
  }
}

inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

size_t sort_workspace_bytes(int64_t nq) { return kSortHistBytes + align256((size_t)nq * 4); }

cudaError_t launch_query_sort(const CloudDevHost& c, const float* q, int32_t q_stride, int64_t nq,
                              void* workspace, int32_t* perm, cudaStream_t stream) {
  char* w = (char*)workspace;
  int32_t* cell = (int32_t*)(w + kSortHistBytes);
  return launch_query_sort_split(c, q, q_stride, nq, workspace, cell, perm, stream);
}

cudaError_t launch_query_sort_split(const CloudDevHost& c, const float* q, int32_t q_stride,
                                    int64_t nq, void* hist_buf, int32_t* cell, int32_t* perm,
                                    cudaStream_t stream) {
  (void)c;  // the grid spans the queries' own bounding box
  int32_t* hist = (int32_t*)hist_buf;
  int32_t* tiles = (int32_t*)((char*)hist_buf + align256((size_t)kSortCells * 4));
  uint32_t* box = (uint32_t*)((char*)tiles + align256((size_t)kSortTiles * 4));
  if (nq == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(hist, 0, (size_t)kSortCells * 4, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(box, 0xff, 12, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(box + 3, 0, 12, stream);
  if (e != cudaSuccess) return e;
  const int threads = 256;
  int64_t blocks = (nq + threads - 1) / threads;
  const int64_t cap = (int64_t)num_sms() * 8;
  if (blocks > cap) blocks = cap;
  qsort_bbox<<<(unsigned)blocks, threads, 0, stream>>>(q, q_stride, nq, box);
  qsort_hist<<<(unsigned)blocks, threads, 0, stream>>>(q, q_stride, nq, box, cell, hist);
  qsort_scan_tiles<<<kSortTiles, kSortTile, 0, stream>>>(hist, tiles);
  qsort_scan_top<<<1, kSortTiles, 0, stream>>>(tiles);
  qsort_scatter<<<(unsigned)blocks, threads, 0, stream>>>(cell, nq, hist, tiles, perm);
  return cudaGetLastError();
}

}  // namespace mknn
