// mknn_knn_noalloc: the query entry point (locality sort + k-NN kernel)
// for callers that must not allocate device memory during a call.
//
// Some callers cannot call cudaMalloc at query time: a process whose
// memory pool has already claimed the device memory it is allowed to use
// (an allocation would fail), or a latency-bound loop that cannot afford
// the device-wide synchronisation cudaMalloc and cudaFree may imply. For
// them, the scratch the locality sort needs (a histogram of cells, the
// cell of each query and the processing order) lives in one fixed
// file-scope device array instead of a library or caller allocation.
//
// The array is kScratchBytes (9 MiB + 1.75 KiB) and holds up to
// kMaxQueries = 2^20 queries per call. Every GPU that loads this library
// keeps it until the process exits. All calls on a device share it, so
// calls whose work overlaps on the GPU (different streams, or different
// host threads) race on it; serialise them. The histogram is cleared at
// the start of every call; the other parts are fully overwritten before
// they are read, so no state from an earlier call is used.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/mknn.h"
#include "batch.h"
#include "cloud.h"
#include "knn_kernels.h"

namespace mknn {
namespace {

constexpr int64_t kMaxQueries = int64_t(1) << 20;
constexpr size_t kHistBytes = kSortHistBytes;  // histogram, tile totals, box: 1 MiB + 1.25 KiB
constexpr size_t kScratchBytes = kHistBytes + 2 * (size_t)kMaxQueries * 4 + 512;
// [histogram + tile totals | cells] [order] for kMaxQueries queries must fit
static_assert(kSortHistBytes + 2 * (((size_t)kMaxQueries * 4 + 255) & ~(size_t)255) <=
                  kScratchBytes,
              "fixed scratch array too small for kMaxQueries");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of g_noalloc_scratch per device, found once per device
// (with that device current) by cudaGetSymbolAddress. In host code the
// array's name is only a host-side stand-in, never a device address.
std::mutex g_mu;
void* g_addr[64] = {};

cudaError_t scratch_address(int dev, void** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace
}  // namespace mknn

using namespace mknn;

extern "C" int64_t mknn_knn_noalloc_max_queries(void) { return kMaxQueries; }

extern "C" mknn_status mknn_knn_noalloc(const mknn_cloud* c, const float* q, int64_t nq,
                                        int32_t q_stride, int32_t k, const int32_t* m,
                                        int32_t m_scalar, int32_t* out_idx, float* out_d2,
                                        mknn_stream_t stream) {
  if (!c) {
    set_error("cloud is NULL");
    return MKNN_EINVAL;
  }
  if (!c->d_pts) {
    set_error("cloud is not uploaded (call mknn_cloud_upload)");
    return MKNN_EINVAL;
  }
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    set_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    return MKNN_ECUDA;
  }
  if (dev != c->device || dev < 0 || dev >= 64) {
    set_error("the cloud does not live on the current device");
    return MKNN_EINVAL;
  }
  if (nq < 0 || nq > kMaxQueries) {
    set_error("nq out of range for mknn_knn_noalloc: at most " + std::to_string(kMaxQueries) +
              " queries per call (the size of its fixed scratch array)");
    return MKNN_EINVAL;
  }
  if (q_stride < 3) {
    set_error("q_stride must be >= 3");
    return MKNN_EINVAL;
  }
  if (k < 1 || k > MKNN_MAX_K) {
    set_error("k must be in [1, 128]");
    return MKNN_EINVAL;
  }
  if (!m) {
    if (m_scalar == 0) m_scalar = (int32_t)c->n;
    if (m_scalar < 1 || m_scalar > c->n) {
      set_error("m_scalar must be in [1, n]");
      return MKNN_EINVAL;
    }
  }
  if (nq == 0) return MKNN_OK;
  if (!q || !out_idx || !out_d2) {
    set_error("NULL device pointer");
    return MKNN_EINVAL;
  }
  void* base = nullptr;
  if ((e = scratch_address(dev, &base)) != cudaSuccess) {
    set_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    return MKNN_ECUDA;
  }
  // the kernel variant mknn_knn would take for this cloud and batch size
  const Mode mode = choose_mode(k, c->n, c->hub_bucket(), nq);
  const int lanes = mode.lanes;
  if (k > plain_max_k(lanes)) {
    set_error("k above what the chosen lane width holds");
    return MKNN_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const mknn::CloudDevHost cd = c->dev();
  // layout: [histogram + cells (sort scratch)] [processing order]; small
  // batches skip the locality sort, as mknn_knn does
  int32_t* perm = nullptr;
  if (nq >= kSortMinQueries) {
    const size_t sort_bytes = sort_workspace_bytes(nq);
    perm = (int32_t*)((char*)base + align256(sort_bytes));
    if ((e = launch_query_sort(cd, q, q_stride, nq, base, perm, s)) != cudaSuccess) {
      set_error(std::string("query sort launch: ") + cudaGetErrorString(e));
      return MKNN_ECUDA;
    }
  }
  PlainLaunch L;
  L.q = q;
  L.q_stride = q_stride;
  L.nq = nq;
  L.k = k;
  L.m = m;
  L.m_scalar = m_scalar;
  L.perm = perm;
  L.out_idx = out_idx;
  L.out_d2 = out_d2;
  L.counters = nullptr;
  L.err = c->d_err;
  L.lanes = lanes;
  L.placement = mode.placement;
  L.blocks_per_sm = 0;
  if ((e = launch_knn_plain(cd, L, s)) != cudaSuccess) {
    set_error(std::string("knn kernel launch: ") + cudaGetErrorString(e));
    return MKNN_ECUDA;
  }
  return MKNN_OK;
}
