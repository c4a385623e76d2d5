// mknn_knn_host: the query entry point on host buffers. Queries are cut
// into chunks; each chunk's upload, query and download run on one of two
// internal streams so that one chunk's copies overlap the other's kernels.
//
// Chunks of 2^20 queries: on the 4M-query torus (k = 16) the call took
// 10.68 ms with 2^19, 10.42 ms with 2^20 and 10.83 ms with 2^21 (a smaller
// chunk's queries are sparser, so neighbouring queries share fewer rows; a
// larger one leaves more of the last download exposed); one chunk for the
// whole batch took 12.0 ms (the 512 MB of results then come back at about
// 190 GB/s after the kernel, not during it), a third stream changed nothing,
// and writing the rows straight into pinned host memory from the kernel
// took 11.9 ms (scattered 64-byte rows over the host link).
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "../../include/mknn.h"
#include "cloud.h"

namespace mknn {
namespace {

constexpr int64_t kChunk = 1 << 20;

struct Slot {
  cudaStream_t s = nullptr;
  float* q = nullptr;
  int32_t* m = nullptr;
  int32_t* idx = nullptr;
  float* d2 = nullptr;
  void* ws = nullptr;
  size_t cap_q = 0, cap_m = 0, cap_idx = 0, cap_d2 = 0, cap_ws = 0;
};

struct DeviceState {
  Slot slot[2];
  bool init = false;
};

std::mutex g_mu;
DeviceState g_dev[64];

cudaError_t grow(void** p, size_t* cap, size_t need) {
  if (*cap >= need) return cudaSuccess;
  cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  cudaError_t e = cudaMalloc(p, need);
  if (e == cudaSuccess) *cap = need;
  return e;
}

}  // namespace
}  // namespace mknn

using namespace mknn;

extern "C" mknn_status mknn_knn_host(const mknn_cloud* c, const float* q, int64_t nq,
                                     int32_t q_stride, int32_t k, const int32_t* m,
                                     int32_t m_scalar, int32_t* out_idx, float* out_d2,
                                     mknn_stream_t stream) {
  if (!c) {
    set_error("cloud is NULL");
    return MKNN_EINVAL;
  }
  if (nq < 0 || q_stride < 3 || k < 1 || k > MKNN_MAX_K) {
    set_error("bad nq, q_stride or k");
    return MKNN_EINVAL;
  }
  if (nq == 0) return MKNN_OK;
  if (!q || !out_idx || !out_d2) {
    set_error("NULL host pointer");
    return MKNN_EINVAL;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) {
    set_error("device index out of range");
    return MKNN_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  DeviceState& D = g_dev[dev];
  cudaError_t e = cudaSuccess;
  if (!D.init) {
    for (auto& sl : D.slot) {
      e = cudaStreamCreateWithFlags(&sl.s, cudaStreamNonBlocking);
      if (e != cudaSuccess) {
        set_error(std::string("stream creation: ") + cudaGetErrorString(e));
        return MKNN_ECUDA;
      }
    }
    D.init = true;
  }
  // work after anything already queued on the caller's stream
  cudaEvent_t ev;
  cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  cudaEventRecord(ev, (cudaStream_t)stream);
  for (auto& sl : D.slot) cudaStreamWaitEvent(sl.s, ev, 0);
  cudaEventDestroy(ev);

  const int64_t chunk = std::min<int64_t>(nq, kChunk);
  mknn_knn_opts opts{};
  const size_t ws_need = mknn_knn_workspace_size(chunk, &opts);
  for (auto& sl : D.slot) {
    if ((e = grow((void**)&sl.q, &sl.cap_q, (size_t)chunk * q_stride * 4)) != cudaSuccess ||
        (e = grow((void**)&sl.idx, &sl.cap_idx, (size_t)chunk * k * 4)) != cudaSuccess ||
        (e = grow((void**)&sl.d2, &sl.cap_d2, (size_t)chunk * k * 4)) != cudaSuccess ||
        (m && (e = grow((void**)&sl.m, &sl.cap_m, (size_t)chunk * 4)) != cudaSuccess) ||
        (e = grow((void**)&sl.ws, &sl.cap_ws, std::max<size_t>(ws_need, 256))) != cudaSuccess) {
      cudaGetLastError();
      set_error(std::string("device allocation: ") + cudaGetErrorString(e));
      return MKNN_ENOMEM;
    }
  }
  mknn_status st = MKNN_OK;
  for (int64_t c0 = 0, ci = 0; c0 < nq; c0 += chunk, ++ci) {
    Slot& sl = D.slot[ci & 1];
    const int64_t len = std::min(chunk, nq - c0);
    if ((e = cudaMemcpyAsync(sl.q, q + c0 * q_stride, (size_t)len * q_stride * 4,
                             cudaMemcpyHostToDevice, sl.s)) != cudaSuccess)
      break;
    if (m && (e = cudaMemcpyAsync(sl.m, m + c0, (size_t)len * 4, cudaMemcpyHostToDevice, sl.s)) !=
                 cudaSuccess)
      break;
    mknn_knn_opts o{};
    o.workspace = sl.ws;
    o.workspace_bytes = sl.cap_ws;
    st = mknn_knn_ex(c, sl.q, len, q_stride, k, m ? sl.m : nullptr, m_scalar, sl.idx, sl.d2, &o,
                     (mknn_stream_t)sl.s);
    if (st != MKNN_OK) break;
    if ((e = cudaMemcpyAsync(out_idx + c0 * k, sl.idx, (size_t)len * k * 4,
                             cudaMemcpyDeviceToHost, sl.s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(out_d2 + c0 * k, sl.d2, (size_t)len * k * 4,
                             cudaMemcpyDeviceToHost, sl.s)) != cudaSuccess)
      break;
  }
  cudaError_t e0 = cudaStreamSynchronize(D.slot[0].s);
  cudaError_t e1 = cudaStreamSynchronize(D.slot[1].s);
  if (st != MKNN_OK) return st;
  if (e == cudaSuccess) e = e0 != cudaSuccess ? e0 : e1;
  if (e != cudaSuccess) {
    set_error(std::string("host-buffer query: ") + cudaGetErrorString(e));
    return MKNN_ECUDA;
  }
  return MKNN_OK;
}
