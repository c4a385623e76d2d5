// Read-bandwidth probe (diagnostic): every thread streams 16-byte loads
// over the buffer, grid-stride, `passes` times, and folds what it read into
// one XOR so the loads cannot be dropped. On a buffer smaller than L2 the
// passes after the first are served by L2: bytes * passes / time is then
// the L2 read bandwidth the query kernels' roofline is set against.
#include <cuda_runtime.h>

#include "../../include/mknn.h"
#include "cloud.h"
#include "knn_kernels.h"

namespace mknn {
namespace {

__global__ void __launch_bounds__(512) read_probe_kernel(const uint4* __restrict__ buf, int64_t n16,
                                                         int passes, uint32_t* __restrict__ sink) {
  uint32_t acc = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int p = 0; p < passes; ++p) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride) {
      const uint4 v = __ldcg(buf + i);  // L2, not L1: the probe measures L2 (or HBM)
      acc ^= v.x ^ v.y ^ v.z ^ v.w;
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc ^= __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31u) == 0) atomicXor(sink, acc);
}

}  // namespace
}  // namespace mknn

extern "C" mknn_status mknn_read_probe(const void* buf, size_t bytes, int32_t passes,
                                       uint32_t* sink, mknn_stream_t stream) {
  if (!buf || !sink || passes < 1 || bytes < 16 || (bytes & 15) || ((uintptr_t)buf & 15)) {
    mknn::set_error("mknn_read_probe: buf and sink non-NULL, buf 16-byte aligned, bytes a "
                    "non-zero multiple of 16, passes >= 1");
    return MKNN_EINVAL;
  }
  const int sms = mknn::num_sms();
  const int64_t n16 = (int64_t)(bytes / 16);
  int64_t blocks = (int64_t)sms * 4;
  if (blocks > (n16 + 511) / 512) blocks = (n16 + 511) / 512;
  mknn::read_probe_kernel<<<(unsigned)blocks, 512, 0, (cudaStream_t)stream>>>(
      (const uint4*)buf, n16, passes, sink);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    mknn::set_error(std::string("read probe launch: ") + cudaGetErrorString(e));
    return MKNN_ECUDA;
  }
  return MKNN_OK;
}
