// The plain query kernel: one cloud, a batch of queries, one group of G
// lanes per query, grid-stride over the (optionally locality-sorted)
// query order. Sized to the SM count times the resident blocks per SM.
#include "knn_device.cuh"
#include "knn_kernels.h"
#include "per_device.h"

namespace mknn {

namespace {

constexpr int kThreads = 256;

template <int G, int S, bool COUNT>
__global__ void __launch_bounds__(kThreads) knn_plain_kernel(
    CloudDev C, const float* __restrict__ q, int q_stride, int64_t nq, int k,
    const int32_t* __restrict__ mq, int m_scalar, const int32_t* __restrict__ perm,
    int32_t* __restrict__ out_idx, float* __restrict__ out_d2, int32_t* __restrict__ counters,
    int32_t* __restrict__ err) {
  const Grp<G> g;
  const int64_t gid = ((int64_t)blockIdx.x * kThreads + threadIdx.x) / G;
  const int64_t ngroups = ((int64_t)gridDim.x * kThreads) / G;
  for (int64_t i = gid; i < nq; i += ngroups) {
    const int64_t qi = perm ? (int64_t)__ldg(perm + i) : i;
    const float* qp = q + qi * q_stride;
    const float qx = __ldg(qp), qy = __ldg(qp + 1), qz = __ldg(qp + 2);
    const int m = mq ? __ldg(mq + qi) : m_scalar;
    if (m < 1 || m > C.n) {
      pad_row(g, k, out_idx + qi * k, out_d2 + qi * k);
      if (g.lane == 0) atomicOr(err, 1);
      continue;
    }
    QueryCounters qc{0, 0, 0, 0};
    knn_query<G, S, COUNT>(C, g, qx, qy, qz, k, m, out_idx, out_d2, (int32_t)qi, qc);
    if (COUNT && g.lane == 0) {
      int32_t* c = counters + 4 * qi;
      c[0] = qc.rows;
      c[1] = qc.entries;
      c[2] = qc.coords;
      c[3] = qc.trans;
    }
  }
}

// One query per thread.
template <int K, bool COUNT>
__global__ void __launch_bounds__(kThreads) knn_plain_thread_kernel(
    CloudDev C, const float* __restrict__ q, int q_stride, int64_t nq, int k,
    const int32_t* __restrict__ mq, int m_scalar, const int32_t* __restrict__ perm,
    int32_t* __restrict__ out_idx, float* __restrict__ out_d2, int32_t* __restrict__ counters,
    int32_t* __restrict__ err) {
  const int64_t stride = (int64_t)gridDim.x * kThreads;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < nq; i += stride) {
    const int64_t qi = perm ? (int64_t)__ldg(perm + i) : i;
    const float* qp = q + qi * q_stride;
    const float qx = __ldg(qp), qy = __ldg(qp + 1), qz = __ldg(qp + 2);
    const int m = mq ? __ldg(mq + qi) : m_scalar;
    int32_t* oi = out_idx + qi * k;
    float* od = out_d2 + qi * k;
    if (m < 1 || m > C.n) {
      for (int p = 0; p < k; ++p) {
        oi[p] = -1;
        od[p] = __int_as_float(0x7f800000);
      }
      atomicOr(err, 1);
      continue;
    }
    QueryCounters qc{0, 0, 0, 0};
    knn_query_thread<K, COUNT>(C, qx, qy, qz, k, m, oi, od, qc);
    if (COUNT) {
      int32_t* c = counters + 4 * qi;
      c[0] = qc.rows;
      c[1] = qc.entries;
      c[2] = qc.coords;
      c[3] = qc.trans;
    }
  }
}

template <int K, bool COUNT>
cudaError_t run_thread(const CloudDevHost& c, const PlainLaunch& L, cudaStream_t stream) {
  static PerDevice<int> occ_of;
  int occ = 0;
  const cudaError_t oe = occ_of.with(current_device(), cudaErrorInvalidDevice, [&](int& o) {
    if (o < 1) {
      cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &o, knn_plain_thread_kernel<K, COUNT>, kThreads, 0);
      if (e != cudaSuccess) {
        o = 0;
        return e;
      }
      if (o < 1) o = 1;
    }
    occ = o;
    return cudaSuccess;
  });
  if (oe != cudaSuccess) return oe;
  const int per_sm = L.blocks_per_sm > 0 ? std::min(L.blocks_per_sm, occ) : occ;
  const int64_t need = (L.nq + kThreads - 1) / kThreads;
  int64_t blocks = (int64_t)num_sms() * per_sm;
  if (need < blocks) blocks = need;
  if (blocks < 1) blocks = 1;
  CloudDev C{(const float4*)c.pts, c.rows, c.succ, c.n, (const float4*)c.ent};
  knn_plain_thread_kernel<K, COUNT><<<(unsigned)blocks, kThreads, 0, stream>>>(
      C, L.q, L.q_stride, L.nq, L.k, L.m, L.m_scalar, L.perm, L.out_idx, L.out_d2, L.counters,
      L.err);
  return cudaGetLastError();
}

// One query per thread, candidate lists in shared memory (kcap =
// list_slots(k) entries per thread, a warp's lists interleaved: thread l of
// warp w owns column l of the warp's [kcap][32] keys). 256-thread blocks are
// held to 48 registers (five blocks per SM, no spills): left alone the
// compiler picks either 40 registers with spills or 64, both measured
// 5%-20% slower, and 4 or 6 blocks per SM were slower too.
// LK: the list kind (8: SortedList of 8 slots, k <= 8; 16: PermList16,
// 9 <= k <= 16; 0: SortedList of k slots searched over 32 W). DEFER (a
// cloud with box trees): a query that gives up (knn_query_smem) is appended
// to defer[0 .. *ndefer) for the one-warp kernel.
template <int THREADS, int W, int LK, bool DEFER>
__global__ void __launch_bounds__(THREADS, THREADS == 256 ? 5 : 1) knn_plain_smem_kernel(
    CloudDev C, const float* __restrict__ q, int q_stride, int64_t nq, int k, int kcap,
    const int32_t* __restrict__ mq, int m_scalar, const int32_t* __restrict__ perm,
    int32_t* __restrict__ out_idx, float* __restrict__ out_d2, int32_t* __restrict__ err,
    int32_t* __restrict__ defer, int32_t* __restrict__ ndefer) {
  extern __shared__ uint64_t smem_lists[];
  const int warp = (int)(threadIdx.x >> 5), lane = (int)(threadIdx.x & 31u);
  uint64_t* col = smem_lists + (size_t)warp * kcap * 32 + lane;
  // 32-bit query indices keep registers free for residency; unsigned, so
  // that i + stride cannot overflow (nq < 2^31 - 1, stride < 2^31).
  // The lanes of a warp take adjacent queries of the locality order and
  // start their next ones together: a lane done early waits at the inner
  // loop's exit. Letting it start its next query at once, in one flat loop
  // over queries and entries, was measured 0.64x as fast (strided queries)
  // and 0.55x (the warp's lanes taking one contiguous range in order): the
  // lanes then sit at different steps of the method, and each iteration
  // runs the descent, expansion and output paths one after another.
  const uint32_t n32 = (uint32_t)nq;
  for (uint32_t i = blockIdx.x * THREADS + threadIdx.x; i < n32; i += gridDim.x * THREADS) {
    // queries and their order are read once: streaming loads
    const int32_t qi = perm ? __ldcs(perm + i) : (int32_t)i;
    const float* qp = q + (int64_t)qi * q_stride;
    const float qx = __ldcs(qp), qy = __ldcs(qp + 1), qz = __ldcs(qp + 2);
    const int m = mq ? __ldg(mq + qi) : m_scalar;
    if (m < 1 || m > C.n) {
      for (int p = 0; p < k; ++p) {
        out_idx[(int64_t)qi * k + p] = -1;
        out_d2[(int64_t)qi * k + p] = __int_as_float(0x7f800000);
      }
      atomicOr(err, 1);
      continue;
    }
    bool done;
    if constexpr (LK == 8)
      done = knn_query_smem<SortedList<8, 1, true>, DEFER>(C, qx, qy, qz, k, m, col, 8, out_idx,
                                                            out_d2, qi);
    else if constexpr (LK == 16)
      done = knn_query_smem<PermList16, DEFER>(C, qx, qy, qz, k, m, col, 16, out_idx, out_d2, qi);
    else
      done = knn_query_smem<SortedList<32 * W, W, false>, DEFER>(C, qx, qy, qz, k, m, col, k,
                                                                 out_idx, out_d2, qi);
    if constexpr (DEFER) {
      if (!done) defer[atomicAdd(ndefer, 1)] = qi;
    }
  }
}

// Shared memory per block for kcap entries per thread.
template <int THREADS>
constexpr size_t smem_bytes(int kcap) {
  return (size_t)THREADS * (size_t)kcap * 8;
}

template <int THREADS, int KMAX, int LK, bool DEFER>
cudaError_t run_smem(const CloudDevHost& c, const PlainLaunch& L, cudaStream_t stream) {
  constexpr int W = KMAX / 32;  // 32-bit words of expanded flags
  const int kcap = list_slots(L.k);
  const size_t smem = smem_bytes<THREADS>(kcap);
  // per device: the raised shared-memory limit and the occupancy per kcap
  struct State {
    bool attr;
    int occ_for[KMAX + 1];
  };
  static PerDevice<State> state;
  int occ = 0;
  const cudaError_t se = state.with(current_device(), cudaErrorInvalidDevice, [&](State& st) {
    if (!st.attr) {
      // once per device, at the largest size any k <= KMAX needs
      cudaError_t e = cudaFuncSetAttribute(knn_plain_smem_kernel<THREADS, W, LK, DEFER>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem_bytes<THREADS>(KMAX));
      if (e != cudaSuccess) return e;
      st.attr = true;
    }
    if (!st.occ_for[kcap]) {
      int o = 0;
      cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &o, knn_plain_smem_kernel<THREADS, W, LK, DEFER>, THREADS, smem);
      if (e != cudaSuccess) return e;
      st.occ_for[kcap] = o < 1 ? 1 : o;
    }
    occ = st.occ_for[kcap];
    return cudaSuccess;
  });
  if (se != cudaSuccess) return se;
  // By default one block per THREADS queries: the block scheduler starts a
  // new block wherever one ends, so every SM stays full to the end of the
  // launch. blocks_per_sm > 0 makes the grid persistent instead (that many
  // resident blocks per SM, each thread looping over queries).
  const int64_t need = (L.nq + THREADS - 1) / THREADS;
  int64_t blocks = need;
  if (L.blocks_per_sm > 0) {
    const int64_t cap = (int64_t)num_sms() * std::min(L.blocks_per_sm, occ);
    if (cap < blocks) blocks = cap;
  }
  if (blocks < 1) blocks = 1;
  CloudDev C{(const float4*)c.pts, c.rows, c.succ, c.n, (const float4*)c.ent, c.hub_of};
  knn_plain_smem_kernel<THREADS, W, LK, DEFER><<<(unsigned)blocks, THREADS, smem, stream>>>(
      C, L.q, L.q_stride, L.nq, L.k, kcap, L.m, L.m_scalar, L.perm, L.out_idx, L.out_d2, L.err,
      DEFER ? L.defer + kDeferHead : nullptr, DEFER ? L.defer : nullptr);
  return cudaGetLastError();
}

// One warp per query, the candidate list in shared memory (KC keys per
// warp: 8 KB per 256-thread block at KC = 128). One block per 8 queries of
// the processing order, started by the hardware wherever a block ends.
template <int KC, bool TREES>
__global__ void __launch_bounds__(kThreads) knn_plain_warp_kernel(
    CloudDev C, const float* __restrict__ q, int q_stride, int64_t nq, int k,
    const int32_t* __restrict__ mq, int m_scalar, const int32_t* __restrict__ perm,
    int32_t* __restrict__ out_idx, float* __restrict__ out_d2, int32_t* __restrict__ err,
    const int32_t* __restrict__ count) {
  __shared__ uint64_t lists[kThreads / 32][TREES ? kWarpListWords(KC) : KC];
  if (count) nq = min(nq, (int64_t)__ldg(count));  // queries a deferring launch handed over
  const int warp = (int)(threadIdx.x >> 5), lane = (int)(threadIdx.x & 31u);
  const int64_t nw = (int64_t)gridDim.x * (kThreads / 32);
  for (int64_t i = (int64_t)blockIdx.x * (kThreads / 32) + warp; i < nq; i += nw) {
    const int64_t qi = perm ? (int64_t)__ldg(perm + i) : i;
    const float* qp = q + qi * q_stride;
    const float qx = __ldg(qp), qy = __ldg(qp + 1), qz = __ldg(qp + 2);
    const int m = mq ? __ldg(mq + qi) : m_scalar;
    if (m < 1 || m > C.n) {
      for (int p = lane; p < k; p += 32) {
        out_idx[qi * k + p] = -1;
        out_d2[qi * k + p] = __int_as_float(0x7f800000);
      }
      if (lane == 0) atomicOr(err, 1);
      continue;
    }
    knn_query_warp<KC, TREES>(C, qx, qy, qz, k, m, lists[warp], out_idx, out_d2, (int32_t)qi);
  }
}

template <int KC, bool TREES>
cudaError_t run_warp(const CloudDevHost& c, const PlainLaunch& L, cudaStream_t stream) {
  constexpr int kWarps = kThreads / 32;
  int64_t blocks = (L.nq + kWarps - 1) / kWarps;
  if (L.blocks_per_sm > 0) {
    static PerDevice<int> occ_of;
    int occ = 0;
    const cudaError_t oe = occ_of.with(current_device(), cudaErrorInvalidDevice, [&](int& o) {
      if (o < 1) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &o, knn_plain_warp_kernel<KC, TREES>, kThreads, 0);
        if (e != cudaSuccess) {
          o = 0;
          return e;
        }
        if (o < 1) o = 1;
      }
      occ = o;
      return cudaSuccess;
    });
    if (oe != cudaSuccess) return oe;
    blocks = std::min<int64_t>(blocks, (int64_t)num_sms() * std::min(L.blocks_per_sm, occ));
  }
  if (blocks < 1) blocks = 1;
  CloudDev C{(const float4*)c.pts, c.rows, c.succ, c.n, (const float4*)c.ent,
             c.hub_of,          (const int4*)c.hub_desc, (const float4*)c.hub_ent,
             (const float4*)c.hub_node};
  knn_plain_warp_kernel<KC, TREES><<<(unsigned)blocks, kThreads, 0, stream>>>(
      C, L.q, L.q_stride, L.nq, L.k, L.m, L.m_scalar, L.perm, L.out_idx, L.out_d2, L.err,
      L.count);
  return cudaGetLastError();
}

// One lane per query on a cloud with box trees: the queries that give up at
// a list with a tree (knn_query_smem's DEFER) are answered afterwards by the
// one-warp kernel, which walks the trees, over a persistent grid that reads
// their number from the device.
cudaError_t run_deferring(const CloudDevHost& c, const PlainLaunch& L, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(L.defer, 0, sizeof(int32_t), stream);
  if (e != cudaSuccess) return e;
  if (L.k <= 8)
    e = run_smem<256, 32, 8, true>(c, L, stream);
  else if (L.k <= 16)
    e = run_smem<256, 32, 16, true>(c, L, stream);
  else if (L.k <= 32)
    e = run_smem<256, 32, 0, true>(c, L, stream);
  else if (L.k <= 64)
    e = run_smem<128, 64, 0, true>(c, L, stream);
  else
    e = run_smem<64, 128, 0, true>(c, L, stream);
  if (e != cudaSuccess) return e;
  PlainLaunch D = L;
  D.perm = L.defer + kDeferHead;
  D.count = L.defer;
  D.defer = nullptr;
  D.lanes = 32;
  D.placement = 2;
  D.blocks_per_sm = 1 << 16;  // as many resident blocks as fit: a persistent grid
  if (L.k <= 32) return run_warp<32, true>(c, D, stream);
  if (L.k <= 64) return run_warp<64, true>(c, D, stream);
  return run_warp<128, true>(c, D, stream);
}

template <bool COUNT>
cudaError_t pick_thread(const CloudDevHost& c, const PlainLaunch& L, cudaStream_t stream) {
  if (!COUNT && L.placement == 2) {
    if (c.hub_of && L.defer) return run_deferring(c, L, stream);
    if (L.k <= 8) return run_smem<256, 32, 8, false>(c, L, stream);
    if (L.k <= 16) return run_smem<256, 32, 16, false>(c, L, stream);
    if (L.k <= 32) return run_smem<256, 32, 0, false>(c, L, stream);
    if (L.k <= 64) return run_smem<128, 64, 0, false>(c, L, stream);
    return run_smem<64, 128, 0, false>(c, L, stream);  // 64 KB of lists per block at k = 128
  }
  if (L.k > 64) return cudaErrorInvalidValue;  // register lists hold k <= 64
  if (L.k <= 8) return run_thread<8, COUNT>(c, L, stream);
  if (L.k <= 16) return run_thread<16, COUNT>(c, L, stream);
  if (L.k <= 32) return run_thread<32, COUNT>(c, L, stream);
  return run_thread<64, COUNT>(c, L, stream);
}

template <int G, int S, bool COUNT>
cudaError_t run(const CloudDevHost& c, const PlainLaunch& L, cudaStream_t stream) {
  static PerDevice<int> occ_of;
  int occ = 0;
  const cudaError_t oe = occ_of.with(current_device(), cudaErrorInvalidDevice, [&](int& o) {
    if (o < 1) {
      cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &o, knn_plain_kernel<G, S, COUNT>, kThreads, 0);
      if (e != cudaSuccess) {
        o = 0;
        return e;
      }
      if (o < 1) o = 1;
    }
    occ = o;
    return cudaSuccess;
  });
  if (oe != cudaSuccess) return oe;
  const int per_sm = L.blocks_per_sm > 0 ? std::min(L.blocks_per_sm, occ) : occ;
  const int64_t need = (L.nq * G + kThreads - 1) / kThreads;
  int64_t blocks = (int64_t)num_sms() * per_sm;
  if (need < blocks) blocks = need;
  if (blocks < 1) blocks = 1;
  CloudDev C{(const float4*)c.pts, c.rows, c.succ, c.n, (const float4*)c.ent};
  knn_plain_kernel<G, S, COUNT><<<(unsigned)blocks, kThreads, 0, stream>>>(
      C, L.q, L.q_stride, L.nq, L.k, L.m, L.m_scalar, L.perm, L.out_idx, L.out_d2, L.counters,
      L.err);
  return cudaGetLastError();
}

template <int G, bool COUNT>
cudaError_t pick_s(const CloudDevHost& c, const PlainLaunch& L, cudaStream_t stream) {
  const int need = (L.k + G - 1) / G;
  if (need <= 1) return run<G, 1, COUNT>(c, L, stream);
  if (need <= 2) return run<G, 2, COUNT>(c, L, stream);
  if constexpr (G == 32) {
    if (need <= 4) return run<G, 4, COUNT>(c, L, stream);  // k <= 128
  }
  if constexpr (G == 16) {
    if (need <= 8) return run<G, 8, COUNT>(c, L, stream);  // k <= 128
  }
  if constexpr (G <= 16) {
    if (need <= 4) return run<G, 4, COUNT>(c, L, stream);
  }
  if constexpr (G <= 8) {
    if (need <= 8) return run<G, 8, COUNT>(c, L, stream);
  }
  if constexpr (G <= 4) {
    if (need <= 16) return run<G, 16, COUNT>(c, L, stream);
  }
  return cudaErrorInvalidValue;
}

template <bool COUNT>
cudaError_t pick_g(const CloudDevHost& c, const PlainLaunch& L, cudaStream_t stream) {
  if (!COUNT && L.lanes == 32 && L.placement == 2) {
    if (c.hub_of) {  // the cloud has box trees over its long lists
      if (L.k <= 32) return run_warp<32, true>(c, L, stream);
      if (L.k <= 64) return run_warp<64, true>(c, L, stream);
      return run_warp<128, true>(c, L, stream);
    }
    if (L.k <= 32) return run_warp<32, false>(c, L, stream);
    if (L.k <= 64) return run_warp<64, false>(c, L, stream);
    return run_warp<128, false>(c, L, stream);
  }
  switch (L.lanes) {
    case 1: return pick_thread<COUNT>(c, L, stream);
    case 4: return pick_s<4, COUNT>(c, L, stream);
    case 8: return pick_s<8, COUNT>(c, L, stream);
    case 16: return pick_s<16, COUNT>(c, L, stream);
    case 32: return pick_s<32, COUNT>(c, L, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

int current_device() {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return dev;
}

int num_sms() {
  static PerDevice<int> sms_of;
  const int dev = current_device();
  return sms_of.with(dev, 1, [&](int& sms) {
    if (sms < 1) {
      if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
          sms < 1) {
        cudaGetLastError();
        return 1;  // not cached: asked again next time
      }
    }
    return sms;
  });
}

// Measured on the 1M-site torus with 4M box queries: one query per thread
// is fastest up to k = 16 (k = 4: 359M q/s vs 264M with 8 lanes; k = 16:
// 124M vs 111M with 16 lanes); above that the 32-slot register list costs
// too much occupancy and 16 lanes win (k = 32: 44M vs 26M with 1 lane).
namespace {

__global__ void fill_entries_kernel(const float4* __restrict__ pts, const int32_t* __restrict__ succ,
                                    int64_t E, float4* __restrict__ ent) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += stride) {
    const int32_t s = __ldg(succ + e);
    const float4 p = __ldg(pts + s);
    ent[e] = make_float4(p.x, p.y, p.z, __int_as_float(s));
  }
}

__global__ void gather_sites_kernel(const float4* __restrict__ pts, int32_t n,
                                    const int32_t* __restrict__ sites, int64_t nq,
                                    const int32_t* __restrict__ m, int32_t m_scalar,
                                    float4* __restrict__ q, int32_t* __restrict__ m_out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nq; i += stride) {
    const int32_t r = __ldg(sites + i);
    const bool ok = r >= 0 && r < n;
    q[i] = ok ? __ldg(pts + r) : make_float4(0.f, 0.f, 0.f, 0.f);
    m_out[i] = ok ? (m ? __ldg(m + i) : m_scalar) : 0;
  }
}

}  // namespace

cudaError_t launch_gather_sites(const CloudDevHost& c, const int32_t* sites, int64_t nq,
                                const int32_t* m, int32_t m_scalar, float4* q, int32_t* m_out,
                                cudaStream_t stream) {
  if (nq <= 0) return cudaSuccess;
  const int64_t blocks = std::min<int64_t>((nq + 255) / 256, (int64_t)num_sms() * 8);
  gather_sites_kernel<<<(unsigned)blocks, 256, 0, stream>>>((const float4*)c.pts, c.n, sites, nq,
                                                            m, m_scalar, q, m_out);
  return cudaGetLastError();
}

cudaError_t launch_fill_entries(const void* pts, const int32_t* succ, int64_t E, void* ent,
                                cudaStream_t stream) {
  if (E <= 0) return cudaSuccess;
  const int64_t blocks = std::min<int64_t>((E + 255) / 256, (int64_t)num_sms() * 8);
  fill_entries_kernel<<<(unsigned)blocks, 256, 0, stream>>>((const float4*)pts, succ, E,
                                                            (float4*)ent);
  return cudaGetLastError();
}

// Measured on the 1M-site torus with 4M box queries (queries/s): one query
// per thread with the list in shared memory against one warp per query with
// the warp's list in shared memory: k = 32: 164M / 120M; k = 64: 51M / 54M;
// k = 100: 21M / 26M; k = 128: 12M / 21M. Register lists over a group of
// 32 (16) lanes: 61M (45M), 21M (7M), 8M (4M), 6M (3M).
int default_lanes(int k) { return k >= kWarpMinK ? 32 : 1; }

int plain_max_k(int lanes) { return (lanes == 4 || lanes == 8) ? 64 : 128; }

// Shared-memory lists for one lane (per thread) and for 32 lanes (per
// warp); the group kernels of 4, 8 and 16 lanes keep theirs in registers.
int default_placement(int k, int lanes) {
  (void)k;
  return (lanes == 1 || lanes == 32) ? 2 : 1;
}

cudaError_t launch_knn_plain(const CloudDevHost& c, const PlainLaunch& L, cudaStream_t stream) {
  if (L.nq == 0) return cudaSuccess;
  if (L.counters) return pick_g<true>(c, L, stream);
  return pick_g<false>(c, L, stream);
}

}  // namespace mknn
