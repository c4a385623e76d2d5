// Appending points to a dynamic cloud: the host continues the build's
// Delaunay insertion (Sec. 3) for the new ranks, and the device copy is
// updated in place. A successor row only grows at its end (every new rank
// is larger than all earlier ones), so an append writes each changed row's
// new tail where the row has room; a row without room moves, whole, to the
// top of an append-only entry arena. New entries are written before the
// (first, end) pairs that make them reachable.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/mknn.h"
#include "cloud.h"
#include "knn_kernels.h"

namespace mknn {

namespace {

mknn_status afail(mknn_status s, const std::string& msg) {
  set_error(msg);
  return s;
}

__global__ void scatter_entries_kernel(const int32_t* __restrict__ pos,
                                       const int32_t* __restrict__ val, int64_t w,
                                       const float4* __restrict__ pts, int32_t* __restrict__ succ,
                                       float4* __restrict__ ent) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < w; i += stride) {
    const int32_t p = pos[i], s = val[i];
    const float4 x = pts[s];
    succ[p] = s;
    ent[p] = make_float4(x.x, x.y, x.z, __int_as_float(s));
  }
}

__global__ void scatter_rows_kernel(const int32_t* __restrict__ idx, const int2* __restrict__ val,
                                    int64_t r, int2* __restrict__ rows) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < r; i += stride)
    rows[idx[i]] = val[i];
}

unsigned grid_for(int64_t w) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((w + 255) / 256, num_sms() * 8));
}

// Moves an allocation to a larger one, keeping its first `keep` bytes.
cudaError_t grow(void** p, size_t keep, size_t bytes, cudaStream_t s) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, bytes);
  if (e != cudaSuccess) return e;
  if (keep) e = cudaMemcpyAsync(q, *p, keep, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaFree(q);
    return e;
  }
  cudaFree(*p);
  *p = q;
  return cudaSuccess;
}

// Device update after the host lists took the entries in `added` (row,
// rank); c->n already counts the new sites. Rows are read from the
// builder's lists.
mknn_status update_device(mknn_cloud* c, int64_t n_old,
                          const std::vector<std::pair<int32_t, int32_t>>& added,
                          cudaStream_t s) {
  const int64_t n_new = c->n;
  cudaError_t e = cudaSuccess;
  // sites: capacity, then the new coordinates
  if (n_new > c->pts_cap) {
    const int64_t cap = std::max<int64_t>(n_new, 2 * c->pts_cap);
    if ((e = grow(&c->d_pts, (size_t)n_old * 16, (size_t)cap * 16, s)) != cudaSuccess ||
        (e = grow((void**)&c->d_rows, (size_t)n_old * 8, (size_t)cap * 8, s)) != cudaSuccess)
      return afail(MKNN_ENOMEM, std::string("growing the site arrays: ") + cudaGetErrorString(e));
    c->dev_bytes += (size_t)(cap - c->pts_cap) * 24;
    c->pts_cap = cap;
  }
  std::vector<float> p4((size_t)(n_new - n_old) * 4);
  for (int64_t i = n_old; i < n_new; ++i) {
    for (int d = 0; d < 3; ++d) p4[(size_t)(i - n_old) * 4 + d] = c->xyz[3 * i + d];
    p4[(size_t)(i - n_old) * 4 + 3] = 0.f;
  }
  c->row_first.resize(n_new, 0);
  c->row_cap.resize(n_new, 0);
  // changed rows, each with its new tail or moved whole
  std::vector<int32_t> rows_changed;
  rows_changed.reserve(added.size());
  for (const auto& a : added) rows_changed.push_back(a.first);
  std::sort(rows_changed.begin(), rows_changed.end());
  std::vector<int32_t> pos, val, ridx, tail;
  std::vector<int2> rval;
  for (size_t a = 0; a < rows_changed.size();) {
    const int32_t i = rows_changed[a];
    size_t b = a;
    while (b < rows_changed.size() && rows_changed[b] == i) ++b;
    const int64_t len = c->inc->row_len(i), len_old = len - (int64_t)(b - a);
    a = b;
    int64_t from = len_old;
    if (len > c->row_cap[i]) {  // no room: the whole row moves to the arena top
      const int64_t cap = len + len / 4 + kRowSlack;
      c->row_first[i] = c->ent_top;
      c->row_cap[i] = cap;
      c->ent_top += cap;
      from = 0;
    }
    tail.clear();
    c->inc->row_tail(i, from, &tail);
    for (size_t t = 0; t < tail.size(); ++t) {
      pos.push_back((int32_t)(c->row_first[i] + from + (int64_t)t));
      val.push_back(tail[t]);
    }
    ridx.push_back(i);
    rval.push_back(make_int2((int32_t)c->row_first[i], (int32_t)(c->row_first[i] + len)));
  }
  if (c->ent_top >= (int64_t)0x7FFFFFFF)
    return afail(MKNN_ENOMEM, "entry arena would exceed 2^31 entries");
  if (c->ent_top > c->ent_cap) {
    const int64_t cap = std::min<int64_t>(std::max<int64_t>(c->ent_top, 2 * c->ent_cap),
                                          (int64_t)0x7FFFFFFE);
    const size_t keep = (size_t)c->ent_cap;
    if ((e = grow((void**)&c->d_succ, keep * 4, (size_t)cap * 4, s)) != cudaSuccess ||
        (e = grow(&c->d_ent, keep * 16, (size_t)cap * 16, s)) != cudaSuccess)
      return afail(MKNN_ENOMEM, std::string("growing the entry arena: ") + cudaGetErrorString(e));
    c->dev_bytes += (size_t)(cap - c->ent_cap) * 20;
    c->ent_cap = cap;
  }
  // the write lists, staged on the device
  const size_t w = pos.size(), r = ridx.size();
  const size_t bytes = w * 8 + r * 12 + 256;
  char* tmp = nullptr;
  if ((e = cudaMalloc((void**)&tmp, bytes)) != cudaSuccess)
    return afail(MKNN_ENOMEM, std::string("append staging: ") + cudaGetErrorString(e));
  int32_t* d_pos = (int32_t*)tmp;
  int32_t* d_val = d_pos + w;
  int32_t* d_ridx = d_val + w;
  int2* d_rval = (int2*)(tmp + ((w * 8 + r * 4 + 15) & ~(size_t)15));
  float4* pts = (float4*)c->d_pts;
  if (n_new > n_old) {
    e = cudaMemcpyAsync(pts + n_old, p4.data(), p4.size() * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemsetAsync(c->d_rows + n_old, 0, (size_t)(n_new - n_old) * 8, s);
  }
  if (e == cudaSuccess && w) {
    e = cudaMemcpyAsync(d_pos, pos.data(), w * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_val, val.data(), w * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
      scatter_entries_kernel<<<grid_for((int64_t)w), 256, 0, s>>>(
          d_pos, d_val, (int64_t)w, pts, c->d_succ, (float4*)c->d_ent);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess && r) {
    e = cudaMemcpyAsync(d_ridx, ridx.data(), r * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_rval, rval.data(), r * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
      scatter_rows_kernel<<<grid_for((int64_t)r), 256, 0, s>>>(d_ridx, d_rval, (int64_t)r,
                                                               c->d_rows);
      e = cudaGetLastError();
    }
  }
  cudaError_t e2 = cudaStreamSynchronize(s);
  cudaFree(tmp);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess)
    return afail(MKNN_ECUDA, std::string("append update: ") + cudaGetErrorString(e));
  return MKNN_OK;
}

// Lays the device table out afresh from the host CSR: rows in rank order,
// each followed by kRowSlack empty slots, the arena's headroom after them.
mknn_status compact_device(mknn_cloud* c, cudaStream_t s) {
  c->sync_csr();
  const int64_t n = c->n, E = (int64_t)c->succ.size(), fresh = E + kRowSlack * n;
  const int64_t cap = std::max<int64_t>(fresh + std::max<int64_t>(E / 4, 1 << 16), 1);
  if (cap >= (int64_t)0x7FFFFFFF) return afail(MKNN_ENOMEM, "entry arena exceeds 2^31 entries");
  std::vector<int2> rows((size_t)n);
  for (int64_t i = 0; i < n; ++i) {
    const int64_t first = c->rowp[i] + kRowSlack * i, len = c->rowp[i + 1] - c->rowp[i];
    rows[i] = make_int2((int32_t)first, (int32_t)(first + len));
    c->row_first[i] = first;
    c->row_cap[i] = len + kRowSlack;
  }
  int32_t* succ = nullptr;
  void* ent = nullptr;
  cudaError_t e;
  if ((e = cudaMalloc((void**)&succ, (size_t)cap * 4)) != cudaSuccess ||
      (e = cudaMalloc(&ent, (size_t)cap * 16)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(succ);
    return afail(MKNN_ENOMEM, std::string("compacting the entry arena: ") + cudaGetErrorString(e));
  }
  e = upload_entries(c, succ, ent, kRowSlack, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->d_rows, rows.data(), (size_t)n * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaFree(succ);
    cudaFree(ent);
    return afail(MKNN_ECUDA, std::string("compacting the entry arena: ") + cudaGetErrorString(e));
  }
  cudaFree(c->d_succ);
  cudaFree(c->d_ent);
  c->d_succ = succ;
  c->d_ent = ent;
  c->dev_bytes = c->dev_bytes - (size_t)c->ent_cap * 20 + (size_t)cap * 20;
  c->ent_cap = cap;
  c->ent_top = fresh;
  return MKNN_OK;
}

}  // namespace

}  // namespace mknn

using namespace mknn;

extern "C" {

mknn_status mknn_cloud_append(mknn_cloud* c, const float* xyz, int64_t count,
                              mknn_stream_t stream) {
  if (!c) return afail(MKNN_EINVAL, "cloud is NULL");
  if (!c->inc) return afail(MKNN_EINVAL, "the cloud was not built with the dynamic option");
  if (!c->inc->can_append())
    return afail(MKNN_EINVAL, "an earlier append failed: the cloud takes no more appends");
  if (count < 0) return afail(MKNN_EINVAL, "count < 0");
  if (count == 0) return MKNN_OK;
  if (!xyz) return afail(MKNN_EINVAL, "xyz is NULL");
  if (c->holders.load() > 0) return afail(MKNN_EBUSY, "cloud is held by a server");
  for (int64_t i = 0; i < 3 * count; ++i)
    if (!std::isfinite(xyz[i]))
      return afail(MKNN_EINVAL, "non-finite coordinate at appended point " + std::to_string(i / 3));
  std::lock_guard<std::mutex> lk(c->mu);
  const int64_t n_old = c->n, n_new = n_old + count;
  if (n_new > (int64_t)0x7FFFFFF0) return afail(MKNN_EINVAL, "n would exceed 2^31 - 16");
  std::vector<std::pair<int32_t, int32_t>> added;
  try {
    c->xyz.insert(c->xyz.end(), xyz, xyz + 3 * count);
    c->order.reserve((size_t)n_new);
    for (int64_t i = n_old; i < n_new; ++i) c->order.push_back(i);
    std::string err;
    if (!c->inc->append(c->xyz.data(), n_new, &added, &err)) {
      // the lists were rolled back: the cloud keeps its old points, table
      // and device copy, and takes no more appends
      c->xyz.resize((size_t)(3 * n_old));
      c->order.resize((size_t)n_old);
      return afail(MKNN_EINVAL, err + " (the cloud keeps its previous points and can no "
                                      "longer be appended to)");
    }
    c->n = n_new;
    c->csr_stale.store(true);
  } catch (const std::bad_alloc&) {
    return afail(MKNN_ENOMEM, "host allocation failed while appending");
  }
  if (c->inc->entries() >= (int64_t)0x7FFFFFFF)
    return afail(MKNN_EINVAL, "successor table exceeds 2^31 entries");
  const double secs = c->stats.seconds;
  c->stats = c->inc->stats();
  c->stats.seconds = secs;
  for (int64_t i = n_old; i < n_new; ++i)
    for (int d = 0; d < 3; ++d) {
      c->lo[d] = std::min(c->lo[d], c->xyz[3 * i + d]);
      c->hi[d] = std::max(c->hi[d], c->xyz[3 * i + d]);
    }
  c->hub_.store(-1);
  c->generation.fetch_add(1);
  if (!c->d_pts) return MKNN_OK;
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != c->device) cudaSetDevice(c->device);
  mknn_status st = update_device(c, n_old, added, (cudaStream_t)stream);
  // moved rows leave their old copies behind: once the arena is 40% larger
  // than a fresh layout would be, the table is laid out afresh (rows in
  // rank order, as after an upload), which keeps the live entries dense in
  // cache lines (queries read through L2)
  const int64_t fresh = c->inc->entries() + kRowSlack * c->n;
  if (st == MKNN_OK && c->ent_top > fresh + fresh * 2 / 5 + (1 << 16))
    st = compact_device(c, (cudaStream_t)stream);
  if (cur != c->device) cudaSetDevice(cur);
  return st;
}

mknn_status mknn_cloud_compact(mknn_cloud* c, mknn_stream_t stream) {
  if (!c) return afail(MKNN_EINVAL, "cloud is NULL");
  if (!c->inc) return afail(MKNN_EINVAL, "the cloud was not built with the dynamic option");
  std::lock_guard<std::mutex> lk(c->mu);
  if (!c->d_pts) return afail(MKNN_EINVAL, "cloud is not uploaded");
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != c->device) cudaSetDevice(c->device);
  const mknn_status st = compact_device(c, (cudaStream_t)stream);
  c->generation.fetch_add(1);  // the entry arrays moved
  if (cur != c->device) cudaSetDevice(cur);
  return st;
}

}  // extern "C"
