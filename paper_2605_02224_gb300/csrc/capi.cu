// C ABI: cloud lifetime, build, checkpoint, query entry points.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>

#include "../../include/mknn.h"
#include "builder.h"
#include "cloud.h"
#include "knn_kernels.h"
#include "predicates.h"
#include "batch.h"
#include "hub_index.h"

namespace mknn {

namespace {
thread_local std::string g_err;
}

void set_error(const std::string& msg) { g_err = msg; }

cudaError_t upload_entries(const mknn_cloud* c, int32_t* d_succ, void* d_ent, int64_t slack,
                           cudaStream_t s) {
  const int64_t n = c->n, E = (int64_t)c->succ.size();
  const int64_t total = E + slack * n;
  if (total <= 0) return cudaSuccess;
  cudaError_t e;
  if (slack == 0) {
    e = cudaMemcpyAsync(d_succ, c->succ.data(), (size_t)E * 4, cudaMemcpyHostToDevice, s);
  } else {
    std::vector<int32_t> spaced((size_t)total, 0);  // empty slots hold rank 0 (never read)
    for (int64_t i = 0; i < n; ++i)
      std::copy(c->succ.begin() + c->rowp[i], c->succ.begin() + c->rowp[i + 1],
                spaced.begin() + c->rowp[i] + slack * i);
    e = cudaMemcpyAsync(d_succ, spaced.data(), (size_t)total * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // before `spaced` goes
  }
  if (e != cudaSuccess) return e;
  return launch_fill_entries(c->d_pts, d_succ, total, d_ent, s);
}
const char* get_error() { return g_err.c_str(); }

namespace {

mknn_status fail(mknn_status s, const std::string& msg) {
  set_error(msg);
  return s;
}

mknn_status cuda_fail(cudaError_t e, const char* what) {
  return fail(MKNN_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void compute_bbox(mknn_cloud* c) {
  if (c->n == 0) return;
  for (int d = 0; d < 3; ++d) {
    c->lo[d] = c->hi[d] = c->xyz[d];
  }
  for (int64_t i = 0; i < c->n; ++i)
    for (int d = 0; d < 3; ++d) {
      const float v = c->xyz[3 * i + d];
      c->lo[d] = std::min(c->lo[d], v);
      c->hi[d] = std::max(c->hi[d], v);
    }
}

void free_device(mknn_cloud* c) {
  if (c->device >= 0) {
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(c->device);
    cudaFree(c->d_pts);
    cudaFree(c->d_rows);
    cudaFree(c->d_succ);
    cudaFree(c->d_ent);
    cudaFree(c->d_err);
    cudaFree(c->d_hub_of);
    cudaFree(c->d_hub_desc);
    cudaFree(c->d_hub_ent);
    cudaFree(c->d_hub_node);
    cudaSetDevice(cur);
  }
  c->d_hub_of = nullptr;
  c->d_hub_desc = c->d_hub_ent = c->d_hub_node = nullptr;
  c->hub_trees = c->hub_entries = 0;
  c->d_pts = nullptr;
  c->d_ent = nullptr;
  c->pts_cap = c->ent_cap = c->ent_top = 0;
  c->row_first.clear();
  c->row_cap.clear();
  c->d_rows = nullptr;
  c->d_succ = c->d_err = nullptr;
  c->device = -1;
  c->dev_bytes = 0;
}

// Library-managed scratch, one buffer per (device, stream), grow-only.
struct ScratchKey {
  int dev;
  cudaStream_t s;
  bool operator<(const ScratchKey& o) const {
    return dev != o.dev ? dev < o.dev : (uintptr_t)s < (uintptr_t)o.s;
  }
};
std::mutex g_scratch_mu;
std::map<ScratchKey, std::pair<void*, size_t>> g_scratch;

cudaError_t scratch_for(cudaStream_t s, size_t bytes, void** out) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  auto& slot = g_scratch[ScratchKey{dev, s}];
  if (slot.second < bytes) {
    if (slot.first) {
      cudaError_t e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return e;
      cudaFree(slot.first);
      slot.first = nullptr;
      slot.second = 0;
    }
    size_t want = std::max(bytes, slot.second * 2);
    cudaError_t e = cudaMalloc(&slot.first, want);
    if (e != cudaSuccess) {
      cudaGetLastError();
      e = cudaMalloc(&slot.first, bytes);
      if (e != cudaSuccess) return e;
      want = bytes;
    }
    slot.second = want;
  }
  *out = slot.first;
  return cudaSuccess;
}

size_t perm_bytes(int64_t nq) { return ((size_t)nq * 4 + 255) & ~(size_t)255; }

// Same-manifold queries: the gathered coordinates (float4) and prefix bounds.
size_t site_q_bytes(int64_t nq) { return ((size_t)nq * 16 + 255) & ~(size_t)255; }
size_t sites_bytes(int64_t nq) { return site_q_bytes(nq) + perm_bytes(nq); }

bool sort_enabled(const mknn_knn_opts* o, int64_t nq) {
  if (o && o->sort < 0) return false;
  if (o && o->sort > 0) return true;
  return nq >= kSortMinQueries;
}

mknn_status check_cloud_dev(const mknn_cloud* c) {
  if (!c) return fail(MKNN_EINVAL, "cloud is NULL");
  if (!c->d_pts) return fail(MKNN_EINVAL, "cloud is not uploaded (call mknn_cloud_upload)");
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != c->device)
    return fail(MKNN_EINVAL, "cloud lives on device " + std::to_string(c->device) +
                                 " but the current device is " + std::to_string(cur));
  return MKNN_OK;
}

}  // namespace
}  // namespace mknn

using namespace mknn;

extern "C" {

const char* mknn_last_error(void) { return get_error(); }

const char* mknn_version(void) { return "mknn-gb300 0.1 (sm_103a)"; }

mknn_status mknn_build(const float* xyz, int64_t n, const int64_t* order,
                       const mknn_build_opts* opts, mknn_cloud** out) {
  if (!out) return fail(MKNN_EINVAL, "out is NULL");
  *out = nullptr;
  if (!xyz && n > 0) return fail(MKNN_EINVAL, "xyz is NULL");
  if (n < 1 || n > (int64_t)0x7FFFFFF0) return fail(MKNN_EINVAL, "n out of range");
  std::unique_ptr<mknn_cloud> c;
  try {
    c.reset(new mknn_cloud());
    c->n = n;
    c->order.resize(n);
    if (order) {
      std::vector<uint8_t> seen(n, 0);
      for (int64_t r = 0; r < n; ++r) {
        const int64_t o = order[r];
        if (o < 0 || o >= n || seen[o])
          return fail(MKNN_EINVAL, "order is not a permutation of 0..n-1");
        seen[o] = 1;
        c->order[r] = o;
      }
    } else {
      for (int64_t r = 0; r < n; ++r) c->order[r] = r;
    }
    c->xyz.resize(3 * n);
    for (int64_t r = 0; r < n; ++r) {
      const float* p = xyz + 3 * c->order[r];
      for (int d = 0; d < 3; ++d) {
        if (!std::isfinite(p[d]))
          return fail(MKNN_EINVAL, "non-finite coordinate at input index " +
                                       std::to_string(c->order[r]));
        c->xyz[3 * r + d] = p[d];
      }
    }
    SuccessorTable t;
    std::string err;
    const bool keep = opts && opts->keep_tets;
    bool ok;
    if (opts && opts->dynamic) {
      c->inc.reset(new IncrementalTable());
      ok = c->inc->build(c->xyz.data(), n, keep, &t, &err);
      if (ok && !c->inc->can_append()) {
        ok = false;
        err = "a dynamic cloud needs points that span 3D (these are all coplanar)";
      }
    } else {
      ok = build_successor_table(c->xyz.data(), n, keep, &t, &err);
    }
    if (!ok) {
      const bool degen = err.find("coplanar") != std::string::npos;
      const bool oom = err.find("memory") != std::string::npos;
      return fail(degen ? MKNN_EDEGENERATE : (oom ? MKNN_ENOMEM : MKNN_EINVAL), err);
    }
    if (t.stats.entries >= (int64_t)0x7FFFFFFF)
      return fail(MKNN_EINVAL, "successor table exceeds 2^31 entries");
    c->rowp = std::move(t.rowp);
    c->succ = std::move(t.succ);
    c->tets = std::move(t.tets);
    c->stats = t.stats;
    compute_bbox(c.get());
  } catch (const std::bad_alloc&) {
    return fail(MKNN_ENOMEM, "host allocation failed");
  }
  *out = c.release();
  return MKNN_OK;
}

mknn_status mknn_cloud_from_table(const float* xyz_ranked, int64_t n, const int64_t* rowp,
                                  const int32_t* succ, mknn_cloud** out) {
  if (!out) return fail(MKNN_EINVAL, "out is NULL");
  *out = nullptr;
  if (n < 1 || n > (int64_t)0x7FFFFFF0) return fail(MKNN_EINVAL, "n out of range");
  if (!xyz_ranked || !rowp) return fail(MKNN_EINVAL, "NULL array");
  if (rowp[0] != 0) return fail(MKNN_EINVAL, "rowp[0] must be 0");
  for (int64_t i = 0; i < n; ++i)
    if (rowp[i + 1] < rowp[i]) return fail(MKNN_EINVAL, "rowp must be nondecreasing");
  const int64_t E = rowp[n];
  if (E >= (int64_t)0x7FFFFFFF) return fail(MKNN_EINVAL, "table exceeds 2^31 entries");
  if (E > 0 && !succ) return fail(MKNN_EINVAL, "succ is NULL");
  for (int64_t i = 0; i < n; ++i) {
    int64_t prev = i;
    for (int64_t e = rowp[i]; e < rowp[i + 1]; ++e) {
      const int64_t s = succ[e];
      if (s <= prev || s >= n)
        return fail(MKNN_EINVAL, "row " + std::to_string(i) +
                                     " must be strictly ascending with entries in (i, n)");
      prev = s;
    }
  }
  for (int64_t i = 0; i < 3 * n; ++i)
    if (!std::isfinite(xyz_ranked[i])) return fail(MKNN_EINVAL, "non-finite coordinate");
  try {
    std::unique_ptr<mknn_cloud> c(new mknn_cloud());
    c->n = n;
    c->xyz.assign(xyz_ranked, xyz_ranked + 3 * n);
    c->order.resize(n);
    for (int64_t r = 0; r < n; ++r) c->order[r] = r;
    c->rowp.assign(rowp, rowp + n + 1);
    c->succ.assign(succ, succ + E);
    c->stats.n = n;
    c->stats.entries = E;
    compute_bbox(c.get());
    *out = c.release();
  } catch (const std::bad_alloc&) {
    return fail(MKNN_ENOMEM, "host allocation failed");
  }
  return MKNN_OK;
}

mknn_status mknn_cloud_upload(mknn_cloud* c, mknn_stream_t stream) {
  if (!c) return fail(MKNN_EINVAL, "cloud is NULL");
  std::lock_guard<std::mutex> lk(c->mu);
  int cur = 0;
  cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (c->d_pts && c->device == cur) return MKNN_OK;
  if (c->d_pts) free_device(c);
  c->sync_csr();
  const int64_t n = c->n, E = c->E();
  // a dynamic cloud gets headroom for appended sites and entries
  const bool dyn = (bool)c->inc;
  const int64_t slack = dyn ? kRowSlack : 0;  // room for appends in every row
  const int64_t pcap = dyn ? n + std::max<int64_t>(n / 4, 4096) : n;
  const int64_t ecap =
      std::max<int64_t>(dyn ? E + slack * n + std::max<int64_t>(E / 4, 1 << 16) : E, 1);
  if (ecap >= (int64_t)0x7FFFFFFF) return fail(MKNN_EINVAL, "entry arena exceeds 2^31 entries");
  std::vector<float> p4;
  std::vector<int2> rows;
  try {
    p4.resize(4 * n);
    rows.resize(n);
    if (dyn) {
      c->row_first.resize(n);
      c->row_cap.resize(n);
    }
  } catch (const std::bad_alloc&) {
    return fail(MKNN_ENOMEM, "host allocation failed");
  }
  for (int64_t i = 0; i < n; ++i) {
    p4[4 * i] = c->xyz[3 * i];
    p4[4 * i + 1] = c->xyz[3 * i + 1];
    p4[4 * i + 2] = c->xyz[3 * i + 2];
    p4[4 * i + 3] = 0.f;
    const int64_t first = c->rowp[i] + slack * i, len = c->rowp[i + 1] - c->rowp[i];
    rows[i] = make_int2((int32_t)first, (int32_t)(first + len));
    if (dyn) {
      c->row_first[i] = first;
      c->row_cap[i] = len + slack;
    }
  }
  c->device = cur;
  const size_t b_pts = (size_t)pcap * 16, b_rows = (size_t)pcap * 8, b_succ = (size_t)ecap * 4,
               b_ent = (size_t)ecap * 16;
  if ((e = cudaMalloc(&c->d_pts, b_pts)) != cudaSuccess ||
      (e = cudaMalloc((void**)&c->d_rows, b_rows)) != cudaSuccess ||
      (e = cudaMalloc((void**)&c->d_succ, b_succ)) != cudaSuccess ||
      (e = cudaMalloc(&c->d_ent, b_ent)) != cudaSuccess ||
      (e = cudaMalloc((void**)&c->d_err, 256)) != cudaSuccess) {
    cudaGetLastError();
    free_device(c);
    return fail(MKNN_ENOMEM, std::string("device allocation failed: ") + cudaGetErrorString(e));
  }
  cudaStream_t s = (cudaStream_t)stream;
  if ((e = cudaMemcpyAsync(c->d_pts, p4.data(), (size_t)n * 16, cudaMemcpyHostToDevice, s)) !=
          cudaSuccess ||
      (e = cudaMemcpyAsync(c->d_rows, rows.data(), (size_t)n * 8, cudaMemcpyHostToDevice, s)) !=
          cudaSuccess ||
      (E > 0 && (e = upload_entries(c, c->d_succ, c->d_ent, slack, s)) != cudaSuccess) ||
      (e = cudaMemsetAsync(c->d_err, 0, 256, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess) {
    free_device(c);
    return cuda_fail(e, "upload");
  }
  // box trees over the long lists (a dynamic cloud's lists change: none)
  size_t b_hub = 0;
  if (!dyn && E > 0) {
    HubIndex H;
    try {
      build_hub_index(n, c->xyz.data(), c->rowp.data(), c->succ.data(), kHubMinRow,
                      kHubMinLongest, &H);
    } catch (const std::bad_alloc&) {
      free_device(c);
      return fail(MKNN_ENOMEM, "host allocation failed");
    }
    if (H.hubs() > 0) {
      const size_t b_of = H.hub_of.size() * 4, b_desc = H.desc.size() * 4,
                   b_hent = H.ent.size() * 4, b_node = H.node.size() * 4;
      if ((e = cudaMalloc((void**)&c->d_hub_of, b_of)) != cudaSuccess ||
          (e = cudaMalloc(&c->d_hub_desc, b_desc)) != cudaSuccess ||
          (e = cudaMalloc(&c->d_hub_ent, b_hent)) != cudaSuccess ||
          (e = cudaMalloc(&c->d_hub_node, b_node)) != cudaSuccess) {
        cudaGetLastError();
        free_device(c);
        return fail(MKNN_ENOMEM, std::string("device allocation failed: ") + cudaGetErrorString(e));
      }
      if ((e = cudaMemcpyAsync(c->d_hub_of, H.hub_of.data(), b_of, cudaMemcpyHostToDevice, s)) !=
              cudaSuccess ||
          (e = cudaMemcpyAsync(c->d_hub_desc, H.desc.data(), b_desc, cudaMemcpyHostToDevice,
                               s)) != cudaSuccess ||
          (e = cudaMemcpyAsync(c->d_hub_ent, H.ent.data(), b_hent, cudaMemcpyHostToDevice, s)) !=
              cudaSuccess ||
          (e = cudaMemcpyAsync(c->d_hub_node, H.node.data(), b_node, cudaMemcpyHostToDevice,
                               s)) != cudaSuccess ||
          (e = cudaStreamSynchronize(s)) != cudaSuccess) {  // before H goes
        free_device(c);
        return cuda_fail(e, "upload");
      }
      b_hub = b_of + b_desc + b_hent + b_node;
      c->hub_trees = H.hubs();
      for (int64_t h = 0; h < H.hubs(); ++h) c->hub_entries += H.desc[4 * h + 1];
    }
  }
  c->pts_cap = pcap;
  c->ent_cap = ecap;
  c->ent_top = E + slack * n;
  c->dev_bytes = b_pts + b_rows + b_succ + b_ent + 256 + b_hub;
  return MKNN_OK;
}

mknn_status mknn_cloud_release_device(mknn_cloud* c) {
  if (!c) return fail(MKNN_EINVAL, "cloud is NULL");
  if (c->holders.load() > 0) return fail(MKNN_EBUSY, "cloud is held by a server");
  std::lock_guard<std::mutex> lk(c->mu);
  free_device(c);
  return MKNN_OK;
}

mknn_status mknn_cloud_free(mknn_cloud* c) {
  if (!c) return MKNN_OK;
  if (c->holders.load() > 0) return fail(MKNN_EBUSY, "cloud is held by a server");
  free_device(c);
  delete c;
  return MKNN_OK;
}

mknn_status mknn_cloud_info(const mknn_cloud* c, int64_t* n, int64_t* E, size_t* dev_bytes) {
  if (!c) return fail(MKNN_EINVAL, "cloud is NULL");
  if (n) *n = c->n;
  if (E) *E = c->E();
  if (dev_bytes) *dev_bytes = c->dev_bytes;
  return MKNN_OK;
}

mknn_status mknn_cloud_trees(const mknn_cloud* c, int64_t* trees, int64_t* entries) {
  if (!c) return fail(MKNN_EINVAL, "cloud is NULL");
  if (trees) *trees = c->hub_trees;
  if (entries) *entries = c->hub_entries;
  return MKNN_OK;
}

mknn_status mknn_cloud_order(const mknn_cloud* c, int64_t* order_out) {
  if (!c || !order_out) return fail(MKNN_EINVAL, "NULL argument");
  std::memcpy(order_out, c->order.data(), (size_t)c->n * 8);
  return MKNN_OK;
}

mknn_status mknn_cloud_table(const mknn_cloud* c, float* xyz_ranked, int64_t* rowp,
                             int32_t* succ) {
  if (!c) return fail(MKNN_EINVAL, "cloud is NULL");
  if (xyz_ranked) std::memcpy(xyz_ranked, c->xyz.data(), c->xyz.size() * 4);
  c->sync_csr();
  if (rowp) std::memcpy(rowp, c->rowp.data(), c->rowp.size() * 8);
  if (succ) std::memcpy(succ, c->succ.data(), c->succ.size() * 4);
  return MKNN_OK;
}

mknn_status mknn_cloud_stats(const mknn_cloud* c, mknn_build_stats* o) {
  if (!c || !o) return fail(MKNN_EINVAL, "NULL argument");
  const BuildStats& s = c->stats;
  o->n = s.n;
  o->entries = s.entries;
  o->duplicates = s.duplicates;
  o->degenerate_prefix = s.degenerate_prefix;
  o->tets_final = s.tets_final;
  o->walk_steps = s.walk_steps;
  o->conflict_tests = s.conflict_tests;
  o->orient_calls = s.orient_calls;
  o->orient_exact = s.orient_exact;
  o->insphere_calls = s.insphere_calls;
  o->insphere_exact = s.insphere_exact;
  o->build_seconds = s.seconds;
  return MKNN_OK;
}

mknn_status mknn_cloud_tets(const mknn_cloud* c, int32_t* tets, int64_t* count) {
  if (!c || !count) return fail(MKNN_EINVAL, "NULL argument");
  *count = (int64_t)(c->tets.size() / 4);
  if (tets) std::memcpy(tets, c->tets.data(), c->tets.size() * 4);
  return MKNN_OK;
}

namespace {
const char kMagic[8] = {'M', 'K', 'N', 'N', 'C', 'L', 'D', '1'};
}

mknn_status mknn_cloud_save(const mknn_cloud* c, const char* path) {
  if (!c || !path) return fail(MKNN_EINVAL, "NULL argument");
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(MKNN_EIO, std::string("cannot open ") + path);
  c->sync_csr();
  const int64_t hdr[4] = {1, c->n, c->E(), 0};
  bool ok = std::fwrite(kMagic, 1, 8, f) == 8 && std::fwrite(hdr, 8, 4, f) == 4 &&
            std::fwrite(c->lo, 4, 3, f) == 3 && std::fwrite(c->hi, 4, 3, f) == 3 &&
            std::fwrite(c->xyz.data(), 4, c->xyz.size(), f) == c->xyz.size() &&
            std::fwrite(c->order.data(), 8, c->order.size(), f) == c->order.size() &&
            std::fwrite(c->rowp.data(), 8, c->rowp.size(), f) == c->rowp.size() &&
            std::fwrite(c->succ.data(), 4, c->succ.size(), f) == c->succ.size();
  ok = (std::fclose(f) == 0) && ok;
  return ok ? MKNN_OK : fail(MKNN_EIO, std::string("write failed: ") + path);
}

mknn_status mknn_cloud_load(const char* path, mknn_cloud** out) {
  if (!path || !out) return fail(MKNN_EINVAL, "NULL argument");
  *out = nullptr;
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(MKNN_EIO, std::string("cannot open ") + path);
  std::unique_ptr<mknn_cloud> c(new mknn_cloud());
  char magic[8];
  int64_t hdr[4];
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kMagic, 8) == 0 &&
            std::fread(hdr, 8, 4, f) == 4 && hdr[0] == 1 && hdr[1] >= 1 && hdr[2] >= 0 &&
            hdr[1] <= (int64_t)0x7FFFFFF0 && hdr[2] < (int64_t)0x7FFFFFFF;
  if (ok) {
    try {
      c->n = hdr[1];
      c->xyz.resize(3 * hdr[1]);
      c->order.resize(hdr[1]);
      c->rowp.resize(hdr[1] + 1);
      c->succ.resize(hdr[2]);
    } catch (const std::bad_alloc&) {
      std::fclose(f);
      return fail(MKNN_ENOMEM, "host allocation failed");
    }
    ok = std::fread(c->lo, 4, 3, f) == 3 && std::fread(c->hi, 4, 3, f) == 3 &&
         std::fread(c->xyz.data(), 4, c->xyz.size(), f) == c->xyz.size() &&
         std::fread(c->order.data(), 8, c->order.size(), f) == c->order.size() &&
         std::fread(c->rowp.data(), 8, c->rowp.size(), f) == c->rowp.size() &&
         std::fread(c->succ.data(), 4, c->succ.size(), f) == c->succ.size();
  }
  std::fclose(f);
  if (!ok) return fail(MKNN_EIO, std::string("bad or truncated cloud file: ") + path);
  if (c->rowp[0] != 0 || c->rowp[c->n] != c->E())
    return fail(MKNN_EIO, std::string("inconsistent table in ") + path);
  c->stats.n = c->n;
  c->stats.entries = c->E();
  *out = c.release();
  return MKNN_OK;
}

size_t mknn_knn_workspace_size(int64_t nq, const mknn_knn_opts* opts) {
  if (nq <= 0) return 0;
  const size_t sort =
      (opts && opts->order) || !sort_enabled(opts, nq) ? 0 : sort_workspace_bytes(nq) + perm_bytes(nq);
  return sort + defer_bytes(nq);
}

size_t mknn_query_order_workspace_size(int64_t nq) {
  return nq < 0 ? 0 : sort_workspace_bytes(nq);
}

mknn_status mknn_query_order(const mknn_cloud* c, const float* q, int64_t nq, int32_t q_stride,
                             int32_t* perm_out, void* workspace, size_t workspace_bytes,
                             mknn_stream_t stream) {
  mknn_status st = check_cloud_dev(c);
  if (st != MKNN_OK) return st;
  if (nq < 0 || nq >= (int64_t)0x7FFFFFFF) return fail(MKNN_EINVAL, "nq out of range");
  if (q_stride < 3) return fail(MKNN_EINVAL, "q_stride must be >= 3");
  if (nq == 0) return MKNN_OK;
  if (!q || !perm_out) return fail(MKNN_EINVAL, "NULL device pointer");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t need = sort_workspace_bytes(nq);
  void* ws = workspace;
  if (ws) {
    if (workspace_bytes < need)
      return fail(MKNN_EINVAL, "workspace smaller than mknn_query_order_workspace_size");
  } else {
    cudaError_t e = scratch_for(s, need, &ws);
    if (e != cudaSuccess) return fail(MKNN_ENOMEM, "workspace allocation failed");
  }
  cudaError_t e = launch_query_sort(c->dev(), q, q_stride, nq, ws, perm_out, s);
  if (e != cudaSuccess) return cuda_fail(e, "query sort launch");
  return MKNN_OK;
}

mknn_status mknn_knn_ex(const mknn_cloud* c, const float* q, int64_t nq, int32_t q_stride,
                        int32_t k, const int32_t* m, int32_t m_scalar, int32_t* out_idx,
                        float* out_d2, const mknn_knn_opts* opts, mknn_stream_t stream) {
  mknn_status st = check_cloud_dev(c);
  if (st != MKNN_OK) return st;
  if (nq < 0 || nq >= (int64_t)0x7FFFFFFF) return fail(MKNN_EINVAL, "nq out of range");
  if (q_stride < 3) return fail(MKNN_EINVAL, "q_stride must be >= 3");
  if (k < 1 || k > MKNN_MAX_K) return fail(MKNN_EINVAL, "k must be in [1, 128]");
  if (!m) {
    if (m_scalar == 0) m_scalar = (int32_t)c->n;
    if (m_scalar < 1 || m_scalar > c->n) return fail(MKNN_EINVAL, "m_scalar must be in [1, n]");
  }
  if (nq == 0) return MKNN_OK;
  if (!q || !out_idx || !out_d2) return fail(MKNN_EINVAL, "NULL device pointer");
  const Mode chosen = choose_mode(k, c->n, c->hub_bucket(), nq, c->d_hub_of != nullptr);
  int lanes = (opts && opts->lanes) ? opts->lanes : chosen.lanes;
  if (lanes != 1 && lanes != 4 && lanes != 8 && lanes != 16 && lanes != 32)
    return fail(MKNN_EINVAL, "lanes must be 1, 4, 8, 16 or 32");
  if (k > plain_max_k(lanes))
    return fail(MKNN_EINVAL, "k above what this lane width holds (4, 8 lanes: 64; 1, 16, 32: 128)");
  if (lanes == 1 && k > 64 && ((opts && opts->counters) || (opts && opts->placement == 1)))
    return fail(MKNN_EINVAL, "one lane with k > 64 needs the shared-memory list (no counters)");
  const int placement = (opts && opts->placement)
                            ? opts->placement
                            : ((opts && opts->lanes) ? default_placement(k, lanes) : chosen.placement);
  if (placement != 1 && placement != 2)
    return fail(MKNN_EINVAL, "placement must be 0, 1 (registers) or 2 (shared memory)");
  cudaStream_t s = (cudaStream_t)stream;
  const int32_t* perm = opts ? opts->order : nullptr;
  // scratch: the sort's (unless an order is given), then the hand-over of
  // queries to the one-warp kernel (one lane on a cloud with box trees)
  const size_t sort_need = (!perm && sort_enabled(opts, nq)) ? sort_workspace_bytes(nq) + perm_bytes(nq) : 0;
  const bool wants_defer =
      c->d_hub_of && lanes == 1 && placement == 2 && !(opts && opts->counters);
  size_t need = sort_need + (wants_defer ? defer_bytes(nq) : 0);
  void* ws = nullptr;
  if (need > 0) {
    if (opts && opts->workspace) {
      if (opts->workspace_bytes < sort_need)
        return fail(MKNN_EINVAL, "workspace smaller than mknn_knn_workspace_size");
      if (opts->workspace_bytes < need) need = sort_need;  // too small to hand over: scan instead
      ws = opts->workspace;
    } else {
      cudaError_t e = scratch_for(s, need, &ws);
      if (e != cudaSuccess) return fail(MKNN_ENOMEM, "workspace allocation failed");
    }
  }
  if (sort_need > 0) {
    int32_t* p = (int32_t*)((char*)ws + sort_workspace_bytes(nq));
    cudaError_t e = launch_query_sort(c->dev(), q, q_stride, nq, ws, p, s);
    if (e != cudaSuccess) return cuda_fail(e, "query sort launch");
    perm = p;
  }
  PlainLaunch L;
  L.defer = need > sort_need ? (int32_t*)((char*)ws + sort_need) : nullptr;
  L.q = q;
  L.q_stride = q_stride;
  L.nq = nq;
  L.k = k;
  L.m = m;
  L.m_scalar = m_scalar;
  L.perm = perm;
  L.out_idx = out_idx;
  L.out_d2 = out_d2;
  L.counters = opts ? opts->counters : nullptr;
  L.err = c->d_err;
  L.lanes = lanes;
  L.blocks_per_sm = opts ? opts->blocks_per_sm : 0;
  L.placement = placement;
  cudaError_t e = launch_knn_plain(c->dev(), L, s);
  if (e != cudaSuccess) return cuda_fail(e, "knn kernel launch");
  return MKNN_OK;
}

size_t mknn_knn_sites_workspace_size(int64_t nq, const mknn_knn_opts* opts) {
  if (nq <= 0) return 0;
  return sites_bytes(nq) + mknn_knn_workspace_size(nq, opts);
}

mknn_status mknn_knn_sites(const mknn_cloud* c, const int32_t* sites, int64_t nq, int32_t k,
                           const int32_t* m, int32_t m_scalar, int32_t* out_idx, float* out_d2,
                           const mknn_knn_opts* opts, mknn_stream_t stream) {
  mknn_status st = check_cloud_dev(c);
  if (st != MKNN_OK) return st;
  if (nq < 0 || nq >= (int64_t)0x7FFFFFFF) return fail(MKNN_EINVAL, "nq out of range");
  if (k < 1 || k > MKNN_MAX_K) return fail(MKNN_EINVAL, "k must be in [1, 128]");
  if (!m) {
    if (m_scalar == 0) m_scalar = (int32_t)c->n;
    if (m_scalar < 1 || m_scalar > c->n) return fail(MKNN_EINVAL, "m_scalar must be in [1, n]");
  }
  if (nq == 0) return MKNN_OK;
  if (!sites || !out_idx || !out_d2) return fail(MKNN_EINVAL, "NULL device pointer");
  if (opts && opts->order) return fail(MKNN_EINVAL, "order is not taken by mknn_knn_sites");
  const size_t own = sites_bytes(nq);
  const size_t need = mknn_knn_sites_workspace_size(nq, opts);
  cudaStream_t s = (cudaStream_t)stream;
  void* ws = nullptr;
  if (opts && opts->workspace) {
    if (opts->workspace_bytes < need)
      return fail(MKNN_EINVAL, "workspace smaller than mknn_knn_sites_workspace_size");
    ws = opts->workspace;
  } else {
    cudaError_t e = scratch_for(s, need, &ws);
    if (e != cudaSuccess) return fail(MKNN_ENOMEM, "workspace allocation failed");
  }
  float4* q4 = (float4*)ws;
  int32_t* m_eff = (int32_t*)((char*)ws + site_q_bytes(nq));
  cudaError_t e = launch_gather_sites(c->dev(), sites, nq, m, m_scalar, q4, m_eff, s);
  if (e != cudaSuccess) return cuda_fail(e, "site gather launch");
  mknn_knn_opts o2{};
  if (opts) o2 = *opts;
  o2.workspace = (char*)ws + own;
  o2.workspace_bytes = need - own;
  return mknn_knn_ex(c, (const float*)q4, nq, 4, k, m_eff, 0, out_idx, out_d2, &o2, stream);
}

mknn_status mknn_knn(const mknn_cloud* c, const float* q, int64_t nq, int32_t q_stride, int32_t k,
                     const int32_t* m, int32_t m_scalar, int32_t* out_idx, float* out_d2,
                     mknn_stream_t stream) {
  return mknn_knn_ex(c, q, nq, q_stride, k, m, m_scalar, out_idx, out_d2, nullptr, stream);
}

mknn_status mknn_cloud_check(const mknn_cloud* c, int32_t* flags) {
  mknn_status st = check_cloud_dev(c);
  if (st != MKNN_OK) return st;
  int32_t v = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&v, c->d_err, 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(c->d_err, 0, 4);
  if (e != cudaSuccess) return cuda_fail(e, "reading error flags");
  if (flags) *flags = v;
  return MKNN_OK;
}

mknn_status mknn_cloud_validate(const mknn_cloud* c, int64_t* bad_orient, int64_t* bad_sphere) {
  if (!c || !bad_orient || !bad_sphere) return fail(MKNN_EINVAL, "NULL argument");
  const int64_t nt = (int64_t)(c->tets.size() / 4);
  int64_t bo = 0, bs = 0;
  const float* X = c->xyz.data();
  for (int64_t t = 0; t < nt; ++t) {
    const int32_t* v = &c->tets[4 * t];
    const float *a = X + 3 * (int64_t)v[0], *b = X + 3 * (int64_t)v[1], *cc = X + 3 * (int64_t)v[2],
                *d = X + 3 * (int64_t)v[3];
    if (orient3d(a, b, cc, d) <= 0) {
      ++bo;
      continue;
    }
    for (int64_t i = 0; i < c->n; ++i) {
      const float* p = X + 3 * i;
      if (insphere(a, b, cc, d, p) > 0) ++bs;
    }
  }
  *bad_orient = bo;
  *bad_sphere = bs;
  return MKNN_OK;
}

int32_t mknn_orient3d(const float* a, const float* b, const float* c, const float* d) {
  return orient3d(a, b, c, d);
}
int32_t mknn_insphere(const float* a, const float* b, const float* c, const float* d,
                      const float* e) {
  return insphere(a, b, c, d, e);
}
int32_t mknn_orient3d_exact(const float* a, const float* b, const float* c, const float* d) {
  return orient3d_exact(a, b, c, d);
}
int32_t mknn_insphere_exact(const float* a, const float* b, const float* c, const float* d,
                            const float* e) {
  return insphere_exact(a, b, c, d, e);
}

}  // extern "C"
