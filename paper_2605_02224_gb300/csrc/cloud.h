// The cloud object behind the opaque mknn_cloud handle (internal).
#pragma once
#include <algorithm>
#include <atomic>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include <memory>

#include "builder.h"
#include "knn_kernels.h"

struct mknn_cloud {
  int64_t n = 0;
  std::vector<float> xyz;        // 3n, rank order
  std::vector<int64_t> order;    // rank -> input index
  // the table as CSR; for a dynamic cloud the builder's lists are the
  // truth and this copy is refreshed on demand after appends (sync_csr)
  mutable std::vector<int64_t> rowp;  // n+1
  mutable std::vector<int32_t> succ;  // E
  mutable std::atomic<bool> csr_stale{false};
  mutable std::mutex csr_mu;
  std::vector<int32_t> tets;     // optional, 4 per finite tetrahedron
  mknn::BuildStats stats;
  float lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  // kept triangulation of a cloud built with the dynamic option (appends)
  std::unique_ptr<mknn::IncrementalTable> inc;
  // bumped by every append: plans made before it refuse to run
  std::atomic<uint64_t> generation{0};
  // device copy
  int device = -1;
  void* d_pts = nullptr;         // float4[n]
  int2* d_rows = nullptr;        // [n]: (first, end) of each row in d_succ / d_ent
  int32_t* d_succ = nullptr;     // [E]
  void* d_ent = nullptr;         // float4[E]: succ with the sites' coordinates inlined
  int32_t* d_err = nullptr;      // error flags
  // box trees over the long lists of a static cloud (hub_index.h), or NULL
  int32_t* d_hub_of = nullptr;   // [n]
  void* d_hub_desc = nullptr;    // int4 per tree
  void* d_hub_ent = nullptr;     // float4 per entry
  void* d_hub_node = nullptr;    // two float4 per node
  int64_t hub_trees = 0, hub_entries = 0;  // trees, and the entries of their lists
  size_t dev_bytes = 0;
  // device capacities: sites (d_pts, d_rows) and entries (d_succ, d_ent);
  // a dynamic cloud's rows live in an append-only arena: row i occupies
  // [row_first[i], row_first[i] + its length) with room up to row_cap[i],
  // and a row that outgrows its room moves to the arena's top
  int64_t pts_cap = 0, ent_cap = 0, ent_top = 0;
  std::vector<int64_t> row_first, row_cap;
  std::atomic<int> holders{0};   // servers referencing the cloud
  mutable std::mutex mu;

  int64_t E() const { return inc ? inc->entries() : (int64_t)succ.size(); }
  void sync_csr() const {
    if (!csr_stale.load()) return;
    std::lock_guard<std::mutex> lk(csr_mu);
    if (!csr_stale.load()) return;
    inc->csr(&rowp, &succ);
    csr_stale.store(false);
  }
  // floor(log2(1 + longest successor list)): the tuning table's cloud shape
  // key (hub rows make queries costly whatever the size)
  int hub_bucket() const {
    int hb = hub_.load(std::memory_order_relaxed);
    if (hb >= 0) return hb;
    int64_t mx = 0;
    if (inc)
      mx = inc->longest_row();
    else
      for (size_t i = 0; i + 1 < rowp.size(); ++i) mx = std::max<int64_t>(mx, rowp[i + 1] - rowp[i]);
    hb = 0;
    while ((int64_t(2) << hb) <= mx + 1) ++hb;
    hub_.store(hb, std::memory_order_relaxed);
    return hb;
  }
  mutable std::atomic<int> hub_{-1};
  mknn::CloudDevHost dev() const {
    mknn::CloudDevHost c;
    c.pts = d_pts;
    c.rows = d_rows;
    c.succ = d_succ;
    c.ent = d_ent;
    c.hub_of = d_hub_of;
    c.hub_desc = d_hub_desc;
    c.hub_ent = d_hub_ent;
    c.hub_node = d_hub_node;
    c.n = (int32_t)n;
    for (int i = 0; i < 3; ++i) {
      c.lo[i] = lo[i];
      c.hi[i] = hi[i];
    }
    return c;
  }
};

namespace mknn {
// Empty slots left after every row of a dynamic cloud when its table is laid
// out (upload, compaction), so that most rows take a few appends in place.
constexpr int64_t kRowSlack = 2;
// Writes the cloud's CSR into device arrays, `slack` empty slots after each
// row (row i starts at rowp[i] + slack * i), and fills ent from it.
cudaError_t upload_entries(const mknn_cloud* c, int32_t* d_succ, void* d_ent, int64_t slack,
                           cudaStream_t s);
void set_error(const std::string& msg);
const char* get_error();
}  // namespace mknn
