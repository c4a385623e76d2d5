// The cloud object behind the opaque mknn_cloud handle (internal).
#pragma once
#include <algorithm>
#include <atomic>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "builder.h"
#include "knn_kernels.h"

struct mknn_cloud {
  int64_t n = 0;
  std::vector<float> xyz;        // 3n, rank order
  std::vector<int64_t> order;    // rank -> input index
  std::vector<int64_t> rowp;     // n+1
  std::vector<int32_t> succ;     // E
  std::vector<int32_t> tets;     // optional, 4 per finite tetrahedron
  mknn::BuildStats stats;
  float lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  // device copy
  int device = -1;
  void* d_pts = nullptr;         // float4[n]
  int32_t* d_rowp = nullptr;     // [n+1]
  int32_t* d_succ = nullptr;     // [E]
  void* d_ent = nullptr;         // float4[E]: succ with the sites' coordinates inlined
  int32_t* d_err = nullptr;      // error flags
  size_t dev_bytes = 0;
  std::atomic<int> holders{0};   // servers referencing the cloud
  mutable std::mutex mu;

  int64_t E() const { return (int64_t)succ.size(); }
  // floor(log2(1 + longest successor list)): the tuning table's cloud shape
  // key (hub rows make queries costly whatever the size)
  int hub_bucket() const {
    int hb = hub_.load(std::memory_order_relaxed);
    if (hb >= 0) return hb;
    int64_t mx = 0;
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
    c.rowp = d_rowp;
    c.succ = d_succ;
    c.ent = d_ent;
    c.n = (int32_t)n;
    for (int i = 0; i < 3; ++i) {
      c.lo[i] = lo[i];
      c.hi[i] = hi[i];
    }
    return c;
  }
};

namespace mknn {
void set_error(const std::string& msg);
const char* get_error();
}  // namespace mknn
