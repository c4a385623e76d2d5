// Box trees over long successor lists: see hub_index.h.
#include "hub_index.h"

#include <algorithm>
#include <cstring>
#include <limits>

namespace mknn {
namespace {

// Spreads the low 10 bits of v to every third bit.
uint32_t spread3(uint32_t v) {
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0x030000ffu;
  v = (v | (v << 8)) & 0x0300f00fu;
  v = (v | (v << 4)) & 0x030c30c3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

float rank_bits(int32_t r) {
  float f;
  std::memcpy(&f, &r, 4);
  return f;
}

int32_t bits_rank(float f) {
  int32_t r;
  std::memcpy(&r, &f, 4);
  return r;
}

}  // namespace

int hub_levels(int64_t len) {
  int64_t c = (len + 31) / 32;
  int levels = 1;
  while (c > 32) {
    c = (c + 31) / 32;
    ++levels;
  }
  return levels <= kHubMaxLevels ? levels : 0;
}

void build_hub_index(int64_t n, const float* xyz, const int64_t* rowp, const int32_t* succ,
                     int64_t min_row, int64_t min_longest, HubIndex* out) {
  out->hub_of.clear();
  out->desc.clear();
  out->ent.clear();
  out->node.clear();
  std::vector<int64_t> long_rows;
  int64_t longest = 0;
  for (int64_t i = 0; i < n; ++i) {
    const int64_t len = rowp[i + 1] - rowp[i];
    longest = std::max(longest, len);
    if (len >= min_row && hub_levels(len) > 0) long_rows.push_back(i);
  }
  if (long_rows.empty() || longest < min_longest) return;
  out->hub_of.assign((size_t)n, -1);
  std::vector<std::pair<uint32_t, int32_t>> keyed;  // (Morton code, rank)
  for (const int64_t i : long_rows) {
    const int64_t first = rowp[i], len = rowp[i + 1] - first;
    const int levels = hub_levels(len);
    float lo[3], hi[3];
    for (int d = 0; d < 3; ++d) lo[d] = hi[d] = xyz[3 * (int64_t)succ[first] + d];
    for (int64_t e = 0; e < len; ++e)
      for (int d = 0; d < 3; ++d) {
        const float v = xyz[3 * (int64_t)succ[first + e] + d];
        lo[d] = std::min(lo[d], v);
        hi[d] = std::max(hi[d], v);
      }
    keyed.resize((size_t)len);
    for (int64_t e = 0; e < len; ++e) {
      const int32_t s = succ[first + e];
      uint32_t code = 0;
      for (int d = 0; d < 3; ++d) {
        const double ext = (double)hi[d] - (double)lo[d];
        const double t = ext > 0 ? ((double)xyz[3 * (int64_t)s + d] - lo[d]) / ext : 0.0;
        const uint32_t cell = (uint32_t)std::min(1023.0, std::max(0.0, t * 1024.0));
        code |= spread3(cell) << d;
      }
      keyed[(size_t)e] = {code, s};
    }
    std::sort(keyed.begin(), keyed.end());
    const int64_t chunks = (len + 31) / 32;
    const int64_t ent0 = (int64_t)out->ent.size() / 4;
    const int64_t node0 = (int64_t)out->node.size() / 8;
    if (ent0 + chunks * 32 >= (int64_t)std::numeric_limits<int32_t>::max()) break;  // int32 offsets
    out->ent.resize((size_t)(ent0 + chunks * 32) * 4);
    float* ent = out->ent.data() + ent0 * 4;
    for (int64_t e = 0; e < chunks * 32; ++e) {
      if (e < len) {
        const int32_t s = keyed[(size_t)e].second;
        ent[4 * e] = xyz[3 * (int64_t)s];
        ent[4 * e + 1] = xyz[3 * (int64_t)s + 1];
        ent[4 * e + 2] = xyz[3 * (int64_t)s + 2];
        ent[4 * e + 3] = rank_bits(s);
      } else {  // pad: a rank no prefix bound admits
        ent[4 * e] = ent[4 * e + 1] = ent[4 * e + 2] = 0.f;
        ent[4 * e + 3] = rank_bits(std::numeric_limits<int32_t>::max());
      }
    }
    int64_t total_nodes = 0;
    for (int l = 0; l < levels; ++l) {
      int64_t off, cnt;
      hub_level(len, l, &off, &cnt);
      total_nodes = off + cnt;
    }
    out->node.resize((size_t)(node0 + total_nodes) * 8);
    float* node = out->node.data() + node0 * 8;
    // level 0: one box per chunk, over its real entries
    for (int64_t c = 0; c < chunks; ++c) {
      float* b = node + 8 * c;
      const int64_t e0 = 32 * c, e1 = std::min(len, e0 + 32);
      int32_t rmin = std::numeric_limits<int32_t>::max(), rmax = 0;
      for (int d = 0; d < 3; ++d) b[d] = b[4 + d] = ent[4 * e0 + d];
      for (int64_t e = e0; e < e1; ++e) {
        for (int d = 0; d < 3; ++d) {
          b[d] = std::min(b[d], ent[4 * e + d]);
          b[4 + d] = std::max(b[4 + d], ent[4 * e + d]);
        }
        const int32_t r = bits_rank(ent[4 * e + 3]);
        rmin = std::min(rmin, r);
        rmax = std::max(rmax, r);
      }
      b[3] = rank_bits(rmin);
      b[7] = rank_bits(rmax);
    }
    // level l: one box per 32 boxes of level l - 1
    for (int l = 1; l < levels; ++l) {
      int64_t off, cnt, coff, ccnt;
      hub_level(len, l, &off, &cnt);
      hub_level(len, l - 1, &coff, &ccnt);
      for (int64_t j = 0; j < cnt; ++j) {
        float* b = node + 8 * (off + j);
        const int64_t c0 = 32 * j, c1 = std::min(ccnt, c0 + 32);
        const float* f = node + 8 * (coff + c0);
        std::memcpy(b, f, 8 * sizeof(float));
        for (int64_t c = c0 + 1; c < c1; ++c) {
          const float* ch = node + 8 * (coff + c);
          for (int d = 0; d < 3; ++d) {
            b[d] = std::min(b[d], ch[d]);
            b[4 + d] = std::max(b[4 + d], ch[4 + d]);
          }
          b[3] = rank_bits(std::min(bits_rank(b[3]), bits_rank(ch[3])));
          b[7] = rank_bits(std::max(bits_rank(b[7]), bits_rank(ch[7])));
        }
      }
    }
    out->hub_of[(size_t)i] = (int32_t)out->hubs();
    out->desc.push_back((int32_t)ent0);
    out->desc.push_back((int32_t)len);
    out->desc.push_back((int32_t)node0);
    out->desc.push_back(levels);
  }
}

}  // namespace mknn
