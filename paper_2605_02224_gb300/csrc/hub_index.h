// Box trees over long successor lists (host side).
//
// On clouds whose sites lie on near-planar patches a few early sites get
// successor lists of 10^4-10^5 entries (every later site of the patch that
// was ever their Delaunay neighbour). Algorithm 1 reads such a list to its
// end whenever no entry is strictly closer than the current site, and
// Algorithm 2 offers all of it whenever the site is among the k-1 nearest,
// so a few queries read hundreds of thousands of entries.
//
// For every list of at least kHubMinRow entries the upload also keeps a
// second copy of its entries, reordered along a Morton curve over the
// list's bounding box and cut into chunks of 32, under a tree of boxes with
// fan-out 32: a level-0 node bounds one chunk, a level-l node bounds 32
// level-(l-1) nodes, up to a top level of at most 32 nodes. Each node keeps
// the smallest rank below it. The one-warp query kernel walks this tree
// instead of scanning such a list: both algorithms only need the entries
// that can be strictly closer than the current site (descent) or below
// the k-th key (expansion), with rank below m, and a box whose nearest
// point is farther, or whose smallest rank is not below m, holds none.
// The list in rank order stays in the table for every other kernel.
#pragma once
#include <cstdint>
#include <vector>

namespace mknn {

// Lists at least this long get a box tree, in a cloud whose longest list
// has at least kHubMinLongest entries. The walk's code slows the one-warp
// kernel's scan of the other lists by about a quarter (registers), which
// only clouds with real hubs win back: on the 1M-site torus (longest list
// 389) trees made k = 100 queries 28% slower; on 1.3M-site patch clouds
// (longest lists 10^5) 4.8x faster.
constexpr int64_t kHubMinRow = 256;
constexpr int64_t kHubMinLongest = 4096;
// Levels of a tree: 32^4 chunks of 32 entries at most; longer lists are
// scanned in rank order.
constexpr int kHubMaxLevels = 4;

struct HubIndex {
  std::vector<int32_t> hub_of;  // [n]: the site's tree, or -1 (empty when no list is long enough)
  std::vector<int32_t> desc;    // 4 per tree: first entry, list length, first node, levels
  std::vector<float> ent;       // 4 per entry (x, y, z, rank bits); chunks of 32, padded
  std::vector<float> node;      // 8 per node: box low corner and smallest rank's bits, high corner
                                // and largest rank's bits
  int64_t hubs() const { return (int64_t)desc.size() / 4; }
};

// Number of nodes at `level` of a tree over `len` entries and the offset of
// that level from the tree's first node (level 0 first).
inline void hub_level(int64_t len, int level, int64_t* offset, int64_t* count) {
  int64_t c = (len + 31) / 32, o = 0;
  for (int l = 0; l < level; ++l) {
    o += c;
    c = (c + 31) / 32;
  }
  *offset = o;
  *count = c;
}

// Levels of the tree over `len` entries (the top level holds at most 32
// nodes), or 0 when that takes more than kHubMaxLevels.
int hub_levels(int64_t len);

// Builds the trees of every list of at least min_row entries when the
// longest list has at least min_longest (else none). xyz holds the sites in
// rank order (3 per site); rowp / succ the table as CSR.
void build_hub_index(int64_t n, const float* xyz, const int64_t* rowp, const int32_t* succ,
                     int64_t min_row, int64_t min_longest, HubIndex* out);

}  // namespace mknn
