// Host-side successor-table builder (Sec. 3; construction as in Sec. 2.2).
//
// Sites are inserted in rank order into an incremental 3D Delaunay
// triangulation (Bowyer-Watson). When p_j is inserted, j is appended to
// the successor list L_i of every Delaunay neighbour p_i of p_j in
// DT(P_{1:j}) (the vertices of the conflict cavity's boundary). Lists are
// therefore ascending. Ranks are 0-based.
#pragma once
#include <cstdint>
#include <memory>
#include <string>
#include <vector>

namespace mknn {

struct BuildStats {
  int64_t n = 0;
  int64_t entries = 0;          // E = sum of list lengths
  int64_t duplicates = 0;       // ranks whose coordinates repeat an earlier rank
  int64_t degenerate_prefix = 0;  // ranks 0..j0 that start with complete lists
  int64_t tets_final = 0;       // finite tetrahedra at the end
  int64_t walk_steps = 0;
  int64_t conflict_tests = 0;
  int64_t orient_calls = 0, orient_exact = 0;
  int64_t insphere_calls = 0, insphere_exact = 0;
  double seconds = 0.0;
};

struct SuccessorTable {
  std::vector<int64_t> rowp;    // n + 1
  std::vector<int32_t> succ;    // E, each row ascending
  std::vector<int32_t> tets;    // 4 * tets_final vertex ranks (only if requested)
  BuildStats stats;
};

// xyz: 3 * n floats in rank order. Returns false and sets *err on failure
// (non-finite coordinates, all points coplanar beyond the complete-table
// limit, out of memory).
bool build_successor_table(const float* xyz, int64_t n, bool keep_tets,
                           SuccessorTable* out, std::string* err);

// Largest all-coplanar input for which a complete table is produced.
constexpr int64_t kMaxCoplanarComplete = 4096;

namespace build_detail {
class Builder;
}

// A successor table that keeps its triangulation, so that points can be
// appended later (ranks n, n+1, ... in append order). Appending continues
// the same insertion, so the lists equal those of one build over all the
// points; an appended rank j only adds entries j to existing lists
// (Delaunay neighbours of p_j in DT(P_{1:j})) and starts its own empty.
class IncrementalTable {
 public:
  IncrementalTable();
  ~IncrementalTable();
  bool build(const float* xyz, int64_t n, bool keep_tets, SuccessorTable* out, std::string* err);
  // xyz holds n_new points in rank order whose first size() are the points
  // already inserted; inserts the others. Each successor entry added is
  // reported as (row, rank) in `added`, in insertion order.
  bool append(const float* xyz, int64_t n_new, std::vector<std::pair<int32_t, int32_t>>* added,
              std::string* err);
  void csr(std::vector<int64_t>* rowp, std::vector<int32_t>* succ) const;
  int64_t size() const;
  int64_t entries() const;
  int64_t row_len(int32_t i) const;
  int64_t longest_row() const;
  // Appends entries [from, row_len(i)) of row i to *out.
  void row_tail(int32_t i, int64_t from, std::vector<int32_t>* out) const;
  bool can_append() const;  // false when the points so far are all coplanar
  BuildStats stats() const;

 private:
  std::unique_ptr<build_detail::Builder> b_;
};

}  // namespace mknn
