/* CPU baselines for the k-NN query path (host code only, no GPU).
 *
 * Two reported baselines, timed next to the GPU kernels on the same host:
 *  - an exact kd-tree with prefix support: every node keeps the smallest
 *    insertion rank below it, so a query restricted to the prefix P_{1:m}
 *    (Sec. 4.2) skips subtrees whose ranks are all >= m;
 *  - Algorithms 1 and 2 (Sec. 4) on the successor table, one query after
 *    another per thread, as the paper runs them on a CPU (Sec. 5.1).
 * Both compute squared distances in float64 from the float32 inputs, in the
 * order ((dx*dx + dy*dy) + dz*dz), and order keys by (distance, rank), the
 * tie rule of Eq. (2); their results are the exact k-NN definition.
 *
 * Points are given in insertion-rank order (row r = rank r). Queries are
 * float32 rows of q_stride floats. m: per-query int32 bounds or NULL, then
 * m_scalar (0 = n). Outputs: int32 ranks and float32 squared distances,
 * nq x k, sorted by (distance, rank), padded with (-1, +inf) past min(k, m).
 * sorted: 0 = queries in input order, 1 = in the Morton order of their
 * cells (1024^3 grid over their bounding box; only the processing order
 * changes). threads: worker threads (0 = all hardware threads). Return 0 on success,
 * a negative value for invalid arguments (nothing is written then).
 * These baselines are not part of the GPU library and share no code with it. */
#pragma once
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mknn_cpu_kdtree mknn_cpu_kdtree;

/* Builds the tree over n ranked points (leaves of at most `leaf` points,
 * 0 = 8). Copies what it needs; the caller keeps xyz. */
int mknn_cpu_kdtree_build(const float* xyz, int64_t n, int32_t leaf, mknn_cpu_kdtree** out);
void mknn_cpu_kdtree_free(mknn_cpu_kdtree* t);
int mknn_cpu_kdtree_knn(const mknn_cpu_kdtree* t, const float* q, int64_t nq, int32_t q_stride,
                        int32_t k, const int32_t* m, int32_t m_scalar, int32_t* out_idx,
                        float* out_d2, int32_t sorted, int32_t threads);

/* Algorithms 1 and 2 over a successor table in CSR form (rowp[n+1] int64,
 * succ[E] int32, each row ascending). counters: NULL or int64[nq * 8] per
 * query: rows opened, entries read, coordinates read, transition sites,
 * offers below the k-th key, offers already in N, insertions, sum of
 * insertion positions. */
int mknn_cpu_dpknn(const float* xyz, int64_t n, const int64_t* rowp, const int32_t* succ,
                   const float* q, int64_t nq, int32_t q_stride, int32_t k, const int32_t* m,
                   int32_t m_scalar, int32_t* out_idx, float* out_d2, int64_t* counters,
                   int32_t sorted, int32_t threads);

/* Hardware threads of this host. */
int32_t mknn_cpu_threads(void);

#ifdef __cplusplus
}
#endif
