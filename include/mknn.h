/*
 * mknn.h - C ABI of the GB300 Manifold k-NN query library.
 *
 * The library answers exact k-nearest-neighbour queries against a point
 * set P = {p_1..p_n} ordered by insertion ("birth") time, optionally
 * restricted to a prefix P_{1:m} (Manifold k-NN, Sec. 3-4). A host-side
 * builder makes the successor table once (Sec. 3: j is in L_i iff p_j is a
 * Delaunay neighbour of p_i in DT(P_{1:j})); queries then run on the GPU:
 * the successor-list descent of Algorithm 1 followed by the expansion of
 * Algorithm 2, whose correctness is Theorem 1.
 *
 * Conventions
 *  - Ranks are 0-based insertion ranks: the paper's p_i is rank i-1.
 *    Results are ranks; mknn_cloud_order maps ranks to input indices.
 *  - Squared Euclidean distances, float32 coordinates.
 *  - Ties are broken by the lower rank (Eq. 2 keeps the earlier site).
 *  - Every function returns a status; none throws. mknn_last_error()
 *    gives a message for the calling thread's last failure.
 *  - Pointers documented as "device" must be CUDA device memory of the
 *    current device (e.g. a torch tensor's data_ptr()); "host" pointers
 *    are ordinary host memory (pinned memory makes copies faster).
 *  - Streams are CUDA stream handles (cudaStream_t); NULL is the legacy
 *    default stream. Device work is asynchronous on the given stream.
 *  - Thread safety: distinct clouds may be used from distinct threads; a
 *    cloud may be queried concurrently, but mknn_cloud_free must not race
 *    with its use.
 */
#ifndef MKNN_H_
#define MKNN_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* mknn_stream_t; /* same type as cudaStream_t */

typedef enum {
  MKNN_OK = 0,
  MKNN_EINVAL = 1,      /* bad argument (k, m, sizes, NULL pointer, NaN coords) */
  MKNN_ENOMEM = 2,      /* host or device allocation failed */
  MKNN_ECUDA = 3,       /* a CUDA runtime call failed */
  MKNN_EBUSY = 4,       /* object in use (e.g. cloud referenced by a server) */
  MKNN_ETIMEOUT = 5,    /* a bounded wait expired */
  MKNN_EDEGENERATE = 6, /* input too degenerate to build (all points coplanar) */
  MKNN_EIO = 7          /* file could not be read or written, or bad format */
} mknn_status;

/* Largest k accepted by the query entry points. */
#define MKNN_MAX_K 128

typedef struct mknn_cloud mknn_cloud;

/* Message describing the calling thread's most recent failure ("" if none).
 * The pointer stays valid until the next library call on the thread. */
const char* mknn_last_error(void);

/* ------------------------------------------------------------------ build
 * mknn_build: the successor table of Sec. 3, made by an incremental 3D
 * Delaunay triangulation with exact predicates on the host.
 *   xyz    host, n*3 float32, input order (row i = point i).
 *   n      number of points, 1 <= n < 2^31 - 16.
 *   order  host int64[n] or NULL. order[r] = input index of the point
 *          inserted at rank r (a permutation of 0..n-1). NULL = identity.
 *   opts   NULL for defaults.
 *   out    receives a new cloud owned by the caller (mknn_cloud_free).
 * Errors: EINVAL (NULL, n out of range, non-finite coordinate, order not a
 * permutation), EDEGENERATE (all points coplanar and n > 4096), ENOMEM.
 * The caller's arrays are copied; they can be freed on return. Nothing is
 * placed on the device until mknn_cloud_upload. Thread-safe for distinct
 * outputs (builds of several clouds may run in parallel threads). */
typedef struct {
  int32_t keep_tets; /* nonzero: keep the final tetrahedra (mknn_cloud_tets) */
  int32_t dynamic;   /* nonzero: keep the triangulation so that points can be
                        appended later (mknn_cloud_append); the points must
                        span 3D (EDEGENERATE otherwise) */
  int32_t reserved[6];
} mknn_build_opts;

mknn_status mknn_build(const float* xyz, int64_t n, const int64_t* order,
                       const mknn_build_opts* opts, mknn_cloud** out);

/* mknn_insertion_order: a birth order for mknn_build (Sec. 5 compares
 * insertion orders; the order changes the successor lists, hence build
 * time and query work, never the answers). order_out receives n input
 * indices, order_out[r] = the point to insert at rank r.
 *   MKNN_ORDER_RANDOM         seeded uniform permutation.
 *   MKNN_ORDER_BRIO_HILBERT   the seeded permutation cut into rounds of
 *                             doubling size (the last holds half the points,
 *                             the first at most 64), each round sorted along
 *                             a 3D Hilbert curve over the bounding box.
 *   MKNN_ORDER_FARTHEST_POINT each next point is the one farthest from those
 *                             already taken (ties to the lower input index),
 *                             from input index 0; seed unused.
 * Host only. Errors: EINVAL (NULL, n < 0, non-finite coordinate, unknown
 * kind), ENOMEM. */
#define MKNN_ORDER_RANDOM 0
#define MKNN_ORDER_BRIO_HILBERT 1
#define MKNN_ORDER_FARTHEST_POINT 2
mknn_status mknn_insertion_order(const float* xyz, int64_t n, int32_t kind, uint64_t seed,
                                 int64_t* order_out);

/* mknn_cloud_from_table: a cloud from an explicit successor table instead
 * of the builder. Any table whose rows are supersets of the true successor
 * lists gives exact results (extra entries are extra candidates), e.g. the
 * complete table L_i = {i+1..n-1}.
 *   xyz_ranked host float32[n*3], rank order.
 *   rowp       host int64[n+1], rowp[0] = 0, nondecreasing, rowp[n] = E.
 *   succ       host int32[E]; row i = succ[rowp[i]..rowp[i+1]), strictly
 *              ascending, every entry in (i, n).
 * Errors: EINVAL (shape or ordering violated, E >= 2^31), ENOMEM. */
mknn_status mknn_cloud_from_table(const float* xyz_ranked, int64_t n, const int64_t* rowp,
                                  const int32_t* succ, mknn_cloud** out);

/* Copies coordinates (as float4 x,y,z,0 in rank order) and the CSR table to
 * the current device, and builds there a second copy of the successor
 * entries with each entry's site inlined (float4 x, y, z, rank), which the
 * query kernels read with one load per entry. Idempotent; synchronous with
 * respect to the host (the copies complete before return). Device bytes:
 * 24 n + 20 E plus a few words of status (a dynamic cloud also reserves
 * room for appends: a quarter more sites and entries, at least 4096 sites
 * and 65536 entries). A cloud without appends whose longest successor list
 * has 4096 entries or more also gets a box tree over every list of 256
 * entries or more (an index for the one-warp
 * query kernel, which searches such a list through its tree instead of
 * reading it in rank order, with the same result; Algorithms 1-2 need
 * only the entries that can be strictly closer than the current site, or
 * below the k-th key): 4 n bytes plus about 17 bytes per entry of those
 * lists (see mknn_cloud_trees). Errors: ENOMEM, ECUDA. */
mknn_status mknn_cloud_upload(mknn_cloud* cloud, mknn_stream_t stream);

/* mknn_cloud_append: inserts `count` new points after the existing ones,
 * in the given order (their birth times follow every existing point:
 * ranks n, n+1, ..., input indices n, n+1, ... for mknn_cloud_order). The
 * cloud must have been built with mknn_build_opts.dynamic. The insertion
 * continues the build's triangulation (Sec. 3), so the table afterwards is
 * the one a build over all the points in this order would make: every
 * existing list gains the new ranks whose insertion made them Delaunay
 * neighbours, and each new rank starts an empty list. Queries with m <= the
 * old n therefore see exactly the old cloud (Sec. 4.2).
 *   xyz    host float32[count*3].
 *   stream used for the device update when the cloud is uploaded.
 * On the device only the changed rows move: a row that outgrows its room is
 * copied to the top of an append-only entry arena, which (like the site
 * arrays) grows by reallocation when full. The call synchronises the
 * stream. Queries on other streams must not overlap it, batch plans made
 * before it must be recreated (mknn_batch_run returns EINVAL), and a cloud
 * held by a server cannot be appended to (EBUSY).
 * Errors: EINVAL (not dynamic, NULL, non-finite coordinate, n would exceed
 * 2^31 - 16, an earlier append failed), EBUSY, ENOMEM, ECUDA. A failure
 * inside the insertion itself leaves the cloud's points and table as they
 * were before the call, and the cloud takes no further appends. */
mknn_status mknn_cloud_append(mknn_cloud* cloud, const float* xyz, int64_t count,
                              mknn_stream_t stream);

/* mknn_cloud_compact: lays a dynamic cloud's device table out afresh (rows
 * in rank order, each followed by two empty slots), dropping the copies
 * that appends left behind. Appends do this on their own once the table has
 * grown 40% beyond a fresh layout; calling it after a burst of appends
 * brings queries back to the speed of a fresh upload. Synchronises the
 * stream; the same rules as for mknn_cloud_append apply (no overlapping
 * queries on other streams; the entry arrays move, so batch plans made
 * before it must be recreated). Errors: EINVAL (not dynamic or not
 * uploaded), ENOMEM, ECUDA. */
mknn_status mknn_cloud_compact(mknn_cloud* cloud, mknn_stream_t stream);

/* Releases device memory of the cloud (keeps the host copy). */
mknn_status mknn_cloud_release_device(mknn_cloud* cloud);

/* Frees the cloud (host and device). EBUSY if a server still holds it. */
mknn_status mknn_cloud_free(mknn_cloud* cloud);

/* Sizes: n, E (total successor entries) and device bytes (0 if not
 * uploaded). Any output pointer may be NULL. */
mknn_status mknn_cloud_info(const mknn_cloud* cloud, int64_t* n, int64_t* E, size_t* dev_bytes);

/* Box trees of the device copy (mknn_cloud_upload): number of trees and
 * the entries of the lists they cover (0 and 0 before upload, for a cloud
 * built for appends, and when no list has 4096 entries). Either output may
 * be NULL. The paper has no such index: it reads every list in rank order. */
mknn_status mknn_cloud_trees(const mknn_cloud* cloud, int64_t* trees, int64_t* entries);

/* order_out host int64[n]: rank -> input index. */
mknn_status mknn_cloud_order(const mknn_cloud* cloud, int64_t* order_out);

/* Copies the table to host arrays: xyz_ranked float[3n], rowp int64[n+1],
 * succ int32[E]. Any pointer may be NULL to skip it. */
mknn_status mknn_cloud_table(const mknn_cloud* cloud, float* xyz_ranked, int64_t* rowp,
                             int32_t* succ);

/* Build statistics. */
typedef struct {
  int64_t n, entries, duplicates, degenerate_prefix, tets_final;
  int64_t walk_steps, conflict_tests;
  int64_t orient_calls, orient_exact, insphere_calls, insphere_exact;
  double build_seconds;
} mknn_build_stats;
mknn_status mknn_cloud_stats(const mknn_cloud* cloud, mknn_build_stats* out);

/* Final finite tetrahedra (rank quadruples, positively oriented) of a cloud
 * built with keep_tets. tets may be NULL to query *count only. */
mknn_status mknn_cloud_tets(const mknn_cloud* cloud, int32_t* tets, int64_t* count);

/* Checkpoint: versioned binary file with n, E, coordinates (rank order),
 * rank order and the CSR table. load gives a host-only cloud. */
mknn_status mknn_cloud_save(const mknn_cloud* cloud, const char* path);
mknn_status mknn_cloud_load(const char* path, mknn_cloud** out);

/* ------------------------------------------------------------------ query
 * mknn_knn: exact k-NN for a batch of queries (Algorithms 1 and 2, with the
 * prefix bound of Sec. 4.2): one query per GPU thread with its candidate
 * list in shared memory, or a group of lanes per query on clouds with very
 * long successor lists and for launches too small to fill the GPU.
 *   cloud     uploaded cloud.
 *   q         device float32, nq rows of q_stride floats (x, y, z first).
 *   nq        number of queries, 0 <= nq < 2^31 - 1.
 *   q_stride  floats per query row, >= 3 (3 = packed xyz, 4 = float4).
 *   k         1 <= k <= MKNN_MAX_K.
 *   m         device int32[nq] per-query prefix bounds, or NULL.
 *   m_scalar  used when m is NULL: 0 means n, otherwise 1 <= m_scalar <= n.
 *   out_idx   device int32[nq*k]: ranks in [0, m), row-major per query.
 *   out_d2    device float32[nq*k]: squared distances (float32 arithmetic).
 *   stream    CUDA stream.
 * Each row is sorted by (distance, rank). If min(k, m) < k the row is padded
 * with (-1, +inf). A per-query m outside [1, n] yields a padded row and
 * sets the cloud's error flag (mknn_cloud_check). Results equal the float64
 * brute force up to the order of distances that differ by less than about
 * 3e-7 relative (float32 rounding). Errors: EINVAL, ECUDA. */
mknn_status mknn_knn(const mknn_cloud* cloud, const float* q, int64_t nq, int32_t q_stride,
                     int32_t k, const int32_t* m, int32_t m_scalar, int32_t* out_idx,
                     float* out_d2, mknn_stream_t stream);

/* Tuning knobs of one query launch; zero-initialise for defaults. */
typedef struct {
  int32_t lanes;        /* lanes per query: 0 = default (1, or 32 from
                           k = 48 up, or more for small batches and
                           clouds with very long successor lists - for
                           k > 8 when the cloud has box trees), or
                           1, 4, 8, 16, 32 (4 and 8 hold k <= 64; one
                           lane above 64 needs placement 2 and no
                           counters) */
  int32_t sort;         /* query locality sort: 0 = default (on from 4096
                           queries), 1 = on, -1 = off */
  int32_t blocks_per_sm;/* 0 = default: one block per 256 queries for the
                           one-lane kernel (the hardware refills SMs as
                           blocks end), as many as fit for the others;
                           > 0 = at most this many resident blocks per SM,
                           each thread looping over queries */
  int32_t* counters;    /* device int32[4*nq] or NULL: per query rows opened,
                           successor entries read, coordinates read and
                           transition sites (descent moves + 1) */
  void* workspace;      /* device scratch or NULL (library-managed) */
  size_t workspace_bytes;
  const int32_t* order; /* device int32[nq] processing order (e.g. from
                           mknn_query_order) or NULL; overrides sort */
  int32_t placement;    /* where the candidate list lives, for 1 and 32
                           lanes: 0 = default (2), 1 = registers (one
                           lane: per thread; 32 lanes: spread over the
                           warp), 2 = shared memory (one lane: a list per
                           thread; 32 lanes: one list per warp, not with
                           counters); 4, 8, 16 lanes use registers */
  int32_t reserved[3];
} mknn_knn_opts;

/* Locality order of a query batch, the one mknn_knn_ex applies when sort
 * is on: queries counting-sorted by the Morton index of their cell in a
 * 64^3 grid over the queries' own bounding box. Changes only the
 * processing order, never a result.
 *   perm_out   device int32[nq]: query indices in processing order.
 *   workspace  device scratch of mknn_query_order_workspace_size(nq) bytes,
 *              or NULL (library-managed, grown on demand).
 * Errors: EINVAL, ENOMEM, ECUDA. */
size_t mknn_query_order_workspace_size(int64_t nq);
mknn_status mknn_query_order(const mknn_cloud* cloud, const float* q, int64_t nq, int32_t q_stride,
                             int32_t* perm_out, void* workspace, size_t workspace_bytes,
                             mknn_stream_t stream);

/* Scratch bytes mknn_knn_ex needs for nq queries with the given options:
 * the locality sort's (none with an order or the sort off) and 4 bytes per
 * query (plus 256) for the hand-over below. */
size_t mknn_knn_workspace_size(int64_t nq, const mknn_knn_opts* opts);

/* mknn_knn with explicit options (opts may be NULL). A caller workspace of
 * at least mknn_knn_workspace_size bytes avoids library allocations.
 * One lane per query with the list in shared memory on a cloud with box
 * trees (mknn_cloud_trees): the queries that would read a list with a tree
 * through are handed over to the one-warp kernel (32 lanes, shared memory),
 * which walks the tree; a second launch on the stream, same results. A
 * caller workspace too small for the hand-over (but not for the sort)
 * leaves it out: the lists are then read in rank order. */
mknn_status mknn_knn_ex(const mknn_cloud* cloud, const float* q, int64_t nq, int32_t q_stride,
                        int32_t k, const int32_t* m, int32_t m_scalar, int32_t* out_idx,
                        float* out_d2, const mknn_knn_opts* opts, mknn_stream_t stream);

/* mknn_knn_sites: same-manifold queries, where each query is one of the
 * cloud's own sites (e.g. normal estimation, Sec. 1 and Sec. 6, or a probe
 * at a site across prefixes, Sec. 5). Query i is the site of rank
 * sites[i]; the rest is mknn_knn: the same Algorithms 1 and 2 with the
 * prefix bound of Sec. 4.2, so the site itself is returned at distance 0
 * when its rank is below m (after any earlier exact duplicate).
 *   sites     device int32[nq] ranks in [0, n). A rank outside it yields a
 *             padded row and sets the cloud's error flag, as a bad m does.
 *   m, m_scalar, k, out_idx, out_d2, stream: as mknn_knn.
 *   opts      as mknn_knn_ex (NULL for defaults), except that `order` must
 *             be NULL (the sites are sorted by locality like queries).
 * Scratch: 20 bytes per query (coordinates and bounds gathered from the
 * cloud) plus mknn_knn_workspace_size; a caller workspace must hold
 * mknn_knn_sites_workspace_size bytes. Errors: EINVAL, ENOMEM, ECUDA. */
size_t mknn_knn_sites_workspace_size(int64_t nq, const mknn_knn_opts* opts);
mknn_status mknn_knn_sites(const mknn_cloud* cloud, const int32_t* sites, int64_t nq, int32_t k,
                           const int32_t* m, int32_t m_scalar, int32_t* out_idx, float* out_d2,
                           const mknn_knn_opts* opts, mknn_stream_t stream);

/* End-to-end form with HOST buffers: copies queries (and m) to the device,
 * runs the query, copies results back, in chunks pipelined over two
 * streams. Returns after the results are in the host buffers.
 *   q host float32 [nq*q_stride]; m host int32[nq] or NULL;
 *   out_idx host int32[nq*k]; out_d2 host float32[nq*k].
 * Pinned host memory is used directly; pageable memory works but is
 * slower. Errors: EINVAL, ENOMEM, ECUDA. */
mknn_status mknn_knn_host(const mknn_cloud* cloud, const float* q, int64_t nq, int32_t q_stride,
                          int32_t k, const int32_t* m, int32_t m_scalar, int32_t* out_idx,
                          float* out_d2, mknn_stream_t stream);

/* mknn_knn_noalloc: mknn_knn (with the locality sort) that allocates no
 * memory at all during the call. The paper has no counterpart; this is an
 * interface for callers that cannot allocate device memory while serving
 * queries, e.g. a process whose memory pool already holds all the device
 * memory it may use (so an allocation would fail), or a latency-bound
 * loop that cannot afford the synchronisation cudaMalloc/cudaFree can
 * cause. Its scratch is a fixed device array inside the library
 * (9 MiB + 1.75 KiB) that every GPU using this entry point holds until the
 * process exits.
 *   Arguments, layout, results and errors are those of mknn_knn, except:
 *   nq must be at most mknn_knn_noalloc_max_queries() (2^20); larger nq
 *   returns EINVAL with a message naming the limit (split the batch).
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture. All calls share the one array: calls whose
 * work overlaps on the GPU (other streams or host threads) race on it and
 * must be serialised by the caller. Nothing carries over between calls:
 * the parts that must start at zero are cleared by each call. */
mknn_status mknn_knn_noalloc(const mknn_cloud* cloud, const float* q, int64_t nq, int32_t q_stride,
                             int32_t k, const int32_t* m, int32_t m_scalar, int32_t* out_idx,
                             float* out_d2, mknn_stream_t stream);
int64_t mknn_knn_noalloc_max_queries(void);

/* Reads and clears the cloud's device error flags (synchronises the
 * device). Bit 0: a per-query m was outside [1, n], or a site rank given to
 * mknn_knn_sites was outside [0, n). */
mknn_status mknn_cloud_check(const mknn_cloud* cloud, int32_t* flags);

/* ------------------------------------------------------- batched queries
 * Many requests, each on its own cloud with its own k and m, answered by
 * persistent kernel launches, one per kernel variant present, each draining
 * its own device work queue (items of a few rounds of one request's
 * queries). Per request the kernel variant
 * (lanes per query, candidate slots) comes from the tuning table, filled by
 * mknn_batch_tune, or a default. A plan captures its launches (query
 * locality sorts + the persistent kernel) in a CUDA graph and replays it.
 * The paper answers queries one at a time on a CPU (Sec. 5.1); batching
 * many clouds into a few launches is this library's GPU form of the same
 * per-query Algorithms 1-2, with identical results. */
typedef struct {
  const mknn_cloud* cloud; /* uploaded on the current device */
  const float* q;          /* device float32, nq rows of q_stride floats */
  int64_t nq;              /* 0 <= nq < 2^31 - 256 */
  int32_t q_stride;        /* >= 3 */
  int32_t k;               /* 1..MKNN_MAX_K */
  const int32_t* m;        /* device int32[nq] or NULL */
  int32_t m_scalar;        /* when m is NULL: 0 = n, else 1..n */
  int32_t* out_idx;        /* device int32[nq*k] */
  float* out_d2;           /* device float32[nq*k] */
} mknn_batch_req;

typedef struct {
  int32_t lanes;          /* 0 = tuned per request, else 1, 4, 8, 16 or 32 for all */
  int32_t sort;           /* 0 = sort requests with >= 4096 queries, 1 = all, -1 = none */
  int32_t item_rounds;    /* rounds of the group width per work item (0 = 1) */
  int32_t blocks_per_sm;  /* 0 = occupancy limit */
  int32_t graph;          /* 0 = capture a CUDA graph (default), -1 = plain launches */
  int32_t placement;      /* with lanes set: 0 = that width's default, 1 = registers,
                             2 = shared memory (only 32 lanes have both: a list
                             per warp in shared memory, or spread over the
                             warp's registers); with lanes 0: tuned per request */
  int32_t reserved[6];
} mknn_batch_opts;

typedef struct mknn_batch mknn_batch;

/* Makes a plan: validates the requests, picks each request's variant,
 * cuts the work items, allocates the plan's device memory (queue, request
 * table, sort scratch) and captures the graph. The request pointers are
 * baked into the plan: the buffers must stay valid while the plan is used;
 * their contents may change between runs. Errors: EINVAL, ENOMEM, ECUDA. */
mknn_status mknn_batch_create(const mknn_batch_req* reqs, int32_t nreq,
                              const mknn_batch_opts* opts, mknn_batch** out);
/* Enqueues one run of the plan on the stream (asynchronous). Runs of one
 * plan must not overlap on the device (they share the queue counter).
 * EINVAL if a request's cloud was appended to after the plan was made. */
mknn_status mknn_batch_run(mknn_batch* plan, mknn_stream_t stream);
/* Lanes chosen per request (int32[nreq], may be NULL), work items, and the
 * blocks of the plan's persistent launches (one launch per kernel variant
 * present, summed). */
mknn_status mknn_batch_info(const mknn_batch* plan, int32_t* lanes, int64_t* items, int32_t* grid);
/* Candidate-list placement chosen per request (int32[nreq]; 2 = shared
 * memory, 1 = registers), beside the lanes mknn_batch_info reports. */
mknn_status mknn_batch_placement(const mknn_batch* plan, int32_t* placement);
mknn_status mknn_batch_free(mknn_batch* plan);
/* One-shot: create (without a graph), run, synchronise the stream, free. */
mknn_status mknn_knn_batch(const mknn_batch_req* reqs, int32_t nreq, const mknn_batch_opts* opts,
                           mknn_stream_t stream);

/* Autotuner: for every distinct (k, floor(log2 n), floor(log2(1 + longest
 * successor list))) among the requests - the last separates clouds with
 * hub rows (nearly coplanar sites), whose queries cost far more -
 * times each kernel variant and list placement: one query per thread with
 * a shared-memory list (lanes 1), a group of 4, 8, 16 or 32 lanes with the
 * list in registers, or one warp per query with the list in shared memory
 * (lanes 32, placement 2). Each candidate runs as the persistent plan
 * variant a plan would run (a one-request plan, no graph, best of 2 after a
 * warm-up) on max(sample, 2 x SMs x 2048) queries of that request (tiled
 * when it has fewer); the fastest (lanes, placement) goes into the
 * process-wide tuning table. Plans, plain launches and the server take the
 * table's entry, widened to more lanes when a launch is too small to fill
 * the GPU one query per thread. If the environment variable MKNN_TUNE_LOG
 * names a file, one line per timed candidate (k, n, hub bucket, sample,
 * lanes, placement, ms) is appended to it. Synchronises the stream.
 * Errors: EINVAL, ENOMEM, ECUDA. */
mknn_status mknn_batch_tune(const mknn_batch_req* reqs, int32_t nreq, int64_t sample,
                            mknn_stream_t stream);
/* Tuning table as text ("k log2n hub lanes placement" per line; a line
 * without placement means that width's default); load merges into the
 * table, clear empties it (the untuned defaults apply again). */
mknn_status mknn_tune_save(const char* path);
mknn_status mknn_tune_load(const char* path);
mknn_status mknn_tune_clear(void);

/* ---------------------------------------------------------------- serving
 * A request loop over resident clouds with continuous batching: a
 * scheduler thread packs pending requests (any cloud, k and m) into the
 * next launch of the persistent kernel as soon as a launch slot and
 * device memory are free; several launches are in flight on separate
 * streams, so requests that arrive while others run are admitted and
 * their copies and kernels overlap on the device. Admission is by device
 * memory: each request needs nq * (12 + 8 k) bytes of the staging budget
 * while it is in flight. Latency = completion time - submit time. */
typedef struct {
  int32_t slots;            /* launches in flight (streams), 0 = 3 */
  int32_t plain;            /* 1 = baseline mode: each request alone, in
                               arrival order, with mknn_knn on one stream */
  size_t mem_budget;        /* device staging bytes, 0 = 3 GiB */
  int64_t max_batch_queries;/* queries packed into one launch, 0 = 2^17 (a larger
                               request still runs, alone) */
  int32_t lanes;            /* 0 = tuned/default per request */
  int32_t reserved[7];
} mknn_server_opts;

typedef struct {
  int32_t cloud;            /* id from mknn_server_add_cloud */
  int32_t k;                /* 1..MKNN_MAX_K */
  int32_t m;                /* prefix bound for every query: 0 = n, else 1..n */
  int32_t reserved;
  const float* q;           /* HOST float32[nq*3], valid until the request is done */
  int64_t nq;               /* 1 <= nq < 2^31 - 256 */
  int32_t* out_idx;         /* HOST int32[nq*k], written when done */
  float* out_d2;            /* HOST float32[nq*k] */
} mknn_request;

typedef struct {
  int64_t submitted, completed, failed, queries, launches;
  double elapsed_s;         /* first submit to last completion */
  double qps;               /* completed queries / elapsed_s */
  double p50_ms, p99_ms, mean_ms, max_ms;
  double mean_requests_per_launch;
  /* GPU time of each phase of a launch, summed over completed launches
   * (stream time between events; launches on different slots overlap):
   * host-to-device copies of the queries (and the pack's request table),
   * kernels (locality sorts + k-NN), device-to-host copies of the results */
  double h2d_ms, kernel_ms, d2h_ms;
} mknn_serving_stats;

typedef struct mknn_server mknn_server;

/* Starts the scheduler thread on the current device. Errors: ENOMEM, ECUDA. */
mknn_status mknn_server_create(const mknn_server_opts* opts, mknn_server** out);
/* Makes a cloud resident (uploads it if needed) and holds it: freeing it
 * returns EBUSY until the server is destroyed. *id receives its index. */
mknn_status mknn_server_add_cloud(mknn_server* s, mknn_cloud* cloud, int32_t* id);
/* Queues a request; *ticket identifies it. EINVAL for a bad request,
 * ENOMEM if it alone exceeds the memory budget. Thread-safe. */
mknn_status mknn_server_submit(mknn_server* s, const mknn_request* req, uint64_t* ticket);
/* *state: 0 pending, 1 done, or minus a status code if it failed. */
mknn_status mknn_server_poll(mknn_server* s, uint64_t ticket, int32_t* state);
/* Waits (at most timeout_s seconds) until every submitted request is done;
 * ETIMEOUT if the wait runs out. */
mknn_status mknn_server_drain(mknn_server* s, double timeout_s);
mknn_status mknn_server_stats(mknn_server* s, mknn_serving_stats* out);
/* Completed requests' latencies in ms, in ticket order; *count = number
 * written (at most cap). Resets nothing. */
mknn_status mknn_server_latencies(mknn_server* s, double* ms, int64_t cap, int64_t* count);
/* Clears the statistics and latency records (not the queue). */
mknn_status mknn_server_reset_stats(mknn_server* s);
/* Drains (up to timeout_s), stops the thread, releases the held clouds. */
mknn_status mknn_server_destroy(mknn_server* s, double timeout_s);

/* ------------------------------------------------------------ diagnostics
 * Exact geometric predicates used by the builder (float32 inputs):
 * orient3d = sign det[b-a; c-a; d-a]; insphere = +1 inside, 0 on, -1
 * outside the sphere through a, b, c, d (positively oriented). */
int32_t mknn_orient3d(const float* a, const float* b, const float* c, const float* d);
int32_t mknn_insphere(const float* a, const float* b, const float* c, const float* d,
                      const float* e);
/* Same predicates without the floating-point filter (exact stage only). */
int32_t mknn_orient3d_exact(const float* a, const float* b, const float* c, const float* d);
int32_t mknn_insphere_exact(const float* a, const float* b, const float* c, const float* d,
                            const float* e);

/* Brute-force check of a cloud built with keep_tets (O(tets * n), for tests
 * on small inputs): *bad_orient = tetrahedra that are not positively
 * oriented, *bad_sphere = (tetrahedron, site) pairs with the site strictly
 * inside the circumsphere. Both 0 for a valid Delaunay triangulation. */
mknn_status mknn_cloud_validate(const mknn_cloud* cloud, int64_t* bad_orient, int64_t* bad_sphere);

/* Position of the cell (x, y, z) of a 2^bits-per-axis grid along the 3D
 * Hilbert curve that MKNN_ORDER_BRIO_HILBERT sorts by (1 <= bits <= 21;
 * 0 otherwise). */
uint64_t mknn_hilbert_index3(uint32_t x, uint32_t y, uint32_t z, int32_t bits);

/* Read-bandwidth probe: reads `bytes` from the device buffer `buf`
 * `passes` times with 16-byte loads through L2 (bypassing L1), spread over
 * every SM, and XORs what it read into *sink (device, 4 bytes). Timed with
 * events around it, bytes * passes / time is the read bandwidth of the
 * level that holds buf: L2 for a buffer well below its size, HBM for one
 * well above. Used to set the L2 roofline of the query kernels (their
 * working set is mostly L2-resident). buf 16-byte aligned, bytes a non-zero
 * multiple of 16, passes >= 1; otherwise EINVAL. Asynchronous on stream. */
mknn_status mknn_read_probe(const void* buf, size_t bytes, int32_t passes, uint32_t* sink,
                            mknn_stream_t stream);

/* Library version string. */
const char* mknn_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MKNN_H_ */
