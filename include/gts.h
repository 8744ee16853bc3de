/*
 * gts.h -- C ABI of a GB300 (sm_103a) library for exact metric range and
 * k-nearest-neighbour search over a GTS index: a pivot-based tree whose nodes
 * are flattened into a node list and a table list (Zhu et al., "GTS:
 * GPU-based Tree Index for Fast Similarity Search", PACMMOD 2024,
 * arXiv 2404.00966).
 *
 * Conventions for every entry point
 *  - No C++ exception crosses this boundary; every call returns a gts_status.
 *    On any status other than GTS_OK, gts_last_error() returns a message
 *    (thread-local, valid until the next call on the same thread), outputs are
 *    left untouched and an index is left as it was before the call.
 *  - All device work runs on the CUDA stream given in the options (NULL = the
 *    legacy default stream) of the device that is current when the index is
 *    built.  Calls return after their results are complete (they synchronise
 *    that stream).
 *  - Input buffers stay owned by the caller and are only read.  A gts_objects
 *    with on_device = 1 holds device pointers of the current device; otherwise
 *    host pointers (pageable or pinned).  Per-query arrays (radii, k, seq)
 *    live on the same side as the queries.
 *  - Object ids are int64.  The objects of gts_build get ids 0 .. n-1 in input
 *    order; gts_insert hands out the next ids in order.  Total ids < 2^31.
 *  - A library built without a usable CUDA device fails every call with
 *    GTS_ECUDA.  There is no CPU fallback.
 *  - An index may be used by one thread at a time.
 */
#ifndef GTS_H
#define GTS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gts_index gts_index; /* opaque; owns all of its device memory */

typedef enum {
    GTS_OK = 0,
    GTS_EINVAL = 1,    /* malformed argument (NaN / negative radius, k <= 0, metric/object mismatch ...) */
    GTS_ENOMEM = 2,    /* a device or host allocation failed */
    GTS_ECUDA = 3,     /* a CUDA runtime error (message in gts_last_error) */
    GTS_ETIMEOUT = 4,  /* a bounded device wait ran out */
    GTS_ENOTFOUND = 5, /* gts_delete: one or more ids are unknown or already deleted (the others were applied) */
    GTS_EOVERFLOW = 6  /* a single query needs more memory than the configured budget allows */
} gts_status;

/* Distance metrics (Section 3, metric-space axioms; Table 2 of the paper).
 *  GTS_EDIT: unit-cost Levenshtein distance between byte strings.
 *  GTS_L1:   sum_i |q_i - x_i| over float32 vectors.
 *  GTS_L2:   sqrt(sum_i (q_i - x_i)^2) over float32 vectors. */
typedef enum { GTS_EDIT = 0, GTS_L1 = 1, GTS_L2 = 2 } gts_metric;

/* Verification precision for L2.  Both give the same result sets:
 *  GTS_PREC_FP32: FP32 CUDA-core distances, FP64 recheck of candidates whose
 *                 FP32 distance lies within a proven error bound of the radius
 *                 or of the running k-th distance.
 *  GTS_PREC_BF16: BF16 tensor-core distance tiles with FP32 accumulation and the
 *                 same FP64 recheck against a (wider) proven BF16 bound.
 * L1 has no product form for the tensor cores: with GTS_PREC_BF16 it runs the
 * same node-major tiles on the CUDA cores in FP32 (the arithmetic and the FP64
 * recheck of GTS_PREC_FP32, batched by node instead of by candidate); this
 * needs dim % 4 == 0 and 16-byte aligned query rows, else the plain path runs.
 * Edit distance ignores this field (exact int). */
typedef enum { GTS_PREC_FP32 = 0, GTS_PREC_BF16 = 1 } gts_precision;

/* A set of objects: vectors (dim > 0) or byte strings (dim == 0).
 *  vectors: data = float32[n * dim], row-major.
 *  strings: data = uint8 bytes, offsets = int64[n + 1], offsets[0] = 0,
 *           string i = data[offsets[i] .. offsets[i+1]); lengths <= 1024. */
typedef struct {
    int64_t n;
    int32_t dim;
    int32_t on_device;
    const void *data;
    const int64_t *offsets;
} gts_objects;

typedef struct {
    void *stream;          /* cudaStream_t */
    int64_t root_pivot;    /* index of the first (root) pivot in [0, n); -1 = drawn from seed (SplitMix64) */
    uint64_t seed;         /* seeds the root pivot of rebuilds and of root_pivot = -1 */
    int64_t cache_limit;   /* stream-update cache list capacity in objects; a larger cache triggers a
                              rebuild (Section 4.4); 0 = default 4096 */
} gts_build_opts;

typedef struct {
    void *stream;            /* cudaStream_t */
    int32_t precision;       /* gts_precision (L2 only) */
    int32_t result_on_device;/* 1: result arrays are device memory owned by the result */
    int64_t memory_budget;   /* bytes for intermediate frontier and candidate tables: size_GPU of the
                                two-stage scheduler (Section 5.1, Algorithm 4); 0 = default 64 GiB */
    const int64_t *seq;      /* optional per-query sequence number (same side as the queries): query i
                                sees the objects inserted before seq[i] and not deleted before seq[i].
                                NULL = the current state.  Must not precede the last rebuild. */
    int64_t *stats;          /* optional host int64[GTS_STATS_LEN] of counters, filled on return */
    double *stage_ms;        /* optional host double[GTS_STAGES_LEN]: device time per stage, measured with
                                CUDA events around every kernel launch of the call (adds the events' cost) */
} gts_query_opts;

/* Stages reported in gts_query_opts.stage_ms (and their launch counts in
 * stage_ms[GTS_STAGES_LEN/2 + stage] as a double). */
enum {
    GTS_STAGE_PIVOT_DIST = 0, /* query-to-pivot distances */
    GTS_STAGE_THRESHOLD = 1,  /* kNN threshold update */
    GTS_STAGE_EXPAND = 2,     /* node pruning and frontier compaction */
    GTS_STAGE_LEAF_SCAN = 3,  /* list-table lower-bound scan and candidate emission */
    GTS_STAGE_VERIFY = 4,     /* metric verification of candidates */
    GTS_STAGE_SELECT = 5,     /* kNN selection with FP64 rechecks */
    GTS_STAGE_OTHER = 6,      /* scans, sorts, regrouping, result assembly */
    GTS_STAGE_TILE = 7,       /* node-major tiles: leaf scan fused with the distance (filter) */
    GTS_STAGES = 8,
    GTS_STAGES_LEN = 16
};

/* Counters written to gts_query_opts.stats. */
enum {
    GTS_STAT_PIVOT_DIST = 0,   /* query-to-pivot distances computed */
    GTS_STAT_FRONTIER = 1,     /* (query, node) entries visited, all levels */
    GTS_STAT_SCANNED_ROWS = 2, /* table-list rows tested in the leaf scan */
    GTS_STAT_CANDIDATES = 3,   /* rows that passed the scan (verified with the metric) */
    GTS_STAT_RECHECKS = 4,     /* FP64 boundary rechecks */
    GTS_STAT_RESULTS = 5,      /* returned (query, object) pairs */
    GTS_STAT_GROUPS = 6,       /* query groups run by the two-stage scheduler */
    GTS_STAT_CACHE_ROWS = 7,   /* cache-list objects compared by brute force */
    GTS_STAT_LAUNCHES = 8,     /* kernels launched by the call */
    GTS_STAT_TILES = 9,        /* tile work items: 128-row blocks of last-level nodes */
    GTS_STAT_TILE_ENTRIES = 10,/* (query, last-level node) entries run against those blocks */
    GTS_STAT_TILE_PAIRS = 11,  /* (query, row) pairs whose distance the tiles computed */
    GTS_STAT_DENSE_PAIRS = 12, /* (query, pivot) distances computed as dense per-level matrices */
    GTS_STAT_DENSE_LAST = 13,  /* 1 if the last level ran as dense matrices (no entry list) */
    GTS_STATS_LEN = 14
};

/* Per-query answers in CSR form: the answers of query i are
 * ids/dist[offsets[i] .. offsets[i+1]).  Range answers are in ascending id
 * order; kNN answers in ascending (distance, id) order.  dist is float32; for
 * GTS_EDIT it holds the exact integer distance.  Allocated by the library
 * (host memory, or device memory when result_on_device = 1); release with
 * gts_result_free. */
typedef struct {
    int64_t nq;
    int64_t *offsets;
    int64_t *ids;
    float *dist;
    int32_t on_device;
    void *priv_;
} gts_result;

/* Build an index over `objects` (Section 4.3, Algorithms 1-3).
 *  n_pivots: number of pivot levels h; 0 = ceil(log_fanout(n + 1)) - 1 (Algorithm 1), at least 1.
 *  fanout:   node capacity N_c, 2 .. 64.
 *  The metric must match the objects (GTS_EDIT <-> strings).  n may be 0. */
gts_status gts_build(const gts_objects *objects, gts_metric metric, int n_pivots, int fanout,
                     const gts_build_opts *opts, gts_index **out);

/* Batched metric range query MRQ(q, r) = { o : d(q, o) <= r } (Section 3,
 * Definition 1; Section 5.1, Algorithm 4).  radii: float32[nq], >= 0 and not
 * NaN; edit-distance radii are read as floor(r). */
gts_status gts_range(gts_index *index, const gts_objects *queries, const float *radii,
                     const gts_query_opts *opts, gts_result *out);

/* Batched metric kNN query (Section 3, Definition 2; Section 5.2, Algorithm
 * 5).  k: int32[nq], each >= 1.  A query gets min(k, visible objects)
 * answers: the first ones in ascending (distance, id) order. */
gts_status gts_knn(gts_index *index, const gts_objects *queries, const int32_t *k,
                   const gts_query_opts *opts, gts_result *out);

/* Stream insert (Section 4.4): the objects go to the cache list and get ids
 * next_id, next_id + 1, ... written to ids_out (host int64[m], may be NULL).
 * When the cache list would exceed cache_limit the index is rebuilt first. */
gts_status gts_insert(gts_index *index, const gts_objects *objects, int64_t *ids_out);

/* Stream delete (Section 4.4): marks the objects with the given ids (host
 * int64[m]) deleted.  Unknown or already deleted ids are skipped and counted
 * in *n_missing (may be NULL); GTS_ENOTFOUND is returned if any was skipped. */
gts_status gts_delete(gts_index *index, const int64_t *ids, int64_t m, int64_t *n_missing);

/* Batch update (Section 4.4): insert `ins` (may be NULL), delete `del` (host
 * int64[m_del]) and rebuild the whole index at once.  New ids go to ids_out. */
gts_status gts_batch_update(gts_index *index, const gts_objects *ins, const int64_t *del, int64_t m_del,
                            int64_t *ids_out);

/* Rebuild the index from its visible objects (index and cache list). */
gts_status gts_rebuild(gts_index *index);

typedef struct {
    int64_t n_tree;      /* objects in the tree (including deleted ones not yet dropped) */
    int64_t n_cache;     /* objects in the cache list */
    int64_t n_live;      /* visible objects now */
    int64_t next_id;
    int64_t seq;         /* sequence number of the next update operation */
    int64_t rebuild_seq; /* sequence number of the last (re)build */
    int32_t h;           /* pivot levels */
    int32_t fanout;
    int32_t metric;
    int32_t dim;
    int64_t device_bytes;/* device memory held by the index */
} gts_index_info;

gts_status gts_info(const gts_index *index, gts_index_info *out);

/* Read back the tree (for checks).  level 0 .. h; arrays of fanout^level
 * entries, host memory, any may be NULL.  pivot (levels 0 .. h-1 only) is the
 * pivot's object id or -1 for an empty node; lo/hi are the node's distance
 * interval to its parent's pivot (level >= 1). */
gts_status gts_tree_level(const gts_index *index, int level, int64_t *pos, int64_t *size, float *lo,
                          float *hi, int64_t *pivot);

/* Read back the table list: ids = int64[n_tree] (row -> object id, leaf
 * order), table = float32[h * n_tree] (column l = distance of each row to its
 * level-l ancestor's pivot).  Host memory; either may be NULL. */
gts_status gts_table(const gts_index *index, int64_t *ids, float *table);

/* Copy a result's arrays into caller buffers (host or device pointers of the
 * index's device; either side of a result works): offsets = int64[nq + 1],
 * ids = int64[total], dist = float32[total], total = offsets[nq].  Any output
 * may be NULL.  Synchronous. */
gts_status gts_result_copy(const gts_result *result, int64_t *offsets, int64_t *ids, float *dist);

/* Launch parameters of the tile kernels and the kNN schedule, held per index.
 * No counterpart in the paper (its kernels are launched per level with fixed
 * shapes).  None of them changes a result: every setting returns the same
 * answers; they trade speed only.
 *  l1_queries: L1 tiles, queries per chunk (64 or 128; default 64).
 *  l1_packed:  L1 tiles, 1 = two coordinates per packed FP32 subtraction
 *              (default), 0 = scalar subtraction (same rounding).
 *  knn_phases: L1 tile kNN, 1 .. 3 launches over growing shares of the
 *              node blocks with tau_q lowered from the answer so far in
 *              between (default 3).
 *  probe_rows: kNN probe, object rows evaluated before the descent to bound
 *              the k-th distance, 0 .. 4096 (default 1024).
 *  tc_queries: BF16 tensor-core tiles for dim <= 128, queries per chunk:
 *              128 (two staging slots, default) or 96 (three slots).
 *  tuned:      output only: 1 once gts_autotune has run on the index. */
typedef struct {
    int32_t l1_queries;
    int32_t l1_packed;
    int32_t knn_phases;
    int32_t probe_rows;
    int32_t tuned;
    int32_t tc_queries;
    int32_t reserved_[2];
} gts_tuning;

/* Read / replace the index's tuning.  A query copies it when it starts, so a
 * change affects later queries only.  Out-of-range values: GTS_EINVAL. */
gts_status gts_get_tuning(gts_index *index, gts_tuning *out);
gts_status gts_set_tuning(gts_index *index, const gts_tuning *tuning);

/* Autotuner: run the sample batch `queries` (range with `radii`, or kNN with
 * `k`: exactly one of the two non-NULL, laid out as for gts_range / gts_knn)
 * `reps` times (1 .. 100) under each candidate setting, coordinate by
 * coordinate starting from the current one, keep the setting with the
 * smallest median wall time, store it in the index (tuned = 1) and return it
 * in *out (may be NULL).  opts as for the query calls (precision, stream,
 * budget); its stats / stage_ms are ignored.  The answers are discarded.  On
 * an error the index keeps the best setting found so far. */
gts_status gts_autotune(gts_index *index, const gts_objects *queries, const float *radii, const int32_t *k,
                        const gts_query_opts *opts, int32_t reps, gts_tuning *out);

/* Diagnostic, no counterpart in the paper: runs the tensor-core tile
 * primitives of the BF16 L2 path (TMA load with 128-byte swizzle, tcgen05.mma
 * with the accumulator in TMEM, tcgen05.ld) on one 128 x N x K product:
 * D[128, N] = bf16(A[128, K]) * bf16(B[N, K])^T in FP32.  A, B, D are host
 * row-major float32; N a multiple of 32 up to 256, K in {64, 128, 192, 256}.
 * a_tmem = 0: A is read from shared memory (TMA); 1: A is first written into
 * TMEM by tcgen05.st, one row per TMEM lane, as the tile kernel holds its node
 * blocks. */
gts_status gts_selftest_tc(const float *A, const float *B, int N, int K, int a_tmem, float *D);

/* Exact kNN over objects held on the device, by scanning every object, with
 * no device memory allocated by the call.  The paper has no counterpart: it is
 * for callers that cannot allocate while they query -- code running during a
 * CUDA graph capture, serving threads that must never enter the device
 * allocator (cudaMalloc may synchronise the device), hosts whose framework
 * owns all device memory.  The work happens in a fixed 16 MiB array of device
 * global memory that the library reserves when it is loaded (every GPU that
 * loads the library holds it until the process exits).
 *  objects: device float32[n * dim], row-major; object i has id i.
 *  queries: device float32[nq * dim].  metric: GTS_L1 or GTS_L2.
 *  k: 1 .. 32, and nq * k <= 2^20 (the array's capacity); larger calls fail
 *     with GTS_EINVAL and do nothing.
 *  ids, dist: device int64[nq * k], float32[nq * k]; query i's answers are at
 *     [i * k, i * k + k) in ascending (distance, id) order, distances from the
 *     same FP64 sums as the reference definition; when n < k the missing
 *     slots hold id -1 and distance +inf.
 *  stream: cudaStream_t (NULL = legacy default stream); returns when done.
 * The first call on a device looks up the array's device address with
 * cudaGetSymbolAddress; make that first call before any stream capture.
 * All calls share the array: calls whose kernels overlap on the GPU (other
 * streams, other host threads) race and must be serialised by the caller. */
gts_status gts_knn_scan_noalloc(const float *objects, int64_t n, int32_t dim, gts_metric metric,
                                const float *queries, int64_t nq, int32_t k, int64_t *ids, float *dist,
                                void *stream);

/* The same scan without the final stream synchronisation: the call only
 * enqueues its two kernels on `stream`, so it can be recorded into a CUDA
 * graph (stream capture) and replayed; results are ready when the stream's
 * work up to this point has finished.  Argument checks and errors as above
 * (an argument error enqueues nothing). */
gts_status gts_knn_scan_noalloc_async(const float *objects, int64_t n, int32_t dim, gts_metric metric,
                                      const float *queries, int64_t nq, int32_t k, int64_t *ids, float *dist,
                                      void *stream);

/* ---------------------------------------------------------------- serving
 * Continuous batching over one index (no counterpart in the paper; the paper
 * answers one batch at a time).  Requests are submitted one by one; worker
 * threads, each with its own CUDA stream, repeatedly form a batch of the
 * oldest pending requests of one kind and run it with the batched search, so
 * requests that arrive while others are on the GPU join the next batch and
 * several batches overlap on the device.  A request is admitted to a batch
 * only while the projected candidate-table bytes of all admitted requests
 * (visible objects x 37 bytes each) fit result_budget.  The index must not be
 * updated while a server runs on it. */
typedef struct gts_server gts_server;

typedef struct {
    int32_t max_batch;      /* requests per device batch; 0 = 1024 */
    int32_t n_streams;      /* worker threads and streams (batches in flight); 0 = 3 */
    int32_t precision;      /* gts_precision of every batch */
    int32_t reserved_;
    int64_t result_budget;  /* admission budget in bytes; 0 = 16 GiB */
    int64_t memory_budget;  /* size_GPU of each batch's two-stage scheduler; 0 = result_budget / n_streams */
} gts_serve_opts;

gts_status gts_serve_start(gts_index *index, const gts_serve_opts *opts, gts_server **out);

/* One request: kind 0 = range (param = radius), 1 = kNN (param = k).  query:
 * host float32[len], len = dim (vectors) or host bytes[len] (strings).  The
 * query is copied; the ticket identifies the request in gts_serve_wait. */
gts_status gts_serve_submit(gts_server *server, const void *query, int64_t len, int32_t kind, double param,
                            int64_t *ticket);

/* Wait for a request (timeout_ms < 0: no limit; GTS_ETIMEOUT if it is not
 * done in time, and the request stays pending).  On GTS_OK *out holds its
 * answers (nq = 1, host memory, free with gts_result_free) and *latency_ms
 * (may be NULL) the time from submit to the answers being ready. */
gts_status gts_serve_wait(gts_server *server, int64_t ticket, int32_t timeout_ms, gts_result *out,
                          double *latency_ms);

/* Counters: int64[4] = batches run, requests run, largest batch, largest
 * projected bytes in flight. */
gts_status gts_serve_stats(gts_server *server, int64_t *out4);

/* Finish the pending requests, join the workers, free the server. */
gts_status gts_serve_stop(gts_server *server);

void gts_result_free(gts_result *result);
void gts_free(gts_index *index);
const char *gts_last_error(void);
const char *gts_status_name(gts_status s);

#ifdef __cplusplus
}
#endif
#endif /* GTS_H */
