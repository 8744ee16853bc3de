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
 *  GTS_L2:   sqrt(sum_i (q_i - x_i)^2) over float32 vectors.
 *  GTS_COS:  the angle between float32 vectors, arccos(q.x / (|q| |x|)) in
 *            radians (Table 2's word cosine distance, read as the angular
 *            distance, a metric on directions).  Objects and queries must not
 *            be zero vectors (GTS_EINVAL).  Exact decisions use the FP64 key
 *            1 - c, c = q.x / (sqrt(|q|^2) sqrt(|x|^2)) from FP64 sums in
 *            coordinate order, clamped to [-1, 1]: range keeps key <= 1 -
 *            cos(r) (r clipped to [0, pi]), kNN orders by (key, id); the
 *            reported distance is arccos(1 - key).  The index is an L2 tree
 *            over the unit vectors (the chord 2 sin(angle / 2) orders like the
 *            angle), so every L2 kernel serves it. */
typedef enum { GTS_EDIT = 0, GTS_L1 = 1, GTS_L2 = 2, GTS_COS = 3 } gts_metric;

/* Verification precision for L2.  Both give the same result sets:
 *  GTS_PREC_FP32: FP32 CUDA-core distances, FP64 recheck of candidates whose
 *                 FP32 distance lies within a proven error bound of the radius
 *                 or of the running k-th distance.
 *  GTS_PREC_BF16: BF16 tensor-core distance tiles with FP32 accumulation and the
 *                 same FP64 recheck against a (wider) proven BF16 bound
 *                 (17 <= dim <= 448; vectors of at most 16 dimensions take the
 *                 node-major table scan, wider ones the FP32 path).
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
    int32_t flags;           /* GTS_QUERY_* bits; 0 = none */
    int32_t reserved_;
} gts_query_opts;

/* gts_query_opts.flags */
enum {
    /* Diagnostics: also count, into stats[GTS_STAT_TABLE_PASS], the (query,
     * row) pairs of the leaves that node pruning kept whose table lower bound
     * max_l |D_l(row) - d(q, p_l)| passes the query's threshold (Lemma 1 /
     * Lemma 2 over every pivot of the row's path) and that are visible: the
     * candidates a per-candidate verification must check, C_q summed over the
     * batch.  Costs an extra pass over those pairs; the answers are unchanged. */
    GTS_QUERY_COUNT_TABLE_PASS = 1,
    /* kNN: also return each answer's FP64 key in gts_result.key (L2: the
     * squared distance summed in FP64 in increasing coordinate order; L1: the
     * FP64 sum; edit: the integer distance), the key that orders answers with
     * ties broken by id -- what gts_merge_knn needs to merge shards exactly. */
    GTS_QUERY_KEYS = 2
};

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
    GTS_STAT_SCANNED_ROWS = 2, /* table-list rows read by the leaf scan (plain scan: per entry; node-major
                                  scan: each row block once) */
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
    GTS_STAT_TABLE_PASS = 14,  /* with GTS_QUERY_COUNT_TABLE_PASS: pairs passing the table bound; else -1 */
    GTS_STAT_SCAN_RECORDS = 15,/* node-major table scan: (query, row block) records tested (each read once) */
    GTS_STATS_LEN = 16
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
    double *key;    /* kNN with GTS_QUERY_KEYS: FP64 key per answer (same side and layout as dist); else NULL */
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

/* Persistence (checkpoint / resume of an index; the paper rebuilds instead,
 * Section 4.4).  gts_save writes the whole index state -- node list and table
 * list (Section 4.2), the objects in leaf order, the cache list and delete
 * marks with their sequence numbers (Section 4.4), the id bookkeeping and the
 * tuning -- to `path` (written to path + ".tmp", then renamed).  gts_load
 * reads it onto the current device (opts: stream and cache_limit are taken,
 * the rest ignored; may be NULL); the loaded index answers exactly as the
 * saved one did, at the same sequence numbers.  A file that is not a GTS
 * index, is truncated or is inconsistent gives GTS_EINVAL before any device
 * allocation. */
gts_status gts_save(const gts_index *index, const char *path);
gts_status gts_load(const char *path, const gts_build_opts *opts, gts_index **out);

/* Merge the answers of indexes over disjoint object sets (shards) for the
 * same nq queries into the answers one index over their union would give.
 * parts[p]: host results (on_device = 0); object id i of part p is global id
 * id_base[p] + i.
 *  gts_merge_knn: parts from gts_knn with GTS_QUERY_KEYS; query q keeps the
 *    first k[q] answers in ascending (FP64 key, global id) order (Definition
 *    2); out carries keys too.
 *  gts_merge_range: all answers of every part, ascending global id
 *    (Definition 1).
 * Host code: no device needed.  out is allocated by the library (host);
 * release it with gts_result_free. */
gts_status gts_merge_knn(const gts_result *const *parts, const int64_t *id_base, int32_t n_parts, const int32_t *k,
                         gts_result *out);
gts_status gts_merge_range(const gts_result *const *parts, const int64_t *id_base, int32_t n_parts, gts_result *out);

/* Multi-column queries (Section 5.2, closing remark): cols[0 .. m), 1 <= m
 * <= 64, are indexes over the same objects, one per column (object id i of every column
 * describes the same object), each with its own vector metric (L1, L2 or
 * angular; not edit distance).  The distance of object o from query q is
 * the sum over columns j, in column order and in FP64, of the column
 * distances d_j(q_j, o_j): sqrt(key) for L2, the key for L1, acos(1 - key)
 * (the C library's acos) for the angle, each key in the single-column
 * operation order of GTS_QUERY_KEYS.
 *  queries: m object sets, all with the same nq and on the same side (host,
 *    or device, copied to the host once; radii / k on the same side);
 *    queries[j] has column j's dim; row i of every set is query i.
 *  gts_multi_range: answers with sum <= radii[i] (finite, >= 0; Definition
 *    1), ascending id.  The candidates are the union of the columns' range answers at
 *    radius radii[i] / m rounded up (pigeonhole principle).
 *  gts_multi_knn: k[i] in 1 .. 1024; the first min(k[i], live objects)
 *    answers in ascending (sum, id) order (Definition 2), by Fagin's
 *    threshold algorithm over the columns' kNN answers with k' doubling from
 *    2 k[i] up to 1024; a query that is still open there sums every live
 *    object (a full scan).
 *  opts: precision and memory_budget pass to the column searches, which
 *    run concurrently, each on a host thread and a non-blocking stream of its
 *    own made for the call (opts->stream is not used; the call returns when
 *    all of it is done; an index given for several columns serves them in
 *    turn); seq must be NULL (the current state) and result_on_device 0;
 *    stats, when given, receives the column searches' counters summed over
 *    columns and rounds (GTS_STAT_LAUNCHES also counts the random-access
 *    kernels), GTS_STAT_RESULTS = the multi-column answers and
 *    GTS_STAT_TABLE_PASS = -1; stage_ms and flags are ignored.
 * Every column must hold the same live ids: GTS_EINVAL when their live
 * counts differ or an answer of one column is not live in another.  out
 * (host) carries dist = (float)sum and key = the FP64 sum; release it with
 * gts_result_free. */
gts_status gts_multi_range(gts_index *const *cols, int32_t m, const gts_objects *queries, const float *radii,
                           const gts_query_opts *opts, gts_result *out);
gts_status gts_multi_knn(gts_index *const *cols, int32_t m, const gts_objects *queries, const int32_t *k,
                         const gts_query_opts *opts, gts_result *out);

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
 *  str_chunk:  edit distance, (query, object) pairs per block of the
 *              bit-parallel DP kernels (pivot distances and verification):
 *              64, 128, 256 (default) or 512.
 *  str_qgram:  edit distance with GTS_PREC_BF16, the 3-gram count filter
 *              before the DP: 0 = off (the table scan alone), or its queries
 *              per tile chunk, 32 or 64 (default).
 *  tuned:      output only: 1 once gts_autotune has run on the index. */
typedef struct {
    int32_t l1_queries;
    int32_t l1_packed;
    int32_t knn_phases;
    int32_t probe_rows;
    int32_t tuned;
    int32_t tc_queries;
    int32_t str_chunk;
    int32_t str_qgram;
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

/* Cost model of Section 5.3.  An object survives the pivots of the first i
 * levels with probability p^i, p = P(|X - Y| <= r) for the distances X, Y of
 * two objects to one pivot (Eq. 2), so a batch of nq queries holds about
 * S_i = nq * fanout^i * p^i (query, node) pairs at level i, and the search
 * costs about  sum_{i=1..h} i^2 ceil(S_i / C) log2(fanout)^2  (the form of
 * Eq. 3, C = the GPU's concurrency in threads), plus the same term for the
 * objects of the surviving leaves, S_{h+1} = nq * n * p^h, which this index
 * verifies after its h pivot levels.  p in [0, 1]; returns the estimate in
 * relative units (only comparisons between shapes are meaningful). */
double gts_cost_model(int64_t n, int64_t nq, double p, int32_t fanout, int32_t h, double concurrency);

/* An index shape (Section 4.2: node capacity and pivot levels) and how it
 * fared under gts_autotune_shape. */
typedef struct {
    int32_t fanout;      /* N_c */
    int32_t n_pivots;    /* h */
    double model_cost;   /* gts_cost_model estimate */
    double measured_ms;  /* median wall time of the sample batch on this shape */
} gts_shape;

/* Shape autotuner: estimates p of Eq. 2 from the index's own table list (the
 * distances of a sample of its objects to the root pivot, all pairs) and the
 * sample batch's radius (range: the median of `radii`; kNN: the mean k-th
 * distance of a run of the batch), ranks the shapes fanout in 4 .. 64, h in 1
 * .. Algorithm 1's height for that fanout, by gts_cost_model, rebuilds the
 * index with the current shape and with `candidates` (1 .. 16) others -- half
 * of them (rounded up) the current shape's neighbours (fanout halved or
 * doubled, one pivot level fewer or more), the rest the model's cheapest --
 * times the sample batch (`reps` runs, median of the wall time;
 * one untimed warm-up run first) on each, and leaves the index rebuilt with
 * the fastest.  A shape whose tree or batch does not fit the device is
 * skipped (reported with measured_ms = +inf).  Ids and answers do not change
 * (every shape answers the same definition).  out: host gts_shape[candidates + 1] (may be NULL), the shapes
 * timed, fastest first; *n_out (may be NULL) their number.  On an error the
 * index holds one of the timed shapes. */
gts_status gts_autotune_shape(gts_index *index, const gts_objects *queries, const float *radii, const int32_t *k,
                              const gts_query_opts *opts, int32_t candidates, int32_t reps, gts_shape *out,
                              int32_t *n_out);

/* Diagnostic, no counterpart in the paper: runs the tensor-core tile
 * primitives of the BF16 L2 path (TMA load with 128-byte swizzle, tcgen05.mma
 * with the accumulator in TMEM, tcgen05.ld) on one 128 x N x K product:
 * D[128, N] = bf16(A[128, K]) * bf16(B[N, K])^T in FP32.  A, B, D are host
 * row-major float32; N a multiple of 32 up to 256, K in {64, 128, 192, 256}.
 * a_tmem = 0: A is read from shared memory (TMA); 1: A is first written into
 * TMEM by tcgen05.st, one row per TMEM lane, as the tile kernel holds its node
 * blocks. */
gts_status gts_selftest_tc(const float *A, const float *B, int N, int K, int a_tmem, float *D);

/* Diagnostic, no counterpart in the paper: checks the bounded waits that
 * every kernel of this library uses on mbarriers.  One thread waits on a
 * barrier that another thread of its block arrives on only if `post` is
 * non-zero; the wait polls at most spin_limit times (1 .. 2^26).  Returns
 * GTS_OK when the arrival came, GTS_ETIMEOUT when the wait ran out (the
 * kernel then records the run-out in a status word and returns; the device
 * stays usable), GTS_EINVAL for a limit out of range. */
gts_status gts_selftest_wait(int32_t post, uint32_t spin_limit);

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
 * Non-finite inputs are not rejected (checking them would cost a pass over
 * the objects): an object whose distance comes out NaN (a NaN coordinate in
 * it or in the query) ranks as distance +inf, after every finite one, by id.
 * The first call in a CUDA context (normally: on a device) looks up the
 * array's device address with cudaGetSymbolAddress and caches it under the
 * context's id; make that first call before any stream capture.  After a
 * cudaDeviceReset the next call looks the address up again.
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
 * fit result_budget.  A request's projection is an upper bound of its
 * candidate rows times 37 bytes: the descent of Section 5.1 run on the host
 * over the top pivot levels of the tree (a snapshot of at most 4096 pivots
 * taken by gts_serve_start; at most 64 pivot distances per request), with
 * Lemma 1's node test on every child's interval (kNN: with the k-th smallest
 * distance to the visible pivots evaluated so far, an upper bound of d_k),
 * summing the rows of the surviving nodes plus the cache list.  The index
 * must not be updated while a server runs on it. */
typedef struct gts_server gts_server;

typedef struct {
    int32_t max_batch;      /* requests per device batch; 0 = 1024 */
    int32_t n_streams;      /* worker threads and streams (batches in flight); 0 = 3 */
    int32_t precision;      /* gts_precision of every batch */
    int32_t batch_quantum;  /* a batch of more than this many requests is cut down to a multiple of it (the
                               rest waits at the head of the queue), so the tiles' query chunks run full;
                               0 or 1 = no rounding */
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

/* Counters, the first n_out of: batches run, requests run, largest batch,
 * largest projected bytes in flight, sum of the projected bytes of every
 * submitted request, requests whose projection was below the worst case
 * (every visible object a candidate). */
gts_status gts_serve_stats(gts_server *server, int64_t *out, int32_t n_out);

/* The admission projection of one request (as gts_serve_submit would compute
 * it) in *bytes, without submitting it. */
gts_status gts_serve_project(gts_server *server, const void *query, int64_t len, int32_t kind, double param,
                             int64_t *bytes);

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
