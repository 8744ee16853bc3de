// Internal declarations of the GTS library (not part of the C ABI).
//
// Data layout in HBM (one index):
//   * X      float32[n * dim]   vectors in leaf order (row r = r-th object of the
//                               table list, Section 4.2), or
//     S/Soff uint8 bytes + int64[n + 1] offsets, strings in leaf order.
//   * row_id int64[n]           row -> object id.
//   * table  float32[h * n]     column l, row r: distance of row r's object to the
//                               pivot of its level-l ancestor (the table list, all
//                               h levels kept).
//   * row_del int64[n]          sequence number at which the row was deleted
//                               (INT64_MAX = never), the deletion mark of Section 4.4.
//   * node list, level by level (Eq. 1, 0-based): level l holds fanout^l nodes, the
//     children of node i are nodes i * fanout + j of level l + 1.  Per node:
//     pos, size (int32, rows [pos, pos + size) of the table list), lo, hi (float32,
//     distance interval to the parent's pivot) and piv (int32 row of the pivot, or
//     -1; levels 0 .. h-1).
//   * cache list (Section 4.4): inserted objects not yet in the tree, with their
//     ids and insert / delete sequence numbers.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>
#include <stdexcept>
#include <string>
#include <vector>

#include "gts.h"

namespace gts {

constexpr int kMaxFanout = 64;
constexpr int kMaxHeight = 12;
constexpr int kMaxStrLen = 1024;
constexpr int64_t kNever = INT64_MAX;

// ------------------------------------------------------------------ errors

struct Error : std::runtime_error {
    gts_status status;
    Error(gts_status s, const std::string &m) : std::runtime_error(m), status(s) {}
};

void set_last_error(const std::string &msg);
void ensure_device();   // GTS_ECUDA unless a CUDA device is usable

#define GTS_CUDA(call)                                                                              \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) {                                                                    \
            if (e_ == cudaErrorMemoryAllocation)                                                    \
                throw ::gts::Error(GTS_ENOMEM, std::string("out of device memory at ") + #call);    \
            throw ::gts::Error(GTS_ECUDA, std::string(cudaGetErrorString(e_)) + " at " + #call +    \
                                              " (" + __FILE__ + ":" + std::to_string(__LINE__) + ")"); \
        }                                                                                           \
    } while (0)

#define GTS_REQUIRE(cond, status, msg)                                                              \
    do {                                                                                            \
        if (!(cond)) throw ::gts::Error(status, msg);                                               \
    } while (0)

inline void check_launch(const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) throw Error(GTS_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// ------------------------------------------------------------------ memory

// Stream-ordered device buffer (cudaMallocAsync / cudaFreeAsync).
template <class T>
struct DBuf {
    T *p = nullptr;
    size_t n = 0;
    cudaStream_t s = nullptr;
    DBuf() = default;
    DBuf(size_t count, cudaStream_t st) { alloc(count, st); }
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    DBuf(DBuf &&o) noexcept { *this = std::move(o); }
    DBuf &operator=(DBuf &&o) noexcept {
        if (this != &o) {
            release();
            p = o.p; n = o.n; s = o.s; keep = o.keep;
            o.p = nullptr; o.n = 0;
        }
        return *this;
    }
    ~DBuf() { release(); }
    void alloc(size_t count, cudaStream_t st) {
        release();
        s = st;
        n = count;
        if (count) GTS_CUDA(cudaMallocAsync((void **)&p, count * sizeof(T), st));
    }
    // Index-owned buffers outlive the stream they were allocated on (a
    // caller's stream, a serving worker's): they are released with the
    // synchronous cudaFree, which needs no stream.
    void persist() { keep = true; }
    void release() {
        if (p) {
            if (keep) cudaFree(p);
            else cudaFreeAsync(p, s);
        }
        p = nullptr;
        n = 0;
    }
    bool keep = false;
    T *get() const { return p; }
    size_t bytes() const { return n * sizeof(T); }
};

// ------------------------------------------------------------------ index

struct Objects {           // a view of caller-provided or library objects
    int64_t n = 0;
    int dim = 0;           // 0 = strings
    const float *X = nullptr;
    const uint8_t *S = nullptr;
    const int64_t *Soff = nullptr;
    int max_len = 0;       // longest string (strings only)
};

// Tensor-core copy of the tree rows (built on the first BF16 query): every
// row split into bf16 hi / lo parts (x = x_hi + x_lo to 2^-16), padded to a
// multiple of 64 columns; the squared norms; the two TMA descriptors.
struct TcCache {
    bool ready = false;
    int dim_p = 0;
    DBuf<uint8_t> Xh, Xl;
    DBuf<float> xn2;
    // every pivot level's pivots as split rows (node order; empty nodes: zero rows)
    bool piv_ready = false;
    DBuf<uint8_t> Ph, Pl;
    DBuf<float> pn2;
};

struct Tree {
    int metric = 0, dim = 0, F = 0, h = 0;
    int64_t n = 0;
    // angular distance (GTS_COS): the tree is an L2 tree over the unit vectors
    // X = x / |x| (normalised in FP64, rounded to FP32); Xr keeps the raw rows
    // (leaf order) for the FP64 keys
    bool cosine = false;
    DBuf<float> Xr;
    DBuf<float> X;
    DBuf<uint8_t> S;
    DBuf<int64_t> Soff;
    DBuf<int64_t> row_id;
    DBuf<float> table;
    DBuf<int64_t> row_del;
    std::vector<int64_t> lvl_off;   // h + 2 entries: first node of each level, last = total nodes
    DBuf<int32_t> npos, nsize, npiv;
    DBuf<float> nlo, nhi;
    int max_len = 0;                // longest string
    int64_t n_deleted = 0;          // rows carrying a delete mark
    TcCache tc;
    DBuf<uint8_t> qg;               // strings: hashed 3-gram counts per row [n, 64] (built on first use)
    bool qg_ready = false;
    size_t device_bytes() const;
    void persist() {   // every buffer the index keeps
        X.persist(); Xr.persist(); S.persist(); Soff.persist(); row_id.persist(); table.persist(); row_del.persist();
        npos.persist(); nsize.persist(); npiv.persist(); nlo.persist(); nhi.persist();
        tc.Xh.persist(); tc.Xl.persist(); tc.xn2.persist(); qg.persist();
    }
};

struct Cache {
    int64_t count = 0, cap = 0;
    DBuf<float> X;                   // cap * dim (unit vectors for GTS_COS)
    DBuf<float> Xr;                  // GTS_COS: the raw rows
    DBuf<uint8_t> S;                 // bytes
    DBuf<int64_t> Soff;              // cap + 1
    int64_t s_bytes = 0, s_cap = 0;
    DBuf<int64_t> id, ins, del;
    std::vector<int64_t> h_Soff;     // host copy of the offsets
    int max_len = 0;
};

// Launch parameters of the tile kernels and of the kNN schedule.  None of
// them changes a result; gts_autotune picks them by timing.
struct Tuning {
    int l1_queries = 64;    // L1 tiles: queries per chunk (64 or 128)
    int l1_packed = 1;      // L1 tiles: packed f32x2 subtraction
    int knn_phases = 3;     // L1 tile kNN: phases (1..3)
    int probe_rows = 1024;  // kNN probe: rows evaluated before the descent (0..4096)
    int tc_queries = 128;   // tensor-core tiles (dim <= 128): queries per chunk, 128 (2 slots) or 96 (3 slots)
    int str_chunk = 256;    // strings: (query, object) pairs per block of the DP kernels
    int str_qgram = 64;     // strings: 3-gram filter off (0) or its queries per chunk (32, 64)
    int tuned = 0;
};

}  // namespace gts

struct gts_index {
    int device = 0;
    cudaStream_t stream = nullptr;
    int metric = 0, dim = 0, F = 0, n_pivots_req = 0;
    gts::Tree tree;
    gts::Cache cache;
    // host bookkeeping: loc[id] >= 0 tree row, <= -2 cache slot (-(slot + 2)), -1 gone
    std::vector<int64_t> loc;
    int64_t next_id = 0, seq = 1, rebuild_seq = 1, n_live = 0;
    int64_t cache_limit = 4096;
    uint64_t seed = 0;
    int64_t rebuilds = 0;
    std::vector<cudaEvent_t> events;   // reused by per-stage timing
    std::mutex tune_mu;
    std::mutex prep_mu;   // lazily built per-index data (BF16 split rows, 3-gram counts)
    gts::Tuning tuning;
    std::atomic<int64_t> tc_pairs_hint[2] = {{0}, {0}}; // last tensor-core output size per query (x1024)
    std::atomic<int64_t> l1_pairs_hint[4] = {{0}, {0}, {0}, {0}};  // L1 tiles: range, kNN phases 0..2 (same unit)
    std::atomic<int64_t> scan_pairs_hint[2] = {{0}, {0}};  // table scan: candidates per query (x1024), range / kNN
    ~gts_index() {
        for (auto e : events) cudaEventDestroy(e);
    }
};

namespace gts {

// api.cu
// FP64 keys of the pairs (queries row pq[j], object id pid[j]) of one index
// (vector metrics), computed on the device on stream st; GTS_EINVAL when an
// id is not live
void pair_keys(gts_index *ix, const gts_objects *queries, const std::vector<int32_t> &pq,
               const std::vector<int64_t> &pid, std::vector<double> &keys, cudaStream_t st);

// build.cu
// raw_rows: angular distance only -- objs holds the unit vectors, raw_rows
// the caller's rows in the same order (kept in leaf order as Tree::Xr)
void build_tree(Tree &t, const Objects &objs, const int64_t *d_ids_or_null, int metric, int F, int h,
                int64_t root_index, cudaStream_t st, const float *raw_rows = nullptr);
int tree_height(int64_t n, int F, int n_pivots);
uint64_t splitmix64(uint64_t x);

// search.cu
struct QueryBatch {
    int64_t nq = 0;
    int dim = 0;
    const float *Q = nullptr;        // device
    const uint8_t *S = nullptr;      // device
    const int64_t *Soff = nullptr;   // device
    int max_len = 0;
    const float *radii = nullptr;    // device (range)
    const int32_t *k = nullptr;      // device (knn)
    const int64_t *seq = nullptr;    // device or null
    int64_t seq_now = 0;
    int64_t max_k = 0;
    bool count_table_pass = false;   // diagnostics: count the pairs passing the table bound
    bool want_keys = false;          // kNN: also return each answer's FP64 key
    // GTS_COS: Q holds the unit query vectors, Qr the raw ones; radii are
    // angles, coslim[i] = 1 - cos(r_i) (FP64, computed on the host)
    const float *Qr = nullptr;
    const double *coslim = nullptr;
};

// GTS_COS: absolute slack (beyond the FP32 relative bound) of every distance
// between unit vectors rounded to FP32: each rounded vector lies within 2^-24
// of the exact one, so a chord moves by at most 2^-23; thresholds carry four
// times that.
constexpr float kCosAbsSlack = 4.8e-7f;

struct QueryOut {
    DBuf<int64_t> offsets, ids;
    DBuf<float> dist;
    DBuf<double> key;   // kNN with GTS_QUERY_KEYS: the FP64 key of each answer
    int64_t total = 0;
};

void run_query(gts_index *ix, const QueryBatch &qb, bool knn, int precision, int64_t budget,
               QueryOut &out, int64_t *stats, double *stage_ms, cudaStream_t st);

}  // namespace gts
