// Tensor-core (tcgen05) verification tiles for L2: declarations shared by the
// search driver and the tile kernel.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "gts_impl.cuh"

namespace gts {

// One (query, last-level node) entry in node-major order: everything the tile
// epilogue needs about the query, 32 bytes (two 16-byte async copies).
struct __align__(16) TileRec {
    int32_t q;
    float thr;       // radius or tau_q
    float alpha, beta;   // tensor-core bound test: keep iff -2 q.x <= beta + alpha |x| + gamma_x
    int64_t seq;     // the query's sequence number
    uint64_t mask;   // surviving leaves of the node
};

struct TileArgs {
    int dim, dim_p, F, h;
    int64_t n;
    const float *xn2;         // |x|^2 of every row (FP64 sum, rounded)
    const __nv_bfloat16 *Xh, *Xl;   // every row, split bf16 [n, dim_p]
    const float *table;       // [h, n]
    const int64_t *row_del;
    const int32_t *npos, *nsize;
    int64_t lvl_last;         // first node of the last pivot level
    const __nv_bfloat16 *Qh, *Ql;   // the batch's queries, split bf16 [nq, dim_p]
    const TileRec *grec;      // entries of the last pivot level regrouped by node
    const int32_t *gq;        // their queries (for the row copies)
    const float *gpath;       // their path distances [*, hp], hp = h rounded up to 4
    int hp;
    const int4 *items;        // (node, first, count, row block | kWindowItem) over the records
    int64_t n_items;
    int *work_counter;
    int32_t *out_q, *out_row;
    float *out_qx;            // null, or each kept pair's q.x~ (d~^2 = |q|^2 + |x|^2 - 2 q.x~ is within E of d^2)
    int64_t cap;
    unsigned long long *out_count;
    int *status;
    float epsc, cE1, cE2;     // pruning slack; error-bound coefficients
    float lslack[kMaxHeight]; // absolute slack of each level's query-to-pivot distances
    int any_deleted;          // 0: no row has a delete mark, skip the visibility test
    // window mode (dense nodes): the node x query bitmap of the regrouping
    const uint32_t *bits;     // [nodes, nw]
    const int32_t *wpre;      // exclusive popcount prefix of each row's words
    const int64_t *noff;      // first record of each node
    int64_t nw;
    int64_t nq;
    // window mode: each node's non-empty windows in ascending order,
    // wlist[node * nwin + k] for k < wcount[node]
    const int32_t *wlist, *wcount;
    int64_t nwin;
    // dense last level: no records; column q of node p takes its leaf mask
    // from dmask[p * nq + q] and its query data from the per-query arrays
    const uint64_t *dmask;    // null: records
    const float2 *ab_q;       // per position: the query's bound constants (alpha, beta)
    const int32_t *qperm;     // position -> query (null: the same)
    const int64_t *seq_q;
};

struct TcQuery {
    int64_t E = 0;
    int64_t nq = 0;
    const __nv_bfloat16 *Qh = nullptr, *Ql = nullptr;   // split bf16 queries [nq, dim_p]
    const float *qn2 = nullptr;                          // |q|^2 (null: not needed, records get 0)
    float cE1 = 0.f, cE2 = 0.f;                          // bf16 error-bound coefficients (tc_bound_coeffs)
    int chunk = 128;                                     // tensor-core tiles up to 128 columns: 128 or 96 queries
    // dense last level: the tiles' column order.  Column (position) i is query
    // perm[i]; Qh / Ql are then in position order, qn2, qseq and thr in query
    // order.  Null: position = query.
    const int32_t *perm = nullptr;
    const int32_t *eq = nullptr, *enode = nullptr;
    const float *path = nullptr;
    const uint64_t *emask = nullptr;
    const float *Q = nullptr;
    const int64_t *qseq = nullptr;
    const float *thr = nullptr;
    float epsc = 0.f;
    float lslack[kMaxHeight] = {};   // absolute slack of each level's path distances
    int any_deleted = 1;
};

// items of nodes that hold at least half of the batch's queries run in window
// mode: chunks are windows of 128 consecutive query ids, loaded by TMA
constexpr int kWindowItem = 1 << 30;

struct TcRegroup {
    const uint64_t *dmask = nullptr;   // dense last level: leaf masks [nodes, nq] (no records)
    DBuf<uint32_t> bits;   // node x query bitmap (when the regrouping used one)
    DBuf<int32_t> wpre;
    DBuf<int64_t> noff;
    int64_t nw = 0;
    DBuf<TileRec> grec;    // entry records grouped by node
    DBuf<int32_t> gq;      // their queries
    DBuf<float> gpath;     // their path distances [*, hp]
    DBuf<int4> items;      // (node, first, count, 0)
    int64_t n_items = 0;
    int64_t n_entries = 0; // entries with a surviving leaf
    int64_t n_chunks = 0;  // query chunks over all blocks (tensor-core tiles)
    int64_t n_pairs = 0;   // (query, row) pairs of all blocks: sum over nodes of entries x rows
};

bool tc_supported(const Tree &t);
// |d~^2 - d^2| <= cE1 |q||x| + cE2 (|q| + |x|)^2 for the split-bf16 products over dim_p columns
void tc_bound_coeffs(int dim_p, float &cE1, float &cE2);
void tc_prepare(Tree &t, TcCache &c, cudaStream_t st);
// split a batch's queries into bf16 hi / lo rows [nq, dim_p] and squared norms
// (sel: row i of the output is query sel[i]; null: query i)
void tc_split_queries(const float *Q, int64_t nq, int dim, int dim_p, DBuf<uint8_t> &Qh, DBuf<uint8_t> &Ql,
                      DBuf<float> &qn2, cudaStream_t st, const int32_t *sel = nullptr);
// whether tc_regroup counts entries per node itself (a node x query bitmap),
// so the caller need not
bool regroup_uses_bits(const Tree &t, int64_t nq, int64_t E);
// regroup the last-level entries by node into tiles; returns the tile count
// counts: entries with a surviving leaf per last-level node, if already known
// window_ok: mark dense nodes' items for window mode (tensor-core tiles with
// 128-query chunks only)
int64_t tc_regroup(const Tree &t, const TcQuery &tq, TcRegroup &rg, cudaStream_t st,
                   const int32_t *counts = nullptr, bool window_ok = false);
// dense last level: work items for every node with a set bit in the node x
// query bitmap `bits` ([nodes, nw] words, nw = ceil(nq / 32)), all in window
// mode; the leaf masks stay in dmask [nodes, nq]
int64_t tc_dense_items(const Tree &t, int64_t nq, const uint64_t *dmask, TcRegroup &rg, cudaStream_t st);
// run the tiles; returns the number of (query, row) pairs written to out_q/out_row
// (and, given out_qx, each pair's q.x~: d~^2 = |q|^2 + |x|^2 - 2 q.x~ is within
// tc_bound_coeffs' E of d^2)
int64_t tc_run(const Tree &t, const TcCache &c, const TcQuery &tq, const TcRegroup &rg, DBuf<int32_t> &out_q,
               DBuf<int32_t> &out_row, int64_t cap_hint, int *launches, cudaStream_t st,
               DBuf<float> *out_qx = nullptr);
// Dense query-to-pivot distances of one pivot level on the tensor cores
// (dim_p <= 256, after tc_prepare and tc_prepare_pivots): out[q, p] for the
// batch's split queries; returns the level's absolute slack, an upper bound of
// |out - d| over the entries not recomputed in FP32 (those are within the FP32
// relative bound).  With perm, the split queries (Qh, Ql, qn2) are in position
// order, position j holding query perm[j]; outT (if given) receives the
// matrix transposed by position, outT[p * nq + j].
bool tc_dense_supported(const Tree &t, const TcCache &c);
void tc_prepare_pivots(const Tree &t, TcCache &c, cudaStream_t st);
float tc_dense_dist(const Tree &t, const TcCache &c, int level, const __nv_bfloat16 *Qh, const __nv_bfloat16 *Ql,
                    const float *qn2, const float *Q, int64_t nq, float *out, cudaStream_t st,
                    const int32_t *perm = nullptr, float *outT = nullptr);
void tc_selftest(const float *hA, const float *hB, int N, int K, int a_tmem, float *hD);
void wait_selftest(int post, uint32_t limit);

}  // namespace gts
