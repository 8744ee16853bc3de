// The list-table pruning scan (Lemma 1 / Lemma 2 over the table list) as a
// node-major, bandwidth-bound pass: declarations shared with the search driver.
#pragma once

#include "gts_impl.cuh"
#include "tile_tc.cuh"

namespace gts {

// dims up to which the batched path verifies by scan + CUDA-core distance
// instead of distance tiles (a row of the table, 4 h + 8 bytes, costs about as
// much as the row itself there)
constexpr int kScanMaxDim = 16;

struct ScanStats {
    int64_t candidates = 0;   // (query, row) pairs that passed the table bound
    int64_t staged_rows = 0;  // table rows read (each block once)
    int64_t records = 0;      // (query, node block) records tested
    int launches = 0;
};

struct ScanQuery {
    float epsc = 0.f;         // pruning slack factor
    int any_deleted = 1;      // 0: no row carries a delete mark (skip the visibility test)
    // range queries on low-dimensional vectors: also compute each passing
    // pair's FP32 distance from the block's rows (staged with the table) and
    // decide it against the radius with the FP32 error band; accepted pairs
    // go straight to the answer, pairs inside the band to the FP64 recheck
    bool fused_range = false;
    const float *Q = nullptr; // queries [nq, dim]
    float rel = 0.f;          // FP32 relative error bound of one distance
};

struct ScanOut {
    DBuf<int32_t> q, row;     // candidates (plain scan) or band pairs (fused range)
    DBuf<uint64_t> key;       // fused range: accepted answers, (query << 32) | object id
    DBuf<float> dist;         // and their FP32 distances
    int64_t n_pairs = 0;      // entries of q / row
    int64_t n_accepted = 0;   // entries of key / dist
};

// Scan the regrouped last-level entries (tc_regroup: records grouped by node,
// items of up to 128 rows of a node): every row of a block is read once from
// the table list and tested against every record of its node; the pairs that
// pass the leaf mask, visibility and the table lower bound are written to
// out.q / out.row (node-major) -- or, with fused_range, decided on the spot.
void scan_run(const Tree &t, const TcRegroup &rg, const ScanQuery &sq, ScanOut &out, int64_t cap_hint,
              ScanStats &stats, cudaStream_t st);

}  // namespace gts
