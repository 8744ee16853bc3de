// L1 verification tiles on the CUDA cores: declarations for the search driver.
#pragma once

#include "gts_impl.cuh"
#include "tile_tc.cuh"

namespace gts {

struct L1Query {
    const float *Q = nullptr;     // the batch's queries [nq, dim]
    const float *thr = nullptr;   // kNN: live tau_q; range: unused (records carry the radius)
    bool knn = false;
    float rel = 0.f;              // FP32 relative error bound of one distance
    int any_deleted = 1;
    int queries = 64;             // queries per chunk: 64 or 128
    bool packed = true;           // packed f32x2 subtraction
};

// the tile path needs dim % 4 == 0 and 16-byte aligned rows and queries
bool l1_tiles_supported(const Tree &t, const float *Q);
// run items [i0, i1) of a regrouping; returns the number of (query, row, FP32
// distance) triples written
int64_t l1_run(const Tree &t, const L1Query &lq, const TcRegroup &rg, int64_t i0, int64_t i1, DBuf<int32_t> &out_q,
               DBuf<int32_t> &out_row, DBuf<float> &out_d, int64_t cap_hint, int *launches, cudaStream_t st);

}  // namespace gts
