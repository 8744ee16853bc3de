// Edit-distance filtering tiles (3-gram count bound): declarations for the
// search driver.
#pragma once

#include "gts_impl.cuh"
#include "tile_tc.cuh"

namespace gts {

struct StrQuery {
    const uint8_t *qg = nullptr;    // the tree rows' 3-gram bucket counts [n, 64]
    const uint8_t *qgq = nullptr;   // the batch's queries' [nq, 64]
    int any_deleted = 1;
    int queries = 64;               // queries per tile chunk: 32 or 64
};

// run the tiles over a regrouping (its records carry each query's threshold);
// returns the number of (query, row) pairs written, the pairs the bound keeps
int64_t qgram_run(const Tree &t, const StrQuery &sq, const TcRegroup &rg, DBuf<int32_t> &out_q,
                  DBuf<int32_t> &out_row, int64_t cap_hint, int *launches, cudaStream_t st);

}  // namespace gts
