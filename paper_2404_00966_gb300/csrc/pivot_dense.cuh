// Dense query-to-pivot distance matrices for one tree level (L1 / L2).
#pragma once

#include "gts_impl.cuh"

namespace gts {

// dim % 4 == 0 and 16-byte aligned rows and queries
bool dense_supported(int metric, int dim, const float *X, const float *Q);
// out[q * P + p] = d(Q[q], X[piv[p]]) in FP32 for q < nq, p < P (piv[p] < 0:
// left unwritten); device pointers, asynchronous on st
void dense_pivot_dist(int metric, const float *X, int dim, const float *Q, int64_t nq, const int32_t *piv, int64_t P,
                      float *out, cudaStream_t st);

}  // namespace gts
