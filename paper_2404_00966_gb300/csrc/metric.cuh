// Device-side distance functions (Section 3: edit distance, L1, L2).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gts {

// ---------------------------------------------------------------- FP32 vectors

// Partial sum over the lanes of a warp; every lane returns the full sum.
// L2 returns the squared distance.  Each lane adds about dim / 32 terms in
// sequence, then five shuffle levels add the lane sums (a binary tree).
template <bool L2>
__device__ __forceinline__ float warp_vec_dist(const float *__restrict__ q, const float *__restrict__ x,
                                               int dim, int lane) {
    float s = 0.f;
    if ((dim & 3) == 0 && ((((uintptr_t)q) | ((uintptr_t)x)) & 15) == 0) {
        const float4 *q4 = reinterpret_cast<const float4 *>(q);
        const float4 *x4 = reinterpret_cast<const float4 *>(x);
        for (int i = lane; i < (dim >> 2); i += 32) {
            float4 a = q4[i], b = __ldg(x4 + i);
            float d0 = a.x - b.x, d1 = a.y - b.y, d2 = a.z - b.z, d3 = a.w - b.w;
            if (L2) s += d0 * d0 + d1 * d1 + d2 * d2 + d3 * d3;
            else s += fabsf(d0) + fabsf(d1) + fabsf(d2) + fabsf(d3);
        }
    } else {
        for (int i = lane; i < dim; i += 32) {
            float d = q[i] - __ldg(x + i);
            s += L2 ? d * d : fabsf(d);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// Same sum with the query already in registers as float4 chunks (NV = dim /
// 128 per lane); NV = 0 falls back to warp_vec_dist.
template <bool L2, int NV>
__device__ __forceinline__ float row_dist_regs(const float4 (&qr)[NV > 0 ? NV : 1], const float *xv, const float *qv,
                                               int dim, int lane) {
    if (NV > 0) {
        const float4 *x4 = reinterpret_cast<const float4 *>(xv);
        float s = 0.f;
#pragma unroll
        for (int v = 0; v < (NV > 0 ? NV : 1); ++v) {
            const float4 b = __ldg(x4 + v * 32 + lane);
            const float4 a = qr[v];
            const float d0 = a.x - b.x, d1 = a.y - b.y, d2 = a.z - b.z, d3 = a.w - b.w;
            if (L2) s += d0 * d0 + d1 * d1 + d2 * d2 + d3 * d3;
            else s += fabsf(d0) + fabsf(d1) + fabsf(d2) + fabsf(d3);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        return s;
    }
    return warp_vec_dist<L2>(qv, xv, dim, lane);
}

// Proven relative error bound of the FP32 distance above against the exact
// distance: with u = 2^-24, any summation order of `dim` non-negative terms,
// each with up to three roundings, stays within gamma_{dim+2}; the square
// root halves it and adds u.  (dim + 8) u covers both with room to spare and
// also covers the FP64 reference's own error (<= (dim + 1) 2^-53).
__host__ __device__ __forceinline__ float fp32_rel_bound(int dim) { return (float)(dim + 8) * 5.9604645e-8f; }
// Absolute floor for results that underflow FP32 (squares below FLT_MIN).
constexpr float kAbsFloor = 1e-17f;

// ---------------------------------------------------------------- FP64 recheck

// The exact operation order of the CPU reference: increasing i, every
// subtraction, product and sum rounded on its own (no fused multiply-add).
__device__ __forceinline__ double l2sq_fp64_seq(const float *q, const float *x, int dim) {
    double s = 0.0;
    for (int i = 0; i < dim; ++i) {
        double t = __dsub_rn((double)q[i], (double)x[i]);
        s = __dadd_rn(s, __dmul_rn(t, t));
    }
    return s;
}

// The angular distance's key, 1 - cos: the three sums q.x, |q|^2, |x|^2 in
// increasing i, every product and sum rounded on its own, c = dot /
// (sqrt(|q|^2) sqrt(|x|^2)) clamped to [-1, 1] -- the reference operation
// order.
__device__ __forceinline__ double cos_key_fp64_seq(const float *q, const float *x, int dim) {
    double dot = 0.0, nq = 0.0, nx = 0.0;
    for (int i = 0; i < dim; ++i) {
        const double a = (double)q[i], b = (double)x[i];
        dot = __dadd_rn(dot, __dmul_rn(a, b));
        nq = __dadd_rn(nq, __dmul_rn(a, a));
        nx = __dadd_rn(nx, __dmul_rn(b, b));
    }
    double c = __ddiv_rn(dot, __dmul_rn(__dsqrt_rn(nq), __dsqrt_rn(nx)));
    c = c > 1.0 ? 1.0 : (c < -1.0 ? -1.0 : c);
    return __dsub_rn(1.0, c);
}

__device__ __forceinline__ double l1_fp64_seq(const float *q, const float *x, int dim) {
    double s = 0.0;
    for (int i = 0; i < dim; ++i) s = __dadd_rn(s, fabs(__dsub_rn((double)q[i], (double)x[i])));
    return s;
}

// ---------------------------------------------------------------- edit distance

// Bit-parallel Levenshtein distance (Myers 1999, in the block form of Hyyro
// 2003) between a pattern of length m, given as match masks Peq[c * W + b]
// (bit i of block b set iff pattern[64 b + i] == c), and a text.  The state is
// the column of vertical deltas of the DP matrix in bit vectors Pv (+1) and Mv
// (-1); every text symbol updates the whole column in O(W) word operations.
// The top boundary row of global edit distance has horizontal delta +1, which
// is shifted into the lowest row of the first block.  Returns the exact
// distance (m >= 1).
template <int W>
__device__ __forceinline__ int myers_edit(const uint64_t *__restrict__ Peq, int m, const uint8_t *__restrict__ text,
                                          int n) {
    uint64_t Pv[W], Mv[W];
#pragma unroll
    for (int b = 0; b < W; ++b) {
        Pv[b] = ~0ull;
        Mv[b] = 0ull;
    }
    const int last = (m - 1) >> 6;
    const uint64_t lastbit = 1ull << ((m - 1) & 63);
    int score = m;
    for (int j = 0; j < n; ++j) {
        const uint64_t *eqc = Peq + (int)text[j] * W;
        int hin = 1;
#pragma unroll
        for (int b = 0; b < W; ++b) {
            if (b <= last) {
                uint64_t Eq = eqc[b];
                const uint64_t pv = Pv[b], mv = Mv[b];
                const uint64_t Xv = Eq | mv;
                if (hin < 0) Eq |= 1ull;
                const uint64_t Xh = (((Eq & pv) + pv) ^ pv) | Eq;
                uint64_t Ph = mv | ~(Xh | pv);
                uint64_t Mh = pv & Xh;
                const uint64_t top = (b == last) ? lastbit : (1ull << 63);
                const int hout = (Ph & top) ? 1 : ((Mh & top) ? -1 : 0);
                Ph <<= 1;
                Mh <<= 1;
                if (hin < 0) Mh |= 1ull;
                else if (hin > 0) Ph |= 1ull;
                Pv[b] = Mh | ~(Xv | Ph);
                Mv[b] = Ph & Xv;
                hin = hout;
            }
        }
        score += hin;
    }
    return score;
}

// Fill the match masks of `pat` (length m, 1 <= m <= 64 W) into shared memory
// `Peq` (256 * W words).  Call with the whole block; ends with __syncthreads().
template <int W>
__device__ __forceinline__ void build_peq(uint64_t *Peq, const uint8_t *pat, int m) {
    for (int i = threadIdx.x; i < 256 * W; i += blockDim.x) Peq[i] = 0ull;
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x)
        atomicOr((unsigned long long *)&Peq[(int)pat[i] * W + (i >> 6)], 1ull << (i & 63));
    __syncthreads();
}

}  // namespace gts
