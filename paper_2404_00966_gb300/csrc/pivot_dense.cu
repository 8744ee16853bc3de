// Query-to-pivot distances of one tree level for a whole batch, as a dense
// FP32 matrix D[q, p] (Section 5.1: the distances d(q, pivot(N)) of the
// frontier entries).  When most (query, node) pairs of a level are in the
// frontier (concentrated distances prune little near the root), computing
// every pair in register tiles costs fewer instructions and far fewer bytes
// than a warp per entry, which reads one query row and one pivot row from L2
// for every entry.  The frontier kernels then read their distance from the
// matrix.
//
// Tile: 128 pivots x 64 queries per CTA, 256 threads; thread (lane, warp)
// sums pivots lane + 32 i (i < 4) against queries 8 warp + j (j < 8) over
// slices of 32 coordinates staged in shared memory by asynchronous 16-byte
// copies (double-buffered).  Per coordinate pair: L2 one packed subtraction
// and one packed fused multiply-add per two coordinates (two partial sums,
// even and odd coordinates), L1 one packed subtraction per two coordinates
// and one absolute-value addition per coordinate.  Every step is FP32 with
// round-to-nearest, so the distance is within the FP32 bound (D + 8) 2^-24
// relative that the search uses for every query-to-pivot distance.
#include "gts_impl.cuh"
#include "pivot_dense.cuh"

namespace gts {

namespace {

constexpr int kPiv = 128;     // pivots per tile
constexpr int kQry = 64;      // queries per tile
constexpr int kThr = 256;
constexpr int kPPT = 4;       // pivots per thread
constexpr int kQPT = 8;       // queries per thread
constexpr int kSlice = 32;    // coordinates per stage
constexpr int kLdS = kSlice + 4;

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp16z(void *dst, const void *src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(saddr(dst)), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}

struct DenseArgs {
    const float *X;        // rows [n, dim]
    const float *Q;        // queries [nq, dim]
    const int32_t *piv;    // pivot row of each of the level's nodes (-1: empty node)
    int64_t P, nq;
    int dim;
    float *out;            // [nq, P]
    int64_t tiles_p;       // ceil(P / kPiv)
};

__device__ __forceinline__ void stage(const DenseArgs &a, int64_t p0, int64_t q0, int k0, float *sP, float *sQ) {
    const int tid = threadIdx.x;
#pragma unroll
    for (int c = tid; c < kPiv * (kSlice / 4); c += kThr) {
        const int r = c >> 3, ch = c & 7, k = k0 + ch * 4;
        const int64_t p = p0 + r;
        const int32_t row = p < a.P ? a.piv[p] : -1;
        const bool v = row >= 0 && k < a.dim;
        cp16z(sP + r * kLdS + ch * 4, v ? a.X + (int64_t)row * a.dim + k : a.X, v);
    }
#pragma unroll
    for (int c = tid; c < kQry * (kSlice / 4); c += kThr) {
        const int j = c >> 3, ch = c & 7, k = k0 + ch * 4;
        const int64_t q = q0 + j;
        const bool v = q < a.nq && k < a.dim;
        cp16z(sQ + j * kLdS + ch * 4, v ? a.Q + q * a.dim + k : a.Q, v);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ void sub2(float &d0, float &d1, float x0, float x1, float q0, float q1) {
    asm("{\n\t.reg .b64 xa, qa, ra;\n\t"
        "mov.b64 xa, {%2, %3};\n\tmov.b64 qa, {%4, %5};\n\t"
        "sub.rn.f32x2 ra, xa, qa;\n\tmov.b64 {%0, %1}, ra;\n\t}"
        : "=f"(d0), "=f"(d1)
        : "f"(x0), "f"(x1), "f"(q0), "f"(q1));
}
// (a0, a1) += (t0 * t0, t1 * t1), each a fused multiply-add
__device__ __forceinline__ void fma2sq(float &a0, float &a1, float t0, float t1) {
    asm("{\n\t.reg .b64 ta, aa;\n\t"
        "mov.b64 ta, {%2, %3};\n\tmov.b64 aa, {%0, %1};\n\t"
        "fma.rn.f32x2 aa, ta, ta, aa;\n\tmov.b64 {%0, %1}, aa;\n\t}"
        : "+f"(a0), "+f"(a1)
        : "f"(t0), "f"(t1));
}

template <bool L2>
__global__ void __launch_bounds__(kThr, 2) k_dense_dist(DenseArgs a) {
    extern __shared__ __align__(16) float smem_d[];
    float *sP = smem_d;                      // 2 x [kPiv][kLdS]
    float *sQ = sP + 2 * kPiv * kLdS;        // 2 x [kQry][kLdS]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nstage = (a.dim + kSlice - 1) / kSlice;
    const int64_t tiles_q = (a.nq + kQry - 1) / kQry;
    for (int64_t t = blockIdx.x; t < a.tiles_p * tiles_q; t += gridDim.x) {
        const int64_t p0 = (t % a.tiles_p) * kPiv, q0 = (t / a.tiles_p) * kQry;
        // two partial sums per pair (even / odd coordinates)
        float acc[kPPT][kQPT][2];
#pragma unroll
        for (int i = 0; i < kPPT; ++i)
#pragma unroll
            for (int j = 0; j < kQPT; ++j) acc[i][j][0] = acc[i][j][1] = 0.f;
        stage(a, p0, q0, 0, sP, sQ);
        for (int s = 0; s < nstage; ++s) {
            const int b = s & 1;
            if (s + 1 < nstage) {
                stage(a, p0, q0, (s + 1) * kSlice, sP + (b ^ 1) * kPiv * kLdS, sQ + (b ^ 1) * kQry * kLdS);
                asm volatile("cp.async.wait_group 1;" ::: "memory");
            } else {
                asm volatile("cp.async.wait_group 0;" ::: "memory");
            }
            __syncthreads();
            const float *ps = sP + b * kPiv * kLdS + lane * kLdS;
            const float *qs = sQ + b * kQry * kLdS + warp * kQPT * kLdS;
#pragma unroll 1
            for (int kk = 0; kk < kSlice; kk += 4) {
                float4 xv[kPPT];
#pragma unroll
                for (int i = 0; i < kPPT; ++i) xv[i] = *reinterpret_cast<const float4 *>(ps + i * 32 * kLdS + kk);
#pragma unroll
                for (int j = 0; j < kQPT; ++j) {
                    const float4 qv = *reinterpret_cast<const float4 *>(qs + j * kLdS + kk);
#pragma unroll
                    for (int i = 0; i < kPPT; ++i) {
                        float t0, t1, t2, t3;
                        sub2(t0, t1, xv[i].x, xv[i].y, qv.x, qv.y);
                        sub2(t2, t3, xv[i].z, xv[i].w, qv.z, qv.w);
                        if (L2) {
                            fma2sq(acc[i][j][0], acc[i][j][1], t0, t1);
                            fma2sq(acc[i][j][0], acc[i][j][1], t2, t3);
                        } else {
                            acc[i][j][0] += fabsf(t0);
                            acc[i][j][1] += fabsf(t1);
                            acc[i][j][0] += fabsf(t2);
                            acc[i][j][1] += fabsf(t3);
                        }
                    }
                }
            }
            __syncthreads();
        }
#pragma unroll
        for (int j = 0; j < kQPT; ++j) {
            const int64_t q = q0 + warp * kQPT + j;
            if (q >= a.nq) break;
#pragma unroll
            for (int i = 0; i < kPPT; ++i) {
                const int64_t p = p0 + lane + 32 * i;
                if (p < a.P) {
                    const float sum = acc[i][j][0] + acc[i][j][1];
                    a.out[q * a.P + p] = L2 ? sqrtf(sum) : sum;
                }
            }
        }
    }
}

}  // namespace

bool dense_supported(int metric, int dim, const float *X, const float *Q) {
    return (metric == GTS_L1 || metric == GTS_L2) && dim > 0 && (dim & 3) == 0 &&
           (((uintptr_t)X | (uintptr_t)Q) & 15) == 0;
}

void dense_pivot_dist(int metric, const float *X, int dim, const float *Q, int64_t nq, const int32_t *piv, int64_t P,
                      float *out, cudaStream_t st) {
    if (nq <= 0 || P <= 0) return;
    int dev = 0, sms = 0;
    GTS_CUDA(cudaGetDevice(&dev));
    GTS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const size_t smem = (size_t)(2 * kPiv * kLdS + 2 * kQry * kLdS) * 4;
    void (*kern)(DenseArgs) = metric == GTS_L2 ? k_dense_dist<true> : k_dense_dist<false>;
    GTS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    GTS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThr, smem));
    if (per_sm < 1) per_sm = 1;
    DenseArgs a;
    a.X = X;
    a.Q = Q;
    a.piv = piv;
    a.P = P;
    a.nq = nq;
    a.dim = dim;
    a.out = out;
    a.tiles_p = (P + kPiv - 1) / kPiv;
    const int64_t tiles = a.tiles_p * ((nq + kQry - 1) / kQry);
    const int64_t grid = std::min<int64_t>(tiles, (int64_t)sms * per_sm);
    kern<<<(unsigned)grid, kThr, smem, st>>>(a);
    check_launch("dense pivot distances");
}

}  // namespace gts
