// L2 verification on the 5th-generation tensor cores (tcgen05 + TMEM + TMA).
//
// After the descent, the surviving (query, last-level node) entries are
// regrouped by node.  A persistent, work-stealing kernel takes one (node,
// chunk of up to kNQ queries) tile at a time:
//   * TMA brings the node's rows -- stored once, centred on the node's
//     centroid and rounded to bf16 -- into shared memory (128-byte swizzle);
//   * the warps load the chunk's queries, centre them on the same centroid,
//     round to bf16 and store them in the same layout;
//   * one thread issues the K/16 tcgen05.mma (M = 128 rows, N = kNQ queries,
//     FP32 accumulation in TMEM);
//   * the epilogue reads the dot products from TMEM, forms
//     d^2 = |q|^2 + |x|^2 - 2 q.x (the centred form), and keeps a (query, row)
//     pair only if the row's leaf survived for the query, the row is visible
//     at the query's sequence number, the table lower bound max_l |D_l - d_l|
//     passes (Lemma 1 / 2) and a proven lower bound of the true distance is
//     within the query's threshold (radius, or tau_q for kNN).
// The pairs kept are a superset of the answers; they are finished by the FP32
// distance with its FP64 boundary recheck, so results equal the plain path's.
//
// Lower bound of d = |q - x| from the bf16 tile (Higham, Accuracy and
// Stability of Numerical Algorithms, 2nd ed., 3.1): with q' = q - c,
// x' = x - c and q^, x^ their bf16 roundings (unit roundoff 2^-8),
//   | |q^ - x^| - |q' - x'| | <= E1 = (2^-8 + 2^-22) (|q'| + |x'|),
// and the FP32 norm form with K-term accumulation (any order, products exact,
// sums allowed to truncate: unit 2^-23) satisfies
//   | d~^2 - |q^ - x^|^2 | <= E2 = gamma_{K+4}(2^-23) (|q^| + |x^|)^2.
// Hence d >= sqrt(max(0, d~^2 - E2)) - E1, shrunk by a further 2^-18
// relative for the FP32 evaluation of the bound itself.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <cub/device/device_scan.cuh>

#include "gts_impl.cuh"
#include "metric.cuh"
#include "tc.cuh"
#include "tile_tc.cuh"

namespace gts {

namespace {

constexpr int kRows = 128;     // MMA M: rows of one node tile
constexpr int kNQ = 128;       // MMA N: queries of one tile
constexpr int kThreads = 256;  // 8 warps
constexpr int kTmemCols = 128; // FP32 accumulator: 128 lanes x kNQ columns
constexpr int kMaxCtasPerSm = 512 / kTmemCols;

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        GTS_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
        GTS_REQUIRE(q == cudaDriverEntryPointSuccess && p != nullptr, GTS_ECUDA, "cuTensorMapEncodeTiled unavailable");
        fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// bf16 rows [rows, dim_p], box 64 columns x 128 rows, 128-byte swizzle
CUtensorMap make_row_map(const void *base, int64_t rows, int dim_p) {
    CUtensorMap m;
    cuuint64_t dims[2] = {(cuuint64_t)dim_p, (cuuint64_t)(rows > 0 ? rows : 1)};
    cuuint64_t strides[1] = {(cuuint64_t)dim_p * 2};
    cuuint32_t box[2] = {64, (cuuint32_t)kRows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box,
                             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    GTS_REQUIRE(r == CUDA_SUCCESS, GTS_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return m;
}

// ---------------------------------------------------------------- preparation

// centroid of every last-level node (FP32 mean of its rows)
__global__ void k_centroids(const float *__restrict__ X, int dim, const int32_t *__restrict__ npos,
                            const int32_t *__restrict__ nsize, int64_t nn, float *__restrict__ cent) {
    const int64_t node = blockIdx.x;
    if (node >= nn) return;
    const int32_t pos = npos[node], size = nsize[node];
    for (int c = threadIdx.x; c < dim; c += blockDim.x) {
        float s = 0.f;
        for (int32_t r = 0; r < size; ++r) s += X[(int64_t)(pos + r) * dim + c];
        cent[node * dim + c] = size > 0 ? s / (float)size : 0.f;
    }
}

// node of every row at the last pivot level, bf16 centred rows and their norms
__global__ void k_center_rows(const float *__restrict__ X, int dim, int dim_p, int64_t n,
                              const int32_t *__restrict__ row_node, const float *__restrict__ cent,
                              __nv_bfloat16 *__restrict__ Xb, float *__restrict__ xn2) {
    const int lane = threadIdx.x & 31;
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (row >= n) return;
    const float *c = cent + (int64_t)row_node[row] * dim;
    float s = 0.f;
    for (int k = lane; k < dim_p; k += 32) {
        float v = 0.f;
        if (k < dim) v = X[row * dim + k] - c[k];
        const __nv_bfloat16 b = __float2bfloat16_rn(v);
        Xb[row * dim_p + k] = b;
        const float bf = __bfloat162float(b);
        s += bf * bf;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) xn2[row] = s;
}

__global__ void k_row_node(const int32_t *__restrict__ npos, const int32_t *__restrict__ nsize, int64_t nn,
                           int32_t *__restrict__ row_node) {
    const int64_t node = blockIdx.x;
    if (node >= nn) return;
    const int32_t pos = npos[node], size = nsize[node];
    for (int32_t r = threadIdx.x; r < size; r += blockDim.x) row_node[pos + r] = (int32_t)node;
}

// ---------------------------------------------------------------- the tile kernel

// Squared-form test of the bf16 lower bound: keep the pair unless
//   sqrt(max(0, d~^2 - E2)) - E1 > thr,  i.e. unless  d~^2 > (thr + E1)^2 + E2,
// with E1 = c1 (|q^| + |x^|), E2 = gK (|q^| + |x^|)^2 as derived above.  thr
// + E1 is inflated by 2^-16 relative, which covers the FP32 evaluation of the
// right-hand side.  No square root per pair.
constexpr float kC1 = 3.9139e-3f;   // (2^-8 + 2^-22) / (1 - 2^-8), with margin

__global__ void __launch_bounds__(kThreads, 1)
    k_tile_l2_tc(const __grid_constant__ CUtensorMap xmap, TileArgs a) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    // 1024-byte alignment of the swizzled operands
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int panels = a.dim_p / 64;
    uint8_t *sA = smem;                                     // panels x 128 rows x 128 B
    uint8_t *sB = sA + panels * kRows * 128;                // panels x kNQ rows x 128 B
    uint64_t *smask = (uint64_t *)(sB + panels * kNQ * 128);// kNQ surviving-leaf masks
    int64_t *sseq = (int64_t *)(smask + kNQ);               // kNQ sequence numbers
    float4 *sq = (float4 *)(sseq + kNQ);                    // kNQ (|q^|^2, |q^|, thr, id)
    float *spath = (float *)(sq + kNQ);                     // kNQ x h
    float *scent = spath + kNQ * a.h;                       // dim_p
    uint64_t *bars = (uint64_t *)(((uintptr_t)(scent + a.dim_p) + 15) & ~(uintptr_t)15);
    uint32_t *tslot = (uint32_t *)(bars + 2);
    int *sitem = (int *)(tslot + 1);
    int *sabort = sitem + 1;
    uint32_t *sphase = (uint32_t *)(sabort + 1);   // phase of the wait that gave up

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) tc::tmem_alloc(tslot, kTmemCols);
    if (tid == 0) {
        tc::mbar_init(&bars[0], 1);
        tc::mbar_init(&bars[1], 1);
        tc::mbar_fence_init();
        *sabort = 0;
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t idesc = tc::idesc_bf16_f32(kRows, kNQ);
    const bool vec4 = (a.dim & 3) == 0 && (((uintptr_t)a.Q) & 15) == 0;
    uint32_t phase = 0;
    for (;;) {
        if (tid == 0) *sitem = atomicAdd(a.work_counter, 1);
        __syncthreads();
        const int item = *sitem;
        if (item >= a.n_items || *sabort) break;
        const int4 it = a.items[item];
        const int64_t node = it.x;
        const int start = it.y, cnt = it.z;
        const int rb = it.w * kRows;   // first row of this 128-row block within the node
        const int64_t g = a.lvl_last + node;
        const int32_t pos = a.npos[g], size = a.nsize[g];
        if (tid == 0) {
            tc::mbar_expect_tx(&bars[0], (uint32_t)(panels * kRows * 128));
            for (int p = 0; p < panels; ++p)
                tc::tma_load_2d(sA + p * kRows * 128, &xmap, p * 64, pos + rb, &bars[0]);
        }
        for (int c = tid; c < a.dim_p; c += kThreads) scent[c] = c < a.dim ? a.cent[node * a.dim + c] : 0.f;
        __syncthreads();
        // ---- per-query metadata, one thread per query (independent loads)
        for (int j = tid; j < cnt; j += kThreads) {
            const int32_t q = a.gq[start + j];
            smask[j] = a.gmask[start + j];
            sseq[j] = a.qseq[q];
            sq[j] = make_float4(0.f, 0.f, a.thr[q], __int_as_float(q));
        }
        for (int t = tid; t < cnt * a.h; t += kThreads) spath[t] = a.gpath[(int64_t)start * a.h + t];
        __syncthreads();
        // ---- query rows: centred on the node centroid, bf16, swizzled.  A warp
        // takes 4 queries at a time so their row loads are in flight together.
        for (int j0 = warp * 4; j0 < cnt; j0 += (kThreads / 32) * 4) {
            float ss[4] = {0.f, 0.f, 0.f, 0.f};
            const float *qv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int j = j0 + u < cnt ? j0 + u : j0;
                qv[u] = a.Q + (int64_t)__float_as_int(sq[j].w) * a.dim;
            }
            for (int k0 = lane * 4; k0 < a.dim_p; k0 += 128) {
                float4 v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (vec4 && k0 + 3 < a.dim) {
                        v[u] = *reinterpret_cast<const float4 *>(qv[u] + k0);
                    } else {
                        if (k0 < a.dim) v[u].x = qv[u][k0];
                        if (k0 + 1 < a.dim) v[u].y = qv[u][k0 + 1];
                        if (k0 + 2 < a.dim) v[u].z = qv[u][k0 + 2];
                        if (k0 + 3 < a.dim) v[u].w = qv[u][k0 + 3];
                    }
                }
                const float4 c = *reinterpret_cast<const float4 *>(scent + k0);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (j0 + u >= cnt) break;
                    const __nv_bfloat162 b0 = __floats2bfloat162_rn(k0 < a.dim ? v[u].x - c.x : 0.f,
                                                                    k0 + 1 < a.dim ? v[u].y - c.y : 0.f);
                    const __nv_bfloat162 b1 = __floats2bfloat162_rn(k0 + 2 < a.dim ? v[u].z - c.z : 0.f,
                                                                    k0 + 3 < a.dim ? v[u].w - c.w : 0.f);
                    uint2 pk;
                    pk.x = *reinterpret_cast<const uint32_t *>(&b0);
                    pk.y = *reinterpret_cast<const uint32_t *>(&b1);
                    *reinterpret_cast<uint2 *>(sB + tc::sw128_offset(j0 + u, k0, kNQ)) = pk;
                    const float2 f0 = __bfloat1622float2(b0), f1 = __bfloat1622float2(b1);
                    ss[u] += f0.x * f0.x + f0.y * f0.y + f1.x * f1.x + f1.y * f1.y;
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                for (int o = 16; o > 0; o >>= 1) ss[u] += __shfl_xor_sync(0xffffffffu, ss[u], o);
            if (lane < 4 && j0 + lane < cnt) {
                const float n2 = lane == 0 ? ss[0] : lane == 1 ? ss[1] : lane == 2 ? ss[2] : ss[3];
                sq[j0 + lane].x = n2;
                sq[j0 + lane].y = sqrtf(n2) * (1.f + 1e-6f);
            }
        }
        tc::fence_proxy_async_smem();
        __syncthreads();
        // ---- MMA: one thread
        if (tid == 0) {
            if (!tc::mbar_wait(&bars[0], phase)) {
                *sabort = 1;
                *sphase = phase;
                atomicExch(a.status, 1);
            } else {
                tc::tc_fence_after();
                const uint32_t aB = tc::smem_u32(sA), bB = tc::smem_u32(sB);
                const int ksteps = a.dim_p / 16;
                for (int s = 0; s < ksteps; ++s) {
                    const int p = s >> 2, w = s & 3;
                    const uint64_t ad = tc::sdesc_k_sw128(aB + p * kRows * 128 + w * 32);
                    const uint64_t bd = tc::sdesc_k_sw128(bB + p * kNQ * 128 + w * 32);
                    tc::mma_bf16(tmem, ad, bd, idesc, s > 0 ? 1u : 0u);
                }
                tc::mma_commit(&bars[1]);
            }
        }
        __syncthreads();
        if (*sabort) break;
        // ---- epilogue: warp w reads lanes 32 (w % 4) .. +32, columns half (w / 4)
        if (!tc::mbar_wait(&bars[1], phase)) {
            *sabort = 1;
            *sphase = phase;
            atomicExch(a.status, 2);
        }
        tc::tc_fence_after();
        const int quad = warp & 3, half = warp >> 2;
        const int r = quad * 32 + lane;                 // TMEM lane = row of the block
        const int nrow = size - rb;                     // rows of the node in this block (may exceed 128)
        const bool valid = r < nrow;
        const int64_t row = (int64_t)pos + rb + r;
        const int32_t avg = size / a.F;
        int32_t jl = avg > 0 ? (rb + r) / avg : a.F - 1;
        if (jl > a.F - 1) jl = a.F - 1;
        // leaves of the warp's rows: a query whose mask misses all of them is
        // skipped by the whole warp at once
        const int rlast = min(quad * 32 + 31, min(nrow, kRows) - 1);
        uint64_t wmask = 0;
        if (rlast >= quad * 32) {
            int32_t j0 = avg > 0 ? (rb + quad * 32) / avg : a.F - 1;
            int32_t j1 = avg > 0 ? (rb + rlast) / avg : a.F - 1;
            j0 = min(j0, a.F - 1);
            j1 = min(j1, a.F - 1);
            wmask = ((j1 >= 63) ? ~0ull : ((1ull << (j1 + 1)) - 1ull)) & ~((1ull << j0) - 1ull);
        }
        float xn2 = 0.f, xn = 0.f;
        int64_t rdel = kNever;
        if (valid) {
            xn2 = a.xn2[row];
            xn = sqrtf(xn2) * (1.f + 1e-6f);
            if (a.any_deleted) rdel = a.row_del[row];
        }
        for (int c0 = half * (kNQ / 2); c0 < (half + 1) * (kNQ / 2) && c0 < cnt; c0 += 32) {
            uint32_t v[32];
            tc::tmem_ld32(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)c0, v);
            tc::tmem_ld_wait();
            uint32_t passbits = 0;
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const int j = c0 + i;
                if (j >= cnt) break;
                const uint64_t m = smask[j];
                if ((m & wmask) == 0) continue;   // warp-uniform
                if (!valid || !((m >> jl) & 1ull)) continue;
                const float4 qm = sq[j];
                const float d2 = fmaf(-2.f, __uint_as_float(v[i]), qm.x + xn2);
                const float sn = qm.y + xn;
                const float t = fmaf(kC1, sn, qm.z) * 1.0000153f;
                if (d2 > fmaf(t, t, a.gK * sn * sn)) continue;
                if (rdel <= sseq[j]) continue;
                // table lower bound (Lemma 1 / 2) on the pair that is left
                bool ok = true;
                for (int l = 0; l < a.h && ok; ++l) {
                    const float T = a.table[(int64_t)l * a.n + row];
                    const float pl = spath[j * a.h + l];
                    const float eps = a.epsc * (T + pl + qm.z);
                    if (fabsf(T - pl) > qm.z + eps) ok = false;
                }
                if (ok) passbits |= 1u << i;
            }
            const int np = __popc(passbits);
            int incl = np;
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            const int wtot = __shfl_sync(0xffffffffu, incl, 31);
            if (wtot == 0) continue;
            unsigned long long base = 0;
            if (lane == 31) base = atomicAdd(a.out_count, (unsigned long long)wtot);
            base = __shfl_sync(0xffffffffu, base, 31);
            unsigned long long o = base + (unsigned long long)(incl - np);
            while (passbits) {
                const int i = __ffs(passbits) - 1;
                passbits &= passbits - 1;
                if ((int64_t)o < a.cap) {
                    a.out_q[o] = __float_as_int(sq[c0 + i].w);
                    a.out_row[o] = (int32_t)row;
                }
                ++o;
            }
        }
        tc::tc_fence_before();
        __syncthreads();
        phase ^= 1u;
    }
    __syncthreads();
    if (*sabort && tid == 0) {
        // let a TMA or MMA still in flight finish (bounded) before the
        // shared memory and the TMEM columns are released
        tc::mbar_wait(&bars[0], *sphase);
        tc::mbar_wait(&bars[1], *sphase);
    }
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

// ---------------------------------------------------------------- node-major regrouping

__global__ void k_node_hist(const int32_t *__restrict__ enode, const uint64_t *__restrict__ emask, int64_t E,
                            int32_t *__restrict__ ncount) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x)
        if (emask[e]) atomicAdd(&ncount[enode[e]], 1);
}

// scatter each entry's payload (query, leaf mask, path distances) to its
// node's slot, so a tile reads its queries' data contiguously
__global__ void k_node_scatter(const int32_t *__restrict__ eq, const int32_t *__restrict__ enode,
                               const uint64_t *__restrict__ emask, const float *__restrict__ path, int h, int64_t E,
                               const int64_t *__restrict__ noff, int32_t *__restrict__ cursor,
                               int32_t *__restrict__ gq, uint64_t *__restrict__ gmask, float *__restrict__ gpath) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t m = emask[e];
        if (!m) continue;
        const int32_t nd = enode[e];
        const int64_t o = noff[nd] + atomicAdd(&cursor[nd], 1);
        gq[o] = eq[e];
        gmask[o] = m;
        for (int l = 0; l < h; ++l) gpath[o * h + l] = path[e * h + l];
    }
}

// tiles of a node: 128-row blocks of its rows x chunks of kNQ of its queries
__global__ void k_items_per_node(const int32_t *__restrict__ ncount, const int32_t *__restrict__ nsize, int64_t nn,
                                 int64_t *__restrict__ nitems) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nn; i += (int64_t)gridDim.x * blockDim.x)
        nitems[i] = (int64_t)((ncount[i] + kNQ - 1) / kNQ) * ((nsize[i] + kRows - 1) / kRows);
    if (blockIdx.x == 0 && threadIdx.x == 0) nitems[nn] = 0;
}

__global__ void k_fill_items(const int32_t *__restrict__ ncount, const int32_t *__restrict__ nsize,
                             const int64_t *__restrict__ noff, const int64_t *__restrict__ ioff, int64_t nn,
                             int4 *__restrict__ items) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nn; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = ncount[i];
        const int32_t blocks = (nsize[i] + kRows - 1) / kRows;
        int64_t o = ioff[i];
        for (int32_t b = 0; b < blocks; ++b)
            for (int32_t s = 0; s < c; s += kNQ, ++o)
                items[o] = make_int4((int)i, (int)(noff[i] + s), c - s < kNQ ? c - s : kNQ, b);
    }
}

__global__ void k_i32_to_i64_tc(const int32_t *a, int64_t n, int64_t *b) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = a[i];
    if (blockIdx.x == 0 && threadIdx.x == 0) b[n] = 0;
}

template <class T>
void exscan(const T *in, T *out, int64_t n, cudaStream_t st) {
    size_t tb = 0;
    cub::DeviceScan::ExclusiveSum(nullptr, tb, in, out, n, st);
    DBuf<uint8_t> tmp(tb ? tb : 1, st);
    GTS_CUDA(cub::DeviceScan::ExclusiveSum(tmp.get(), tb, in, out, n, st));
}

inline unsigned nblk(int64_t n, int per = 256) {
    int64_t b = (n + per - 1) / per;
    if (b < 1) b = 1;
    if (b > 0x7fffffffLL) b = 0x7fffffffLL;
    return (unsigned)b;
}

size_t tile_smem_bytes(int dim_p, int h, int dim) {
    const int panels = dim_p / 64;
    size_t b = 1024;                                  // alignment slack
    b += (size_t)panels * kRows * 128 + (size_t)panels * kNQ * 128;
    b += (size_t)kNQ * (8 + 8 + 16) + sizeof(float) * kNQ * h + sizeof(float) * dim_p;
    b += 16 + 16 + 16 + 16 + 16 + 16;
    (void)dim;
    return b;
}

}  // namespace

bool tc_supported(const Tree &t) { return t.metric == GTS_L2 && t.dim > 0 && t.dim <= 256 && t.n > 0; }

void tc_prepare(Tree &t, TcCache &c, cudaStream_t st) {
    if (c.ready) return;
    const int64_t nn = t.lvl_off[t.h] - t.lvl_off[t.h - 1];
    c.dim_p = ((t.dim + 63) / 64) * 64;
    c.cent.alloc((size_t)nn * t.dim, st);
    c.xn2.alloc(t.n, st);
    c.Xb.alloc((size_t)t.n * c.dim_p * 2, st);
    DBuf<int32_t> row_node(t.n, st);
    const int32_t *npos = t.npos.get() + t.lvl_off[t.h - 1];
    const int32_t *nsize = t.nsize.get() + t.lvl_off[t.h - 1];
    k_row_node<<<(unsigned)nn, 128, 0, st>>>(npos, nsize, nn, row_node.get());
    k_centroids<<<(unsigned)nn, 128, 0, st>>>(t.X.get(), t.dim, npos, nsize, nn, c.cent.get());
    k_center_rows<<<nblk(t.n * 32), 256, 0, st>>>(t.X.get(), t.dim, c.dim_p, t.n, row_node.get(), c.cent.get(),
                                                (__nv_bfloat16 *)c.Xb.get(), c.xn2.get());
    check_launch("bf16 preparation");
    c.map = make_row_map(c.Xb.get(), t.n, c.dim_p);
    GTS_CUDA(cudaStreamSynchronize(st));
    c.ready = true;
}

int64_t tc_regroup(const Tree &t, const TcQuery &tq, TcRegroup &rg, cudaStream_t st) {
    const int64_t E = tq.E;
    const int64_t nn = t.lvl_off[t.h] - t.lvl_off[t.h - 1];
    DBuf<int32_t> ncount(nn, st), cursor(nn, st);
    GTS_CUDA(cudaMemsetAsync(ncount.get(), 0, nn * 4, st));
    GTS_CUDA(cudaMemsetAsync(cursor.get(), 0, nn * 4, st));
    k_node_hist<<<nblk(E), 256, 0, st>>>(tq.enode, tq.emask, E, ncount.get());
    DBuf<int64_t> c64(nn + 1, st), noff(nn + 1, st), nitems(nn + 1, st), ioff(nn + 1, st);
    k_i32_to_i64_tc<<<nblk(nn), 256, 0, st>>>(ncount.get(), nn, c64.get());
    exscan(c64.get(), noff.get(), nn + 1, st);
    int64_t total_entries = 0;
    GTS_CUDA(cudaMemcpyAsync(&total_entries, noff.get() + nn, 8, cudaMemcpyDeviceToHost, st));
    GTS_CUDA(cudaStreamSynchronize(st));
    const int64_t ne = total_entries > 0 ? total_entries : 1;
    rg.gq.alloc(ne, st);
    rg.gmask.alloc(ne, st);
    rg.gpath.alloc(ne * t.h, st);
    k_node_scatter<<<nblk(E), 256, 0, st>>>(tq.eq, tq.enode, tq.emask, tq.path, t.h, E, noff.get(), cursor.get(),
                                            rg.gq.get(), rg.gmask.get(), rg.gpath.get());
    const int32_t *lsize = t.nsize.get() + t.lvl_off[t.h - 1];
    k_items_per_node<<<nblk(nn), 256, 0, st>>>(ncount.get(), lsize, nn, nitems.get());
    exscan(nitems.get(), ioff.get(), nn + 1, st);
    int64_t total_items = 0;
    GTS_CUDA(cudaMemcpyAsync(&total_items, ioff.get() + nn, 8, cudaMemcpyDeviceToHost, st));
    GTS_CUDA(cudaStreamSynchronize(st));
    rg.n_items = total_items;
    rg.n_entries = total_entries;
    if (total_items > 0) {
        rg.items.alloc(total_items, st);
        k_fill_items<<<nblk(nn), 256, 0, st>>>(ncount.get(), lsize, noff.get(), ioff.get(), nn, rg.items.get());
    }
    check_launch("tile regroup");
    return total_items;
}

int64_t tc_run(const Tree &t, const TcCache &c, const TcQuery &tq, const TcRegroup &rg, DBuf<int32_t> &out_q,
               DBuf<int32_t> &out_row, int64_t cap_hint, int *launches, cudaStream_t st) {
    *launches = 0;
    if (rg.n_items == 0) return 0;
    int dev = 0, sms = 0;
    GTS_CUDA(cudaGetDevice(&dev));
    GTS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const size_t smem = tile_smem_bytes(c.dim_p, t.h, t.dim);
    GTS_CUDA(cudaFuncSetAttribute(k_tile_l2_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // CTAs per SM: shared memory (each CTA also has 1 KB reserved), the 512
    // TMEM columns, and the occupancy calculator (registers)
    int smem_sm = 0, regs_sm = 0;
    GTS_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    GTS_CUDA(cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev));
    cudaFuncAttributes fa;
    GTS_CUDA(cudaFuncGetAttributes(&fa, k_tile_l2_tc));
    int per_sm = (int)(smem_sm / (smem + 1024));
    const int regs_cta = ((fa.numRegs + 7) / 8) * 8 * kThreads;
    if (regs_cta > 0 && per_sm > regs_sm / regs_cta) per_sm = regs_sm / regs_cta;
    if (per_sm > kMaxCtasPerSm) per_sm = kMaxCtasPerSm;
    if (per_sm < 1) per_sm = 1;
    const int64_t grid = std::min<int64_t>(rg.n_items, (int64_t)sms * per_sm);
    DBuf<int> counter(1, st), status(1, st);
    DBuf<unsigned long long> count(1, st);
    int64_t cap = cap_hint > 0 ? cap_hint : 1 << 20;
    for (int attempt = 0; attempt < 2; ++attempt) {
        out_q.alloc(cap, st);
        out_row.alloc(cap, st);
        GTS_CUDA(cudaMemsetAsync(counter.get(), 0, 4, st));
        GTS_CUDA(cudaMemsetAsync(status.get(), 0, 4, st));
        GTS_CUDA(cudaMemsetAsync(count.get(), 0, 8, st));
        TileArgs a;
        a.dim = t.dim;
        a.dim_p = c.dim_p;
        a.F = t.F;
        a.h = t.h;
        a.n = t.n;
        a.cent = c.cent.get();
        a.xn2 = c.xn2.get();
        a.table = t.table.get();
        a.row_del = t.row_del.get();
        a.npos = t.npos.get();
        a.nsize = t.nsize.get();
        a.lvl_last = t.lvl_off[t.h - 1];
        a.Q = tq.Q;
        a.qseq = tq.qseq;
        a.thr = tq.thr;
        a.gq = rg.gq.get();
        a.gpath = rg.gpath.get();
        a.gmask = rg.gmask.get();
        a.items = rg.items.get();
        a.n_items = rg.n_items;
        a.work_counter = counter.get();
        a.out_q = out_q.get();
        a.out_row = out_row.get();
        a.cap = cap;
        a.out_count = count.get();
        a.status = status.get();
        a.epsc = tq.epsc;
        a.gK = (float)(c.dim_p + 4) * 1.1920929e-7f * 1.01f;
        a.any_deleted = tq.any_deleted;
        k_tile_l2_tc<<<(unsigned)grid, kThreads, smem, st>>>(c.map, a);
        ++*launches;
        check_launch("tensor-core tile");
        unsigned long long hcount = 0;
        int hstatus = 0;
        GTS_CUDA(cudaMemcpyAsync(&hcount, count.get(), 8, cudaMemcpyDeviceToHost, st));
        GTS_CUDA(cudaMemcpyAsync(&hstatus, status.get(), 4, cudaMemcpyDeviceToHost, st));
        GTS_CUDA(cudaStreamSynchronize(st));
        GTS_REQUIRE(hstatus == 0, GTS_ETIMEOUT,
                    "tensor-core tile: a bounded mbarrier wait ran out (status " + std::to_string(hstatus) + ")");
        if ((int64_t)hcount <= cap) return (int64_t)hcount;
        cap = (int64_t)hcount;
    }
    throw Error(GTS_ECUDA, "tensor-core tile: output count changed between launches");
}

// ---------------------------------------------------------------- self-test

namespace {

constexpr int kSelfN = 256;   // self-test tile: N up to 256, its own TMEM allocation

__global__ void __launch_bounds__(128, 1)
    k_selftest_tc(const __grid_constant__ CUtensorMap amap, const __nv_bfloat16 *__restrict__ B, int N, int K,
                  float *__restrict__ D, int *status) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int panels = K / 64;
    uint8_t *sA = smem;
    uint8_t *sB = sA + panels * kRows * 128;
    uint64_t *bars = (uint64_t *)(sB + panels * kSelfN * 128);
    uint32_t *tslot = (uint32_t *)(bars + 2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) tc::tmem_alloc(tslot, kSelfN);
    if (tid == 0) {
        tc::mbar_init(&bars[0], 1);
        tc::mbar_init(&bars[1], 1);
        tc::mbar_fence_init();
        tc::mbar_expect_tx(&bars[0], (uint32_t)(panels * kRows * 128));
        for (int p = 0; p < panels; ++p) tc::tma_load_2d(sA + p * kRows * 128, &amap, p * 64, 0, &bars[0]);
    }
    for (int j = tid; j < N; j += blockDim.x)
        for (int k = 0; k < K; ++k) *(__nv_bfloat16 *)(sB + tc::sw128_offset(j, k, kSelfN)) = B[(int64_t)j * K + k];
    tc::fence_proxy_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tslot;
    if (tid == 0) {
        if (!tc::mbar_wait(&bars[0], 0)) {
            atomicExch(status, 1);
        } else {
            const uint32_t idesc = tc::idesc_bf16_f32(kRows, kSelfN);
            for (int s = 0; s < K / 16; ++s) {
                const int p = s >> 2, w = s & 3;
                tc::mma_bf16(tmem, tc::sdesc_k_sw128(tc::smem_u32(sA) + p * kRows * 128 + w * 32),
                             tc::sdesc_k_sw128(tc::smem_u32(sB) + p * kSelfN * 128 + w * 32), idesc, s > 0 ? 1u : 0u);
            }
            tc::mma_commit(&bars[1]);
        }
    }
    __syncthreads();
    const bool ok = *status == 0 && tc::mbar_wait(&bars[1], 0);
    if (!ok) atomicExch(status, 2);
    tc::tc_fence_after();
    if (ok) {
        for (int c0 = 0; c0 < N; c0 += 32) {
            uint32_t v[32];
            tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            tc::tmem_ld_wait();
            const int r = warp * 32 + lane;
            for (int i = 0; i < 32; ++i)
                if (c0 + i < N) D[(int64_t)r * N + c0 + i] = __uint_as_float(v[i]);
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (tid == 0 && !ok) {
        tc::mbar_wait(&bars[0], 0);
        tc::mbar_wait(&bars[1], 0);
    }
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kSelfN);
}

__global__ void k_f32_to_bf16(const float *a, int64_t n, __nv_bfloat16 *b) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = __float2bfloat16_rn(a[i]);
}

}  // namespace

void tc_selftest(const float *hA, const float *hB, int N, int K, float *hD) {
    GTS_REQUIRE(N >= 32 && N <= kSelfN && N % 32 == 0, GTS_EINVAL, "N must be a multiple of 32 in 32 .. 256");
    GTS_REQUIRE(K >= 64 && K <= 256 && K % 64 == 0, GTS_EINVAL, "K must be 64, 128, 192 or 256");
    cudaStream_t st = nullptr;
    DBuf<float> fA((size_t)kRows * K, st), fB((size_t)N * K, st), D((size_t)kRows * N, st);
    DBuf<__nv_bfloat16> bA((size_t)kRows * K, st), bB((size_t)N * K, st);
    DBuf<int> status(1, st);
    GTS_CUDA(cudaMemcpyAsync(fA.get(), hA, (size_t)kRows * K * 4, cudaMemcpyHostToDevice, st));
    GTS_CUDA(cudaMemcpyAsync(fB.get(), hB, (size_t)N * K * 4, cudaMemcpyHostToDevice, st));
    GTS_CUDA(cudaMemsetAsync(status.get(), 0, 4, st));
    k_f32_to_bf16<<<64, 256, 0, st>>>(fA.get(), (int64_t)kRows * K, bA.get());
    k_f32_to_bf16<<<64, 256, 0, st>>>(fB.get(), (int64_t)N * K, bB.get());
    CUtensorMap m = make_row_map(bA.get(), kRows, K);
    const size_t smem = 1024 + (size_t)(K / 64) * (kRows + kSelfN) * 128 + 64;
    GTS_CUDA(cudaFuncSetAttribute(k_selftest_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_selftest_tc<<<1, 128, smem, st>>>(m, bB.get(), N, K, D.get(), status.get());
    check_launch("tensor-core self-test");
    int hs = 0;
    GTS_CUDA(cudaMemcpyAsync(&hs, status.get(), 4, cudaMemcpyDeviceToHost, st));
    GTS_CUDA(cudaMemcpyAsync(hD, D.get(), (size_t)kRows * N * 4, cudaMemcpyDeviceToHost, st));
    GTS_CUDA(cudaStreamSynchronize(st));
    GTS_REQUIRE(hs == 0, GTS_ETIMEOUT, "tensor-core self-test: a bounded wait ran out");
}

}  // namespace gts
