// L1 verification tiles on the CUDA cores.
//
// L1 has no product form, so it cannot use the tensor cores: every (query,
// object) pair costs a subtraction and an absolute-value addition per
// coordinate, and the work is bound by the FP32 pipes.  When the lower bounds
// of Lemma 1 / 2 prune little (high-dimensional, concentrated distances), the
// pairs left after the descent are most of the n x nq pairs and the paper's
// candidate-by-candidate verification reads one object row per pair.  Here
// the surviving (query, last-level node) entries are regrouped by node (the
// same regrouping the tensor-core tiles use) and one CTA computes a block of
// up to 128 node rows against up to 128 of the node's queries at once:
//   * both operands are streamed through shared memory in slices of 32
//     coordinates (asynchronous 16-byte copies, double-buffered), so each row
//     slice is read once per query chunk and each query slice once per block;
//   * thread (lane, warp) holds the FP32 sums of rows lane + 32 i (i < 4) for
//     queries 16 warp + j (j < 16) in registers and adds the coordinates of a
//     pair in increasing order;
//   * the epilogue keeps a pair only if the row's leaf survived for the query,
//     the row is visible at the query's sequence number and the FP32 distance
//     minus its error bound is within the query's threshold; the pair is
//     written with its FP32 distance, so nothing re-reads the row later except
//     the FP64 recheck of distances within the error band of the threshold.
// Error bound: the FP32 sum of D rounded terms |q_i - x_i| lies within
// (D + 8) 2^-24 of the exact sum in relative terms (recursive summation,
// Higham 2nd ed. 4.2), the band the plain path uses as well.
#include <cub/device/device_scan.cuh>

#include "gts_impl.cuh"
#include "metric.cuh"
#include "tile_l1.cuh"

namespace gts {

namespace {

constexpr int kRowsL1 = 128;   // rows of one node block (the regrouping's block size)
constexpr int kNQL1 = 128;     // queries of one chunk, at most (8 warps x QPT)
constexpr int kThreadsL1 = 256;
constexpr int kRPT = 4;        // rows per thread: lane + 32 i
constexpr int kKC = 32;        // coordinates per pipeline stage
constexpr int kLd = kKC + 4;   // padded shared-memory row stride (floats): conflict-free 16-byte loads

struct L1Args {
    int dim, F;
    const float *X;            // rows in leaf order [n, dim]
    const float *Q;            // queries [nq, dim]
    const int64_t *row_del;
    const int32_t *npos, *nsize;
    int64_t lvl_last;
    const TileRec *grec;
    const int32_t *gq;
    const float *thr_live;     // kNN: the current tau_q (lowered between phases)
    int knn;
    const int4 *items;
    int64_t i1;                // items [work_counter start, i1)
    int *work_counter;
    int32_t *out_q, *out_row;
    float *out_d;
    int64_t cap;
    unsigned long long *out_count;
    float rel;
    int any_deleted;
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
// 16-byte asynchronous copy; with valid == false nothing is read and the
// destination is filled with zeros
__device__ __forceinline__ void cp16(void *dst, const void *src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_addr(dst)), "l"(src),
                 "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// copy coordinates [k0, k0 + 32) of the block's rows and of the chunk's
// queries; coordinates past dim and rows / queries past the block are zeros
template <int NQ>
__device__ __forceinline__ void stage_slice(const L1Args &a, int64_t row0, int nrow, const int32_t *sq, int cnt,
                                            int k0, float *sX, float *sQ) {
    const int tid = threadIdx.x;
#pragma unroll
    for (int c = tid; c < kRowsL1 * (kKC / 4); c += kThreadsL1) {
        const int r = c >> 3, ch = c & 7, k = k0 + ch * 4;
        const bool v = r < nrow && k < a.dim;
        const float *src = v ? a.X + (row0 + r) * a.dim + k : a.X;
        cp16(sX + r * kLd + ch * 4, src, v);
    }
#pragma unroll
    for (int c = tid; c < NQ * (kKC / 4); c += kThreadsL1) {
        const int j = c >> 3, ch = c & 7, k = k0 + ch * 4;
        const bool v = j < cnt && k < a.dim;
        const float *src = v ? a.Q + (int64_t)sq[j] * a.dim + k : a.Q;
        cp16(sQ + j * kLd + ch * 4, src, v);
    }
}

// acc += |x_0 - q_0| + ... + |x_3 - q_3| in coordinate order.  X2 forms the
// four differences with two packed FP32 subtractions (sub.rn.f32x2, two
// IEEE round-to-nearest results per instruction, the same values as four
// scalar subtractions), so a pair costs 1.5 instead of 2 instructions per
// coordinate.
template <bool X2>
__device__ __forceinline__ float l1_step4(float acc, const float4 &x, const float4 &q) {
    float d0, d1, d2, d3;
    if (X2) {
        asm("{\n\t.reg .b64 xa, qa, ra;\n\t"
            "mov.b64 xa, {%2, %3};\n\tmov.b64 qa, {%4, %5};\n\t"
            "sub.rn.f32x2 ra, xa, qa;\n\tmov.b64 {%0, %1}, ra;\n\t}"
            : "=f"(d0), "=f"(d1)
            : "f"(x.x), "f"(x.y), "f"(q.x), "f"(q.y));
        asm("{\n\t.reg .b64 xa, qa, ra;\n\t"
            "mov.b64 xa, {%2, %3};\n\tmov.b64 qa, {%4, %5};\n\t"
            "sub.rn.f32x2 ra, xa, qa;\n\tmov.b64 {%0, %1}, ra;\n\t}"
            : "=f"(d2), "=f"(d3)
            : "f"(x.z), "f"(x.w), "f"(q.z), "f"(q.w));
    } else {
        d0 = x.x - q.x;
        d1 = x.y - q.y;
        d2 = x.z - q.z;
        d3 = x.w - q.w;
    }
    acc += fabsf(d0);
    acc += fabsf(d1);
    acc += fabsf(d2);
    acc += fabsf(d3);
    return acc;
}

// QPT queries per thread (a chunk of 8 QPT queries); X2: packed subtraction
template <int QPT, bool X2>
__global__ void __launch_bounds__(kThreadsL1, 2) k_tile_l1(L1Args a) {
    constexpr int NQ = 8 * QPT;
    constexpr int kQPT = QPT;
    extern __shared__ __align__(16) float smem_l1[];
    float *sX = smem_l1;                                 // 2 x [128][kLd]
    float *sQ = sX + 2 * kRowsL1 * kLd;                  // 2 x [128][kLd]
    TileRec *sRec = reinterpret_cast<TileRec *>(sQ + 2 * kNQL1 * kLd);   // [128]
    float *sThr = reinterpret_cast<float *>(sRec + kNQL1);                // [128]
    int32_t *sQid = reinterpret_cast<int32_t *>(sThr + kNQL1);           // [128]
    __shared__ uint64_t sRowBit[kRowsL1];
    __shared__ int64_t sRowDel[kRowsL1];
    __shared__ int s_item;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nstage = (a.dim + kKC - 1) / kKC;
    for (;;) {
        if (tid == 0) s_item = atomicAdd(a.work_counter, 1);
        __syncthreads();
        const int64_t item = s_item;
        if (item >= a.i1) break;
        const int4 it = a.items[item];
        const int64_t g = a.lvl_last + it.x;
        const int first = it.y, total = it.z;
        const int rb = it.w * kRowsL1;
        const int32_t pos = a.npos[g], size = a.nsize[g];
        const int nrow = min(kRowsL1, size - rb);
        const int64_t row0 = (int64_t)pos + rb;
        // per-row constants: leaf bit within the node (even split, remainder
        // in the last child) and delete mark
        if (tid < kRowsL1) {
            const int32_t avg = size / a.F;
            int32_t jl = avg > 0 ? (rb + tid) / avg : a.F - 1;
            if (jl > a.F - 1) jl = a.F - 1;
            sRowBit[tid] = tid < nrow ? (1ull << jl) : 0ull;
            sRowDel[tid] = (tid < nrow && a.any_deleted) ? a.row_del[row0 + tid] : kNever;
        }
        for (int c0 = 0; c0 < total; c0 += NQ) {
            const int cnt = min(NQ, total - c0);
            for (int j = tid; j < cnt; j += kThreadsL1) {
                const TileRec rc = a.grec[first + c0 + j];
                sRec[j] = rc;
                sQid[j] = rc.q;
                sThr[j] = a.knn ? fminf(rc.thr, a.thr_live[rc.q]) : rc.thr;
            }
            __syncthreads();
            const bool active = warp * kQPT < cnt;   // warp-uniform: this warp has queries in the chunk
            float acc[kRPT][kQPT];
#pragma unroll
            for (int i = 0; i < kRPT; ++i)
#pragma unroll
                for (int j = 0; j < kQPT; ++j) acc[i][j] = 0.f;
            stage_slice<NQ>(a, row0, nrow, sQid, cnt, 0, sX, sQ);
            cp_commit();
            for (int s = 0; s < nstage; ++s) {
                const int b = s & 1;
                if (s + 1 < nstage) {
                    stage_slice<NQ>(a, row0, nrow, sQid, cnt, (s + 1) * kKC, sX + (b ^ 1) * kRowsL1 * kLd,
                                    sQ + (b ^ 1) * kNQL1 * kLd);
                    cp_commit();
                    cp_wait<1>();
                } else {
                    cp_wait<0>();
                }
                __syncthreads();
                if (active) {
                    const float *xs = sX + b * kRowsL1 * kLd + lane * kLd;
                    const float *qs = sQ + b * kNQL1 * kLd + warp * kQPT * kLd;
#pragma unroll 1
                    for (int kk = 0; kk < kKC; kk += 4) {
                        float4 xv[kRPT];
#pragma unroll
                        for (int i = 0; i < kRPT; ++i) xv[i] = *reinterpret_cast<const float4 *>(xs + i * 32 * kLd + kk);
#pragma unroll
                        for (int j = 0; j < kQPT; ++j) {
                            const float4 qv = *reinterpret_cast<const float4 *>(qs + j * kLd + kk);
#pragma unroll
                            for (int i = 0; i < kRPT; ++i) acc[i][j] = l1_step4<X2>(acc[i][j], xv[i], qv);
                        }
                    }
                }
                __syncthreads();   // the buffer is refilled next stage
            }
            // ---- epilogue: leaf, visibility and threshold tests; emit kept pairs
            uint64_t pass = 0;
            if (active) {
#pragma unroll
                for (int j = 0; j < kQPT; ++j) {
                    const int jj = warp * kQPT + j;
                    if (jj >= cnt) break;
                    const uint64_t mk = sRec[jj].mask;
                    const int64_t seq = sRec[jj].seq;
                    const float t = sThr[jj];
#pragma unroll
                    for (int i = 0; i < kRPT; ++i) {
                        const int r = lane + 32 * i;
                        const float lo = acc[i][j] * (1.f - 2.f * a.rel) - kAbsFloor;
                        if (lo <= t && (mk & sRowBit[r]) && sRowDel[r] > seq) pass |= 1ull << (i * kQPT + j);
                    }
                }
            }
            const int np = __popcll(pass);
            int incl = np;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            const int wtot = __shfl_sync(0xffffffffu, incl, 31);
            if (wtot > 0) {
                unsigned long long base = 0;
                if (lane == 31) base = atomicAdd(a.out_count, (unsigned long long)wtot);
                base = __shfl_sync(0xffffffffu, base, 31);
                if (pass) {
                    unsigned long long o = base + (unsigned long long)(incl - np);
#pragma unroll
                    for (int i = 0; i < kRPT; ++i)
#pragma unroll
                        for (int j = 0; j < kQPT; ++j)
                            if ((pass >> (i * kQPT + j)) & 1ull) {
                                if ((int64_t)o < a.cap) {
                                    a.out_q[o] = sQid[warp * kQPT + j];
                                    a.out_row[o] = (int32_t)(row0 + lane + 32 * i);
                                    a.out_d[o] = acc[i][j];
                                }
                                ++o;
                            }
                }
            }
            __syncthreads();   // sRec / sQid are rewritten by the next chunk
        }
    }
}

size_t l1_smem_bytes() {
    return (size_t)(2 * kRowsL1 * kLd + 2 * kNQL1 * kLd) * 4 + (size_t)kNQL1 * (sizeof(TileRec) + 4 + 4);
}

}  // namespace

bool l1_tiles_supported(const Tree &t, const float *Q) {
    return t.metric == GTS_L1 && t.dim > 0 && (t.dim & 3) == 0 && t.n > 0 && t.n < ((int64_t)1 << 31) &&
           (((uintptr_t)Q | (uintptr_t)t.X.get()) & 15) == 0;
}

int64_t l1_run(const Tree &t, const L1Query &lq, const TcRegroup &rg, int64_t i0, int64_t i1, DBuf<int32_t> &out_q,
               DBuf<int32_t> &out_row, DBuf<float> &out_d, int64_t cap_hint, int *launches, cudaStream_t st) {
    *launches = 0;
    if (i1 <= i0) return 0;
    int dev = 0, sms = 0;
    GTS_CUDA(cudaGetDevice(&dev));
    GTS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const size_t smem = l1_smem_bytes();
    void (*kern)(L1Args) = lq.queries <= 64 ? (lq.packed ? k_tile_l1<8, true> : k_tile_l1<8, false>)
                                            : (lq.packed ? k_tile_l1<16, true> : k_tile_l1<16, false>);
    GTS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    GTS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreadsL1, smem));
    if (per_sm < 1) per_sm = 1;
    const int64_t grid = std::min<int64_t>(i1 - i0, (int64_t)sms * per_sm);
    DBuf<int> counter(1, st);
    DBuf<unsigned long long> count(1, st);
    int64_t cap = cap_hint > 0 ? cap_hint : 1 << 20;
    for (int attempt = 0; attempt < 2; ++attempt) {
        out_q.alloc(cap, st);
        out_row.alloc(cap, st);
        out_d.alloc(cap, st);
        const int c0 = (int)i0;
        GTS_CUDA(cudaMemcpyAsync(counter.get(), &c0, 4, cudaMemcpyHostToDevice, st));
        GTS_CUDA(cudaMemsetAsync(count.get(), 0, 8, st));
        L1Args a;
        a.dim = t.dim;
        a.F = t.F;
        a.X = t.X.get();
        a.Q = lq.Q;
        a.row_del = t.row_del.get();
        a.npos = t.npos.get();
        a.nsize = t.nsize.get();
        a.lvl_last = t.lvl_off[t.h - 1];
        a.grec = rg.grec.get();
        a.gq = rg.gq.get();
        a.thr_live = lq.thr;
        a.knn = lq.knn ? 1 : 0;
        a.items = rg.items.get();
        a.i1 = i1;
        a.work_counter = counter.get();
        a.out_q = out_q.get();
        a.out_row = out_row.get();
        a.out_d = out_d.get();
        a.cap = cap;
        a.out_count = count.get();
        a.rel = lq.rel;
        a.any_deleted = lq.any_deleted;
        kern<<<(unsigned)grid, kThreadsL1, smem, st>>>(a);
        ++*launches;
        check_launch("L1 tile");
        unsigned long long hcount = 0;
        GTS_CUDA(cudaMemcpyAsync(&hcount, count.get(), 8, cudaMemcpyDeviceToHost, st));
        GTS_CUDA(cudaStreamSynchronize(st));
        if ((int64_t)hcount <= cap) return (int64_t)hcount;
        cap = (int64_t)hcount;   // rerun with room for every pair
    }
    GTS_REQUIRE(false, GTS_ECUDA, "L1 tile: output count changed between identical runs");
    return 0;
}

}  // namespace gts
