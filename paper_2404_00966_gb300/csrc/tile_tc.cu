// L2 verification on the 5th-generation tensor cores (tcgen05 + TMEM + TMA).
//
// After the descent, the surviving (query, last-level node) entries are
// regrouped by node.  A persistent, work-stealing, warp-specialised kernel
// takes one 128-row block of one node at a time (the A operand, loaded once by
// TMA and kept in shared memory) and runs it against the node's queries in
// chunks of kNQ (the B operand); producer warps stage the chunks, one thread
// issues the MMAs and epilogue warps test the results, handing chunks on
// through mbarriers:
//   * rows and queries are stored once as split bf16 pairs x = x_hi + x_lo
//     (x_hi = bf16(x), x_lo = bf16(x - x_hi)); a chunk's query pairs are
//     copied into shared memory in the 128-byte swizzled layout;
//   * one thread issues three tcgen05.mma per 16-wide k-step,
//     D += A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T, FP32 accumulator in TMEM;
//   * the epilogue reads q.x from TMEM, forms d~^2 = |q|^2 + |x|^2 - 2 q.x and
//     keeps a (query, row) pair only if the row's leaf survived for the query,
//     the row is visible at the query's sequence number, a proven lower bound
//     of the distance is within the query's threshold (radius, or tau_q for
//     kNN) and the table lower bound max_l |D_l - d_l| passes (Lemma 1 / 2).
// The pairs kept are a superset of the answers; they are finished by the FP32
// distance with its FP64 boundary recheck, so results equal the plain path's.
//
// Error bound (Higham, Accuracy and Stability of Numerical Algorithms, 2nd
// ed., 3.1).  With |x - x_hi| <= 2^-8 |x| and |x - x_hi - x_lo| <= 2^-16 |x|
// per coordinate (the same for q), the three products miss at most
// 3.01 * 2^-16 sum_i |q_i x_i| <= 3.01 * 2^-16 |q| |x|; the 3K exact products
// are summed in FP32, possibly truncating (unit 2^-23), within
// gamma_{3K+2} |q| |x|.  The norms come from FP64 sums rounded to FP32.  So
//   | d~^2 - d^2 | <= E = cE1 |q| |x| + cE2 (|q| + |x|)^2,
//   cE1 = 2.02 (3.01 * 2^-16 + gamma_{3K+2}(2^-23)),  cE2 = 2^-21,
// and d <= thr is possible only if d~^2 <= thr^2 + E.
#include <cstring>

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

constexpr int kRows = 128;     // MMA M: rows of one node block
// MMA N (queries per chunk) NQ, the number SB of query-row buffers (B, hi and
// lo) and the number SM of chunk slots (records, path distances and one FP32
// TMEM accumulator of 128 lanes x NQ columns each) are template parameters,
// chosen so that the node block (dim_p TMEM columns, hi and lo) and the SM
// accumulators fit TMEM's 512 columns and the SB buffers and the slots fit
// shared memory:
//   dim_p <= 128: 128 queries (SB = SM = 3) or 96 (4, 4), the tuning chooses;
//   192: 64 (4, 4);  256: 32 (4, 4);  320: 64 (2, 3);  384: 32 (2, 4);
//   448: 32 (2, 2).
// A B buffer is released when the MMAs that read it are done, a slot when the
// epilogue has tested its chunk: the producers restage B while the epilogue
// still works on older chunks.
struct TileShape {
    int nq, sb, sm;
};
inline TileShape shape_for(int dim_p, int pref) {
    if (dim_p <= 128) return pref == 96 ? TileShape{96, 4, 4} : TileShape{128, 3, 3};
    if (dim_p <= 192) return {64, 4, 4};
    if (dim_p <= 256) return {32, 4, 4};
    if (dim_p <= 320) return {64, 2, 3};
    if (dim_p <= 384) return {32, 2, 4};
    return {32, 2, 2};
}
inline int nq_for(int dim_p, int pref) { return shape_for(dim_p, pref).nq; }

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

// bf16 rows [rows, dim_p], box 64 columns x box_rows rows, 128-byte swizzle
CUtensorMap make_row_map(const void *base, int64_t rows, int dim_p, int box_rows) {
    CUtensorMap m;
    cuuint64_t dims[2] = {(cuuint64_t)dim_p, (cuuint64_t)(rows > 0 ? rows : 1)};
    cuuint64_t strides[1] = {(cuuint64_t)dim_p * 2};
    cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box,
                             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    GTS_REQUIRE(r == CUDA_SUCCESS, GTS_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return m;
}

// The same rows as (64 coordinates, row, 64-coordinate panel): one box
// {64, box_rows, dim_p / 64} lands as the panels one after another, each
// box_rows x 128 bytes in the 128-byte swizzle -- a chunk's rows of all panels
// in one copy.
CUtensorMap make_panel_map(const void *base, int64_t rows, int dim_p, int box_rows) {
    CUtensorMap m;
    cuuint64_t dims[3] = {64, (cuuint64_t)(rows > 0 ? rows : 1), (cuuint64_t)(dim_p / 64)};
    cuuint64_t strides[2] = {(cuuint64_t)dim_p * 2, 128};
    cuuint32_t box[3] = {64, (cuuint32_t)box_rows, (cuuint32_t)(dim_p / 64)};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(base), dims, strides, box,
                             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    GTS_REQUIRE(r == CUDA_SUCCESS, GTS_ECUDA, "cuTensorMapEncodeTiled (3-D) failed (" + std::to_string((int)r) + ")");
    return m;
}

// ---------------------------------------------------------------- preparation

// Split every float32 row into bf16 hi / lo parts (padded with zeros to
// dim_p columns) and its squared norm, summed in FP64 and rounded once
// (output row i from input row sel[i] when sel is given).
__global__ void k_split_rows(const float *__restrict__ X, int dim, int dim_p, int64_t n,
                             __nv_bfloat16 *__restrict__ Xh, __nv_bfloat16 *__restrict__ Xl,
                             float *__restrict__ n2, const int32_t *__restrict__ sel) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; row < n; row += nw) {
        // output row `row` takes input row `src` (a negative src: a zero row)
        const int64_t src = sel ? (int64_t)sel[row] : row;
        double s = 0.0;
        for (int k = lane; k < dim_p; k += 32) {
            const float v = k < dim && src >= 0 ? X[src * dim + k] : 0.f;
            const __nv_bfloat16 h = __float2bfloat16_rn(v);
            const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
            Xh[row * dim_p + k] = h;
            Xl[row * dim_p + k] = l;
            s += (double)v * (double)v;
        }
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) n2[row] = __double2float_rn(s);
    }
}

// ---------------------------------------------------------------- the tile kernel

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc::smem_u32(smem_dst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// (d0, d1) = (a0 + b0, a1 + b1), one packed FP32 addition (round to nearest)
__device__ __forceinline__ void add2(float &d0, float &d1, float a0, float a1, float b0, float b1) {
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d0), "=f"(d1)
        : "f"(a0), "f"(a1), "f"(b0), "f"(b1));
}
// (d0, d1) = (a0 b0 + c0, a1 b1 + c1), one packed FP32 fused multiply-add
__device__ __forceinline__ void fma2(float &d0, float &d1, float a0, float a1, float b0, float b1, float c0,
                                     float c1) {
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d0), "=f"(d1)
        : "f"(a0), "f"(a1), "f"(b0), "f"(b1), "f"(c0), "f"(c1));
}

__device__ __forceinline__ void bound_consts(float thr, float qn2, float cE1, float cE2, float &alpha, float &beta);

// The per-chunk data the producer hands to the MMA thread and the epilogue.
struct ChunkDesc {
    int32_t stop;       // 1: no more work
    int32_t new_item;   // first chunk of a node block (the epilogue writes the block's rows into TMEM)
    int32_t first;      // first record of the chunk
    int32_t cnt;        // queries in the chunk
    int32_t pos, size;  // the node's rows [pos, pos + size)
    int32_t rb;         // first row of the block within the node
    int32_t pad_;
};

// Roles: warps 0-15 epilogue (TMEM lane quadrant w % 4, 32 query columns
// each), warps 16-19 producers, warp 20 (lane 0) the MMA issuer.
constexpr int kEpiWarps = 16;
constexpr int kProducers = 128;
constexpr int kProdWarp0 = kEpiWarps;
constexpr int kMmaWarp = kEpiWarps + kProducers / 32;
constexpr int kThreadsWS = (kMmaWarp + 1) * 32;

// Stage chunk [start, start + cnt) of a block's queries with asynchronous
// copies by the producer threads: the records and path distances (contiguous,
// node-major), and the split bf16 query rows into the 128-byte swizzled
// layout (each thread first reads the query ids of the rows it copies).
template <int NQ>
__device__ __forceinline__ void stage_chunk(const TileArgs &a, int start, int cnt, TileRec *mrec, float *mpath,
                                            uint8_t *sBh, uint8_t *sBl, int chunks16, int ptid, int32_t *sqid) {
    const uint8_t *rsrc = reinterpret_cast<const uint8_t *>(a.grec + start);
    for (int t = ptid; t < cnt * 2; t += kProducers) cp_async16(reinterpret_cast<uint8_t *>(mrec) + t * 16, rsrc + t * 16);
    const uint8_t *psrc = reinterpret_cast<const uint8_t *>(a.gpath + (int64_t)start * a.hp);
    const int pch = cnt * a.hp / 4;
    for (int t = ptid; t < pch; t += kProducers) cp_async16(reinterpret_cast<uint8_t *>(mpath) + t * 16, psrc + t * 16);
    // query ids first (one load per thread), then the rows: consecutive
    // threads copy consecutive 16-byte pieces of a row, so every warp
    // instruction reads whole 32-byte sectors
    tc::named_sync(1, kProducers);   // every producer is done with the previous chunk's ids
    for (int j = ptid; j < cnt; j += kProducers) sqid[j] = a.gq[start + j];
    tc::named_sync(1, kProducers);
    const int per_q = 2 * chunks16;                  // 16-byte copies per query (hi and lo)
#pragma unroll 4
    for (int t = ptid; t < cnt * per_q; t += kProducers) {
        const int j = t / per_q, c = t - j * per_q;
        const int32_t q = sqid[j];
        const int comp = c / chunks16, k16 = c - comp * chunks16;
        const __nv_bfloat16 *src = (comp ? a.Ql : a.Qh) + (int64_t)q * a.dim_p + k16 * 8;
        uint8_t *dst = (comp ? sBl : sBh) + (k16 >> 3) * (NQ * 128) + j * 128 + (((k16 & 7) ^ (j & 7)) << 4);
        cp_async16(dst, src);
    }
}

// Warp-specialised persistent kernel.  When a node block starts, the epilogue
// warps write its split rows (A, hi and lo) into TMEM, each thread its own row
// (TMEM lane = block row); the producer warps stage chunk g's query rows into
// B buffer g % SB once the MMAs of chunk g - SB are done, and its records into
// slot g % SM once the epilogue has released chunk g - SM; one thread issues
// the MMAs of chunk g (A from TMEM, B from shared memory) into accumulator
// g % SM; the epilogue warps test chunk g when its MMAs are done and release
// the slot.  mbarriers carry every hand-off (the barriers of slot g % SM;
// chunk g's phase parity is (g / SM) & 1), so no block-wide barrier runs per
// chunk.
//
// TMEM columns: [0, dim_p / 2) A_hi and [dim_p / 2, dim_p) A_lo (two
// consecutive coordinates per 32-bit column), then SM accumulators of NQ
// columns.  With A in TMEM the shared-memory port serves B alone: with both
// operands in shared memory a 128 x 128 x 16 MMA reads 8 KB, all that the port
// delivers in the MMA's 64 cycles, and the MMAs ran at about 60 % of the
// tensor rate.
template <int NQ, int SB, int SM>
__global__ void __launch_bounds__(kThreadsWS, 1)
    k_tile_l2_tc(const __grid_constant__ CUtensorMap map_qh, const __grid_constant__ CUtensorMap map_ql, TileArgs a) {
    static_assert(SB <= SM, "a B buffer is reused no later than its slot");
    constexpr int kNQ = NQ;
    constexpr int kTmemCols = 512;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int panels = a.dim_p / 64;
    const int bpanel = kNQ * 128;
    uint8_t *sB = smem;                                     // SB buffers x (hi, lo) x panels x kNQ x 128 B
    const int bbuf = 2 * panels * bpanel;                   // bytes of one buffer
    uint8_t *mbase = sB + SB * bbuf;
    // slot: records [kNQ], path distances [kNQ][hp], bound constants [kNQ / 2][4], descriptor
    const int mbytes = kNQ * (int)sizeof(TileRec) + kNQ * a.hp * 4 + kNQ * 8 + (int)sizeof(ChunkDesc);
    auto mrec = [&](int sl) { return (TileRec *)(mbase + sl * mbytes); };
    auto mpath = [&](int sl) { return (float *)(mbase + sl * mbytes + kNQ * sizeof(TileRec)); };
    // columns 2i, 2i + 1 as (alpha_2i, alpha_2i+1, beta_2i, beta_2i+1), for packed FP32 tests
    auto mab = [&](int sl) { return (float *)(mbase + sl * mbytes + kNQ * sizeof(TileRec) + kNQ * a.hp * 4); };
    auto mdesc = [&](int sl) {
        return (ChunkDesc *)(mbase + sl * mbytes + kNQ * sizeof(TileRec) + kNQ * a.hp * 4 + kNQ * 8);
    };
    uint64_t *bars = (uint64_t *)(mbase + SM * mbytes);    // full[SM], mma_done[SM], epi_done[SM], a_full
    uint64_t *full = bars, *mma_done = bars + SM, *epi_done = bars + 2 * SM, *a_full = bars + 3 * SM;
    uint32_t *tslot = (uint32_t *)(bars + 3 * SM + 1);
    int *sitem = (int *)(tslot + 1);
    volatile int *sabort = sitem + 1;
    int32_t *sqid = sitem + 4;     // the staged chunk's query ids (producers only), kNQ

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) tc::tmem_alloc(tslot, kTmemCols);
    if (tid == 0) {
        for (int i = 0; i < SM; ++i) {
            tc::mbar_init(&full[i], kProducers);
            tc::mbar_init(&mma_done[i], 1);
            tc::mbar_init(&epi_done[i], kEpiWarps);
        }
        tc::mbar_init(a_full, kEpiWarps);
        tc::mbar_fence_init();
        *sabort = 0;
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t tacc = tmem + (uint32_t)a.dim_p;        // accumulator 0
    const int chunks16 = a.dim_p / 8;                       // 16-byte chunks per bf16 row
    auto fail = [&](int code) {
        *sabort = 1;
        atomicExch(a.status, code);
    };

    if (warp >= kProdWarp0 && warp < kMmaWarp) {
        // ================================================= producer warps
        const int ptid = tid - kProdWarp0 * 32;
        uint32_t g = 0;
        for (;;) {
            if (ptid == 0) *sitem = atomicAdd(a.work_counter, 1);
            tc::named_sync(1, kProducers);
            const int item = *sitem;
            tc::named_sync(1, kProducers);
            const bool stop = item >= a.n_items || *sabort;
            int4 it = make_int4(0, 0, 0, 0);
            int32_t pos = 0, size = 0;
            if (!stop) {
                it = a.items[item];
                const int64_t gnode = a.lvl_last + it.x;
                pos = a.npos[gnode];
                size = a.nsize[gnode];
            }
            const int total = it.z;
            const bool window = !stop && (it.w & kWindowItem) != 0;
            const int rbk = it.w & (kWindowItem - 1);
            // gather mode: chunks of the node's records; window mode: the node's
            // non-empty windows of kNQ consecutive query ids (from its list)
            const int32_t *wl = window ? a.wlist + (int64_t)it.x * a.nwin : nullptr;
            const int nchunks = stop ? 1 : window ? a.wcount[it.x] : (total + kNQ - 1) / kNQ;
            // window mode: this thread's column of window c (query c * kNQ +
            // ptid; threads past kNQ have none): its bitmap word and, for the
            // dense last level, its leaf mask and query data.  Loaded one
            // window ahead, so the loads overlap the previous window's work
            // (no barrier runs in between: a barrier would wait for them).
            struct Col {
                uint32_t word;
                uint64_t dmask;
                float2 ab;   // the query's bound constants (alpha, beta)
                int64_t seq;
                int32_t qid; // the query of the column
            };
            // (every load is predicated, so nothing waits for a load before its use)
            auto load_col = [&](int c) {
                Col w;
                w.word = 0;
                w.dmask = 0;
                w.ab = make_float2(0.f, 0.f);
                w.seq = 0;
                w.qid = (int32_t)((int64_t)c * kNQ + ptid);
                const int64_t wi = (int64_t)c * (kNQ / 32) + (ptid >> 5);
                const int64_t q = (int64_t)c * kNQ + ptid;
                if (window && ptid < kNQ && wi < a.nw) w.word = a.bits[(int64_t)it.x * a.nw + wi];
                if (window && a.dmask && ptid < kNQ && q < a.nq) {
                    w.dmask = a.dmask[(int64_t)it.x * a.nq + q];
                    w.ab = a.ab_q[q];
                    w.seq = a.seq_q[q];
                    if (a.qperm) w.qid = a.qperm[q];
                }
                return w;
            };
            // the window of chunk k + 1 and of chunk k + 2 are read ahead
            int wnext = (window && nchunks > 0) ? wl[0] : 0;
            Col nxt = load_col(wnext);
            int wnn = (window && nchunks > 1) ? wl[1] : 0;
            bool first_chunk = true;
            for (int k = 0; k < nchunks; ++k) {
                const int c = window ? wnext : k;   // window index, or chunk of the node's records
                const Col cur = nxt;
                wnext = wnn;
                nxt = load_col(wnext);
                wnn = (window && k + 2 < nchunks) ? wl[k + 2] : 0;
                const int sl = g % SM, sb = g % SB;
                // B buffer sb: the MMAs of chunk g - SB are done (every phase
                // of full[sl] up to chunk g - SM completed before that)
                if (g >= SB && !tc::mbar_wait(&mma_done[(g - SB) % SM], ((g - SB) / SM) & 1)) fail(4);
                if (window && ptid == 0) {
                    // the window's query rows, every panel of hi and of lo
                    tc::mbar_expect_tx_only(&full[sl], (uint32_t)(2 * panels * bpanel));
                    tc::tma_load_3d(sB + sb * bbuf, &map_qh, 0, c * kNQ, 0, &full[sl]);
                    tc::tma_load_3d(sB + sb * bbuf + panels * bpanel, &map_ql, 0, c * kNQ, 0, &full[sl]);
                }
                // slot sl (records, path distances, accumulator): chunk g - SM tested
                if (g >= SM && !tc::mbar_wait(&epi_done[sl], ((g - SM) / SM) & 1)) fail(7);
                int cnt;
                float *ab = mab(sl);
                if (stop) {
                    cnt = 0;
                } else if (window) {
                    cnt = kNQ;
                    // column ptid: its record, path distances and bound constants, or an empty record
                    if (ptid < kNQ) {
                        TileRec *mr = mrec(sl) + ptid;
                        const bool has = (cur.word >> (ptid & 31)) & 1u;
                        if (a.dmask) {
                            // dense last level: the record from the per-query arrays
                            // (no threshold: only the table test reads it, and
                            // dense chunks skip that test)
                            TileRec r;
                            r.q = cur.qid;
                            r.thr = 0.f;
                            r.seq = cur.seq;
                            r.mask = has ? cur.dmask : 0ull;
                            r.alpha = cur.ab.x;
                            r.beta = cur.ab.y;
                            *mr = r;
                            ab[(ptid >> 1) * 4 + (ptid & 1)] = r.alpha;
                            ab[(ptid >> 1) * 4 + 2 + (ptid & 1)] = r.beta;
                        } else if (has) {
                            const int64_t wi = (int64_t)it.x * a.nw + (int64_t)c * (kNQ / 32) + (ptid >> 5);
                            const int64_t o =
                                a.noff[it.x] + a.wpre[wi] + __popc(cur.word & ((1u << (ptid & 31)) - 1u));
                            const TileRec r = a.grec[o];
                            *mr = r;
                            ab[(ptid >> 1) * 4 + (ptid & 1)] = r.alpha;
                            ab[(ptid >> 1) * 4 + 2 + (ptid & 1)] = r.beta;
                            float *mp = mpath(sl) + ptid * a.hp;
                            for (int l = 0; l < a.hp; ++l) mp[l] = a.gpath[o * a.hp + l];
                        } else {
                            mr->mask = 0;
                            mr->q = c * kNQ + ptid;
                        }
                    }
                } else {
                    cnt = total - c * kNQ < kNQ ? total - c * kNQ : kNQ;
                    stage_chunk<NQ>(a, it.y + c * kNQ, cnt, mrec(sl), mpath(sl), sB + sb * bbuf,
                                    sB + sb * bbuf + panels * bpanel, chunks16, ptid, sqid);
                    // the bound constants, once every producer's record copies have landed
                    cp_async_wait_all();
                    tc::named_sync(1, kProducers);
                    for (int j = ptid; j < cnt; j += kProducers) {
                        const TileRec &r = mrec(sl)[j];
                        ab[(j >> 1) * 4 + (j & 1)] = r.alpha;
                        ab[(j >> 1) * 4 + 2 + (j & 1)] = r.beta;
                    }
                }
                if (ptid == 0) {
                    ChunkDesc dsc;
                    dsc.stop = stop ? 1 : 0;
                    dsc.new_item = first_chunk ? 1 : 0;
                    dsc.first = it.y + c * kNQ;
                    dsc.cnt = cnt;
                    dsc.pos = pos;
                    dsc.size = size;
                    dsc.rb = rbk * kRows;
                    dsc.pad_ = 0;
                    *mdesc(sl) = dsc;
                }
                first_chunk = false;
                // gather mode: the copies have landed and are visible to the
                // tensor cores (async proxy) before this thread arrives (window
                // mode: B comes by TMA, the async proxy itself)
                if (!window) {
                    cp_async_wait_all();
                    tc::fence_proxy_async_smem();
                }
                tc::mbar_arrive(&full[sl]);
                ++g;
            }
            if (stop) break;
        }
        cp_async_wait_all();
    } else if (warp == kMmaWarp) {
        // ================================================= MMA issuer
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_bf16_f32(kRows, kNQ);
            const uint32_t alo = tmem + (uint32_t)(a.dim_p / 2);   // A_lo
            const uint64_t bdesc0 = tc::sdesc_k_sw128(tc::smem_u32(sB));
            uint32_t a_par = 0;
            int64_t last_issued = -1;
            for (uint32_t g = 0;; ++g) {
                const int sl = g % SM;
                if (!tc::mbar_wait(&full[sl], (g / SM) & 1)) {
                    fail(5);
                    break;
                }
                const ChunkDesc dsc = *mdesc(sl);
                if (dsc.stop || *sabort) break;
                if (dsc.new_item) {
                    // the block's rows are in TMEM
                    if (!tc::mbar_wait(a_full, a_par)) {
                        fail(1);
                        break;
                    }
                    a_par ^= 1u;
                }
                tc::tc_fence_after();
                // descriptors of B's k-steps: the start address field holds
                // address / 16 in 14 bits, and shared addresses stay below
                // 2^18, so an offset adds to the descriptor without carry
                const uint64_t bh = bdesc0 + (uint64_t)(((g % SB) * bbuf) >> 4);
                const uint64_t bl = bh + (uint64_t)((panels * bpanel) >> 4);
                const uint32_t dt = tacc + (uint32_t)(sl * kNQ);
                for (int pnl = 0; pnl < panels; ++pnl) {
                    const uint64_t po = (uint64_t)((pnl * bpanel) >> 4);
                    const uint32_t ka = 32 * pnl;   // A columns of the panel (8 per k-step)
#pragma unroll
                    for (int s = 0; s < 4; ++s) {
                        tc::mma_bf16_ts(dt, tmem + ka + 8 * s, bh + po + 2 * s, idesc, (pnl | s) != 0);
                        tc::mma_bf16_ts(dt, tmem + ka + 8 * s, bl + po + 2 * s, idesc, 1u);
                        tc::mma_bf16_ts(dt, alo + ka + 8 * s, bh + po + 2 * s, idesc, 1u);
                    }
                }
                tc::mma_commit(&mma_done[sl]);
                last_issued = g;
            }
            // on an early exit, let issued MMAs finish before TMEM is released
            if (last_issued >= 0 && *sabort)
                tc::mbar_wait(&mma_done[last_issued % SM], (uint32_t)((last_issued / SM) & 1));
        }
    } else if (warp < kEpiWarps) {
        // ================================================= epilogue warps
        const int quad = warp & 3;                 // TMEM lane quadrant of this warp
        const int cc = (warp >> 2) * 32;           // its query columns [cc, cc + 32)
        const int r = quad * 32 + lane;            // row of the block
        const uint32_t tlane = (uint32_t)(quad * 32) << 16;
        bool valid = false;
        int64_t row = 0, rdel = kNever;
        uint64_t rowbit = 0, wmask = 0;
        float xn = 0.f, gx = 0.f;
        for (uint32_t g = 0;; ++g) {
            const int sl = g % SM;
            if (!tc::mbar_wait(&full[sl], (g / SM) & 1)) {
                fail(6);
                break;
            }
            const ChunkDesc dsc = *mdesc(sl);
            if (dsc.stop || *sabort) break;
            if (dsc.new_item) {
                // per-row constants of this block (thread = TMEM lane of its quadrant)
                const int nrow = dsc.size - dsc.rb;
                valid = r < nrow;
                row = (int64_t)dsc.pos + dsc.rb + r;
                const int32_t avg = dsc.size / a.F;
                int32_t jl = avg > 0 ? (dsc.rb + r) / avg : a.F - 1;
                if (jl > a.F - 1) jl = a.F - 1;
                const int rlast = min(quad * 32 + 31, min(nrow, kRows) - 1);
                wmask = 0;
                if (rlast >= quad * 32) {
                    int32_t j0 = avg > 0 ? (dsc.rb + quad * 32) / avg : a.F - 1;
                    int32_t j1 = avg > 0 ? (dsc.rb + rlast) / avg : a.F - 1;
                    j0 = min(j0, a.F - 1);
                    j1 = min(j1, a.F - 1);
                    wmask = ((j1 >= 63) ? ~0ull : ((1ull << (j1 + 1)) - 1ull)) & ~((1ull << j0) - 1ull);
                }
                float xn2 = 0.f;
                xn = 0.f;
                rdel = kNever;
                if (valid) {
                    xn2 = a.xn2[row];
                    xn = sqrtf(xn2) * (1.f + 1e-6f);
                    if (a.any_deleted) rdel = a.row_del[row];
                }
                // rows outside the node block match no leaf bit
                rowbit = valid ? (1ull << jl) : 0ull;
                // gamma_x = (cE2 - 1) |x|^2, rounded toward +inf (keeps the test conservative)
                gx = __fmul_ru(a.cE2 - 1.f, xn2) + 4.f * 1.1920929e-7f * xn2;
                // the row's split coordinates into TMEM (rows outside the block:
                // zeros).  Every MMA of the previous block is done: this warp
                // has waited for the previous chunk's.
                const int ncol = a.dim_p / 4;                  // this warp's share of A's dim_p columns
                for (int p = 0; p < ncol; p += 16) {
                    const int col = (warp >> 2) * ncol + p;
                    const bool lo = col >= a.dim_p / 2;
                    const int k0 = 2 * (lo ? col - a.dim_p / 2 : col);   // first coordinate
                    uint32_t v[16];
                    if (valid) {
                        const uint4 *src = reinterpret_cast<const uint4 *>((lo ? a.Xl : a.Xh) + row * a.dim_p + k0);
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const uint4 x = src[j];
                            v[4 * j] = x.x;
                            v[4 * j + 1] = x.y;
                            v[4 * j + 2] = x.z;
                            v[4 * j + 3] = x.w;
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; ++j) v[j] = 0u;
                    }
                    __syncwarp();   // tcgen05.st is warp-wide
                    tc::tmem_st16(tmem + tlane + (uint32_t)col, v);
                }
                tc::tmem_st_wait();
                tc::tc_fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(a_full);
            }
            if (!tc::mbar_wait(&mma_done[sl], (g / SM) & 1)) {
                fail(2);
                break;
            }
            tc::tc_fence_after();
            const int cnt = dsc.cnt;
            const TileRec *rec = mrec(sl);
            const float *pth = mpath(sl);
            // columns (queries) with a surviving leaf among the warp's 32 rows
            const unsigned live = (cc < kNQ && cc < cnt)
                                      ? __ballot_sync(0xffffffffu, cc + lane < cnt && (rec[cc + lane].mask & wmask) != 0)
                                      : 0u;
            if (live) {   // warp-uniform
                uint32_t v[32];
                tc::tmem_ld32(tacc + tlane + (uint32_t)(sl * kNQ + cc), v);
                tc::tmem_ld_wait();
                // bound test of all 32 columns, two at a time in packed FP32:
                // d~^2 <= thr^2 + E  <=>  -2 q.x <= w = fma(alpha_q, |x|, beta_q + gamma_x)
                // <=>  t = 2 q.x + w >= 0.  t is rounded once from the exact
                // sum, so its sign is that of the exact sum, and it is never
                // -0 (w >= +0 when it is zero): its sign bit marks a failed test.
                const float4 *abp = reinterpret_cast<const float4 *>(mab(sl) + cc * 2);
                uint32_t failbits = 0;
#pragma unroll
                for (int i = 0; i < 32; i += 2) {
                    const float4 c4 = abp[i / 2];   // alpha_i, alpha_i+1, beta_i, beta_i+1
                    float w0, w1, t0, t1;
                    add2(w0, w1, c4.z, c4.w, gx, gx);
                    fma2(w0, w1, c4.x, c4.y, xn, xn, w0, w1);
                    fma2(t0, t1, 2.f, 2.f, __uint_as_float(v[i]), __uint_as_float(v[i + 1]), w0, w1);
                    failbits |= ((__float_as_uint(t0) >> 31) << i) | ((__float_as_uint(t1) >> 31) << (i + 1));
                }
                uint32_t cand = ~failbits & live;
                // the few survivors: the row's leaf, visibility and the table lower bound
                uint32_t passbits = 0;
                while (cand) {
                    const int i = __ffs(cand) - 1;
                    cand &= cand - 1;
                    const TileRec &rc = rec[cc + i];
                    if (!(rc.mask & rowbit) || rdel <= rc.seq) continue;
                    bool ok = true;
                    // (the table lower bound can only drop a pair that the
                    // distance bound already dropped; dense chunks skip it)
                    for (int l = 0; l < a.h && ok && !a.dmask; ++l) {
                        const float T = a.table[(int64_t)l * a.n + row];
                        const float pl = pth[(cc + i) * a.hp + l];
                        const float eps = a.epsc * (T + pl + rc.thr) + a.lslack[l];
                        if (fabsf(T - pl) > rc.thr + eps) ok = false;
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
                if (wtot > 0) {
                    unsigned long long base = 0;
                    if (lane == 31) base = atomicAdd(a.out_count, (unsigned long long)wtot);
                    base = __shfl_sync(0xffffffffu, base, 31);
                    unsigned long long o = base + (unsigned long long)(incl - np);
                    while (passbits) {
                        const int i = __ffs(passbits) - 1;
                        passbits &= passbits - 1;
                        if ((int64_t)o < a.cap) {
                            a.out_q[o] = rec[cc + i].q;
                            a.out_row[o] = (int32_t)row;
                            if (a.out_qx) {
                                // q.x of column i, picked from the registers by a
                                // select tree on the bits of i (an indexed load
                                // would put v in local memory)
                                float e16[16], e8[8], e4[4], e2[2];
#pragma unroll
                                for (int k = 0; k < 16; ++k) e16[k] = __uint_as_float((i & 1) ? v[2 * k + 1] : v[2 * k]);
#pragma unroll
                                for (int k = 0; k < 8; ++k) e8[k] = (i & 2) ? e16[2 * k + 1] : e16[2 * k];
#pragma unroll
                                for (int k = 0; k < 4; ++k) e4[k] = (i & 4) ? e8[2 * k + 1] : e8[2 * k];
#pragma unroll
                                for (int k = 0; k < 2; ++k) e2[k] = (i & 8) ? e4[2 * k + 1] : e4[2 * k];
                                a.out_qx[o] = (i & 16) ? e2[1] : e2[0];
                            }
                        }
                        ++o;
                    }
                }
            }
            tc::tc_fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&epi_done[sl]);
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

// ---------------------------------------------------------------- node-major regrouping

__global__ void k_node_hist(const int32_t *__restrict__ enode, const uint64_t *__restrict__ emask, int64_t E,
                            int32_t *__restrict__ ncount) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x)
        if (emask[e]) atomicAdd(&ncount[enode[e]], 1);
}

// scatter each entry's record (query, threshold, norms, sequence number,
// leaf mask) and path distances to its node's slot, so a tile reads its
// queries' data contiguously
// the per-query constants of the squared-form bound test, all rounded up:
// keep iff d~^2 <= thr^2 + cE1 |q||x| + cE2 (|q| + |x|)^2 with
// d~^2 = |q|^2 + |x|^2 - 2 q.x, i.e. -2 q.x <= beta + alpha |x| + gamma_x,
// alpha = (cE1 + 2 cE2) |q|, beta = thr^2 + (cE2 - 1) |q|^2
__device__ __forceinline__ void bound_consts(float thr, float qn2, float cE1, float cE2, float &alpha, float &beta) {
    const float qn = sqrtf(qn2) * (1.f + 1e-6f);
    const float t = thr * 1.0000039f;
    alpha = __fmul_ru(cE1 + 2.f * cE2, qn) * 1.000001f;
    beta = __fadd_ru(__fmul_ru(t, t), __fmul_ru(cE2 - 1.f, qn2)) + 4.f * 1.1920929e-7f * (t * t + qn2);
}

// For every node, its non-empty windows (windows of wpw bitmap words) in
// ascending order, and their number: a warp per node.
__global__ void k_window_list(const uint32_t *__restrict__ bits, int64_t nn, int64_t nw, int wpw, int64_t nwin,
                              int32_t *__restrict__ wl, int32_t *__restrict__ wcnt) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t node = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; node < nn; node += nwarps) {
        int cnt = 0;
        for (int64_t c0 = 0; c0 < nwin; c0 += 32) {
            const int64_t c = c0 + lane;
            uint32_t any = 0;
            if (c < nwin)
                for (int j = 0; j < wpw; ++j) {
                    const int64_t w = c * wpw + j;
                    if (w < nw) any |= bits[node * nw + w];
                }
            const unsigned b = __ballot_sync(0xffffffffu, any != 0u);
            if (any) wl[node * nwin + cnt + __popc(b & ((1u << lane) - 1u))] = (int32_t)c;
            cnt += __popc(b);
        }
        if (lane == 0) wcnt[node] = cnt;
    }
}

// the bound constants (alpha, beta) and the sequence number of the query in
// each column position of the dense last level (query perm[i] at position i)
__global__ void k_query_consts(const float *__restrict__ thr, const float *__restrict__ qn2,
                               const int64_t *__restrict__ qseq, const int32_t *__restrict__ perm, int64_t nq,
                               float cE1, float cE2, float2 *__restrict__ ab, int64_t *__restrict__ seq) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nq; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = perm ? (int64_t)perm[i] : i;
        float al, be;
        bound_consts(thr[q], qn2 ? qn2[q] : 0.f, cE1, cE2, al, be);
        ab[i] = make_float2(al, be);
        seq[i] = qseq[q];
    }
}

__global__ void k_node_scatter(const int32_t *__restrict__ eq, const int32_t *__restrict__ enode,
                               const uint64_t *__restrict__ emask, const float *__restrict__ path, int h, int hp,
                               int64_t E, const float *__restrict__ thr, const float *__restrict__ qn2, float cE1,
                               float cE2, const int64_t *__restrict__ qseq, const int64_t *__restrict__ noff,
                               int32_t *__restrict__ cursor, TileRec *__restrict__ grec, int32_t *__restrict__ gq,
                               float *__restrict__ gpath) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t m = emask[e];
        if (!m) continue;
        const int32_t nd = enode[e];
        const int64_t o = noff[nd] + atomicAdd(&cursor[nd], 1);
        const int32_t q = eq[e];
        TileRec r;
        r.q = q;
        r.thr = thr[q];
        bound_consts(r.thr, qn2 ? qn2[q] : 0.f, cE1, cE2, r.alpha, r.beta);
        r.seq = qseq[q];
        r.mask = m;
        grec[o] = r;
        gq[o] = q;
        for (int l = 0; l < hp; ++l) gpath[o * hp + l] = l < h ? path[e * h + l] : 0.f;
    }
}

// Regrouping through a (node x query) bitmap: bit q of row p is set when the
// entry (q, p) has a surviving leaf.  Row popcounts give the per-node counts,
// and an entry's slot within its node is the number of set bits before it,
// so entries of a node land in ascending query order with no contended
// atomics (each 32-bit word collects at most 32 entries).
__global__ void k_bits_set(const int32_t *__restrict__ eq, const int32_t *__restrict__ enode,
                           const uint64_t *__restrict__ emask, int64_t E, int64_t nw, uint32_t *__restrict__ bits) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
        if (!emask[e]) continue;
        const int32_t q = eq[e];
        atomicOr(&bits[(int64_t)enode[e] * nw + (q >> 5)], 1u << (q & 31));
    }
}

// block per row: exclusive popcount prefix of the row's words, and the count
__global__ void k_bits_rows(const uint32_t *__restrict__ bits, int64_t nn, int64_t nw, int32_t *__restrict__ wpre,
                            int32_t *__restrict__ ncount) {
    __shared__ int32_t warp_tot[32];
    __shared__ int32_t carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    for (int64_t row = blockIdx.x; row < nn; row += gridDim.x) {
        if (tid == 0) carry = 0;
        __syncthreads();
        for (int64_t w0 = 0; w0 < nw; w0 += blockDim.x) {
            const int64_t w = w0 + tid;
            const int32_t c = w < nw ? __popc(bits[row * nw + w]) : 0;
            int32_t incl = c;
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            if (lane == 31) warp_tot[warp] = incl;
            __syncthreads();
            int32_t before = carry;
            for (int i = 0; i < warp; ++i) before += warp_tot[i];
            if (w < nw) wpre[row * nw + w] = before + incl - c;
            __syncthreads();
            if (tid == 0) {
                int32_t t = 0;
                for (int i = 0; i < nwarps; ++i) t += warp_tot[i];
                carry += t;
            }
            __syncthreads();
        }
        if (tid == 0) ncount[row] = carry;
        __syncthreads();
    }
}

__device__ __forceinline__ void write_rec(int64_t e, int64_t o, const int32_t *eq, const uint64_t *emask,
                                          const float *path, int h, int hp, const float *thr, const float *qn2,
                                          float cE1, float cE2, const int64_t *qseq, TileRec *grec, int32_t *gq,
                                          float *gpath) {
    const int32_t q = eq[e];
    TileRec r;
    r.q = q;
    r.thr = thr[q];
    bound_consts(r.thr, qn2 ? qn2[q] : 0.f, cE1, cE2, r.alpha, r.beta);
    r.seq = qseq[q];
    r.mask = emask[e];
    grec[o] = r;
    gq[o] = q;
    for (int l = 0; l < hp; ++l) gpath[o * hp + l] = l < h ? path[e * h + l] : 0.f;
}

__global__ void k_node_scatter_bits(const int32_t *__restrict__ eq, const int32_t *__restrict__ enode,
                                    const uint64_t *__restrict__ emask, const float *__restrict__ path, int h, int hp,
                                    int64_t E, const float *__restrict__ thr, const float *__restrict__ qn2,
                                    float cE1, float cE2, const int64_t *__restrict__ qseq,
                                    const int64_t *__restrict__ noff, const uint32_t *__restrict__ bits, const int32_t *__restrict__ wpre, int64_t nw,
                                    TileRec *__restrict__ grec, int32_t *__restrict__ gq, float *__restrict__ gpath) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
        if (!emask[e]) continue;
        const int32_t q = eq[e];
        const int64_t wi = (int64_t)enode[e] * nw + (q >> 5);
        const int64_t o = noff[enode[e]] + wpre[wi] + __popc(bits[wi] & ((1u << (q & 31)) - 1u));
        write_rec(e, o, eq, emask, path, h, hp, thr, qn2, cE1, cE2, qseq, grec, gq, gpath);
    }
}

// work items: one per 128-row block of every node that has entries
// (also sums the (query, row) pairs the blocks hold into *pairs)
__global__ void k_items_per_node(const int32_t *__restrict__ ncount, const int32_t *__restrict__ nsize, int64_t nn,
                                 int64_t *__restrict__ nitems, unsigned long long *__restrict__ pairs) {
    unsigned long long p = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nn; i += (int64_t)gridDim.x * blockDim.x) {
        nitems[i] = ncount[i] > 0 ? (int64_t)((nsize[i] + kRows - 1) / kRows) : 0;
        p += (unsigned long long)ncount[i] * (unsigned long long)nsize[i];
    }
    for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
    if ((threadIdx.x & 31) == 0 && p) atomicAdd(pairs, p);
    if (blockIdx.x == 0 && threadIdx.x == 0) nitems[nn] = 0;
}

// win_min: nodes with at least this many entries get window-mode items
__global__ void k_fill_items(const int32_t *__restrict__ ncount, const int32_t *__restrict__ nsize,
                             const int64_t *__restrict__ noff, const int64_t *__restrict__ ioff, int64_t nn,
                             int64_t win_min, int4 *__restrict__ items) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nn; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = ncount[i];
        if (c == 0) continue;
        const int32_t blocks = (nsize[i] + kRows - 1) / kRows;
        const int flag = c >= win_min ? kWindowItem : 0;
        for (int32_t b = 0; b < blocks; ++b) items[ioff[i] + b] = make_int4((int)i, (int)noff[i], c, b | flag);
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

size_t tile_smem_bytes(int dim_p, int h, int kNQ, int SB, int SM) {
    const int panels = dim_p / 64;
    size_t b = 1024;                                              // alignment slack
    b += (size_t)SB * 2 * panels * kNQ * 128;
    b += SM * ((size_t)kNQ * sizeof(TileRec) + (size_t)kNQ * ((h + 3) & ~3) * 4 + (size_t)kNQ * 8 + 32);
    b += (3 * SM + 1) * 8 + 4 + 4 * 4 + 16 + (size_t)kNQ * 4;
    return b;
}

}  // namespace

void tc_bound_coeffs(int dim_p, float &cE1, float &cE2) {
    // |d~^2 - d^2| <= cE1 |q||x| + cE2 (|q| + |x|)^2 (see the file comment)
    const double u23 = 1.0 / 8388608.0;
    const double kterms = 3.0 * dim_p + 2.0;
    const double gam = kterms * u23 / (1.0 - kterms * u23);
    cE1 = (float)(2.02 * (3.01 / 65536.0 + gam) * 1.01);
    cE2 = (float)(1.0 / 2097152.0);
}

bool tc_supported(const Tree &t) { return t.metric == GTS_L2 && t.dim > 0 && t.dim <= 448 && t.n > 0; }

void tc_prepare(Tree &t, TcCache &c, cudaStream_t st) {
    if (c.ready) return;
    c.dim_p = ((t.dim + 63) / 64) * 64;
    c.Xh.alloc((size_t)t.n * c.dim_p * 2, st);
    c.Xl.alloc((size_t)t.n * c.dim_p * 2, st);
    c.xn2.alloc(t.n, st);
    k_split_rows<<<nblk(t.n * 32), 256, 0, st>>>(t.X.get(), t.dim, c.dim_p, t.n, (__nv_bfloat16 *)c.Xh.get(),
                                                (__nv_bfloat16 *)c.Xl.get(), c.xn2.get(), nullptr);
    check_launch("split rows");
    GTS_CUDA(cudaStreamSynchronize(st));
    c.Xh.persist();
    c.Xl.persist();
    c.xn2.persist();
    c.ready = true;
}

void tc_split_queries(const float *Q, int64_t nq, int dim, int dim_p, DBuf<uint8_t> &Qh, DBuf<uint8_t> &Ql,
                      DBuf<float> &qn2, cudaStream_t st, const int32_t *sel) {
    Qh.alloc((size_t)(nq > 0 ? nq : 1) * dim_p * 2, st);
    Ql.alloc((size_t)(nq > 0 ? nq : 1) * dim_p * 2, st);
    qn2.alloc(nq > 0 ? nq : 1, st);
    if (nq > 0)
        k_split_rows<<<nblk(nq * 32), 256, 0, st>>>(Q, dim, dim_p, nq, (__nv_bfloat16 *)Qh.get(),
                                                   (__nv_bfloat16 *)Ql.get(), qn2.get(), sel);
    check_launch("split queries");
}

bool regroup_uses_bits(const Tree &t, int64_t nq, int64_t E) {
    // the bitmap costs a pass over nodes x query words; it pays when the
    // entries are dense in it (at least one per four words) and it stays small
    const int64_t nn = t.lvl_off[t.h] - t.lvl_off[t.h - 1];
    const int64_t words = nn * ((nq + 31) / 32);
    return words * 8 <= ((int64_t)1 << 30) && words <= 4 * E;
}

int64_t tc_regroup(const Tree &t, const TcQuery &tq, TcRegroup &rg, cudaStream_t st, const int32_t *counts,
                   bool window_ok) {
    const int64_t E = tq.E;
    const int64_t nn = t.lvl_off[t.h] - t.lvl_off[t.h - 1];
    // the bitmap form when its two (node x query-word) arrays stay small
    const int64_t nw = (tq.nq + 31) / 32;
    const bool use_bits = regroup_uses_bits(t, tq.nq, E);
    DBuf<uint32_t> &bits = rg.bits;
    DBuf<int32_t> &wpre = rg.wpre;
    bits.alloc(use_bits ? nn * nw : 0, st);
    wpre.alloc(use_bits ? nn * nw : 0, st);
    rg.nw = use_bits ? nw : 0;
    DBuf<int32_t> own((counts && !use_bits) ? 0 : nn, st), cursor(use_bits ? 0 : nn, st);
    if (use_bits) {
        GTS_CUDA(cudaMemsetAsync(bits.get(), 0, nn * nw * 4, st));
        k_bits_set<<<nblk(E), 256, 0, st>>>(tq.eq, tq.enode, tq.emask, E, nw, bits.get());
        k_bits_rows<<<(unsigned)std::min<int64_t>(nn, 65535), 256, 0, st>>>(bits.get(), nn, nw, wpre.get(), own.get());
    } else {
        GTS_CUDA(cudaMemsetAsync(cursor.get(), 0, nn * 4, st));
        if (!counts) {
            GTS_CUDA(cudaMemsetAsync(own.get(), 0, nn * 4, st));
            k_node_hist<<<nblk(E), 256, 0, st>>>(tq.enode, tq.emask, E, own.get());
        }
    }
    const int32_t *ncnt = (counts && !use_bits) ? counts : own.get();
    DBuf<int64_t> c64(nn + 1, st), nitems(nn + 1, st), ioff(nn + 1, st);
    DBuf<int64_t> &noff = rg.noff;
    noff.alloc(nn + 1, st);
    k_i32_to_i64_tc<<<nblk(nn), 256, 0, st>>>(ncnt, nn, c64.get());
    exscan(c64.get(), noff.get(), nn + 1, st);
    int64_t total_entries = 0;
    GTS_CUDA(cudaMemcpyAsync(&total_entries, noff.get() + nn, 8, cudaMemcpyDeviceToHost, st));
    GTS_CUDA(cudaStreamSynchronize(st));
    const int64_t ne = total_entries > 0 ? total_entries : 1;
    const int hp = (t.h + 3) & ~3;
    rg.grec.alloc(ne, st);
    rg.gq.alloc(ne, st);
    rg.gpath.alloc(ne * hp, st);
    if (use_bits)
        k_node_scatter_bits<<<nblk(E), 256, 0, st>>>(tq.eq, tq.enode, tq.emask, tq.path, t.h, hp, E, tq.thr, tq.qn2,
                                                     tq.cE1, tq.cE2, tq.qseq, noff.get(), bits.get(), wpre.get(), nw, rg.grec.get(),
                                                     rg.gq.get(), rg.gpath.get());
    else
        k_node_scatter<<<nblk(E), 256, 0, st>>>(tq.eq, tq.enode, tq.emask, tq.path, t.h, hp, E, tq.thr, tq.qn2,
                                                tq.cE1, tq.cE2, tq.qseq, noff.get(), cursor.get(), rg.grec.get(), rg.gq.get(),
                                                rg.gpath.get());
    const int32_t *lsize = t.nsize.get() + t.lvl_off[t.h - 1];
    DBuf<unsigned long long> pairs(1, st);
    GTS_CUDA(cudaMemsetAsync(pairs.get(), 0, 8, st));
    k_items_per_node<<<nblk(nn), 256, 0, st>>>(ncnt, lsize, nn, nitems.get(), pairs.get());
    exscan(nitems.get(), ioff.get(), nn + 1, st);
    int64_t total_items = 0;
    unsigned long long total_pairs = 0;
    GTS_CUDA(cudaMemcpyAsync(&total_items, ioff.get() + nn, 8, cudaMemcpyDeviceToHost, st));
    GTS_CUDA(cudaMemcpyAsync(&total_pairs, pairs.get(), 8, cudaMemcpyDeviceToHost, st));
    GTS_CUDA(cudaStreamSynchronize(st));
    rg.n_pairs = (int64_t)total_pairs;
    rg.n_items = total_items;
    rg.n_entries = total_entries;
    rg.n_chunks = (total_entries + 127) / 128;
    if (total_items > 0) {
        rg.items.alloc(total_items, st);
        // window mode for nodes holding at least half of the batch
        const int64_t win_min = (use_bits && window_ok) ? std::max<int64_t>(1, (tq.nq + 1) / 2) : INT64_MAX;
        k_fill_items<<<nblk(nn), 256, 0, st>>>(ncnt, lsize, noff.get(), ioff.get(), nn, win_min, rg.items.get());
    }
    check_launch("tile regroup");
    return total_items;
}

int64_t tc_dense_items(const Tree &t, int64_t nq, const uint64_t *dmask, TcRegroup &rg, cudaStream_t st) {
    const int64_t nn = t.lvl_off[t.h] - t.lvl_off[t.h - 1];
    const int64_t nw = rg.nw;
    DBuf<int32_t> ncnt(nn, st);
    rg.wpre.alloc(nn * nw, st);
    k_bits_rows<<<(unsigned)std::min<int64_t>(nn, 65535), 256, 0, st>>>(rg.bits.get(), nn, nw, rg.wpre.get(),
                                                                         ncnt.get());
    DBuf<int64_t> c64(nn + 1, st), nitems(nn + 1, st), ioff(nn + 1, st);
    rg.noff.alloc(nn + 1, st);
    k_i32_to_i64_tc<<<nblk(nn), 256, 0, st>>>(ncnt.get(), nn, c64.get());
    exscan(c64.get(), rg.noff.get(), nn + 1, st);
    const int32_t *lsize = t.nsize.get() + t.lvl_off[t.h - 1];
    DBuf<unsigned long long> pairs(1, st);
    GTS_CUDA(cudaMemsetAsync(pairs.get(), 0, 8, st));
    k_items_per_node<<<nblk(nn), 256, 0, st>>>(ncnt.get(), lsize, nn, nitems.get(), pairs.get());
    exscan(nitems.get(), ioff.get(), nn + 1, st);
    int64_t total_items = 0, total_entries = 0;
    unsigned long long total_pairs = 0;
    GTS_CUDA(cudaMemcpyAsync(&total_items, ioff.get() + nn, 8, cudaMemcpyDeviceToHost, st));
    GTS_CUDA(cudaMemcpyAsync(&total_entries, rg.noff.get() + nn, 8, cudaMemcpyDeviceToHost, st));
    GTS_CUDA(cudaMemcpyAsync(&total_pairs, pairs.get(), 8, cudaMemcpyDeviceToHost, st));
    GTS_CUDA(cudaStreamSynchronize(st));
    rg.dmask = dmask;
    rg.n_items = total_items;
    rg.n_entries = total_entries;
    rg.n_pairs = (int64_t)total_pairs;
    rg.n_chunks = 0;
    if (total_items > 0) {
        rg.items.alloc(total_items, st);
        k_fill_items<<<nblk(nn), 256, 0, st>>>(ncnt.get(), lsize, rg.noff.get(), ioff.get(), nn, 0, rg.items.get());
    }
    check_launch("dense tile items");
    return total_items;
}

int64_t tc_run(const Tree &t, const TcCache &c, const TcQuery &tq, const TcRegroup &rg, DBuf<int32_t> &out_q,
               DBuf<int32_t> &out_row, int64_t cap_hint, int *launches, cudaStream_t st, DBuf<float> *out_qx) {
    *launches = 0;
    if (rg.n_items == 0) return 0;
    int dev = 0, sms = 0;
    GTS_CUDA(cudaGetDevice(&dev));
    GTS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const TileShape shp = shape_for(c.dim_p, tq.chunk);
    const int nq_chunk = shp.nq;
    int smem_optin = 0;
    GTS_CUDA(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    // TMEM: A (dim_p columns) and the slots' accumulators share 512 columns
    GTS_REQUIRE(c.dim_p + shp.sm * nq_chunk <= 512, GTS_ECUDA, "tensor-core tile: TMEM columns");
    const size_t smem = tile_smem_bytes(c.dim_p, t.h, nq_chunk, shp.sb, shp.sm);
    GTS_REQUIRE(smem <= (size_t)smem_optin, GTS_ECUDA, "tensor-core tile: shared memory");
    void (*kern)(const CUtensorMap, const CUtensorMap, TileArgs) =
        nq_chunk == 96    ? k_tile_l2_tc<96, 4, 4>
        : nq_chunk == 128 ? k_tile_l2_tc<128, 3, 3>
        : shp.sb == 4     ? (nq_chunk == 64 ? k_tile_l2_tc<64, 4, 4> : k_tile_l2_tc<32, 4, 4>)
        : nq_chunk == 64  ? k_tile_l2_tc<64, 2, 3>
        : shp.sm == 4     ? k_tile_l2_tc<32, 2, 4>
                          : k_tile_l2_tc<32, 2, 2>;
    GTS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // CTAs per SM: shared memory (each CTA also has 1 KB reserved), the 512
    // TMEM columns, and registers
    int smem_sm = 0, regs_sm = 0;
    GTS_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    GTS_CUDA(cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev));
    cudaFuncAttributes fa;
    GTS_CUDA(cudaFuncGetAttributes(&fa, kern));
    int per_sm = (int)(smem_sm / (smem + 1024));
    const int regs_cta = ((fa.numRegs + 7) / 8) * 8 * kThreadsWS;
    if (regs_cta > 0 && per_sm > regs_sm / regs_cta) per_sm = regs_sm / regs_cta;
    if (per_sm > 1) per_sm = 1;   // TMEM: every CTA takes all 512 columns
    if (per_sm < 1) per_sm = 1;
    const int64_t grid = std::min<int64_t>(rg.n_items, (int64_t)sms * per_sm);
    // the batch's split query rows, for window-mode chunks (TMA, 128 rows)
    const CUtensorMap map_qh = make_panel_map(tq.Qh, tq.nq, c.dim_p, nq_chunk);
    const CUtensorMap map_ql = make_panel_map(tq.Ql, tq.nq, c.dim_p, nq_chunk);
    DBuf<int> counter(1, st), status(1, st);
    DBuf<unsigned long long> count(1, st);
    int64_t cap = cap_hint > 0 ? cap_hint : 1 << 20;
    float cE1 = 0.f, cE2 = 0.f;
    tc_bound_coeffs(c.dim_p, cE1, cE2);
    // window mode: every node's non-empty windows
    const int64_t nn = t.lvl_off[t.h] - t.lvl_off[t.h - 1];
    const int64_t nwin = (tq.nq + nq_chunk - 1) / nq_chunk;
    const bool wl_on = rg.bits.get() != nullptr && rg.nw > 0;
    DBuf<int32_t> wl(wl_on ? nn * nwin : 1, st), wcnt(wl_on ? nn : 1, st);
    if (wl_on) {
        k_window_list<<<nblk(nn * 32), 256, 0, st>>>(rg.bits.get(), nn, rg.nw, nq_chunk / 32, nwin, wl.get(),
                                                     wcnt.get());
        check_launch("window lists");
        ++*launches;
    }
    // dense last level: the queries' bound constants and sequence numbers in
    // column order, once per batch
    DBuf<float2> abq(rg.dmask ? tq.nq : 1, st);
    DBuf<int64_t> seqp(rg.dmask ? tq.nq : 1, st);
    if (rg.dmask) {
        k_query_consts<<<nblk(tq.nq), 256, 0, st>>>(tq.thr, tq.qn2, tq.qseq, tq.perm, tq.nq, cE1, cE2, abq.get(),
                                                    seqp.get());
        check_launch("query bound constants");
        ++*launches;
    }
    for (int attempt = 0; attempt < 2; ++attempt) {
        out_q.alloc(cap, st);
        out_row.alloc(cap, st);
        if (out_qx) out_qx->alloc(cap, st);
        GTS_CUDA(cudaMemsetAsync(counter.get(), 0, 4, st));
        GTS_CUDA(cudaMemsetAsync(status.get(), 0, 4, st));
        GTS_CUDA(cudaMemsetAsync(count.get(), 0, 8, st));
        TileArgs a;
        a.dim = t.dim;
        a.dim_p = c.dim_p;
        a.F = t.F;
        a.h = t.h;
        a.n = t.n;
        a.xn2 = c.xn2.get();
        a.Xh = reinterpret_cast<const __nv_bfloat16 *>(c.Xh.get());
        a.Xl = reinterpret_cast<const __nv_bfloat16 *>(c.Xl.get());
        a.table = t.table.get();
        a.row_del = t.row_del.get();
        a.npos = t.npos.get();
        a.nsize = t.nsize.get();
        a.lvl_last = t.lvl_off[t.h - 1];
        a.Qh = tq.Qh;
        a.Ql = tq.Ql;
        a.grec = rg.grec.get();
        a.gq = rg.gq.get();
        a.gpath = rg.gpath.get();
        a.hp = (t.h + 3) & ~3;
        a.items = rg.items.get();
        a.n_items = rg.n_items;
        a.work_counter = counter.get();
        a.out_q = out_q.get();
        a.out_row = out_row.get();
        a.out_qx = out_qx ? out_qx->get() : nullptr;
        a.cap = cap;
        a.out_count = count.get();
        a.status = status.get();
        a.epsc = tq.epsc;
        for (int l = 0; l < kMaxHeight; ++l) a.lslack[l] = tq.lslack[l];
        a.cE1 = cE1;
        a.cE2 = cE2;
        a.any_deleted = tq.any_deleted;
        a.bits = rg.bits.get();
        a.wpre = rg.wpre.get();
        a.noff = rg.noff.get();
        a.nw = rg.nw;
        a.nq = tq.nq;
        a.dmask = rg.dmask;
        a.ab_q = abq.get();
        a.seq_q = seqp.get();
        a.qperm = tq.perm;
        a.wlist = wl.get();
        a.wcount = wcnt.get();
        a.nwin = nwin;
        kern<<<(unsigned)grid, kThreadsWS, smem, st>>>(map_qh, map_ql, a);
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

// ---------------------------------------------------------------- dense pivot distances

namespace {

constexpr int kDenseQ = 128;   // queries per CTA (MMA N)

struct DenseTcArgs {
    const __nv_bfloat16 *Ph, *Pl;   // the level's pivots, split bf16 rows [P, dim_p]
    const float *pn2, *pnu;         // their squared norms (FP64 sums, rounded) and norms rounded up
    const float *qn2, *qnu;         // the same for the queries
    const int32_t *piv;             // pivot row of each node (-1: empty), for the exact recomputation
    const float *X, *Q;             // FP32 rows and queries
    int dim, dim_p;
    int64_t P, nq;
    float cE1, cE2;
    float *out;                     // [nq, P]: out[query * P + p]
    // optional: the columns (B rows) are positions, position j holding query
    // perm[j] (null: j), and outT[p * nq + j] receives the same entries
    // transposed (the layout of the dense leaf masks)
    const int32_t *perm;
    float *outT;
    unsigned *slack;                // the largest |d~ - d| bound written (float bits)
    int *status;
};

// PTX approximations; every use below checks its own result (a residual),
// so no error bound of theirs is relied on
__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// |x| rounded up, for the error bound
__global__ void k_norms_up(const float *__restrict__ n2, int64_t n, float *__restrict__ nu) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        nu[i] = __fmul_ru(__fsqrt_ru(n2[i]), 1.f + 1e-6f);
}

// D[q, p] for 128 pivots x 128 queries per CTA: the pivots' split rows into
// TMEM (TMEM lane = pivot), the queries' by one TMA copy into shared memory,
// three MMAs per 16-wide k-step, then per entry d~^2 = (|p|^2 + |q|^2) -
// 2 p.q~ with |d~^2 - d^2| <= E (the tile kernel's bound, here with 2 cE2).
// The entry stores t ~ sqrt(d~^2) and the level's absolute slack takes an
// upper bound of |t - d|: |t - sqrt(d~^2)| <= |t^2 - d~^2| / t (the residual
// of t, computed by one fused multiply-add) and |sqrt(d~^2) - d| = |d~^2 -
// d^2| / (sqrt(d~^2) + d) <= E / ((1 + sqrt(15 / 16)) sqrt(d~^2)) when d~^2 >
// 16 E (d >= sqrt(d~^2 - E)), with 1 / t from an approximate reciprocal
// checked by its own residual (0.5085 covers 1 / (1 + sqrt(15 / 16)) and
// 1 / (1 - 2^-13)).  An entry near the pivot (d~^2 <= 16 E, or a bound above
// 2^-12 (|p| + |q|), where the product form cancels) is recomputed in FP32 as
// the sum of squared differences instead, within the FP32 relative bound the
// search allows for any distance, and adds nothing to the slack.
// Warp w: TMEM lane quadrant w % 4 (32 pivots); A columns (w / 4 = 0: hi,
// 1: lo) and accumulator columns [64 (w / 4), 64 (w / 4) + 64).
__global__ void __launch_bounds__(256, 1)
    k_dense_tc(const __grid_constant__ CUtensorMap map_qh, const __grid_constant__ CUtensorMap map_ql, DenseTcArgs a) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int panels = a.dim_p / 64;
    const int bpanel = kDenseQ * 128;
    uint8_t *sB = smem;                                   // hi panels, then lo panels
    uint64_t *bars = (uint64_t *)(sB + 2 * panels * bpanel);
    uint32_t *tslot = (uint32_t *)(bars + 2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quad = warp & 3, half = warp >> 2;
    const int ncols = a.dim_p + kDenseQ <= 256 ? 256 : 512;
    const int64_t p0 = (int64_t)blockIdx.x * kRows, q0 = (int64_t)blockIdx.y * kDenseQ;
    if (warp == 0) tc::tmem_alloc(tslot, ncols);
    if (tid == 0) {
        tc::mbar_init(&bars[0], 1);
        tc::mbar_init(&bars[1], 1);
        tc::mbar_fence_init();
        tc::mbar_expect_tx(&bars[0], (uint32_t)(2 * panels * bpanel));
        tc::tma_load_3d(sB, &map_qh, 0, (int32_t)q0, 0, &bars[0]);
        tc::tma_load_3d(sB + panels * bpanel, &map_ql, 0, (int32_t)q0, 0, &bars[0]);
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t tacc = tmem + (uint32_t)a.dim_p;
    const uint32_t tlane = (uint32_t)(quad * 32) << 16;
    // A: this thread's pivot row, hi in columns [0, dim_p / 2), lo after
    const int64_t p = p0 + quad * 32 + lane;
    const bool pv = p < a.P;
    for (int c = 0; c < a.dim_p / 2; c += 16) {
        const int col = half * (a.dim_p / 2) + c;
        uint32_t v[16];
        if (pv) {
            const uint4 *src = reinterpret_cast<const uint4 *>((half ? a.Pl : a.Ph) + p * a.dim_p + 2 * c);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint4 x = src[j];
                v[4 * j] = x.x;
                v[4 * j + 1] = x.y;
                v[4 * j + 2] = x.z;
                v[4 * j + 3] = x.w;
            }
        } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = 0u;
        }
        tc::tmem_st16(tmem + tlane + (uint32_t)col, v);
    }
    tc::tmem_st_wait();
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (tid == 0) {
        if (!tc::mbar_wait(&bars[0], 0)) {
            atomicExch(a.status, 1);
        } else {
            const uint32_t idesc = tc::idesc_bf16_f32(kRows, kDenseQ);
            const uint32_t alo = tmem + (uint32_t)(a.dim_p / 2);
            const uint64_t bh = tc::sdesc_k_sw128(tc::smem_u32(sB));
            const uint64_t bl = bh + (uint64_t)((panels * bpanel) >> 4);
            for (int pnl = 0; pnl < panels; ++pnl) {
                const uint64_t po = (uint64_t)((pnl * bpanel) >> 4);
                const uint32_t ka = 32 * pnl;
#pragma unroll
                for (int s4 = 0; s4 < 4; ++s4) {
                    tc::mma_bf16_ts(tacc, tmem + ka + 8 * s4, bh + po + 2 * s4, idesc, (pnl | s4) != 0);
                    tc::mma_bf16_ts(tacc, tmem + ka + 8 * s4, bl + po + 2 * s4, idesc, 1u);
                    tc::mma_bf16_ts(tacc, alo + ka + 8 * s4, bh + po + 2 * s4, idesc, 1u);
                }
            }
            tc::mma_commit(&bars[1]);
        }
    }
    __syncthreads();
    // (warp-uniform: the TMEM loads below are warp-wide)
    const bool ok = __all_sync(0xffffffffu, *(volatile int *)a.status == 0 && tc::mbar_wait(&bars[1], 0));
    tc::tc_fence_after();
    float umax = 0.f;
    if (ok) {
        const float p2 = pv ? a.pn2[p] : 0.f;
        const float pn = pv ? a.pnu[p] : 0.f;
        const int32_t prow = pv ? a.piv[p] : -1;
        for (int c0 = half * (kDenseQ / 2); c0 < (half + 1) * (kDenseQ / 2); c0 += 32) {
            uint32_t v[32];
            tc::tmem_ld32(tacc + tlane + (uint32_t)c0, v);
            tc::tmem_ld_wait();
            uint32_t redo = 0;   // entries near the pivot, recomputed below
            float tv[32];        // this thread's 32 entries, for the transposed copy
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const int64_t j = q0 + c0 + i;   // column (position)
                tv[i] = 0.f;
                if (!pv || j >= a.nq) continue;
                const int64_t q = a.perm ? (int64_t)a.perm[j] : j;
                const float q2 = a.qn2[j], qn = a.qnu[j];
                const float sn = __fadd_ru(pn, qn);
                const float E = __fadd_ru(__fmul_ru(a.cE1, __fmul_ru(pn, qn)), __fmul_ru(2.f * a.cE2, __fmul_ru(sn, sn)));
                const float d2 = fmaf(-2.f, __uint_as_float(v[i]), p2 + q2);
                bool near = !(d2 > 16.f * E);
                float t = 0.f, u = 0.f;
                if (!near) {
                    t = sqrt_approx(d2);
                    const float r = fabsf(fmaf(t, t, -d2));               // |t^2 - d~^2|, one rounding
                    const float inv = rcp_approx(t);
                    const float e = fabsf(fmaf(-t, inv, 1.f));            // 1 - t inv
                    const float ih = __fmul_ru(inv, __fadd_ru(1.f, __fadd_ru(2.f * e, 2.384185791015625e-7f)));
                    const float e1 = __fmul_ru(__fmul_ru(r, 1.0000002f), ih);   // >= |t - sqrt(d~^2)|
                    u = __fadd_ru(e1, __fmul_ru(__fmul_ru(E, ih), 0.5085f));
                    // (written so that a NaN anywhere counts as near)
                    near = !(e1 <= 1.220703125e-4f * t) || !(u <= 2.44140625e-4f * sn);
                }
                if (near && prow >= 0) {
                    redo |= 1u << i;
                } else {
                    if (!near) umax = fmaxf(umax, u);
                    const float val = near ? sqrtf(fmaxf(d2, 0.f)) : t;   // (near with no pivot: an empty node)
                    a.out[q * a.P + p] = val;
                    tv[i] = val;
                }
            }
            if (a.outT && pv) {   // (entries recomputed below are rewritten there)
                float *dst = a.outT + p * a.nq + q0 + c0;
                const int64_t nv = a.nq - (q0 + c0) < 32 ? a.nq - (q0 + c0) : 32;
                if (nv == 32 && ((reinterpret_cast<uintptr_t>(dst) & 15) == 0)) {
#pragma unroll
                    for (int i = 0; i < 32; i += 4)
                        *reinterpret_cast<float4 *>(dst + i) = make_float4(tv[i], tv[i + 1], tv[i + 2], tv[i + 3]);
                } else {
#pragma unroll
                    for (int i = 0; i < 32; ++i)
                        if (i < nv) dst[i] = tv[i];
                }
            }
            while (redo) {   // near the pivot: the sum of squared differences in FP32
                const int i = __ffs(redo) - 1;
                redo &= redo - 1;
                const int64_t j = q0 + c0 + i;
                const int64_t q = a.perm ? (int64_t)a.perm[j] : j;
                const float *xr = a.X + (int64_t)prow * a.dim, *qr = a.Q + q * a.dim;
                float sum = 0.f;
                for (int k = 0; k < a.dim; ++k) {
                    const float d = qr[k] - xr[k];
                    sum = fmaf(d, d, sum);
                }
                a.out[q * a.P + p] = sqrtf(sum);
                if (a.outT) a.outT[p * a.nq + j] = sqrtf(sum);
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) umax = fmaxf(umax, __shfl_xor_sync(0xffffffffu, umax, o));
    if (lane == 0 && umax > 0.f) atomicMax(a.slack, __float_as_uint(umax));
    tc::tc_fence_before();
    __syncthreads();
    if (tid == 0 && !ok) {   // let an issued copy or MMA land before TMEM and shared memory go
        tc::mbar_wait(&bars[0], 0);
        tc::mbar_wait(&bars[1], 0);
    }
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}

// (at least 80 KB: at most two CTAs per SM, as many as TMEM holds)
size_t dense_tc_smem(int dim_p) {
    const size_t b = 1024 + 2 * (size_t)(dim_p / 64) * kDenseQ * 128 + 64;
    return b < 81920 ? 81920 : b;
}

}  // namespace

bool tc_dense_supported(const Tree &t, const TcCache &c) {
    return c.ready && c.dim_p > 0 && c.dim_p <= 256 && t.h >= 1;
}

void tc_prepare_pivots(const Tree &t, TcCache &c, cudaStream_t st) {
    if (c.piv_ready) return;
    const int64_t nodes = t.lvl_off[t.h];   // every pivot level's nodes
    c.Ph.alloc((size_t)(nodes > 0 ? nodes : 1) * c.dim_p * 2, st);
    c.Pl.alloc((size_t)(nodes > 0 ? nodes : 1) * c.dim_p * 2, st);
    c.pn2.alloc(nodes > 0 ? nodes : 1, st);
    if (nodes > 0)
        k_split_rows<<<nblk(nodes * 32), 256, 0, st>>>(t.X.get(), t.dim, c.dim_p, nodes, (__nv_bfloat16 *)c.Ph.get(),
                                                       (__nv_bfloat16 *)c.Pl.get(), c.pn2.get(), t.npiv.get());
    check_launch("split pivots");
    GTS_CUDA(cudaStreamSynchronize(st));
    c.Ph.persist();
    c.Pl.persist();
    c.pn2.persist();
    c.piv_ready = true;
}

float tc_dense_dist(const Tree &t, const TcCache &c, int level, const __nv_bfloat16 *Qh, const __nv_bfloat16 *Ql,
                    const float *qn2, const float *Q, int64_t nq, float *out, cudaStream_t st, const int32_t *perm,
                    float *outT) {
    const int64_t base = t.lvl_off[level], P = t.lvl_off[level + 1] - base;
    if (P == 0 || nq == 0) return 0.f;
    const size_t smem = dense_tc_smem(c.dim_p);
    GTS_CUDA(cudaFuncSetAttribute(k_dense_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const CUtensorMap mh = make_panel_map(Qh, nq, c.dim_p, kDenseQ);
    const CUtensorMap ml = make_panel_map(Ql, nq, c.dim_p, kDenseQ);
    DBuf<unsigned> slack(1, st);
    DBuf<int> status(1, st);
    DBuf<float> pnu(P, st), qnu(nq, st);
    k_norms_up<<<nblk(P), 256, 0, st>>>(c.pn2.get() + base, P, pnu.get());
    k_norms_up<<<nblk(nq), 256, 0, st>>>(qn2, nq, qnu.get());
    GTS_CUDA(cudaMemsetAsync(slack.get(), 0, 4, st));
    GTS_CUDA(cudaMemsetAsync(status.get(), 0, 4, st));
    DenseTcArgs a;
    a.Ph = reinterpret_cast<const __nv_bfloat16 *>(c.Ph.get()) + base * c.dim_p;
    a.Pl = reinterpret_cast<const __nv_bfloat16 *>(c.Pl.get()) + base * c.dim_p;
    a.pn2 = c.pn2.get() + base;
    a.pnu = pnu.get();
    a.qn2 = qn2;
    a.qnu = qnu.get();
    a.piv = t.npiv.get() + base;
    a.X = t.X.get();
    a.Q = Q;
    a.dim = t.dim;
    a.dim_p = c.dim_p;
    a.P = P;
    a.nq = nq;
    tc_bound_coeffs(c.dim_p, a.cE1, a.cE2);
    a.out = out;
    a.perm = perm;
    a.outT = outT;
    a.slack = slack.get();
    a.status = status.get();
    const dim3 grid((unsigned)((P + kRows - 1) / kRows), (unsigned)((nq + kDenseQ - 1) / kDenseQ));
    k_dense_tc<<<grid, 256, smem, st>>>(mh, ml, a);
    check_launch("dense pivot distances (tensor cores)");
    unsigned hs = 0;
    int hst = 0;
    GTS_CUDA(cudaMemcpyAsync(&hs, slack.get(), 4, cudaMemcpyDeviceToHost, st));
    GTS_CUDA(cudaMemcpyAsync(&hst, status.get(), 4, cudaMemcpyDeviceToHost, st));
    GTS_CUDA(cudaStreamSynchronize(st));
    GTS_REQUIRE(hst == 0, GTS_ETIMEOUT, "dense pivot distances: a bounded mbarrier wait ran out");
    float f;
    std::memcpy(&f, &hs, 4);
    return f;
}

// ---------------------------------------------------------------- self-test

namespace {

constexpr int kSelfN = 256;   // self-test tile: N up to 256 accumulator columns, then A (a_tmem) in TMEM

// D = A B^T for one 128 x N x K tile, A from shared memory (loaded by TMA) or,
// with a_tmem, from TMEM (written by the four warps, thread = row, as the
// tile kernel writes its node blocks).
__global__ void __launch_bounds__(128, 1)
    k_selftest_tc(const __grid_constant__ CUtensorMap amap, const __nv_bfloat16 *__restrict__ A,
                  const __nv_bfloat16 *__restrict__ B, int N, int K, int a_tmem, float *__restrict__ D, int *status) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int panels = K / 64;
    uint8_t *sA = smem;
    uint8_t *sB = sA + panels * kRows * 128;
    uint64_t *bars = (uint64_t *)(sB + panels * kSelfN * 128);
    uint32_t *tslot = (uint32_t *)(bars + 2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) tc::tmem_alloc(tslot, 2 * kSelfN);
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
    const uint32_t ta = tmem + kSelfN;   // A in TMEM: K / 2 columns
    if (a_tmem) {
        // thread = row = TMEM lane; 16 columns (32 coordinates) per store
        for (int c = 0; c < K / 2; c += 16) {
            uint32_t v[16];
            const uint4 *src = reinterpret_cast<const uint4 *>(A + (int64_t)tid * K + 2 * c);
            for (int j = 0; j < 4; ++j) {
                const uint4 x = src[j];
                v[4 * j] = x.x;
                v[4 * j + 1] = x.y;
                v[4 * j + 2] = x.z;
                v[4 * j + 3] = x.w;
            }
            tc::tmem_st16(ta + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
        }
        tc::tmem_st_wait();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (tid == 0) {
        if (!tc::mbar_wait(&bars[0], 0)) {
            atomicExch(status, 1);
        } else {
            const uint32_t idesc = tc::idesc_bf16_f32(kRows, kSelfN);
            for (int s = 0; s < K / 16; ++s) {
                const int p = s >> 2, w = s & 3;
                const uint64_t bd = tc::sdesc_k_sw128(tc::smem_u32(sB) + p * kSelfN * 128 + w * 32);
                if (a_tmem)
                    tc::mma_bf16_ts(tmem, ta + 8 * s, bd, idesc, s > 0 ? 1u : 0u);
                else
                    tc::mma_bf16(tmem, tc::sdesc_k_sw128(tc::smem_u32(sA) + p * kRows * 128 + w * 32), bd, idesc,
                                 s > 0 ? 1u : 0u);
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
    if (warp == 0) tc::tmem_dealloc(tmem, 2 * kSelfN);
}

// Bounded-wait check: thread 0 waits on an mbarrier of arrival count 1 that
// thread 32 arrives on only if `post` is set.  Without the arrival the wait
// gives up after `limit` polls and the kernel records status 1 and returns,
// as every waiting kernel of this library does when a wait runs out.
__global__ void k_selftest_wait(int post, uint32_t limit, int *status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        tc::mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 32 && post) tc::mbar_arrive(&bar);
    if (threadIdx.x == 0) *status = tc::mbar_wait_limit(&bar, 0, limit) ? 0 : 1;
}

__global__ void k_f32_to_bf16(const float *a, int64_t n, __nv_bfloat16 *b) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = __float2bfloat16_rn(a[i]);
}

}  // namespace

void wait_selftest(int post, uint32_t limit) {
    GTS_REQUIRE(limit >= 1 && limit <= tc::kSpinLimit, GTS_EINVAL, "spin limit must be in 1 .. 2^26");
    cudaStream_t st = nullptr;
    DBuf<int> status(1, st);
    GTS_CUDA(cudaMemsetAsync(status.get(), 0xff, 4, st));
    k_selftest_wait<<<1, 64, 0, st>>>(post ? 1 : 0, limit, status.get());
    check_launch("bounded-wait self-test");
    int hs = -1;
    GTS_CUDA(cudaMemcpyAsync(&hs, status.get(), 4, cudaMemcpyDeviceToHost, st));
    GTS_CUDA(cudaStreamSynchronize(st));
    GTS_REQUIRE(hs != -1, GTS_ECUDA, "bounded-wait self-test: status not written");
    GTS_REQUIRE(hs == 0, GTS_ETIMEOUT, "bounded-wait self-test: the wait ran out after its poll limit");
}

void tc_selftest(const float *hA, const float *hB, int N, int K, int a_tmem, float *hD) {
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
    CUtensorMap m = make_row_map(bA.get(), kRows, K, kRows);
    const size_t smem = 1024 + (size_t)(K / 64) * (kRows + kSelfN) * 128 + 64;
    GTS_CUDA(cudaFuncSetAttribute(k_selftest_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_selftest_tc<<<1, 128, smem, st>>>(m, bA.get(), bB.get(), N, K, a_tmem ? 1 : 0, D.get(), status.get());
    check_launch("tensor-core self-test");
    int hs = 0;
    GTS_CUDA(cudaMemcpyAsync(&hs, status.get(), 4, cudaMemcpyDeviceToHost, st));
    GTS_CUDA(cudaMemcpyAsync(hD, D.get(), (size_t)kRows * N * 4, cudaMemcpyDeviceToHost, st));
    GTS_CUDA(cudaStreamSynchronize(st));
    GTS_REQUIRE(hs == 0, GTS_ETIMEOUT, "tensor-core self-test: a bounded wait ran out");
}

}  // namespace gts
