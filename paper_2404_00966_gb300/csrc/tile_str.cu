// Edit-distance filtering tiles: the 3-gram count bound over (node rows x
// queries) blocks.
//
// For strings the lower bounds of Lemma 1 / 2 prune little when the distances
// concentrate (random-like sequences), and most (query, row) pairs of the
// surviving leaves reach verification.  Before the bit-parallel DP, each pair
// is tested against the 3-gram count bound: the L1 distance between the
// strings' hashed 3-gram bucket counts is at most 6 times the edit distance
// (a substitution changes at most 3 of a string's 3-grams, an insertion or a
// deletion at most 2 old and 3 new ones; summing counts into buckets and
// capping them at 255 can only lower the L1 distance), so L1 > 6 t proves
// d > t.  The surviving (query, last-level node) entries are regrouped by
// node; one CTA takes a block of up to 128 node rows (each thread holds one
// row's 64-byte bucket vector in registers) and the node's queries in chunks
// of 32 or 64 (their vectors in shared memory); a pair is kept if the row's leaf
// survived for the query, the row is visible
// at the query's sequence number and the bound does not exclude it.  The
// kept pairs go on to the exact DP.
#include "gts_impl.cuh"
#include "tile_str.cuh"

namespace gts {

namespace {

constexpr int kRowsS = 128;     // rows of one node block (the regrouping's block size)
constexpr int kThreadsS = 256;  // thread = (row tid % 128, query half tid / 128)
constexpr int kWords = 16;      // 64 one-byte buckets as 16 words

struct StrArgs {
    int F;
    const int32_t *npos, *nsize;
    int64_t lvl_last;
    const int64_t *row_del;
    int any_deleted;
    const uint8_t *qg;          // rows' bucket counts [n, 64]
    const uint8_t *qgq;         // queries' bucket counts [nq, 64]
    const TileRec *grec;
    const int4 *items;
    int64_t i1;
    int *work_counter;
    int32_t *out_q, *out_row;
    int64_t cap;
    unsigned long long *out_count;
};

// NQS: queries per chunk (32 or 64; a tuning parameter), NQS / 2 per thread
template <int NQS>
__global__ void __launch_bounds__(kThreadsS) k_tile_qgram(StrArgs a) {
    constexpr int kNQS = NQS;
    constexpr int kQPTS = NQS / 2;
    __shared__ __align__(16) uint32_t sQ[kNQS][kWords + 1];
    __shared__ uint64_t sMask[kNQS];
    __shared__ int64_t sSeq[kNQS];
    __shared__ float sLim[kNQS];
    __shared__ int32_t sQid[kNQS];
    __shared__ int s_item;
    const int tid = threadIdx.x, lane = tid & 31;
    const int r = tid % kRowsS, half = tid / kRowsS;
    for (;;) {
        if (tid == 0) s_item = atomicAdd(a.work_counter, 1);
        __syncthreads();
        const int64_t item = s_item;
        if (item >= a.i1) break;
        const int4 it = a.items[item];
        const int64_t g = a.lvl_last + it.x;
        const int first = it.y, total = it.z;
        const int rb = it.w * kRowsS;
        const int32_t pos = a.npos[g], size = a.nsize[g];
        const int nrow = min(kRowsS, size - rb);
        const int64_t row = (int64_t)pos + rb + r;
        const bool valid = r < nrow;
        // this thread's row: bucket counts, leaf bit, delete mark
        const int32_t avg = size / a.F;
        int32_t jl = avg > 0 ? (rb + r) / avg : a.F - 1;
        if (jl > a.F - 1) jl = a.F - 1;
        const uint64_t rowbit = valid ? (1ull << jl) : 0ull;
        const int64_t rdel = (valid && a.any_deleted) ? a.row_del[row] : kNever;
        uint32_t rw[kWords];
        if (valid) {
            const uint4 *src = reinterpret_cast<const uint4 *>(a.qg + row * 64);
#pragma unroll
            for (int v = 0; v < kWords / 4; ++v) {
                const uint4 x = src[v];
                rw[4 * v] = x.x;
                rw[4 * v + 1] = x.y;
                rw[4 * v + 2] = x.z;
                rw[4 * v + 3] = x.w;
            }
        } else {
#pragma unroll
            for (int w = 0; w < kWords; ++w) rw[w] = 0;
        }
        for (int c0 = 0; c0 < total; c0 += kNQS) {
            const int cnt = min(kNQS, total - c0);
            __syncthreads();   // the previous chunk's shared data is no longer read
            for (int j = tid; j < cnt; j += kThreadsS) {
                const TileRec rc = a.grec[first + c0 + j];
                sMask[j] = rc.mask;
                sSeq[j] = rc.seq;
                sLim[j] = 6.f * rc.thr;   // keep iff L1 <= 6 t
                sQid[j] = rc.q;
            }
            for (int t = tid; t < cnt * kWords; t += kThreadsS) {
                const int j = t / kWords, w = t - j * kWords;
                sQ[j][w] = reinterpret_cast<const uint32_t *>(a.qgq + (int64_t)a.grec[first + c0 + j].q * 64)[w];
            }
            __syncthreads();
            uint32_t pass = 0;
#pragma unroll 1
            for (int jj = 0; jj < kQPTS; ++jj) {
                const int j = half * kQPTS + jj;
                if (j >= cnt) break;
                if (!(sMask[j] & rowbit) || rdel <= sSeq[j]) continue;
                uint32_t l1 = 0;
#pragma unroll
                for (int w = 0; w < kWords; ++w) l1 = __vsadu4(rw[w], sQ[j][w]) + l1;
                if ((float)l1 <= sLim[j]) pass |= 1u << jj;
            }
            const int np = __popc(pass);
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
                unsigned long long o = base + (unsigned long long)(incl - np);
                while (pass) {
                    const int jj = __ffs(pass) - 1;
                    pass &= pass - 1;
                    if ((int64_t)o < a.cap) {
                        a.out_q[o] = sQid[half * kQPTS + jj];
                        a.out_row[o] = (int32_t)row;
                    }
                    ++o;
                }
            }
        }
        __syncthreads();
    }
}

}  // namespace

int64_t qgram_run(const Tree &t, const StrQuery &sq, const TcRegroup &rg, DBuf<int32_t> &out_q,
                  DBuf<int32_t> &out_row, int64_t cap_hint, int *launches, cudaStream_t st) {
    *launches = 0;
    if (rg.n_items == 0) return 0;
    int dev = 0, sms = 0;
    GTS_CUDA(cudaGetDevice(&dev));
    GTS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int per_sm = 0;
    if (sq.queries == 32)
        GTS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tile_qgram<32>, kThreadsS, 0));
    else
        GTS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tile_qgram<64>, kThreadsS, 0));
    if (per_sm < 1) per_sm = 1;
    const int64_t grid = std::min<int64_t>(rg.n_items, (int64_t)sms * per_sm);
    DBuf<int> counter(1, st);
    DBuf<unsigned long long> count(1, st);
    int64_t cap = cap_hint > 0 ? cap_hint : 1 << 20;
    for (int attempt = 0; attempt < 2; ++attempt) {
        out_q.alloc(cap, st);
        out_row.alloc(cap, st);
        GTS_CUDA(cudaMemsetAsync(counter.get(), 0, 4, st));
        GTS_CUDA(cudaMemsetAsync(count.get(), 0, 8, st));
        StrArgs a;
        a.F = t.F;
        a.npos = t.npos.get();
        a.nsize = t.nsize.get();
        a.lvl_last = t.lvl_off[t.h - 1];
        a.row_del = t.row_del.get();
        a.any_deleted = sq.any_deleted;
        a.qg = sq.qg;
        a.qgq = sq.qgq;
        a.grec = rg.grec.get();
        a.items = rg.items.get();
        a.i1 = rg.n_items;
        a.work_counter = counter.get();
        a.out_q = out_q.get();
        a.out_row = out_row.get();
        a.cap = cap;
        a.out_count = count.get();
        if (sq.queries == 32)
            k_tile_qgram<32><<<(unsigned)grid, kThreadsS, 0, st>>>(a);
        else
            k_tile_qgram<64><<<(unsigned)grid, kThreadsS, 0, st>>>(a);
        ++*launches;
        check_launch("3-gram tile");
        unsigned long long hcount = 0;
        GTS_CUDA(cudaMemcpyAsync(&hcount, count.get(), 8, cudaMemcpyDeviceToHost, st));
        GTS_CUDA(cudaStreamSynchronize(st));
        if ((int64_t)hcount <= cap) return (int64_t)hcount;
        cap = (int64_t)hcount;   // rerun with room for every pair
    }
    GTS_REQUIRE(false, GTS_ECUDA, "3-gram tile: output count changed between identical runs");
    return 0;
}

}  // namespace gts
