// List-table pruning scan (the table list of Section 4.2; Lemma 1 for range
// queries, Lemma 2 for kNN, Section 5), node-major and bandwidth-bound.
//
// The last-level (query, node) entries are regrouped by node (tc_regroup:
// records of 32 bytes -- query, threshold, sequence number, leaf mask -- and
// the entry's path distances d(q, p_l), l < h).  A work item is a block of up
// to 128 consecutive rows of one node together with all records of that node.
// Each warp takes items on its own from a global counter (work stealing:
// nodes carry very different numbers of queries; no block-wide barrier, since
// a typical item holds only a few records).  Per item:
//   * the records and their pivot-distance tiles (h distances each) are staged
//     16 at a time by the TMA engine (cp.async.bulk into the warp's shared
//     memory, completion on the warp's mbarrier), issued first so that they
//     land while the lanes load the block;
//   * the block's h table columns are read once with 16-byte vector loads from
//     a 16-byte aligned start, with its delete marks, into shared memory;
//   * the warp tests each record against the block's rows, a row per lane in
//     32-row strips: the leaf bit of the row's leaf, visibility at the query's
//     sequence number and the table lower bound
//         lb = max_l |D_l(row) - d(q, p_l)|  <=  t + eps_l
//     (t = radius or tau_q; eps_l = epsc (D_l + d(q, p_l) + t), the FP32 slack
//     the whole search uses, 0 for exact integer distances).  Survivors are
//     compacted by ballot and a warp prefix count and appended with one atomic
//     per (record, output) on one of 32 striped counters (each stripe owns a
//     slice of the output), so that the atomics of different warps do not
//     queue on one address; the slices are packed together afterwards.
// Every row is read from HBM once per item however many queries test it, so
// the pass streams the table at the memory's rate when the batch touches more
// rows than fit in L2.
//
// Range queries on vectors of at most 16 dimensions take a fused form: the
// block's rows are staged beside the table, and every pair that passes the
// table bound gets its FP32 distance (the query row in registers) and is
// decided against the radius with the FP32 error band of the whole search,
// |d32 - d| <= 2 (D + 8) 2^-24 d: clearly inside -> the answer (query, object
// id, distance); clearly outside -> dropped; inside the band -> listed for
// the FP64 recheck in the reference operation order.  A separate verification
// pass over the candidates would gather every candidate's row again; at low
// dimension that gather costs more than the arithmetic.
#include "metric.cuh"
#include "scan.cuh"
#include "tc.cuh"

namespace gts {

namespace {

constexpr int kRowsB = 128;                          // rows per item (the regrouping's blocks)
constexpr int kWarpsPerCta = 4;
constexpr int kThreads = 32 * kWarpsPerCta;
constexpr int kRecW = 16;                            // records staged per warp at a time
constexpr int kTPad = kRowsB + 4;                    // a column window with up to 3 leading floats
constexpr int kV4 = (3 + kRowsB + 3) / 4;            // 16-byte loads per column window
constexpr int kStripes = 32;                         // striped output counters / slices
constexpr unsigned kFull = 0xffffffffu;

struct ScanArgs {
    int F, h, hp;
    int64_t n;
    const float *table;        // [h, n]
    const int64_t *row_del;    // [n]
    const int32_t *npos, *nsize;
    int64_t lvl_last;          // first node of the last pivot level
    const TileRec *grec;       // records grouped by node
    const float *gpath;        // their path distances [*, hp]
    const int4 *items;         // (node, first record, record count, row block)
    int64_t n_items;
    int *work;
    float epsc;
    int any_deleted;
    // outputs, stripe s owning [s * cap, (s + 1) * cap) of each array
    int32_t *out_q, *out_row;  // candidates, or band pairs (fused)
    int64_t cap;
    uint64_t *out_key;         // fused: accepted answers
    float *out_dist;
    int64_t cap_acc;
    unsigned long long *counts;   // [s] pairs of stripe s, [kStripes + s] accepted of stripe s,
                                  // [2 kStripes] rows staged, [+1] records tested, [+2] pairs passing the bound
    int *status;
    // fused range decisions (dim <= kScanMaxDim)
    int dim, l2;
    const float *X, *Q;
    const int64_t *row_id;
    float rel;
    int warp_bytes;            // shared memory per warp
    int claim;                 // items a warp takes per atomic on the work counter
};

// Per-warp shared-memory layout (bytes), from h, hp and dim.
struct WarpLayout {
    int bar, rec, path, del, T, X, qrow, toff, leaf, bytes;
};

__host__ __device__ inline WarpLayout warp_layout(int h, int hp, int dim, bool fused) {
    WarpLayout L;
    int o = 0;
    L.bar = o;
    o += 16;
    L.rec = o;
    o += kRecW * (int)sizeof(TileRec);
    L.path = o;
    o += kRecW * hp * 4;
    L.del = o;
    o += kRowsB * 8;
    L.T = o;
    o += h * kTPad * 4;
    L.X = o;
    o += fused ? ((kRowsB * (dim | 1) * 4 + 15) & ~15) : 0;
    L.qrow = o;                 // fused: the current record's query row
    o += fused ? kScanMaxDim * 4 : 0;
    L.toff = o;                 // each column's window offset in T
    o += kMaxHeight * 4;
    L.leaf = o;
    o += kRowsB;
    L.bytes = (o + 15) & ~15;
    return L;
}

__device__ __forceinline__ void issue_records(const ScanArgs &a, TileRec *rec, float *path, uint64_t *bar,
                                              int64_t rec0, int k) {
    const uint32_t rb = (uint32_t)k * (uint32_t)sizeof(TileRec);
    const uint32_t pb = (uint32_t)(k * a.hp) * 4u;
    tc::fence_proxy_async_smem();   // the warp's earlier generic reads of the buffer come first
    tc::mbar_expect_tx(bar, rb + pb);
    tc::bulk_load(rec, a.grec + rec0, rb, bar);
    tc::bulk_load(path, a.gpath + rec0 * a.hp, pb, bar);
}

// append the lanes flagged in the strips' ballots (bits[s], a 32-row strip
// each) to a striped output: one atomic for the warp
template <class Write>
__device__ __forceinline__ void emit(const uint32_t *bits, int nstrips, int total, unsigned long long *counter,
                                     int lane, Write write) {
    if (!total) return;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(counter, (unsigned long long)total);
    base = __shfl_sync(kFull, base, 0);
    int before = 0;
#pragma unroll
    for (int s = 0; s < kRowsB / 32; ++s) {
        if (s < nstrips) {
            if ((bits[s] >> lane) & 1u) write(s, base + before + __popc(bits[s] & ((1u << lane) - 1u)));
            before += __popc(bits[s]);
        }
    }
}

template <bool FUSED>
__global__ void __launch_bounds__(kThreads, FUSED ? 6 : 8) k_scan_warps(ScanArgs a) {
    extern __shared__ __align__(16) uint8_t dyn[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const WarpLayout L = warp_layout(a.h, a.hp, a.dim, FUSED);
    uint8_t *wb = dyn + warp * a.warp_bytes;
    uint64_t *bar = reinterpret_cast<uint64_t *>(wb + L.bar);
    TileRec *rec = reinterpret_cast<TileRec *>(wb + L.rec);
    float *path = reinterpret_cast<float *>(wb + L.path);
    int64_t *del = reinterpret_cast<int64_t *>(wb + L.del);
    float *T = reinterpret_cast<float *>(wb + L.T);
    float *Xs = reinterpret_cast<float *>(wb + L.X);
    float *qrow = reinterpret_cast<float *>(wb + L.qrow);
    int *toffs = reinterpret_cast<int *>(wb + L.toff);
    uint8_t *leaf = wb + L.leaf;
    const int xs = a.dim | 1;
    if (lane == 0) {
        tc::mbar_init(bar, 1);
        tc::mbar_fence_init();
    }
    __syncwarp();
    uint32_t phase = 0;
    const int stripe = (int)((blockIdx.x * (unsigned)kWarpsPerCta + warp) % kStripes);
    unsigned long long *cnt_pairs = a.counts + stripe;
    unsigned long long *cnt_acc = a.counts + kStripes + stripe;
    int32_t *oq = a.out_q + (int64_t)stripe * a.cap;
    int32_t *orow = a.out_row + (int64_t)stripe * a.cap;
    uint64_t *okey = FUSED ? a.out_key + (int64_t)stripe * a.cap_acc : nullptr;
    float *odist = FUSED ? a.out_dist + (int64_t)stripe * a.cap_acc : nullptr;
    unsigned long long staged = 0, tested = 0, passed = 0;
    const int64_t hn = (int64_t)a.h * a.n;
    bool ok = true;
    // items are claimed a run of a.claim at a time: one atomic on the shared
    // counter per run instead of per item (the counter's address serialises
    // its atomics)
    int run_next = 0, run_end = 0;
    for (;;) {
        if (run_next == run_end) {
            int it = 0;
            if (lane == 0) it = atomicAdd(a.work, a.claim);
            it = __shfl_sync(kFull, it, 0);
            run_next = it;
            run_end = (int)min((int64_t)it + a.claim, a.n_items);
        }
        if (run_next >= a.n_items) break;
        const int it = run_next++;
        const int4 w = a.items[it];
        const int64_t node = a.lvl_last + w.x;
        const int64_t first = w.y;
        const int cnt = w.z, blk = w.w;
        const int32_t pos = a.npos[node], size = a.nsize[node];
        const int32_t avg = size / a.F;
        const int r0 = blk * kRowsB;
        const int nr = min(kRowsB, size - r0);
        const int64_t g0 = (int64_t)pos + r0;
        // the first records by the TMA engine, while the lanes load the block
        if (lane == 0) issue_records(a, rec, path, bar, first, min(kRecW, cnt));
        for (int idx = lane; idx < a.h * kV4; idx += 32) {
            const int l = idx / kV4, v = idx - l * kV4;
            const int64_t c0 = (int64_t)l * a.n + g0;
            const int64_t al = c0 & ~(int64_t)3;
            if (v < ((int)(c0 - al) + nr + 3) >> 2) {
                const int64_t e = al + 4 * v;
                float4 x;
                if (e + 3 < hn) {
                    x = __ldg(reinterpret_cast<const float4 *>(a.table + e));
                } else {
                    x.x = e < hn ? a.table[e] : 0.f;
                    x.y = e + 1 < hn ? a.table[e + 1] : 0.f;
                    x.z = e + 2 < hn ? a.table[e + 2] : 0.f;
                    x.w = 0.f;
                }
                *reinterpret_cast<float4 *>(&T[l * kTPad + 4 * v]) = x;
            }
        }
        for (int rr = lane; rr < nr; rr += 32) {
            if (a.any_deleted) del[rr] = a.row_del[g0 + rr];
            const int j = avg > 0 ? (r0 + rr) / avg : a.F - 1;
            leaf[rr] = (uint8_t)(j > a.F - 1 ? a.F - 1 : j);
        }
        if (FUSED)   // the block's rows: nr x dim consecutive floats
            for (int e = lane; e < nr * a.dim; e += 32) {
                const int rr = e / a.dim, i = e - rr * a.dim;
                Xs[rr * xs + i] = a.X[g0 * a.dim + e];
            }
        if (lane < a.h) toffs[lane] = (int)(((int64_t)lane * a.n + g0) & 3) + lane * kTPad;
        __syncwarp();
        staged += (unsigned long long)nr;
        const int nstrips = (nr + 31) >> 5;
        for (int c0 = 0; c0 < cnt; c0 += kRecW) {
            const int k = min(kRecW, cnt - c0);
            ok = __all_sync(kFull, tc::mbar_wait(bar, phase & 1u));
            if (!ok) break;
            ++phase;
            for (int i = 0; i < k; ++i) {
                const TileRec rc = rec[i];
                const float thr = rc.thr;
                const float *dq = path + i * a.hp;   // this record's pivot-distance tile (shared memory)
                if (FUSED) {
                    __syncwarp();                    // the previous record's query row is read
                    if (lane < a.dim) qrow[lane] = a.Q[(int64_t)rc.q * a.dim + lane];
                    __syncwarp();
                }
                uint32_t pb[kRowsB / 32], ab[kRowsB / 32];
                float dv[FUSED ? kRowsB / 32 : 1];
                int tot = 0, tot_acc = 0;
#pragma unroll
                for (int s = 0; s < kRowsB / 32; ++s) {
                    pb[s] = ab[s] = 0u;
                    if (s >= nstrips) continue;
                    const int rr = s * 32 + lane;
                    bool pass = rr < nr && ((rc.mask >> leaf[rr]) & 1ull) && (!a.any_deleted || del[rr] > rc.seq);
                    if (pass) {
                        // loops bounded by the tree's h and the data's dim:
                        // no predicated-off iterations
#pragma unroll 2
                        for (int l = 0; l < a.h; ++l) {
                            const float Tv = T[toffs[l] + rr];
                            const float dl = dq[l];
                            const float eps = a.epsc * (Tv + dl + thr);
                            if (fabsf(Tv - dl) > thr + eps) pass = false;
                        }
                    }
                    bool take = false;
                    if (FUSED) {
                        passed += __popc(__ballot_sync(kFull, pass));
                        dv[s] = 0.f;
                        if (pass) {
                            // the pair's FP32 distance and the band decision (the
                            // same bound as the candidate verification)
                            float sum = 0.f;
                            const float *xr = Xs + rr * xs;
                            if (a.l2) {
#pragma unroll 2
                                for (int c2 = 0; c2 < a.dim; ++c2) {
                                    const float t = qrow[c2] - xr[c2];
                                    sum = fmaf(t, t, sum);
                                }
                            } else {
#pragma unroll 2
                                for (int c2 = 0; c2 < a.dim; ++c2) sum += fabsf(qrow[c2] - xr[c2]);
                            }
                            const float d32 = a.l2 ? sqrtf(sum) : sum;
                            const float hi = d32 * (1.f + 2.f * a.rel) + kAbsFloor;
                            const float lo = d32 * (1.f - 2.f * a.rel) - kAbsFloor;
                            if (hi < thr * (1.f - 1e-9f)) {
                                take = true;
                                pass = false;
                            } else if (lo > thr * (1.f + 1e-9f)) {
                                pass = false;
                            }
                            dv[s] = d32;
                        }
                    }
                    pb[s] = __ballot_sync(kFull, pass);
                    ab[s] = __ballot_sync(kFull, take);
                    tot += __popc(pb[s]);
                    tot_acc += __popc(ab[s]);
                }
                tested += 1;
                const int32_t q = rc.q;
                emit(pb, nstrips, tot, cnt_pairs, lane, [&](int s, unsigned long long o) {
                    if ((int64_t)o < a.cap) {
                        oq[o] = q;
                        orow[o] = (int32_t)(g0 + s * 32 + lane);
                    }
                });
                if (FUSED)
                    emit(ab, nstrips, tot_acc, cnt_acc, lane, [&](int s, unsigned long long o) {
                        if ((int64_t)o < a.cap_acc) {
                            okey[o] = ((uint64_t)(uint32_t)q << 32) | (uint64_t)(uint32_t)a.row_id[g0 + s * 32 + lane];
                            odist[o] = dv[s];
                        }
                    });
            }
            __syncwarp();   // the buffer is read: the next chunk may land in it
            if (c0 + kRecW < cnt && lane == 0) issue_records(a, rec, path, bar, first + c0 + kRecW, min(kRecW, cnt - c0 - kRecW));
        }
        if (!ok) break;
    }
    if (!ok && lane == 0) {
        // a bounded wait ran out: record it, let the copy in flight land (again
        // bounded) and leave
        atomicExch(a.status, 1);
        tc::mbar_wait(bar, phase & 1u);
    }
    if (lane == 0) {
        if (staged) atomicAdd(&a.counts[2 * kStripes], staged);
        if (tested) atomicAdd(&a.counts[2 * kStripes + 1], tested);
        if (FUSED && passed) atomicAdd(&a.counts[2 * kStripes + 2], passed);
    }
}

// pack the stripes' slices [s * cap, s * cap + count_s) one after another
template <class T>
__global__ void k_pack_stripes(const T *__restrict__ src, const unsigned long long *__restrict__ counts, int64_t cap,
                               T *__restrict__ dst) {
    const int s = blockIdx.y;
    int64_t off = 0;
    for (int t = 0; t < s; ++t) off += min((int64_t)counts[t], cap);
    const int64_t c = min((int64_t)counts[s], cap);   // (the host relaunches until no slice overflows)
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < c; i += (int64_t)gridDim.x * blockDim.x)
        dst[off + i] = src[(int64_t)s * cap + i];
}

template <class T>
void pack(DBuf<T> &buf, const unsigned long long *dcounts, int64_t cap, int64_t total, cudaStream_t st) {
    DBuf<T> out(total > 0 ? total : 1, st);
    if (total > 0) {
        dim3 grid((unsigned)std::min<int64_t>((total / kStripes + 255) / 256 + 1, 64), kStripes);
        k_pack_stripes<T><<<grid, 256, 0, st>>>(buf.get(), dcounts, cap, out.get());
        check_launch("pack stripes");
    }
    buf = std::move(out);
}

}  // namespace

void scan_run(const Tree &t, const TcRegroup &rg, const ScanQuery &sq, ScanOut &out, int64_t cap_hint,
              ScanStats &stats, cudaStream_t st) {
    stats = ScanStats();
    out.n_pairs = out.n_accepted = 0;
    if (rg.n_items == 0) return;
    GTS_REQUIRE(t.h >= 1 && t.h <= kMaxHeight && t.F <= kMaxFanout, GTS_EINVAL, "tree shape out of range for the scan");
    GTS_REQUIRE(!rg.dmask && rg.grec.get() && rg.gpath.get(), GTS_EINVAL, "the scan needs regrouped records");
    GTS_REQUIRE(!sq.fused_range || (t.dim >= 1 && t.dim <= kScanMaxDim && sq.Q), GTS_EINVAL,
                "fused range scan needs vectors of at most 16 dimensions");
    const bool fused = sq.fused_range;
    const int hp = (t.h + 3) & ~3;
    const WarpLayout L = warp_layout(t.h, hp, t.dim, fused);
    const int smem = L.bytes * kWarpsPerCta;
    int dev = 0, sms = 0, per_sm = 0;
    GTS_CUDA(cudaGetDevice(&dev));
    GTS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (fused) {
        GTS_CUDA(cudaFuncSetAttribute(k_scan_warps<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        GTS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_scan_warps<true>, kThreads, smem));
    } else {
        GTS_CUDA(cudaFuncSetAttribute(k_scan_warps<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        GTS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_scan_warps<false>, kThreads, smem));
    }
    const int64_t warps_needed = (rg.n_items + 0);
    const int64_t resident = (int64_t)(sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((warps_needed + kWarpsPerCta - 1) / kWarpsPerCta, resident));
    const int nc = 2 * kStripes + 3;
    DBuf<unsigned long long> counts(nc, st);
    DBuf<int> work(1, st), status(1, st);
    // per-stripe slices; fused: most passing pairs are accepted answers, few fall in the band
    int64_t cap = std::max<int64_t>((fused ? cap_hint / 16 : cap_hint) / kStripes + 1, 1 << 12);
    int64_t cap_acc = fused ? std::max<int64_t>(cap_hint / kStripes + 1, 1 << 12) : 0;
    std::vector<unsigned long long> hc(nc, 0);
    // Work stealing spreads the items over the warps (and so over the
    // stripes) differently on every launch: a relaunch sized by one launch's
    // stripe counts can still overflow a slice, so the launch repeats, with
    // slices grown past the largest count seen, until no stripe overflows.
    bool fits = false;
    for (int attempt = 0; attempt < 8 && !fits; ++attempt) {
        out.q.alloc(cap * kStripes, st);
        out.row.alloc(cap * kStripes, st);
        out.key.alloc(fused ? cap_acc * kStripes : 1, st);
        out.dist.alloc(fused ? cap_acc * kStripes : 1, st);
        GTS_CUDA(cudaMemsetAsync(counts.get(), 0, nc * sizeof(unsigned long long), st));
        GTS_CUDA(cudaMemsetAsync(work.get(), 0, sizeof(int), st));
        GTS_CUDA(cudaMemsetAsync(status.get(), 0, sizeof(int), st));
        ScanArgs a;
        a.F = t.F;
        a.h = t.h;
        a.hp = hp;
        a.n = t.n;
        a.table = t.table.get();
        a.row_del = t.row_del.get();
        a.npos = t.npos.get();
        a.nsize = t.nsize.get();
        a.lvl_last = t.lvl_off[t.h - 1];
        a.grec = rg.grec.get();
        a.gpath = rg.gpath.get();
        a.items = rg.items.get();
        a.n_items = rg.n_items;
        a.work = work.get();
        a.epsc = sq.epsc;
        a.any_deleted = sq.any_deleted;
        a.out_q = out.q.get();
        a.out_row = out.row.get();
        a.cap = cap;
        a.out_key = out.key.get();
        a.out_dist = out.dist.get();
        a.cap_acc = cap_acc;
        a.counts = counts.get();
        a.status = status.get();
        a.dim = t.dim;
        a.l2 = t.metric == GTS_L2 ? 1 : 0;
        a.X = t.X.get();
        a.Q = sq.Q;
        a.row_id = t.row_id.get();
        a.rel = sq.rel;
        a.warp_bytes = L.bytes;
        // runs of consecutive items: about 16 runs per warp, 1 .. 16 items each
        a.claim = (int)std::max<int64_t>(1, std::min<int64_t>(16, rg.n_items / ((int64_t)grid * kWarpsPerCta * 16)));
        if (fused)
            k_scan_warps<true><<<grid, kThreads, smem, st>>>(a);
        else
            k_scan_warps<false><<<grid, kThreads, smem, st>>>(a);
        check_launch("table scan");
        stats.launches += 1;
        int hs = 0;
        GTS_CUDA(cudaMemcpyAsync(hc.data(), counts.get(), nc * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
        GTS_CUDA(cudaMemcpyAsync(&hs, status.get(), sizeof(int), cudaMemcpyDeviceToHost, st));
        GTS_CUDA(cudaStreamSynchronize(st));
        GTS_REQUIRE(hs == 0, GTS_ETIMEOUT, "table scan: a bounded wait for a staged record chunk ran out");
        int64_t mx = 0, mxa = 0;
        for (int s2 = 0; s2 < kStripes; ++s2) {
            mx = std::max<int64_t>(mx, (int64_t)hc[s2]);
            mxa = std::max<int64_t>(mxa, (int64_t)hc[kStripes + s2]);
        }
        fits = mx <= cap && mxa <= cap_acc;
        if (!fits) {
            cap = std::max(cap, mx + mx / 4 + 1024);
            cap_acc = fused ? std::max(cap_acc, mxa + mxa / 4 + 1024) : 0;
        }
    }
    GTS_REQUIRE(fits, GTS_ECUDA, "table scan: output slices kept overflowing");
    int64_t np = 0, na = 0;
    for (int s2 = 0; s2 < kStripes; ++s2) {
        np += (int64_t)hc[s2];
        na += (int64_t)hc[kStripes + s2];
    }
    pack(out.q, counts.get(), cap, np, st);
    pack(out.row, counts.get(), cap, np, st);
    if (fused) {
        pack(out.key, counts.get() + kStripes, cap_acc, na, st);
        pack(out.dist, counts.get() + kStripes, cap_acc, na, st);
    }
    out.n_pairs = np;
    out.n_accepted = na;
    stats.candidates = fused ? (int64_t)hc[2 * kStripes + 2] : np;
    stats.staged_rows = (int64_t)hc[2 * kStripes];
    stats.records = (int64_t)hc[2 * kStripes + 1];
}

}  // namespace gts
