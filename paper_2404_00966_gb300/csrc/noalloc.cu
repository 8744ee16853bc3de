// Exact kNN by brute-force scan with no device allocation.
//
// Some callers of this library cannot allocate device memory at query time:
// code that runs while a CUDA graph is being captured (an allocation there is
// an error or is baked into the graph), latency-critical serving threads that
// must not call into the allocator (cudaMalloc may synchronise the device and
// stall every stream), and host frameworks that own all device memory through
// their own pool and forbid any other allocator.  gts_knn_scan_noalloc serves
// them: it answers exact kNN over an object set the caller holds on the device
// by scanning every object, the same brute-force table scan that GTS uses for
// its cache list, and keeps its intermediate lists in a fixed array in device
// global memory that the library reserves once, when it is loaded.
//
// Scratch: a file-scope __device__ array of kScratchEntries (key, id) pairs
// (16 MiB).  Every GPU that loads the library holds it until the process exits.
// Every call uses the same array, so calls whose kernels overlap on the GPU
// (different streams, or different host threads) race on it; serialise them.
// Nothing in it has to start at zero: each call writes every entry it reads.
//
// Non-finite inputs: a distance that comes out NaN (a NaN coordinate in the
// object or the query) is ranked as +inf, so such objects sort after every
// finite one, by id, and never displace a real neighbour.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <unordered_map>

#include "gts_impl.cuh"
#include "metric.cuh"

namespace gts {
namespace {

constexpr int64_t kScratchEntries = 1 << 20;
constexpr int kScanMaxK = 32;

struct ScanPair {
    double key;
    int64_t id;
};

static __device__ __align__(256) ScanPair g_scan_scratch[kScratchEntries];

__device__ __forceinline__ bool pair_less(double ka, int64_t ia, double kb, int64_t ib) {
    return ka < kb || (ka == kb && ia < ib);
}

// One warp per (query, slice): every lane keeps its own ascending top-k of
// (FP64 key, id) over the objects it scans, then the warp merges the 32 lists
// by k rounds of argmin and writes k pairs to the scratch array (+inf padding
// when the slice holds fewer than k objects).
__global__ void k_scan_partial(const float *__restrict__ X, int64_t n, int dim, int l2, const float *__restrict__ Q,
                               int64_t nq, int k, int slices, ScanPair *__restrict__ scratch) {
    const int lane = threadIdx.x & 31;
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (w >= nq * slices) return;
    const int64_t q = w / slices;
    const int p = (int)(w - q * slices);
    const int64_t o0 = n * p / slices, o1 = n * (p + 1) / slices;
    const float *qv = Q + q * dim;
    double kk[kScanMaxK];
    int64_t ii[kScanMaxK];
    int len = 0;
    for (int64_t o = o0 + lane; o < o1; o += 32) {
        const float *xv = X + o * dim;
        double key = l2 ? l2sq_fp64_seq(qv, xv, dim) : l1_fp64_seq(qv, xv, dim);
        if (key != key) key = __longlong_as_double(0x7ff0000000000000ll);   // NaN ranks as +inf
        if (len == k && !pair_less(key, o, kk[k - 1], ii[k - 1])) continue;
        int pos = len < k ? len : k - 1;
        while (pos > 0 && pair_less(key, o, kk[pos - 1], ii[pos - 1])) {
            kk[pos] = kk[pos - 1];
            ii[pos] = ii[pos - 1];
            --pos;
        }
        kk[pos] = key;
        ii[pos] = o;
        if (len < k) ++len;
    }
    ScanPair *out = scratch + w * k;
    int head = 0;
    for (int r = 0; r < k; ++r) {
        double hk = head < len ? kk[head] : __longlong_as_double(0x7ff0000000000000ll);
        int64_t hi = head < len ? ii[head] : INT64_MAX;
        double bk = hk;
        int64_t bi = hi;
        for (int off = 16; off > 0; off >>= 1) {
            const double ok = __shfl_xor_sync(0xffffffffu, bk, off);
            const int64_t oi = __shfl_xor_sync(0xffffffffu, bi, off);
            if (pair_less(ok, oi, bk, bi)) {
                bk = ok;
                bi = oi;
            }
        }
        if (lane == 0) out[r] = ScanPair{bk, bi};
        if (head < len && hk == bk && hi == bi) ++head;
    }
}

// One warp per query: merge its `slices` ascending lists of k pairs.
__global__ void k_scan_merge(const ScanPair *__restrict__ scratch, int64_t nq, int k, int slices, int l2,
                             int64_t *__restrict__ ids, float *__restrict__ dist) {
    const int lane = threadIdx.x & 31;
    const int64_t q = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (q >= nq) return;
    const ScanPair *lists = scratch + q * slices * k;
    int head = 0;   // lane s < slices owns list s
    for (int r = 0; r < k; ++r) {
        double hk = __longlong_as_double(0x7ff0000000000000ll);
        int64_t hi = INT64_MAX;
        if (lane < slices && head < k) {
            hk = lists[lane * k + head].key;
            hi = lists[lane * k + head].id;
        }
        double bk = hk;
        int64_t bi = hi;
        for (int off = 16; off > 0; off >>= 1) {
            const double ok = __shfl_xor_sync(0xffffffffu, bk, off);
            const int64_t oi = __shfl_xor_sync(0xffffffffu, bi, off);
            if (pair_less(ok, oi, bk, bi)) {
                bk = ok;
                bi = oi;
            }
        }
        if (lane < slices && head < k && hk == bk && hi == bi && bi != INT64_MAX) ++head;
        if (lane == 0) {
            const bool real = bi != INT64_MAX;
            ids[q * k + r] = real ? bi : -1;
            dist[q * k + r] = real ? __double2float_rn(l2 ? __dsqrt_rn(bk) : bk) : __int_as_float(0x7f800000);
        }
    }
}

// Device address of the scratch array.  In host code the array's name is
// only a host-side stand-in, not a device address, so the address is fetched
// through cudaGetSymbolAddress, once per CUDA context (with the caller's
// device current), and cached under the context's unique id: after a
// cudaDeviceReset the device gets a new primary context, with a new id, and
// the address is looked up again instead of reusing a stale one.
using CtxGetCurrentFn = int (*)(void **);
using CtxGetIdFn = int (*)(void *, unsigned long long *);

unsigned long long current_context_id() {
    static CtxGetCurrentFn get_ctx = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
        void *f1 = nullptr, *f2 = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess)
            get_ctx = (CtxGetCurrentFn)f1;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q2 == cudaDriverEntryPointSuccess)
            get_id = (CtxGetIdFn)f2;
    });
    GTS_REQUIRE(get_ctx && get_id, GTS_ECUDA, "driver entry points cuCtxGetCurrent / cuCtxGetId not found");
    void *ctx = nullptr;
    GTS_REQUIRE(get_ctx(&ctx) == 0, GTS_ECUDA, "cuCtxGetCurrent failed");
    if (!ctx) return 0;
    unsigned long long id = 0;
    GTS_REQUIRE(get_id(ctx, &id) == 0, GTS_ECUDA, "cuCtxGetId failed");
    return id;
}

ScanPair *scratch_ptr() {
    static std::mutex mu;
    static std::unordered_map<unsigned long long, ScanPair *> ptrs;
    std::lock_guard<std::mutex> lock(mu);
    unsigned long long ctx = current_context_id();
    if (ctx != 0) {
        auto it = ptrs.find(ctx);
        if (it != ptrs.end()) return it->second;
    }
    void *p = nullptr;
    GTS_CUDA(cudaGetSymbolAddress(&p, g_scan_scratch));   // also makes the runtime's context current
    GTS_REQUIRE(p != nullptr, GTS_ECUDA, "cudaGetSymbolAddress returned no address");
    ctx = current_context_id();
    GTS_REQUIRE(ctx != 0, GTS_ECUDA, "no current CUDA context after cudaGetSymbolAddress");
    ptrs[ctx] = (ScanPair *)p;
    return (ScanPair *)p;
}

}  // namespace

void knn_scan_noalloc(const float *X, int64_t n, int dim, int metric, const float *Q, int64_t nq, int k,
                      int64_t *ids, float *dist, cudaStream_t st, bool sync) {
    GTS_REQUIRE(metric == GTS_L1 || metric == GTS_L2, GTS_EINVAL, "metric must be GTS_L1 or GTS_L2");
    GTS_REQUIRE(k >= 1 && k <= kScanMaxK, GTS_EINVAL, "k must be in 1 .. 32");
    GTS_REQUIRE(dim >= 1, GTS_EINVAL, "dim must be >= 1");
    GTS_REQUIRE(n >= 0 && n < ((int64_t)1 << 31) && nq >= 0, GTS_EINVAL, "n or nq out of range");
    GTS_REQUIRE(nq * (int64_t)k <= kScratchEntries, GTS_EINVAL,
                "nq * k = " + std::to_string(nq * (int64_t)k) + " exceeds the fixed scratch of " +
                    std::to_string(kScratchEntries) + " entries");
    GTS_REQUIRE(nq == 0 || (Q && ids && dist), GTS_EINVAL, "NULL query or output pointer");
    GTS_REQUIRE(n == 0 || X, GTS_EINVAL, "NULL object pointer");
    if (nq == 0) return;
    ScanPair *scratch = scratch_ptr();
    // slices per query: as many as fit the scratch, up to one per warp lane
    int64_t slices = kScratchEntries / (nq * (int64_t)k);
    if (slices > 32) slices = 32;
    if (slices > n) slices = n > 0 ? n : 1;
    if (slices < 1) slices = 1;
    const int64_t warps = nq * slices;
    k_scan_partial<<<(unsigned)((warps + 7) / 8), 256, 0, st>>>(X, n, dim, metric == GTS_L2, Q, nq, k, (int)slices,
                                                                scratch);
    check_launch("scan partial");
    k_scan_merge<<<(unsigned)((nq + 7) / 8), 256, 0, st>>>(scratch, nq, k, (int)slices, metric == GTS_L2, ids, dist);
    check_launch("scan merge");
    if (sync) GTS_CUDA(cudaStreamSynchronize(st));
}

}  // namespace gts

static gts_status scan_entry(const float *objects, int64_t n, int32_t dim, gts_metric metric, const float *queries,
                             int64_t nq, int32_t k, int64_t *ids, float *dist, void *stream, bool sync) {
    try {
        gts::knn_scan_noalloc(objects, n, dim, (int)metric, queries, nq, k, ids, dist, (cudaStream_t)stream, sync);
        return GTS_OK;
    } catch (const gts::Error &e) {
        gts::set_last_error(e.what());
        return e.status;
    } catch (const std::exception &e) {
        gts::set_last_error(e.what());
        return GTS_ECUDA;
    } catch (...) {
        gts::set_last_error("unknown internal error");
        return GTS_ECUDA;
    }
}

extern "C" gts_status gts_knn_scan_noalloc(const float *objects, int64_t n, int32_t dim, gts_metric metric,
                                           const float *queries, int64_t nq, int32_t k, int64_t *ids, float *dist,
                                           void *stream) {
    return scan_entry(objects, n, dim, metric, queries, nq, k, ids, dist, stream, true);
}

extern "C" gts_status gts_knn_scan_noalloc_async(const float *objects, int64_t n, int32_t dim, gts_metric metric,
                                                 const float *queries, int64_t nq, int32_t k, int64_t *ids,
                                                 float *dist, void *stream) {
    return scan_entry(objects, n, dim, metric, queries, nq, k, ids, dist, stream, false);
}
