// Batched range and kNN search over a GTS index (Section 5, Algorithms 4-5).
//
// One query batch walks the tree level by level.  The frontier (the paper's
// Q_Res) is a query-major list of (query, node) entries; each entry carries the
// query's distances to the pivots on the node's path.  Per level l:
//   1. pivot distances d(q, pivot(N)) of every entry (FP32 for vectors, exact
//      bit-parallel DP for strings);
//   2. kNN only: the threshold tau_q, the k-th smallest distance among distinct
//      visible objects evaluated so far (the pivots), kept as an upper bound in
//      FP64 (Section 5.2: the distance bound starts at infinity and narrows);
//   3. expansion: a child c of entry (q, N) survives unless the interval
//      [d(q,p) - t, d(q,p) + t] misses [lo_c, hi_c], t = r (Lemma 1) or tau_q
//      (Lemma 2, pruning only on a strict miss), with a proven FP32 slack.
// Before each expansion the two-stage scheduler (Section 5.1) bounds the next
// level's table to budget / ((h - l) * fanout) bytes and, if it would not fit,
// runs the entries in groups, depth first.  At the last pivot level the
// surviving leaves of an entry form a bit mask; the leaf scan walks the rows of
// the entry's node (the leaves of one node are contiguous in the table list),
// keeps rows of surviving leaves whose table lower bound max_l |D_l - d_l|
// passes, and emits (query, row) candidates with warp ballots and prefix sums.
// Candidates are verified with the true metric; float metrics carry a proven
// error band and candidates inside it are recomputed in FP64 in the reference
// operation order.  The cache list is scanned by brute force (Section 4.4).
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>
#include <unordered_map>

#include "gts_impl.cuh"
#include "metric.cuh"
#include "pivot_dense.cuh"
#include "tile_l1.cuh"
#include "tile_str.cuh"
#include "tile_tc.cuh"
#include "scan.cuh"

namespace gts {
namespace {

constexpr int kT = 256;
constexpr int kWarpsPerBlock = kT / 32;
constexpr int kKeepCap = 2048;   // exact-key candidates staged in shared memory per query

inline unsigned nblocks(int64_t work, int per) {
    int64_t b = (work + per - 1) / per;
    if (b < 1) b = 1;
    if (b > 0x7fffffffLL) b = 0x7fffffffLL;
    return (unsigned)b;
}

struct Dev {
    int metric, dim, F, h;
    int64_t n;
    const float *X;
    const uint8_t *S;
    const int64_t *Soff;
    const int64_t *row_id;
    const float *table;
    const int64_t *row_del;
    const int32_t *npos, *nsize, *npiv;
    const float *nlo, *nhi;
    int64_t cn;
    const float *cX;
    const uint8_t *cS;
    const int64_t *cSoff, *cid, *cins, *cdel;
    const float *Q;
    const uint8_t *QS;
    const int64_t *QSoff;
    const int64_t *qseq;
    float rel;     // FP32 relative error bound of one distance (0 for edit distance)
    const uint8_t *qg;    // strings: hashed 3-gram counts of the tree rows [n, 64]
    const uint8_t *qgq;   // the same for the batch's queries [nq, 64]
    float epsc;    // pruning slack factor (0 for edit distance)
    // absolute slack of each pivot level's query-to-pivot distances: 0 for
    // FP32 distances (their error is within epsc's relative bound), the
    // tensor-core bound for levels whose dense matrix the tensor cores computed
    float lslack[kMaxHeight];
    float absf;    // absolute floor of every FP32 distance bound (angular distance: the unit-vector rounding)
    // angular distance: the kernels work on unit vectors (X, Q, cX); the FP64
    // keys come from the raw rows and queries
    int cosine;
    const float *Xr, *cXr, *Qr;
    const double *coslim;   // range: 1 - cos(r) per query
};

__device__ __forceinline__ const float *vrow(const Dev &d, int64_t row) {
    return row < d.n ? d.X + row * d.dim : d.cX + (row - d.n) * d.dim;
}
__device__ __forceinline__ bool row_visible(const Dev &d, int64_t row, int64_t s) {
    if (row < d.n) return d.row_del[row] > s;
    const int64_t c = row - d.n;
    return d.cins[c] < s && s < d.cdel[c];
}
__device__ __forceinline__ const float *vrow_raw(const Dev &d, int64_t row) {
    return row < d.n ? d.Xr + row * d.dim : d.cXr + (row - d.n) * d.dim;
}
// The FP64 key of (query, row) in the reference operation order: L2 the
// squared sum, L1 the sum, angular distance 1 - cos on the raw vectors.
template <bool L2>
__device__ __forceinline__ double fp64_key(const Dev &d, int64_t q, int64_t row) {
    if (d.cosine) return cos_key_fp64_seq(d.Qr + q * d.dim, vrow_raw(d, row), d.dim);
    const float *qv = d.Q + q * d.dim, *xv = vrow(d, row);
    return L2 ? l2sq_fp64_seq(qv, xv, d.dim) : l1_fp64_seq(qv, xv, d.dim);
}
// the range limit on the FP64 key and the reported distance of a key
template <bool L2>
__device__ __forceinline__ double fp64_limit(const Dev &d, int64_t q, float r) {
    if (d.cosine) return d.coslim[q];
    return L2 ? __dmul_rn((double)r, (double)r) : (double)r;
}
__device__ __forceinline__ float key_distance(const Dev &d, bool l2, double key) {
    if (d.cosine) return __double2float_rn(acos(__dsub_rn(1.0, key)));
    return __double2float_rn(l2 ? __dsqrt_rn(key) : key);
}

__device__ __forceinline__ int64_t row_oid(const Dev &d, int64_t row) {
    return row < d.n ? d.row_id[row] : d.cid[row - d.n];
}
__device__ __forceinline__ void srow(const Dev &d, int64_t row, const uint8_t *&p, int &len) {
    if (row < d.n) {
        p = d.S + d.Soff[row];
        len = (int)(d.Soff[row + 1] - d.Soff[row]);
    } else {
        const int64_t c = row - d.n;
        p = d.cS + d.cSoff[c];
        len = (int)(d.cSoff[c + 1] - d.cSoff[c]);
    }
}

// first index in [a, b) with v[i] >= x (v sorted ascending)
__device__ __forceinline__ int64_t lower_bound_i32(const int32_t *v, int64_t a, int64_t b, int32_t x) {
    while (a < b) {
        int64_t m = (a + b) >> 1;
        if (v[m] < x) a = m + 1;
        else b = m;
    }
    return a;
}

__global__ void k_fill_f32(float *a, int64_t n, float v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = v;
}
__global__ void k_fill_i64(int64_t *a, int64_t n, int64_t v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = v;
}
__global__ void k_root_entries(int32_t *eq, int32_t *enode, int64_t nq) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nq; i += (int64_t)gridDim.x * blockDim.x) {
        eq[i] = (int32_t)i;
        enode[i] = 0;
    }
}
// Range thresholds in the kernels' distance: the radius (edit distance: its
// floor); angular distance: the chord sqrt(2 (1 - cos r)) of the FP64 limit,
// rounded up, plus the unit-vector slack.
__global__ void k_thresholds(const float *radii, int64_t nq, bool floor_r, const double *coslim, float absf,
                             float *thr) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nq; i += (int64_t)gridDim.x * blockDim.x) {
        if (coslim) {
            const double lim = coslim[i];
            thr[i] = lim < 0.0 ? -1.f : __double2float_ru(__dsqrt_ru(__dmul_ru(2.0, lim))) + absf;
        } else {
            thr[i] = floor_r ? floorf(radii[i]) : radii[i];
        }
    }
}
__global__ void k_k_to_i64(const int32_t *k, int64_t nq, int64_t *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nq; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = k[i];
    if (blockIdx.x == 0 && threadIdx.x == 0) out[nq] = 0;
}

// ---------------------------------------------------------------- pivot distances

// A warp takes runs of kPivGroup consecutive entries (query-major, so the
// query mostly stays in registers); grid-stride over the runs.
constexpr int kPivGroup = 4;

template <bool L2, int NV>
__global__ void k_pivdist_vec(Dev d, const int32_t *__restrict__ eq, const int32_t *__restrict__ enode,
                              int64_t lvl_base, int64_t e0, int64_t e1, float *__restrict__ path, int l) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    float4 qr[NV > 0 ? NV : 1];
    for (int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; e0 + w * kPivGroup < e1; w += nw) {
        const int64_t a0 = e0 + w * kPivGroup;
        const int64_t a1 = a0 + kPivGroup < e1 ? a0 + kPivGroup : e1;
        int32_t cur = -1;
        const float *qv = nullptr;
        for (int64_t e = a0; e < a1; ++e) {
            const int32_t q = eq[e];
            if (q != cur) {
                cur = q;
                qv = d.Q + (int64_t)q * d.dim;
                if (NV > 0) {
                    const float4 *q4 = reinterpret_cast<const float4 *>(qv);
#pragma unroll
                    for (int v = 0; v < (NV > 0 ? NV : 1); ++v) qr[v] = q4[v * 32 + lane];
                }
            }
            const int32_t prow = d.npiv[lvl_base + enode[e]];
            const float s = row_dist_regs<L2, NV>(qr, d.X + (int64_t)prow * d.dim, qv, d.dim, lane);
            if (lane == 0) path[e * d.h + l] = L2 ? sqrtf(s) : s;
        }
    }
}

// Frontier entries of a level whose distances are in a dense matrix.
__global__ void k_pivdist_lookup(const int32_t *__restrict__ eq, const int32_t *__restrict__ enode, int64_t e0,
                                 int64_t e1, const float *__restrict__ dense, int64_t P, float *__restrict__ path,
                                 int h, int l) {
    for (int64_t e = e0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < e1; e += (int64_t)gridDim.x * blockDim.x)
        path[e * h + l] = dense[(int64_t)eq[e] * P + enode[e]];
}

// Strings: blocks take runs of entries; entries of one query share the
// query's match masks (pattern = query, text = pivot).
template <int W>
__global__ void k_pivdist_str(Dev d, const int32_t *__restrict__ eq, const int32_t *__restrict__ enode,
                              int64_t lvl_base, int64_t e0, int64_t e1, int chunk, float *__restrict__ path, int l) {
    __shared__ uint64_t Peq[256 * W];
    const int64_t a0 = e0 + (int64_t)blockIdx.x * chunk;
    const int64_t a1 = a0 + chunk < e1 ? a0 + chunk : e1;
    int64_t s = a0;
    while (s < a1) {
        const int32_t q = eq[s];
        const int64_t t = lower_bound_i32(eq, s, a1, q + 1);
        const int m = (int)(d.QSoff[q + 1] - d.QSoff[q]);
        if (m > 0) build_peq<W>(Peq, d.QS + d.QSoff[q], m);
        for (int64_t e = s + threadIdx.x; e < t; e += blockDim.x) {
            const int32_t prow = d.npiv[lvl_base + enode[e]];
            const uint8_t *tx;
            int len;
            srow(d, prow, tx, len);
            path[e * d.h + l] = (float)(m > 0 ? myers_edit<W>(Peq, m, tx, len) : len);
        }
        __syncthreads();
        s = t;
    }
}

// ---------------------------------------------------------------- kNN threshold

// Insert (u, id) into the ascending list D/I of n (<= K) distinct ids if it
// belongs among the K smallest (u, id).  Warp-cooperative: every lane passes
// the same arguments and gets the same n back; the duplicate test, the
// insert position and the shift take n / 32 steps per lane.
__device__ __forceinline__ void warp_tau_insert(double *D, int64_t *I, int &n, int K, double u, int64_t id,
                                                int lane) {
    if (n >= K && !(u < D[K - 1] || (u == D[K - 1] && id < I[K - 1]))) return;
    bool dup = false;
    int below = 0;
    for (int i = lane; i < n; i += 32) {
        const double di = D[i];
        const int64_t ii = I[i];
        dup |= ii == id;
        below += (di < u || (di == u && ii < id)) ? 1 : 0;
    }
    if (__any_sync(0xffffffffu, dup)) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) below += __shfl_xor_sync(0xffffffffu, below, o);
    const int last = n < K ? n : K - 1;   // entries [below, last) move up one; a full list drops entry K-1
    for (int top = last - 1; top >= below; top -= 32) {
        const int i = top - lane;
        double dv = 0.0;
        int64_t iv = 0;
        if (i >= below) {
            dv = D[i];
            iv = I[i];
        }
        __syncwarp();
        if (i >= below) {
            D[i + 1] = dv;
            I[i + 1] = iv;
        }
        __syncwarp();
    }
    if (lane == 0) {
        D[below] = u;
        I[below] = id;
    }
    __syncwarp();
    if (n < K) ++n;
}

// A query's threshold list as one warp works on it: the K smallest (bound,
// id) of distinct objects, ascending.  With K <= 32 the warp holds it in
// registers (lane i: entry i) between load() and store(); longer lists stay in
// global memory (warp_tau_insert).  insert() keeps exactly the entries that
// warp_tau_insert keeps.  Every member function is warp-uniform.
struct TauList {
    double *D;
    int64_t *I;
    int n, K, lane;
    bool reg;
    double rd;    // lane i's entry (register form)
    int64_t ri;
    __device__ __forceinline__ void load(double *D_, int64_t *I_, int n_, int K_, int lane_) {
        D = D_;
        I = I_;
        n = n_;
        K = K_;
        lane = lane_;
        reg = K <= 32;
        rd = __longlong_as_double(0x7ff0000000000000ll);
        ri = 0x7fffffffffffffffll;
        if (reg && lane < n) {
            rd = D[lane];
            ri = I[lane];
        }
    }
    // entry K - 1 (meaningful once n >= K)
    __device__ __forceinline__ double kd() const { return reg ? __shfl_sync(0xffffffffu, rd, K - 1) : D[K - 1]; }
    __device__ __forceinline__ int64_t kid() const {
        return reg ? (int64_t)__shfl_sync(0xffffffffu, (long long)ri, K - 1) : I[K - 1];
    }
    __device__ __forceinline__ void insert(double u, int64_t id) {
        if (!reg) {
            warp_tau_insert(D, I, n, K, u, id, lane);
            return;
        }
        if (n >= K) {
            const double k_d = kd();
            const int64_t k_i = kid();
            if (!(u < k_d || (u == k_d && id < k_i))) return;
        }
        const bool live = lane < n;
        if (__any_sync(0xffffffffu, live && ri == id)) return;
        const int below = __popc(__ballot_sync(0xffffffffu, live && (rd < u || (rd == u && ri < id))));
        const double pd = __shfl_up_sync(0xffffffffu, rd, 1);
        const int64_t pi = (int64_t)__shfl_up_sync(0xffffffffu, (long long)ri, 1);
        const int last = n < K ? n : K - 1;   // entries [below, last) move up one; a full list drops entry K-1
        if (lane > below && lane <= last) {
            rd = pd;
            ri = pi;
        }
        if (lane == below) {
            rd = u;
            ri = id;
        }
        if (n < K) ++n;
    }
    __device__ __forceinline__ void store() const {
        if (reg && lane < n) {
            D[lane] = rd;
            I[lane] = ri;
        }
        __syncwarp();
    }
};

// the first index of each query's run in the query-sorted entries or candidates
// (and C at nq): one binary search per query, shared by the selection kernels
__global__ void k_query_runs(const int32_t *__restrict__ cq, int64_t C, int64_t nq, int64_t *__restrict__ qoff) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q <= nq; q += (int64_t)gridDim.x * blockDim.x)
        qoff[q] = q == nq ? C : lower_bound_i32(cq, 0, C, (int32_t)q);
}

// Warp per query.  The query's list of the k smallest (upper bound, id) of
// distinct visible pivots seen so far is merged with this level's entries;
// tau_q = the k-th bound, rounded up to float, or +inf while fewer than k.
__global__ void k_tau(Dev d, const int64_t *__restrict__ qrun, const int32_t *__restrict__ enode, int64_t lvl_base,
                      int64_t e0, int64_t e1, const float *__restrict__ path, int l, int64_t nq,
                      const int32_t *__restrict__ kq, const int64_t *__restrict__ koff, double *tk_d, int64_t *tk_id,
                      int32_t *tk_n, float *tau) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t q = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; q < nq; q += nw) {
    const int64_t a = e0 + qrun[q], b = e0 + qrun[q + 1];
    if (a == b) continue;
    const int K = kq[q];
    TauList L;
    L.load(tk_d + koff[q], tk_id + koff[q], tk_n[q], K, lane);
    const int64_t s = d.qseq[q];
    const double up = 1.0 + 2.0 * (double)d.rel;
    for (int64_t base = a; base < b; base += 32) {
        const int64_t e = base + lane;
        const bool full = L.n >= K;
        const double k_d = full ? L.kd() : 0.0;
        const int64_t k_i = full ? L.kid() : 0;
        bool cand = false;
        double ub = 0.0;
        int64_t id = 0;
        if (e < b) {
            const float dv = path[e * d.h + l];
            ub = d.rel > 0.f ? (double)dv * up + (double)d.absf + (double)d.lslack[l] : (double)dv;
            if (!full || ub <= k_d) {   // the bound test before the pivot's delete mark
                const int32_t prow = d.npiv[lvl_base + enode[e]];
                if (row_visible(d, prow, s)) {
                    id = d.row_id[prow];
                    cand = !full || ub < k_d || (ub == k_d && id < k_i);
                }
            }
        }
        unsigned bal = __ballot_sync(0xffffffffu, cand);
        while (bal) {
            const int src = __ffs(bal) - 1;
            bal &= bal - 1;
            const double u = __shfl_sync(0xffffffffu, ub, src);
            const int64_t iid = __shfl_sync(0xffffffffu, id, src);
            L.insert(u, iid);
        }
    }
    L.store();
    const double k_fin = L.n >= K ? L.kd() : 0.0;
    if (lane == 0) {
        tk_n[q] = L.n;
        tau[q] = L.n >= K ? __double2float_ru(k_fin) : __int_as_float(0x7f800000);
    }
    }
}

struct LevelOffsets {
    int64_t v[kMaxHeight + 2];
};

constexpr int kProbeNodes = 4;   // last-level nodes whose rows the kNN probe evaluates

// Probe for kNN (warp per query).  Section 3 notes that MkNNQ(q, k) is
// MRQ(q, d_k) once d_k is known; the probe bounds d_k from above before the
// batched descent.  It follows one root-to-last-level path: at every level it
// computes the distances from q to the pivots of all non-empty children and
// descends into the child whose pivot is nearest; at the last pivot level it
// computes the distances to the rows (up to `cap` in all) of the kProbeNodes
// nodes with the nearest pivots.  Every visible object so
// evaluated enters the query's threshold list, so tau_q starts at (an upper
// bound of) the k-th smallest of them instead of +inf.
// One lane's distance from q to one row (coordinates in increasing order;
// L2 returns the square).  The FP32 bound of the plain path covers any order.
template <bool L2>
__device__ __forceinline__ float lane_vec_dist(const float *__restrict__ q, const float *__restrict__ x, int dim) {
    float s = 0.f;
    if ((dim & 3) == 0 && ((((uintptr_t)q) | ((uintptr_t)x)) & 15) == 0) {
        const float4 *q4 = reinterpret_cast<const float4 *>(q);
        const float4 *x4 = reinterpret_cast<const float4 *>(x);
        for (int i = 0; i < (dim >> 2); ++i) {
            const float4 a = q4[i], b = __ldg(x4 + i);
            const float d0 = a.x - b.x, d1 = a.y - b.y, d2 = a.z - b.z, d3 = a.w - b.w;
            if (L2) s += d0 * d0 + d1 * d1 + d2 * d2 + d3 * d3;
            else s += fabsf(d0) + fabsf(d1) + fabsf(d2) + fabsf(d3);
        }
    } else {
        for (int i = 0; i < dim; ++i) {
            const float t = q[i] - __ldg(x + i);
            s += L2 ? t * t : fabsf(t);
        }
    }
    return s;
}

// Rows [pos, pos + m) into the threshold list, a row per lane.
template <bool L2>
__device__ __forceinline__ void probe_rows(const Dev &d, const float *qv, int64_t pos, int32_t m, int64_t s,
                                           TauList &L, double up, int lane) {
    for (int32_t r0 = 0; r0 < m; r0 += 32) {
        const int32_t r = r0 + lane;
        const bool full = L.n >= L.K;
        const double k_d = full ? L.kd() : 0.0;
        const int64_t k_i = full ? L.kid() : 0;
        bool cand = false;
        double ub = 0.0;
        int64_t id = 0;
        if (r < m) {
            const int64_t row = pos + r;
            if (d.row_del[row] > s) {
                const float sq = lane_vec_dist<L2>(qv, d.X + row * d.dim, d.dim);
                const float dv = L2 ? sqrtf(sq) : sq;
                ub = (double)dv * up + (double)d.absf;
                id = d.row_id[row];
                cand = !full || ub < k_d || (ub == k_d && id < k_i);
            }
        }
        unsigned bal = __ballot_sync(0xffffffffu, cand);
        while (bal) {
            const int src = __ffs(bal) - 1;
            bal &= bal - 1;
            const double u = __shfl_sync(0xffffffffu, ub, src);
            const int64_t iid = __shfl_sync(0xffffffffu, id, src);
            L.insert(u, iid);
        }
    }
}

// Probe for kNN (warp per query).  Section 3 notes that MkNNQ(q, k) is
// MRQ(q, d_k) once d_k is known; the probe bounds d_k from above before the
// batched descent.  It follows one root-to-last-level path: at every level it
// computes the distances from q to the pivots of all non-empty children and
// descends into the child whose pivot is nearest; at the last pivot level it
// computes the distances to the rows (up to `cap` in all) of the kProbeNodes
// nodes with the nearest pivots.  Every visible object so evaluated enters
// the query's threshold list, so tau_q starts at (an upper bound of) the k-th
// smallest of them instead of +inf.  The last-level node the path ended in is
// the query's key: queries with equal or nearby keys lie in the same region.
template <bool L2>
__global__ void k_probe_vec(Dev d, LevelOffsets lo_off, int64_t nq, int cap, const int32_t *__restrict__ kq,
                            const int64_t *__restrict__ koff, double *tk_d, int64_t *tk_id, int32_t *tk_n,
                            float *tau, int32_t *__restrict__ key) {
    const int lane = threadIdx.x & 31;
    const int64_t q = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (q >= nq) return;
    const int K = kq[q];
    TauList L;
    L.load(tk_d + koff[q], tk_id + koff[q], tk_n[q], K, lane);
    const int64_t s = d.qseq[q];
    const float *qv = d.Q + q * d.dim;
    const double up = 1.0 + 2.0 * (double)d.rel;
    // root pivot
    {
        const int32_t prow = d.npiv[lo_off.v[0]];
        const float sq = warp_vec_dist<L2>(qv, d.X + (int64_t)prow * d.dim, d.dim, lane);
        const float dq = L2 ? sqrtf(sq) : sq;
        if (d.row_del[prow] > s) L.insert((double)dq * up + (double)d.absf, d.row_id[prow]);
    }
    int64_t node = 0;
    if (d.h == 1) {   // one pivot level: the root's own rows
        const int32_t m = d.nsize[lo_off.v[0]] < cap ? d.nsize[lo_off.v[0]] : cap;
        probe_rows<L2>(d, qv, d.npos[lo_off.v[0]], m, s, L, up, lane);
    }
    for (int l = 1; l < d.h; ++l) {
        // the kProbeNodes children with the nearest pivots (ascending), kept by every lane
        float bd[kProbeNodes];
        int64_t bn[kProbeNodes];
#pragma unroll
        for (int i = 0; i < kProbeNodes; ++i) {
            bd[i] = __int_as_float(0x7f800000);
            bn[i] = -1;
        }
        // the children 32 at a time, a child per lane: their pivot distances
        // are computed together, then taken in child order
        for (int j0 = 0; j0 < d.F; j0 += 32) {
            const int j = j0 + lane;
            float dq = 0.f;
            bool live = false, vis = false;
            int64_t id = 0;
            if (j < d.F) {
                const int64_t g = lo_off.v[l] + node * d.F + j;
                if (d.nsize[g] != 0) {
                    const int32_t prow = d.npiv[g];
                    const float sq = lane_vec_dist<L2>(qv, d.X + (int64_t)prow * d.dim, d.dim);
                    dq = L2 ? sqrtf(sq) : sq;
                    live = true;
                    vis = d.row_del[prow] > s;
                    if (vis) id = d.row_id[prow];
                }
            }
            // the visible pivots into the threshold list (a register copy of
            // its K-th bound skips the pivots that cannot enter it)
            const double ub = (double)dq * up + (double)d.absf;
            const bool full = L.n >= K;
            const double kth = full ? L.kd() : 0.0;
            unsigned bal = __ballot_sync(0xffffffffu, vis && (!full || ub <= kth));
            while (bal) {
                const int src = __ffs(bal) - 1;
                bal &= bal - 1;
                const double uu = __shfl_sync(0xffffffffu, ub, src);
                const int64_t iid = __shfl_sync(0xffffffffu, id, src);
                L.insert(uu, iid);
            }
            // the nearest children, in child order (ties keep the earlier child)
            unsigned lv = __ballot_sync(0xffffffffu, live);
            while (lv) {
                const int src = __ffs(lv) - 1;
                lv &= lv - 1;
                float vd = __shfl_sync(0xffffffffu, dq, src);
                int64_t vn = node * d.F + j0 + src;
                if (vd < bd[kProbeNodes - 1]) {
#pragma unroll
                    for (int i = 0; i < kProbeNodes; ++i) {
                        if (vd < bd[i]) {
                            const float td = bd[i];
                            const int64_t tn = bn[i];
                            bd[i] = vd;
                            bn[i] = vn;
                            vd = td;
                            vn = tn;
                        }
                    }
                }
            }
        }
        if (bn[0] < 0) break;   // no non-empty child (cannot happen for a non-empty node)
        node = bn[0];
        if (l == d.h - 1) {
            // last pivot level: the rows of the nearest kProbeNodes nodes
            int budget = cap;
#pragma unroll
            for (int i = 0; i < kProbeNodes; ++i) {
                if (bn[i] < 0 || budget <= 0) continue;
                const int64_t g = lo_off.v[l] + bn[i];
                const int32_t m = d.nsize[g] < budget ? d.nsize[g] : budget;
                budget -= m;
                probe_rows<L2>(d, qv, d.npos[g], m, s, L, up, lane);
            }
        }
    }
    L.store();
    const double k_fin = L.n >= K ? L.kd() : 0.0;
    if (lane == 0) {
        tk_n[q] = L.n;
        tau[q] = L.n >= K ? __double2float_ru(k_fin) : __int_as_float(0x7f800000);
        if (key) key[q] = (int32_t)node;   // where the path ended: a locality key for the query
    }
}

// ---------------------------------------------------------------- expansion

__device__ __forceinline__ bool interval_hit(float dq, float thr, float lo, float hi, float epsc, float abs_slack) {
    const float eps = (epsc > 0.f ? epsc * (dq + thr + fabsf(hi)) : 0.f) + abs_slack;
    return (dq - thr <= hi + eps) && (dq + thr + eps >= lo);
}

// MODE 0: test the children of every entry, write the survivor bit mask and
// its population count; 1: write the survivors named by the mask as the next
// level's entries (the mask fixes the count, whatever the threshold has
// become since: kNN thresholds only shrink while earlier groups run); 2: last
// pivot level, write the surviving-leaf mask only.
template <int MODE>
__global__ void k_expand(Dev d, const int32_t *__restrict__ eq, const int32_t *__restrict__ enode,
                         const float *__restrict__ path, int l, int64_t lvl_next, int64_t e0, int64_t e1,
                         const float *__restrict__ thr_q, int32_t *__restrict__ cnt, const int64_t *__restrict__ off,
                         int32_t *__restrict__ nq_out, int32_t *__restrict__ nnode_out, float *__restrict__ npath_out,
                         uint64_t *__restrict__ mask_io) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    if (MODE != 1) {
        // 32 entries per warp step: lane i loads entry i's data, the warp
        // tests each entry's children in turn (a child per lane), lane i
        // keeps entry i's mask, and the masks are written together
        for (int64_t g0 = e0 + ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5) * 32; g0 < e1; g0 += nw * 32) {
            const int64_t eg = g0 + lane;
            const bool in = eg < e1;
            const int32_t gnode = in ? enode[eg] : 0;
            const float gdq = in ? path[eg * d.h + l] : 0.f;
            const float gthr = in ? thr_q[eq[eg]] : 0.f;
            const int ne = e1 - g0 < 32 ? (int)(e1 - g0) : 32;
            uint64_t my_m = 0;
            for (int i = 0; i < ne; ++i) {
                const int32_t node = __shfl_sync(0xffffffffu, gnode, i);
                const float dq = __shfl_sync(0xffffffffu, gdq, i);
                const float thr = __shfl_sync(0xffffffffu, gthr, i);
                uint64_t m = 0;
                for (int j0 = 0; j0 < d.F; j0 += 32) {
                    const int j = j0 + lane;
                    bool keep = false;
                    if (j < d.F) {
                        const int64_t c = lvl_next + (int64_t)node * d.F + j;
                        keep = d.nsize[c] > 0 && interval_hit(dq, thr, d.nlo[c], d.nhi[c], d.epsc, d.lslack[l]);
                    }
                    m |= (uint64_t)__ballot_sync(0xffffffffu, keep) << j0;
                }
                if (lane == i) my_m = m;
            }
            if (in) {
                mask_io[eg - e0] = my_m;
                if (MODE == 0) cnt[eg - e0] = __popcll(my_m);
            }
        }
        return;
    }
    for (int64_t e = e0 + ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5); e < e1; e += nw) {
    const int32_t q = eq[e];
    const int32_t node = enode[e];
    if (MODE == 1) {
        const uint64_t m = mask_io[e - e0];
        const int64_t base = off[e - e0];
        for (int j0 = 0; j0 < d.F; j0 += 32) {
            const int j = j0 + lane;
            if (j < d.F && ((m >> j) & 1ull)) {
                const int64_t o = base + __popcll(m & ((1ull << j) - 1ull));
                nq_out[o] = q;
                nnode_out[o] = node * d.F + j;
                for (int t = 0; t <= l; ++t) npath_out[o * d.h + t] = path[e * d.h + t];
            }
        }
        continue;
    }
    const float dq = path[e * d.h + l];
    const float thr = thr_q[q];
    uint64_t m = 0;
    for (int j0 = 0; j0 < d.F; j0 += 32) {
        const int j = j0 + lane;
        bool keep = false;
        if (j < d.F) {
            const int64_t c = lvl_next + (int64_t)node * d.F + j;
            keep = d.nsize[c] > 0 && interval_hit(dq, thr, d.nlo[c], d.nhi[c], d.epsc, d.lslack[l]);
        }
        m |= (uint64_t)__ballot_sync(0xffffffffu, keep) << j0;
    }
    if (lane == 0) {
        mask_io[e - e0] = m;
        if (MODE == 0) cnt[e - e0] = __popcll(m);
    }
    }
}

// Last pivot level, tensor-core path: one pass per entry computes d(q, pivot),
// tests the node's leaf children against [d - t, d + t] (Lemma 1 / 2) into a
// bit mask, and counts the entries with a surviving leaf per node for the
// regrouping.  A warp takes kLastGroup consecutive entries and issues each
// stage's loads for all of them before using any (entry ids, pivot rows,
// query rows, leaf intervals), so the dependent-load latencies overlap.
constexpr int kLastGroup = 8;

template <bool L2, int NV>
__global__ void k_last_level_vec(Dev d, const int32_t *__restrict__ eq, const int32_t *__restrict__ enode,
                                 int64_t lvl_base, int64_t lvl_next, int64_t e0, int64_t e1,
                                 float *__restrict__ path, int l, const float *__restrict__ thr_q,
                                 uint64_t *__restrict__ mask_out, int32_t *__restrict__ ncount,
                                 const float *__restrict__ dense, int64_t P) {
    constexpr int G = kLastGroup;
    constexpr int V = NV > 0 ? NV : 1;
    const float lab = dense ? d.lslack[l] : 0.f;   // the slack of the dense matrix's distances
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; e0 + w * G < e1; w += nw) {
        const int64_t a0 = e0 + w * G;
        const int cnt = (int)(e1 - a0 < G ? e1 - a0 : G);
        // stage 1: entry ids, nodes, pivots, thresholds (lane i < cnt loads entry i)
        int32_t my_q = 0, my_node = 0, my_prow = 0;
        float my_thr = 0.f;
        if (lane < cnt) {
            my_q = eq[a0 + lane];
            my_node = enode[a0 + lane];
        }
        if (lane < cnt) {
            my_prow = d.npiv[lvl_base + my_node];
            my_thr = thr_q[my_q];
        }
        float dq[G];
        if (dense) {   // distances from the level's dense matrix
            const float my_d = lane < cnt ? dense[(int64_t)my_q * P + my_node] : 0.f;
#pragma unroll
            for (int i = 0; i < G; ++i) dq[i] = __shfl_sync(0xffffffffu, my_d, i);
        } else {
        // stage 2: pivot rows and query rows of all entries
        float4 pr[G][V], qr[G][V];
#pragma unroll
        for (int i = 0; i < G; ++i) {
            const int32_t prow = __shfl_sync(0xffffffffu, my_prow, i);
            const int32_t q = __shfl_sync(0xffffffffu, my_q, i);
            if (i < cnt) {
                if (NV > 0) {
                    const float4 *p4 = reinterpret_cast<const float4 *>(d.X + (int64_t)prow * d.dim);
                    const float4 *q4 = reinterpret_cast<const float4 *>(d.Q + (int64_t)q * d.dim);
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        pr[i][v] = __ldg(p4 + v * 32 + lane);
                        qr[i][v] = __ldg(q4 + v * 32 + lane);
                    }
                }
            }
        }
        // stage 3: distances
#pragma unroll
        for (int i = 0; i < G; ++i) {
            dq[i] = 0.f;
            if (i < cnt) {
                float sq;
                if (NV > 0) {
                    sq = 0.f;
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        const float4 x = pr[i][v], y = qr[i][v];
                        const float t0 = y.x - x.x, t1 = y.y - x.y, t2 = y.z - x.z, t3 = y.w - x.w;
                        sq += L2 ? t0 * t0 + t1 * t1 + t2 * t2 + t3 * t3 : fabsf(t0) + fabsf(t1) + fabsf(t2) + fabsf(t3);
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
                } else {
                    const int32_t prow = __shfl_sync(0xffffffffu, my_prow, i);
                    const int32_t q = __shfl_sync(0xffffffffu, my_q, i);
                    sq = warp_vec_dist<L2>(d.Q + (int64_t)q * d.dim, d.X + (int64_t)prow * d.dim, d.dim, lane);
                }
                dq[i] = L2 ? sqrtf(sq) : sq;
            }
        }
        }
        // stage 4: leaf intervals of all entries, then the tests; lane i
        // collects entry i's mask
        uint64_t my_mask = 0;
        for (int j0 = 0; j0 < d.F; j0 += 32) {
            const int j = j0 + lane;
            int32_t sz[G];
            float lo[G], hi[G];
#pragma unroll
            for (int i = 0; i < G; ++i) {
                const int32_t node = __shfl_sync(0xffffffffu, my_node, i);
                sz[i] = 0;
                lo[i] = hi[i] = 0.f;
                if (i < cnt && j < d.F) {
                    const int64_t c = lvl_next + (int64_t)node * d.F + j;
                    sz[i] = d.nsize[c];
                    lo[i] = d.nlo[c];
                    hi[i] = d.nhi[c];
                }
            }
#pragma unroll
            for (int i = 0; i < G; ++i) {
                const float thr = __shfl_sync(0xffffffffu, my_thr, i);
                const bool keep = i < cnt && j < d.F && sz[i] > 0 && interval_hit(dq[i], thr, lo[i], hi[i], d.epsc, lab);
                const uint64_t m = (uint64_t)__ballot_sync(0xffffffffu, keep) << j0;
                if (lane == i) my_mask |= m;
            }
        }
        float my_dq = 0.f;
#pragma unroll
        for (int i = 0; i < G; ++i)
            if (lane == i) my_dq = dq[i];
        if (lane < cnt) {
            path[(a0 + lane) * d.h + l] = my_dq;
            mask_out[a0 + lane - e0] = my_mask;
            if (my_mask && ncount) atomicAdd(&ncount[my_node], 1);
        }
    }
}

// Last pivot level with the distances in a dense matrix: thread per entry,
// the leaf mask from the node's children intervals (Lemma 1 / 2).
__global__ void k_leaf_masks_dense(Dev d, const int32_t *__restrict__ eq, const int32_t *__restrict__ enode,
                                   int64_t lvl_next, int64_t e0, int64_t e1, const float *__restrict__ dense,
                                   int64_t P, float *__restrict__ path, int l, const float *__restrict__ thr_q,
                                   uint64_t *__restrict__ mask_out) {
    for (int64_t e = e0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < e1; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t q = eq[e], node = enode[e];
        const float dq = dense[(int64_t)q * P + node];
        const float thr = thr_q[q];
        const int64_t c0 = lvl_next + (int64_t)node * d.F;
        uint64_t m = 0;
        for (int j = 0; j < d.F; ++j)
            if (d.nsize[c0 + j] > 0 && interval_hit(dq, thr, d.nlo[c0 + j], d.nhi[c0 + j], d.epsc, d.lslack[l]))
                m |= 1ull << j;
        path[e * d.h + l] = dq;
        mask_out[e - e0] = m;
    }
}

// ---------------------------------------------------------------- leaf scan

// Warp per last-level entry: rows of the entry's node, in 32-row strips; a
// row passes if its leaf survived, it is visible at the query's sequence
// number and its table lower bound max_l |D_l(row) - d(q, p_l)| is within the
// threshold (Lemma 1 / Lemma 2 on every pivot of the path).
template <bool WRITE>
__global__ void k_leafscan(Dev d, const int32_t *__restrict__ eq, const int32_t *__restrict__ enode,
                           const float *__restrict__ path, int64_t lvl_last, int64_t e0, int64_t e1,
                           const uint64_t *__restrict__ mask, const float *__restrict__ thr_q,
                           int32_t *__restrict__ cnt, const int64_t *__restrict__ off, int32_t *__restrict__ cq,
                           int32_t *__restrict__ crow, unsigned long long *__restrict__ scanned) {
    const int lane = threadIdx.x & 31;
    const int64_t e = e0 + ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    if (e >= e1) return;
    const uint64_t m = mask[e - e0];
    if (m == 0) {
        if (!WRITE && lane == 0) cnt[e - e0] = 0;
        return;
    }
    const int32_t q = eq[e];
    const int64_t node = lvl_last + enode[e];
    const int32_t pos = d.npos[node], size = d.nsize[node];
    const int32_t avg = size / d.F;
    const int64_t s = d.qseq[q];
    const float thr = thr_q[q];
    float dq[kMaxHeight];
#pragma unroll
    for (int t = 0; t < kMaxHeight; ++t) dq[t] = t < d.h ? path[e * d.h + t] : 0.f;
    int64_t count = 0, tested = 0;
    const int64_t base = WRITE ? off[e - e0] : 0;
    // the write pass re-tests with the same thresholds as the count pass; the
    // bound keeps every write inside this entry's slot regardless
    const int64_t lim = WRITE ? off[e - e0 + 1] : 0;
    for (int32_t r0 = 0; r0 < size; r0 += 32) {
        const int32_t r = r0 + lane;
        bool pass = false, test = false;
        if (r < size) {
            int32_t j = avg > 0 ? r / avg : d.F - 1;
            if (j > d.F - 1) j = d.F - 1;
            if ((m >> j) & 1ull) {
                test = true;
                const int64_t row = pos + r;
                if (d.row_del[row] > s) {
                    pass = true;
#pragma unroll
                    for (int t = 0; t < kMaxHeight; ++t) {
                        if (t < d.h) {
                            const float T = d.table[(int64_t)t * d.n + row];
                            const float eps = (d.epsc > 0.f ? d.epsc * (T + dq[t] + thr) : 0.f) + d.lslack[t];
                            if (fabsf(T - dq[t]) > thr + eps) pass = false;
                        }
                    }
                }
            }
        }
        const unsigned b = __ballot_sync(0xffffffffu, pass);
        if (WRITE && pass) {
            const int64_t o = base + count + __popc(b & ((1u << lane) - 1u));
            if (o < lim) {
                cq[o] = q;
                crow[o] = pos + r;
            }
        }
        count += __popc(b);
        tested += __popc(__ballot_sync(0xffffffffu, test));
    }
    if (!WRITE && lane == 0) {
        cnt[e - e0] = (int32_t)count;
        atomicAdd(scanned, (unsigned long long)tested);
    }
}

// ---------------------------------------------------------------- diagnostics

// Per-query distances to every pivot level, for the count below.
struct DenseLevels {
    const float *D[kMaxHeight];   // level l: [nq, P_l], query-major
    int64_t P[kMaxHeight];
};

// Diagnostics (not on the answer path): the dense last level's (query, row)
// pairs that pass visibility and the table lower bound of Lemma 1 / 2 on
// every pivot of the row's path, with the search's FP32 slack -- the
// candidates C_q a per-candidate verification would check.  Thread per
// (last-level node, column position) pair of the leaf-mask matrix M.
__global__ void k_count_table_pass_dense(Dev d, DenseLevels dl, const uint64_t *__restrict__ M,
                                         const int32_t *__restrict__ perm, int64_t P, int64_t nq, int64_t lvl_leaf,
                                         const float *__restrict__ thr_q, unsigned long long *__restrict__ count) {
    unsigned long long c = 0;
    const int64_t total = P * nq;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t m = M[t];
        if (!m) continue;
        const int64_t p = t / nq, pos = t - p * nq;
        const int64_t q = perm ? (int64_t)perm[pos] : pos;
        float dq[kMaxHeight];
        int64_t anc = p;   // the level-l ancestor of node p (Eq. 1: parent = child / F)
        for (int l = d.h - 1; l >= 0; --l) {
            dq[l] = dl.D[l][q * dl.P[l] + anc];
            anc /= d.F;
        }
        const float thr = thr_q[q];
        const int64_t s = d.qseq[q];
        for (int j = 0; j < d.F; ++j) {
            if (!((m >> j) & 1ull)) continue;
            const int64_t leaf = lvl_leaf + p * d.F + j;
            const int64_t r0 = d.npos[leaf], r1 = r0 + d.nsize[leaf];
            for (int64_t r = r0; r < r1; ++r) {
                if (d.row_del[r] <= s) continue;
                bool pass = true;
                for (int l = 0; l < d.h && pass; ++l) {
                    const float T = d.table[(int64_t)l * d.n + r];
                    const float eps = (d.epsc > 0.f ? d.epsc * (T + dq[l] + thr) : 0.f) + d.lslack[l];
                    if (fabsf(T - dq[l]) > thr + eps) pass = false;
                }
                c += pass ? 1 : 0;
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

__global__ void k_sum_i32(const int32_t *__restrict__ a, int64_t n, unsigned long long *__restrict__ out) {
    unsigned long long c = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        c += (unsigned long long)a[i];
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

// Cache list (Section 4.4): every (query, cache slot) pair of a query range.
__global__ void k_cache_cands(int64_t qa, int64_t qb, int64_t n, int64_t cn, int32_t *cq, int32_t *crow) {
    const int64_t total = (qb - qa) * cn;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = qa + i / cn;
        cq[i] = (int32_t)q;
        crow[i] = (int32_t)(n + i % cn);
    }
}

// ---------------------------------------------------------------- verification

// A warp takes kVerifyGroup consecutive candidates (query-major, so they
// mostly share a query, which then stays in registers), sums their distances
// one after another, and then decides them together, a lane per candidate.
// Range: accept when
// the FP32 upper bound is below r, reject when the lower bound is above r,
// otherwise decide in FP64 exactly as the CPU reference does.  kNN: keep the
// candidate if its lower bound is within the query's threshold tau_q (an
// upper bound of the k-th distance; a farther candidate cannot be in the top
// k) and store its FP32 distance.
constexpr int kVerifyGroup = 32;   // pairs per warp in k_verify_vec (at most 32: one per lane)

template <bool L2, bool KNN, int NV>
__global__ void k_verify_vec(Dev d, const int32_t *__restrict__ cq, const int32_t *__restrict__ crow, int64_t C,
                             const float *__restrict__ thr_q, float *__restrict__ cdist, uint8_t *__restrict__ keep,
                             unsigned long long *__restrict__ rechecks) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    float4 qr[NV > 0 ? NV : 1];
    for (int64_t c0 = ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5) * kVerifyGroup; c0 < C;
         c0 += nw * kVerifyGroup) {
    const int64_t c1 = c0 + kVerifyGroup < C ? c0 + kVerifyGroup : C;
    const int ng = (int)(c1 - c0);
    // the group's pairs (lane i: pair c0 + i); the warp sums each pair's
    // distance in turn and lane i keeps pair i's, then the lanes decide
    // their pairs together
    const int32_t gq = lane < ng ? cq[c0 + lane] : 0;
    const int32_t grow = lane < ng ? crow[c0 + lane] : 0;
    float my_d32 = 0.f;
    bool my_vis = true;
    int32_t cur = -1;
    const float *qv = nullptr;
    for (int i = 0; i < ng; ++i) {
        const int32_t q = __shfl_sync(0xffffffffu, gq, i);
        const int64_t row = __shfl_sync(0xffffffffu, grow, i);
        if (q != cur) {
            cur = q;
            qv = d.Q + (int64_t)q * d.dim;
            if (NV > 0) {
                const float4 *q4 = reinterpret_cast<const float4 *>(qv);
#pragma unroll
                for (int v = 0; v < (NV > 0 ? NV : 1); ++v) qr[v] = q4[v * 32 + lane];
            }
        }
        const bool vis = !(row >= d.n && !row_visible(d, row, d.qseq[q]));
        float sq = 0.f;
        if (vis) sq = row_dist_regs<L2, NV>(qr, vrow(d, row), qv, d.dim, lane);
        if (lane == i) {
            my_vis = vis;
            my_d32 = L2 ? sqrtf(sq) : sq;
        }
    }
    if (lane < ng) {
        const int64_t c = c0 + lane;
        if (!my_vis) {
            cdist[c] = __int_as_float(0x7f800000);
            keep[c] = 0;
        } else {
        const int32_t q = gq;
        const float d32 = my_d32;
        const float r = thr_q[q];
        const float hi = d32 * (1.f + 2.f * d.rel) + d.absf;
        const float lo = d32 * (1.f - 2.f * d.rel) - d.absf;
        if (KNN) {
            cdist[c] = d32;
            keep[c] = lo <= r ? 1 : 0;
        } else if (!d.cosine && hi < r * (1.f - 1e-9f)) {   // (angular: the FP64 key decides every kept pair)
            keep[c] = 1;
            cdist[c] = d32;
        } else if (lo > r * (1.f + 1e-9f)) {
            keep[c] = 0;
        } else {
            const double key = fp64_key<L2>(d, q, (int64_t)grow);
            keep[c] = key <= fp64_limit<L2>(d, q, r) ? 1 : 0;
            cdist[c] = key_distance(d, L2, key);
            atomicAdd(rechecks, 1ull);
        }
        }
    }
    }
}

// The same verification for vectors of at most 16 dimensions, a thread per
// pair: at low dimension a warp per pair leaves most lanes idle, while a
// thread reads its whole row (consecutive pairs of a query read consecutive
// rows) and sums it in FP32 in coordinate order, within the same error bound.
template <bool L2, bool KNN>
__global__ void k_verify_lowdim(Dev d, const int32_t *__restrict__ cq, const int32_t *__restrict__ crow, int64_t C,
                                const float *__restrict__ thr_q, float *__restrict__ cdist,
                                uint8_t *__restrict__ keep, unsigned long long *__restrict__ rechecks) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < C; c += (int64_t)gridDim.x * blockDim.x) {
        const int32_t q = cq[c];
        const int64_t row = crow[c];
        if (row >= d.n && !row_visible(d, row, d.qseq[q])) {
            cdist[c] = __int_as_float(0x7f800000);
            keep[c] = 0;
            continue;
        }
        const float *qv = d.Q + (int64_t)q * d.dim;
        const float *xv = vrow(d, row);
        float sum = 0.f;
        for (int i = 0; i < d.dim; ++i) {
            const float t = qv[i] - xv[i];
            sum = L2 ? fmaf(t, t, sum) : sum + fabsf(t);
        }
        const float d32 = L2 ? sqrtf(sum) : sum;
        const float r = thr_q[q];
        const float hi = d32 * (1.f + 2.f * d.rel) + d.absf;
        const float lo = d32 * (1.f - 2.f * d.rel) - d.absf;
        if (KNN) {
            cdist[c] = d32;
            keep[c] = lo <= r ? 1 : 0;
        } else if (!d.cosine && hi < r * (1.f - 1e-9f)) {   // (angular: the FP64 key decides every kept pair)
            keep[c] = 1;
            cdist[c] = d32;
        } else if (lo > r * (1.f + 1e-9f)) {
            keep[c] = 0;
        } else {
            const double key = fp64_key<L2>(d, q, row);
            keep[c] = key <= fp64_limit<L2>(d, q, r) ? 1 : 0;
            cdist[c] = key_distance(d, L2, key);
            atomicAdd(rechecks, 1ull);
        }
    }
}

// Cache list (Section 4.4), range queries over vectors of at most 16
// dimensions: every (query, cache slot) pair of the queries [qa, qb) is
// verified as k_verify_lowdim verifies it (the same FP32 sum in coordinate
// order, the same band, the same FP64 decision), and the kept pairs go
// straight into the answer keys (query << 32 | id) and distances, a warp's
// kept pairs at one atomic -- no candidate list is written.  rkey / rdist
// hold (qb - qa) * cn entries, at least the pairs kept.
template <bool L2>
__global__ void k_cache_range_lowdim(Dev d, int64_t qa, int64_t qb, int64_t cn, const float *__restrict__ thr_q,
                                     uint64_t *__restrict__ rkey, float *__restrict__ rdist,
                                     unsigned long long *__restrict__ count,
                                     unsigned long long *__restrict__ rechecks) {
    const int lane = threadIdx.x & 31;
    const int64_t total = (qb - qa) * cn;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // base is the warp's first pair: every lane runs the same iterations
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < total; base += stride) {
        const int64_t i = base + lane;
        bool kept = false;
        float dist = 0.f;
        int64_t q = 0, row = 0;
        if (i < total) {
            q = qa + i / cn;
            row = d.n + i % cn;
            if (row_visible(d, row, d.qseq[q])) {
                const float *qv = d.Q + q * d.dim;
                const float *xv = vrow(d, row);
                float sum = 0.f;
                for (int k = 0; k < d.dim; ++k) {
                    const float t = qv[k] - xv[k];
                    sum = L2 ? fmaf(t, t, sum) : sum + fabsf(t);
                }
                const float d32 = L2 ? sqrtf(sum) : sum;
                const float r = thr_q[q];
                const float hi = d32 * (1.f + 2.f * d.rel) + d.absf;
                const float lo = d32 * (1.f - 2.f * d.rel) - d.absf;
                if (!d.cosine && hi < r * (1.f - 1e-9f)) {   // (angular: the FP64 key decides every kept pair)
                    kept = true;
                    dist = d32;
                } else if (!(lo > r * (1.f + 1e-9f))) {
                    const double key = fp64_key<L2>(d, q, row);
                    kept = key <= fp64_limit<L2>(d, q, r);
                    dist = key_distance(d, L2, key);
                    atomicAdd(rechecks, 1ull);
                }
            }
        }
        const unsigned m = __ballot_sync(0xffffffffu, kept);
        if (m) {
            unsigned long long b = 0;
            if (lane == 0) b = atomicAdd(count, (unsigned long long)__popc(m));
            b = __shfl_sync(0xffffffffu, b, 0);
            if (kept) {
                const unsigned long long o = b + (unsigned long long)__popc(m & ((1u << lane) - 1u));
                rkey[o] = ((uint64_t)(uint32_t)q << 32) | (uint64_t)(uint32_t)row_oid(d, row);
                rdist[o] = dist;
            }
        }
    }
}

__global__ void k_compact_cands(const int32_t *__restrict__ cq, const int32_t *__restrict__ crow,
                                const float *__restrict__ cdist, const uint8_t *__restrict__ keep, int64_t C,
                                const int64_t *__restrict__ pos, int32_t *__restrict__ oq, int32_t *__restrict__ orow,
                                float *__restrict__ od) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < C; c += (int64_t)gridDim.x * blockDim.x) {
        if (!keep[c]) continue;
        const int64_t o = pos[c];
        oq[o] = cq[c];
        orow[o] = crow[c];
        od[o] = cdist[c];
    }
}

// ---------------------------------------------------------------- q-gram count filter
//
// A lower bound for edit distance from the counts of the strings' 3-grams
// (Ukkonen 1992, q-gram distance): a substitution changes at most 3 of a
// string's 3-grams and an insertion or deletion at most 2 old and 3 new ones,
// so the L1 distance between the two 3-gram count vectors is at most 6 times
// the edit distance.  Counting the 3-grams in 64 hashed buckets (sums of the
// exact counts) and capping a count at 255 can only lower that L1 distance,
// so L1(buckets) > 6 t proves d > t, and such a pair is not verified.
constexpr int kQgBuckets = 64;

__device__ __forceinline__ uint32_t qgram_bucket(uint32_t a, uint32_t b, uint32_t c) {
    return ((((a << 16) | (b << 8) | c) * 0x9E3779B1u) >> 26) & (kQgBuckets - 1);
}

// thread per string: its 64 bucket counts (saturating at 255)
__global__ void k_qgram_hist(const uint8_t *__restrict__ S, const int64_t *__restrict__ Soff, int64_t n,
                             uint8_t *__restrict__ out) {
    __shared__ uint8_t hb[256][kQgBuckets];
    uint8_t *h = hb[threadIdx.x];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i - threadIdx.x < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (i >= n) continue;
        for (int b = 0; b < kQgBuckets; ++b) h[b] = 0;
        const uint8_t *s = S + Soff[i];
        const int64_t len = Soff[i + 1] - Soff[i];
        for (int64_t j = 0; j + 2 < len; ++j) {
            const uint32_t b = qgram_bucket(s[j], s[j + 1], s[j + 2]);
            if (h[b] < 255) ++h[b];
        }
        uint32_t *o = reinterpret_cast<uint32_t *>(out + i * kQgBuckets);
        const uint32_t *hw = reinterpret_cast<const uint32_t *>(h);
        for (int w = 0; w < kQgBuckets / 4; ++w) o[w] = hw[w];
    }
}

template <int W, bool KNN>
__global__ void k_verify_str(Dev d, const int32_t *__restrict__ cq, const int32_t *__restrict__ crow, int64_t C,
                             int chunk, const float *__restrict__ thr_q, float *__restrict__ cdist,
                             uint8_t *__restrict__ keep) {
    __shared__ uint64_t Peq[256 * W];
    const int64_t a0 = (int64_t)blockIdx.x * chunk;
    const int64_t a1 = a0 + chunk < C ? a0 + chunk : C;
    int64_t s = a0;
    while (s < a1) {
        const int32_t q = cq[s];
        const int64_t t = lower_bound_i32(cq, s, a1, q + 1);
        const int m = (int)(d.QSoff[q + 1] - d.QSoff[q]);
        if (m > 0) build_peq<W>(Peq, d.QS + d.QSoff[q], m);
        const float r = thr_q[q];
        uint32_t qw[kQgBuckets / 4];
        if (d.qg) {
#pragma unroll
            for (int w = 0; w < kQgBuckets / 4; ++w) qw[w] = reinterpret_cast<const uint32_t *>(d.qgq + (int64_t)q * kQgBuckets)[w];
        }
        for (int64_t c = s + threadIdx.x; c < t; c += blockDim.x) {
            const int64_t row = crow[c];
            if (row >= d.n && !row_visible(d, row, d.qseq[q])) {
                cdist[c] = __int_as_float(0x7f800000);
                keep[c] = 0;
                continue;
            }
            if (d.qg && row < d.n && r < 1e9f) {   // the 3-gram bound: d >= L1 / 6
                const uint4 *ow = reinterpret_cast<const uint4 *>(d.qg + row * kQgBuckets);
                uint32_t l1 = 0;
#pragma unroll
                for (int v = 0; v < kQgBuckets / 16; ++v) {
                    const uint4 o = ow[v];
                    l1 = __vsadu4(qw[4 * v], o.x) + l1;
                    l1 = __vsadu4(qw[4 * v + 1], o.y) + l1;
                    l1 = __vsadu4(qw[4 * v + 2], o.z) + l1;
                    l1 = __vsadu4(qw[4 * v + 3], o.w) + l1;
                }
                if ((float)l1 > 6.f * r) {
                    cdist[c] = __int_as_float(0x7f800000);
                    keep[c] = 0;
                    continue;
                }
            }
            const uint8_t *tx;
            int len;
            srow(d, row, tx, len);
            const float dist = (float)(m > 0 ? myers_edit<W>(Peq, m, tx, len) : len);
            cdist[c] = dist;
            keep[c] = dist <= r ? 1 : 0;   // kNN: r = tau_q, an upper bound of the k-th distance
        }
        __syncthreads();
        s = t;
    }
}

// ---------------------------------------------------------------- kNN merge

__device__ __forceinline__ uint64_t dbits(double x) { return (uint64_t)__double_as_longlong(x); }

// Selection with 8-bit digits (the rank-th smallest as block_select below,
// half the passes): 256 bins, the bin holding the rank found by a block-wide
// prefix sum (blockDim.x == 256).
template <int BITS, class Get>
__device__ uint64_t block_select8(int64_t M, int64_t rank, Get get, unsigned *hist, int64_t *sh) {
    __shared__ unsigned wsum[8];
    uint64_t prefix = 0, pmask = 0;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    for (int shift = BITS - 8; shift >= 0; shift -= 8) {
        hist[t] = 0;
        __syncthreads();
        for (int64_t i = t; i < M; i += blockDim.x) {
            uint64_t v;
            if (get(i, v) && (v & pmask) == prefix) atomicAdd(&hist[(v >> shift) & 255u], 1u);
        }
        __syncthreads();
        const unsigned c = hist[t];
        unsigned incl = c;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        unsigned before = 0;
        for (int w = 0; w < warp; ++w) before += wsum[w];
        const int64_t lo = (int64_t)before + incl - c, hi = (int64_t)before + incl;
        if (c > 0 && lo < rank && rank <= hi) {   // exactly one bin holds the rank
            sh[0] = t;
            sh[1] = rank - lo;
        }
        __syncthreads();
        prefix |= (uint64_t)sh[0] << shift;
        pmask |= 255ull << shift;
        rank = sh[1];
        __syncthreads();
    }
    return prefix;
}

// rank-th smallest (1-based) value among those enumerated by get(i, &v) for
// i in [0, M); values are non-negative keys compared as unsigned integers.
// Whole block; returns the same value in every thread.
template <int BITS, class Get>
__device__ uint64_t block_select(int64_t M, int64_t rank, Get get, unsigned *hist, int64_t *sh) {
    uint64_t prefix = 0, pmask = 0;
    for (int shift = BITS - 4; shift >= 0; shift -= 4) {
        if (threadIdx.x < 16) hist[threadIdx.x] = 0;
        __syncthreads();
        for (int64_t i = threadIdx.x; i < M; i += blockDim.x) {
            uint64_t v;
            if (get(i, v) && (v & pmask) == prefix) atomicAdd(&hist[(v >> shift) & 15u], 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int64_t c = 0, r = sh[1] = rank;
            int sel = 15;
            for (int b = 0; b < 16; ++b) {
                if (c + hist[b] >= r) { sel = b; break; }
                c += hist[b];
            }
            sh[0] = sel;
            sh[1] = r - c;
        }
        __syncthreads();
        prefix |= (uint64_t)sh[0] << shift;
        pmask |= 15ull << shift;
        rank = sh[1];
        __syncthreads();
    }
    return prefix;
}

__device__ __forceinline__ int64_t block_sum(int64_t v, int64_t *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    int64_t t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    __syncthreads();
    return t;
}

// One block per query.  Merges this group's candidates into the query's
// running answer (exact keys: FP64 key for L1/L2, the integer for edit):
//  A. float metrics: U = k-th smallest upper bound over the answer so far and
//     the candidates' FP32 intervals; only candidates whose lower bound is
//     <= U can reach the top k, and only those get an FP64 key;
//  B. the k-th smallest exact (key, id) over answer + kept candidates, ties
//     to the smaller id, gives exactly min(k, total) survivors, which are
//     sorted and written back as the new answer.
// PASS 0 (L1 / L2): step A; the candidates that need an FP64 key are listed
// in rlist and get it from k_recheck_keys (a thread per candidate: the
// sequential FP64 sums then keep every lane of the FP64 pipe busy).  PASS 1:
// step B (and, for edit distance, the keys from the exact distances).
// Warp-per-query forms of the two selection steps of k_knn_merge for k <= 32
// (a block per query spends most of its time in barriers at these sizes).
//  Step A: U = the k-th smallest upper bound over answer + candidates (k
//  rounds at most: the smallest value above the last one and its
//  multiplicity), then every candidate whose lower bound is <= U is listed
//  for its FP64 key -- the same U and the same list as the block form.
constexpr int kBoundStage = 1024;   // candidate bounds a warp stages in shared memory

template <int METRIC>
__global__ void __launch_bounds__(256) k_knn_bound_warp(Dev d, const int64_t *__restrict__ qoff,
                                                        const float *__restrict__ cdist, int64_t C,
                                                        const int32_t *__restrict__ kq,
                                                        const int64_t *__restrict__ koff,
                                                        const double *__restrict__ bd,
                                                        const int32_t *__restrict__ bn, double *__restrict__ ckey,
                                                        int64_t *__restrict__ rlist,
                                                        unsigned long long *__restrict__ rcount,
                                                        const float *__restrict__ chi, int64_t nq) {
    __shared__ uint32_t sx[8][kBoundStage];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t q = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (q >= nq) return;
    const int64_t a = qoff[q], b = qoff[q + 1];
    if (a == b) return;
    const int64_t M = b - a;
    const int K = kq[q];
    const int nb = bn[q];
    const float up = 1.f + 2.f * d.rel, dn = 1.f - 2.f * d.rel;
    // upper bounds as float bits (x >= +0: bit order is value order)
    auto cand_bits = [&](int64_t i) -> uint32_t {
        return __float_as_uint(chi ? chi[a + i] + d.absf : cdist[a + i] * up + d.absf);
    };
    uint32_t U = 0x7f800000u;
    if ((int64_t)nb + M > K) {
        // the answer's bounds, one per lane (nb <= k <= 32), formed once
        uint32_t ans = 0xffffffffu;
        if (lane < nb) {
            const double v = bd[koff[q] + lane];
            const double ex = d.cosine ? __dsqrt_ru(__dmul_ru(2.0, v)) : (METRIC == GTS_L2 ? __dsqrt_rn(v) : v);
            ans = __float_as_uint(__double2float_ru(ex) + (d.cosine ? d.absf : 0.f));
        }
        // U' = the k-th smallest of the 32 lane minima: a subset's k-th
        // smallest, so U' >= U, and every value <= U is <= U'.  Only those
        // are staged (a few dozen, typically); the exact rounds run on them.
        uint32_t lmin = lane < nb ? ans : 0xffffffffu;
        for (int64_t i = lane; i < M; i += 32) lmin = min(lmin, cand_bits(i));
        uint32_t srt = lmin;   // ascending across lanes (bitonic)
        for (int k2 = 2; k2 <= 32; k2 <<= 1)
            for (int j = k2 >> 1; j > 0; j >>= 1) {
                const uint32_t o = __shfl_xor_sync(0xffffffffu, srt, j);
                const bool lower = (lane & j) == 0, asc = (lane & k2) == 0;
                srt = lower == asc ? min(srt, o) : max(srt, o);
            }
        const uint32_t Up = __shfl_sync(0xffffffffu, srt, K - 1);
        int ns = 0;   // values <= U' staged
        {
            const bool keep = lane < nb && ans <= Up;
            const unsigned bal = __ballot_sync(0xffffffffu, keep);
            if (keep) sx[w][__popc(bal & ((1u << lane) - 1u))] = ans;
            ns = __popc(bal);
        }
        for (int64_t i0 = 0; i0 < M; i0 += 32) {
            const int64_t i = i0 + lane;
            const uint32_t x = i < M ? cand_bits(i) : 0xffffffffu;
            const bool keep = i < M && x <= Up;
            const unsigned bal = __ballot_sync(0xffffffffu, keep);
            const int slot = ns + __popc(bal & ((1u << lane) - 1u));
            if (keep && slot < kBoundStage) sx[w][slot] = x;
            ns += __popc(bal);
        }
        __syncwarp();
        const bool staged = ns <= kBoundStage;
        // the k-th smallest over the staged values (or, past the stage's
        // capacity, over every value): k rounds at most, each the smallest
        // value above the last one and its multiplicity
        int remaining = K;
        bool first = true;
        uint32_t prev = 0;
        for (;;) {
            uint32_t mn = 0xffffffffu;
            if (staged) {
                for (int i = lane; i < ns; i += 32) {
                    const uint32_t x = sx[w][i];
                    if ((first || x > prev) && x < mn) mn = x;
                }
            } else {
                if (lane < nb && (first || ans > prev)) mn = ans;
                for (int64_t i = lane; i < M; i += 32) {
                    const uint32_t x = cand_bits(i);
                    if ((first || x > prev) && x < mn) mn = x;
                }
            }
            mn = __reduce_min_sync(0xffffffffu, mn);
            if (mn == 0xffffffffu) break;
            unsigned cnt = 0;
            if (staged) {
                for (int i = lane; i < ns; i += 32) cnt += sx[w][i] == mn ? 1u : 0u;
            } else {
                cnt = lane < nb && ans == mn ? 1u : 0u;
                for (int64_t i = lane; i < M; i += 32) cnt += cand_bits(i) == mn ? 1u : 0u;
            }
            cnt = __reduce_add_sync(0xffffffffu, cnt);
            if ((int)cnt >= remaining) {
                U = mn;
                break;
            }
            remaining -= (int)cnt;
            prev = mn;
            first = false;
        }
    }
    const float Uf = __uint_as_float(U);
    // the candidates whose lower bound reaches U: counted first, then one
    // atomic per warp reserves their places in the list (a counter that every
    // warp hits once per candidate serialises)
    auto listed = [&](int64_t i) -> bool {
        const float dv = cdist[a + i];
        return (chi ? dv : dv * dn) - d.absf <= Uf && dv != __int_as_float(0x7f800000);
    };
    unsigned cnt = 0;
    for (int64_t i = lane; i < M; i += 32) cnt += listed(i) ? 1u : 0u;
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    unsigned long long base = 0;
    if (lane == 0 && cnt) base = atomicAdd(rcount, (unsigned long long)cnt);
    base = __shfl_sync(0xffffffffu, base, 0);
    for (int64_t i0 = 0; i0 < M; i0 += 32) {
        const int64_t i = i0 + lane;
        const bool l = i < M && listed(i);
        if (i < M) ckey[a + i] = __longlong_as_double(0x7ff0000000000000ll);   // +inf: not a candidate
        const unsigned bal = __ballot_sync(0xffffffffu, l);
        if (l) rlist[base + __popc(bal & ((1u << lane) - 1u))] = a + i;
        base += __popc(bal);
    }
}

//  Step B: the first min(k, finite keys) in (key, id) order over answer +
//  candidates with an FP64 key, when there are at most 64 of them (staged in
//  shared memory, then a warp bitonic sort, two entries per lane); a query
//  with more is flagged in `more` for the block form, untouched.
constexpr int kSelWarpCap = 64;

__device__ __forceinline__ bool key_id_less(uint64_t ka, int64_t ia, uint64_t kb, int64_t ib) {
    return ka < kb || (ka == kb && ia < ib);
}

template <int METRIC>
__global__ void __launch_bounds__(256) k_knn_select_warp(Dev d, const int64_t *__restrict__ qoff,
                                                         const int32_t *__restrict__ crow, int64_t C,
                                                         const int32_t *__restrict__ kq,
                                                         const int64_t *__restrict__ koff, double *__restrict__ bd,
                                                         int64_t *__restrict__ bi, int32_t *__restrict__ bn,
                                                         const double *__restrict__ ckey, int64_t nq,
                                                         uint8_t *__restrict__ more) {
    __shared__ uint64_t sk[8][kSelWarpCap];
    __shared__ int64_t si[8][kSelWarpCap];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t q = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (q >= nq) return;
    if (lane == 0) more[q] = 0;
    const int64_t a = qoff[q], b = qoff[q + 1];
    if (a == b) return;
    const int64_t M = b - a;
    const int K = kq[q];
    const int nb = bn[q];
    double *BD = bd + koff[q];
    int64_t *BI = bi + koff[q];
    const uint64_t INF = 0x7ff0000000000000ull;
    const int64_t n = (int64_t)nb + M;
    int total = 0;
    for (int64_t base = 0; base < n; base += 32) {
        const int64_t i = base + lane;
        uint64_t v = INF;
        if (i < n) v = i < nb ? dbits(BD[i]) : dbits(ckey[a + i - nb]);
        const bool fin = v < INF;
        const unsigned bal = __ballot_sync(0xffffffffu, fin);
        const int slot = total + __popc(bal & ((1u << lane) - 1u));
        if (fin && slot < kSelWarpCap) {
            sk[w][slot] = v;
            si[w][slot] = i < nb ? BI[i] : row_oid(d, crow[a + i - nb]);
        }
        total += __popc(bal);
    }
    if (total > kSelWarpCap) {
        if (lane == 0) more[q] = 1;
        return;
    }
    __syncwarp();
    uint64_t k0 = lane < total ? sk[w][lane] : ~0ull, k1 = lane + 32 < total ? sk[w][lane + 32] : ~0ull;
    int64_t i0 = lane < total ? si[w][lane] : INT64_MAX, i1 = lane + 32 < total ? si[w][lane + 32] : INT64_MAX;
    // bitonic sort of the 64 entries e = lane + 32 r by (key, id), ascending
    for (int k2 = 2; k2 <= 64; k2 <<= 1) {
        for (int j = k2 >> 1; j > 0; j >>= 1) {
            if (j == 32) {   // (only with k2 = 64: ascending) entries lane and lane + 32
                if (key_id_less(k1, i1, k0, i0)) {
                    const uint64_t tk = k0;
                    k0 = k1;
                    k1 = tk;
                    const int64_t ti = i0;
                    i0 = i1;
                    i1 = ti;
                }
                continue;
            }
            const bool lower = (lane & j) == 0;
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                uint64_t &kr = r ? k1 : k0;
                int64_t &ir = r ? i1 : i0;
                const int e = lane + 32 * r;
                const bool asc = (e & k2) == 0;
                const uint64_t pk = __shfl_xor_sync(0xffffffffu, kr, j);
                const int64_t pi = __shfl_xor_sync(0xffffffffu, ir, j);
                const bool take_other = lower == asc ? key_id_less(pk, pi, kr, ir) : key_id_less(kr, ir, pk, pi);
                if (take_other) {
                    kr = pk;
                    ir = pi;
                }
            }
        }
    }
    const int take = total < K ? total : K;   // <= 32: entries 0 .. take - 1 are every lane's first
    if (lane < take) {
        BD[lane] = __longlong_as_double((long long)k0);
        BI[lane] = i0;
    }
    if (lane == 0) bn[q] = take;
}

// Tensor-core tile estimates to distance intervals: from the tile's q.x~,
// d~^2 = (|q|^2 + |x|^2) - 2 q.x~ (the tile's own operation order) is within
// E = cE1 |q||x| + cE2 (|q| + |x|)^2 of d^2 (the tile kernel's bound, taken
// here with 2 cE2), so d lies in [sqrt(d~^2 - E), sqrt(d~^2 + E)], each end
// rounded outwards.  lo overwrites the input.
__global__ void k_tile_intervals(const int32_t *__restrict__ cq, const int32_t *__restrict__ crow, int64_t C,
                                 const float *__restrict__ qn2, const float *__restrict__ xn2, float cE1, float cE2,
                                 float *__restrict__ qxlo, float *__restrict__ hi) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < C; c += (int64_t)gridDim.x * blockDim.x) {
        const float q2 = qn2[cq[c]], x2 = xn2[crow[c]];
        const float qn = __fmul_ru(__fsqrt_ru(q2), 1.f + 1e-6f);
        const float xn = __fmul_ru(__fsqrt_ru(x2), 1.f + 1e-6f);
        const float sn = __fadd_ru(qn, xn);
        const float E = __fadd_ru(__fmul_ru(cE1, __fmul_ru(qn, xn)), __fmul_ru(2.f * cE2, __fmul_ru(sn, sn)));
        const float v = fmaf(-2.f, qxlo[c], q2 + x2);
        hi[c] = __fsqrt_ru(__fadd_ru(v, E));
        const float l = __fsub_rd(v, E);
        qxlo[c] = l > 0.f ? __fsqrt_rd(l) : 0.f;
    }
}

// With chi (tensor-core tiles' kNN pairs, no FP32 verification): candidate
// i's distance lies in [cdist[i], chi[i]] instead of within the FP32 band of
// cdist[i].
template <int METRIC, int PASS>
__global__ void k_knn_merge(Dev d, const int64_t *__restrict__ qoff, const int32_t *__restrict__ crow,
                            const float *__restrict__ cdist, int64_t C, const int32_t *__restrict__ kq,
                            const int64_t *__restrict__ koff, double *__restrict__ bd, int64_t *__restrict__ bi,
                            int32_t *__restrict__ bn, double *__restrict__ ckey, int64_t *__restrict__ rlist,
                            unsigned long long *__restrict__ rcount, const float *__restrict__ chi,
                            const uint8_t *__restrict__ only) {
    __shared__ unsigned hist[256];
    __shared__ int64_t sh[4];
    __shared__ int64_t red[kWarpsPerBlock];
    __shared__ double kk[kKeepCap];
    __shared__ int64_t ki[kKeepCap];
    __shared__ int nkeep;
    const int32_t q = blockIdx.x;
    if (only && !only[q]) return;   // (the warp kernel finished this query)
    const int64_t a = qoff[q], b = qoff[q + 1];
    if (a == b) return;
    const int64_t M = b - a;
    const int K = kq[q];
    const int nb = bn[q];
    double *BD = bd + koff[q];
    int64_t *BI = bi + koff[q];
    constexpr bool FLOAT_METRIC = METRIC != GTS_EDIT;
    const float up = 1.f + 2.f * d.rel, dn = 1.f - 2.f * d.rel;
    // ---- A: candidates that can still enter the top k
    if (FLOAT_METRIC && PASS == 0) {
        uint64_t U = 0x7f800000ull;   // +inf as float bits
        if ((int64_t)nb + M > K) {
            auto get_hi = [&](int64_t i, uint64_t &v) -> bool {
                float x;
                if (i < nb) {
                    // the answer's FP64 key as an upper bound in the kernels' distance
                    // (angular: the chord sqrt(2 key) of the exact unit vectors, plus
                    // the unit-vector rounding)
                    const double ex = d.cosine ? __dsqrt_ru(__dmul_ru(2.0, BD[i]))
                                               : (METRIC == GTS_L2 ? __dsqrt_rn(BD[i]) : BD[i]);
                    x = __double2float_ru(ex) + (d.cosine ? d.absf : 0.f);
                } else {
                    x = chi ? chi[a + i - nb] + d.absf : cdist[a + i - nb] * up + d.absf;
                }
                v = __float_as_uint(x);
                return true;
            };
            U = block_select8<32>((int64_t)nb + M, K, get_hi, hist, sh);
        }
        const float Uf = __uint_as_float((uint32_t)U);
        for (int64_t i = threadIdx.x; i < M; i += blockDim.x) {
            const float dv = cdist[a + i];
            ckey[a + i] = __longlong_as_double(0x7ff0000000000000ll);   // +inf: not a candidate
            if ((chi ? dv : dv * dn) - d.absf <= Uf && dv != __int_as_float(0x7f800000))
                rlist[atomicAdd(rcount, 1ull)] = a + i;   // its FP64 key comes next
        }
        return;
    }
    if (!FLOAT_METRIC) {
        for (int64_t i = threadIdx.x; i < M; i += blockDim.x) {
            const float dv = cdist[a + i];
            ckey[a + i] = dv == __int_as_float(0x7f800000) ? __longlong_as_double(0x7ff0000000000000ll) : (double)dv;
        }
    }
    __syncthreads();
    // ---- B: exact selection over answer-so-far (first nb) and candidates
    const uint64_t INF = 0x7ff0000000000000ull;
    auto get_key = [&](int64_t i, uint64_t &v) -> bool {
        v = i < nb ? dbits(BD[i]) : dbits(ckey[a + i - nb]);
        return v < INF;
    };
    int64_t total = 0;
    for (int64_t i = threadIdx.x; i < (int64_t)nb + M; i += blockDim.x) {
        uint64_t v;
        total += get_key(i, v) ? 1 : 0;
    }
    total = block_sum(total, red);
    const int64_t take = total < K ? total : K;
    if (take == 0) return;
    uint64_t Vk = INF, Ik = 0x7fffffffffffffffull;
    // few exact keys (the common case): stage them all and sort; else select
    // the k-th (key, id) first and stage only those up to it
    if (total > kKeepCap) {
        Vk = block_select<64>((int64_t)nb + M, K, get_key, hist, sh);
        int64_t lt = 0;
        for (int64_t i = threadIdx.x; i < (int64_t)nb + M; i += blockDim.x) {
            uint64_t v;
            if (get_key(i, v) && v < Vk) ++lt;
        }
        lt = block_sum(lt, red);
        auto get_id = [&](int64_t i, uint64_t &v) -> bool {
            uint64_t key;
            if (!get_key(i, key) || key != Vk) return false;
            v = (uint64_t)(i < nb ? BI[i] : row_oid(d, crow[a + i - nb]));
            return true;
        };
        Ik = block_select<32>((int64_t)nb + M, K - lt, get_id, hist, sh);
    }
    if (threadIdx.x == 0) nkeep = 0;
    __syncthreads();
    for (int64_t i = threadIdx.x; i < (int64_t)nb + M; i += blockDim.x) {
        uint64_t v;
        if (!get_key(i, v)) continue;
        const int64_t id = i < nb ? BI[i] : row_oid(d, crow[a + i - nb]);
        if (v < Vk || (v == Vk && (uint64_t)id <= Ik)) {
            const int p = atomicAdd(&nkeep, 1);
            if (p < kKeepCap) {
                kk[p] = __longlong_as_double((long long)v);
                ki[p] = id;
            }
        }
    }
    __syncthreads();
    // bitonic sort of the survivors by (key, id)
    const int staged = nkeep < kKeepCap ? nkeep : kKeepCap;
    int L = 1;
    while (L < take || L < staged) L <<= 1;
    for (int i = threadIdx.x; i < L; i += blockDim.x)
        if (i >= staged) {
            kk[i] = __longlong_as_double(0x7ff0000000000000ll);
            ki[i] = 0x7fffffffffffffffll;
        }
    __syncthreads();
    for (int k2 = 2; k2 <= L; k2 <<= 1) {
        for (int j = k2 >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < L; i += blockDim.x) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const bool asc = (i & k2) == 0;
                    const bool gt = kk[i] > kk[ixj] || (kk[i] == kk[ixj] && ki[i] > ki[ixj]);
                    if (gt == asc) {
                        const double tk = kk[i];
                        kk[i] = kk[ixj];
                        kk[ixj] = tk;
                        const int64_t ti = ki[i];
                        ki[i] = ki[ixj];
                        ki[ixj] = ti;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < take; i += blockDim.x) {
        BD[i] = kk[i];
        BI[i] = ki[i];
    }
    if (threadIdx.x == 0) bn[q] = (int32_t)take;
}

// L1 tiles, range queries: decide the (query, row) pairs the tiles kept from
// their FP32 distance; a pair within the error band of the radius takes the
// FP64 distance in the CPU reference's operation order.
__global__ void k_decide_range_l1(Dev d, const int32_t *__restrict__ cq, const int32_t *__restrict__ crow,
                                  float *__restrict__ cdist, int64_t C, const float *__restrict__ thr_q,
                                  uint8_t *__restrict__ keep, unsigned long long *__restrict__ rechecks) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < C; c += (int64_t)gridDim.x * blockDim.x) {
        const int32_t q = cq[c];
        const float d32 = cdist[c];
        const float r = thr_q[q];
        const float hi = d32 * (1.f + 2.f * d.rel) + d.absf;
        const float lo = d32 * (1.f - 2.f * d.rel) - d.absf;
        if (hi < r * (1.f - 1e-9f)) {
            keep[c] = 1;
        } else if (lo > r * (1.f + 1e-9f)) {
            keep[c] = 0;
        } else {
            const double key = l1_fp64_seq(d.Q + (int64_t)q * d.dim, vrow(d, crow[c]), d.dim);
            keep[c] = key <= (double)r ? 1 : 0;
            cdist[c] = __double2float_rn(key);
            atomicAdd(rechecks, 1ull);
        }
    }
}

__global__ void k_add_u64(const unsigned long long *__restrict__ src, unsigned long long *__restrict__ dst) {
    *dst += *src;
}

// FP64 keys (the CPU reference's operation order) of the listed candidates,
// a thread per candidate
template <int METRIC>
__global__ void k_recheck_keys(Dev d, const int32_t *__restrict__ cq, const int32_t *__restrict__ crow,
                               const int64_t *__restrict__ rlist, const unsigned long long *__restrict__ rcount,
                               double *__restrict__ ckey) {
    const int64_t n = (int64_t)*rcount;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = rlist[i];
        ckey[c] = fp64_key<METRIC == GTS_L2>(d, cq[c], crow[c]);
    }
}

// kNN: once a query's answer so far holds k objects, its k-th FP64 distance
// (rounded up) bounds tau_q from above.
__global__ void k_tau_from_answer(const int32_t *__restrict__ kq, const int64_t *__restrict__ koff,
                                  const double *__restrict__ bd, const int32_t *__restrict__ bn, int64_t nq, int l2,
                                  float *__restrict__ thr) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nq; q += (int64_t)gridDim.x * blockDim.x) {
        const int K = kq[q];
        if (bn[q] < K) continue;
        const double v = bd[koff[q] + K - 1];
        const float t = __double2float_ru(l2 ? __dsqrt_ru(v) : v);
        if (t < thr[q]) thr[q] = t;
    }
}

__global__ void k_pack_row_dist(const int32_t *__restrict__ row, const float *__restrict__ dist, int64_t C,
                                uint64_t *__restrict__ out) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < C; c += (int64_t)gridDim.x * blockDim.x)
        out[c] = ((uint64_t)(uint32_t)row[c] << 32) | (uint64_t)__float_as_uint(dist[c]);
}

__global__ void k_unpack_row_dist(const uint64_t *__restrict__ in, int64_t C, int32_t *__restrict__ row,
                                  float *__restrict__ dist) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < C; c += (int64_t)gridDim.x * blockDim.x) {
        row[c] = (int32_t)(in[c] >> 32);
        dist[c] = __uint_as_float((uint32_t)in[c]);
    }
}

// ---------------------------------------------------------------- dense last level
//
// When the frontier of the last pivot level covers most (query, node) pairs,
// it is kept as matrices instead of an entry list: the child masks of the
// level above, CM[parent][q]; the query-to-pivot distances, DT[node][q]; the
// leaf masks, M[node][q]; and a node x query bitmap of the pairs with a
// surviving leaf.  The tiles read these directly (node-major, 128 queries at
// a time), so no per-entry records are written or regrouped.

__global__ void k_cm_scatter(const int32_t *__restrict__ eq, const int32_t *__restrict__ enode, int64_t e0,
                             int64_t e1, const uint64_t *__restrict__ cmask, int64_t nq, uint64_t *__restrict__ cm) {
    for (int64_t e = e0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < e1; e += (int64_t)gridDim.x * blockDim.x)
        cm[(int64_t)enode[e] * nq + eq[e]] = cmask[e - e0];
}

constexpr int64_t kDenseTcMinPivots = 2048;   // the smallest level whose dense matrix runs on the tensor cores
constexpr int kTauUnroll = 4;   // pivots per lane whose loads k_tau_dense issues together

// member(node, q): the node's bit in its parent's child mask for q
// (node indices of one level fit 32 bits: a 32-bit division, far cheaper than a 64-bit one)
__device__ __forceinline__ bool dense_member(const uint64_t *cm, int64_t node, int64_t q, int64_t nq, int F) {
    const uint32_t nu = (uint32_t)node, par = nu / (uint32_t)F, rem = nu - par * (uint32_t)F;
    return (cm[(int64_t)par * nq + q] >> rem) & 1ull;
}

// kNN threshold from this level's pivots (warp per query; the same candidates
// as k_tau over the entry list: the pivots of the member nodes)
__global__ void k_tau_dense(Dev d, const float *__restrict__ D, int64_t P, const uint64_t *__restrict__ cm,
                            int64_t lvl_base, int64_t nq, const int32_t *__restrict__ kq,
                            const int64_t *__restrict__ koff, double *tk_d, int64_t *tk_id, int32_t *tk_n,
                            float *tau) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const float lab = d.lslack[d.h - 1];   // the last pivot level's absolute slack
    for (int64_t q = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; q < nq; q += nw) {
        const int K = kq[q];
        TauList L;
        L.load(tk_d + koff[q], tk_id + koff[q], tk_n[q], K, lane);
        const int64_t s = d.qseq[q];
        const double up = 1.0 + 2.0 * (double)d.rel;
        // the list's current K-th entry, kept in registers (read again after
        // inserts), and an FP32 distance above which a pivot's bound exceeds
        // it: (double)dv * up + floor <= kth implies dv <= fthr, so the FP64
        // bound is formed only for the few pivots at or below fthr
        double kth = 0.0;
        int64_t kthid = 0;
        float fthr = __int_as_float(0x7f800000);
        auto refresh = [&]() {
            if (L.n >= K) {
                kth = L.kd();
                kthid = L.kid();
                // one float step above the quotient absorbs its FP64 rounding
                fthr = nextafterf(__double2float_ru((kth - (double)d.absf - (double)lab) / up),
                                  __int_as_float(0x7f800000));
            }
        };
        refresh();
        for (int64_t p0 = 0; p0 < P; p0 += 32 * kTauUnroll) {
            // kTauUnroll pivots per lane: their membership and distance loads
            // are issued together, then they are tested in pivot order
            bool mem[kTauUnroll];
            float dv[kTauUnroll];
#pragma unroll
            for (int u = 0; u < kTauUnroll; ++u) {
                const int64_t p = p0 + 32 * u + lane;
                mem[u] = p < P && dense_member(cm, p, q, nq, d.F);
                dv[u] = p < P ? D[q * P + p] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < kTauUnroll; ++u) {
                const int64_t p = p0 + 32 * u + lane;
                bool cand = false;
                double ub = 0.0;
                int64_t id = 0;
                if (mem[u] && dv[u] <= fthr) {
                    ub = (double)dv[u] * up + (double)d.absf + (double)lab;
                    // the bound test first: most pivots fail it, and then the
                    // pivot's delete mark and id are never read
                    if ((L.n < K) || ub <= kth) {
                        const int32_t prow = d.npiv[lvl_base + p];
                        if (prow >= 0 && row_visible(d, prow, s)) {
                            id = d.row_id[prow];
                            cand = (L.n < K) || ub < kth || (ub == kth && id < kthid);
                        }
                    }
                }
                unsigned bal = __ballot_sync(0xffffffffu, cand);
                if (bal) {
                    while (bal) {
                        const int src = __ffs(bal) - 1;
                        bal &= bal - 1;
                        const double uu = __shfl_sync(0xffffffffu, ub, src);
                        const int64_t iid = __shfl_sync(0xffffffffu, id, src);
                        L.insert(uu, iid);
                    }
                    refresh();
                }
            }
        }
        L.store();
        const double k_fin = L.n >= K ? L.kd() : 0.0;
        if (lane == 0) {
            tk_n[q] = L.n;
            tau[q] = L.n >= K ? __double2float_ru(k_fin) : __int_as_float(0x7f800000);
        }
    }
}

// out[c * rows + r] = in[sel(r) * cols + c], sel(r) = rowsel[r] (or r)
__global__ void k_transpose_f32(const float *__restrict__ in, int64_t rows, int64_t cols, float *__restrict__ out,
                                const int32_t *__restrict__ rowsel) {
    __shared__ float tile[32][33];
    const int64_t tr = (int64_t)blockIdx.y * 32, tc = (int64_t)blockIdx.x * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t r = tr + i, c = tc + threadIdx.x;
        tile[i][threadIdx.x] = (r < rows && c < cols) ? in[(rowsel ? (int64_t)rowsel[r] : r) * cols + c] : 0.f;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t c = tc + i, r = tr + threadIdx.x;
        if (r < rows && c < cols) out[c * rows + r] = tile[threadIdx.x][i];
    }
}

// Leaf masks of every member pair (Lemma 1 / 2 on the node's children
// intervals, the same test as the entry kernels), the node x query bitmap of
// the pairs with a surviving leaf, and the counts of member pairs and of
// pairs with a surviving leaf.  Queries are taken in column order: position i
// is query perm[i] (DT, M and the bitmap are in position order).  A block takes one node at a time and all of
// its queries, 256 per step.
// packed FP32 pairs, round to nearest: (a0 + b0, a1 + b1), (a0 - b0, a1 - b1), (a0 b0, a1 b1)
__device__ __forceinline__ float2 add2f(float2 a, float2 b) {
    float2 r;
    asm("{\n\t.reg .b64 x, y, z;\n\tmov.b64 x, {%2, %3};\n\tmov.b64 y, {%4, %5};\n\t"
        "add.rn.f32x2 z, x, y;\n\tmov.b64 {%0, %1}, z;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 sub2f(float2 a, float2 b) {
    float2 r;
    asm("{\n\t.reg .b64 x, y, z;\n\tmov.b64 x, {%2, %3};\n\tmov.b64 y, {%4, %5};\n\t"
        "sub.rn.f32x2 z, x, y;\n\tmov.b64 {%0, %1}, z;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 mul2f(float2 a, float2 b) {
    float2 r;
    asm("{\n\t.reg .b64 x, y, z;\n\tmov.b64 x, {%2, %3};\n\tmov.b64 y, {%4, %5};\n\t"
        "mul.rn.f32x2 z, x, y;\n\tmov.b64 {%0, %1}, z;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}

__global__ void k_leaf_dense(Dev d, const float *__restrict__ DT, const uint64_t *__restrict__ cm, int64_t P,
                             int64_t nq, int64_t lvl_next, const float *__restrict__ thr_q,
                             const int32_t *__restrict__ perm, uint64_t *__restrict__ M,
                             uint32_t *__restrict__ bits, int64_t nw, unsigned long long *__restrict__ counts) {
    // the node's children two at a time: (hi_j, hi_j+1, |hi_j|, |hi_j+1|) and
    // (lo_j, lo_j+1) for j = 2 i; and the mask of the non-empty children
    __shared__ float4 sph[32];
    __shared__ float2 spl[32];
    __shared__ unsigned long long s_ne;
    // the same children in order, for the sorted form (below)
    __shared__ float s_hi[64], s_lo[64];
    __shared__ int s_sorted, s_j0;
    const int lane = threadIdx.x & 31;
    const float epsc = d.epsc;
    unsigned long long nmem = 0, nlive = 0;
    // one node per block iteration, all of its queries: the children are read once
    for (int64_t p = blockIdx.x; p < P; p += gridDim.x) {
        __syncthreads();   // the previous node's children are no longer read
        if (threadIdx.x == 0) s_ne = 0ull;
        __syncthreads();
        if (threadIdx.x < 64) {
            const int j = threadIdx.x;
            float lo = 0.f, hi = 0.f;
            if (j < d.F) {
                const int64_t c = lvl_next + p * d.F + j;
                const bool ne = d.nsize[c] > 0;
                if (ne) {
                    lo = d.nlo[c];
                    hi = d.nhi[c];
                    atomicOr(&s_ne, 1ull << j);
                }
            }
            float *h4 = reinterpret_cast<float *>(&sph[j >> 1]);
            float *l2 = reinterpret_cast<float *>(&spl[j >> 1]);
            h4[j & 1] = hi;
            h4[2 + (j & 1)] = fabsf(hi);
            l2[j & 1] = lo;
            s_hi[j] = hi;
            s_lo[j] = lo;
        }
        __syncthreads();
        const uint64_t nonempty = s_ne;
        // Sorted form: the build cuts a node's rows, in ascending distance to
        // its pivot, into consecutive children, so the non-empty children
        // are a suffix whose [lo, hi] rise with j.  Then the children that
        // pass the test with one eps >= every child's (the one of the largest
        // hi) are the range [ja, jb] found by two binary searches -- a
        // superset of the per-child test's, so no surviving leaf is lost.
        // Checked per node; a node that is not so ordered takes the per-child
        // test.
        if (threadIdx.x < 32) {
            bool bad = false;
            for (int j = threadIdx.x; j + 1 < d.F; j += 32) {
                const bool ne0 = (nonempty >> j) & 1ull, ne1 = (nonempty >> (j + 1)) & 1ull;
                if (ne0 && (!ne1 || s_hi[j] > s_hi[j + 1] || s_lo[j] > s_lo[j + 1] || s_lo[j] < 0.f ||
                            s_hi[j] < s_lo[j]))
                    bad = true;
            }
            bad = __any_sync(0xffffffffu, bad);
            if (threadIdx.x == 0) {
                s_sorted = !bad && nonempty != 0ull && s_hi[d.F - 1] >= s_lo[d.F - 1];
                s_j0 = nonempty ? __ffsll((long long)nonempty) - 1 : d.F;
            }
        }
        __syncthreads();
        const bool sorted = s_sorted != 0;
        const int j0 = s_j0;
        const float himax = s_hi[d.F - 1];
        for (int64_t q0 = 0; q0 < nq; q0 += blockDim.x) {
            const int64_t q = q0 + threadIdx.x;                          // column position
            const int64_t qq = q < nq && perm ? (int64_t)perm[q] : q;    // its query
            const bool member = q < nq && dense_member(cm, p, qq, nq, d.F);
            uint64_t m = 0;
            if (member) {
                const float dq = DT[p * nq + q];
                const float thr = thr_q[qq];
                // interval_hit for two children at a time in packed FP32, its
                // query terms formed once (the same operations in the same
                // order): eps = epsc (sq + |hi|) + the level's absolute slack,
                // keep iff u <= hi + eps and sq + eps >= lo.  A failed test
                // shows as the sign bit of (hi + eps) - u or of (sq + eps) -
                // lo: both differences are rounded once from the exact ones
                // and are never -0 (eps >= +0, so hi + eps and sq + eps are
                // not -0).
                const float u = dq - thr, sq = dq + thr;
                if (sorted) {
                    const float eps = (epsc > 0.f ? epsc * (sq + himax) : 0.f) + d.lslack[d.h - 1];
                    // ja: the first child with (hi + eps) - u >= +0; jb + 1: the
                    // first with (sq + eps) - lo < 0 (sign bits, as below)
                    int a0 = j0, a1 = d.F;
                    while (a0 < a1) {
                        const int mid = (a0 + a1) >> 1;
                        if (__float_as_uint((s_hi[mid] + eps) - u) >> 31) a0 = mid + 1;
                        else a1 = mid;
                    }
                    const int ja = a0;
                    a0 = j0;
                    a1 = d.F;
                    while (a0 < a1) {
                        const int mid = (a0 + a1) >> 1;
                        if (__float_as_uint((sq + eps) - s_lo[mid]) >> 31) a1 = mid;
                        else a0 = mid + 1;
                    }
                    const int jb = a0 - 1;
                    if (ja <= jb)
                        m = ((jb >= 63) ? ~0ull : ((1ull << (jb + 1)) - 1ull)) & ~((1ull << ja) - 1ull) & nonempty;
                } else {
                    const float2 u2 = make_float2(u, u), sq2 = make_float2(sq, sq);
                    const float2 ec2 = make_float2(epsc, epsc);
                    const float2 lab2 = make_float2(d.lslack[d.h - 1], d.lslack[d.h - 1]);
                    uint64_t fail = 0;
#pragma unroll 2
                    for (int j = 0; j < d.F; j += 2) {
                        const float4 h = sph[j >> 1];
                        const float2 lo = spl[j >> 1];
                        const float2 eps = add2f(epsc > 0.f ? mul2f(ec2, add2f(sq2, make_float2(h.z, h.w)))
                                                            : make_float2(0.f, 0.f),
                                                 lab2);
                        const float2 d1 = sub2f(add2f(make_float2(h.x, h.y), eps), u2);
                        const float2 d2 = sub2f(add2f(sq2, eps), lo);
                        const uint32_t f0 = (__float_as_uint(d1.x) | __float_as_uint(d2.x)) >> 31;
                        const uint32_t f1 = (__float_as_uint(d1.y) | __float_as_uint(d2.y)) >> 31;
                        fail |= (uint64_t)(f0 | (f1 << 1)) << j;
                    }
                    m = ~fail & nonempty;
                }
            }
            if (q < nq) M[p * nq + q] = m;
            const unsigned live = __ballot_sync(0xffffffffu, m != 0ull);
            const unsigned mem = __ballot_sync(0xffffffffu, member);
            const int64_t w = (q - lane) >> 5;   // the warp's word
            if (lane == 0 && w < nw) bits[p * nw + w] = live;
            if (lane == 0) {
                nmem += __popc(mem);
                nlive += __popc(live);
            }
        }
    }
    if (lane == 0) {
        if (nmem) atomicAdd(&counts[0], nmem);
        if (nlive) atomicAdd(&counts[1], nlive);
    }
}

// ---------------------------------------------------------------- results

__global__ void k_range_pack(const int32_t *__restrict__ cq, const int32_t *__restrict__ crow,
                             const float *__restrict__ cdist, const uint8_t *__restrict__ keep, int64_t C,
                             const int64_t *__restrict__ pos, Dev d, uint64_t *__restrict__ rkey,
                             float *__restrict__ rdist) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < C; c += (int64_t)gridDim.x * blockDim.x) {
        if (!keep[c]) continue;
        const int64_t o = pos[c];
        rkey[o] = ((uint64_t)(uint32_t)cq[c] << 32) | (uint64_t)(uint32_t)row_oid(d, crow[c]);
        rdist[o] = cdist[c];
    }
}

__global__ void k_iota_i32(int32_t *a, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = (int32_t)i;
}

__global__ void k_u8_to_i64(const uint8_t *a, int64_t n, int64_t *b) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = a[i];
    if (blockIdx.x == 0 && threadIdx.x == 0) b[n] = 0;
}

// Range answer keys (query << 32 | id), as the kernels emit them, repacked
// to (query << idbits | id) with every id < 2^idbits, so that the sort by
// (query, id) runs over the bits in use only.
__global__ void k_repack_keys(const uint64_t *__restrict__ in, int64_t n, int idbits, uint64_t *__restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = in[i];
        out[i] = ((k >> 32) << idbits) | (k & 0xffffffffull);
    }
}

// Range answers sorted by (query << idbits | id): query q's answers start at
// the first key >= q << idbits (a binary search per query, no atomics), and
// each answer's id is the key's low idbits bits.
__global__ void k_range_offsets(const uint64_t *__restrict__ rkey, int64_t R, int64_t nq, int idbits,
                                int64_t *__restrict__ offsets) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q <= nq; q += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t x = (uint64_t)q << idbits;
        int64_t a = 0, b = R;
        while (a < b) {
            const int64_t m = (a + b) >> 1;
            if (rkey[m] < x) a = m + 1;
            else b = m;
        }
        offsets[q] = a;
    }
}

__global__ void k_range_ids(const uint64_t *__restrict__ rkey, int64_t R, int idbits, int64_t *__restrict__ ids) {
    const uint64_t mask = (1ull << idbits) - 1ull;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < R; i += (int64_t)gridDim.x * blockDim.x)
        ids[i] = (int64_t)(rkey[i] & mask);
}

__global__ void k_knn_counts(const int32_t *bn, int64_t nq, int64_t *counts) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nq; i += (int64_t)gridDim.x * blockDim.x)
        counts[i] = bn[i];
    if (blockIdx.x == 0 && threadIdx.x == 0) counts[nq] = 0;
}

__global__ void k_knn_emit(const int64_t *__restrict__ offsets, const int64_t *__restrict__ koff,
                           const double *__restrict__ bd, const int64_t *__restrict__ bi, const int32_t *__restrict__ bn,
                           int64_t nq, bool l2, bool cosine, int64_t *__restrict__ ids, float *__restrict__ dist,
                           double *__restrict__ keys) {
    const int64_t q = blockIdx.x;
    if (q >= nq) return;
    for (int i = threadIdx.x; i < bn[q]; i += blockDim.x) {
        const double key = bd[koff[q] + i];
        ids[offsets[q] + i] = bi[koff[q] + i];
        dist[offsets[q] + i] = __double2float_rn(cosine ? acos(__dsub_rn(1.0, key)) : (l2 ? __dsqrt_rn(key) : key));
        if (keys) keys[offsets[q] + i] = key;
    }
}

// first entry index at which the running count reaches each group boundary
__global__ void k_group_bounds(const int64_t *__restrict__ off, int64_t E, int64_t G, int64_t total,
                               int64_t *__restrict__ bounds) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g <= G; g += (int64_t)gridDim.x * blockDim.x) {
        if (g == 0) { bounds[0] = 0; continue; }
        if (g == G) { bounds[G] = E; continue; }
        const int64_t target = (total / G) * g;
        int64_t lo = 0, hi = E;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (off[mid] < target) lo = mid + 1;
            else hi = mid;
        }
        bounds[g] = lo;
    }
}

// ---------------------------------------------------------------- host driver

__global__ void k_shift(const int64_t *in, int64_t n, int64_t sub, int64_t *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = in[i] - sub;
}


template <class T>
void exclusive_scan(const T *in, T *out, int64_t n, cudaStream_t st) {
    size_t tb = 0;
    cub::DeviceScan::ExclusiveSum(nullptr, tb, in, out, n, st);
    DBuf<uint8_t> tmp(tb ? tb : 1, st);
    GTS_CUDA(cub::DeviceScan::ExclusiveSum(tmp.get(), tb, in, out, n, st));
}

__global__ void k_i32_to_i64(const int32_t *a, int64_t n, int64_t *b) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = a[i];
    if (blockIdx.x == 0 && threadIdx.x == 0) b[n] = 0;
}

int64_t d2h_i64(const int64_t *p, cudaStream_t st) {
    int64_t v = 0;
    GTS_CUDA(cudaMemcpyAsync(&v, p, 8, cudaMemcpyDeviceToHost, st));
    GTS_CUDA(cudaStreamSynchronize(st));
    return v;
}

struct Level {
    int64_t E = 0;
    DBuf<int32_t> q, node;
    DBuf<float> path;
};

// Per-stage device time: CUDA events recorded on the query stream around
// every launch of a stage (only when the caller asks for stage times).  The
// events come from a pool owned by the index, so timing costs one record each.
struct StageClock {
    bool on = false;
    cudaStream_t st = nullptr;
    std::vector<cudaEvent_t> *pool = nullptr;
    size_t used = 0;
    struct Rec {
        int stage;
        cudaEvent_t a, b;
    };
    std::vector<Rec> recs;
    int64_t launches[GTS_STAGES] = {0};
    int cur = -1;
    cudaEvent_t cur_a = nullptr;
    cudaEvent_t take() {
        if (used == pool->size()) {
            cudaEvent_t e;
            GTS_CUDA(cudaEventCreate(&e));
            pool->push_back(e);
        }
        return (*pool)[used++];
    }
    void begin(int stage, int nlaunch = 1) {
        launches[stage] += nlaunch;
        if (!on) return;
        cur = stage;
        cur_a = take();
        GTS_CUDA(cudaEventRecord(cur_a, st));
    }
    void end() {
        if (!on) return;
        cudaEvent_t b = take();
        GTS_CUDA(cudaEventRecord(b, st));
        recs.push_back({cur, cur_a, b});
    }
    void collect(double *out) {
        for (int i = 0; i < GTS_STAGES_LEN; ++i) out[i] = 0.0;
        for (auto &r : recs) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) out[r.stage] += ms;
        }
        for (int s = 0; s < GTS_STAGES; ++s) out[GTS_STAGES + s] = (double)launches[s];
    }
    int64_t total_launches() const {
        int64_t t = 0;
        for (int s = 0; s < GTS_STAGES; ++s) t += launches[s];
        return t;
    }
};

// Grid of a grid-stride kernel: at most one wave (SMs x the blocks of this
// kernel that fit on an SM at once), so that no partial second wave runs on
// a few SMs while the rest idle.
template <typename Kern>
unsigned wave_grid(Kern kern, int64_t blocks, int threads) {
    static std::mutex mu;
    static std::unordered_map<const void *, int> per_sm_of;
    int dev = 0, sms = 0, per_sm = 0;
    GTS_CUDA(cudaGetDevice(&dev));
    GTS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    {
        std::lock_guard<std::mutex> g(mu);
        auto it = per_sm_of.find(reinterpret_cast<const void *>(kern));
        if (it != per_sm_of.end()) {
            per_sm = it->second;
        } else {
            GTS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0));
            if (per_sm < 1) per_sm = 1;
            per_sm_of[reinterpret_cast<const void *>(kern)] = per_sm;
        }
    }
    const int64_t cap = (int64_t)sms * per_sm;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(blocks, cap));
}

struct Runner {
    gts_index *ix;
    const QueryBatch &qb;
    bool knn;
    int64_t budget;
    cudaStream_t st;
    Dev d;
    int h, F, W;
    DBuf<float> thr;
    // kNN state
    DBuf<int64_t> koff;
    DBuf<double> tk_d, bd;
    DBuf<int64_t> tk_id, bi;
    DBuf<int32_t> tk_n, bn;
    // range results, appended per group
    std::vector<DBuf<uint64_t>> rkeys;
    std::vector<DBuf<float>> rdists;
    std::vector<int64_t> rcounts;
    DBuf<unsigned long long> counters;   // [0] rechecks, [1] scanned rows
    int64_t st_pivots = 0, st_frontier = 0, st_cands = 0, st_groups = 0, st_cache = 0;
    int64_t st_tiles = 0, st_tile_entries = 0, st_table_pass = 0;
    int64_t st_scan_rows = 0, st_scan_records = 0;   // node-major scan: table rows read, records tested
    StageClock clk;
    bool use_tc = false;   // BF16 tensor-core tiles at the last level (L2)
    bool use_l1 = false;   // FP32 CUDA-core tiles at the last level (L1)
    bool use_qg = false;   // 3-gram filtering tiles at the last level (edit distance)
    bool use_scan = false; // low-dim vectors: node-major table scan + CUDA-core verification
    Tuning tu;             // launch parameters (a copy of the index's)
    // dense query-to-pivot matrices per level (tile paths): state 0 undecided, 1 ready, 2 not used
    std::vector<DBuf<float>> dense;
    std::vector<int> dense_state;
    int64_t st_tile_pairs = 0, st_dense_pairs = 0;
    bool whole_batch = true;   // no level has been split into groups so far
    int64_t st_dense_last = 0;
    DBuf<uint8_t> tcQh, tcQl;   // the batch's queries as split bf16 rows (tensor-core path)
    DBuf<float> tcqn2;
    DBuf<int32_t> qkey;         // kNN: the probe's last-level node per query (qkey_ok once written)
    bool qkey_ok = false;
    DBuf<unsigned long long> tp_count;   // diagnostics: [0] pairs passing the table bound, [1] scratch

    Runner(gts_index *i, const QueryBatch &b, bool k, int64_t bud, cudaStream_t s)
        : ix(i), qb(b), knn(k), budget(bud), st(s) {
        clk.st = s;
        clk.pool = &i->events;
    }

    unsigned max_blocks = 152 * 8;   // grid cap for the grid-stride kernels (set from the SM count)
    unsigned cap(unsigned b) const { return b < max_blocks ? b : max_blocks; }

    int64_t limit_bytes(int l) const {   // Algorithm 4: size_GPU / ((h - layer + 1) * N_c), layer = l + 1
        return budget / ((int64_t)(h - l) * F);
    }

    void scan_i32(const DBuf<int32_t> &cnt, int64_t E, DBuf<int64_t> &off) {
        DBuf<int64_t> c64(E + 1, st);
        off.alloc(E + 1, st);
        clk.begin(GTS_STAGE_OTHER, 2);
        k_i32_to_i64<<<nblocks(E, kT), kT, 0, st>>>(cnt.get(), E, c64.get());
        exclusive_scan(c64.get(), off.get(), E + 1, st);
        clk.end();
    }

    // Level l's query-to-pivot matrix: on the tensor cores when the batch
    // runs the BF16 tiles (with the level's absolute slack), else in FP32.
    void level_matrix(int l, float *out) {
        const int64_t P = ix->tree.lvl_off[l + 1] - ix->tree.lvl_off[l];
        clk.begin(GTS_STAGE_PIVOT_DIST);
        // (levels of fewer than kDenseTcMinPivots pivots: the FP32 kernel, which
        // needs no host round trip for the slack and is as fast at that size)
        if (use_tc && P >= kDenseTcMinPivots && tc_dense_supported(ix->tree, ix->tree.tc) &&
            ix->tree.tc.piv_ready) {
            d.lslack[l] = tc_dense_dist(ix->tree, ix->tree.tc, l, (const __nv_bfloat16 *)tcQh.get(),
                                        (const __nv_bfloat16 *)tcQl.get(), tcqn2.get(), d.Q, qb.nq, out, st);
        } else {
            dense_pivot_dist(d.metric, d.X, d.dim, d.Q, qb.nq, d.npiv + ix->tree.lvl_off[l], P, out, st);
        }
        clk.end();
    }

    // The level's dense distance matrix, computed on the first group that
    // reaches the level if its frontier holds at least a quarter of the
    // batch's (query, node) pairs and the matrix fits an eighth of the budget.
    const float *dense_for(int l, int64_t E) {
        if (!(use_tc || use_l1 || use_scan) || d.dim == 0) return nullptr;
        if ((int)dense_state.size() < h) {
            dense_state.assign(h, 0);
            dense.resize(h);
        }
        if (dense_state[l] == 1) return dense[l].get();
        if (dense_state[l] == 2) return nullptr;
        const int64_t P = ix->tree.lvl_off[l + 1] - ix->tree.lvl_off[l];
        const int64_t pairs = qb.nq * P;
        dense_state[l] = 2;
        if (!dense_supported(d.metric, d.dim, d.X, d.Q) || 4 * E < pairs || pairs * 4 > budget / 8) return nullptr;
        dense[l].alloc(pairs, st);
        level_matrix(l, dense[l].get());
        st_dense_pairs += pairs;
        dense_state[l] = 1;
        return dense[l].get();
    }

    void pivdist(Level &L, int64_t e0, int64_t e1, int l) {
        if (e1 <= e0) return;
        if (const float *dm = dense_for(l, e1 - e0)) {
            const int64_t P = ix->tree.lvl_off[l + 1] - ix->tree.lvl_off[l];
            clk.begin(GTS_STAGE_PIVOT_DIST);
            k_pivdist_lookup<<<cap(nblocks(e1 - e0, kT)), kT, 0, st>>>(L.q.get(), L.node.get(), e0, e1, dm, P,
                                                                        L.path.get(), h, l);
            clk.end();
            check_launch("pivot distance lookup");
            st_pivots += e1 - e0;
            st_frontier += e1 - e0;
            if (knn) {
                const int64_t base = ix->tree.lvl_off[l];
                clk.begin(GTS_STAGE_THRESHOLD);
                k_tau<<<cap(nblocks(qb.nq, kWarpsPerBlock)), kT, 0, st>>>(d, query_runs(L, e0, e1), L.node.get(), base,
                                                                          e0, e1,
                                                                          L.path.get(), l, qb.nq, qb.k, koff.get(),
                                                                          tk_d.get(), tk_id.get(), tk_n.get(),
                                                                          thr.get());
                clk.end();
                check_launch("knn threshold");
            }
            return;
        }
        const int64_t base = ix->tree.lvl_off[l];
        const int64_t E = e1 - e0;
        clk.begin(GTS_STAGE_PIVOT_DIST);
        if (d.dim > 0) {
            const bool aligned = ((uintptr_t)d.Q & 15) == 0;
            const int nv = (aligned && d.dim % 128 == 0 && d.dim <= 512) ? d.dim / 128 : 0;
            const unsigned grid = cap(nblocks((E + kPivGroup - 1) / kPivGroup, kWarpsPerBlock));
#define GTS_PV(L2V, NVV) \
    k_pivdist_vec<L2V, NVV><<<grid, kT, 0, st>>>(d, L.q.get(), L.node.get(), base, e0, e1, L.path.get(), l)
            if (d.metric == GTS_L2) {
                switch (nv) { case 1: GTS_PV(true, 1); break; case 2: GTS_PV(true, 2); break;
                              case 3: GTS_PV(true, 3); break; case 4: GTS_PV(true, 4); break;
                              default: GTS_PV(true, 0); }
            } else {
                switch (nv) { case 1: GTS_PV(false, 1); break; case 2: GTS_PV(false, 2); break;
                              case 3: GTS_PV(false, 3); break; case 4: GTS_PV(false, 4); break;
                              default: GTS_PV(false, 0); }
            }
#undef GTS_PV
        } else {
            const int chunk = tu.str_chunk;
#define GTS_PIV(WW)                                                                                                  \
    k_pivdist_str<WW><<<nblocks(E, chunk), 128, 0, st>>>(d, L.q.get(), L.node.get(), base, e0, e1, chunk, L.path.get(), \
                                                         l)
            if (W <= 1) GTS_PIV(1);
            else if (W <= 2) GTS_PIV(2);
            else if (W <= 4) GTS_PIV(4);
            else if (W <= 8) GTS_PIV(8);
            else GTS_PIV(16);
#undef GTS_PIV
        }
        clk.end();
        check_launch("pivot distances");
        st_pivots += E;
        st_frontier += E;
        if (knn) {
            clk.begin(GTS_STAGE_THRESHOLD);
            k_tau<<<cap(nblocks(qb.nq, kWarpsPerBlock)), kT, 0, st>>>(d, query_runs(L, e0, e1), L.node.get(), base,
                                                                          e0, e1, L.path.get(),
                                                                 l, qb.nq, qb.k, koff.get(), tk_d.get(), tk_id.get(),
                                                                 tk_n.get(), thr.get());
            clk.end();
            check_launch("knn threshold");
        }
    }

    // split [0, E) into groups whose cumulative counts stay near the limit
    std::vector<int64_t> groups(const DBuf<int64_t> &off, int64_t E, int64_t total, int64_t limit_items) {
        int64_t G = limit_items > 0 ? (total + limit_items - 1) / limit_items : total;
        if (G < 1) G = 1;
        if (G > E) G = E > 0 ? E : 1;
        std::vector<int64_t> b(G + 1);
        if (G == 1) {
            b[0] = 0;
            b[1] = E;
            return b;
        }
        DBuf<int64_t> db(G + 1, st);
        clk.begin(GTS_STAGE_OTHER);
        k_group_bounds<<<nblocks(G + 1, kT), kT, 0, st>>>(off.get(), E, G, total, db.get());
        clk.end();
        GTS_CUDA(cudaMemcpyAsync(b.data(), db.get(), (G + 1) * 8, cudaMemcpyDeviceToHost, st));
        GTS_CUDA(cudaStreamSynchronize(st));
        std::vector<int64_t> out;
        out.push_back(0);
        for (int64_t g = 1; g <= G; ++g)
            if (b[g] > out.back()) out.push_back(b[g]);
        if (out.back() != E) out.push_back(E);
        return out;
    }

    void group_range(const DBuf<int64_t> &off, int64_t g0, int64_t g1, int64_t &o0, int64_t &o1,
                     DBuf<int64_t> &offg) {
        GTS_CUDA(cudaMemcpyAsync(&o0, off.get() + g0, 8, cudaMemcpyDeviceToHost, st));
        GTS_CUDA(cudaMemcpyAsync(&o1, off.get() + g1, 8, cudaMemcpyDeviceToHost, st));
        GTS_CUDA(cudaStreamSynchronize(st));
        offg.alloc(g1 - g0 + 1, st);
        clk.begin(GTS_STAGE_OTHER);
        k_shift<<<nblocks(g1 - g0 + 1, kT), kT, 0, st>>>(off.get() + g0, g1 - g0 + 1, o0, offg.get());
        clk.end();
    }

    void process(Level &L, int64_t e0, int64_t e1, int l) {
        if (e1 <= e0) return;
        if ((use_tc || use_l1 || use_scan) && l == h - 1) {
            last_level_tc(L, e0, e1, l);
            return;
        }
        pivdist(L, e0, e1, l);
        const int64_t E = e1 - e0;
        const int64_t lvl_next = ix->tree.lvl_off[l + 1];
        if (l < h - 1) {
            DBuf<int32_t> cnt(E, st);
            DBuf<uint64_t> cmask(E, st);
            clk.begin(GTS_STAGE_EXPAND);
            k_expand<0><<<wave_grid(k_expand<0>, nblocks((E + 31) / 32, kWarpsPerBlock), kT), kT, 0, st>>>(d, L.q.get(), L.node.get(), L.path.get(), l,
                                                                   lvl_next, e0, e1, thr.get(), cnt.get(), nullptr,
                                                                   nullptr, nullptr, nullptr, cmask.get());
            clk.end();
            check_launch("expand count");
            DBuf<int64_t> off;
            scan_i32(cnt, E, off);
            const int64_t total = d2h_i64(off.get() + E, st);
            if (use_tc && l == h - 2 && dense_last_ok(total)) {
                dense_last_level(L, e0, e1, cmask);
                return;
            }
            const int64_t entry_bytes = 8 + 4 * (int64_t)h;
            auto gb = groups(off, E, total, limit_bytes(l) / entry_bytes);
            if (gb.size() > 2) {
                st_groups += (int64_t)gb.size() - 1;
                whole_batch = false;
            }
            for (size_t g = 0; g + 1 < gb.size(); ++g) {
                const int64_t g0 = gb[g], g1 = gb[g + 1];
                int64_t o0 = 0, o1 = 0;
                DBuf<int64_t> offg;
                group_range(off, g0, g1, o0, o1, offg);
                Level N;
                N.E = o1 - o0;
                if (N.E == 0) continue;
                N.q.alloc(N.E, st);
                N.node.alloc(N.E, st);
                N.path.alloc(N.E * h, st);
                clk.begin(GTS_STAGE_EXPAND);
                k_expand<1><<<cap(nblocks(g1 - g0, kWarpsPerBlock)), kT, 0, st>>>(
                    d, L.q.get(), L.node.get(), L.path.get(), l, lvl_next, e0 + g0, e0 + g1, thr.get(), nullptr,
                    offg.get(), N.q.get(), N.node.get(), N.path.get(), cmask.get() + g0);
                clk.end();
                check_launch("expand write");
                process(N, 0, N.E, l + 1);
            }
        } else {
            DBuf<uint64_t> mask(E, st);
            clk.begin(GTS_STAGE_EXPAND);
            k_expand<2><<<wave_grid(k_expand<2>, nblocks((E + 31) / 32, kWarpsPerBlock), kT), kT, 0, st>>>(d, L.q.get(), L.node.get(), L.path.get(), l,
                                                                   lvl_next, e0, e1, thr.get(), nullptr, nullptr,
                                                                   nullptr, nullptr, nullptr, mask.get());
            clk.end();
            if (use_tc) {
                tc_leaf(L, e0, e1, mask);
                return;
            }
            if (use_qg) {
                count_table_pass(L, e0, e1, mask);
                str_leaf(L, e0, e1, mask);
                return;
            }
            DBuf<int32_t> cnt(E, st);
            const int64_t lvl_last = ix->tree.lvl_off[h - 1];
            clk.begin(GTS_STAGE_LEAF_SCAN);
            k_leafscan<false><<<nblocks(E, kWarpsPerBlock), kT, 0, st>>>(d, L.q.get(), L.node.get(), L.path.get(),
                                                                         lvl_last, e0, e1, mask.get(), thr.get(),
                                                                         cnt.get(), nullptr, nullptr, nullptr,
                                                                         counters.get() + 1);
            clk.end();
            check_launch("leaf scan count");
            DBuf<int64_t> off;
            scan_i32(cnt, E, off);
            const int64_t total = d2h_i64(off.get() + E, st);
            st_table_pass += total;   // the plain scan's candidates are exactly the pairs passing the bound
            if (total == 0) return;
            const int64_t cand_bytes = 4 + 4 + 4 + 1 + 8 + 16;
            auto gb = groups(off, E, total, (budget / 2) / cand_bytes);
            for (size_t g = 0; g + 1 < gb.size(); ++g) {
                const int64_t g0 = gb[g], g1 = gb[g + 1];
                int64_t o0 = 0, o1 = 0;
                DBuf<int64_t> offg;
                group_range(off, g0, g1, o0, o1, offg);
                const int64_t C = o1 - o0;
                if (C == 0) continue;
                DBuf<int32_t> cq(C, st), crow(C, st);
                clk.begin(GTS_STAGE_LEAF_SCAN);
                k_leafscan<true><<<nblocks(g1 - g0, kWarpsPerBlock), kT, 0, st>>>(
                    d, L.q.get(), L.node.get(), L.path.get(), lvl_last, e0 + g0, e0 + g1, mask.get() + g0, thr.get(),
                    nullptr, offg.get(), cq.get(), crow.get(), nullptr);
                clk.end();
                check_launch("leaf scan write");
                verify_and_collect(cq, crow, C);
                ++st_groups;
            }
        }
    }

    // Last pivot level on the tensor-core path: the fused pass computes the
    // pivot distances, the leaf masks and the per-node counts; the threshold
    // list then takes this level's pivots (kNN); the tiles follow.
    void last_level_tc(Level &L, int64_t e0, int64_t e1, int l) {
        const int64_t E = e1 - e0;
        const int64_t base = ix->tree.lvl_off[l], lvl_next = ix->tree.lvl_off[l + 1];
        const int64_t nn = ix->tree.lvl_off[l + 1] - ix->tree.lvl_off[l];
        DBuf<uint64_t> mask(E, st);
        const bool need_counts = !regroup_uses_bits(ix->tree, qb.nq, E);
        DBuf<int32_t> ncount(need_counts ? nn : 0, st);
        if (need_counts) GTS_CUDA(cudaMemsetAsync(ncount.get(), 0, nn * 4, st));
        const bool aligned = ((uintptr_t)d.Q & 15) == 0;
        const int nv = (aligned && d.dim % 128 == 0 && d.dim <= 512) ? d.dim / 128 : 0;
        const unsigned grid = cap(nblocks((E + kLastGroup - 1) / kLastGroup, kWarpsPerBlock));
        const float *dm = dense_for(l, E);
        // with the distances known up front, this level's pivots lower tau_q
        // before the leaf masks are formed
        const bool tau_first = dm != nullptr && knn;
        if (tau_first) {   // k_tau reads this level's distances from the path
            clk.begin(GTS_STAGE_PIVOT_DIST);
            k_pivdist_lookup<<<cap(nblocks(E, kT)), kT, 0, st>>>(L.q.get(), L.node.get(), e0, e1, dm, nn,
                                                                  L.path.get(), h, l);
            clk.end();
            clk.begin(GTS_STAGE_THRESHOLD);
            k_tau<<<cap(nblocks(qb.nq, kWarpsPerBlock)), kT, 0, st>>>(d, query_runs(L, e0, e1), L.node.get(), base,
                                                                          e0, e1,
                                                                      L.path.get(), l, qb.nq, qb.k, koff.get(),
                                                                      tk_d.get(), tk_id.get(), tk_n.get(), thr.get());
            clk.end();
            check_launch("knn threshold");
        }
        clk.begin(GTS_STAGE_PIVOT_DIST);
#define GTS_LL(L2V, NVV)                                                                                 \
    k_last_level_vec<L2V, NVV><<<grid, kT, 0, st>>>(d, L.q.get(), L.node.get(), base, lvl_next, e0, e1, \
                                                   L.path.get(), l, thr.get(), mask.get(),               \
                                                   need_counts ? ncount.get() : nullptr, dm, nn)
        if (dm && !need_counts) {
            k_leaf_masks_dense<<<cap(nblocks(E, kT)), kT, 0, st>>>(d, L.q.get(), L.node.get(), lvl_next, e0, e1, dm,
                                                                    nn, L.path.get(), l, thr.get(), mask.get());
        } else if (d.metric == GTS_L2) {
            switch (nv) {
                case 1: GTS_LL(true, 1); break;
                case 2: GTS_LL(true, 2); break;
                case 3: GTS_LL(true, 3); break;
                case 4: GTS_LL(true, 4); break;
                default: GTS_LL(true, 0); break;
            }
        } else {
            switch (nv) {
                case 1: GTS_LL(false, 1); break;
                case 2: GTS_LL(false, 2); break;
                case 3: GTS_LL(false, 3); break;
                case 4: GTS_LL(false, 4); break;
                default: GTS_LL(false, 0); break;
            }
        }
#undef GTS_LL
        clk.end();
        check_launch("last level");
        st_pivots += E;
        st_frontier += E;
        if (knn && !tau_first) {
            clk.begin(GTS_STAGE_THRESHOLD);
            k_tau<<<cap(nblocks(qb.nq, kWarpsPerBlock)), kT, 0, st>>>(d, query_runs(L, e0, e1), L.node.get(), base,
                                                                          e0, e1,
                                                                      L.path.get(), l, qb.nq, qb.k, koff.get(),
                                                                      tk_d.get(), tk_id.get(), tk_n.get(), thr.get());
            clk.end();
            check_launch("knn threshold");
        }
        tc_leaf(L, e0, e1, mask, need_counts ? &ncount : nullptr);
    }

    // Last level on the tensor cores: regroup the entries by node, run the
    // tiles (leaf scan + bf16 distance prefilter), then finish the kept pairs
    // with the FP32 distance and its FP64 boundary recheck.
    // The dense last level applies when the whole batch reaches the level
    // above the last in one group, every level so far used dense pivot
    // matrices, the last level's frontier (`total` entries) covers at least a
    // quarter of its (query, node) pairs, and its matrices fit a quarter of
    // the budget.
    bool dense_last_ok(int64_t total) {
        // (window chunks: the tensor-core tiles with dim_p <= 128)
        if (!whole_batch || d.dim == 0 || h < 2 || qb.nq == 0 || qb.nq > 2000000 || ix->tree.tc.dim_p > 128)
            return false;
        if ((int)dense_state.size() < h) return false;
        for (int l = 0; l <= h - 2; ++l)
            if (dense_state[l] != 1) return false;
        if (!dense_supported(d.metric, d.dim, d.X, d.Q)) return false;
        const int64_t P = ix->tree.lvl_off[h] - ix->tree.lvl_off[h - 1];
        const int64_t Pp = ix->tree.lvl_off[h - 1] - ix->tree.lvl_off[h - 2];
        const int64_t pairs = qb.nq * P;
        if (4 * total < pairs) return false;
        const int64_t nw = (qb.nq + 31) / 32;
        const int64_t bytes = pairs * (4 + 4 + 8) + P * nw * 8 + Pp * qb.nq * 8;
        return bytes <= budget / 4;
    }

    void dense_last_level(Level &L, int64_t e0, int64_t e1, DBuf<uint64_t> &cmask) {
        const int ll = h - 1;
        const int64_t nq = qb.nq;
        const int64_t base = ix->tree.lvl_off[ll];
        const int64_t P = ix->tree.lvl_off[h] - base;
        const int64_t Pp = base - ix->tree.lvl_off[ll - 1];
        // kNN: the tiles take the queries in the order of their probe keys, so
        // the windows of consecutive columns hold queries of one region (a
        // node's live columns cluster and whole windows drop out)
        DBuf<int32_t> perm;
        DBuf<uint8_t> pQh, pQl;
        DBuf<float> pqn2;
        if (knn && qkey_ok && nq > 1) {
            clk.begin(GTS_STAGE_OTHER, 5);
            DBuf<int32_t> idx(nq, st), key2(nq, st);
            perm.alloc(nq, st);
            k_iota_i32<<<nblocks(nq, kT), kT, 0, st>>>(idx.get(), nq);
            // keys: last-level node indices in [0, P) (a stable sort keeps
            // equal keys in query order)
            int kbits = 1;
            while (kbits < 31 && ((int64_t)1 << kbits) < P) ++kbits;
            size_t tb = 0;
            cub::DeviceRadixSort::SortPairs(nullptr, tb, qkey.get(), key2.get(), idx.get(), perm.get(), nq, 0, kbits,
                                            st);
            DBuf<uint8_t> tmp(tb > 0 ? tb : 1, st);
            GTS_CUDA(cub::DeviceRadixSort::SortPairs(tmp.get(), tb, qkey.get(), key2.get(), idx.get(), perm.get(), nq,
                                                     0, kbits, st));
            tc_split_queries(d.Q, nq, d.dim, ix->tree.tc.dim_p, pQh, pQl, pqn2, st, perm.get());
            clk.end();
            check_launch("query order");
        }
        // the last level's distances (forced: the frontier is dense), in query
        // order (D) and transposed by position (DT); on the tensor cores both
        // come from the one kernel
        DBuf<float> DT(nq * P, st);
        bool have_dt = false;
        if (dense_state[ll] != 1) {
            dense[ll].alloc(nq * P, st);
            if (use_tc && P >= kDenseTcMinPivots && tc_dense_supported(ix->tree, ix->tree.tc) &&
                ix->tree.tc.piv_ready) {
                clk.begin(GTS_STAGE_PIVOT_DIST);
                d.lslack[ll] = tc_dense_dist(
                    ix->tree, ix->tree.tc, ll, (const __nv_bfloat16 *)(perm.get() ? pQh.get() : tcQh.get()),
                    (const __nv_bfloat16 *)(perm.get() ? pQl.get() : tcQl.get()), perm.get() ? pqn2.get() : tcqn2.get(),
                    d.Q, nq, dense[ll].get(), st, perm.get(), DT.get());
                clk.end();
                have_dt = true;
            } else {
                level_matrix(ll, dense[ll].get());
            }
            st_dense_pairs += nq * P;
            dense_state[ll] = 1;
        }
        const float *D = dense[ll].get();
        st_dense_last = 1;
        DBuf<uint64_t> cm(Pp * nq, st);
        GTS_CUDA(cudaMemsetAsync(cm.get(), 0, Pp * nq * 8, st));
        clk.begin(GTS_STAGE_EXPAND);
        k_cm_scatter<<<cap(nblocks(e1 - e0, kT)), kT, 0, st>>>(L.q.get(), L.node.get(), e0, e1, cmask.get(), nq,
                                                               cm.get());
        clk.end();
        if (knn) {
            clk.begin(GTS_STAGE_THRESHOLD);
            k_tau_dense<<<wave_grid(k_tau_dense, nblocks(nq, kWarpsPerBlock), kT), kT, 0, st>>>(d, D, P, cm.get(), base, nq, qb.k,
                                                                         koff.get(), tk_d.get(), tk_id.get(),
                                                                         tk_n.get(), thr.get());
            clk.end();
            check_launch("dense knn threshold");
        }
        DBuf<uint64_t> M(nq * P, st);
        TcRegroup rg;
        rg.nw = (nq + 31) / 32;
        rg.bits.alloc(P * rg.nw, st);
        GTS_CUDA(cudaMemsetAsync(rg.bits.get(), 0, P * rg.nw * 4, st));
        DBuf<unsigned long long> cnt(2, st);
        GTS_CUDA(cudaMemsetAsync(cnt.get(), 0, 16, st));
        clk.begin(GTS_STAGE_PIVOT_DIST, 2);
        {
            dim3 tb(32, 8), tg((unsigned)((P + 31) / 32), (unsigned)((nq + 31) / 32));
            if (!have_dt) k_transpose_f32<<<tg, tb, 0, st>>>(D, nq, P, DT.get(), perm.get());
            k_leaf_dense<<<wave_grid(k_leaf_dense, P, 256), 256, 0, st>>>(
                d, DT.get(), cm.get(), P, nq, ix->tree.lvl_off[h], thr.get(), perm.get(), M.get(), rg.bits.get(),
                rg.nw, cnt.get());
        }
        clk.end();
        check_launch("dense leaf masks");
        unsigned long long hc[2] = {0, 0};
        GTS_CUDA(cudaMemcpyAsync(hc, cnt.get(), 16, cudaMemcpyDeviceToHost, st));
        GTS_CUDA(cudaStreamSynchronize(st));
        st_pivots += (int64_t)hc[0];
        st_frontier += (int64_t)hc[0];
        clk.begin(GTS_STAGE_OTHER, 6);
        tc_dense_items(ix->tree, nq, M.get(), rg, st);
        clk.end();
        if (qb.count_table_pass) {
            DenseLevels dl;
            for (int l = 0; l < h; ++l) {
                dl.D[l] = dense[l].get();
                dl.P[l] = ix->tree.lvl_off[l + 1] - ix->tree.lvl_off[l];
            }
            k_count_table_pass_dense<<<cap(nblocks(P * nq, kT)), kT, 0, st>>>(
                d, dl, M.get(), perm.get(), P, nq, ix->tree.lvl_off[h], thr.get(), tp_count.get());
            check_launch("dense table-pass count");
        }
        TcQuery tq = tc_query_base();
        if (perm.get()) {
            tq.perm = perm.get();
            tq.Qh = (const __nv_bfloat16 *)pQh.get();
            tq.Ql = (const __nv_bfloat16 *)pQl.get();
        }
        tc_finish(tq, rg);
    }

    // Diagnostics (GTS_QUERY_COUNT_TABLE_PASS): the pairs of the last-level
    // entries [e0, e1) that pass visibility and the table bound, with the
    // thresholds the leaf stage is about to use.
    void count_table_pass(Level &L, int64_t e0, int64_t e1, DBuf<uint64_t> &mask) {
        if (!qb.count_table_pass || e1 <= e0) return;
        const int64_t E = e1 - e0;
        DBuf<int32_t> cnt(E, st);
        k_leafscan<false><<<nblocks(E, kWarpsPerBlock), kT, 0, st>>>(d, L.q.get(), L.node.get(), L.path.get(),
                                                                     ix->tree.lvl_off[h - 1], e0, e1, mask.get(),
                                                                     thr.get(), cnt.get(), nullptr, nullptr, nullptr,
                                                                     tp_count.get() + 1);
        k_sum_i32<<<cap(nblocks(E, kT)), kT, 0, st>>>(cnt.get(), E, tp_count.get());
        check_launch("table-pass count");
    }

    TcQuery tc_query_base() {
        TcQuery tq;
        tq.nq = qb.nq;
        tq.Qh = (const __nv_bfloat16 *)tcQh.get();
        tq.Ql = (const __nv_bfloat16 *)tcQl.get();
        tq.qn2 = tcqn2.get();
        tq.chunk = tu.tc_queries;
        tc_bound_coeffs(ix->tree.tc.dim_p, tq.cE1, tq.cE2);
        tq.Q = d.Q;
        tq.qseq = d.qseq;
        tq.thr = thr.get();
        tq.epsc = d.epsc;
        for (int l = 0; l < kMaxHeight; ++l) tq.lslack[l] = d.lslack[l];
        tq.any_deleted = ix->tree.n_deleted > 0 ? 1 : 0;
        return tq;
    }

    // run the regrouped tiles, then finish the kept pairs with the FP32
    // distance and its FP64 boundary recheck
    void tc_finish(TcQuery &tq, TcRegroup &rg) {
        st_tiles += rg.n_items;
        st_tile_entries += rg.n_entries;
        st_tile_pairs += rg.n_pairs;
        DBuf<int32_t> oq, orow;
        int nl = 0;
        // output capacity: twice the last call's size (per query), at least 1 M
        // pairs; a larger output triggers one relaunch with the exact size
        const int64_t per_q = ix->tc_pairs_hint[knn ? 1 : 0].load();
        const int64_t hint = std::max<int64_t>(1 << 20, 2 * per_q * (qb.nq > 0 ? qb.nq : 1) / 1024);
        // kNN: the tiles also give each kept pair's q.x~, whose proven distance
        // interval stands in for the FP32 distance (the answers' distances
        // come from their FP64 keys), so the pairs skip the FP32 verification
        DBuf<float> od2;
        clk.begin(GTS_STAGE_TILE);
        const int64_t C = tc_run(ix->tree, ix->tree.tc, tq, rg, oq, orow, hint, &nl, st, knn ? &od2 : nullptr);
        clk.end();
        if (rg.n_items > 0 && qb.nq > 0)
            ix->tc_pairs_hint[knn ? 1 : 0].store(std::max<int64_t>(per_q, C * 1024 / qb.nq));
        ++st_groups;
        if (C == 0) return;
        if (knn) {
            st_cands += C;
            knn_from_intervals(oq, orow, od2, C, tq);
            return;
        }
        // verified in the tiles' node-major order (consecutive pairs share
        // their object row); range pairs kept are then sorted by query and id
        verify_and_collect(oq, orow, C, /*query_major=*/false);
    }

    // kNN pairs of the tensor-core tiles with their estimates d~^2: put them
    // in query order, turn each estimate into its distance interval, and
    // merge (FP64 keys for the candidates whose interval reaches the k-th
    // upper bound)
    void knn_from_intervals(DBuf<int32_t> &cq, DBuf<int32_t> &crow, DBuf<float> &cd2, int64_t C, const TcQuery &tq) {
        DBuf<uint64_t> v1(C, st), v2(C, st);
        DBuf<int32_t> q3(C, st), r3(C, st);
        DBuf<float> d3(C, st), hi(C, st);
        int qbits = 1;
        while (((int64_t)1 << qbits) < qb.nq) ++qbits;
        size_t tb = 0;
        cub::DeviceRadixSort::SortPairs(nullptr, tb, cq.get(), q3.get(), v1.get(), v2.get(), C, 0, qbits, st);
        DBuf<uint8_t> tmp(tb ? tb : 1, st);
        clk.begin(GTS_STAGE_OTHER, 4);
        k_pack_row_dist<<<cap(nblocks(C, kT)), kT, 0, st>>>(crow.get(), cd2.get(), C, v1.get());
        GTS_CUDA(cub::DeviceRadixSort::SortPairs(tmp.get(), tb, cq.get(), q3.get(), v1.get(), v2.get(), C, 0, qbits,
                                                 st));
        k_unpack_row_dist<<<cap(nblocks(C, kT)), kT, 0, st>>>(v2.get(), C, r3.get(), d3.get());
        k_tile_intervals<<<cap(nblocks(C, kT)), kT, 0, st>>>(q3.get(), r3.get(), C, tq.qn2, ix->tree.tc.xn2.get(),
                                                            tq.cE1, tq.cE2, d3.get(), hi.get());
        clk.end();
        check_launch("tile intervals");
        merge_knn(q3, r3, d3, C, hi.get());
    }

    void tc_leaf(Level &L, int64_t e0, int64_t e1, DBuf<uint64_t> &mask, DBuf<int32_t> *ncount = nullptr) {
        count_table_pass(L, e0, e1, mask);
        if (use_scan) {
            scan_leaf(L, e0, e1, mask, ncount);
            return;
        }
        if (use_l1) {
            l1_leaf(L, e0, e1, mask, ncount);
            return;
        }
        TcQuery tq = tc_query_base();
        tq.E = e1 - e0;
        tq.eq = L.q.get() + e0;
        tq.enode = L.node.get() + e0;
        tq.path = L.path.get() + e0 * h;
        tq.emask = mask.get();
        TcRegroup rg;
        clk.begin(GTS_STAGE_OTHER, 6);
        tc_regroup(ix->tree, tq, rg, st, ncount ? ncount->get() : nullptr, ix->tree.tc.dim_p <= 128);
        clk.end();
        tc_finish(tq, rg);
    }

    // Last level of low-dimensional vectors: regroup the entries by node, scan
    // each node block's table rows once against all of its queries (leaf
    // mask, visibility, Lemma 1 / 2 lower bound), then verify the candidates
    // with the FP32 distance and its FP64 boundary recheck.
    void scan_leaf(Level &L, int64_t e0, int64_t e1, DBuf<uint64_t> &mask, DBuf<int32_t> *ncount) {
        TcQuery tq;
        tq.E = e1 - e0;
        tq.nq = qb.nq;
        tq.eq = L.q.get() + e0;
        tq.enode = L.node.get() + e0;
        tq.path = L.path.get() + e0 * h;
        tq.emask = mask.get();
        tq.Q = d.Q;
        tq.qseq = d.qseq;
        tq.thr = thr.get();
        tq.epsc = d.epsc;
        tq.any_deleted = ix->tree.n_deleted > 0 ? 1 : 0;
        TcRegroup rg;
        clk.begin(GTS_STAGE_OTHER, 6);
        tc_regroup(ix->tree, tq, rg, st, ncount ? ncount->get() : nullptr, false);
        clk.end();
        st_tiles += rg.n_items;
        st_tile_entries += rg.n_entries;
        const int64_t per_q = ix->scan_pairs_hint[knn ? 1 : 0].load();
        const int64_t hint = std::max<int64_t>(1 << 20, 2 * per_q * (qb.nq > 0 ? qb.nq : 1) / 1024);
        ScanQuery sq;
        sq.epsc = d.epsc;
        sq.any_deleted = tq.any_deleted;
        // range: decide the pairs in the scan (low dimension; the angular
        // distance takes its FP64 key for every pair, so not there)
        sq.fused_range = !knn && !d.cosine;
        sq.Q = d.Q;
        sq.rel = d.rel;
        ScanOut so;
        ScanStats ss;
        clk.begin(GTS_STAGE_LEAF_SCAN);
        scan_run(ix->tree, rg, sq, so, hint, ss, st);
        clk.end();
        clk.launches[GTS_STAGE_LEAF_SCAN] += ss.launches > 1 ? ss.launches - 1 : 0;
        st_scan_rows += ss.staged_rows;
        st_scan_records += ss.records;
        if (rg.n_items > 0 && qb.nq > 0)
            ix->scan_pairs_hint[knn ? 1 : 0].store(std::max<int64_t>(per_q, ss.candidates * 1024 / qb.nq));
        ++st_groups;
        if (sq.fused_range) {
            // the method's candidates are the pairs that passed the table
            // bound; the accepted ones are answers already, the band pairs get
            // their FP64 recheck
            st_cands += ss.candidates - so.n_pairs;
            if (so.n_accepted > 0) {
                rkeys.push_back(std::move(so.key));
                rdists.push_back(std::move(so.dist));
                rcounts.push_back(so.n_accepted);
            }
            if (so.n_pairs > 0) verify_and_collect(so.q, so.row, so.n_pairs, /*query_major=*/false);
            return;
        }
        if (so.n_pairs == 0) return;
        verify_and_collect(so.q, so.row, so.n_pairs, /*query_major=*/false);
    }

    // Last level for strings on the 3-gram tiles: regroup the entries by
    // node, keep the pairs the 3-gram count bound does not exclude, then run
    // the exact bit-parallel DP on those (query-major for its match masks).
    void str_leaf(Level &L, int64_t e0, int64_t e1, DBuf<uint64_t> &mask) {
        TcQuery tq;
        tq.E = e1 - e0;
        tq.nq = qb.nq;
        tq.eq = L.q.get() + e0;
        tq.enode = L.node.get() + e0;
        tq.path = L.path.get() + e0 * h;
        tq.emask = mask.get();
        tq.qseq = d.qseq;
        tq.thr = thr.get();
        tq.any_deleted = ix->tree.n_deleted > 0 ? 1 : 0;
        TcRegroup rg;
        clk.begin(GTS_STAGE_OTHER, 6);
        tc_regroup(ix->tree, tq, rg, st, nullptr, false);
        clk.end();
        st_tiles += rg.n_items;
        st_tile_entries += rg.n_entries;
        st_tile_pairs += rg.n_pairs;
        StrQuery sq;
        sq.qg = d.qg;
        sq.qgq = d.qgq;
        sq.any_deleted = tq.any_deleted;
        sq.queries = tu.str_qgram == 32 ? 32 : 64;
        const int64_t per_q = ix->tc_pairs_hint[knn ? 1 : 0].load();
        const int64_t hint = std::max<int64_t>(1 << 20, 2 * per_q * (qb.nq > 0 ? qb.nq : 1) / 1024);
        DBuf<int32_t> oq, orow;
        int nl = 0;
        clk.begin(GTS_STAGE_TILE);
        const int64_t C = qgram_run(ix->tree, sq, rg, oq, orow, hint, &nl, st);
        clk.end();
        if (rg.n_items > 0 && qb.nq > 0)
            ix->tc_pairs_hint[knn ? 1 : 0].store(std::max<int64_t>(per_q, C * 1024 / qb.nq));
        ++st_groups;
        if (C == 0) return;
        DBuf<int32_t> q2(C, st), r2(C, st);
        int qbits = 1;
        while (((int64_t)1 << qbits) < qb.nq) ++qbits;
        size_t tb = 0;
        cub::DeviceRadixSort::SortPairs(nullptr, tb, oq.get(), q2.get(), orow.get(), r2.get(), C, 0, qbits, st);
        DBuf<uint8_t> tmp(tb ? tb : 1, st);
        clk.begin(GTS_STAGE_OTHER);
        GTS_CUDA(cub::DeviceRadixSort::SortPairs(tmp.get(), tb, oq.get(), q2.get(), orow.get(), r2.get(), C, 0, qbits,
                                                 st));
        clk.end();
        verify_and_collect(q2, r2, C);
    }

    // Last level on the L1 tiles: regroup the entries by node, run the tiles
    // (leaf mask, visibility and FP32 distance with its error band), then
    // decide the kept pairs (range) or merge them into the answer (kNN).  kNN
    // runs the blocks in three phases (1/64, 7/64, 56/64 of them); after each
    // phase the k-th distance of the answer so far lowers tau_q, so the later
    // blocks keep few pairs even where the lower bounds prune nothing.
    void l1_leaf(Level &L, int64_t e0, int64_t e1, DBuf<uint64_t> &mask, DBuf<int32_t> *ncount) {
        TcQuery tq;
        tq.E = e1 - e0;
        tq.nq = qb.nq;
        tq.eq = L.q.get() + e0;
        tq.enode = L.node.get() + e0;
        tq.path = L.path.get() + e0 * h;
        tq.emask = mask.get();
        tq.Q = d.Q;
        tq.qseq = d.qseq;
        tq.thr = thr.get();
        tq.epsc = d.epsc;
        tq.any_deleted = ix->tree.n_deleted > 0 ? 1 : 0;
        TcRegroup rg;
        clk.begin(GTS_STAGE_OTHER, 6);
        tc_regroup(ix->tree, tq, rg, st, ncount ? ncount->get() : nullptr);
        clk.end();
        st_tiles += rg.n_items;
        st_tile_entries += rg.n_entries;
        st_tile_pairs += rg.n_pairs;
        L1Query lq;
        lq.Q = d.Q;
        lq.thr = thr.get();
        lq.knn = knn;
        lq.rel = d.rel;
        lq.any_deleted = tq.any_deleted;
        lq.queries = tu.l1_queries;
        lq.packed = tu.l1_packed != 0;
        std::vector<int64_t> bounds = {0};
        if (knn && tu.knn_phases > 1) {
            const int64_t fr[2] = {tu.knn_phases >= 3 ? 64 : 0, 8};
            for (int64_t f : fr) {
                if (f == 0) continue;
                const int64_t b = rg.n_items / f;
                if (b > bounds.back()) bounds.push_back(b);
            }
        }
        if (rg.n_items > bounds.back()) bounds.push_back(rg.n_items);
        for (size_t p = 0; p + 1 < bounds.size(); ++p) {
            const int slot = knn ? 1 + (int)std::min<size_t>(p, 2) : 0;
            const int64_t per_q = ix->l1_pairs_hint[slot].load();
            const int64_t hint = std::max<int64_t>(1 << 20, 2 * per_q * (qb.nq > 0 ? qb.nq : 1) / 1024);
            DBuf<int32_t> oq, orow;
            DBuf<float> od;
            int nl = 0;
            clk.begin(GTS_STAGE_TILE);
            const int64_t C = l1_run(ix->tree, lq, rg, bounds[p], bounds[p + 1], oq, orow, od, hint, &nl, st);
            clk.end();
            if (qb.nq > 0) ix->l1_pairs_hint[slot].store(std::max<int64_t>(per_q, C * 1024 / qb.nq));
            ++st_groups;
            if (C == 0) continue;
            st_cands += C;
            DBuf<uint8_t> keep(C, st);
            if (knn) {   // the merge wants query-major order
                DBuf<uint64_t> v1(C, st), v2(C, st);
                DBuf<int32_t> q2(C, st), r2(C, st);
                DBuf<float> d2(C, st);
                int qbits = 1;
                while (((int64_t)1 << qbits) < qb.nq) ++qbits;
                size_t tb = 0;
                cub::DeviceRadixSort::SortPairs(nullptr, tb, oq.get(), q2.get(), v1.get(), v2.get(), C, 0, qbits, st);
                DBuf<uint8_t> tmp(tb ? tb : 1, st);
                clk.begin(GTS_STAGE_OTHER, 3);
                k_pack_row_dist<<<cap(nblocks(C, kT)), kT, 0, st>>>(orow.get(), od.get(), C, v1.get());
                GTS_CUDA(cub::DeviceRadixSort::SortPairs(tmp.get(), tb, oq.get(), q2.get(), v1.get(), v2.get(), C, 0,
                                                         qbits, st));
                k_unpack_row_dist<<<cap(nblocks(C, kT)), kT, 0, st>>>(v2.get(), C, r2.get(), d2.get());
                clk.end();
                merge_knn(q2, r2, d2, C);
                clk.begin(GTS_STAGE_THRESHOLD);
                k_tau_from_answer<<<cap(nblocks(qb.nq, kT)), kT, 0, st>>>(qb.k, koff.get(), bd.get(), bn.get(), qb.nq,
                                                                         0, thr.get());
                clk.end();
                check_launch("L1 tau update");
            } else {
                clk.begin(GTS_STAGE_VERIFY);
                k_decide_range_l1<<<cap(nblocks(C, kT)), kT, 0, st>>>(d, oq.get(), orow.get(), od.get(), C, thr.get(),
                                                                      keep.get(), counters.get());
                clk.end();
                check_launch("L1 range decision");
                collect(oq, orow, od, keep, C);
            }
        }
    }

    template <bool L2, bool KNN>
    void launch_verify_vec(const DBuf<int32_t> &cq, const DBuf<int32_t> &crow, int64_t C, DBuf<float> &cdist,
                           DBuf<uint8_t> &keep) {
        if (d.dim <= kScanMaxDim) {   // a thread per pair
            k_verify_lowdim<L2, KNN><<<wave_grid(k_verify_lowdim<L2, KNN>, nblocks(C, kT), kT), kT, 0, st>>>(
                d, cq.get(), crow.get(), C, thr.get(), cdist.get(), keep.get(), counters.get());
            return;
        }
        const int64_t warps = (C + kVerifyGroup - 1) / kVerifyGroup;
        const unsigned grid = cap(nblocks(warps, kWarpsPerBlock));
        const bool aligned = ((uintptr_t)d.Q & 15) == 0;
        const int nv = (aligned && d.dim % 128 == 0 && d.dim <= 512) ? d.dim / 128 : 0;
#define GTS_VV(NVV)                                                                                          \
    k_verify_vec<L2, KNN, NVV><<<wave_grid(k_verify_vec<L2, KNN, NVV>, grid, kT), kT, 0, st>>>(                     \
        d, cq.get(), crow.get(), C, thr.get(), cdist.get(), keep.get(), counters.get())
        switch (nv) {
            case 1: GTS_VV(1); break;
            case 2: GTS_VV(2); break;
            case 3: GTS_VV(3); break;
            case 4: GTS_VV(4); break;
            default: GTS_VV(0); break;
        }
#undef GTS_VV
    }

    // query_major: the pairs come sorted by query (the kNN merge needs that
    // order; otherwise the kept pairs are sorted first; strings must come
    // sorted, the bit-parallel DP keeps one query's match masks per run)
    void verify_and_collect(DBuf<int32_t> &cq, DBuf<int32_t> &crow, int64_t C, bool query_major = true) {
        st_cands += C;
        DBuf<float> cdist(C, st);
        DBuf<uint8_t> keep(C, st);
        clk.begin(GTS_STAGE_VERIFY);
        if (d.dim > 0) {
            if (d.metric == GTS_L2) {
                if (knn) launch_verify_vec<true, true>(cq, crow, C, cdist, keep);
                else launch_verify_vec<true, false>(cq, crow, C, cdist, keep);
            } else {
                if (knn) launch_verify_vec<false, true>(cq, crow, C, cdist, keep);
                else launch_verify_vec<false, false>(cq, crow, C, cdist, keep);
            }
        } else {
            const int chunk = tu.str_chunk;
#define GTS_VER(WW)                                                                                              \
    do {                                                                                                         \
        if (knn)                                                                                                 \
            k_verify_str<WW, true><<<nblocks(C, chunk), 128, 0, st>>>(d, cq.get(), crow.get(), C, chunk,         \
                                                                      thr.get(), cdist.get(), keep.get());       \
        else                                                                                                     \
            k_verify_str<WW, false><<<nblocks(C, chunk), 128, 0, st>>>(d, cq.get(), crow.get(), C, chunk,        \
                                                                       thr.get(), cdist.get(), keep.get());      \
    } while (0)
            if (W <= 1) GTS_VER(1);
            else if (W <= 2) GTS_VER(2);
            else if (W <= 4) GTS_VER(4);
            else if (W <= 8) GTS_VER(8);
            else GTS_VER(16);
#undef GTS_VER
        }
        clk.end();
        check_launch("verify");
        collect(cq, crow, cdist, keep, C, query_major);
    }

    // Keep the pairs flagged in `keep`: range pairs are appended to the
    // answer; kNN pairs are merged into each query's answer so far.
    void collect(DBuf<int32_t> &cq, DBuf<int32_t> &crow, DBuf<float> &cdist, DBuf<uint8_t> &keep, int64_t C,
                 bool query_major = true) {
        DBuf<int64_t> k64(C + 1, st), pos(C + 1, st);
        clk.begin(GTS_STAGE_OTHER, 2);
        k_u8_to_i64<<<nblocks(C, kT), kT, 0, st>>>(keep.get(), C, k64.get());
        exclusive_scan(k64.get(), pos.get(), C + 1, st);
        clk.end();
        const int64_t R = d2h_i64(pos.get() + C, st);
        if (R == 0) return;
        if (knn) {
            // only candidates within tau_q can reach the top k
            DBuf<int32_t> kq2(R, st), krow2(R, st);
            DBuf<float> kd2(R, st);
            clk.begin(GTS_STAGE_OTHER);
            k_compact_cands<<<nblocks(C, kT), kT, 0, st>>>(cq.get(), crow.get(), cdist.get(), keep.get(), C, pos.get(),
                                                           kq2.get(), krow2.get(), kd2.get());
            clk.end();
            if (query_major) {
                merge_knn(kq2, krow2, kd2, R);
            } else {   // stable radix sort by query, (row, distance) carried along
                DBuf<uint64_t> v1(R, st), v2(R, st);
                DBuf<int32_t> q3(R, st), r3(R, st);
                DBuf<float> d3(R, st);
                int qbits = 1;
                while (((int64_t)1 << qbits) < qb.nq) ++qbits;
                size_t tb = 0;
                cub::DeviceRadixSort::SortPairs(nullptr, tb, kq2.get(), q3.get(), v1.get(), v2.get(), R, 0, qbits, st);
                DBuf<uint8_t> tmp(tb ? tb : 1, st);
                clk.begin(GTS_STAGE_OTHER, 3);
                k_pack_row_dist<<<cap(nblocks(R, kT)), kT, 0, st>>>(krow2.get(), kd2.get(), R, v1.get());
                GTS_CUDA(cub::DeviceRadixSort::SortPairs(tmp.get(), tb, kq2.get(), q3.get(), v1.get(), v2.get(), R, 0,
                                                         qbits, st));
                k_unpack_row_dist<<<cap(nblocks(R, kT)), kT, 0, st>>>(v2.get(), R, r3.get(), d3.get());
                clk.end();
                merge_knn(q3, r3, d3, R);
            }
        } else {
            DBuf<uint64_t> rk(R, st);
            DBuf<float> rd(R, st);
            clk.begin(GTS_STAGE_OTHER);
            k_range_pack<<<nblocks(C, kT), kT, 0, st>>>(cq.get(), crow.get(), cdist.get(), keep.get(), C, pos.get(), d,
                                                        rk.get(), rd.get());
            clk.end();
            check_launch("range pack");
            rkeys.push_back(std::move(rk));
            rdists.push_back(std::move(rd));
            rcounts.push_back(R);
        }
    }

    // the first entry of each query's run among entries [e0, e1) of a
    // query-sorted level (relative to e0), for the per-query threshold kernel
    DBuf<int64_t> qrun_buf;
    const int64_t *query_runs(Level &L, int64_t e0, int64_t e1) {
        qrun_buf.alloc(qb.nq + 1, st);
        k_query_runs<<<cap(nblocks(qb.nq + 1, kT)), kT, 0, st>>>(L.q.get() + e0, e1 - e0, qb.nq, qrun_buf.get());
        return qrun_buf.get();
    }

    // merge R query-major (query, row, FP32 distance) candidates into the
    // per-query answers (exact (key, id) selection with FP64 keys)
    void merge_knn(DBuf<int32_t> &kq2, DBuf<int32_t> &krow2, DBuf<float> &kd2, int64_t R,
                   const float *chi = nullptr) {
        DBuf<double> ckey(R, st);
        const unsigned grid = (unsigned)qb.nq;
        DBuf<int64_t> qoff(qb.nq + 1, st);
        clk.begin(GTS_STAGE_SELECT, 5);
        k_query_runs<<<cap(nblocks(qb.nq + 1, kT)), kT, 0, st>>>(kq2.get(), R, qb.nq, qoff.get());
        if (d.metric == GTS_EDIT) {
            k_knn_merge<GTS_EDIT, 1><<<grid, kT, 0, st>>>(d, qoff.get(), krow2.get(), kd2.get(), R, qb.k, koff.get(),
                                                          bd.get(), bi.get(), bn.get(), ckey.get(), nullptr, nullptr,
                                                          nullptr, nullptr);
        } else {
            // step A lists the candidates that need an FP64 key, a thread per
            // candidate computes it, step B selects; the list's length is
            // added to the recheck counter (counters[0])
            DBuf<int64_t> rlist(R, st);
            DBuf<unsigned long long> rc(1, st);
            GTS_CUDA(cudaMemsetAsync(rc.get(), 0, 8, st));
            // k <= 32: a warp per query for both selection steps (step B falls
            // back to the block form for a query with more than 64 keys)
            const bool warp_sel = qb.max_k <= 32;
            const unsigned wgrid = (unsigned)((qb.nq + 7) / 8);
            DBuf<uint8_t> more(warp_sel ? qb.nq : 1, st);
#define GTS_MERGE(MT)                                                                                            \
    do {                                                                                                         \
        if (warp_sel)                                                                                            \
            k_knn_bound_warp<MT><<<wgrid, 256, 0, st>>>(d, qoff.get(), kd2.get(), R, qb.k, koff.get(), bd.get(),  \
                                                        bn.get(), ckey.get(), rlist.get(), rc.get(), chi, qb.nq); \
        else                                                                                                     \
            k_knn_merge<MT, 0><<<grid, kT, 0, st>>>(d, qoff.get(), krow2.get(), kd2.get(), R, qb.k, koff.get(), \
                                                    bd.get(), bi.get(), bn.get(), ckey.get(), rlist.get(),      \
                                                    rc.get(), chi, nullptr);                                     \
        k_recheck_keys<MT><<<cap(nblocks(R, kT)), kT, 0, st>>>(d, kq2.get(), krow2.get(), rlist.get(), rc.get(), \
                                                              ckey.get());                                     \
        if (warp_sel)                                                                                            \
            k_knn_select_warp<MT><<<wgrid, 256, 0, st>>>(d, qoff.get(), krow2.get(), R, qb.k, koff.get(),         \
                                                         bd.get(), bi.get(), bn.get(), ckey.get(), qb.nq,        \
                                                         more.get());                                            \
        k_knn_merge<MT, 1><<<grid, kT, 0, st>>>(d, qoff.get(), krow2.get(), kd2.get(), R, qb.k, koff.get(),     \
                                                bd.get(), bi.get(), bn.get(), ckey.get(), rlist.get(), rc.get(),  \
                                                chi, warp_sel ? more.get() : nullptr);                            \
        k_add_u64<<<1, 1, 0, st>>>(rc.get(), counters.get());                                                   \
    } while (0)
            if (d.metric == GTS_L2) GTS_MERGE(GTS_L2);
            else GTS_MERGE(GTS_L1);
#undef GTS_MERGE
        }
        clk.end();
        check_launch("knn merge");
    }

    void cache_pass() {
        const int64_t cn = ix->cache.count;
        if (cn == 0) return;
        int64_t qchunk = ((budget / 2) / 40) / cn;
        if (qchunk < 1) qchunk = 1;
        // range queries over low-dimensional vectors: verified and kept in
        // one pass (the general path writes every pair as a candidate first)
        const bool fused = !knn && d.dim > 0 && d.dim <= kScanMaxDim;
        for (int64_t qa = 0; qa < qb.nq; qa += qchunk) {
            const int64_t qe = qa + qchunk < qb.nq ? qa + qchunk : qb.nq;
            const int64_t C = (qe - qa) * cn;
            if (fused) {
                st_cache += C;
                DBuf<uint64_t> rk(C, st);
                DBuf<float> rd(C, st);
                DBuf<unsigned long long> kept(1, st);
                GTS_CUDA(cudaMemsetAsync(kept.get(), 0, 8, st));
                clk.begin(GTS_STAGE_VERIFY);
                if (d.metric == GTS_L2)
                    k_cache_range_lowdim<true><<<wave_grid(k_cache_range_lowdim<true>, nblocks(C, kT), kT), kT, 0,
                                                 st>>>(d, qa, qe, cn, thr.get(), rk.get(), rd.get(), kept.get(),
                                                       counters.get());
                else
                    k_cache_range_lowdim<false><<<wave_grid(k_cache_range_lowdim<false>, nblocks(C, kT), kT), kT,
                                                  0, st>>>(d, qa, qe, cn, thr.get(), rk.get(), rd.get(), kept.get(),
                                                           counters.get());
                clk.end();
                check_launch("cache range");
                const int64_t R = d2h_i64(reinterpret_cast<const int64_t *>(kept.get()), st);
                if (R > 0) {
                    rkeys.push_back(std::move(rk));
                    rdists.push_back(std::move(rd));
                    rcounts.push_back(R);
                }
                continue;
            }
            DBuf<int32_t> cq(C, st), crow(C, st);
            clk.begin(GTS_STAGE_OTHER);
            k_cache_cands<<<nblocks(C, kT), kT, 0, st>>>(qa, qe, ix->tree.n, cn, cq.get(), crow.get());
            clk.end();
            st_cache += C;
            verify_and_collect(cq, crow, C);
            st_cands -= C;
        }
    }
};

}  // namespace

void run_query(gts_index *ix, const QueryBatch &qb, bool knn, int precision, int64_t budget, QueryOut &out,
               int64_t *stats, double *stage_ms, cudaStream_t st) {
    Tree &t = ix->tree;
    Cache &c = ix->cache;
    const int64_t nq = qb.nq;
    Runner R(ix, qb, knn, budget, st);
    {
        std::lock_guard<std::mutex> g(ix->tune_mu);
        R.tu = ix->tuning;
    }
    R.clk.on = stage_ms != nullptr;
    {
        int dev = 0, sms = 0;
        GTS_CUDA(cudaGetDevice(&dev));
        GTS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        R.max_blocks = (unsigned)(sms > 0 ? sms : 1) * 8u;
    }
    const bool low_dim = t.dim > 0 && t.dim <= kScanMaxDim && (t.metric == GTS_L1 || t.metric == GTS_L2) &&
                         t.n > 0 && t.n < ((int64_t)1 << 31);
    if (precision == GTS_PREC_BF16 && low_dim) R.use_scan = true;
    if (precision == GTS_PREC_BF16 && !low_dim && l1_tiles_supported(t, qb.Q)) R.use_l1 = true;
    if (precision == GTS_PREC_BF16 && t.dim == 0 && t.n > 0 && t.n < ((int64_t)1 << 31) && R.tu.str_qgram > 0)
        R.use_qg = true;
    if (precision == GTS_PREC_BF16 && !low_dim && tc_supported(t)) {
        {
            std::lock_guard<std::mutex> g(ix->prep_mu);   // concurrent queries build it once
            tc_prepare(t, t.tc, st);
            if (tc_dense_supported(t, t.tc)) tc_prepare_pivots(t, t.tc, st);
        }
        R.use_tc = true;
        R.clk.begin(GTS_STAGE_OTHER);
        tc_split_queries(qb.Q, nq, t.dim, t.tc.dim_p, R.tcQh, R.tcQl, R.tcqn2, st);
        R.clk.end();
    }
    R.h = t.h;
    R.F = t.F;
    R.W = (qb.max_len + 63) / 64;
    if (R.W < 1) R.W = 1;
    Dev &d = R.d;
    d.metric = t.metric;
    d.dim = t.dim;
    d.F = t.F;
    d.h = t.h;
    d.n = t.n;
    d.X = t.X.get();
    d.S = t.S.get();
    d.Soff = t.Soff.get();
    d.row_id = t.row_id.get();
    d.table = t.table.get();
    d.row_del = t.row_del.get();
    d.npos = t.npos.get();
    d.nsize = t.nsize.get();
    d.npiv = t.npiv.get();
    d.nlo = t.nlo.get();
    d.nhi = t.nhi.get();
    d.cn = c.count;
    d.cX = c.X.get();
    d.cS = c.S.get();
    d.cSoff = c.Soff.get();
    d.cid = c.id.get();
    d.cins = c.ins.get();
    d.cdel = c.del.get();
    d.Q = qb.Q;
    d.QS = qb.S;
    d.QSoff = qb.Soff;
    d.rel = t.dim > 0 ? fp32_rel_bound(t.dim) : 0.f;
    d.qg = nullptr;
    d.qgq = nullptr;
    DBuf<uint8_t> qgq;
    if (t.dim == 0 && t.n > 0 && nq > 0) {   // strings: 3-gram counts of the rows (once) and the queries
        R.clk.begin(GTS_STAGE_OTHER, 2);
        {
            std::lock_guard<std::mutex> g(ix->prep_mu);   // concurrent queries build it once
            if (!t.qg_ready) {
                t.qg.alloc(t.n * kQgBuckets, st);
                k_qgram_hist<<<nblocks(t.n, 256), 256, 0, st>>>(t.S.get(), t.Soff.get(), t.n, t.qg.get());
                GTS_CUDA(cudaStreamSynchronize(st));
                t.qg.persist();
                t.qg_ready = true;
            }
        }
        qgq.alloc(nq * kQgBuckets, st);
        k_qgram_hist<<<nblocks(nq, 256), 256, 0, st>>>(qb.S, qb.Soff, nq, qgq.get());
        R.clk.end();
        check_launch("3-gram counts");
        d.qg = t.qg.get();
        d.qgq = qgq.get();
    }
    d.epsc = t.dim > 0 ? 4.f * d.rel : 0.f;
    for (int l = 0; l < kMaxHeight; ++l) d.lslack[l] = 0.f;
    // angular distance: the unit vectors' chords stand within kCosAbsSlack of
    // the exact unit vectors'; a bound crosses between the two twice at most
    d.cosine = t.cosine ? 1 : 0;
    d.absf = t.cosine ? 2.f * kCosAbsSlack : kAbsFloor;
    d.Xr = t.Xr.get();
    d.cXr = c.Xr.get();
    d.Qr = qb.Qr;
    d.coslim = qb.coslim;
    DBuf<int64_t> qseq(nq, st);
    R.clk.begin(GTS_STAGE_OTHER);
    if (qb.seq)
        GTS_CUDA(cudaMemcpyAsync(qseq.get(), qb.seq, nq * 8, cudaMemcpyDeviceToDevice, st));
    else
        k_fill_i64<<<nblocks(nq, kT), kT, 0, st>>>(qseq.get(), nq, qb.seq_now);
    R.clk.end();
    d.qseq = qseq.get();
    R.thr.alloc(nq, st);
    R.counters.alloc(2, st);
    GTS_CUDA(cudaMemsetAsync(R.counters.get(), 0, 16, st));
    if (qb.count_table_pass) {
        R.tp_count.alloc(2, st);
        GTS_CUDA(cudaMemsetAsync(R.tp_count.get(), 0, 16, st));
    }
    if (knn) {
        DBuf<int64_t> k64(nq + 1, st);
        R.koff.alloc(nq + 1, st);
        R.clk.begin(GTS_STAGE_OTHER, 2);
        k_k_to_i64<<<nblocks(nq, kT), kT, 0, st>>>(qb.k, nq, k64.get());
        exclusive_scan(k64.get(), R.koff.get(), nq + 1, st);
        R.clk.end();
        const int64_t ktot = d2h_i64(R.koff.get() + nq, st);
        R.tk_d.alloc(ktot, st);
        R.tk_id.alloc(ktot, st);
        R.bd.alloc(ktot, st);
        R.bi.alloc(ktot, st);
        R.tk_n.alloc(nq, st);
        R.bn.alloc(nq, st);
        R.qkey.alloc(nq, st);
        GTS_CUDA(cudaMemsetAsync(R.tk_n.get(), 0, nq * 4, st));
        GTS_CUDA(cudaMemsetAsync(R.bn.get(), 0, nq * 4, st));
        R.clk.begin(GTS_STAGE_OTHER);
        k_fill_f32<<<nblocks(nq, kT), kT, 0, st>>>(R.thr.get(), nq, INFINITY);
        R.clk.end();
    } else {
        R.clk.begin(GTS_STAGE_OTHER);
        k_thresholds<<<nblocks(nq, kT), kT, 0, st>>>(qb.radii, nq, t.dim == 0, t.cosine ? qb.coslim : nullptr,
                                                      d.absf, R.thr.get());
        R.clk.end();
    }
    check_launch("query setup");
    if (knn && t.n > 0 && nq > 0 && t.dim > 0) {
        LevelOffsets lo_off;
        for (int l = 0; l <= t.h && l < kMaxHeight + 2; ++l) lo_off.v[l] = t.lvl_off[l];
        const int cap = R.tu.probe_rows;
        R.clk.begin(GTS_STAGE_THRESHOLD);
        if (t.metric == GTS_L2)
            k_probe_vec<true><<<nblocks(nq, kWarpsPerBlock), kT, 0, st>>>(d, lo_off, nq, cap, qb.k, R.koff.get(),
                                                                          R.tk_d.get(), R.tk_id.get(), R.tk_n.get(),
                                                                          R.thr.get(), R.qkey.get());
        else
            k_probe_vec<false><<<nblocks(nq, kWarpsPerBlock), kT, 0, st>>>(d, lo_off, nq, cap, qb.k, R.koff.get(),
                                                                           R.tk_d.get(), R.tk_id.get(), R.tk_n.get(),
                                                                           R.thr.get(), R.qkey.get());
        R.qkey_ok = true;
        R.clk.end();
        check_launch("knn probe");
        R.st_pivots += nq * (int64_t)t.h;
    }
    if (t.n > 0 && nq > 0) {
        Level L0;
        L0.E = nq;
        L0.q.alloc(nq, st);
        L0.node.alloc(nq, st);
        L0.path.alloc(nq * t.h, st);
        R.clk.begin(GTS_STAGE_OTHER);
        k_root_entries<<<nblocks(nq, kT), kT, 0, st>>>(L0.q.get(), L0.node.get(), nq);
        R.clk.end();
        R.process(L0, 0, nq, 0);
    }
    if (nq > 0) R.cache_pass();
    // ---- assemble the CSR answer
    out.offsets.alloc(nq + 1, st);
    if (knn) {
        DBuf<int64_t> counts(nq + 1, st);
        R.clk.begin(GTS_STAGE_OTHER, 2);
        k_knn_counts<<<nblocks(nq, kT), kT, 0, st>>>(R.bn.get(), nq, counts.get());
        exclusive_scan(counts.get(), out.offsets.get(), nq + 1, st);
        R.clk.end();
        out.total = d2h_i64(out.offsets.get() + nq, st);
        out.ids.alloc(out.total ? out.total : 1, st);
        out.dist.alloc(out.total ? out.total : 1, st);
        if (qb.want_keys) out.key.alloc(out.total ? out.total : 1, st);
        R.clk.begin(GTS_STAGE_OTHER);
        k_knn_emit<<<(unsigned)(nq > 0 ? nq : 1), 128, 0, st>>>(out.offsets.get(), R.koff.get(), R.bd.get(),
                                                                R.bi.get(), R.bn.get(), nq, t.metric == GTS_L2,
                                                                t.cosine, out.ids.get(), out.dist.get(),
                                                                out.key.get());
        R.clk.end();
    } else {
        int64_t Rt = 0;
        for (auto v : R.rcounts) Rt += v;
        DBuf<uint64_t> keys(Rt ? Rt : 1, st), keys2(Rt ? Rt : 1, st);
        DBuf<float> dd(Rt ? Rt : 1, st);
        out.dist.alloc(Rt ? Rt : 1, st);
        out.ids.alloc(Rt ? Rt : 1, st);
        // ids are below next_id (< 2^31): the keys keep idbits id bits
        int idbits = 1;
        while (idbits < 32 && ((int64_t)1 << idbits) < ix->next_id) ++idbits;
        int64_t o = 0;
        R.clk.begin(GTS_STAGE_OTHER, (int)R.rkeys.size());
        for (size_t i = 0; i < R.rkeys.size(); ++i) {
            k_repack_keys<<<R.cap(nblocks(R.rcounts[i], kT)), kT, 0, st>>>(R.rkeys[i].get(), R.rcounts[i], idbits,
                                                                         keys.get() + o);
            GTS_CUDA(cudaMemcpyAsync(dd.get() + o, R.rdists[i].get(), R.rcounts[i] * 4, cudaMemcpyDeviceToDevice, st));
            o += R.rcounts[i];
        }
        R.clk.end();
        check_launch("repack range keys");
        R.rkeys.clear();
        R.rdists.clear();
        if (Rt > 0) {
            int qbits = 1;
            while (((int64_t)1 << qbits) < nq) ++qbits;
            size_t tb = 0;
            cub::DeviceRadixSort::SortPairs(nullptr, tb, keys.get(), keys2.get(), dd.get(), out.dist.get(), Rt, 0,
                                            idbits + qbits, st);
            DBuf<uint8_t> tmp(tb, st);
            R.clk.begin(GTS_STAGE_OTHER, 3);
            GTS_CUDA(cub::DeviceRadixSort::SortPairs(tmp.get(), tb, keys.get(), keys2.get(), dd.get(), out.dist.get(),
                                                     Rt, 0, idbits + qbits, st));
            k_range_ids<<<R.cap(nblocks(Rt, kT)), kT, 0, st>>>(keys2.get(), Rt, idbits, out.ids.get());
            k_range_offsets<<<nblocks(nq + 1, kT), kT, 0, st>>>(keys2.get(), Rt, nq, idbits, out.offsets.get());
            R.clk.end();
        } else {
            GTS_CUDA(cudaMemsetAsync(out.offsets.get(), 0, (nq + 1) * 8, st));
        }
        out.total = Rt;
    }
    check_launch("assemble");
    unsigned long long hc[2] = {0, 0}, htp[2] = {0, 0};
    GTS_CUDA(cudaMemcpyAsync(hc, R.counters.get(), 16, cudaMemcpyDeviceToHost, st));
    if (qb.count_table_pass) GTS_CUDA(cudaMemcpyAsync(htp, R.tp_count.get(), 16, cudaMemcpyDeviceToHost, st));
    GTS_CUDA(cudaStreamSynchronize(st));
    if (stage_ms) R.clk.collect(stage_ms);
    if (stats) {
        stats[GTS_STAT_PIVOT_DIST] = R.st_pivots;
        stats[GTS_STAT_FRONTIER] = R.st_frontier;
        stats[GTS_STAT_SCANNED_ROWS] = (int64_t)hc[1] + R.st_scan_rows;
        stats[GTS_STAT_CANDIDATES] = R.st_cands;
        stats[GTS_STAT_RECHECKS] = (int64_t)hc[0];
        stats[GTS_STAT_RESULTS] = out.total;
        stats[GTS_STAT_GROUPS] = R.st_groups;
        stats[GTS_STAT_CACHE_ROWS] = R.st_cache;
        stats[GTS_STAT_LAUNCHES] = R.clk.total_launches();
        stats[GTS_STAT_TILES] = R.st_tiles;
        stats[GTS_STAT_TILE_ENTRIES] = R.st_tile_entries;
        stats[GTS_STAT_TILE_PAIRS] = R.st_tile_pairs;
        stats[GTS_STAT_DENSE_PAIRS] = R.st_dense_pairs;
        stats[GTS_STAT_DENSE_LAST] = R.st_dense_last;
        stats[GTS_STAT_TABLE_PASS] = qb.count_table_pass ? (int64_t)htp[0] + R.st_table_pass : -1;
        stats[GTS_STAT_SCAN_RECORDS] = R.st_scan_records;
    }
}

}  // namespace gts
