// The extern "C" entry points of include/gts.h: argument checks, host/device
// marshalling, stream updates with sequence numbers (Section 4.4), rebuilds
// and result ownership.  No C++ exception leaves this file.
#include <cub/device/device_radix_sort.cuh>

#include <algorithm>
#include <cmath>
#include <chrono>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <new>

#include "gts_impl.cuh"
#include "metric.cuh"
#include "tile_tc.cuh"

namespace gts {

static thread_local std::string g_last_error;

void set_last_error(const std::string &msg) { g_last_error = msg; }

namespace {

constexpr int kT = 256;
inline unsigned nb(int64_t n) {
    int64_t b = (n + kT - 1) / kT;
    if (b < 1) b = 1;
    if (b > 0x7fffffffLL) b = 0x7fffffffLL;
    return (unsigned)b;
}

template <class F>
gts_status guarded(F &&f) {
    try {
        f();
        return GTS_OK;
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.status;
    } catch (const std::bad_alloc &) {
        set_last_error("host allocation failed");
        return GTS_ENOMEM;
    } catch (const std::exception &e) {
        set_last_error(e.what());
        return GTS_ECUDA;
    } catch (...) {
        set_last_error("unknown internal error");
        return GTS_ECUDA;
    }
}

}  // namespace

// Throws GTS_ECUDA when no device is usable; sets the stream-ordered pool
// to keep freed memory cached (once per device).
void ensure_device() {
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n == 0)
        throw Error(GTS_ECUDA, std::string("no usable CUDA device: ") + (e != cudaSuccess ? cudaGetErrorString(e) : "0 devices"));
    static std::atomic<bool> pool_set[64] = {};
    int dev = 0;
    GTS_CUDA(cudaGetDevice(&dev));
    if (dev < 64 && !pool_set[dev]) {
        // keep freed stream-ordered memory cached in the pool between calls
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t thr = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
        pool_set[dev] = true;
    }
}

namespace {

__global__ void k_nonfinite(const float *x, int64_t n, int *flag) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(x[i])) *flag = 1;
}

// Unit vectors for the angular distance: a warp per row sums the squares in
// FP64, every coordinate is divided in FP64 and rounded to FP32 once (so the
// rounded vector lies within 2^-24 of the exact unit vector).  A zero row
// sets *zero (it has no direction).
__global__ void k_unit_rows(const float *__restrict__ X, int64_t n, int dim, float *__restrict__ out, int *zero) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < n; r += nw) {
        const float *x = X + r * dim;
        double s = 0.0;
        for (int i = lane; i < dim; i += 32) s += (double)x[i] * (double)x[i];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (s == 0.0) {
            if (lane == 0) *zero = 1;
            continue;
        }
        const double inv = 1.0 / sqrt(s);
        for (int i = lane; i < dim; i += 32) out[r * dim + i] = (float)((double)x[i] * inv);
    }
}

// Device copy of a caller's object set (or a view when it is already on the device).
struct DevObjects {
    Objects v;
    DBuf<float> X;
    DBuf<uint8_t> S;
    DBuf<int64_t> Soff;
    std::vector<int64_t> h_off;   // host offsets (strings)
};

void load_objects(const gts_objects *o, int want_dim_or_neg, DevObjects &out, cudaStream_t st, const char *what) {
    GTS_REQUIRE(o != nullptr, GTS_EINVAL, std::string(what) + " is NULL");
    GTS_REQUIRE(o->n >= 0, GTS_EINVAL, std::string(what) + ": negative n");
    GTS_REQUIRE(o->n < ((int64_t)1 << 31), GTS_EINVAL, std::string(what) + ": n >= 2^31");
    GTS_REQUIRE(o->dim >= 0, GTS_EINVAL, std::string(what) + ": negative dim");
    if (want_dim_or_neg >= 0)
        GTS_REQUIRE(o->dim == want_dim_or_neg, GTS_EINVAL,
                    std::string(what) + ": dim " + std::to_string(o->dim) + " does not match the index (" +
                        std::to_string(want_dim_or_neg) + ")");
    const int64_t n = o->n;
    out.v.n = n;
    out.v.dim = o->dim;
    if (o->dim > 0) {
        GTS_REQUIRE(n == 0 || o->data != nullptr, GTS_EINVAL, std::string(what) + ": data is NULL");
        const size_t cnt = (size_t)n * o->dim;
        if (o->on_device) {
            out.v.X = (const float *)o->data;
        } else {
            out.X.alloc(cnt, st);
            if (cnt) GTS_CUDA(cudaMemcpyAsync(out.X.get(), o->data, cnt * 4, cudaMemcpyHostToDevice, st));
            out.v.X = out.X.get();
        }
        if (cnt) {
            DBuf<int> flag(1, st);
            GTS_CUDA(cudaMemsetAsync(flag.get(), 0, 4, st));
            k_nonfinite<<<std::min<int64_t>(nb((int64_t)cnt), 4096), kT, 0, st>>>(out.v.X, (int64_t)cnt, flag.get());
            int h = 0;
            GTS_CUDA(cudaMemcpyAsync(&h, flag.get(), 4, cudaMemcpyDeviceToHost, st));
            GTS_CUDA(cudaStreamSynchronize(st));
            GTS_REQUIRE(h == 0, GTS_EINVAL, std::string(what) + ": NaN or infinite coordinate");
        }
    } else {
        GTS_REQUIRE(o->offsets != nullptr, GTS_EINVAL, std::string(what) + ": strings need offsets");
        out.h_off.resize(n + 1);
        if (o->on_device) {
            GTS_CUDA(cudaMemcpyAsync(out.h_off.data(), o->offsets, (n + 1) * 8, cudaMemcpyDeviceToHost, st));
            GTS_CUDA(cudaStreamSynchronize(st));
        } else {
            std::memcpy(out.h_off.data(), o->offsets, (n + 1) * 8);
        }
        GTS_REQUIRE(out.h_off[0] == 0, GTS_EINVAL, std::string(what) + ": offsets[0] != 0");
        int ml = 0;
        for (int64_t i = 0; i < n; ++i) {
            const int64_t L = out.h_off[i + 1] - out.h_off[i];
            GTS_REQUIRE(L >= 0, GTS_EINVAL, std::string(what) + ": offsets not non-decreasing");
            GTS_REQUIRE(L <= kMaxStrLen, GTS_EINVAL, std::string(what) + ": string longer than 1024 bytes");
            ml = std::max<int>(ml, (int)L);
        }
        out.v.max_len = ml;
        const int64_t bytes = out.h_off[n];
        GTS_REQUIRE(bytes == 0 || o->data != nullptr, GTS_EINVAL, std::string(what) + ": data is NULL");
        if (o->on_device) {
            out.v.S = (const uint8_t *)o->data;
            out.v.Soff = o->offsets;
        } else {
            out.S.alloc(bytes > 0 ? bytes : 1, st);
            out.Soff.alloc(n + 1, st);
            if (bytes) GTS_CUDA(cudaMemcpyAsync(out.S.get(), o->data, bytes, cudaMemcpyHostToDevice, st));
            GTS_CUDA(cudaMemcpyAsync(out.Soff.get(), out.h_off.data(), (n + 1) * 8, cudaMemcpyHostToDevice, st));
            out.v.S = out.S.get();
            out.v.Soff = out.Soff.get();
        }
    }
}

// GTS_COS: the unit vectors of a loaded vector set into `unit` (rejects zero rows)
void unit_vectors(const Objects &v, DBuf<float> &unit, cudaStream_t st, const char *what) {
    const size_t cnt = (size_t)v.n * v.dim;
    unit.alloc(cnt > 0 ? cnt : 1, st);
    if (!cnt) return;
    DBuf<int> flag(1, st);
    GTS_CUDA(cudaMemsetAsync(flag.get(), 0, 4, st));
    k_unit_rows<<<std::min<int64_t>(nb(v.n * 32), 4096), kT, 0, st>>>(v.X, v.n, v.dim, unit.get(), flag.get());
    int h = 0;
    GTS_CUDA(cudaMemcpyAsync(&h, flag.get(), 4, cudaMemcpyDeviceToHost, st));
    GTS_CUDA(cudaStreamSynchronize(st));
    GTS_REQUIRE(h == 0, GTS_EINVAL, std::string(what) + ": a zero vector has no angle (GTS_COS)");
}

template <class T>
void copy_small_to_device(const T *src, int64_t n, bool on_device, DBuf<T> &dst, std::vector<T> &host,
                          cudaStream_t st) {
    host.resize(n);
    dst.alloc(n > 0 ? n : 1, st);
    if (n == 0) return;
    if (on_device) {
        GTS_CUDA(cudaMemcpyAsync(host.data(), src, n * sizeof(T), cudaMemcpyDeviceToHost, st));
        GTS_CUDA(cudaMemcpyAsync(dst.get(), src, n * sizeof(T), cudaMemcpyDeviceToDevice, st));
        GTS_CUDA(cudaStreamSynchronize(st));
    } else {
        std::memcpy(host.data(), src, n * sizeof(T));
        GTS_CUDA(cudaMemcpyAsync(dst.get(), src, n * sizeof(T), cudaMemcpyHostToDevice, st));
    }
}

__global__ void k_scatter_marks(int64_t *dst, const int64_t *pos, const int64_t *val, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[pos[i]] = val[i];
}

// loc[id] = tree row of every id after a build (-1: none), scattered on the
// device and copied back in one transfer
__global__ void k_loc_scatter(const int64_t *__restrict__ row_id, int64_t n, int64_t *__restrict__ loc) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        loc[row_id[r]] = r;
}
__global__ void k_fill_loc(int64_t *a, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = -1;
}

void refresh_loc(gts_index *ix) {
    Tree &t = ix->tree;
    cudaStream_t st = ix->stream;
    if (t.n == 0 || ix->next_id == 0) {
        ix->loc.assign(ix->next_id, -1);
        return;
    }
    // room for the stream inserts until the next rebuild (at most the cache
    // limit), so no insert has to move the whole table
    const size_t need = (size_t)ix->next_id + (size_t)std::max<int64_t>(ix->cache_limit, 0);
    if (ix->loc.capacity() < need) ix->loc.reserve(need + (size_t)ix->next_id / 8);
    ix->loc.resize(ix->next_id);   // every entry is overwritten by the copy below
    DBuf<int64_t> locd(ix->next_id, st);
    k_fill_loc<<<std::min<int64_t>(nb(ix->next_id), 4096), kT, 0, st>>>(locd.get(), ix->next_id);
    k_loc_scatter<<<std::min<int64_t>(nb(t.n), 4096), kT, 0, st>>>(t.row_id.get(), t.n, locd.get());
    GTS_CUDA(cudaMemcpyAsync(ix->loc.data(), locd.get(), ix->next_id * 8, cudaMemcpyDeviceToHost, st));
    GTS_CUDA(cudaStreamSynchronize(st));
}

// ---------------------------------------------------------------- cache list

__global__ void k_set_i64(int64_t *a, int64_t start, int64_t count, int64_t v0, int64_t step) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        a[start + i] = v0 + i * step;
}

template <class T>
void grow(DBuf<T> &b, size_t used, size_t need, cudaStream_t st) {
    if (b.n >= need) return;
    size_t cap = std::max<size_t>(need, b.n * 2);
    DBuf<T> nbuf(cap, st);
    if (used) GTS_CUDA(cudaMemcpyAsync(nbuf.get(), b.get(), used * sizeof(T), cudaMemcpyDeviceToDevice, st));
    GTS_CUDA(cudaStreamSynchronize(st));   // the old buffer is freed synchronously below
    nbuf.persist();
    b = std::move(nbuf);
}

void cache_append(gts_index *ix, const DevObjects &o, int64_t *ids_out) {
    Cache &c = ix->cache;
    cudaStream_t st = ix->stream;
    const int64_t m = o.v.n;
    if (m == 0) return;
    const int64_t need = c.count + m;
    grow(c.id, c.count, need, st);
    grow(c.ins, c.count, need, st);
    grow(c.del, c.count, need, st);
    if (ix->dim > 0) {
        grow(c.X, (size_t)c.count * ix->dim, (size_t)need * ix->dim, st);
        const float *rows = o.v.X;
        DBuf<float> unit;
        if (ix->metric == GTS_COS) {   // unit vectors for the L2 kernels, the raw rows for the FP64 keys
            unit_vectors(o.v, unit, st, "objects");
            rows = unit.get();
            grow(c.Xr, (size_t)c.count * ix->dim, (size_t)need * ix->dim, st);
            GTS_CUDA(cudaMemcpyAsync(c.Xr.get() + (size_t)c.count * ix->dim, o.v.X, (size_t)m * ix->dim * 4,
                                     cudaMemcpyDeviceToDevice, st));
        }
        GTS_CUDA(cudaMemcpyAsync(c.X.get() + (size_t)c.count * ix->dim, rows, (size_t)m * ix->dim * 4,
                                 cudaMemcpyDeviceToDevice, st));
        GTS_CUDA(cudaStreamSynchronize(st));
    } else {
        if (c.h_Soff.empty()) c.h_Soff.push_back(0);
        const int64_t add = o.h_off[m];
        grow(c.S, c.s_bytes, c.s_bytes + add + 1, st);
        if (add) GTS_CUDA(cudaMemcpyAsync(c.S.get() + c.s_bytes, o.v.S, add, cudaMemcpyDeviceToDevice, st));
        for (int64_t i = 1; i <= m; ++i) c.h_Soff.push_back(c.s_bytes + o.h_off[i]);
        c.s_bytes += add;
        grow(c.Soff, 0, need + 1, st);
        GTS_CUDA(cudaMemcpyAsync(c.Soff.get(), c.h_Soff.data(), (need + 1) * 8, cudaMemcpyHostToDevice, st));
        c.max_len = std::max(c.max_len, o.v.max_len);
    }
    k_set_i64<<<nb(m), kT, 0, st>>>(c.id.get(), c.count, m, ix->next_id, 1);
    k_set_i64<<<nb(m), kT, 0, st>>>(c.ins.get(), c.count, m, ix->seq, 1);
    k_set_i64<<<nb(m), kT, 0, st>>>(c.del.get(), c.count, m, kNever, 0);
    check_launch("cache append");
    ix->loc.resize(ix->next_id + m, -1);
    for (int64_t i = 0; i < m; ++i) {
        ix->loc[ix->next_id + i] = -(c.count + i + 2);
        if (ids_out) ids_out[i] = ix->next_id + i;
    }
    ix->next_id += m;
    ix->seq += m;
    c.count += m;
    ix->n_live += m;
    GTS_CUDA(cudaStreamSynchronize(st));
}

// ---------------------------------------------------------------- rebuild

// sort keys of the tree rows: the id of a visible row, `none` (above every
// id) for a deleted one
__global__ void k_visible_rows(const int64_t *row_del, const int64_t *row_id, int64_t n, uint64_t none,
                               uint64_t *key, int64_t *val) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const bool vis = row_del[r] == kNever;
        key[r] = vis ? (uint64_t)row_id[r] : none;
        val[r] = r;
    }
}
// the number of keys below `none` in the sorted keys (a binary search)
__global__ void k_count_below(const uint64_t *key, int64_t n, uint64_t none, int64_t *out) {
    int64_t a = 0, b = n;
    while (a < b) {
        const int64_t m = (a + b) >> 1;
        if (key[m] < none) a = m + 1;
        else b = m;
    }
    *out = a;
}

__global__ void k_gather_vec_rows(const float *X, const float *cX, int dim, int64_t n_tree, const int64_t *src,
                                  int64_t m, float *out) {
    const int64_t total = m * (int64_t)dim;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / dim;
        const int c = (int)(t - i * dim);
        const int64_t s = src[i];
        out[t] = s < n_tree ? X[s * dim + c] : cX[(s - n_tree) * dim + c];
    }
}

__global__ void k_gather_str_rows(const uint8_t *S, const int64_t *Soff, const uint8_t *cS, const int64_t *cSoff,
                                  int64_t n_tree, const int64_t *src, int64_t m, const int64_t *ooff, uint8_t *out) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = w0; i < m; i += nw) {
        const int64_t s = src[i];
        const uint8_t *p;
        int64_t len;
        if (s < n_tree) {
            p = S + Soff[s];
            len = Soff[s + 1] - Soff[s];
        } else {
            p = cS + cSoff[s - n_tree];
            len = cSoff[s - n_tree + 1] - cSoff[s - n_tree];
        }
        for (int64_t j = lane; j < len; j += 32) out[ooff[i] + j] = p[j];
    }
}

__global__ void k_gather_ids(const int64_t *row_id, const int64_t *cid, int64_t n_tree, const int64_t *src, int64_t m,
                             int64_t *ids) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = src[i];
        ids[i] = s < n_tree ? row_id[s] : cid[s - n_tree];
    }
}

// FP64 keys of (query, object) pairs for random access (multi-column
// queries): the reference operation order of each metric (L2: the squared
// sum; L1: the sum; angular distance: 1 - cos on the raw vectors); rows <
// n_tree are tree rows, the rest cache slots.
__global__ void k_pair_keys(const float *__restrict__ Q, int dim, int metric, const float *__restrict__ X,
                            const float *__restrict__ cX, int64_t n_tree, const int32_t *__restrict__ pq,
                            const int64_t *__restrict__ prow, int64_t n, double *__restrict__ keys) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const float *q = Q + (int64_t)pq[j] * dim;
        const int64_t r = prow[j];
        const float *x = r < n_tree ? X + r * dim : cX + (r - n_tree) * dim;
        keys[j] = metric == GTS_COS ? cos_key_fp64_seq(q, x, dim)
                  : metric == GTS_L2 ? l2sq_fp64_seq(q, x, dim)
                                     : l1_fp64_seq(q, x, dim);
    }
}

}  // namespace

void pair_keys(gts_index *ix, const gts_objects *queries, const std::vector<int32_t> &pq,
               const std::vector<int64_t> &pid, std::vector<double> &keys, cudaStream_t st) {
    GTS_REQUIRE(ix->dim > 0, GTS_EINVAL, "multi-column queries take vector columns (L1, L2, angular)");
    GTS_CUDA(cudaSetDevice(ix->device));
    const int64_t n = (int64_t)pq.size();
    keys.assign(n, 0.0);
    if (n == 0) return;
    DevObjects dq;
    load_objects(queries, ix->dim, dq, st, "queries");
    const Tree &t = ix->tree;
    const Cache &c = ix->cache;
    std::vector<int64_t> rows(n);
    for (int64_t j = 0; j < n; ++j) {
        const int64_t id = pid[j];
        GTS_REQUIRE(id >= 0 && id < (int64_t)ix->loc.size() && ix->loc[id] != -1, GTS_EINVAL,
                    "object " + std::to_string(id) + " is not live in every column");
        GTS_REQUIRE(pq[j] >= 0 && pq[j] < dq.v.n, GTS_EINVAL, "query index out of range");
        const int64_t L = ix->loc[id];
        rows[j] = L >= 0 ? L : t.n + (-(L + 2));
    }
    DBuf<int32_t> dpq(n, st);
    DBuf<int64_t> drow(n, st);
    DBuf<double> dk(n, st);
    GTS_CUDA(cudaMemcpyAsync(dpq.get(), pq.data(), n * 4, cudaMemcpyHostToDevice, st));
    GTS_CUDA(cudaMemcpyAsync(drow.get(), rows.data(), n * 8, cudaMemcpyHostToDevice, st));
    const bool cosr = ix->metric == GTS_COS;
    k_pair_keys<<<std::min<int64_t>(nb(n), 4096), kT, 0, st>>>(
        dq.v.X, ix->dim, ix->metric, cosr ? t.Xr.get() : t.X.get(), cosr ? c.Xr.get() : c.X.get(), t.n, dpq.get(),
        drow.get(), n, dk.get());
    check_launch("pair keys");
    GTS_CUDA(cudaMemcpyAsync(keys.data(), dk.get(), n * 8, cudaMemcpyDeviceToHost, st));
    GTS_CUDA(cudaStreamSynchronize(st));
}

namespace {

void rebuild(gts_index *ix) {
    cudaStream_t st = ix->stream;
    Tree &t = ix->tree;
    Cache &c = ix->cache;
    // visible tree rows in id order (sorted on the device by id, over the
    // bits the ids use), then visible cache slots (their ids are newer)
    int64_t vis = 0;
    DBuf<int64_t> val2(t.n > 0 ? t.n : 1, st);
    if (t.n) {
        int idbits = 1;
        while (idbits < 62 && ((int64_t)1 << idbits) <= ix->next_id) ++idbits;
        const uint64_t none = (uint64_t)1 << idbits;
        DBuf<uint64_t> key(t.n, st), key2(t.n, st);
        DBuf<int64_t> val(t.n, st), cnt(1, st);
        k_visible_rows<<<nb(t.n), kT, 0, st>>>(t.row_del.get(), t.row_id.get(), t.n, none, key.get(), val.get());
        size_t tb = 0;
        cub::DeviceRadixSort::SortPairs(nullptr, tb, key.get(), key2.get(), val.get(), val2.get(), t.n, 0,
                                        idbits + 1, st);
        DBuf<uint8_t> tmp(tb, st);
        GTS_CUDA(cub::DeviceRadixSort::SortPairs(tmp.get(), tb, key.get(), key2.get(), val.get(), val2.get(), t.n, 0,
                                                 idbits + 1, st));
        k_count_below<<<1, 1, 0, st>>>(key2.get(), t.n, none, cnt.get());
        GTS_CUDA(cudaMemcpyAsync(&vis, cnt.get(), 8, cudaMemcpyDeviceToHost, st));
        GTS_CUDA(cudaStreamSynchronize(st));
    }
    std::vector<int64_t> csrc;   // visible cache slots, as sources t.n + slot
    if (c.count) {
        std::vector<int64_t> cdel(c.count);
        GTS_CUDA(cudaMemcpyAsync(cdel.data(), c.del.get(), c.count * 8, cudaMemcpyDeviceToHost, st));
        GTS_CUDA(cudaStreamSynchronize(st));
        for (int64_t s2 = 0; s2 < c.count; ++s2)
            if (cdel[s2] == kNever) csrc.push_back(t.n + s2);
    }
    const int64_t m = vis + (int64_t)csrc.size();
    DBuf<int64_t> dsrc(m > 0 ? m : 1, st), ids(m > 0 ? m : 1, st);
    if (vis) GTS_CUDA(cudaMemcpyAsync(dsrc.get(), val2.get(), vis * 8, cudaMemcpyDeviceToDevice, st));
    if (!csrc.empty())
        GTS_CUDA(cudaMemcpyAsync(dsrc.get() + vis, csrc.data(), csrc.size() * 8, cudaMemcpyHostToDevice, st));
    // strings size their rows on the host: the sources there too
    std::vector<int64_t> src;
    if (ix->dim == 0 && m > 0) {
        src.resize(m);
        GTS_CUDA(cudaMemcpyAsync(src.data(), dsrc.get(), m * 8, cudaMemcpyDeviceToHost, st));
        GTS_CUDA(cudaStreamSynchronize(st));
    }
    k_gather_ids<<<nb(m), kT, 0, st>>>(t.row_id.get(), c.id.get(), t.n, dsrc.get(), m, ids.get());
    Objects o;
    o.n = m;
    o.dim = ix->dim;
    DBuf<float> X;
    DBuf<uint8_t> S;
    DBuf<int64_t> Soff;
    DBuf<float> Xr;
    if (ix->dim > 0) {
        X.alloc((size_t)(m > 0 ? m : 1) * ix->dim, st);
        k_gather_vec_rows<<<nb(m * (int64_t)ix->dim), kT, 0, st>>>(t.X.get(), c.X.get(), ix->dim, t.n, dsrc.get(), m,
                                                                   X.get());
        o.X = X.get();
        if (ix->metric == GTS_COS) {
            Xr.alloc((size_t)(m > 0 ? m : 1) * ix->dim, st);
            k_gather_vec_rows<<<nb(m * (int64_t)ix->dim), kT, 0, st>>>(t.Xr.get(), c.Xr.get(), ix->dim, t.n,
                                                                       dsrc.get(), m, Xr.get());
        }
    } else {
        // lengths on the host from the two offset tables
        std::vector<int64_t> toff(t.n + 1, 0);
        if (t.n) {
            GTS_CUDA(cudaMemcpyAsync(toff.data(), t.Soff.get(), (t.n + 1) * 8, cudaMemcpyDeviceToHost, st));
            GTS_CUDA(cudaStreamSynchronize(st));
        }
        std::vector<int64_t> noff(m + 1, 0);
        int ml = 0;
        for (int64_t i = 0; i < m; ++i) {
            const int64_t s = src[i];
            const int64_t L = s < t.n ? toff[s + 1] - toff[s] : c.h_Soff[s - t.n + 1] - c.h_Soff[s - t.n];
            noff[i + 1] = noff[i] + L;
            ml = std::max<int>(ml, (int)L);
        }
        Soff.alloc(m + 1, st);
        GTS_CUDA(cudaMemcpyAsync(Soff.get(), noff.data(), (m + 1) * 8, cudaMemcpyHostToDevice, st));
        S.alloc(noff[m] > 0 ? noff[m] : 1, st);
        k_gather_str_rows<<<nb(m * 32), kT, 0, st>>>(t.S.get(), t.Soff.get(), c.S.get(), c.Soff.get(), t.n, dsrc.get(),
                                                    m, Soff.get(), S.get());
        o.S = S.get();
        o.Soff = Soff.get();
        o.max_len = ml;
    }
    check_launch("rebuild gather");
    Tree nt;
    ix->rebuilds += 1;
    const int h = tree_height(m, ix->F, ix->n_pivots_req);
    const int64_t root = m > 0 ? (int64_t)(splitmix64(ix->seed + (uint64_t)ix->rebuilds) % (uint64_t)m) : 0;
    build_tree(nt, o, ids.get(), ix->metric == GTS_COS ? GTS_L2 : ix->metric, ix->F, h, root, st,
               ix->metric == GTS_COS ? Xr.get() : nullptr);
    ix->tree = std::move(nt);
    ix->cache = Cache();
    ix->rebuild_seq = ix->seq;
    ix->n_live = m;
    refresh_loc(ix);
}

struct ResultPriv {
    QueryOut out;
};

void fill_result(gts_result *res, int64_t nq, QueryOut &qo, bool on_device, cudaStream_t st) {
    res->nq = nq;
    res->on_device = on_device ? 1 : 0;
    res->key = nullptr;
    const bool keys = qo.key.get() != nullptr;
    if (on_device) {
        auto *p = new ResultPriv();
        p->out = std::move(qo);
        res->offsets = p->out.offsets.get();
        res->ids = p->out.ids.get();
        res->dist = p->out.dist.get();
        res->key = keys ? p->out.key.get() : nullptr;
        res->priv_ = p;
        return;
    }
    const int64_t tot = qo.total;
    res->offsets = (int64_t *)std::malloc(sizeof(int64_t) * (nq + 1));
    res->ids = (int64_t *)std::malloc(sizeof(int64_t) * (tot > 0 ? tot : 1));
    res->dist = (float *)std::malloc(sizeof(float) * (tot > 0 ? tot : 1));
    if (keys) res->key = (double *)std::malloc(sizeof(double) * (tot > 0 ? tot : 1));
    res->priv_ = nullptr;
    if (!res->offsets || !res->ids || !res->dist || (keys && !res->key)) {
        std::free(res->offsets);
        std::free(res->ids);
        std::free(res->dist);
        std::free(res->key);
        res->offsets = nullptr;
        res->ids = nullptr;
        res->dist = nullptr;
        res->key = nullptr;
        throw std::bad_alloc();
    }
    GTS_CUDA(cudaMemcpyAsync(res->offsets, qo.offsets.get(), (nq + 1) * 8, cudaMemcpyDeviceToHost, st));
    if (tot) {
        GTS_CUDA(cudaMemcpyAsync(res->ids, qo.ids.get(), tot * 8, cudaMemcpyDeviceToHost, st));
        GTS_CUDA(cudaMemcpyAsync(res->dist, qo.dist.get(), tot * 4, cudaMemcpyDeviceToHost, st));
        if (keys) GTS_CUDA(cudaMemcpyAsync(res->key, qo.key.get(), tot * 8, cudaMemcpyDeviceToHost, st));
    }
    GTS_CUDA(cudaStreamSynchronize(st));
}

gts_status query_common(gts_index *ix, const gts_objects *q, const float *radii, const int32_t *k,
                        const gts_query_opts *opts, gts_result *out, bool knn) {
    return guarded([&] {
        GTS_REQUIRE(ix != nullptr, GTS_EINVAL, "index is NULL");
        GTS_REQUIRE(out != nullptr, GTS_EINVAL, "result is NULL");
        ensure_device();
        GTS_CUDA(cudaSetDevice(ix->device));
        cudaStream_t st = opts ? (cudaStream_t)opts->stream : nullptr;
        GTS_REQUIRE(q != nullptr, GTS_EINVAL, "queries are NULL");
        GTS_REQUIRE((ix->metric == GTS_EDIT) == (q->dim == 0), GTS_EINVAL, "query kind does not match the metric");
        DevObjects dq;
        load_objects(q, ix->dim, dq, st, "queries");
        const int64_t nq = dq.v.n;
        QueryBatch qb;
        qb.nq = nq;
        qb.dim = ix->dim;
        qb.Q = dq.v.X;
        DBuf<float> qunit;
        if (ix->metric == GTS_COS) {   // unit query vectors for the L2 kernels, the raw ones for the FP64 keys
            unit_vectors(dq.v, qunit, st, "queries");
            qb.Q = qunit.get();
            qb.Qr = dq.v.X;
        }
        qb.S = dq.v.S;
        qb.Soff = dq.v.Soff;
        qb.max_len = dq.v.max_len;
        qb.seq_now = ix->seq;
        DBuf<float> drad;
        DBuf<int32_t> dk;
        DBuf<int64_t> dseq;
        std::vector<float> hrad;
        std::vector<int32_t> hk;
        std::vector<int64_t> hseq;
        if (knn) {
            GTS_REQUIRE(nq == 0 || k != nullptr, GTS_EINVAL, "k is NULL");
            copy_small_to_device(k, nq, q->on_device != 0, dk, hk, st);
            for (int64_t i = 0; i < nq; ++i) {
                GTS_REQUIRE(hk[i] >= 1 && hk[i] <= 1024, GTS_EINVAL, "k must be in 1 .. 1024");
                qb.max_k = std::max<int64_t>(qb.max_k, hk[i]);
            }
            qb.k = dk.get();
        } else {
            GTS_REQUIRE(nq == 0 || radii != nullptr, GTS_EINVAL, "radii is NULL");
            copy_small_to_device(radii, nq, q->on_device != 0, drad, hrad, st);
            for (int64_t i = 0; i < nq; ++i)
                GTS_REQUIRE(std::isfinite(hrad[i]) && hrad[i] >= 0.f, GTS_EINVAL, "radius must be finite and >= 0");
            qb.radii = drad.get();
        }
        DBuf<double> dlim;
        if (!knn && ix->metric == GTS_COS && nq > 0) {
            // the FP64 limits 1 - cos(r) of the range test, on the host
            std::vector<double> lim(nq);
            for (int64_t i = 0; i < nq; ++i) {
                double r = (double)hrad[i];
                if (r > 3.14159265358979323846) r = 3.14159265358979323846;
                lim[i] = 1.0 - std::cos(r);
            }
            dlim.alloc(nq, st);
            GTS_CUDA(cudaMemcpyAsync(dlim.get(), lim.data(), nq * 8, cudaMemcpyHostToDevice, st));
            GTS_CUDA(cudaStreamSynchronize(st));
            qb.coslim = dlim.get();
        }
        if (opts && opts->seq) {
            copy_small_to_device(opts->seq, nq, q->on_device != 0, dseq, hseq, st);
            for (int64_t i = 0; i < nq; ++i)
                GTS_REQUIRE(hseq[i] >= ix->rebuild_seq && hseq[i] <= ix->seq, GTS_EINVAL,
                            "query sequence number before the last rebuild or after the current state");
            qb.seq = dseq.get();
        }
        const int64_t budget = opts && opts->memory_budget > 0 ? opts->memory_budget : ((int64_t)64 << 30);
        qb.count_table_pass = opts && (opts->flags & GTS_QUERY_COUNT_TABLE_PASS) != 0;
        qb.want_keys = knn && opts && (opts->flags & GTS_QUERY_KEYS) != 0;
        QueryOut qo;
        run_query(ix, qb, knn, opts ? opts->precision : 0, budget, qo, opts ? opts->stats : nullptr,
                  opts ? opts->stage_ms : nullptr, st);
        fill_result(out, nq, qo, opts && opts->result_on_device, st);
    });
}

void check_tuning(const gts_tuning *t) {
    GTS_REQUIRE(t != nullptr, GTS_EINVAL, "tuning is NULL");
    GTS_REQUIRE(t->l1_queries == 64 || t->l1_queries == 128, GTS_EINVAL, "l1_queries must be 64 or 128");
    GTS_REQUIRE(t->l1_packed == 0 || t->l1_packed == 1, GTS_EINVAL, "l1_packed must be 0 or 1");
    GTS_REQUIRE(t->knn_phases >= 1 && t->knn_phases <= 3, GTS_EINVAL, "knn_phases must be in 1 .. 3");
    GTS_REQUIRE(t->probe_rows >= 0 && t->probe_rows <= 4096, GTS_EINVAL, "probe_rows must be in 0 .. 4096");
    GTS_REQUIRE(t->tc_queries == 96 || t->tc_queries == 128, GTS_EINVAL, "tc_queries must be 96 or 128");
    GTS_REQUIRE(t->str_chunk == 64 || t->str_chunk == 128 || t->str_chunk == 256 || t->str_chunk == 512, GTS_EINVAL,
                "str_chunk must be 64, 128, 256 or 512");
    GTS_REQUIRE(t->str_qgram == 0 || t->str_qgram == 32 || t->str_qgram == 64, GTS_EINVAL,
                "str_qgram must be 0, 32 or 64");
}

gts_tuning to_c(const Tuning &t) {
    gts_tuning o;
    std::memset(&o, 0, sizeof(o));
    o.l1_queries = t.l1_queries;
    o.l1_packed = t.l1_packed;
    o.knn_phases = t.knn_phases;
    o.probe_rows = t.probe_rows;
    o.tc_queries = t.tc_queries;
    o.str_chunk = t.str_chunk;
    o.str_qgram = t.str_qgram;
    o.tuned = t.tuned;
    return o;
}

Tuning from_c(const gts_tuning &o, int tuned) {
    Tuning t;
    t.l1_queries = o.l1_queries;
    t.l1_packed = o.l1_packed;
    t.knn_phases = o.knn_phases;
    t.probe_rows = o.probe_rows;
    t.tc_queries = o.tc_queries;
    t.str_chunk = o.str_chunk;
    t.str_qgram = o.str_qgram;
    t.tuned = tuned;
    return t;
}

}  // namespace
}  // namespace gts

using namespace gts;

extern "C" {

const char *gts_last_error(void) { return g_last_error.c_str(); }

const char *gts_status_name(gts_status s) {
    switch (s) {
        case GTS_OK: return "GTS_OK";
        case GTS_EINVAL: return "GTS_EINVAL";
        case GTS_ENOMEM: return "GTS_ENOMEM";
        case GTS_ECUDA: return "GTS_ECUDA";
        case GTS_ETIMEOUT: return "GTS_ETIMEOUT";
        case GTS_ENOTFOUND: return "GTS_ENOTFOUND";
        case GTS_EOVERFLOW: return "GTS_EOVERFLOW";
    }
    return "unknown";
}

gts_status gts_build(const gts_objects *objects, gts_metric metric, int n_pivots, int fanout,
                     const gts_build_opts *opts, gts_index **out) {
    return guarded([&] {
        GTS_REQUIRE(out != nullptr, GTS_EINVAL, "out is NULL");
        GTS_REQUIRE(metric == GTS_EDIT || metric == GTS_L1 || metric == GTS_L2 || metric == GTS_COS, GTS_EINVAL,
                    "unknown metric");
        GTS_REQUIRE(fanout >= 2 && fanout <= kMaxFanout, GTS_EINVAL, "fanout must be in 2 .. 64");
        GTS_REQUIRE(n_pivots >= 0 && n_pivots <= kMaxHeight, GTS_EINVAL, "n_pivots must be in 0 .. 12");
        GTS_REQUIRE(objects != nullptr, GTS_EINVAL, "objects is NULL");
        GTS_REQUIRE((metric == GTS_EDIT) == (objects->dim == 0), GTS_EINVAL,
                    "GTS_EDIT needs strings (dim 0); L1/L2 need vectors (dim > 0)");
        ensure_device();
        std::unique_ptr<gts_index> ix(new gts_index());
        GTS_CUDA(cudaGetDevice(&ix->device));
        ix->stream = opts ? (cudaStream_t)opts->stream : nullptr;
        ix->metric = metric;
        ix->dim = objects->dim;
        ix->F = fanout;
        ix->n_pivots_req = n_pivots;
        ix->seed = opts ? opts->seed : 0;
        ix->cache_limit = opts && opts->cache_limit > 0 ? opts->cache_limit : 4096;
        DevObjects o;
        load_objects(objects, -1, o, ix->stream, "objects");
        const int64_t n = o.v.n;
        int64_t root = opts ? opts->root_pivot : -1;
        if (n > 0) {
            if (root < 0) root = (int64_t)(splitmix64(ix->seed) % (uint64_t)n);
            GTS_REQUIRE(root < n, GTS_EINVAL, "root_pivot out of range");
        } else {
            root = 0;
        }
        const int h = tree_height(n, fanout, n_pivots);
        if (metric == GTS_COS) {   // an L2 tree over the unit vectors; the raw rows kept for the FP64 keys
            DBuf<float> unit;
            unit_vectors(o.v, unit, ix->stream, "objects");
            Objects uv = o.v;
            uv.X = unit.get();
            build_tree(ix->tree, uv, nullptr, GTS_L2, fanout, h, root, ix->stream, o.v.X);
        } else {
            build_tree(ix->tree, o.v, nullptr, metric, fanout, h, root, ix->stream);
        }
        ix->next_id = n;
        ix->n_live = n;
        refresh_loc(ix.get());
        *out = ix.release();
    });
}

gts_status gts_range(gts_index *index, const gts_objects *queries, const float *radii, const gts_query_opts *opts,
                     gts_result *out) {
    return query_common(index, queries, radii, nullptr, opts, out, false);
}

gts_status gts_knn(gts_index *index, const gts_objects *queries, const int32_t *k, const gts_query_opts *opts,
                   gts_result *out) {
    return query_common(index, queries, nullptr, k, opts, out, true);
}

gts_status gts_insert(gts_index *ix, const gts_objects *objects, int64_t *ids_out) {
    return guarded([&] {
        GTS_REQUIRE(ix != nullptr, GTS_EINVAL, "index is NULL");
        ensure_device();
        GTS_CUDA(cudaSetDevice(ix->device));
        GTS_REQUIRE(objects != nullptr, GTS_EINVAL, "objects is NULL");
        GTS_REQUIRE((ix->metric == GTS_EDIT) == (objects->dim == 0), GTS_EINVAL, "object kind does not match the metric");
        DevObjects o;
        load_objects(objects, ix->dim, o, ix->stream, "objects");
        GTS_REQUIRE(ix->next_id + o.v.n < ((int64_t)1 << 31), GTS_EINVAL, "object ids would reach 2^31");
        cache_append(ix, o, ids_out);
        if (ix->cache.count > ix->cache_limit) rebuild(ix);
    });
}

gts_status gts_delete(gts_index *ix, const int64_t *ids, int64_t m, int64_t *n_missing) {
    int64_t missing = 0;
    gts_status s = guarded([&] {
        GTS_REQUIRE(ix != nullptr, GTS_EINVAL, "index is NULL");
        GTS_REQUIRE(m >= 0 && (m == 0 || ids != nullptr), GTS_EINVAL, "bad id list");
        ensure_device();
        GTS_CUDA(cudaSetDevice(ix->device));
        std::vector<int64_t> tree_rows, tree_seq, cache_slots, cache_seq;
        for (int64_t i = 0; i < m; ++i) {
            const int64_t id = ids[i];
            if (id < 0 || id >= (int64_t)ix->loc.size() || ix->loc[id] == -1) {
                ++missing;
                continue;
            }
            const int64_t L = ix->loc[id];
            if (L >= 0) {
                tree_rows.push_back(L);
                tree_seq.push_back(ix->seq);
                ix->tree.n_deleted += 1;
            } else {
                cache_slots.push_back(-(L + 2));
                cache_seq.push_back(ix->seq);
            }
            ix->loc[id] = -1;
            ix->seq += 1;
            ix->n_live -= 1;
        }
        cudaStream_t st = ix->stream;
        // the delete marks: (position, sequence) pairs to the device in one
        // copy per list, then scattered
        for (int k = 0; k < 2; ++k) {
            auto &pos = k == 0 ? tree_rows : cache_slots;
            auto &sq = k == 0 ? tree_seq : cache_seq;
            if (pos.empty()) continue;
            int64_t *dst = k == 0 ? ix->tree.row_del.get() : ix->cache.del.get();
            const int64_t cnt = (int64_t)pos.size();
            DBuf<int64_t> dp(2 * cnt, st);
            GTS_CUDA(cudaMemcpyAsync(dp.get(), pos.data(), cnt * 8, cudaMemcpyHostToDevice, st));
            GTS_CUDA(cudaMemcpyAsync(dp.get() + cnt, sq.data(), cnt * 8, cudaMemcpyHostToDevice, st));
            k_scatter_marks<<<nb(cnt), kT, 0, st>>>(dst, dp.get(), dp.get() + cnt, cnt);
        }
        check_launch("delete marks");
        GTS_CUDA(cudaStreamSynchronize(st));
    });
    if (n_missing) *n_missing = missing;
    if (s == GTS_OK && missing > 0) {
        set_last_error(std::to_string(missing) + " id(s) unknown or already deleted");
        return GTS_ENOTFOUND;
    }
    return s;
}

gts_status gts_batch_update(gts_index *ix, const gts_objects *ins, const int64_t *del, int64_t m_del,
                            int64_t *ids_out) {
    gts_status s = guarded([&] {
        GTS_REQUIRE(ix != nullptr, GTS_EINVAL, "index is NULL");
        ensure_device();
        GTS_CUDA(cudaSetDevice(ix->device));
        if (ins) {
            GTS_REQUIRE((ix->metric == GTS_EDIT) == (ins->dim == 0), GTS_EINVAL, "object kind does not match the metric");
            DevObjects o;
            load_objects(ins, ix->dim, o, ix->stream, "objects");
            GTS_REQUIRE(ix->next_id + o.v.n < ((int64_t)1 << 31), GTS_EINVAL, "object ids would reach 2^31");
            cache_append(ix, o, ids_out);
        }
    });
    if (s != GTS_OK) return s;
    int64_t missing = 0;
    if (m_del > 0) {
        s = gts_delete(ix, del, m_del, &missing);
        if (s != GTS_OK && s != GTS_ENOTFOUND) return s;
    }
    s = guarded([&] { rebuild(ix); });
    if (s == GTS_OK && missing > 0) {
        set_last_error(std::to_string(missing) + " id(s) unknown or already deleted");
        return GTS_ENOTFOUND;
    }
    return s;
}

gts_status gts_rebuild(gts_index *ix) {
    return guarded([&] {
        GTS_REQUIRE(ix != nullptr, GTS_EINVAL, "index is NULL");
        ensure_device();
        GTS_CUDA(cudaSetDevice(ix->device));
        rebuild(ix);
    });
}

gts_status gts_info(const gts_index *ix, gts_index_info *out) {
    return guarded([&] {
        GTS_REQUIRE(ix != nullptr && out != nullptr, GTS_EINVAL, "NULL argument");
        out->n_tree = ix->tree.n;
        out->n_cache = ix->cache.count;
        out->n_live = ix->n_live;
        out->next_id = ix->next_id;
        out->seq = ix->seq;
        out->rebuild_seq = ix->rebuild_seq;
        out->h = ix->tree.h;
        out->fanout = ix->F;
        out->metric = ix->metric;
        out->dim = ix->dim;
        const Cache &c = ix->cache;
        out->device_bytes = (int64_t)(ix->tree.device_bytes() + c.X.bytes() + c.S.bytes() + c.Soff.bytes() +
                                      c.id.bytes() + c.ins.bytes() + c.del.bytes());
    });
}

gts_status gts_tree_level(const gts_index *ix, int level, int64_t *pos, int64_t *size, float *lo, float *hi,
                          int64_t *pivot) {
    return guarded([&] {
        GTS_REQUIRE(ix != nullptr, GTS_EINVAL, "index is NULL");
        const Tree &t = ix->tree;
        GTS_REQUIRE(level >= 0 && level <= t.h, GTS_EINVAL, "level out of range");
        GTS_CUDA(cudaSetDevice(ix->device));
        cudaStream_t st = ix->stream;
        const int64_t a = t.lvl_off[level], cnt = t.lvl_off[level + 1] - a;
        std::vector<int32_t> p(cnt), s(cnt), pv(cnt);
        std::vector<float> l(cnt), hh(cnt);
        GTS_CUDA(cudaMemcpyAsync(p.data(), t.npos.get() + a, cnt * 4, cudaMemcpyDeviceToHost, st));
        GTS_CUDA(cudaMemcpyAsync(s.data(), t.nsize.get() + a, cnt * 4, cudaMemcpyDeviceToHost, st));
        GTS_CUDA(cudaMemcpyAsync(pv.data(), t.npiv.get() + a, cnt * 4, cudaMemcpyDeviceToHost, st));
        GTS_CUDA(cudaMemcpyAsync(l.data(), t.nlo.get() + a, cnt * 4, cudaMemcpyDeviceToHost, st));
        GTS_CUDA(cudaMemcpyAsync(hh.data(), t.nhi.get() + a, cnt * 4, cudaMemcpyDeviceToHost, st));
        std::vector<int64_t> rid(t.n);
        if (t.n) GTS_CUDA(cudaMemcpyAsync(rid.data(), t.row_id.get(), t.n * 8, cudaMemcpyDeviceToHost, st));
        GTS_CUDA(cudaStreamSynchronize(st));
        for (int64_t i = 0; i < cnt; ++i) {
            if (pos) pos[i] = p[i];
            if (size) size[i] = s[i];
            if (lo) lo[i] = l[i];
            if (hi) hi[i] = hh[i];
            if (pivot) pivot[i] = (level < t.h && pv[i] >= 0) ? rid[pv[i]] : -1;
        }
    });
}

gts_status gts_table(const gts_index *ix, int64_t *ids, float *table) {
    return guarded([&] {
        GTS_REQUIRE(ix != nullptr, GTS_EINVAL, "index is NULL");
        const Tree &t = ix->tree;
        GTS_CUDA(cudaSetDevice(ix->device));
        cudaStream_t st = ix->stream;
        if (ids && t.n) GTS_CUDA(cudaMemcpyAsync(ids, t.row_id.get(), t.n * 8, cudaMemcpyDeviceToHost, st));
        if (table && t.n)
            GTS_CUDA(cudaMemcpyAsync(table, t.table.get(), (size_t)t.h * t.n * 4, cudaMemcpyDeviceToHost, st));
        GTS_CUDA(cudaStreamSynchronize(st));
    });
}

gts_status gts_result_copy(const gts_result *r, int64_t *offsets, int64_t *ids, float *dist) {
    return guarded([&] {
        GTS_REQUIRE(r != nullptr && r->offsets != nullptr, GTS_EINVAL, "empty result");
        int64_t total = 0;
        GTS_CUDA(cudaMemcpy(&total, r->offsets + r->nq, 8, cudaMemcpyDefault));
        if (offsets) GTS_CUDA(cudaMemcpy(offsets, r->offsets, (r->nq + 1) * 8, cudaMemcpyDefault));
        if (ids && total) GTS_CUDA(cudaMemcpy(ids, r->ids, total * 8, cudaMemcpyDefault));
        if (dist && total) GTS_CUDA(cudaMemcpy(dist, r->dist, total * 4, cudaMemcpyDefault));
    });
}

gts_status gts_selftest_tc(const float *A, const float *B, int N, int K, int a_tmem, float *D) {
    return guarded([&] {
        GTS_REQUIRE(A && B && D, GTS_EINVAL, "NULL argument");
        ensure_device();
        tc_selftest(A, B, N, K, a_tmem, D);
    });
}

gts_status gts_selftest_wait(int32_t post, uint32_t spin_limit) {
    return guarded([&] {
        ensure_device();
        wait_selftest(post, spin_limit);
    });
}

gts_status gts_get_tuning(gts_index *ix, gts_tuning *out) {
    return guarded([&] {
        GTS_REQUIRE(ix != nullptr && out != nullptr, GTS_EINVAL, "index or output is NULL");
        std::lock_guard<std::mutex> g(ix->tune_mu);
        *out = to_c(ix->tuning);
    });
}

gts_status gts_set_tuning(gts_index *ix, const gts_tuning *t) {
    return guarded([&] {
        GTS_REQUIRE(ix != nullptr, GTS_EINVAL, "index is NULL");
        check_tuning(t);
        std::lock_guard<std::mutex> g(ix->tune_mu);
        ix->tuning = from_c(*t, ix->tuning.tuned);
    });
}

gts_status gts_autotune(gts_index *ix, const gts_objects *queries, const float *radii, const int32_t *k,
                        const gts_query_opts *opts, int32_t reps, gts_tuning *out) {
    gts_tuning best;
    gts_status s = guarded([&] {
        GTS_REQUIRE(ix != nullptr, GTS_EINVAL, "index is NULL");
        GTS_REQUIRE((radii == nullptr) != (k == nullptr), GTS_EINVAL, "give radii (range) or k (kNN), not both");
        GTS_REQUIRE(reps >= 1 && reps <= 100, GTS_EINVAL, "reps must be in 1 .. 100");
        std::lock_guard<std::mutex> g(ix->tune_mu);
        best = to_c(ix->tuning);
    });
    if (s != GTS_OK) return s;
    const bool knn = k != nullptr;
    gts_query_opts o;
    std::memset(&o, 0, sizeof(o));
    if (opts) o = *opts;
    o.stats = nullptr;
    o.stage_ms = nullptr;
    o.flags = 0;
    o.result_on_device = 1;
    // one setting: the median wall time of `reps` runs of the sample batch
    auto time_it = [&](const gts_tuning &t, double &ms) -> gts_status {
        gts_status r = gts_set_tuning(ix, &t);
        if (r != GTS_OK) return r;
        std::vector<double> v;
        for (int i = 0; i < reps; ++i) {
            gts_result res;
            std::memset(&res, 0, sizeof(res));
            const auto t0 = std::chrono::steady_clock::now();
            r = query_common(ix, queries, radii, k, &o, &res, knn);
            const auto t1 = std::chrono::steady_clock::now();
            if (r != GTS_OK) return r;
            gts_result_free(&res);
            v.push_back(std::chrono::duration<double, std::milli>(t1 - t0).count());
        }
        std::sort(v.begin(), v.end());
        ms = v[v.size() / 2];
        return GTS_OK;
    };
    // coordinate descent over the parameters that apply to this index
    std::vector<std::pair<int32_t gts_tuning::*, std::vector<int32_t>>> space;
    if (ix->metric == GTS_L1) {
        space.push_back({&gts_tuning::l1_queries, {64, 128}});
        space.push_back({&gts_tuning::l1_packed, {0, 1}});
        if (knn) space.push_back({&gts_tuning::knn_phases, {1, 2, 3}});
    }
    if (knn && ix->metric != GTS_EDIT) space.push_back({&gts_tuning::probe_rows, {0, 256, 1024, 4096}});
    if ((ix->metric == GTS_L2 || ix->metric == GTS_COS) && ix->dim <= 128)
        space.push_back({&gts_tuning::tc_queries, {128, 96}});
    if (ix->metric == GTS_EDIT) {
        space.push_back({&gts_tuning::str_chunk, {64, 128, 256, 512}});
        if (o.precision == GTS_PREC_BF16) space.push_back({&gts_tuning::str_qgram, {0, 32, 64}});
    }
    double best_ms = 0.0;
    s = time_it(best, best_ms);   // the first run also warms every lazily built structure
    if (s == GTS_OK) s = time_it(best, best_ms);
    for (auto &dim : space) {
        if (s != GTS_OK) break;
        for (int32_t v : dim.second) {
            if (best.*(dim.first) == v) continue;
            gts_tuning t = best;
            t.*(dim.first) = v;
            double ms = 0.0;
            s = time_it(t, ms);
            if (s != GTS_OK) break;
            if (ms < best_ms) {
                best_ms = ms;
                best = t;
            }
        }
    }
    gts_status s2 = guarded([&] {
        std::lock_guard<std::mutex> g(ix->tune_mu);
        ix->tuning = from_c(best, s == GTS_OK ? 1 : ix->tuning.tuned);
        best = to_c(ix->tuning);
    });
    if (out) *out = best;
    return s != GTS_OK ? s : s2;
}

double gts_cost_model(int64_t n, int64_t nq, double p, int32_t fanout, int32_t h, double concurrency) {
    if (n < 0 || nq < 0 || fanout < 2 || h < 1 || !(concurrency >= 1.0) || !(p >= 0.0 && p <= 1.0)) return -1.0;
    const double lf = std::log2((double)fanout);
    double cost = 0.0, level = (double)nq;   // S_i = nq (fanout p)^i
    for (int i = 1; i <= h; ++i) {
        level *= (double)fanout * p;
        cost += (double)i * i * std::ceil(level / concurrency) * lf * lf;
    }
    const double objs = (double)nq * (double)n * std::pow(p, h);   // objects of the surviving leaves
    cost += (double)(h + 1) * (h + 1) * std::ceil(objs / concurrency) * lf * lf;
    return cost;
}

namespace {

// P(|X - Y| <= r) over all pairs of a sample of one pivot's distances (Eq. 2)
double pair_prob(std::vector<float> x, double r) {
    std::sort(x.begin(), x.end());
    const size_t m = x.size();
    if (m < 2) return 1.0;
    double within = 0.0;
    size_t j = 0;
    for (size_t i = 0; i < m; ++i) {   // pairs (j, i), j < i, with x_i - x_j <= r
        while ((double)x[i] - (double)x[j] > r) ++j;
        within += (double)(i - j);
    }
    return within / ((double)m * (double)(m - 1) / 2.0);
}

}  // namespace

gts_status gts_autotune_shape(gts_index *ix, const gts_objects *queries, const float *radii, const int32_t *k,
                              const gts_query_opts *opts, int32_t candidates, int32_t reps, gts_shape *out,
                              int32_t *n_out) {
    std::vector<gts_shape> timed;
    gts_status s = guarded([&] {
        GTS_REQUIRE(ix != nullptr && queries != nullptr, GTS_EINVAL, "index or queries is NULL");
        GTS_REQUIRE((radii == nullptr) != (k == nullptr), GTS_EINVAL, "give radii (range) or k (kNN), not both");
        GTS_REQUIRE(reps >= 1 && reps <= 100, GTS_EINVAL, "reps must be in 1 .. 100");
        GTS_REQUIRE(candidates >= 1 && candidates <= 16, GTS_EINVAL, "candidates must be in 1 .. 16");
        GTS_REQUIRE(queries->n > 0, GTS_EINVAL, "the sample batch is empty");
        ensure_device();
        GTS_CUDA(cudaSetDevice(ix->device));
        const bool knn = k != nullptr;
        gts_query_opts o;
        std::memset(&o, 0, sizeof(o));
        if (opts) o = *opts;
        o.stats = nullptr;
        o.stage_ms = nullptr;
        o.flags = 0;
        // the radius of Eq. 2: range -> the median radius; kNN -> the mean k-th distance
        double r = 0.0;
        {
            gts_query_opts oh = o;
            oh.result_on_device = 0;
            gts_result res;
            std::memset(&res, 0, sizeof(res));
            gts_status q = query_common(ix, queries, radii, k, &oh, &res, knn);
            if (q != GTS_OK) throw Error(q, gts_last_error());
            if (knn) {
                double sum = 0.0;
                int64_t cnt = 0;
                for (int64_t i = 0; i < res.nq; ++i)
                    if (res.offsets[i + 1] > res.offsets[i]) {
                        sum += res.dist[res.offsets[i + 1] - 1];
                        ++cnt;
                    }
                r = cnt ? sum / (double)cnt : 0.0;
            } else {
                std::vector<float> hr(queries->n);
                if (queries->on_device)
                    GTS_CUDA(cudaMemcpy(hr.data(), radii, queries->n * 4, cudaMemcpyDeviceToHost));
                else
                    std::memcpy(hr.data(), radii, queries->n * 4);
                std::nth_element(hr.begin(), hr.begin() + hr.size() / 2, hr.end());
                r = hr[hr.size() / 2];
            }
            gts_result_free(&res);
        }
        // p from the table list: distances of a sample of rows to the root pivot
        const Tree &t = ix->tree;
        const int64_t n = t.n;
        double p = 1.0;
        if (n > 1) {
            const int64_t m = std::min<int64_t>(n, 4096);
            std::vector<float> col(n);
            GTS_CUDA(cudaMemcpy(col.data(), t.table.get(), n * 4, cudaMemcpyDeviceToHost));
            std::vector<float> smp(m);
            for (int64_t i = 0; i < m; ++i) smp[i] = col[(i * n) / m];
            p = pair_prob(std::move(smp), r);
        }
        int sms = 0;
        GTS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ix->device));
        const double C = (double)(sms > 0 ? sms : 1) * 2048.0;
        const int64_t nq = queries->n;
        // rank every shape by the model
        std::vector<gts_shape> all;
        for (int F : {4, 6, 8, 10, 12, 16, 20, 24, 32, 40, 48, 64}) {
            const int hmax = tree_height(n + ix->cache.count, F, 0);
            for (int h = 1; h <= hmax; ++h) {
                gts_shape sh;
                sh.fanout = F;
                sh.n_pivots = h;
                sh.model_cost = gts_cost_model(n, nq, p, F, h, C);
                sh.measured_ms = 0.0;
                all.push_back(sh);
            }
        }
        std::stable_sort(all.begin(), all.end(),
                         [](const gts_shape &a, const gts_shape &b) { return a.model_cost < b.model_cost; });
        // candidates: the current shape, its neighbours (fanout halved /
        // doubled, one pivot level fewer / more) and the model's cheapest,
        // `candidates` in all besides the current one
        std::vector<gts_shape> cand;
        auto add = [&](int F, int h) {
            if (F < 2 || F > kMaxFanout || h < 1 || h > tree_height(n + ix->cache.count, F, 0)) return;
            for (auto &c : cand)
                if (c.fanout == F && c.n_pivots == h) return;
            gts_shape sh;
            sh.fanout = F;
            sh.n_pivots = h;
            sh.model_cost = gts_cost_model(n, nq, p, F, h, C);
            sh.measured_ms = 0.0;
            cand.push_back(sh);
        };
        add(ix->F, ix->tree.h);
        const int F0 = ix->F, h0 = ix->tree.h;
        const int nb[][2] = {{F0, h0 - 1}, {F0, h0 + 1}, {F0 * 2, h0 - 1}, {F0 / 2, h0 + 1}, {F0 * 2, h0}, {F0 / 2, h0}};
        const size_t want = 1 + (size_t)candidates;
        for (auto &v : nb)
            if (cand.size() < 1 + ((size_t)candidates + 1) / 2) add(v[0], v[1]);
        for (auto &sh : all)
            if (cand.size() < want) add(sh.fanout, sh.n_pivots);
        o.result_on_device = 1;
        auto time_shape = [&](gts_shape &sh) {
            ix->F = sh.fanout;
            ix->n_pivots_req = sh.n_pivots;
            rebuild(ix);
            std::vector<double> v;
            for (int i = 0; i <= reps; ++i) {   // run 0 warms the lazily built per-index data
                gts_result res;
                std::memset(&res, 0, sizeof(res));
                const auto t0 = std::chrono::steady_clock::now();
                gts_status q = query_common(ix, queries, radii, k, &o, &res, knn);
                const auto t1 = std::chrono::steady_clock::now();
                if (q != GTS_OK) throw Error(q, gts_last_error());
                gts_result_free(&res);
                if (i > 0) v.push_back(std::chrono::duration<double, std::milli>(t1 - t0).count());
            }
            std::sort(v.begin(), v.end());
            sh.measured_ms = v[v.size() / 2];
        };
        for (auto &sh : cand) {
            try {
                time_shape(sh);
            } catch (const Error &e) {
                // a shape whose tree or batch does not fit the device is
                // skipped (recorded with an infinite time); other errors stand
                if (e.status != GTS_ENOMEM && e.status != GTS_EOVERFLOW) throw;
                cudaGetLastError();
                sh.measured_ms = INFINITY;
            }
            timed.push_back(sh);
        }
        GTS_REQUIRE(std::isfinite(std::min_element(timed.begin(), timed.end(),
                                                   [](const gts_shape &a, const gts_shape &b) {
                                                       return a.measured_ms < b.measured_ms;
                                                   })->measured_ms),
                    GTS_ENOMEM, "no candidate shape fits the device");
        std::stable_sort(timed.begin(), timed.end(),
                         [](const gts_shape &a, const gts_shape &b) { return a.measured_ms < b.measured_ms; });
        const gts_shape &best = timed.front();
        if (ix->F != best.fanout || ix->tree.h != best.n_pivots) {
            ix->F = best.fanout;
            ix->n_pivots_req = best.n_pivots;
            rebuild(ix);
        }
    });
    if (out)
        for (size_t i = 0; i < timed.size(); ++i) out[i] = timed[i];
    if (n_out) *n_out = (int32_t)timed.size();
    return s;
}

void gts_result_free(gts_result *r) {
    if (!r) return;
    if (r->priv_) {
        delete (ResultPriv *)r->priv_;
    } else {
        std::free(r->offsets);
        std::free(r->ids);
        std::free(r->dist);
        std::free(r->key);
    }
    r->offsets = nullptr;
    r->ids = nullptr;
    r->dist = nullptr;
    r->key = nullptr;
    r->priv_ = nullptr;
    r->nq = 0;
}

void gts_free(gts_index *ix) {
    if (!ix) return;
    cudaSetDevice(ix->device);
    cudaStreamSynchronize(ix->stream);
    delete ix;
}

}  // extern "C"
