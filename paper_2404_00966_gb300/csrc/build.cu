// Index construction on the GPU (Section 4.3, Algorithms 1-3).
//
// All nodes of one level are processed together (the paper's level-parallel
// construction).  Per pivot level l = 0 .. h-1:
//   1. pivot choice (Algorithm 2, FFT): one block per node picks the object
//      whose smallest distance to the pivots of its ancestors is largest
//      (ties to the smallest id); the root pivot is given.
//   2. mapping (Algorithm 2): every object's distance to its node's pivot,
//      computed exactly (FP64 in the reference operation order for L1/L2,
//      bit-parallel integer DP for edit distance), stored as float32.
//   3. partitioning (Algorithm 3): one global radix sort of 64-bit keys
//      (node index << 32 | distance bits) over objects listed in id order;
//      the sort is stable, so ties fall to the smaller id.  This plays the
//      role of the paper's encoded key i + dis / (max + 1) without its
//      floating-point collisions at large node indices.
//   4. even split of each node into fanout children by count, the last child
//      taking the remainder; a child's [lo, hi] is its first and last distance.
// Objects stay in input order while the levels are built (per-object columns);
// at the end they are gathered once into leaf order.
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include "gts_impl.cuh"
#include "metric.cuh"

namespace gts {

uint64_t splitmix64(uint64_t x) {
    // SplitMix64 (Steele, Lea, Flood 2014): one output for state x.
    uint64_t z = x + 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

int tree_height(int64_t n, int F, int n_pivots) {
    if (n_pivots > 0) return n_pivots < kMaxHeight ? n_pivots : kMaxHeight;
    // ceil(log_F(n + 1)) - 1 (Algorithm 1), in integers; at least one pivot level
    int t = 0;
    long double p = 1;
    while (p < (long double)n + 1) {
        p *= F;
        ++t;
    }
    // at least one pivot level; at most kMaxHeight (small fanouts over large sets)
    const int h = t - 1 < 1 ? 1 : t - 1;
    return h < kMaxHeight ? h : kMaxHeight;
}

size_t Tree::device_bytes() const {
    return X.bytes() + S.bytes() + Soff.bytes() + row_id.bytes() + table.bytes() + row_del.bytes() + npos.bytes() +
           nsize.bytes() + npiv.bytes() + nlo.bytes() + nhi.bytes() + tc.Xh.bytes() + tc.Xl.bytes() + tc.xn2.bytes() +
           qg.bytes();
}

namespace {

constexpr int kThreads = 256;

inline unsigned blocks_for(int64_t n, int per = kThreads) {
    int64_t b = (n + per - 1) / per;
    if (b < 1) b = 1;
    if (b > 0x7fffffff) b = 0x7fffffff;
    return (unsigned)b;
}

__global__ void k_iota_i32(int32_t *a, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = (int32_t)i;
}

__global__ void k_fill_i32(int32_t *a, int64_t n, int32_t v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = v;
}

__global__ void k_fill_i64(int64_t *a, int64_t n, int64_t v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = v;
}

// FFT pivot of every node of level l >= 1.  Key = (score bits << 32) |
// (0x7fffffff - object index): the maximum has the largest score, then the
// smallest index (objects are listed in increasing id order).
__global__ void k_fft_pivot(const int32_t *__restrict__ perm, const float *__restrict__ T, int64_t n, int l,
                            const int32_t *__restrict__ lpos, const int32_t *__restrict__ lsize,
                            int32_t *__restrict__ piv_obj) {
    const int node = blockIdx.x;
    const int32_t s = lpos[node], c = lsize[node];
    if (c == 0) {
        if (threadIdx.x == 0) piv_obj[node] = -1;
        return;
    }
    unsigned long long best = 0ull;
    for (int32_t r = threadIdx.x; r < c; r += blockDim.x) {
        const int32_t o = perm[s + r];
        float sc = T[o];
        for (int a = 1; a < l; ++a) sc = fminf(sc, T[(int64_t)a * n + o]);
        const unsigned long long key =
            ((unsigned long long)__float_as_uint(sc) << 32) | (unsigned long long)(0x7fffffffu - (uint32_t)o);
        best = key > best ? key : best;
    }
    __shared__ unsigned long long red[kThreads / 32];
    for (int off = 16; off > 0; off >>= 1) {
        unsigned long long o2 = __shfl_xor_sync(0xffffffffu, best, off);
        best = o2 > best ? o2 : best;
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long b = red[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) b = red[w] > b ? red[w] : b;
        piv_obj[node] = (int32_t)(0x7fffffffu - (uint32_t)(b & 0xffffffffull));
    }
}

// Mapping for vectors: one thread per table position, FP64 in the reference
// order, rounded once to float32.  Also records each object's node.
template <bool L2>
__global__ void k_map_vec(const float *__restrict__ X, int dim, const int32_t *__restrict__ perm,
                          const int32_t *__restrict__ pos_node, const int32_t *__restrict__ piv_obj, int64_t n,
                          float *__restrict__ Tl, int32_t *__restrict__ node_of) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t o = perm[p];
        const int32_t node = pos_node[p];
        const int32_t pv = piv_obj[node];
        const float *a = X + (int64_t)o * dim;
        const float *b = X + (int64_t)pv * dim;
        double d = L2 ? l2sq_fp64_seq(a, b, dim) : l1_fp64_seq(a, b, dim);
        if (L2) d = __dsqrt_rn(d);
        Tl[o] = __double2float_rn(d);
        node_of[o] = node;
    }
}

// Mapping for strings: a block takes a run of table positions; for every node
// in the run it loads the node pivot's match masks into shared memory and each
// thread computes one object's distance to the pivot (pattern = pivot).
template <int W>
__global__ void k_map_str(const uint8_t *__restrict__ S, const int64_t *__restrict__ Soff,
                          const int32_t *__restrict__ perm, const int32_t *__restrict__ pos_node,
                          const int32_t *__restrict__ piv_obj, const int32_t *__restrict__ lpos,
                          const int32_t *__restrict__ lsize, int64_t n, int chunk, float *__restrict__ Tl,
                          int32_t *__restrict__ node_of) {
    __shared__ uint64_t Peq[256 * W];
    const int64_t p0 = (int64_t)blockIdx.x * chunk;
    const int64_t p1 = p0 + chunk < n ? p0 + chunk : n;
    int64_t s = p0;
    while (s < p1) {
        const int32_t node = pos_node[s];
        int64_t e = (int64_t)lpos[node] + lsize[node];
        if (e > p1) e = p1;
        const int32_t pv = piv_obj[node];
        const int m = (int)(Soff[pv + 1] - Soff[pv]);
        if (m > 0) build_peq<W>(Peq, S + Soff[pv], m);
        for (int64_t p = s + threadIdx.x; p < e; p += blockDim.x) {
            const int32_t o = perm[p];
            const int len = (int)(Soff[o + 1] - Soff[o]);
            const int d = m > 0 ? myers_edit<W>(Peq, m, S + Soff[o], len) : len;
            Tl[o] = (float)d;
            node_of[o] = node;
        }
        __syncthreads();
        s = e;
    }
}

__global__ void k_keys(const int32_t *__restrict__ node_of, const float *__restrict__ Tl, int64_t n,
                       uint64_t *__restrict__ keys, int32_t *__restrict__ vals) {
    for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n; o += (int64_t)gridDim.x * blockDim.x) {
        keys[o] = ((uint64_t)(uint32_t)node_of[o] << 32) | (uint64_t)__float_as_uint(Tl[o]);
        vals[o] = (int32_t)o;
    }
}

// Children of every node of level l: even split by count (Algorithm 3).
__global__ void k_children(const int32_t *__restrict__ lpos, const int32_t *__restrict__ lsize, int64_t nn, int F,
                           const int32_t *__restrict__ perm, const float *__restrict__ Tl,
                           int32_t *__restrict__ cpos, int32_t *__restrict__ csize, float *__restrict__ clo,
                           float *__restrict__ chi) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nn * F; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / F;
        const int j = (int)(t - i * F);
        const int32_t s = lpos[i], c = lsize[i];
        const int32_t avg = c / F;
        const int32_t cs = s + j * avg;
        const int32_t cc = j < F - 1 ? avg : c - avg * (F - 1);
        cpos[t] = cs;
        csize[t] = cc;
        if (cc > 0) {
            clo[t] = Tl[perm[cs]];
            chi[t] = Tl[perm[cs + cc - 1]];
        } else {
            clo[t] = __int_as_float(0x7f800000);   // +inf
            chi[t] = __int_as_float(0xff800000);   // -inf
        }
    }
}

__global__ void k_next_pos_node(int32_t *__restrict__ pos_node, int64_t n, const int32_t *__restrict__ lpos,
                                const int32_t *__restrict__ lsize, int F) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t node = pos_node[p];
        const int32_t s = lpos[node], c = lsize[node];
        const int32_t avg = c / F;
        int32_t j = avg > 0 ? (int32_t)((p - s) / avg) : F - 1;
        if (j > F - 1) j = F - 1;
        pos_node[p] = node * F + j;
    }
}

__global__ void k_gather_rows(const float *__restrict__ X, int dim, const int32_t *__restrict__ perm, int64_t n,
                              float *__restrict__ Xl) {
    const int64_t total = n * (int64_t)dim;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = t / dim;
        const int c = (int)(t - p * dim);
        Xl[t] = X[(int64_t)perm[p] * dim + c];
    }
}

__global__ void k_gather_meta(const int32_t *__restrict__ perm, int64_t n, int h, const float *__restrict__ T,
                              const int64_t *__restrict__ ids_in, float *__restrict__ table,
                              int64_t *__restrict__ row_id, int32_t *__restrict__ inv) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t o = perm[p];
        for (int l = 0; l < h; ++l) table[(int64_t)l * n + p] = T[(int64_t)l * n + o];
        row_id[p] = ids_in ? ids_in[o] : (int64_t)o;
        inv[o] = (int32_t)p;
    }
}

__global__ void k_str_lengths(const int64_t *__restrict__ Soff, const int32_t *__restrict__ perm, int64_t n,
                              int64_t *__restrict__ len) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t o = perm[p];
        len[p] = Soff[o + 1] - Soff[o];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) len[n] = 0;
}

__global__ void k_gather_str(const uint8_t *__restrict__ S, const int64_t *__restrict__ Soff,
                             const int32_t *__restrict__ perm, int64_t n, const int64_t *__restrict__ Loff,
                             uint8_t *__restrict__ SL) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t p = warp; p < n; p += nw) {
        const int32_t o = perm[p];
        const int64_t a = Soff[o], len = Soff[o + 1] - a, d = Loff[p];
        for (int64_t i = lane; i < len; i += 32) SL[d + i] = S[a + i];
    }
}

__global__ void k_piv_rows(int32_t *__restrict__ piv, int64_t cnt, const int32_t *__restrict__ inv) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x)
        if (piv[i] >= 0) piv[i] = inv[piv[i]];
}

template <int W>
void launch_map_str(const Objects &o, const int32_t *perm, const int32_t *pos_node, const int32_t *piv,
                    const int32_t *lpos, const int32_t *lsize, int64_t n, float *Tl, int32_t *node_of,
                    cudaStream_t st) {
    const int chunk = 256;
    k_map_str<W><<<blocks_for(n, chunk), 128, 0, st>>>(o.S, o.Soff, perm, pos_node, piv, lpos, lsize, n, chunk, Tl,
                                                       node_of);
}

}  // namespace

void build_tree(Tree &t, const Objects &objs, const int64_t *d_ids, int metric, int F, int h, int64_t root,
                cudaStream_t st, const float *raw_rows) {
    const int64_t n = objs.n;
    t.metric = metric;
    t.cosine = raw_rows != nullptr;
    t.dim = objs.dim;
    t.F = F;
    t.h = h;
    t.n = n;
    t.lvl_off.assign(h + 2, 0);
    int64_t cnt = 1;
    for (int l = 0; l <= h; ++l) {
        t.lvl_off[l + 1] = t.lvl_off[l] + cnt;
        if (l < h) {
            cnt *= F;
            GTS_REQUIRE(t.lvl_off[l + 1] + cnt <= (int64_t)1 << 28, GTS_EINVAL,
                        "fanout^height too large: more than 2^28 tree nodes");
        }
    }
    const int64_t total_nodes = t.lvl_off[h + 1];
    t.npos.alloc(total_nodes, st);
    t.nsize.alloc(total_nodes, st);
    t.npiv.alloc(total_nodes, st);
    t.nlo.alloc(total_nodes, st);
    t.nhi.alloc(total_nodes, st);
    k_fill_i32<<<blocks_for(total_nodes), kThreads, 0, st>>>(t.npiv.get(), total_nodes, -1);
    {
        int32_t zero = 0, nn32 = (int32_t)n;
        float ninf = -INFINITY, pinf = INFINITY;
        GTS_CUDA(cudaMemcpyAsync(t.npos.get(), &zero, 4, cudaMemcpyHostToDevice, st));
        GTS_CUDA(cudaMemcpyAsync(t.nsize.get(), &nn32, 4, cudaMemcpyHostToDevice, st));
        GTS_CUDA(cudaMemcpyAsync(t.nlo.get(), &ninf, 4, cudaMemcpyHostToDevice, st));
        GTS_CUDA(cudaMemcpyAsync(t.nhi.get(), &pinf, 4, cudaMemcpyHostToDevice, st));
        GTS_CUDA(cudaStreamSynchronize(st));
    }
    t.row_del.alloc(n, st);
    t.row_id.alloc(n, st);
    t.table.alloc((size_t)h * n, st);
    if (n == 0) {
        if (objs.dim == 0) {
            t.Soff.alloc(1, st);
            GTS_CUDA(cudaMemsetAsync(t.Soff.get(), 0, 8, st));
        }
        GTS_CUDA(cudaStreamSynchronize(st));
        return;
    }
    t.max_len = objs.dim == 0 ? objs.max_len : 0;
    DBuf<int32_t> perm(n, st), perm2(n, st), pos_node(n, st), node_of(n, st), inv(n, st);
    DBuf<float> T((size_t)h * n, st);
    DBuf<uint64_t> keys(n, st), keys2(n, st);
    k_iota_i32<<<blocks_for(n), kThreads, 0, st>>>(perm.get(), n);
    k_fill_i32<<<blocks_for(n), kThreads, 0, st>>>(pos_node.get(), n, 0);
    {
        int32_t r32 = (int32_t)root;
        GTS_CUDA(cudaMemcpyAsync(t.npiv.get(), &r32, 4, cudaMemcpyHostToDevice, st));
        GTS_CUDA(cudaStreamSynchronize(st));
    }
    size_t sort_tmp_bytes = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, sort_tmp_bytes, keys.get(), keys2.get(), perm.get(), perm2.get(), n, 0,
                                    64, st);
    DBuf<uint8_t> sort_tmp(sort_tmp_bytes, st);
    int W = 1;   // 64-bit words per pivot pattern (strings)
    for (int l = 0; l < h; ++l) {
        const int64_t nn = t.lvl_off[l + 1] - t.lvl_off[l];
        int32_t *lpos = t.npos.get() + t.lvl_off[l];
        int32_t *lsize = t.nsize.get() + t.lvl_off[l];
        int32_t *lpiv = t.npiv.get() + t.lvl_off[l];
        float *Tl = T.get() + (int64_t)l * n;
        if (l > 0) k_fft_pivot<<<(unsigned)nn, kThreads, 0, st>>>(perm.get(), T.get(), n, l, lpos, lsize, lpiv);
        check_launch("fft pivot");
        if (objs.dim > 0) {
            if (metric == GTS_L2)
                k_map_vec<true><<<blocks_for(n), kThreads, 0, st>>>(objs.X, objs.dim, perm.get(), pos_node.get(), lpiv,
                                                                    n, Tl, node_of.get());
            else
                k_map_vec<false><<<blocks_for(n), kThreads, 0, st>>>(objs.X, objs.dim, perm.get(), pos_node.get(), lpiv,
                                                                     n, Tl, node_of.get());
        } else {
            W = (t.max_len + 63) / 64;
            if (W <= 1) launch_map_str<1>(objs, perm.get(), pos_node.get(), lpiv, lpos, lsize, n, Tl, node_of.get(), st);
            else if (W <= 2) launch_map_str<2>(objs, perm.get(), pos_node.get(), lpiv, lpos, lsize, n, Tl, node_of.get(), st);
            else if (W <= 4) launch_map_str<4>(objs, perm.get(), pos_node.get(), lpiv, lpos, lsize, n, Tl, node_of.get(), st);
            else if (W <= 8) launch_map_str<8>(objs, perm.get(), pos_node.get(), lpiv, lpos, lsize, n, Tl, node_of.get(), st);
            else launch_map_str<16>(objs, perm.get(), pos_node.get(), lpiv, lpos, lsize, n, Tl, node_of.get(), st);
        }
        check_launch("mapping");
        k_keys<<<blocks_for(n), kThreads, 0, st>>>(node_of.get(), Tl, n, keys.get(), perm2.get());
        int node_bits = 0;
        while (((int64_t)1 << node_bits) < nn) ++node_bits;
        size_t tb = sort_tmp_bytes;
        GTS_CUDA(cub::DeviceRadixSort::SortPairs(sort_tmp.get(), tb, keys.get(), keys2.get(), perm2.get(), perm.get(),
                                                 n, 0, 32 + node_bits, st));
        k_children<<<blocks_for(nn * F), kThreads, 0, st>>>(lpos, lsize, nn, F, perm.get(), Tl,
                                                           t.npos.get() + t.lvl_off[l + 1],
                                                           t.nsize.get() + t.lvl_off[l + 1],
                                                           t.nlo.get() + t.lvl_off[l + 1], t.nhi.get() + t.lvl_off[l + 1]);
        k_next_pos_node<<<blocks_for(n), kThreads, 0, st>>>(pos_node.get(), n, lpos, lsize, F);
        check_launch("partitioning");
    }
    // final gather into leaf order
    k_gather_meta<<<blocks_for(n), kThreads, 0, st>>>(perm.get(), n, h, T.get(), d_ids, t.table.get(),
                                                      t.row_id.get(), inv.get());
    k_piv_rows<<<blocks_for(t.lvl_off[h]), kThreads, 0, st>>>(t.npiv.get(), t.lvl_off[h], inv.get());
    k_fill_i64<<<blocks_for(n), kThreads, 0, st>>>(t.row_del.get(), n, kNever);
    if (objs.dim > 0) {
        t.X.alloc((size_t)n * objs.dim, st);
        k_gather_rows<<<blocks_for(n * (int64_t)objs.dim), kThreads, 0, st>>>(objs.X, objs.dim, perm.get(), n,
                                                                             t.X.get());
        if (raw_rows) {   // angular distance: the raw rows in the same (leaf) order
            t.Xr.alloc((size_t)(n > 0 ? n : 1) * objs.dim, st);
            k_gather_rows<<<blocks_for(n * (int64_t)objs.dim), kThreads, 0, st>>>(raw_rows, objs.dim, perm.get(), n,
                                                                                 t.Xr.get());
        }
    } else {
        DBuf<int64_t> len(n + 1, st);
        t.Soff.alloc(n + 1, st);
        k_str_lengths<<<blocks_for(n), kThreads, 0, st>>>(objs.Soff, perm.get(), n, len.get());
        size_t tb = 0;
        cub::DeviceScan::ExclusiveSum(nullptr, tb, len.get(), t.Soff.get(), n + 1, st);
        DBuf<uint8_t> tmp(tb, st);
        GTS_CUDA(cub::DeviceScan::ExclusiveSum(tmp.get(), tb, len.get(), t.Soff.get(), n + 1, st));
        int64_t total = 0;
        GTS_CUDA(cudaMemcpyAsync(&total, t.Soff.get() + n, 8, cudaMemcpyDeviceToHost, st));
        GTS_CUDA(cudaStreamSynchronize(st));
        t.S.alloc(total > 0 ? total : 1, st);
        k_gather_str<<<blocks_for(n * 32), kThreads, 0, st>>>(objs.S, objs.Soff, perm.get(), n, t.Soff.get(),
                                                            t.S.get());
    }
    check_launch("gather");
    GTS_CUDA(cudaStreamSynchronize(st));
    t.persist();
}

}  // namespace gts
