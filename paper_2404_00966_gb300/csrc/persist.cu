// Index persistence and the merge of sharded answers.
//
// gts_save / gts_load write and read the whole index state -- the node list
// and table list of Section 4.2, the objects in leaf order, the cache list
// and the delete marks of Section 4.4, the id and sequence bookkeeping and the
// tuning -- so a loaded index answers exactly as the saved one did, at the
// same sequence numbers.  The format is a flat sequence of little-endian
// fields (the byte order of every host this library builds for): a magic and
// version, the scalars, then each array as a byte count followed by its bytes.
// Data derived from those arrays on first use (the split bf16 rows, the
// 3-gram counts) is not stored and is rebuilt lazily.
//
// gts_merge_knn / gts_merge_range combine the answers of several indexes over
// disjoint object sets (shards) for the same queries: kNN keeps the first k by
// (FP64 key, global id), the order of Definition 2 that one index over the
// union would produce; range concatenates and sorts by global id (Definition
// 1).  Both are host code and need no device.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "gts_impl.cuh"

namespace gts {

namespace {

constexpr char kMagic[8] = {'G', 'T', 'S', 'I', 'D', 'X', '0', '1'};
// version 2 adds the string tunings and, for the angular distance, the raw rows
constexpr int32_t kVersion = 2;

struct File {
    FILE *f = nullptr;
    ~File() {
        if (f) std::fclose(f);
    }
};

struct Writer {
    FILE *f;
    void raw(const void *p, size_t n) {
        if (n && std::fwrite(p, 1, n, f) != n) throw Error(GTS_EINVAL, "write failed");
    }
    template <class T>
    void pod(const T &v) {
        raw(&v, sizeof(T));
    }
    template <class T>
    void host(const std::vector<T> &v) {
        pod<int64_t>((int64_t)(v.size() * sizeof(T)));
        raw(v.data(), v.size() * sizeof(T));
    }
    // `count` elements of a device buffer
    template <class T>
    void dev(const DBuf<T> &b, size_t count) {
        GTS_REQUIRE(count <= b.n, GTS_EINVAL, "internal: array shorter than its count");
        std::vector<T> h(count);
        if (count) GTS_CUDA(cudaMemcpy(h.data(), b.get(), count * sizeof(T), cudaMemcpyDeviceToHost));
        host(h);
    }
};

struct Reader {
    FILE *f;
    int64_t left;   // bytes not read yet
    void raw(void *p, size_t n) {
        GTS_REQUIRE((int64_t)n <= left, GTS_EINVAL, "index file is truncated");
        if (n && std::fread(p, 1, n, f) != n) throw Error(GTS_EINVAL, "index file is truncated");
        left -= (int64_t)n;
    }
    template <class T>
    T pod() {
        T v;
        raw(&v, sizeof(T));
        return v;
    }
    template <class T>
    std::vector<T> host() {
        const int64_t bytes = pod<int64_t>();
        GTS_REQUIRE(bytes >= 0 && bytes <= left && bytes % (int64_t)sizeof(T) == 0, GTS_EINVAL,
                    "index file is corrupt (array size)");
        std::vector<T> v((size_t)(bytes / (int64_t)sizeof(T)));
        raw(v.data(), (size_t)bytes);
        return v;
    }
    // an array into a new device buffer of at least `min_count` elements
    template <class T>
    int64_t dev(DBuf<T> &b, int64_t min_count, cudaStream_t st) {
        std::vector<T> h = host<T>();
        const int64_t count = (int64_t)h.size();
        b.alloc((size_t)std::max<int64_t>(std::max<int64_t>(count, min_count), 1), st);
        if (count) GTS_CUDA(cudaMemcpyAsync(b.get(), h.data(), count * sizeof(T), cudaMemcpyHostToDevice, st));
        GTS_CUDA(cudaStreamSynchronize(st));
        return count;
    }
};

}  // namespace

}  // namespace gts

using namespace gts;

extern "C" gts_status gts_save(const gts_index *ix, const char *path) {
    try {
        GTS_REQUIRE(ix != nullptr && path != nullptr, GTS_EINVAL, "index or path is NULL");
        GTS_CUDA(cudaSetDevice(ix->device));
        GTS_CUDA(cudaStreamSynchronize(ix->stream));
        const Tree &t = ix->tree;
        const Cache &c = ix->cache;
        const std::string tmp = std::string(path) + ".tmp";
        {
            File fh;
            fh.f = std::fopen(tmp.c_str(), "wb");
            GTS_REQUIRE(fh.f != nullptr, GTS_EINVAL, std::string("cannot open ") + tmp + " for writing");
            Writer w{fh.f};
            w.raw(kMagic, 8);
            w.pod(kVersion);
            w.pod<int32_t>(ix->metric);
            w.pod<int32_t>(ix->dim);
            w.pod<int32_t>(ix->F);
            w.pod<int32_t>(ix->n_pivots_req);
            w.pod<int32_t>(t.h);
            w.pod<int32_t>(t.max_len);
            w.pod<int64_t>(t.n);
            w.pod<int64_t>(t.n_deleted);
            w.pod<int64_t>(ix->next_id);
            w.pod<int64_t>(ix->seq);
            w.pod<int64_t>(ix->rebuild_seq);
            w.pod<int64_t>(ix->n_live);
            w.pod<int64_t>(ix->cache_limit);
            w.pod<int64_t>(ix->rebuilds);
            w.pod<uint64_t>(ix->seed);
            const Tuning &tu = ix->tuning;
            const int32_t tv[8] = {tu.l1_queries, tu.l1_packed, tu.knn_phases, tu.probe_rows,
                                   tu.tc_queries, tu.tuned,      tu.str_chunk,  tu.str_qgram};
            w.raw(tv, sizeof(tv));
            w.host(t.lvl_off);
            const int64_t nodes = t.lvl_off.empty() ? 0 : t.lvl_off.back();
            if (ix->dim > 0) {
                w.dev(t.X, (size_t)t.n * ix->dim);
                if (t.cosine) w.dev(t.Xr, (size_t)t.n * ix->dim);
            } else {
                std::vector<int64_t> soff(t.n + 1, 0);
                if (t.n) GTS_CUDA(cudaMemcpy(soff.data(), t.Soff.get(), (t.n + 1) * 8, cudaMemcpyDeviceToHost));
                w.host(soff);
                w.dev(t.S, (size_t)soff[t.n]);
            }
            w.dev(t.row_id, t.n);
            w.dev(t.table, (size_t)t.h * t.n);
            w.dev(t.row_del, t.n);
            w.dev(t.npos, nodes);
            w.dev(t.nsize, nodes);
            w.dev(t.npiv, nodes);
            w.dev(t.nlo, nodes);
            w.dev(t.nhi, nodes);
            // cache list
            w.pod<int64_t>(c.count);
            w.pod<int32_t>(c.max_len);
            if (ix->dim > 0) {
                w.dev(c.X, (size_t)c.count * ix->dim);
                if (t.cosine) w.dev(c.Xr, (size_t)c.count * ix->dim);
            } else {
                w.host(c.h_Soff);
                w.dev(c.S, (size_t)c.s_bytes);
            }
            w.dev(c.id, c.count);
            w.dev(c.ins, c.count);
            w.dev(c.del, c.count);
            w.host(ix->loc);
            if (std::fflush(fh.f) != 0) throw Error(GTS_EINVAL, "write failed");
        }
        GTS_REQUIRE(std::rename(tmp.c_str(), path) == 0, GTS_EINVAL, std::string("cannot rename ") + tmp);
        return GTS_OK;
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.status;
    } catch (const std::exception &e) {
        set_last_error(e.what());
        return GTS_ENOMEM;
    }
}

extern "C" gts_status gts_load(const char *path, const gts_build_opts *opts, gts_index **out) {
    try {
        GTS_REQUIRE(path != nullptr && out != nullptr, GTS_EINVAL, "path or out is NULL");
        File fh;
        fh.f = std::fopen(path, "rb");
        GTS_REQUIRE(fh.f != nullptr, GTS_EINVAL, std::string("cannot open ") + path);
        std::fseek(fh.f, 0, SEEK_END);
        const long size = std::ftell(fh.f);
        std::fseek(fh.f, 0, SEEK_SET);
        Reader r{fh.f, (int64_t)(size > 0 ? size : 0)};
        char magic[8];
        r.raw(magic, 8);
        GTS_REQUIRE(std::memcmp(magic, kMagic, 8) == 0, GTS_EINVAL, "not a GTS index file");
        const int32_t version = r.pod<int32_t>();
        GTS_REQUIRE(version == 1 || version == kVersion, GTS_EINVAL, "unsupported index file version");
        std::unique_ptr<gts_index> ix(new gts_index());
        ix->metric = r.pod<int32_t>();
        ix->dim = r.pod<int32_t>();
        ix->F = r.pod<int32_t>();
        ix->n_pivots_req = r.pod<int32_t>();
        const int32_t h = r.pod<int32_t>();
        const int32_t max_len = r.pod<int32_t>();
        GTS_REQUIRE(ix->metric >= GTS_EDIT && ix->metric <= (version == 1 ? GTS_L2 : GTS_COS) && ix->dim >= 0 &&
                        (ix->metric == GTS_EDIT) == (ix->dim == 0) && ix->F >= 2 && ix->F <= kMaxFanout && h >= 1 &&
                        h <= kMaxHeight && max_len >= 0 && max_len <= kMaxStrLen,
                    GTS_EINVAL, "index file is corrupt (header)");
        const int64_t n = r.pod<int64_t>();
        const int64_t n_deleted = r.pod<int64_t>();
        ix->next_id = r.pod<int64_t>();
        ix->seq = r.pod<int64_t>();
        ix->rebuild_seq = r.pod<int64_t>();
        ix->n_live = r.pod<int64_t>();
        ix->cache_limit = r.pod<int64_t>();
        ix->rebuilds = r.pod<int64_t>();
        ix->seed = r.pod<uint64_t>();
        GTS_REQUIRE(n >= 0 && n < ((int64_t)1 << 31) && ix->next_id >= n && ix->next_id < ((int64_t)1 << 31) &&
                        n_deleted >= 0 && n_deleted <= n,
                    GTS_EINVAL, "index file is corrupt (sizes)");
        int32_t tv[8] = {0, 0, 0, 0, 0, 0, 256, 64};
        r.raw(tv, version == 1 ? 6 * sizeof(int32_t) : sizeof(tv));
        ix->tuning.l1_queries = tv[0];
        ix->tuning.l1_packed = tv[1];
        ix->tuning.knn_phases = tv[2];
        ix->tuning.probe_rows = tv[3];
        ix->tuning.tc_queries = tv[4];
        ix->tuning.tuned = tv[5];
        ix->tuning.str_chunk = tv[6];
        ix->tuning.str_qgram = tv[7];
        GTS_REQUIRE((tv[6] == 64 || tv[6] == 128 || tv[6] == 256 || tv[6] == 512) && (tv[7] == 0 || tv[7] == 32 || tv[7] == 64),
                    GTS_EINVAL, "index file is corrupt (tuning)");
        // the device work starts here
        ensure_device();
        GTS_CUDA(cudaGetDevice(&ix->device));
        ix->stream = opts ? (cudaStream_t)opts->stream : nullptr;
        if (opts && opts->cache_limit > 0) ix->cache_limit = opts->cache_limit;
        cudaStream_t st = ix->stream;
        Tree &t = ix->tree;
        // the angular distance is an L2 tree over unit vectors with the raw rows beside
        t.metric = ix->metric == GTS_COS ? GTS_L2 : ix->metric;
        t.cosine = ix->metric == GTS_COS;
        t.dim = ix->dim;
        t.F = ix->F;
        t.h = h;
        t.n = n;
        t.max_len = max_len;
        t.n_deleted = n_deleted;
        t.lvl_off = r.host<int64_t>();
        GTS_REQUIRE((int)t.lvl_off.size() == h + 2, GTS_EINVAL, "index file is corrupt (levels)");
        const int64_t nodes = t.lvl_off.back();
        auto expect = [&](int64_t got, int64_t want, const char *what) {
            GTS_REQUIRE(got == want, GTS_EINVAL, std::string("index file is corrupt (") + what + ")");
        };
        if (ix->dim > 0) {
            expect(r.dev(t.X, 1, st), n * ix->dim, "objects");
            if (t.cosine) expect(r.dev(t.Xr, 1, st), n * ix->dim, "raw objects");
        } else {
            std::vector<int64_t> soff = r.host<int64_t>();
            expect((int64_t)soff.size(), n + 1, "string offsets");
            t.Soff.alloc(n + 1, st);
            GTS_CUDA(cudaMemcpyAsync(t.Soff.get(), soff.data(), (n + 1) * 8, cudaMemcpyHostToDevice, st));
            expect(r.dev(t.S, 1, st), soff[n], "strings");
        }
        expect(r.dev(t.row_id, 1, st), n, "ids");
        expect(r.dev(t.table, 1, st), (int64_t)h * n, "table");
        expect(r.dev(t.row_del, 1, st), n, "delete marks");
        expect(r.dev(t.npos, 1, st), nodes, "node positions");
        expect(r.dev(t.nsize, 1, st), nodes, "node sizes");
        expect(r.dev(t.npiv, 1, st), nodes, "pivots");
        expect(r.dev(t.nlo, 1, st), nodes, "node bounds");
        expect(r.dev(t.nhi, 1, st), nodes, "node bounds");
        t.persist();
        Cache &c = ix->cache;
        c.count = r.pod<int64_t>();
        c.max_len = r.pod<int32_t>();
        GTS_REQUIRE(c.count >= 0 && c.count <= ix->next_id, GTS_EINVAL, "index file is corrupt (cache)");
        if (ix->dim > 0) {
            expect(r.dev(c.X, 1, st), c.count * ix->dim, "cache objects");
            if (t.cosine) expect(r.dev(c.Xr, 1, st), c.count * ix->dim, "raw cache objects");
        } else {
            c.h_Soff = r.host<int64_t>();
            GTS_REQUIRE((int64_t)c.h_Soff.size() == (c.count > 0 ? c.count + 1 : (int64_t)c.h_Soff.size()),
                        GTS_EINVAL, "index file is corrupt (cache offsets)");
            c.s_bytes = c.h_Soff.empty() ? 0 : c.h_Soff.back();
            expect(r.dev(c.S, 1, st), c.s_bytes, "cache strings");
            c.Soff.alloc(c.h_Soff.size() + 1, st);
            if (!c.h_Soff.empty())
                GTS_CUDA(cudaMemcpyAsync(c.Soff.get(), c.h_Soff.data(), c.h_Soff.size() * 8, cudaMemcpyHostToDevice,
                                         st));
            c.Soff.persist();
        }
        expect(r.dev(c.id, 1, st), c.count, "cache ids");
        expect(r.dev(c.ins, 1, st), c.count, "cache insert marks");
        expect(r.dev(c.del, 1, st), c.count, "cache delete marks");
        c.cap = c.count;
        c.X.persist();
        c.Xr.persist();
        c.S.persist();
        c.id.persist();
        c.ins.persist();
        c.del.persist();
        ix->loc = r.host<int64_t>();
        expect((int64_t)ix->loc.size(), ix->next_id, "id locations");
        GTS_CUDA(cudaStreamSynchronize(st));
        *out = ix.release();
        return GTS_OK;
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.status;
    } catch (const std::bad_alloc &) {
        set_last_error("host allocation failed");
        return GTS_ENOMEM;
    } catch (const std::exception &e) {
        set_last_error(e.what());
        return GTS_EINVAL;
    }
}

namespace {

gts_status alloc_host_result(gts_result *out, int64_t nq, int64_t total, bool keys) {
    out->nq = nq;
    out->on_device = 0;
    out->priv_ = nullptr;
    out->offsets = (int64_t *)std::malloc(sizeof(int64_t) * (nq + 1));
    out->ids = (int64_t *)std::malloc(sizeof(int64_t) * (total > 0 ? total : 1));
    out->dist = (float *)std::malloc(sizeof(float) * (total > 0 ? total : 1));
    out->key = keys ? (double *)std::malloc(sizeof(double) * (total > 0 ? total : 1)) : nullptr;
    if (!out->offsets || !out->ids || !out->dist || (keys && !out->key)) {
        gts_result_free(out);
        set_last_error("host allocation failed");
        return GTS_ENOMEM;
    }
    return GTS_OK;
}

gts_status check_parts(const gts_result *const *parts, const int64_t *id_base, int32_t n_parts, bool need_keys,
                       int64_t &nq) {
    if (!parts || !id_base || n_parts < 1) {
        set_last_error("parts / id_base NULL or n_parts < 1");
        return GTS_EINVAL;
    }
    nq = parts[0] ? parts[0]->nq : -1;
    for (int32_t p = 0; p < n_parts; ++p) {
        const gts_result *r = parts[p];
        if (!r || r->on_device || r->nq != nq || nq < 0 || !r->offsets || (need_keys && !r->key) || id_base[p] < 0) {
            set_last_error("every part must be a host result of the same query count" +
                           std::string(need_keys ? ", with keys (GTS_QUERY_KEYS)" : "") + ", id_base >= 0");
            return GTS_EINVAL;
        }
    }
    return GTS_OK;
}

}  // namespace

extern "C" gts_status gts_merge_knn(const gts_result *const *parts, const int64_t *id_base, int32_t n_parts,
                                    const int32_t *k, gts_result *out) {
    int64_t nq = 0;
    gts_status s = check_parts(parts, id_base, n_parts, true, nq);
    if (s != GTS_OK) return s;
    if (!k || !out) {
        set_last_error("k or out is NULL");
        return GTS_EINVAL;
    }
    struct Ent {
        double key;
        int64_t id;
        float dist;
    };
    std::vector<std::vector<Ent>> best((size_t)nq);
    int64_t total = 0;
    for (int64_t q = 0; q < nq; ++q) {
        if (k[q] < 1) {
            set_last_error("k must be >= 1");
            return GTS_EINVAL;
        }
        std::vector<Ent> &v = best[(size_t)q];
        for (int32_t p = 0; p < n_parts; ++p) {
            const gts_result *r = parts[p];
            for (int64_t i = r->offsets[q]; i < r->offsets[q + 1]; ++i)
                v.push_back(Ent{r->key[i], r->ids[i] + id_base[p], r->dist[i]});
        }
        std::sort(v.begin(), v.end(),
                  [](const Ent &a, const Ent &b) { return a.key < b.key || (a.key == b.key && a.id < b.id); });
        if ((int64_t)v.size() > k[q]) v.resize((size_t)k[q]);
        total += (int64_t)v.size();
    }
    s = alloc_host_result(out, nq, total, true);
    if (s != GTS_OK) return s;
    int64_t o = 0;
    for (int64_t q = 0; q < nq; ++q) {
        out->offsets[q] = o;
        for (const Ent &e : best[(size_t)q]) {
            out->key[o] = e.key;
            out->ids[o] = e.id;
            out->dist[o] = e.dist;
            ++o;
        }
    }
    out->offsets[nq] = o;
    return GTS_OK;
}

extern "C" gts_status gts_merge_range(const gts_result *const *parts, const int64_t *id_base, int32_t n_parts,
                                      gts_result *out) {
    int64_t nq = 0;
    gts_status s = check_parts(parts, id_base, n_parts, false, nq);
    if (s != GTS_OK) return s;
    if (!out) {
        set_last_error("out is NULL");
        return GTS_EINVAL;
    }
    int64_t total = 0;
    for (int32_t p = 0; p < n_parts; ++p) total += parts[p]->offsets[nq];
    s = alloc_host_result(out, nq, total, false);
    if (s != GTS_OK) return s;
    std::vector<std::pair<int64_t, float>> v;
    int64_t o = 0;
    for (int64_t q = 0; q < nq; ++q) {
        v.clear();
        for (int32_t p = 0; p < n_parts; ++p) {
            const gts_result *r = parts[p];
            for (int64_t i = r->offsets[q]; i < r->offsets[q + 1]; ++i)
                v.push_back({r->ids[i] + id_base[p], r->dist[i]});
        }
        std::sort(v.begin(), v.end(),
                  [](const std::pair<int64_t, float> &a, const std::pair<int64_t, float> &b) { return a.first < b.first; });
        out->offsets[q] = o;
        for (auto &e : v) {
            out->ids[o] = e.first;
            out->dist[o] = e.second;
            ++o;
        }
    }
    out->offsets[nq] = o;
    return GTS_OK;
}
