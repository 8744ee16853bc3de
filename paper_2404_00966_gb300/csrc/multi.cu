// Multi-column queries (Section 5.2, closing remark): one index per column
// over the same object ids, the distance of an object the sum of its column
// distances (a sum of metrics is a metric), and a query combined from the
// columns' own answers.
//
//  * Range (pigeonhole principle): when the m column distances sum to at most
//    r, at least one of them is at most r / m.  The union of the columns'
//    range answers at radius r / m (rounded up) holds every answer; each
//    candidate's sum is then computed from all columns and kept when <= r.
//  * kNN (Fagin's threshold algorithm): sorted access is each column's k'
//    nearest, random access the FP64 key of a (query, object) pair in a
//    column.  An object that no column returned is at least as far as each
//    column's k'-th answer in every column, so its sum is at least T, the sum
//    of those k'-th distances; the search stops once the k-th best seen sum is
//    below T (or a column returned every object), else k' doubles.
//
// Every sum is the FP64 column distances (L2: sqrt of the FP64 key; L1: the
// key; angular: the C library's acos(1 - key)) added in column order from 0.
// Column searches run on the device through the single-column entry points;
// the combination (unions, threshold tests, selection) is host bookkeeping.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <unordered_map>
#include <vector>

#include "gts_impl.cuh"

namespace gts {
namespace {

double column_distance(int metric, double key) {
    if (metric == GTS_L2) return std::sqrt(key);
    if (metric == GTS_COS) return std::acos(1.0 - key);
    return key;
}

// Owns one column's host result.
struct ColResult {
    gts_result r{};
    ~ColResult() { gts_result_free(&r); }
};

void raise_status(gts_status s, const char *what) {
    if (s != GTS_OK) throw Error(s, std::string(what) + ": " + gts_last_error());
}

struct Columns {
    std::vector<gts_index *> ix;
    std::vector<int> metric;
    int64_t nq = 0, n_live = 0;
    gts_query_opts base{};
};

Columns check_columns(gts_index *const *cols, int32_t m, const gts_objects *queries, const gts_query_opts *opts) {
    GTS_REQUIRE(cols != nullptr && queries != nullptr, GTS_EINVAL, "columns or queries NULL");
    GTS_REQUIRE(m >= 1 && m <= 64, GTS_EINVAL, "number of columns must be 1 .. 64");
    Columns c;
    if (opts) c.base = *opts;
    GTS_REQUIRE(c.base.seq == nullptr, GTS_EINVAL, "multi-column queries run on the current state (seq must be NULL)");
    GTS_REQUIRE(c.base.result_on_device == 0, GTS_EINVAL, "multi-column results are host memory");
    c.base.stats = nullptr;
    c.base.stage_ms = nullptr;
    c.base.flags = 0;
    for (int32_t j = 0; j < m; ++j) {
        gts_index *ix = cols[j];
        GTS_REQUIRE(ix != nullptr, GTS_EINVAL, "column index NULL");
        GTS_REQUIRE(ix->dim > 0 && ix->metric != GTS_EDIT, GTS_EINVAL,
                    "multi-column queries take vector columns (L1, L2, angular)");
        const gts_objects &q = queries[j];
        GTS_REQUIRE(q.on_device == 0, GTS_EINVAL, "multi-column queries are host rows");
        GTS_REQUIRE(q.dim == ix->dim, GTS_EINVAL, "column " + std::to_string(j) + ": query dim does not match");
        GTS_REQUIRE(q.n >= 0 && (q.n == 0 || q.data != nullptr), GTS_EINVAL, "column queries: bad n or NULL data");
        if (j == 0) {
            c.nq = q.n;
            c.n_live = ix->n_live;
        }
        GTS_REQUIRE(q.n == c.nq, GTS_EINVAL, "every column needs the same number of queries");
        GTS_REQUIRE(ix->n_live == c.n_live, GTS_EINVAL, "columns hold different numbers of live objects");
        c.ix.push_back(ix);
        c.metric.push_back(ix->metric);
    }
    return c;
}

// Sums of the column distances of the pairs (query pq[j] of `queries`, id pid[j]).
std::vector<double> pair_sums(const Columns &c, const gts_objects *queries, const std::vector<int32_t> &pq,
                              const std::vector<int64_t> &pid) {
    std::vector<double> sum(pq.size(), 0.0), keys;
    for (size_t j = 0; j < c.ix.size(); ++j) {
        pair_keys(c.ix[j], &queries[j], pq, pid, keys);
        for (size_t p = 0; p < pq.size(); ++p) sum[p] += column_distance(c.metric[j], keys[p]);
    }
    return sum;
}

void host_result(gts_result *out, int64_t nq, const std::vector<int64_t> &off, const std::vector<int64_t> &ids,
                 const std::vector<double> &sums) {
    const int64_t total = (int64_t)ids.size();
    out->nq = nq;
    out->on_device = 0;
    out->priv_ = nullptr;
    out->offsets = (int64_t *)std::malloc(sizeof(int64_t) * (nq + 1));
    out->ids = (int64_t *)std::malloc(sizeof(int64_t) * (total > 0 ? total : 1));
    out->dist = (float *)std::malloc(sizeof(float) * (total > 0 ? total : 1));
    out->key = (double *)std::malloc(sizeof(double) * (total > 0 ? total : 1));
    if (!out->offsets || !out->ids || !out->dist || !out->key) {
        gts_result_free(out);
        throw Error(GTS_ENOMEM, "host allocation failed");
    }
    std::memcpy(out->offsets, off.data(), sizeof(int64_t) * (nq + 1));
    for (int64_t i = 0; i < total; ++i) {
        out->ids[i] = ids[i];
        out->dist[i] = (float)sums[i];
        out->key[i] = sums[i];
    }
}

// Rows `rows` of every column's queries, gathered on the host.
struct SubQueries {
    std::vector<std::vector<float>> data;
    std::vector<gts_objects> obj;
    SubQueries(const Columns &c, const gts_objects *queries, const std::vector<int64_t> &rows) {
        const size_t m = c.ix.size();
        data.resize(m);
        obj.resize(m);
        for (size_t j = 0; j < m; ++j) {
            const int d = queries[j].dim;
            const float *src = (const float *)queries[j].data;
            data[j].resize(rows.size() * (size_t)d + 1);
            for (size_t i = 0; i < rows.size(); ++i)
                std::memcpy(&data[j][i * d], src + rows[i] * d, sizeof(float) * d);
            obj[j] = gts_objects{(int64_t)rows.size(), d, 0, data[j].data(), nullptr};
        }
    }
};

void multi_range(const Columns &c, const gts_objects *queries, const float *radii, gts_result *out) {
    const int64_t nq = c.nq;
    const int m = (int)c.ix.size();
    GTS_REQUIRE(nq == 0 || radii != nullptr, GTS_EINVAL, "radii NULL");
    std::vector<float> rcol(nq > 0 ? nq : 1);
    for (int64_t q = 0; q < nq; ++q) {
        GTS_REQUIRE(std::isfinite(radii[q]) && radii[q] >= 0.f, GTS_EINVAL, "radii must be finite and >= 0");
        // r / m rounded up to FP32, with a relative margin far above the FP64
        // rounding of an m-term sum, so the column radius never falls below
        // the pigeonhole bound
        const double t = (double)radii[q] / m * (1.0 + 1e-12);
        float f = (float)t;
        if ((double)f < t) f = std::nextafter(f, std::numeric_limits<float>::infinity());
        rcol[q] = f;
    }
    // union of the column answers, per query ascending id
    std::vector<std::vector<int64_t>> cand(nq);
    for (int j = 0; j < m; ++j) {
        ColResult r;
        raise_status(gts_range(c.ix[j], &queries[j], rcol.data(), &c.base, &r.r), "column range query");
        for (int64_t q = 0; q < nq; ++q)
            cand[q].insert(cand[q].end(), r.r.ids + r.r.offsets[q], r.r.ids + r.r.offsets[q + 1]);
    }
    std::vector<int32_t> pq;
    std::vector<int64_t> pid;
    for (int64_t q = 0; q < nq; ++q) {
        std::sort(cand[q].begin(), cand[q].end());
        cand[q].erase(std::unique(cand[q].begin(), cand[q].end()), cand[q].end());
        for (int64_t id : cand[q]) {
            pq.push_back((int32_t)q);
            pid.push_back(id);
        }
    }
    const std::vector<double> sum = pair_sums(c, queries, pq, pid);
    std::vector<int64_t> off(nq + 1, 0), ids;
    std::vector<double> sums;
    for (size_t p = 0; p < pq.size(); ++p)
        if (sum[p] <= (double)radii[pq[p]]) {
            ids.push_back(pid[p]);
            sums.push_back(sum[p]);
            ++off[pq[p] + 1];
        }
    for (int64_t q = 0; q < nq; ++q) off[q + 1] += off[q];
    host_result(out, nq, off, ids, sums);
}

constexpr int64_t kMaxK = 1024;   // the single-column kNN limit

// kNN by random access to every live object (the columns' lists at the k'
// limit did not settle the threshold test), queries in chunks of at most
// 2^24 pairs.
void full_scan(const Columns &c, const gts_objects *queries, const int32_t *k, const std::vector<int64_t> &rows,
               std::vector<std::vector<std::pair<double, int64_t>>> &answer) {
    std::vector<int64_t> live;
    const std::vector<int64_t> &loc = c.ix[0]->loc;
    for (int64_t id = 0; id < (int64_t)loc.size(); ++id)
        if (loc[id] != -1) live.push_back(id);
    const int64_t n = (int64_t)live.size();
    const int64_t per = std::max<int64_t>(1, ((int64_t)1 << 24) / std::max<int64_t>(n, 1));
    for (size_t c0 = 0; c0 < rows.size(); c0 += per) {
        const std::vector<int64_t> chunk(rows.begin() + c0, rows.begin() + std::min(rows.size(), c0 + (size_t)per));
        SubQueries sub(c, queries, chunk);
        std::vector<int32_t> pq;
        std::vector<int64_t> pid;
        pq.reserve(chunk.size() * n);
        pid.reserve(chunk.size() * n);
        for (size_t i = 0; i < chunk.size(); ++i)
            for (int64_t id : live) {
                pq.push_back((int32_t)i);
                pid.push_back(id);
            }
        const std::vector<double> sum = pair_sums(c, sub.obj.data(), pq, pid);
        for (size_t i = 0; i < chunk.size(); ++i) {
            const int64_t q = chunk[i];
            std::vector<std::pair<double, int64_t>> v(n);
            for (int64_t p = 0; p < n; ++p) v[p] = {sum[i * n + p], live[p]};
            const size_t kk = std::min<size_t>((size_t)k[q], v.size());
            std::partial_sort(v.begin(), v.begin() + kk, v.end());
            v.resize(kk);
            answer[q] = std::move(v);
        }
    }
}

void multi_knn(const Columns &c, const gts_objects *queries, const int32_t *k, gts_result *out) {
    const int64_t nq = c.nq;
    const int m = (int)c.ix.size();
    GTS_REQUIRE(nq == 0 || k != nullptr, GTS_EINVAL, "k NULL");
    for (int64_t q = 0; q < nq; ++q) GTS_REQUIRE(k[q] >= 1 && k[q] <= kMaxK, GTS_EINVAL, "k must be in 1 .. 1024");
    // k' stops at the single-column limit; a query whose threshold test
    // still fails there takes the full scan below
    const int64_t kmax = std::min<int64_t>(std::max<int64_t>(c.n_live, 1), kMaxK);
    std::vector<int64_t> full;
    std::vector<std::unordered_map<int64_t, double>> seen(nq);
    std::vector<std::vector<std::pair<double, int64_t>>> answer(nq);
    std::vector<int64_t> active(nq);
    std::vector<int32_t> kp(nq);
    for (int64_t q = 0; q < nq; ++q) {
        active[q] = q;
        kp[q] = (int32_t)std::min<int64_t>(k[q], kmax);
    }
    gts_query_opts o = c.base;
    o.flags = GTS_QUERY_KEYS;
    while (!active.empty()) {
        const int64_t na = (int64_t)active.size();
        SubQueries sub(c, queries, active);
        std::vector<int32_t> ka(na);
        for (int64_t i = 0; i < na; ++i) ka[i] = kp[active[i]];
        // sorted access: each column's k' nearest; T = sum of the k'-th distances
        std::vector<double> T(na, 0.0);
        std::vector<char> all_seen(na, 0);
        std::vector<int32_t> pq;
        std::vector<int64_t> pid;
        for (int j = 0; j < m; ++j) {
            ColResult r;
            raise_status(gts_knn(c.ix[j], &sub.obj[j], ka.data(), &o, &r.r), "column kNN query");
            for (int64_t i = 0; i < na; ++i) {
                const int64_t a = r.r.offsets[i], b = r.r.offsets[i + 1];
                if (b - a < ka[i] || b - a >= c.n_live) all_seen[i] = 1;
                if (b > a) T[i] += column_distance(c.metric[j], r.r.key[b - 1]);
                auto &s = seen[active[i]];
                for (int64_t p = a; p < b; ++p)
                    if (s.emplace(r.r.ids[p], -1.0).second) {   // first sight: random access below
                        pq.push_back((int32_t)i);
                        pid.push_back(r.r.ids[p]);
                    }
            }
        }
        // random access: the full sum of every object seen for the first time
        const std::vector<double> sum = pair_sums(c, sub.obj.data(), pq, pid);
        for (size_t p = 0; p < pq.size(); ++p) seen[active[pq[p]]][pid[p]] = sum[p];
        std::vector<int64_t> next;
        for (int64_t i = 0; i < na; ++i) {
            const int64_t q = active[i];
            std::vector<std::pair<double, int64_t>> v;
            v.reserve(seen[q].size());
            for (const auto &e : seen[q]) v.emplace_back(e.second, e.first);
            const size_t kk = std::min<size_t>((size_t)k[q], v.size());
            std::partial_sort(v.begin(), v.begin() + kk, v.end());
            v.resize(kk);
            if (all_seen[i] || (kk == (size_t)k[q] && v.back().first < T[i])) {
                answer[q] = std::move(v);
            } else if (kp[q] >= kmax) {
                full.push_back(q);
            } else {
                kp[q] = (int32_t)std::min<int64_t>(2 * (int64_t)kp[q], kmax);
                next.push_back(q);
            }
        }
        active.swap(next);
    }
    if (!full.empty()) full_scan(c, queries, k, full, answer);
    std::vector<int64_t> off(nq + 1, 0), ids;
    std::vector<double> sums;
    for (int64_t q = 0; q < nq; ++q) {
        for (const auto &e : answer[q]) {
            sums.push_back(e.first);
            ids.push_back(e.second);
        }
        off[q + 1] = (int64_t)ids.size();
    }
    host_result(out, nq, off, ids, sums);
}

template <class F>
gts_status guarded_multi(gts_result *out, F &&f) {
    try {
        GTS_REQUIRE(out != nullptr, GTS_EINVAL, "out NULL");
        std::memset(out, 0, sizeof(*out));
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
    }
}

}  // namespace
}  // namespace gts

using namespace gts;

extern "C" {

gts_status gts_multi_range(gts_index *const *cols, int32_t m, const gts_objects *queries, const float *radii,
                           const gts_query_opts *opts, gts_result *out) {
    return guarded_multi(out, [&] { multi_range(check_columns(cols, m, queries, opts), queries, radii, out); });
}

gts_status gts_multi_knn(gts_index *const *cols, int32_t m, const gts_objects *queries, const int32_t *k,
                         const gts_query_opts *opts, gts_result *out) {
    return guarded_multi(out, [&] { multi_knn(check_columns(cols, m, queries, opts), queries, k, out); });
}

}  // extern "C"
