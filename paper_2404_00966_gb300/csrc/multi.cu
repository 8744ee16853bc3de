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
// Column searches run on the device through the single-column entry points,
// the columns concurrently (one host thread and one non-blocking stream per
// column); the combination (unions, threshold tests, selection) is host
// bookkeeping.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <exception>
#include <future>
#include <limits>
#include <memory>
#include <thread>
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
    ColResult() = default;
    ColResult(const ColResult &) = delete;
    ColResult &operator=(const ColResult &) = delete;
    ~ColResult() { gts_result_free(&r); }
};

void raise_status(gts_status s, const char *what) {
    if (s != GTS_OK) throw Error(s, std::string(what) + ": " + gts_last_error());
}

struct Columns {
    std::vector<gts_index *> ix;
    std::vector<int> metric;
    std::vector<cudaStream_t> stream;   // one non-blocking stream per column, owned
    bool distinct = true;               // no index serves two columns
    int64_t nq = 0, n_live = 0;
    gts_query_opts base{};
    int64_t *user_stats = nullptr;      // the caller's counters, filled on return
    // per column, its searches' counters summed (written by its own thread only)
    mutable std::vector<std::array<int64_t, GTS_STATS_LEN>> acc;
    Columns() = default;
    Columns(const Columns &) = delete;
    Columns &operator=(const Columns &) = delete;
    Columns(Columns &&o) noexcept
        : ix(std::move(o.ix)), metric(std::move(o.metric)), stream(std::move(o.stream)), distinct(o.distinct),
          nq(o.nq), n_live(o.n_live), base(o.base), user_stats(o.user_stats), acc(std::move(o.acc)) {
        o.stream.clear();
    }
    ~Columns() {
        for (cudaStream_t st : stream) cudaStreamDestroy(st);
    }
    // column j's options: the caller's, on the column's own stream, its
    // counters into st
    gts_query_opts opts(int j, int32_t flags, int64_t *st) const {
        gts_query_opts o = base;
        o.stream = stream[j];
        o.flags = flags;
        o.stats = st;
        return o;
    }
    void add(int j, const int64_t *st) const {
        for (int s = 0; s < GTS_STATS_LEN; ++s)
            if (st[s] > 0) acc[j][s] += st[s];
    }
    // the caller's counters: the columns' sums, the multi-column answers
    void report(int64_t results) const {
        if (!user_stats) return;
        for (int s = 0; s < GTS_STATS_LEN; ++s) {
            int64_t t = 0;
            for (const auto &a : acc) t += a[s];
            user_stats[s] = t;
        }
        user_stats[GTS_STAT_RESULTS] = results;
        user_stats[GTS_STAT_TABLE_PASS] = -1;
    }
};

// f(j) for every column j, each on a thread of its own (in turn when an
// index serves two columns: an index is used by one thread at a time); the
// first error is rethrown once every column has finished.
template <class F>
void for_columns(const Columns &c, F &&f) {
    const int m = (int)c.ix.size();
    if (m == 1 || !c.distinct) {
        for (int j = 0; j < m; ++j) f(j);
        return;
    }
    std::vector<std::future<void>> fs;
    for (int j = 0; j < m; ++j) fs.push_back(std::async(std::launch::async, [&f, j] { f(j); }));
    std::exception_ptr first;
    for (auto &x : fs) try {
            x.get();
        } catch (...) {
            if (!first) first = std::current_exception();
        }
    if (first) std::rethrow_exception(first);
}

Columns check_columns(gts_index *const *cols, int32_t m, const gts_objects *queries, const gts_query_opts *opts) {
    GTS_REQUIRE(cols != nullptr && queries != nullptr, GTS_EINVAL, "columns or queries NULL");
    GTS_REQUIRE(m >= 1 && m <= 64, GTS_EINVAL, "number of columns must be 1 .. 64");
    Columns c;
    if (opts) c.base = *opts;
    c.user_stats = c.base.stats;
    c.acc.assign(m, std::array<int64_t, GTS_STATS_LEN>{});
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
        GTS_REQUIRE(q.on_device == queries[0].on_device, GTS_EINVAL,
                    "every column's queries must be on the same side");
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
    for (int32_t j = 0; j < m; ++j)
        for (int32_t i = 0; i < j; ++i)
            if (c.ix[i] == c.ix[j]) c.distinct = false;
    for (int32_t j = 0; j < m; ++j) {
        GTS_CUDA(cudaSetDevice(c.ix[j]->device));
        cudaStream_t st = nullptr;
        GTS_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        c.stream.push_back(st);
    }
    return c;
}

int host_threads() {
    static const int t = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    return t;
}

// f(begin, end) over [0, n) in contiguous chunks of at least `grain` items,
// one host thread per chunk (up to host_threads()); the first error is
// rethrown after every chunk has finished.
template <class F>
void parallel_for(int64_t n, int64_t grain, F &&f) {
    const int64_t T = std::min<int64_t>(host_threads(), (n + grain - 1) / grain);
    if (T <= 1) {
        if (n > 0) f((int64_t)0, n);
        return;
    }
    std::vector<std::thread> th;
    std::vector<std::exception_ptr> err(T);
    for (int64_t t = 0; t < T; ++t)
        th.emplace_back([&, t] {
            try {
                f(n * t / T, n * (t + 1) / T);
            } catch (...) {
                err[t] = std::current_exception();
            }
        });
    for (auto &x : th) x.join();
    for (auto &e : err)
        if (e) std::rethrow_exception(e);
}

// Sums of the column distances of the pairs (query pq[p] of `queries`, id
// pid[p]): each column's keys on its own stream, converted to distances in
// its thread, then added in column order from 0.
std::vector<double> pair_sums(const Columns &c, const gts_objects *queries, const std::vector<int32_t> &pq,
                              const std::vector<int64_t> &pid) {
    const int m = (int)c.ix.size();
    const int64_t n = (int64_t)pq.size();
    std::vector<std::vector<double>> dist(m);
    for_columns(c, [&](int j) {
        pair_keys(c.ix[j], &queries[j], pq, pid, dist[j], c.stream[j]);
        if (n > 0) c.acc[j][GTS_STAT_LAUNCHES] += 1;   // k_pair_keys
        double *d = dist[j].data();
        const int metric = c.metric[j];
        parallel_for(n, 1 << 14, [&](int64_t b, int64_t e) {
            for (int64_t p = b; p < e; ++p) d[p] = column_distance(metric, d[p]);
        });
    });
    std::vector<double> sum(n);
    parallel_for(n, 1 << 15, [&](int64_t b, int64_t e) {
        for (int64_t p = b; p < e; ++p) {
            double s = 0.0;
            for (int j = 0; j < m; ++j) s += dist[j][p];
            sum[p] = s;
        }
    });
    return sum;
}

// A host result from per-query answers, allocated for gts_result_free.
struct Answers {
    std::vector<int64_t> off;                 // nq + 1
    std::vector<int64_t> ids;
    std::vector<double> sums;
};

void host_result(gts_result *out, int64_t nq, const Answers &a) {
    const int64_t total = (int64_t)a.ids.size();
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
    std::memcpy(out->offsets, a.off.data(), sizeof(int64_t) * (nq + 1));
    if (total) {
        std::memcpy(out->ids, a.ids.data(), sizeof(int64_t) * total);
        std::memcpy(out->key, a.sums.data(), sizeof(double) * total);
    }
    for (int64_t i = 0; i < total; ++i) out->dist[i] = (float)a.sums[i];
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

// Per query i, the ids all columns returned for it (res[j] rows i), sorted
// and without repeats: cand[off[i] .. off[i] + cnt[i]).
void union_ids(const std::vector<ColResult> &res, int64_t nq, std::vector<int64_t> &off, std::vector<int64_t> &cand,
               std::vector<int64_t> &cnt) {
    off.assign(nq + 1, 0);
    for (const auto &r : res)
        for (int64_t i = 0; i < nq; ++i) off[i + 1] += r.r.offsets[i + 1] - r.r.offsets[i];
    for (int64_t i = 0; i < nq; ++i) off[i + 1] += off[i];
    cand.resize(off[nq]);
    cnt.resize(nq);
    parallel_for(nq, 256, [&](int64_t b, int64_t e) {
        for (int64_t i = b; i < e; ++i) {
            int64_t *w = cand.data() + off[i];
            for (const auto &r : res) w = std::copy(r.r.ids + r.r.offsets[i], r.r.ids + r.r.offsets[i + 1], w);
            int64_t *s = cand.data() + off[i];
            std::sort(s, w);
            cnt[i] = std::unique(s, w) - s;
        }
    });
}

// The pairs (i, cand[off[i] + t]), t < cnt[i], flattened in query order.
void flatten_pairs(const std::vector<int64_t> &off, const std::vector<int64_t> &cand, const std::vector<int64_t> &cnt,
                   std::vector<int64_t> &poff, std::vector<int32_t> &pq, std::vector<int64_t> &pid) {
    const int64_t nq = (int64_t)cnt.size();
    poff.assign(nq + 1, 0);
    for (int64_t i = 0; i < nq; ++i) poff[i + 1] = poff[i] + cnt[i];
    pq.resize(poff[nq]);
    pid.resize(poff[nq]);
    parallel_for(nq, 256, [&](int64_t b, int64_t e) {
        for (int64_t i = b; i < e; ++i)
            for (int64_t t = 0; t < cnt[i]; ++t) {
                pq[poff[i] + t] = (int32_t)i;
                pid[poff[i] + t] = cand[off[i] + t];
            }
    });
}

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
    std::vector<ColResult> res(m);
    for_columns(c, [&](int j) {
        int64_t st[GTS_STATS_LEN] = {};
        const gts_query_opts o = c.opts(j, 0, st);
        raise_status(gts_range(c.ix[j], &queries[j], rcol.data(), &o, &res[j].r), "column range query");
        c.add(j, st);
    });
    std::vector<int64_t> off, cand, cnt, poff, pid;
    std::vector<int32_t> pq;
    union_ids(res, nq, off, cand, cnt);
    flatten_pairs(off, cand, cnt, poff, pq, pid);
    const std::vector<double> sum = pair_sums(c, queries, pq, pid);
    // keep the pairs whose sum is <= r (ascending id within each query)
    std::vector<int64_t> kept(nq);
    parallel_for(nq, 256, [&](int64_t b, int64_t e) {
        for (int64_t i = b; i < e; ++i) {
            int64_t w = poff[i];
            for (int64_t p = poff[i]; p < poff[i + 1]; ++p)
                if (sum[p] <= (double)radii[i]) ++w;
            kept[i] = w - poff[i];
        }
    });
    Answers a;
    a.off.assign(nq + 1, 0);
    for (int64_t i = 0; i < nq; ++i) a.off[i + 1] = a.off[i] + kept[i];
    a.ids.resize(a.off[nq]);
    a.sums.resize(a.off[nq]);
    parallel_for(nq, 256, [&](int64_t b, int64_t e) {
        for (int64_t i = b; i < e; ++i) {
            int64_t w = a.off[i];
            for (int64_t p = poff[i]; p < poff[i + 1]; ++p)
                if (sum[p] <= (double)radii[i]) {
                    a.ids[w] = pid[p];
                    a.sums[w++] = sum[p];
                }
        }
    });
    c.report((int64_t)a.ids.size());
    host_result(out, nq, a);
}

constexpr int64_t kMaxK = 1024;   // the single-column kNN limit

using Best = std::vector<std::pair<double, int64_t>>;   // (sum, id), ascending
using Seen = std::vector<std::pair<int64_t, double>>;   // (id, sum), ascending id

// The first k of n (sum, id) pairs in ascending order.
Best best_k(Best v, int64_t k) {
    const size_t kk = std::min<size_t>((size_t)k, v.size());
    std::partial_sort(v.begin(), v.begin() + kk, v.end());
    v.resize(kk);
    return v;
}

// kNN by random access to every live object (the columns' lists at the k'
// limit did not settle the threshold test), queries in chunks of at most
// 2^24 pairs.
void full_scan(const Columns &c, const gts_objects *queries, const int32_t *k, const std::vector<int64_t> &rows,
               std::vector<Best> &answer) {
    std::vector<int64_t> live;
    const std::vector<int64_t> &loc = c.ix[0]->loc;
    for (int64_t id = 0; id < (int64_t)loc.size(); ++id)
        if (loc[id] != -1) live.push_back(id);
    const int64_t n = (int64_t)live.size();
    const int64_t per = std::max<int64_t>(1, ((int64_t)1 << 24) / std::max<int64_t>(n, 1));
    for (size_t c0 = 0; c0 < rows.size(); c0 += per) {
        const std::vector<int64_t> chunk(rows.begin() + c0, rows.begin() + std::min(rows.size(), c0 + (size_t)per));
        const int64_t nc = (int64_t)chunk.size();
        SubQueries sub(c, queries, chunk);
        std::vector<int32_t> pq(nc * n);
        std::vector<int64_t> pid(nc * n);
        parallel_for(nc, 1, [&](int64_t b, int64_t e) {
            for (int64_t i = b; i < e; ++i)
                for (int64_t p = 0; p < n; ++p) {
                    pq[i * n + p] = (int32_t)i;
                    pid[i * n + p] = live[p];
                }
        });
        const std::vector<double> sum = pair_sums(c, sub.obj.data(), pq, pid);
        parallel_for(nc, 1, [&](int64_t b, int64_t e) {
            for (int64_t i = b; i < e; ++i) {
                Best v(n);
                for (int64_t p = 0; p < n; ++p) v[p] = {sum[i * n + p], live[p]};
                answer[chunk[i]] = best_k(std::move(v), k[chunk[i]]);
            }
        });
    }
}

void multi_knn(const Columns &c, const gts_objects *queries, const int32_t *k, gts_result *out) {
    const int64_t nq = c.nq;
    const int m = (int)c.ix.size();
    GTS_REQUIRE(nq == 0 || k != nullptr, GTS_EINVAL, "k NULL");
    for (int64_t q = 0; q < nq; ++q) GTS_REQUIRE(k[q] >= 1 && k[q] <= kMaxK, GTS_EINVAL, "k must be in 1 .. 1024");
    // k' stops at the single-column limit; a query whose threshold test
    // still fails there takes the full scan
    const int64_t kmax = std::min<int64_t>(std::max<int64_t>(c.n_live, 1), kMaxK);
    std::vector<Seen> seen(nq);
    std::vector<Best> answer(nq);
    std::vector<int64_t> active(nq), full;
    std::vector<int32_t> kp(nq);
    // k' starts at 2k: the threshold test rarely holds at k' = k, since the
    // k-th best sum must fall below the sum of the columns' k'-th distances
    for (int64_t q = 0; q < nq; ++q) {
        active[q] = q;
        kp[q] = (int32_t)std::min<int64_t>(2 * (int64_t)k[q], kmax);
    }
    for (int round = 0; !active.empty(); ++round) {
        const int64_t na = (int64_t)active.size();
        const bool first = round == 0;  // nothing seen yet
        std::unique_ptr<SubQueries> sub;
        const gts_objects *qo = queries;
        if (na != nq) {                 // else every query, in order: no gather
            sub.reset(new SubQueries(c, queries, active));
            qo = sub->obj.data();
        }
        std::vector<int32_t> ka(na);
        for (int64_t i = 0; i < na; ++i) ka[i] = kp[active[i]];
        // sorted access: each column's k' nearest
        std::vector<ColResult> res(m);
        for_columns(c, [&](int j) {
            int64_t st[GTS_STATS_LEN] = {};
            const gts_query_opts o = c.opts(j, GTS_QUERY_KEYS, st);
            raise_status(gts_knn(c.ix[j], &qo[j], ka.data(), &o, &res[j].r), "column kNN query");
            c.add(j, st);
        });
        // T = the sum of the columns' k'-th distances (column order); a column
        // that returned fewer than k' answers, or all live objects, returned
        // every object
        std::vector<double> T(na, 0.0);
        std::vector<char> all_seen(na, 0);
        for (int j = 0; j < m; ++j) {
            const gts_result &r = res[j].r;
            for (int64_t i = 0; i < na; ++i) {
                const int64_t a = r.offsets[i], b = r.offsets[i + 1];
                if (b - a < ka[i] || b - a >= c.n_live) all_seen[i] = 1;
                if (b > a) T[i] += column_distance(c.metric[j], r.key[b - 1]);
            }
        }
        // random access for the ids not seen in an earlier round
        std::vector<int64_t> off, cand, cnt, poff, pid;
        std::vector<int32_t> pq;
        union_ids(res, na, off, cand, cnt);
        if (!first)
            parallel_for(na, 256, [&](int64_t b, int64_t e) {
                for (int64_t i = b; i < e; ++i) {
                    int64_t *s = cand.data() + off[i];
                    const Seen &S = seen[active[i]];
                    int64_t w = 0;
                    size_t t = 0;
                    for (int64_t u = 0; u < cnt[i]; ++u) {
                        while (t < S.size() && S[t].first < s[u]) ++t;
                        if (t < S.size() && S[t].first == s[u]) continue;
                        s[w++] = s[u];
                    }
                    cnt[i] = w;
                }
            });
        flatten_pairs(off, cand, cnt, poff, pq, pid);
        const std::vector<double> sum = pair_sums(c, qo, pq, pid);
        // merge into each query's seen set; settled once the k-th best sum is
        // below T (an unseen object's sum is at least T)
        std::vector<char> settled(na, 0);
        parallel_for(na, 64, [&](int64_t b, int64_t e) {
            for (int64_t i = b; i < e; ++i) {
                const int64_t q = active[i];
                Seen &S = seen[q];
                Seen merged;
                merged.reserve(S.size() + cnt[i]);
                size_t a = 0;
                int64_t t = poff[i];
                while (a < S.size() || t < poff[i + 1]) {
                    if (t == poff[i + 1] || (a < S.size() && S[a].first < pid[t]))
                        merged.push_back(S[a++]);
                    else {
                        merged.emplace_back(pid[t], sum[t]);
                        ++t;
                    }
                }
                S.swap(merged);
                Best v(S.size());
                for (size_t u = 0; u < S.size(); ++u) v[u] = {S[u].second, S[u].first};
                v = best_k(std::move(v), k[q]);
                if (all_seen[i] || ((int64_t)v.size() == k[q] && v.back().first < T[i])) {
                    answer[q] = std::move(v);
                    settled[i] = 1;
                    Seen().swap(S);
                }
            }
        });
        std::vector<int64_t> next;
        for (int64_t i = 0; i < na; ++i) {
            const int64_t q = active[i];
            if (settled[i]) continue;
            if (kp[q] >= kmax) {
                full.push_back(q);
            } else {
                kp[q] = (int32_t)std::min<int64_t>(2 * (int64_t)kp[q], kmax);
                next.push_back(q);
            }
        }
        active.swap(next);
    }
    if (!full.empty()) full_scan(c, queries, k, full, answer);
    Answers a;
    a.off.assign(nq + 1, 0);
    for (int64_t q = 0; q < nq; ++q) a.off[q + 1] = a.off[q] + (int64_t)answer[q].size();
    a.ids.resize(a.off[nq]);
    a.sums.resize(a.off[nq]);
    parallel_for(nq, 1024, [&](int64_t b, int64_t e) {
        for (int64_t q = b; q < e; ++q)
            for (size_t t = 0; t < answer[q].size(); ++t) {
                a.sums[a.off[q] + t] = answer[q][t].first;
                a.ids[a.off[q] + t] = answer[q][t].second;
            }
    });
    c.report((int64_t)a.ids.size());
    host_result(out, nq, a);
}

// Device-resident queries (and their per-query array, on the same side)
// copied to the host once: the combination works on host rows.
struct HostSide {
    std::vector<std::vector<float>> rows;
    std::vector<gts_objects> obj;
    std::vector<uint8_t> per_query;
    const gts_objects *queries;
    const void *pq;
    HostSide(gts_index *const *cols, int32_t m, const gts_objects *q, const void *per, size_t elem)
        : queries(q), pq(per) {
        if (!cols || !q || m < 1 || m > 64 || !q[0].on_device) return;
        GTS_REQUIRE(cols[0] != nullptr, GTS_EINVAL, "column index NULL");
        GTS_CUDA(cudaSetDevice(cols[0]->device));
        rows.resize(m);
        obj.resize(m);
        for (int32_t j = 0; j < m; ++j) {
            GTS_REQUIRE(q[j].on_device && q[j].dim > 0 && q[j].n >= 0 && (q[j].n == 0 || q[j].data), GTS_EINVAL,
                        "multi-column queries: bad device query set");
            const size_t cnt = (size_t)q[j].n * q[j].dim;
            rows[j].resize(cnt + 1);
            if (cnt) GTS_CUDA(cudaMemcpy(rows[j].data(), q[j].data, cnt * 4, cudaMemcpyDefault));
            obj[j] = gts_objects{q[j].n, q[j].dim, 0, rows[j].data(), nullptr};
        }
        queries = obj.data();
        if (per && q[0].n > 0) {
            per_query.resize((size_t)q[0].n * elem);
            GTS_CUDA(cudaMemcpy(per_query.data(), per, per_query.size(), cudaMemcpyDefault));
            pq = per_query.data();
        }
    }
};

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
    return guarded_multi(out, [&] {
        const HostSide h(cols, m, queries, radii, sizeof(float));
        multi_range(check_columns(cols, m, h.queries, opts), h.queries, (const float *)h.pq, out);
    });
}

gts_status gts_multi_knn(gts_index *const *cols, int32_t m, const gts_objects *queries, const int32_t *k,
                         const gts_query_opts *opts, gts_result *out) {
    return guarded_multi(out, [&] {
        const HostSide h(cols, m, queries, k, sizeof(int32_t));
        multi_knn(check_columns(cols, m, h.queries, opts), h.queries, (const int32_t *)h.pq, out);
    });
}

}  // extern "C"
