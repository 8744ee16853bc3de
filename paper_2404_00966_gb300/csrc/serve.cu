// Continuous-batching request loop over one index.
//
// Requests (one query each: a range query with its radius or a kNN query
// with its k) are submitted one at a time from any host thread.  A pool of
// worker threads, each with its own CUDA stream, repeatedly takes the oldest
// pending requests of one kind, as many as fit both the batch size and the
// admission budget, and runs them as one batched search (the same device
// path as gts_range / gts_knn).  Requests that arrive while batches are on
// the GPU are admitted into the next batch a worker forms, so several batches
// overlap on the device.
//
// Admission: every request carries a projected device footprint -- an upper
// bound of the candidate rows it can produce times the bytes one candidate
// occupies in the search's tables -- and a request is admitted only while the
// projections of all requests in flight fit the result budget (the oldest
// request is always admitted when nothing is in flight).  Each batch's own
// intermediate tables are further bounded by the two-stage scheduler with
// memory_budget.
//
// The projection is the descent of Section 5.1 run on the host over the
// top levels of the tree (a snapshot taken when the server starts, at most
// 4096 pivots), evaluating at most 64 pivots per request: the request's
// distances to the pivots of the surviving nodes (FP64, or exact edit
// distance), the node test of Lemma 1 on every child's [lo, hi] interval
// (with the radius, or for kNN with the k-th smallest distance to a visible
// pivot evaluated so far, which bounds d_k from above since the pivots are
// objects), and the row counts of the nodes that survive at the deepest level
// reached.
// Every candidate row of the full search lies in one of those nodes (or in
// the cache list), so the sum bounds the candidates from above.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <string>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "gts_impl.cuh"

struct gts_server;

namespace gts {
namespace {

constexpr int64_t kCandidateBytes = 37;   // (query, row, distance, keep, key) in the candidate tables

double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
    int64_t ticket;
    int32_t kind;    // 0 range, 1 kNN
    float radius;
    int32_t k;
    std::vector<uint8_t> payload;   // float32[dim] or string bytes
    int64_t proj;
    double t_submit;
};

struct Done {
    std::vector<int64_t> ids;
    std::vector<float> dist;
    double latency_ms;
    gts_status status;
};

// Host snapshot of the tree's top `levels` pivot levels (Section 4.2 node
// list, Eq. 1 numbering) for the admission projection.
struct TopLevels {
    int levels = 0, F = 0, dim = 0, metric = 0;
    bool cosine = false;                   // angular distance: pivots are unit vectors, distances chords
    std::vector<int64_t> lvl_off;          // first node of levels 0 .. levels
    std::vector<float> pv;                 // pivot vectors of levels < levels, [node, dim]
    std::vector<std::string> ps;           // pivot strings
    std::vector<uint8_t> has_piv, piv_live;
    std::vector<float> lo, hi;             // every node of levels 1 .. levels
    std::vector<int64_t> size;             // every node of levels 0 .. levels
    int64_t cache_rows = 0, n_live = 0;
};

double host_distance(const TopLevels &t, int64_t node, const uint8_t *q, int64_t len) {
    if (t.dim > 0) {
        const float *x = &t.pv[(size_t)node * t.dim];
        const float *qq = reinterpret_cast<const float *>(q);
        double s = 0.0;
        for (int i = 0; i < t.dim; ++i) {
            const double d = (double)qq[i] - (double)x[i];
            s += t.metric == GTS_L2 ? d * d : std::fabs(d);
        }
        return t.metric == GTS_L2 ? std::sqrt(s) : s;
    }
    const std::string &b = t.ps[(size_t)node];   // unit-cost Levenshtein, two rows
    const int64_t lb = (int64_t)b.size();
    std::vector<int64_t> prev(lb + 1), cur(lb + 1);
    for (int64_t j = 0; j <= lb; ++j) prev[j] = j;
    for (int64_t i = 1; i <= len; ++i) {
        cur[0] = i;
        for (int64_t j = 1; j <= lb; ++j)
            cur[j] = std::min(std::min(prev[j] + 1, cur[j - 1] + 1),
                              prev[j - 1] + (q[i - 1] != (uint8_t)b[(size_t)j - 1] ? 1 : 0));
        std::swap(prev, cur);
    }
    return (double)prev[lb];
}

// Upper bound of the candidate rows of one request (see the file comment):
// the descent of Algorithm 4 / 5 over the snapshot levels, evaluating only the
// pivots of the nodes that survive (at most kMaxEvals of them per request; past
// that, or where no radius bound exists yet, the rows of the current frontier
// are the bound).
constexpr int kMaxEvals = 64;

int64_t project_rows(const TopLevels &t, const uint8_t *q, int64_t len, int32_t kind, double param) {
    if (t.levels == 0) return t.n_live + t.cache_rows;
    std::vector<float> unit;
    if (t.cosine) {   // the descent runs on chords between unit vectors, as the tree does
        const float *qq = reinterpret_cast<const float *>(q);
        double s = 0.0;
        for (int i = 0; i < t.dim; ++i) s += (double)qq[i] * (double)qq[i];
        if (!(s > 0.0)) return t.n_live + t.cache_rows;
        const double inv = 1.0 / std::sqrt(s);
        unit.resize(t.dim);
        for (int i = 0; i < t.dim; ++i) unit[i] = (float)((double)qq[i] * inv);
        q = reinterpret_cast<const uint8_t *>(unit.data());
        if (kind == 0) param = std::sqrt(2.0 * (1.0 - std::cos(std::min(param, 3.14159265358979323846)))) + 1e-6;
    }
    std::vector<int64_t> frontier{0}, next;   // node indices within the current level
    std::vector<double> live;                 // exact distances to the visible pivots evaluated so far
    std::vector<double> dnode;
    auto rows_of = [&](int l) {
        int64_t rows = t.cache_rows;
        for (int64_t c : frontier) rows += t.size[t.lvl_off[l] + c];
        return rows;
    };
    int evals = 0;
    const size_t k = kind == 1 ? (size_t)param : 0;
    for (int l = 0; l < t.levels; ++l) {
        if (evals + (int)frontier.size() > kMaxEvals) return rows_of(l);
        dnode.assign(frontier.size(), 0.0);
        for (size_t i = 0; i < frontier.size(); ++i) {
            const int64_t v = t.lvl_off[l] + frontier[i];
            if (!t.has_piv[v]) continue;
            dnode[i] = host_distance(t, v, q, len);
            ++evals;
            if (t.piv_live[v]) live.push_back(dnode[i]);
        }
        double r;
        if (kind == 0) {
            r = t.dim > 0 ? param : std::floor(param);
        } else {
            if (live.size() < k) return rows_of(l);   // no bound on d_k yet: nothing can be pruned
            std::vector<double> tmp(live);
            std::nth_element(tmp.begin(), tmp.begin() + (k - 1), tmp.end());
            r = tmp[k - 1];   // the k-th smallest distance to an object evaluated so far >= d_k
        }
        next.clear();
        for (size_t i = 0; i < frontier.size(); ++i) {
            const int64_t node = frontier[i], v = t.lvl_off[l] + node;
            if (!t.has_piv[v]) continue;   // an empty node has no rows
            const double dq = dnode[i];
            for (int j = 0; j < t.F; ++j) {
                const int64_t c = node * t.F + j, cv = t.lvl_off[l + 1] + c;
                if (t.size[cv] == 0) continue;
                const double lo = t.lo[cv - 1], hi = t.hi[cv - 1];   // lo/hi hold levels >= 1
                // at least the search's own FP32 slack, 4 (D + 8) 2^-24 of the same terms
                const double rel = std::max(1e-5, 8.0 * (t.dim + 8) * 5.9604644775390625e-8);
                const double slack = t.dim > 0 ? rel * (std::fabs(dq) + r + std::fabs(lo) + std::fabs(hi)) + 1e-6 : 0.0;
                if (dq - r <= hi + slack && dq + r >= lo - slack) next.push_back(c);
            }
        }
        frontier.swap(next);
    }
    return rows_of(t.levels);
}

}  // namespace
}  // namespace gts

struct gts_server {
    gts_index *ix = nullptr;
    gts_serve_opts opts;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<gts::Request> pending;
    std::unordered_map<int64_t, gts::Done> done;
    int64_t next_ticket = 1;
    bool stopping = false;
    int64_t in_flight = 0;        // projected bytes of admitted requests
    int64_t max_in_flight = 0;
    int64_t batches = 0, requests_run = 0, max_batch_seen = 0;
    int64_t proj_total = 0, proj_below_worst = 0;
    gts::TopLevels top;
    std::vector<std::thread> workers;
};

namespace gts {
namespace {

void worker_loop(gts_server *sv, int wid) {
    cudaSetDevice(sv->ix->device);
    cudaStream_t st;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    std::vector<Request> batch;
    const int dim = sv->ix->dim;
    (void)wid;
    for (;;) {
        batch.clear();
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            sv->cv_work.wait(lk, [&] { return sv->stopping || !sv->pending.empty(); });
            if (sv->pending.empty() && sv->stopping) break;
            // oldest-first batch of one kind, within the batch size and the admission budget
            const int32_t kind = sv->pending.front().kind;
            for (auto it = sv->pending.begin(); it != sv->pending.end() && (int)batch.size() < sv->opts.max_batch;) {
                if (it->kind != kind) {
                    ++it;
                    continue;
                }
                const bool fits = sv->in_flight + it->proj <= sv->opts.result_budget;
                if (!fits && !(sv->in_flight == 0 && batch.empty())) break;
                sv->in_flight += it->proj;
                batch.push_back(std::move(*it));
                it = sv->pending.erase(it);
            }
            // a batch above the quantum keeps a multiple of it; the newest
            // requests go back to the head of the queue, in order
            const size_t bq = sv->opts.batch_quantum > 1 ? (size_t)sv->opts.batch_quantum : 0;
            if (bq && batch.size() > bq && batch.size() % bq != 0) {
                const size_t keep = batch.size() / bq * bq;
                for (size_t i = batch.size(); i-- > keep;) {
                    sv->in_flight -= batch[i].proj;
                    sv->pending.push_front(std::move(batch[i]));
                }
                batch.resize(keep);
                sv->cv_work.notify_one();
            }
            if (sv->in_flight > sv->max_in_flight) sv->max_in_flight = sv->in_flight;
            if (batch.empty()) {   // nothing admissible yet: wait for a batch to finish
                sv->cv_done.wait(lk);
                continue;
            }
            sv->batches += 1;
            sv->requests_run += (int64_t)batch.size();
            if ((int64_t)batch.size() > sv->max_batch_seen) sv->max_batch_seen = (int64_t)batch.size();
        }
        // ---- marshal the batch (host buffers) and run it on this worker's stream
        const int64_t nb = (int64_t)batch.size();
        gts_objects qo;
        std::memset(&qo, 0, sizeof(qo));
        std::vector<float> qv;
        std::vector<uint8_t> qs;
        std::vector<int64_t> qoff;
        if (dim > 0) {
            qv.resize((size_t)nb * dim);
            for (int64_t i = 0; i < nb; ++i) std::memcpy(&qv[(size_t)i * dim], batch[i].payload.data(), (size_t)dim * 4);
            qo.n = nb;
            qo.dim = dim;
            qo.data = qv.data();
        } else {
            qoff.resize(nb + 1, 0);
            for (int64_t i = 0; i < nb; ++i) qoff[i + 1] = qoff[i] + (int64_t)batch[i].payload.size();
            qs.resize(qoff[nb] > 0 ? qoff[nb] : 1);
            for (int64_t i = 0; i < nb; ++i)
                if (!batch[i].payload.empty())
                    std::memcpy(&qs[qoff[i]], batch[i].payload.data(), batch[i].payload.size());
            qo.n = nb;
            qo.dim = 0;
            qo.data = qs.data();
            qo.offsets = qoff.data();
        }
        gts_query_opts o;
        std::memset(&o, 0, sizeof(o));
        o.stream = st;
        o.precision = sv->opts.precision;
        o.memory_budget = sv->opts.memory_budget;
        gts_result res;
        std::memset(&res, 0, sizeof(res));
        gts_status s;
        if (batch[0].kind == 0) {
            std::vector<float> r(nb);
            for (int64_t i = 0; i < nb; ++i) r[i] = batch[i].radius;
            s = gts_range(sv->ix, &qo, r.data(), &o, &res);
        } else {
            std::vector<int32_t> k(nb);
            for (int64_t i = 0; i < nb; ++i) k[i] = batch[i].k;
            s = gts_knn(sv->ix, &qo, k.data(), &o, &res);
        }
        const double t_done = now_ms();
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            for (int64_t i = 0; i < nb; ++i) {
                Done dn;
                dn.status = s;
                dn.latency_ms = t_done - batch[i].t_submit;
                if (s == GTS_OK) {
                    const int64_t a = res.offsets[i], b = res.offsets[i + 1];
                    dn.ids.assign(res.ids + a, res.ids + b);
                    dn.dist.assign(res.dist + a, res.dist + b);
                }
                sv->done.emplace(batch[i].ticket, std::move(dn));
                sv->in_flight -= batch[i].proj;
            }
        }
        if (s == GTS_OK) gts_result_free(&res);
        sv->cv_done.notify_all();
        sv->cv_work.notify_all();
    }
    cudaStreamDestroy(st);
}

// The host snapshot of the top pivot levels: the deepest l <= h whose levels
// above it hold at most 4096 pivots (Eq. 1: levels 0 .. l-1 hold lvl_off[l] nodes).
void snapshot_top_levels(gts_index *ix, TopLevels &t) {
    const Tree &tr = ix->tree;
    t = TopLevels();
    t.F = tr.F;
    t.dim = tr.dim;
    t.metric = tr.metric;
    t.cosine = tr.cosine;
    t.cache_rows = ix->cache.count;
    t.n_live = ix->n_live;
    if (tr.n == 0 || tr.h < 1) return;
    int L = 1;
    while (L < tr.h && tr.lvl_off[L + 1] <= 4096) ++L;
    t.levels = L;
    t.lvl_off.assign(tr.lvl_off.begin(), tr.lvl_off.begin() + L + 1);
    const int64_t nodes = tr.lvl_off[L + 1], npiv = tr.lvl_off[L];
    std::vector<int32_t> piv(npiv), sz(nodes);
    t.lo.resize(nodes - 1);
    t.hi.resize(nodes - 1);
    GTS_CUDA(cudaMemcpy(piv.data(), tr.npiv.get(), npiv * 4, cudaMemcpyDeviceToHost));
    GTS_CUDA(cudaMemcpy(sz.data(), tr.nsize.get(), nodes * 4, cudaMemcpyDeviceToHost));
    GTS_CUDA(cudaMemcpy(t.lo.data(), tr.nlo.get() + 1, (nodes - 1) * 4, cudaMemcpyDeviceToHost));
    GTS_CUDA(cudaMemcpy(t.hi.data(), tr.nhi.get() + 1, (nodes - 1) * 4, cudaMemcpyDeviceToHost));
    t.size.assign(sz.begin(), sz.end());
    t.has_piv.assign(npiv, 0);
    t.piv_live.assign(npiv, 0);
    if (t.dim > 0) t.pv.assign((size_t)npiv * t.dim, 0.f);
    else t.ps.assign(npiv, std::string());
    for (int64_t v = 0; v < npiv; ++v) {
        const int32_t row = piv[v];
        if (row < 0) continue;
        t.has_piv[v] = 1;
        int64_t del = 0;
        GTS_CUDA(cudaMemcpy(&del, tr.row_del.get() + row, 8, cudaMemcpyDeviceToHost));
        t.piv_live[v] = del == kNever ? 1 : 0;
        if (t.dim > 0) {
            GTS_CUDA(cudaMemcpy(&t.pv[(size_t)v * t.dim], tr.X.get() + (int64_t)row * t.dim, (size_t)t.dim * 4,
                                cudaMemcpyDeviceToHost));
        } else {
            int64_t off[2];
            GTS_CUDA(cudaMemcpy(off, tr.Soff.get() + row, 16, cudaMemcpyDeviceToHost));
            std::string str((size_t)(off[1] - off[0]), '\0');
            if (off[1] > off[0])
                GTS_CUDA(cudaMemcpy(&str[0], tr.S.get() + off[0], (size_t)(off[1] - off[0]), cudaMemcpyDeviceToHost));
            t.ps[v] = std::move(str);
        }
    }
}

template <class F>
gts_status guard(F &&f) {
    try {
        f();
        return GTS_OK;
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.status;
    } catch (const std::exception &e) {
        set_last_error(e.what());
        return GTS_ECUDA;
    }
}

}  // namespace
}  // namespace gts

using namespace gts;

extern "C" {

gts_status gts_serve_start(gts_index *ix, const gts_serve_opts *opts, gts_server **out) {
    return guard([&] {
        GTS_REQUIRE(ix && out, GTS_EINVAL, "NULL argument");
        std::unique_ptr<gts_server> sv(new gts_server());
        sv->ix = ix;
        std::memset(&sv->opts, 0, sizeof(sv->opts));
        if (opts) sv->opts = *opts;
        if (sv->opts.max_batch <= 0) sv->opts.max_batch = 1024;
        if (sv->opts.n_streams <= 0) sv->opts.n_streams = 3;
        if (sv->opts.result_budget <= 0) sv->opts.result_budget = (int64_t)16 << 30;
        if (sv->opts.memory_budget <= 0) sv->opts.memory_budget = sv->opts.result_budget / sv->opts.n_streams;
        GTS_CUDA(cudaSetDevice(ix->device));
        // warm the tensor-core copy before any worker runs (it is built lazily)
        if (sv->opts.precision == GTS_PREC_BF16 && (ix->metric == GTS_L2 || ix->metric == GTS_COS) &&
            ix->tree.n > 0) {
            std::vector<float> q((size_t)ix->dim, 0.f);
            q[0] = 1.f;   // (the angular distance has no zero vector)
            gts_objects qo;
            std::memset(&qo, 0, sizeof(qo));
            qo.n = 1;
            qo.dim = ix->dim;
            qo.data = q.data();
            int32_t k = 1;
            gts_query_opts o;
            std::memset(&o, 0, sizeof(o));
            o.stream = ix->stream;
            o.precision = GTS_PREC_BF16;
            gts_result r;
            if (gts_knn(ix, &qo, &k, &o, &r) == GTS_OK) gts_result_free(&r);
        }
        snapshot_top_levels(ix, sv->top);
        gts_server *p = sv.get();
        for (int i = 0; i < sv->opts.n_streams; ++i) sv->workers.emplace_back(worker_loop, p, i);
        *out = sv.release();
    });
}

gts_status gts_serve_submit(gts_server *sv, const void *query, int64_t len, int32_t kind, double param,
                            int64_t *ticket) {
    return guard([&] {
        GTS_REQUIRE(sv && ticket, GTS_EINVAL, "NULL argument");
        GTS_REQUIRE(kind == 0 || kind == 1, GTS_EINVAL, "kind must be 0 (range) or 1 (kNN)");
        const int dim = sv->ix->dim;
        Request r;
        r.kind = kind;
        if (kind == 0) {
            GTS_REQUIRE(param >= 0.0 && param == param, GTS_EINVAL, "radius must be >= 0");
            r.radius = (float)param;
            r.k = 0;
        } else {
            GTS_REQUIRE(param >= 1.0 && param <= 1024.0, GTS_EINVAL, "k must be in 1 .. 1024");
            r.k = (int32_t)param;
            r.radius = 0.f;
        }
        if (dim > 0) {
            GTS_REQUIRE(len == dim && query, GTS_EINVAL, "a vector query must have dim coordinates");
            r.payload.resize((size_t)dim * 4);
            std::memcpy(r.payload.data(), query, (size_t)dim * 4);
        } else {
            GTS_REQUIRE(len >= 0 && len <= kMaxStrLen && (len == 0 || query), GTS_EINVAL, "bad string query");
            r.payload.assign((const uint8_t *)query, (const uint8_t *)query + len);
        }
        const int64_t rows = project_rows(sv->top, r.payload.data(), (int64_t)r.payload.size(), kind, param);
        r.proj = (rows > 0 ? rows : 1) * kCandidateBytes;
        r.t_submit = now_ms();
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            GTS_REQUIRE(!sv->stopping, GTS_EINVAL, "server is stopping");
            r.ticket = sv->next_ticket++;
            *ticket = r.ticket;
            sv->proj_total += r.proj;
            if (rows < sv->top.n_live + sv->top.cache_rows) sv->proj_below_worst += 1;
            sv->pending.push_back(std::move(r));
        }
        sv->cv_work.notify_one();
    });
}

gts_status gts_serve_wait(gts_server *sv, int64_t ticket, int32_t timeout_ms, gts_result *out, double *latency_ms) {
    gts_status inner = GTS_OK;
    gts_status s = guard([&] {
        GTS_REQUIRE(sv && out, GTS_EINVAL, "NULL argument");
        std::unique_lock<std::mutex> lk(sv->mu);
        auto ready = [&] { return sv->done.count(ticket) > 0; };
        if (timeout_ms < 0) {
            sv->cv_done.wait(lk, ready);
        } else if (!sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) {
            throw Error(GTS_ETIMEOUT, "request not finished yet");
        }
        Done dn = std::move(sv->done[ticket]);
        sv->done.erase(ticket);
        lk.unlock();
        inner = dn.status;
        if (latency_ms) *latency_ms = dn.latency_ms;
        if (dn.status != GTS_OK) throw Error(dn.status, "request failed");
        const int64_t m = (int64_t)dn.ids.size();
        out->nq = 1;
        out->on_device = 0;
        out->priv_ = nullptr;
        out->key = nullptr;
        out->offsets = (int64_t *)std::malloc(16);
        out->ids = (int64_t *)std::malloc(sizeof(int64_t) * (m > 0 ? m : 1));
        out->dist = (float *)std::malloc(sizeof(float) * (m > 0 ? m : 1));
        if (!out->offsets || !out->ids || !out->dist) throw std::bad_alloc();
        out->offsets[0] = 0;
        out->offsets[1] = m;
        if (m) {
            std::memcpy(out->ids, dn.ids.data(), sizeof(int64_t) * m);
            std::memcpy(out->dist, dn.dist.data(), sizeof(float) * m);
        }
    });
    (void)inner;
    return s;
}

gts_status gts_serve_stats(gts_server *sv, int64_t *out, int32_t n_out) {
    return guard([&] {
        GTS_REQUIRE(sv && out && n_out >= 0, GTS_EINVAL, "NULL argument");
        std::lock_guard<std::mutex> lk(sv->mu);
        const int64_t v[6] = {sv->batches, sv->requests_run, sv->max_batch_seen, sv->max_in_flight,
                              sv->proj_total, sv->proj_below_worst};
        for (int i = 0; i < n_out && i < 6; ++i) out[i] = v[i];
    });
}

gts_status gts_serve_project(gts_server *sv, const void *query, int64_t len, int32_t kind, double param,
                             int64_t *bytes) {
    return guard([&] {
        GTS_REQUIRE(sv && bytes, GTS_EINVAL, "NULL argument");
        GTS_REQUIRE(kind == 0 || kind == 1, GTS_EINVAL, "kind must be 0 (range) or 1 (kNN)");
        GTS_REQUIRE(kind == 1 ? (param >= 1.0 && param <= 1024.0) : (param >= 0.0 && param == param), GTS_EINVAL,
                    "bad radius or k");
        const int dim = sv->ix->dim;
        GTS_REQUIRE(dim > 0 ? (len == dim && query) : (len >= 0 && len <= kMaxStrLen && (len == 0 || query)),
                    GTS_EINVAL, "bad query");
        const int64_t rows = project_rows(sv->top, (const uint8_t *)query, dim > 0 ? (int64_t)dim * 4 : len, kind,
                                          param);
        *bytes = (rows > 0 ? rows : 1) * kCandidateBytes;
    });
}

gts_status gts_serve_stop(gts_server *sv) {
    return guard([&] {
        GTS_REQUIRE(sv, GTS_EINVAL, "NULL argument");
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            sv->stopping = true;
        }
        sv->cv_work.notify_all();
        sv->cv_done.notify_all();
        for (auto &t : sv->workers) t.join();
        delete sv;
    });
}

}  // extern "C"
