/*
 * CPU oracle for GTS metric range / kNN search (arXiv 2404.00966).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library path calls, links or
 * loads this file: only tests/, the smoke check of __graft_entry__ and the
 * CPU-baseline leg of bench.py do.  It shares no code, header or constant with
 * the CUDA library.
 *
 * What it computes is the plain definition of the two queries, by brute force
 * over every live object:
 *   range (Section 3, Definition 1):  MRQ(q, r) = { o in O : d(q, o) <= r }
 *   kNN   (Section 3, Definition 2):  a set S of k objects with
 *         d(q, s) <= d(q, o) for every s in S and o outside S.  Where ties
 *         leave several valid sets, the oracle returns the first k objects in
 *         ascending (distance, id) order.
 * Pruning by Lemma 1 / Lemma 2 (Section 5) is exact, so an index-based search
 * must reach exactly these sets.
 *
 * Metrics (Section 3; Table 2):
 *   edit: unit-cost Levenshtein distance over bytes (insert, delete, replace),
 *         the textbook dynamic programme.  For range queries a band of width r
 *         around the diagonal (Ukkonen's cut-off) gives min(d, r + 1) exactly.
 *   l2:   key = sum_i ((double)q_i - (double)x_i)^2, summed in increasing i in
 *         FP64 with every operation rounded on its own (build with
 *         -ffp-contract=off).  Range compares key <= (double)r * (double)r;
 *         kNN orders by key (the square root is monotone, and the squared
 *         value keeps distinct FP64 sums distinct).  Reported d = sqrt(key).
 *   l1:   key = sum_i |(double)q_i - (double)x_i|, in increasing i, FP64.
 *   cos:  the angle between the vectors, d = arccos(c), c = q.x / (|q| |x|)
 *         (the word cosine distance of Table 2, read as the angular distance,
 *         a metric on directions).  The three sums q.x, |q|^2, |x|^2 run in
 *         increasing i in FP64, c = dot / (sqrt(|q|^2) * sqrt(|x|^2)) clamped
 *         to [-1, 1], key = 1 - c (monotone in the angle).  Range compares
 *         key <= 1 - cos((double)r) (r clipped to [0, pi]); kNN orders by key.
 *         Reported d = arccos(1 - key).  Zero vectors have no direction and
 *         are not accepted by the library.
 *
 * Stream updates (Section 4.4) are modelled by sequence numbers: object o is
 * visible to a query with sequence s iff ins_seq[o] < s < del_seq[o]
 * (del_seq = INT64_MAX when never deleted).  Null sequence arrays mean every
 * object is visible.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { OR_EDIT = 0, OR_L1 = 1, OR_L2 = 2, OR_COS = 3 };

int orc_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------- metrics */

/* Textbook Levenshtein DP, two rows. */
int64_t orc_edit_full(const uint8_t *a, int64_t la, const uint8_t *b, int64_t lb) {
    if (la == 0) return lb;
    if (lb == 0) return la;
    int64_t *prev = (int64_t *)malloc(sizeof(int64_t) * (size_t)(lb + 1));
    int64_t *cur = (int64_t *)malloc(sizeof(int64_t) * (size_t)(lb + 1));
    for (int64_t j = 0; j <= lb; ++j) prev[j] = j;
    for (int64_t i = 1; i <= la; ++i) {
        cur[0] = i;
        for (int64_t j = 1; j <= lb; ++j) {
            int64_t sub = prev[j - 1] + (a[i - 1] != b[j - 1] ? 1 : 0);
            int64_t del = prev[j] + 1;
            int64_t ins = cur[j - 1] + 1;
            int64_t v = sub < del ? sub : del;
            cur[j] = v < ins ? v : ins;
        }
        int64_t *t = prev; prev = cur; cur = t;
    }
    int64_t d = prev[lb];
    free(prev); free(cur);
    return d;
}

/* Levenshtein distance restricted to the diagonal band |i - j| <= r, with
 * every value capped at r + 1.  Cells outside the band have true value
 * >= |i - j| > r, and capping commutes with min and +1, so the result is
 * min(d, r + 1). */
int64_t orc_edit_banded(const uint8_t *a, int64_t la, const uint8_t *b, int64_t lb, int64_t r) {
    if (r < 0) return r + 1; /* min(d, r + 1) with d >= 0 */
    const int64_t INF = r + 1;
    int64_t diff = la > lb ? la - lb : lb - la;
    if (diff > r) return INF;
    int64_t *prev = (int64_t *)malloc(sizeof(int64_t) * (size_t)(lb + 2));
    int64_t *cur = (int64_t *)malloc(sizeof(int64_t) * (size_t)(lb + 2));
    for (int64_t j = 0; j <= lb + 1; ++j) prev[j] = (j <= r && j <= lb) ? j : INF;
    for (int64_t i = 1; i <= la; ++i) {
        int64_t jlo = i - r > 1 ? i - r : 1;
        int64_t jhi = i + r < lb ? i + r : lb;
        for (int64_t j = 0; j <= lb + 1; ++j) cur[j] = INF;
        cur[0] = i <= r ? i : INF;
        for (int64_t j = jlo; j <= jhi; ++j) {
            int64_t sub = prev[j - 1] + (a[i - 1] != b[j - 1] ? 1 : 0);
            int64_t del = prev[j] + 1;
            int64_t ins = cur[j - 1] + 1;
            int64_t v = sub < del ? sub : del;
            v = v < ins ? v : ins;
            cur[j] = v < INF ? v : INF;
        }
        int64_t *t = prev; prev = cur; cur = t;
    }
    int64_t d = prev[lb] < INF ? prev[lb] : INF;
    free(prev); free(cur);
    return d;
}

double orc_l2sq(const float *a, const float *b, int64_t dim) {
    double s = 0.0;
    for (int64_t i = 0; i < dim; ++i) {
        double t = (double)a[i] - (double)b[i];
        double p = t * t;
        s = s + p;
    }
    return s;
}

double orc_l1(const float *a, const float *b, int64_t dim) {
    double s = 0.0;
    for (int64_t i = 0; i < dim; ++i) {
        double t = (double)a[i] - (double)b[i];
        s = s + fabs(t);
    }
    return s;
}

/* 1 - cos of the angle, the three FP64 sums in increasing i, c clamped to [-1, 1]. */
double orc_cos_key(const float *a, const float *b, int64_t dim) {
    double dot = 0.0, na = 0.0, nb = 0.0;
    for (int64_t i = 0; i < dim; ++i) {
        double x = (double)a[i], y = (double)b[i];
        double p = x * y;
        dot = dot + p;
        double pa = x * x;
        na = na + pa;
        double pb = y * y;
        nb = nb + pb;
    }
    double den = sqrt(na) * sqrt(nb);
    double c = dot / den;
    if (c > 1.0) c = 1.0;
    if (c < -1.0) c = -1.0;
    return 1.0 - c;
}

/* the range limit on the key for an angle r */
double orc_cos_limit(double r) {
    const double pi = 3.14159265358979323846;
    if (r > pi) r = pi;
    return 1.0 - cos(r);
}

/* Angles of FP64 cosine keys: acos(1 - key) from the C library, element by
 * element (the multi-column sum of Section 5.2's closing remark adds these). */
void orc_cos_angles(const double *keys, int64_t n, double *out) {
    for (int64_t i = 0; i < n; ++i) out[i] = acos(1.0 - keys[i]);
}

static double vec_key(int metric, const float *q, const float *x, int64_t dim) {
    if (metric == OR_COS) return orc_cos_key(q, x, dim);
    return metric == OR_L2 ? orc_l2sq(q, x, dim) : orc_l1(q, x, dim);
}

static int visible(const int64_t *ins, const int64_t *del, int64_t o, int64_t s) {
    if (!ins) return 1;
    return ins[o] < s && s < del[o];
}

/* Distance keys from one query to every object (no visibility filter). */
void orc_keys_vec(int metric, const float *X, int64_t n, int64_t dim, const float *q, double *out) {
#pragma omp parallel for schedule(static)
    for (int64_t o = 0; o < n; ++o) out[o] = vec_key(metric, q, X + o * dim, dim);
}

void orc_keys_str(const uint8_t *data, const int64_t *offs, int64_t n, const uint8_t *q, int64_t lq,
                  int64_t *out) {
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t o = 0; o < n; ++o)
        out[o] = orc_edit_full(q, lq, data + offs[o], offs[o + 1] - offs[o]);
}

/* ------------------------------------------------------------ range query */

/* Two calls: with ids == NULL only counts[q] is written; with ids != NULL the
 * matches of query q go to ids/keys[offsets[q] ...] in ascending id order. */
void orc_range_vec(int metric, const float *X, int64_t n, int64_t dim, const float *Q, int64_t nq,
                   const float *radii, const int64_t *ins, const int64_t *del, const int64_t *qseq,
                   int64_t *counts, const int64_t *offsets, int64_t *ids, double *keys) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t qi = 0; qi < nq; ++qi) {
        const float *q = Q + qi * dim;
        double r = (double)radii[qi];
        double lim = metric == OR_L2 ? r * r : (metric == OR_COS ? orc_cos_limit(r) : r);
        int64_t s = qseq ? qseq[qi] : 0;
        int64_t c = 0;
        for (int64_t o = 0; o < n; ++o) {
            if (!visible(ins, del, o, s)) continue;
            double k = vec_key(metric, q, X + o * dim, dim);
            if (k <= lim) {
                if (ids) { ids[offsets[qi] + c] = o; keys[offsets[qi] + c] = k; }
                ++c;
            }
        }
        counts[qi] = c;
    }
}

void orc_range_str(const uint8_t *data, const int64_t *offs, int64_t n, const uint8_t *qdata,
                   const int64_t *qoffs, int64_t nq, const float *radii, const int64_t *ins,
                   const int64_t *del, const int64_t *qseq, int64_t *counts, const int64_t *offsets,
                   int64_t *ids, double *keys) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t qi = 0; qi < nq; ++qi) {
        const uint8_t *q = qdata + qoffs[qi];
        int64_t lq = qoffs[qi + 1] - qoffs[qi];
        int64_t r = (int64_t)floor((double)radii[qi]);
        int64_t s = qseq ? qseq[qi] : 0;
        int64_t c = 0;
        for (int64_t o = 0; o < n; ++o) {
            if (!visible(ins, del, o, s)) continue;
            int64_t d = orc_edit_banded(q, lq, data + offs[o], offs[o + 1] - offs[o], r);
            if (d <= r) {
                if (ids) { ids[offsets[qi] + c] = o; keys[offsets[qi] + c] = (double)d; }
                ++c;
            }
        }
        counts[qi] = c;
    }
}

/* -------------------------------------------------------------- kNN query */

/* Insert (key, id) into the ascending list (keys, ids) of length *len, capacity
 * k, if it belongs among the first k in (key, id) order. */
static void topk_push(double *kk, int64_t *ii, int64_t *len, int64_t k, double key, int64_t id) {
    int64_t L = *len;
    if (L == k) {
        if (key > kk[L - 1] || (key == kk[L - 1] && id > ii[L - 1])) return;
        L = k - 1;
    }
    int64_t p = L;
    while (p > 0 && (kk[p - 1] > key || (kk[p - 1] == key && ii[p - 1] > id))) {
        kk[p] = kk[p - 1]; ii[p] = ii[p - 1]; --p;
    }
    kk[p] = key; ii[p] = id;
    *len = L + 1;
}

/* Query q's answer goes to ids/keys[offsets[q] .. offsets[q] + counts[q]),
 * counts[q] = min(k[q], visible objects), ascending (key, id). */
void orc_knn_vec(int metric, const float *X, int64_t n, int64_t dim, const float *Q, int64_t nq,
                 const int32_t *k, const int64_t *ins, const int64_t *del, const int64_t *qseq,
                 const int64_t *offsets, int64_t *ids, double *keys, int64_t *counts) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t qi = 0; qi < nq; ++qi) {
        const float *q = Q + qi * dim;
        int64_t s = qseq ? qseq[qi] : 0;
        int64_t len = 0;
        double *kk = keys + offsets[qi];
        int64_t *ii = ids + offsets[qi];
        for (int64_t o = 0; o < n; ++o) {
            if (!visible(ins, del, o, s)) continue;
            topk_push(kk, ii, &len, k[qi], vec_key(metric, q, X + o * dim, dim), o);
        }
        counts[qi] = len;
    }
}

void orc_knn_str(const uint8_t *data, const int64_t *offs, int64_t n, const uint8_t *qdata,
                 const int64_t *qoffs, int64_t nq, const int32_t *k, const int64_t *ins,
                 const int64_t *del, const int64_t *qseq, const int64_t *offsets, int64_t *ids,
                 double *keys, int64_t *counts) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t qi = 0; qi < nq; ++qi) {
        const uint8_t *q = qdata + qoffs[qi];
        int64_t lq = qoffs[qi + 1] - qoffs[qi];
        int64_t s = qseq ? qseq[qi] : 0;
        int64_t len = 0;
        double *kk = keys + offsets[qi];
        int64_t *ii = ids + offsets[qi];
        for (int64_t o = 0; o < n; ++o) {
            if (!visible(ins, del, o, s)) continue;
            int64_t d = orc_edit_full(q, lq, data + offs[o], offs[o + 1] - offs[o]);
            topk_push(kk, ii, &len, k[qi], (double)d, o);
        }
        counts[qi] = len;
    }
}
