/*
 * Plain CPU oracle for the BBC large-k IVF search path (arxiv 2604.01960).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file; only the tests, the smoke check and the benchmark's CPU
 * baseline use it.  It shares no code with the CUDA library.
 *
 * Single-threaded, written for clarity over speed.  Floating point is FP64
 * except where the method fixes FP32 (the PQ lookup table recipe).  Compile
 * with -ffp-contract=off so that no multiply-add is fused.
 *
 * What each function follows:
 *   oracle_probe          Section 2 "Quantization": IVF routes a query to the
 *                         n_probe nearest centroids; Algorithm 4 visits them
 *                         nearest first.  Ties go to the smaller list id.
 *   oracle_lut_f32/16     Section 2 "Quantization", step (1): distances from
 *                         the query to every codebook vector, per sub-space;
 *                         then the uint16 integer quantisation of the table
 *                         (oracle_lut_q: the same recipe with a smaller top
 *                         level, e.g. 2047, whose entries FP16 holds exactly).
 *   oracle_adc            step (2): estimated distance = sum over sub-spaces
 *                         of the table entry picked by the code.
 *   oracle_lut16_scale, oracle_resid_a/_base/_w/_v, oracle_adc_resid
 *                         the same step when the PQ codes quantise the
 *                         residual o - c_l of each list's objects (residual
 *                         IVF-PQ): the table plus a per-(query, list) and a
 *                         per-object term, in the table's integer units.
 *   oracle_topkc_sort     the n_cand candidates by estimated distance
 *                         (Section 2, unbounded methods), by a full sort.
 *   oracle_topkc_heap     the same set through a binary max-heap collector,
 *                         the baseline collector of Section 2 "Top-k Collector".
 *   oracle_bucket_collect Algorithm 1 (Push, Update, Collect) with the
 *                         sampled equal-width -> equal-depth codebook of
 *                         Section 3.2 and the bucket id of Eq. (remap).
 *   oracle_alg4           Algorithm 4 (IVF+PQ with early re-ranking) on
 *                         Algorithm 1's buffer: which objects get their
 *                         exact distance while their list is scanned.
 *   oracle_rerank         exact distances of the candidates (FP64).
 *   oracle_topk_final     the k smallest exact distances, ascending.
 *   oracle_search         the whole path for a batch of queries.
 *   oracle_bruteforce     exact kNN over the whole data set (FP64).
 *   oracle_sign_encode, oracle_sign_bounds, oracle_rotation_eps
 *                         the 1-bit sign quantizer of the bounded re-rank
 *                         (Section 3.4): codes of the rotated residual and
 *                         hard per-object distance bounds.
 *   oracle_sign_bounds_rq the same objects' bounds from the RaBitQ estimator
 *                         and its probabilistic error bound (the method
 *                         Section 3.4 builds on, with the Section 4.1 setting
 *                         epsilon_0 = 1.9): not hard; the true distance lies
 *                         inside with high probability.
 *   oracle_alg2           Algorithm 2, minimal re-ranking with two heaps.
 *   oracle_obs1_count     the set of Observation 1 (bounds enclosing Dist_k).
 *   oracle_oneshot        the one-pass sure-in / sure-out classification.
 *   oracle_rounds         the bounded re-rank in two rounds with exact
 *                         returned distances (batched Algorithm 3).
 *   oracle_bf16_*, oracle_e4m3_*, oracle_prec_copy
 *                         the low-precision copies of the vectors used by the
 *                         precision form of the re-rank (the paper re-ranks
 *                         "with exact distances", Section 2; the copies and
 *                         their per-vector error e_v are this implementation's
 *                         reading of how to do that cheaply).  Written from
 *                         the two formats' definitions: bfloat16 = binary32
 *                         with 7 stored fraction bits; OCP E4M3 = 4 exponent
 *                         bits (bias 7), 3 fraction bits, largest finite 448.
 *
 * Orders: every "smallest" is by (value, id) ascending, id breaking ties.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_L2 0
#define ORACLE_IP 1

/* ------------------------------------------------------------------ */
/* comparators                                                          */
/* ------------------------------------------------------------------ */
typedef struct { double s; int64_t id; } dkey;
typedef struct { uint32_t e; int64_t id; } ukey;

static int cmp_dkey(const void* a, const void* b) {
    const dkey* x = (const dkey*)a;
    const dkey* y = (const dkey*)b;
    if (x->s < y->s) return -1;
    if (x->s > y->s) return 1;
    if (x->id < y->id) return -1;
    if (x->id > y->id) return 1;
    return 0;
}

static int cmp_ukey(const void* a, const void* b) {
    const ukey* x = (const ukey*)a;
    const ukey* y = (const ukey*)b;
    if (x->e < y->e) return -1;
    if (x->e > y->e) return 1;
    if (x->id < y->id) return -1;
    if (x->id > y->id) return 1;
    return 0;
}

static int cmp_double(const void* a, const void* b) {
    const double x = *(const double*)a, y = *(const double*)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

static int ukey_less(ukey a, ukey b) { return a.e < b.e || (a.e == b.e && a.id < b.id); }

/* ------------------------------------------------------------------ */
/* distances                                                            */
/* ------------------------------------------------------------------ */
/* Squared L2, or negated inner product, in FP64 over ascending dimension. */
double oracle_dist(const float* a, const float* b, int32_t d, int32_t metric) {
    double s = 0.0;
    if (metric == ORACLE_L2) {
        for (int32_t i = 0; i < d; ++i) {
            double t = (double)a[i] - (double)b[i];
            s = s + t * t;
        }
    } else {
        for (int32_t i = 0; i < d; ++i) s = s + (double)a[i] * (double)b[i];
        s = -s;
    }
    return s;
}

/* ------------------------------------------------------------------ */
/* IVF probe                                                            */
/* ------------------------------------------------------------------ */
int oracle_probe(const float* q, const float* centroids, int32_t nlist, int32_t d,
                 int32_t metric, int32_t nprobe, int32_t* out_lists, double* out_scores) {
    if (nprobe < 1 || nprobe > nlist) return -1;
    dkey* all = (dkey*)malloc(sizeof(dkey) * (size_t)nlist);
    if (!all) return -4;
    for (int32_t l = 0; l < nlist; ++l) {
        all[l].s = oracle_dist(q, centroids + (size_t)l * d, d, metric);
        all[l].id = l;
    }
    qsort(all, (size_t)nlist, sizeof(dkey), cmp_dkey);
    for (int32_t j = 0; j < nprobe; ++j) {
        out_lists[j] = (int32_t)all[j].id;
        if (out_scores) out_scores[j] = all[j].s;
    }
    free(all);
    return 0;
}

/* ------------------------------------------------------------------ */
/* PQ lookup table                                                      */
/* ------------------------------------------------------------------ */
/* FP32 table: entry [m][j] = ||q_m - y_{m,j}||^2 (L2) or -<q_m, y_{m,j}> (IP),
 * accumulated in FP32 over ascending dimension, one rounding per operation. */
void oracle_lut_f32(const float* q, const float* books, int32_t d, int32_t M, int32_t bits,
                    int32_t metric, float* lut) {
    const int32_t K = 1 << bits, ds = d / M;
    for (int32_t m = 0; m < M; ++m) {
        const float* qm = q + (size_t)m * ds;
        for (int32_t j = 0; j < K; ++j) {
            const float* y = books + ((size_t)m * K + j) * ds;
            float acc = 0.0f;
            if (metric == ORACLE_L2) {
                for (int32_t i = 0; i < ds; ++i) {
                    float t = qm[i] - y[i];
                    float t2 = t * t;
                    acc = acc + t2;
                }
            } else {
                for (int32_t i = 0; i < ds; ++i) {
                    float p = qm[i] * y[i];
                    acc = acc + p;
                }
                acc = -acc;
            }
            lut[(size_t)m * K + j] = acc;
        }
    }
}

/* Integer table with top level T (65535 for the uint16 table): per
 * sub-space offset lo_m = min_j L[m][j]; one scale for the query,
 * inv = T / span with span = max_m (max_j L[m][j] - lo_m);
 * entry = min(T, floor((L - lo_m) * inv + 0.5)).  span == 0 gives zeros. */
/* lo_m and the query's scale inv of the integer table from the FP32 table. */
static float lut_offsets(const float* lut, int32_t M, int32_t K, float top, float* lo) {
    float span = 0.0f;
    for (int32_t m = 0; m < M; ++m) {
        float mn = lut[(size_t)m * K], mx = mn;
        for (int32_t j = 1; j < K; ++j) {
            float v = lut[(size_t)m * K + j];
            if (v < mn) mn = v;
            if (v > mx) mx = v;
        }
        lo[m] = mn;
        float w = mx - mn;
        if (w > span) span = w;
    }
    float inv = span > 0.0f ? top / span : 0.0f;
    if (!(inv <= FLT_MAX)) inv = 0.0f;
    return inv;
}

/* The integer table with top level `levels` (1 .. 65535). */
void oracle_lut_q(const float* q, const float* books, int32_t d, int32_t M, int32_t bits,
                  int32_t metric, int32_t levels, uint16_t* lut16, float* lut_f32_out) {
    const int32_t K = 1 << bits;
    const float top = (float)levels;
    float* lut = (float*)malloc(sizeof(float) * (size_t)M * K);
    float* lo = (float*)malloc(sizeof(float) * (size_t)M);
    oracle_lut_f32(q, books, d, M, bits, metric, lut);
    const float inv = lut_offsets(lut, M, K, top, lo);
    for (int32_t m = 0; m < M; ++m) {
        for (int32_t j = 0; j < K; ++j) {
            float t = lut[(size_t)m * K + j] - lo[m];
            float u = t * inv;
            float v = floorf(u + 0.5f);
            if (v > top) v = top;
            lut16[(size_t)m * K + j] = (uint16_t)v;
        }
    }
    if (lut_f32_out) memcpy(lut_f32_out, lut, sizeof(float) * (size_t)M * K);
    free(lut);
    free(lo);
}

void oracle_lut16(const float* q, const float* books, int32_t d, int32_t M, int32_t bits,
                  int32_t metric, uint16_t* lut16, float* lut_f32_out) {
    oracle_lut_q(q, books, d, M, bits, metric, 65535, lut16, lut_f32_out);
}

/* ------------------------------------------------------------------ */
/* ADC estimated distance                                               */
/* ------------------------------------------------------------------ */
static int32_t code_of(const uint8_t* row, int32_t m, int32_t bits) {
    if (bits == 8) return row[m];
    uint8_t b = row[m >> 1];
    return (m & 1) ? (b >> 4) : (b & 0x0F);
}

void oracle_adc(const uint16_t* lut16, const uint8_t* codes, int64_t n, int32_t M, int32_t bits,
                uint32_t* out_e) {
    const int32_t K = 1 << bits, cb = M * bits / 8;
    for (int64_t i = 0; i < n; ++i) {
        const uint8_t* row = codes + (size_t)i * cb;
        uint32_t e = 0;
        for (int32_t m = 0; m < M; ++m) e += lut16[(size_t)m * K + code_of(row, m, bits)];
        out_e[i] = e;
    }
}

/* The query's table scale inv (integer units per unit of distance) and the
 * per-sub-space offsets' sum, sum_m lo_m (FP64 sum of the FP32 offsets). */
float oracle_lut16_scale(const float* q, const float* books, int32_t d, int32_t M, int32_t bits,
                         int32_t metric, double* lo_sum) {
    const int32_t K = 1 << bits;
    float* lut = (float*)malloc(sizeof(float) * (size_t)M * K);
    float* lo = (float*)malloc(sizeof(float) * (size_t)M);
    oracle_lut_f32(q, books, d, M, bits, metric, lut);
    const float inv = lut_offsets(lut, M, K, 65535.0f, lo);
    if (lo_sum) {
        double s = 0.0;
        for (int32_t m = 0; m < M; ++m) s += (double)lo[m];
        *lo_sum = s;
    }
    free(lut);
    free(lo);
    return inv;
}

/* ------------------------------------------------------------------ */
/* Residual IVF-PQ (Section 2 "Quantization", with the codes of o - c_l) */
/* ------------------------------------------------------------------ */
/* An object o of list l is coded by the PQ code of its residual o - c_l;
 * y = the code's reconstruction (codeword m of sub-space m in dimensions
 * m*d/M ..).  Its estimated distance splits into the query's table, a
 * per-(query, list) term and a per-object term:
 *   L2  ||q - c_l - y||^2 = ||q - y||^2 + (||c_l||^2 - 2 <q, c_l>) + 2 <c_l, y>
 *                        = sum_m L[m][code_m] + A_ql + V_o;
 *   IP  -<q, c_l + y>     = sum_m L[m][code_m] + A_ql,  A_ql = -<q, c_l>, V_o = 0;
 * L the query's table of oracle_lut_f32 (the same formula as for plain PQ).
 * In the uint16 table's integer units (scale inv) the object's key is
 *   key = sum_m LUT16[m][code_m] + base_ql + w_o,
 *   base_ql = 2^30 + rint(clamp(A_ql * inv, -2^29, 2^29)),
 *   w_o     = rint(clamp(V_o * inv, -2^28, 2^28)),
 * i.e. (key - 2^30) / inv ~ the estimated distance minus sum_m lo_m; 2^30
 * keeps keys positive, the clamps keep them below 2^31 (reached only when the
 * table's span is tiny against the centroid terms).  A_ql and V_o are
 * evaluated in FP32 with fused multiply-adds over ascending dimension, the
 * precision in which the keys -- and so the candidate set -- are decided:
 *   A_ql: s = sum_i q_i c_i, n = sum_i c_i c_i (each a chain of fmaf from 0),
 *         A = fmaf(-2, s, n) (L2) or -s (IP);
 *   V_o:  t = sum_i c_i y_i (a chain of fmaf from 0), V = 2 t (L2), 0 (IP). */
#define RESID_BIAS 1073741824.0 /* 2^30 */

static int32_t resid_round(float x, float lim) {
    x = fmaxf(x, -lim);
    x = fminf(x, lim);
    return (int32_t)rintf(x);
}

float oracle_resid_a(const float* q, const float* c, int32_t d, int32_t metric) {
    float s = 0.0f, n = 0.0f;
    for (int32_t i = 0; i < d; ++i) {
        s = fmaf(q[i], c[i], s);
        n = fmaf(c[i], c[i], n);
    }
    return metric == ORACLE_L2 ? fmaf(-2.0f, s, n) : -s;
}

int32_t oracle_resid_base(float a, float inv) {
    return (int32_t)RESID_BIAS + resid_round(a * inv, 536870912.0f);
}

int32_t oracle_resid_w(float v, float inv) { return resid_round(v * inv, 268435456.0f); }

/* V_o of n code rows (canonical layout) of list centroid c. */
void oracle_resid_v(const float* c, const uint8_t* codes, int64_t n, const float* books, int32_t d,
                    int32_t M, int32_t bits, int32_t metric, float* out_v) {
    const int32_t K = 1 << bits, ds = d / M, cb = M * bits / 8;
    for (int64_t o = 0; o < n; ++o) {
        const uint8_t* row = codes + (size_t)o * cb;
        float t = 0.0f;
        for (int32_t m = 0; m < M; ++m) {
            const float* y = books + ((size_t)m * K + code_of(row, m, bits)) * ds;
            for (int32_t i = 0; i < ds; ++i) t = fmaf(c[m * ds + i], y[i], t);
        }
        out_v[o] = metric == ORACLE_L2 ? 2.0f * t : 0.0f;
    }
}

/* Residual keys of n objects of one list: the plain sums of oracle_adc plus
 * base_ql and each object's w_o (see above). */
void oracle_adc_resid(const uint16_t* lut16, const uint8_t* codes, int64_t n, int32_t M, int32_t bits,
                      const float* q, const float* c, const float* books, int32_t d, int32_t metric,
                      float inv, uint32_t* out_e) {
    float* v = (float*)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
    oracle_adc(lut16, codes, n, M, bits, out_e);
    oracle_resid_v(c, codes, n, books, d, M, bits, metric, v);
    const int64_t base = oracle_resid_base(oracle_resid_a(q, c, d, metric), inv);
    for (int64_t o = 0; o < n; ++o) out_e[o] = (uint32_t)((int64_t)out_e[o] + base + oracle_resid_w(v[o], inv));
    free(v);
}

/* ------------------------------------------------------------------ */
/* candidate collectors                                                 */
/* ------------------------------------------------------------------ */
/* Sort-based: the Kc smallest (e, id); returns how many were written. */
int64_t oracle_topkc_sort(const uint32_t* e, const int64_t* ids, int64_t n, int64_t Kc,
                          int64_t* out_ids, uint32_t* out_e) {
    ukey* a = (ukey*)malloc(sizeof(ukey) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) { a[i].e = e[i]; a[i].id = ids[i]; }
    qsort(a, (size_t)n, sizeof(ukey), cmp_ukey);
    int64_t c = n < Kc ? n : Kc;
    for (int64_t i = 0; i < c; ++i) { out_ids[i] = a[i].id; if (out_e) out_e[i] = a[i].e; }
    free(a);
    return c;
}

/* Binary max-heap of capacity Kc keyed by (e, id); output in ascending order. */
static void heap_sift_down(ukey* h, int64_t n, int64_t i) {
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, big = i;
        if (l < n && ukey_less(h[big], h[l])) big = l;
        if (r < n && ukey_less(h[big], h[r])) big = r;
        if (big == i) return;
        ukey t = h[i]; h[i] = h[big]; h[big] = t;
        i = big;
    }
}

static void heap_sift_up(ukey* h, int64_t i) {
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (!ukey_less(h[p], h[i])) return;
        ukey t = h[i]; h[i] = h[p]; h[p] = t;
        i = p;
    }
}

int64_t oracle_topkc_heap(const uint32_t* e, const int64_t* ids, int64_t n, int64_t Kc,
                          int64_t* out_ids, uint32_t* out_e) {
    if (Kc <= 0) return 0;
    ukey* h = (ukey*)malloc(sizeof(ukey) * (size_t)Kc);
    int64_t sz = 0;
    for (int64_t i = 0; i < n; ++i) {
        ukey x = {e[i], ids[i]};
        if (sz < Kc) { h[sz] = x; heap_sift_up(h, sz); ++sz; }
        else if (ukey_less(x, h[0])) { h[0] = x; heap_sift_down(h, sz, 0); }
    }
    /* pop in descending order, write back to front */
    int64_t c = sz;
    while (sz > 0) {
        out_ids[sz - 1] = h[0].id;
        if (out_e) out_e[sz - 1] = h[0].e;
        h[0] = h[sz - 1];
        --sz;
        heap_sift_down(h, sz, 0);
    }
    free(h);
    return c;
}

/* ------------------------------------------------------------------ */
/* Bucket-based result buffer (Algorithm 1)                             */
/* ------------------------------------------------------------------ */
/* Codebook of Section 3.2 on integer estimated distances.
 *   sample   = the first lists in probe order: at least min(sample_min, P)
 *              lists, extended until they hold min(Kc, S_q) objects;
 *   t        = min(Kc, |sample|); d_min = smallest, d_max = t-th smallest
 *              sampled estimated distance (the sample's local top-Kc);
 *   delta    = 2^sh, the smallest power of two with (d_max - d_min) >> sh
 *              <= 255, so n_ew = 256 equal-width bins cover [d_min, d_max];
 *   bin(e)   = clamp(floor((e - d_min) / delta), 0, 255)          (Eq. remap)
 *   h[b]     = sampled objects with e <= d_max in bin b, T = sum h;
 *   map[b]   = min(m - 1, floor(m * sum_{b'<b} h[b'] / T)), a monotone
 *              equal-width -> equal-depth remap;
 *   bucket   = map[bin(e)] in [0, m).  tau = m stands for "infinity". */
typedef struct {
    uint32_t d_min, d_max;
    int32_t sh;
    int32_t m;
    int32_t sample_lists;
    int64_t sample_size;
    int32_t tau;            /* final threshold bucket (Update on the final buffer) */
    int64_t pushed;         /* objects appended to the buffer over the whole scan */
    int64_t below;          /* objects in buckets < tau */
    uint8_t map[256];
} oracle_codebook;

static int32_t bin_of(uint32_t e, const oracle_codebook* cb) {
    if (e <= cb->d_min) return 0;
    uint32_t b = (e - cb->d_min) >> cb->sh;
    return b > 255u ? 255 : (int32_t)b;
}

static int32_t bucket_of(uint32_t e, const oracle_codebook* cb) { return cb->map[bin_of(e, cb)]; }

/* Update (Algorithm 1): first bucket whose running count reaches
 * Kc ("reaches or exceeds", Section 3.2 text and the Figure 3 example). */
int32_t oracle_update(const int64_t* counts, int32_t m, int64_t Kc) {
    int64_t s = 0;
    for (int32_t i = 0; i < m; ++i) {
        s += counts[i];
        if (s >= Kc) return i;
    }
    return m;
}

static int cmp_u32(const void* a, const void* b) {
    uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

void oracle_build_codebook(const uint32_t* sample_e, int64_t ns, int64_t Kc, int32_t m,
                           oracle_codebook* cb) {
    memset(cb->map, 0, sizeof(cb->map));
    cb->m = m;
    cb->sample_size = ns;
    if (ns <= 0) { cb->d_min = cb->d_max = 0; cb->sh = 0; return; }
    uint32_t* s = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)ns);
    memcpy(s, sample_e, sizeof(uint32_t) * (size_t)ns);
    qsort(s, (size_t)ns, sizeof(uint32_t), cmp_u32);            /* partial sort, done fully */
    int64_t t = ns < Kc ? ns : Kc;
    cb->d_min = s[0];
    cb->d_max = s[t - 1];
    int32_t sh = 0;
    while (((cb->d_max - cb->d_min) >> sh) > 255u) ++sh;
    cb->sh = sh;
    int64_t h[256];
    memset(h, 0, sizeof(h));
    int64_t T = 0;
    for (int64_t i = 0; i < ns; ++i) {
        if (s[i] > cb->d_max) break;
        h[bin_of(s[i], cb)]++;
        ++T;
    }
    int64_t cum = 0;
    for (int32_t b = 0; b < 256; ++b) {
        int64_t v = (int64_t)m * cum / T;
        cb->map[b] = (uint8_t)(v > m - 1 ? m - 1 : v);
        cum += h[b];
    }
    free(s);
}

/* Collect (Algorithm 1) over the scanned lists in probe order.
 * e/ids hold the scanned objects list after list; list_ofs[j]..list_ofs[j+1]
 * is list j.  Outputs the Kc candidates (ascending (e, id)), the codebook,
 * the final bucket counts (counts[m]) and returns the number written. */
int64_t oracle_bucket_collect(const uint32_t* e, const int64_t* ids, const int64_t* list_ofs,
                              int32_t nl, int64_t Kc, int32_t m, int32_t sample_min,
                              oracle_codebook* cb, int64_t* counts_out,
                              int64_t* out_ids, uint32_t* out_e) {
    const int64_t Sq = list_ofs[nl] - list_ofs[0];
    const int64_t want = Kc < Sq ? Kc : Sq;
    int32_t ns_lists = sample_min < nl ? sample_min : nl;
    while (ns_lists < nl && list_ofs[ns_lists] - list_ofs[0] < want) ++ns_lists;
    int64_t ns = list_ofs[ns_lists] - list_ofs[0];
    oracle_build_codebook(e + list_ofs[0], ns, Kc, m, cb);
    cb->sample_lists = ns_lists;

    /* buckets: linear buffers appended at the tail (one shared arena, per-bucket chains) */
    int64_t* cnt = (int64_t*)calloc((size_t)m, sizeof(int64_t));
    int64_t* cap = (int64_t*)calloc((size_t)m, sizeof(int64_t));
    ukey** B = (ukey**)calloc((size_t)m, sizeof(ukey*));
    int32_t tau = m;                                  /* tau starts at infinity */
    int64_t pushed = 0;
    for (int32_t j = 0; j < nl; ++j) {                /* each cluster in probe order */
        for (int64_t i = list_ofs[j]; i < list_ofs[j + 1]; ++i) {
            int32_t a = bucket_of(e[i], cb);           /* Push: bucket of the estimate */
            if (a <= tau) {                            /* Push: admitted when at or below tau */
                if (cnt[a] == cap[a]) {
                    cap[a] = cap[a] ? 2 * cap[a] : 64;
                    B[a] = (ukey*)realloc(B[a], sizeof(ukey) * (size_t)cap[a]);
                }
                B[a][cnt[a]].e = e[i];
                B[a][cnt[a]].id = ids[i];
                cnt[a]++;
                ++pushed;
            }
        }
        tau = oracle_update(cnt, m, Kc);              /* Update after the cluster */
    }
    int64_t nres = 0;
    if (tau >= m) {                                    /* fewer than Kc objects in total */
        ukey* all = (ukey*)malloc(sizeof(ukey) * (size_t)(pushed > 0 ? pushed : 1));
        for (int32_t a = 0; a < m; ++a)
            for (int64_t i = 0; i < cnt[a]; ++i) all[nres++] = B[a][i];
        qsort(all, (size_t)nres, sizeof(ukey), cmp_ukey);
        for (int64_t i = 0; i < nres; ++i) { out_ids[i] = all[i].id; if (out_e) out_e[i] = all[i].e; }
        free(all);
        cb->below = nres;
    } else {
        /* buckets before tau, then the top-s of bucket tau */
        ukey* res = (ukey*)malloc(sizeof(ukey) * (size_t)Kc);
        for (int32_t a = 0; a < tau; ++a)
            for (int64_t i = 0; i < cnt[a]; ++i) res[nres++] = B[a][i];
        cb->below = nres;
        int64_t s = Kc - nres;
        qsort(B[tau], (size_t)cnt[tau], sizeof(ukey), cmp_ukey);
        for (int64_t i = 0; i < s; ++i) res[nres++] = B[tau][i];
        qsort(res, (size_t)nres, sizeof(ukey), cmp_ukey);
        for (int64_t i = 0; i < nres; ++i) { out_ids[i] = res[i].id; if (out_e) out_e[i] = res[i].e; }
        free(res);
    }
    cb->tau = tau;
    cb->pushed = pushed;
    if (counts_out) for (int32_t a = 0; a < m; ++a) counts_out[a] = cnt[a];
    for (int32_t a = 0; a < m; ++a) free(B[a]);
    free(B); free(cnt); free(cap);
    return nres;
}

/* ------------------------------------------------------------------ */
/* re-rank and final top-k                                              */
/* ------------------------------------------------------------------ */
void oracle_rerank(const float* q, const float* vectors, int32_t d, int32_t metric,
                   const int64_t* ids, int64_t n, double* out_d) {
    for (int64_t i = 0; i < n; ++i)
        out_d[i] = oracle_dist(q, vectors + (size_t)ids[i] * d, d, metric);
}

/* k smallest (dist, id) ascending; pads with id -1 and +inf when n < k. */
void oracle_topk_final(const double* dist, const int64_t* ids, int64_t n, int32_t k,
                       int64_t* out_ids, double* out_d) {
    dkey* a = (dkey*)malloc(sizeof(dkey) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) { a[i].s = dist[i]; a[i].id = ids[i]; }
    qsort(a, (size_t)n, sizeof(dkey), cmp_dkey);
    for (int32_t i = 0; i < k; ++i) {
        if (i < n) { out_ids[i] = a[i].id; out_d[i] = a[i].s; }
        else { out_ids[i] = -1; out_d[i] = INFINITY; }
    }
    free(a);
}

/* ------------------------------------------------------------------ */
/* whole path                                                           */
/* ------------------------------------------------------------------ */
typedef struct {
    int64_t n;
    int32_t d, nlist, metric, M, bits;
    const float* centroids;      /* [nlist*d] */
    const int64_t* list_offsets; /* [nlist+1] */
    const int64_t* ids;          /* [n] list order */
    const uint8_t* codes;        /* [n*code_bytes] list order */
    const float* books;          /* [M*2^bits*d/M] */
    const float* vectors;        /* [n*d] id order */
    int32_t residual;            /* 1: codes are PQ codes of o - c_l (residual IVF-PQ) */
    int32_t lut_levels;          /* top level of the integer table (0: 65535) */
} oracle_ivfpq;

/* collector: 0 = sort, 1 = heap, 2 = bucket (Algorithm 1).
 * Kc = candidates kept for the re-rank (the paper's n_cand).
 * stats (optional, per query): [0] S_q scanned, [1] candidates, [2] tau,
 * [3] pushed (bucket collector only). */
int oracle_search(const oracle_ivfpq* ix, const float* queries, int64_t nq, int32_t k,
                  int32_t nprobe, int64_t Kc, int32_t collector, int32_t m, int32_t sample_min,
                  int64_t* out_ids, double* out_d, int64_t* stats) {
    if (k <= 0 || nprobe < 1 || nprobe > ix->nlist || Kc < 1) return -1;
    if (ix->lut_levels < 0 || ix->lut_levels > 65535) return -1;
    /* the residual keys are defined on the uint16 table's scale */
    if (ix->residual && ix->lut_levels != 0 && ix->lut_levels != 65535) return -1;
    const int32_t d = ix->d, K = 1 << ix->bits, cb = ix->M * ix->bits / 8;
    int32_t* lists = (int32_t*)malloc(sizeof(int32_t) * (size_t)nprobe);
    uint16_t* lut = (uint16_t*)malloc(sizeof(uint16_t) * (size_t)ix->M * K);
    int64_t sq_max = 0;
    for (int32_t l = 0; l < ix->nlist; ++l) {
        int64_t s = ix->list_offsets[l + 1] - ix->list_offsets[l];
        sq_max += s;
    }
    uint32_t* e = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(sq_max + 1));
    int64_t* sid = (int64_t*)malloc(sizeof(int64_t) * (size_t)(sq_max + 1));
    int64_t* lofs = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nprobe + 1));
    int64_t* cand = (int64_t*)malloc(sizeof(int64_t) * (size_t)Kc);
    double* cd = (double*)malloc(sizeof(double) * (size_t)Kc);
    int64_t* cnts = (int64_t*)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
    for (int64_t qi = 0; qi < nq; ++qi) {
        const float* q = queries + (size_t)qi * d;
        oracle_probe(q, ix->centroids, ix->nlist, d, ix->metric, nprobe, lists, NULL);
        oracle_lut_q(q, ix->books, d, ix->M, ix->bits, ix->metric, ix->lut_levels > 0 ? ix->lut_levels : 65535,
                     lut, NULL);
        const float inv = ix->residual ? oracle_lut16_scale(q, ix->books, d, ix->M, ix->bits, ix->metric, NULL)
                                       : 0.0f;
        int64_t sq = 0;
        lofs[0] = 0;
        for (int32_t j = 0; j < nprobe; ++j) {
            int64_t a = ix->list_offsets[lists[j]], b = ix->list_offsets[lists[j] + 1];
            if (ix->residual)
                oracle_adc_resid(lut, ix->codes + (size_t)a * cb, b - a, ix->M, ix->bits, q,
                                 ix->centroids + (size_t)lists[j] * d, ix->books, d, ix->metric, inv, e + sq);
            else
                oracle_adc(lut, ix->codes + (size_t)a * cb, b - a, ix->M, ix->bits, e + sq);
            for (int64_t i = a; i < b; ++i) sid[sq + (i - a)] = ix->ids[i];
            sq += b - a;
            lofs[j + 1] = sq;
        }
        int64_t nc;
        oracle_codebook cbk;
        memset(&cbk, 0, sizeof(cbk));
        if (collector == 0) nc = oracle_topkc_sort(e, sid, sq, Kc, cand, NULL);
        else if (collector == 1) nc = oracle_topkc_heap(e, sid, sq, Kc, cand, NULL);
        else nc = oracle_bucket_collect(e, sid, lofs, nprobe, Kc, m, sample_min, &cbk, cnts, cand, NULL);
        oracle_rerank(q, ix->vectors, d, ix->metric, cand, nc, cd);
        oracle_topk_final(cd, cand, nc, k, out_ids + (size_t)qi * k, out_d + (size_t)qi * k);
        if (stats) {
            stats[qi * 4 + 0] = sq;
            stats[qi * 4 + 1] = nc;
            stats[qi * 4 + 2] = collector == 2 ? cbk.tau : -1;
            stats[qi * 4 + 3] = collector == 2 ? cbk.pushed : -1;
        }
    }
    free(lists); free(lut); free(e); free(sid); free(lofs); free(cand); free(cd); free(cnts);
    return 0;
}

/* Algorithm 4 (Improved Search Algorithm of IVF+PQ) on the result buffer of
 * Algorithm 1, lists in probe order:
 *   1-3. the sample and its codebook as in oracle_bucket_collect (the sampled
 *        lists' objects enter the buffer with their quantised distances);
 *   4.   tau_pred = the bucket of the r-th smallest quantised distance of the
 *        scanned objects, r = ceil(|O_scanned| / |O| * n_cand) (at least 1),
 *        O the objects of all probed lists;
 *   5-13 every other list: an object whose bucket a <= tau enters the buffer;
 *        if also a < tau_pred, its exact distance is computed now (early);
 *   14.  after each list tau_pred (rule 4) and tau (Update) are refreshed;
 *   15.  the candidates are Collect's n_cand (Algorithm 1), and the re-rank
 *        computes the exact distance of those without one.
 * Reading: the buffer orders objects by their quantised distance (the bucket
 * ids come from it), and an early exact distance travels with its object, so
 * the candidates are those of Algorithm 1 and the results those of the plain
 * re-rank; what changes is when exact distances are computed.  Returns the
 * number of candidates (written to out_ids, ascending by (e, id)); early_flag
 * (per candidate, may be NULL) marks the early ones; *n_early = objects
 * scored early, *n_early_cand = those among the candidates. */
int64_t oracle_alg4(const uint32_t* e, const int64_t* ids, const int64_t* list_ofs, int32_t nl, int64_t Kc,
                    int32_t m, int32_t sample_min, int64_t* out_ids, uint8_t* early_flag, int64_t* n_early,
                    int64_t* n_early_cand) {
    const int64_t Sq = list_ofs[nl] - list_ofs[0];
    const int64_t want = Kc < Sq ? Kc : Sq;
    int32_t ns_lists = sample_min < nl ? sample_min : nl;
    while (ns_lists < nl && list_ofs[ns_lists] - list_ofs[0] < want) ++ns_lists;
    const int64_t ns = list_ofs[ns_lists] - list_ofs[0];
    oracle_codebook cb;
    memset(&cb, 0, sizeof(cb));
    oracle_build_codebook(e + list_ofs[0], ns, Kc, m, &cb);
    int64_t* cnt = (int64_t*)calloc((size_t)m, sizeof(int64_t));
    uint32_t* seen = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(Sq > 0 ? Sq : 1));
    uint32_t* sorted = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(Sq > 0 ? Sq : 1));
    char* early = (char*)calloc((size_t)(Sq > 0 ? Sq : 1), 1);
    char* in_buf = (char*)calloc((size_t)(Sq > 0 ? Sq : 1), 1);
    int64_t nseen = 0, ne = 0;
    int32_t tau = m, tau_pred = m;
    for (int32_t j = 0; j < nl; ++j) {
        const int sampled = j < ns_lists;
        for (int64_t i = list_ofs[j]; i < list_ofs[j + 1]; ++i) {
            const int32_t a = bucket_of(e[i], &cb);
            if (a <= tau) {
                in_buf[i - list_ofs[0]] = 1;
                cnt[a]++;
                if (!sampled && a < tau_pred) { early[i - list_ofs[0]] = 1; ++ne; }
            }
            seen[nseen++] = e[i];
        }
        tau = oracle_update(cnt, m, Kc);
        if (j + 1 >= ns_lists && nseen > 0) {
            /* rule 4 on every object scanned so far */
            int64_t r = (int64_t)ceil((double)nseen / (double)Sq * (double)Kc);
            if (r < 1) r = 1;
            if (r > nseen) r = nseen;
            memcpy(sorted, seen, sizeof(uint32_t) * (size_t)nseen);
            qsort(sorted, (size_t)nseen, sizeof(uint32_t), cmp_u32);
            tau_pred = bucket_of(sorted[r - 1], &cb);
        }
    }
    /* Collect: the Kc smallest (e, id) of the buffer (Algorithm 1) */
    int64_t nb = 0;
    ukey* all = (ukey*)malloc(sizeof(ukey) * (size_t)(Sq > 0 ? Sq : 1));
    int64_t* pos = (int64_t*)malloc(sizeof(int64_t) * (size_t)(Sq > 0 ? Sq : 1));
    for (int64_t i = 0; i < Sq; ++i)
        if (in_buf[i]) { all[nb].e = e[list_ofs[0] + i]; all[nb].id = ids[list_ofs[0] + i]; pos[nb] = i; ++nb; }
    /* sort by (e, id); ids are unique, so the position follows from the id */
    qsort(all, (size_t)nb, sizeof(ukey), cmp_ukey);
    const int64_t nc = nb < Kc ? nb : Kc;
    int64_t nec = 0;
    for (int64_t t = 0; t < nc; ++t) {
        out_ids[t] = all[t].id;
        int64_t u = 0;                                 /* the object's position among the scanned */
        while (ids[list_ofs[0] + u] != all[t].id) ++u;
        const int ee = early[u];
        if (early_flag) early_flag[t] = (uint8_t)ee;
        nec += ee;
    }
    *n_early = ne;
    *n_early_cand = nec;
    free(cnt); free(seen); free(sorted); free(early); free(in_buf); free(all); free(pos);
    return nc;
}

/* Exact kNN over all n vectors, FP64. */
void oracle_bruteforce(const float* queries, int64_t nq, const float* x, int64_t n, int32_t d,
                       int32_t metric, int32_t k, int64_t* out_ids, double* out_d) {
    double* dist = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    int64_t* ids = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) ids[i] = i;
    for (int64_t qi = 0; qi < nq; ++qi) {
        for (int64_t i = 0; i < n; ++i)
            dist[i] = oracle_dist(queries + (size_t)qi * d, x + (size_t)i * d, d, metric);
        oracle_topk_final(dist, ids, n, k, out_ids + (size_t)qi * k, out_d + (size_t)qi * k);
    }
    free(dist);
    free(ids);
}

/* ------------------------------------------------------------------ */
/* low-precision copies (precision form of the re-rank)                 */
/* ------------------------------------------------------------------ */
/* bfloat16 bits of x: binary32's sign and 8 exponent bits with the fraction
 * rounded to 7 bits, to nearest, ties to even.  Values below 2^-126 sit on
 * the subnormal grid of spacing 2^-133.  NaN -> 0x7FC0. */
uint16_t oracle_bf16_bits(float x) {
    if (isnan(x)) return 0x7FC0;
    const double a = fabs((double)x);
    double r;
    if (a == 0.0 || isinf(x)) {
        r = a;
    } else if (a < ldexp(1.0, -126)) {
        r = ldexp(nearbyint(ldexp(a, 133)), -133);
    } else {
        int e;
        frexp(a, &e);                                  /* a in [2^(e-1), 2^e) */
        r = ldexp(nearbyint(ldexp(a, 8 - e)), e - 8);  /* 8 significant bits */
    }
    float y = r >= ldexp(1.0, 128) ? INFINITY : (float)r;   /* exact below the overflow */
    if (signbit(x)) y = -y;
    uint32_t u;
    memcpy(&u, &y, 4);
    return (uint16_t)(u >> 16);
}

double oracle_bf16_value(uint16_t b) {
    uint32_t u = (uint32_t)b << 16;
    float f;
    memcpy(&f, &u, 4);
    return (double)f;
}

/* E4M3 bits of x: normals (1 + f/8) 2^(e-7), e = 1..15 (e = 15, f = 7 is
 * NaN), subnormals f 2^-9; nearest, ties to even; |x| >= 448 saturates to
 * 448.  NaN -> 0x7F. */
uint8_t oracle_e4m3_bits(float x) {
    if (isnan(x)) return 0x7F;
    const uint8_t sgn = signbit(x) ? 0x80 : 0x00;
    const double a = fabs((double)x);
    if (a >= 448.0) return (uint8_t)(sgn | 0x7E);
    if (a < ldexp(1.0, -6)) return (uint8_t)(sgn | (uint8_t)nearbyint(a * 512.0));   /* 8 -> 2^-6 */
    int e;
    frexp(a, &e);
    int E = e - 1;                                     /* a = 1.f * 2^E, E >= -6 */
    double q = nearbyint(ldexp(a, 3 - E));             /* 8..16 */
    if (q == 16.0) { q = 8.0; E += 1; }
    return (uint8_t)(sgn | (uint8_t)(((E + 7) << 3) | ((int)q - 8)));
}

double oracle_e4m3_value(uint8_t b) {
    const int e = (b >> 3) & 15, f = b & 7;
    const double v = e == 0 ? ldexp((double)f, -9) : ldexp((double)(8 + f), e - 10);
    return (b & 0x80) ? -v : v;
}

/* Copy of n vectors [n*d] into rows [n*dpad] (zero padded): prec 1 = BF16 bits
 * (u16), prec 2 = E4M3 bytes of x / s with s = amax / 448 in FP32 (1 when that
 * is not a positive finite number).  meta4 per vector: s, e_v = ||x - v~||_2
 * (v~ = the copy's value times s), ||x||_2, 0 -- FP64, not rounded. */
void oracle_prec_copy(const float* v, int64_t n, int32_t d, int32_t dpad, int32_t prec, void* rows,
                      double* meta4) {
    for (int64_t i = 0; i < n; ++i) {
        const float* x = v + (size_t)i * d;
        float amax = 0.0f;
        for (int32_t j = 0; j < d; ++j) amax = fabsf(x[j]) > amax ? fabsf(x[j]) : amax;
        float s = 1.0f;
        if (prec == 2) {
            s = amax / 448.0f;
            if (!(s > 0.0f) || !isfinite(s)) s = 1.0f;
        }
        double e2 = 0.0, n2 = 0.0;
        for (int32_t j = 0; j < dpad; ++j) {
            const float xj = j < d ? x[j] : 0.0f;
            double vt;
            if (prec == 2) {
                const float y = xj / s;
                const uint8_t c = oracle_e4m3_bits(y);
                ((uint8_t*)rows)[(size_t)i * dpad + j] = c;
                vt = oracle_e4m3_value(c) * (double)s;
            } else {
                const uint16_t b = oracle_bf16_bits(xj);
                ((uint16_t*)rows)[(size_t)i * dpad + j] = b;
                vt = oracle_bf16_value(b);
            }
            e2 += ((double)xj - vt) * ((double)xj - vt);
            n2 += (double)xj * (double)xj;
        }
        meta4[i * 4 + 0] = s;
        meta4[i * 4 + 1] = sqrt(e2);
        meta4[i * 4 + 2] = sqrt(n2);
        meta4[i * 4 + 3] = 0.0;
    }
}

/* ------------------------------------------------------------------ */
/* 1-bit sign quantizer with per-object bounds (bounded re-rank)        */
/* ------------------------------------------------------------------ */
/* Codes of the rotated residual (Section 2 cites RaBitQ for bounded
 * methods without stating its estimator; this is the deterministic reading
 * used here).  For object o in list l: u = o - c_l, r = P u (FP64, P the
 * FP32-stored rotation), s_i = +1 if r_i > 0 else -1, alpha = <s, r> / d =
 * mean |r_i|, e = ||r - alpha s||, un2 = ||u||^2.  Codes are d/32 words per
 * object (bit i of word w = [r_(32w+i) > 0]), in list order.  fac[4] =
 * {alpha, e, un2, popcount of the code}. */
void oracle_sign_encode(const float* vectors, int32_t d, const float* centroids, int32_t nlist,
                        const int64_t* list_offsets, const int64_t* ids, const float* rot,
                        uint32_t* codes, double* fac) {
    const int32_t W = d / 32;
    double* u = (double*)malloc(sizeof(double) * (size_t)d);
    double* r = (double*)malloc(sizeof(double) * (size_t)d);
    for (int32_t l = 0; l < nlist; ++l) {
        for (int64_t p = list_offsets[l]; p < list_offsets[l + 1]; ++p) {
            const float* o = vectors + (size_t)ids[p] * d;
            const float* c = centroids + (size_t)l * d;
            double un2 = 0.0;
            for (int32_t i = 0; i < d; ++i) { u[i] = (double)o[i] - (double)c[i]; un2 += u[i] * u[i]; }
            double sabs = 0.0;
            for (int32_t i = 0; i < d; ++i) {
                double t = 0.0;
                for (int32_t j = 0; j < d; ++j) t += (double)rot[(size_t)i * d + j] * u[j];
                r[i] = t;
                sabs += fabs(t);
            }
            const double alpha = sabs / d;
            double e2 = 0.0;
            int64_t pc = 0;
            uint32_t* cw = codes + (size_t)p * W;
            for (int32_t w = 0; w < W; ++w) cw[w] = 0;
            for (int32_t i = 0; i < d; ++i) {
                const double s = r[i] > 0.0 ? 1.0 : -1.0;
                if (r[i] > 0.0) { cw[i / 32] |= 1u << (i % 32); ++pc; }
                e2 += (r[i] - alpha * s) * (r[i] - alpha * s);
            }
            fac[p * 4 + 0] = alpha;
            fac[p * 4 + 1] = sqrt(e2);
            fac[p * 4 + 2] = un2;
            fac[p * 4 + 3] = (double)pc;
        }
    }
    free(u);
    free(r);
}

/* ||P^T P - I||_F in FP64: bounds |<P t, P u> - <t, u>| <= eps ||t|| ||u||. */
double oracle_rotation_eps(const float* rot, int32_t d) {
    double s = 0.0;
    for (int32_t i = 0; i < d; ++i) {
        for (int32_t j = 0; j < d; ++j) {
            double t = 0.0;
            for (int32_t k = 0; k < d; ++k) t += (double)rot[(size_t)k * d + i] * (double)rot[(size_t)k * d + j];
            if (i == j) t -= 1.0;
            s += t * t;
        }
    }
    return sqrt(s);
}

/* Bounds [lb, ub] on ||q - o||^2 for the objects of list l (positions
 * list_offsets[l] .. list_offsets[l+1]), all in FP64:
 *   t = q - c_l, q' = P t; 4-bit query: lo = min q', Delta = (max q' - lo) / 15,
 *   u_i = nearest integer to (q'_i - lo) / Delta in [0, 15], q~ = lo + Delta u,
 *   eta = ||q' - q~||;
 *   X = <q~, s> = lo (2 pc - d) + Delta (2 sum_i u_i b_i - sum_i u_i)   (b = code bits);
 *   <q', r> in alpha X +- scale (||q'|| e + |alpha| eta sqrt(d));
 *   ||q - o||^2 = ||t||^2 + ||u||^2 - 2 <t, u>, |<t, u> - <q', r>| <= eps ||t|| ||u||;
 * plus a relative FP64 allowance of 1e-12.  scale multiplies the two
 * Cauchy-Schwarz terms; 1 gives hard bounds. */
void oracle_sign_bounds(const float* q, int32_t d, const float* centroid, const float* rot, double eps,
                        const uint32_t* codes, const double* fac, int64_t n, double scale,
                        double* lb, double* ub) {
    const int32_t W = d / 32;
    double* t = (double*)malloc(sizeof(double) * (size_t)d);
    double* qr = (double*)malloc(sizeof(double) * (size_t)d);
    int32_t* uq = (int32_t*)malloc(sizeof(int32_t) * (size_t)d);
    double tn2 = 0.0;
    for (int32_t i = 0; i < d; ++i) { t[i] = (double)q[i] - (double)centroid[i]; tn2 += t[i] * t[i]; }
    double lo = INFINITY, hi = -INFINITY, qn2 = 0.0;
    for (int32_t i = 0; i < d; ++i) {
        double a = 0.0;
        for (int32_t j = 0; j < d; ++j) a += (double)rot[(size_t)i * d + j] * t[j];
        qr[i] = a;
        qn2 += a * a;
        if (a < lo) lo = a;
        if (a > hi) hi = a;
    }
    const double delta = (hi - lo) / 15.0;
    double eta2 = 0.0;
    int64_t usum = 0;
    for (int32_t i = 0; i < d; ++i) {
        int32_t ui = 0;
        if (delta > 0.0) {
            double v = nearbyint((qr[i] - lo) / delta);
            ui = v < 0.0 ? 0 : (v > 15.0 ? 15 : (int32_t)v);
        }
        uq[i] = ui;
        usum += ui;
        const double diff = qr[i] - (lo + delta * ui);
        eta2 += diff * diff;
    }
    const double eta = sqrt(eta2), qn = sqrt(qn2), tn = sqrt(tn2), sd = sqrt((double)d);
    for (int64_t p = 0; p < n; ++p) {
        const uint32_t* cw = codes + (size_t)p * W;
        int64_t ub_sum = 0;
        for (int32_t i = 0; i < d; ++i)
            if ((cw[i / 32] >> (i % 32)) & 1u) ub_sum += uq[i];
        const double alpha = fac[p * 4 + 0], e = fac[p * 4 + 1], un2 = fac[p * 4 + 2], pc = fac[p * 4 + 3];
        const double X = lo * (2.0 * pc - d) + delta * (2.0 * (double)ub_sum - (double)usum);
        const double est = alpha * X;
        const double half = scale * (qn * e + fabs(alpha) * eta * sd);
        const double rot_err = 2.0 * eps * tn * sqrt(un2);
        const double base = tn2 + un2;
        const double slack = 1e-12 * (base + 2.0 * fabs(est) + 2.0 * half + rot_err);
        double l = base - 2.0 * (est + half) - rot_err - slack;
        lb[p] = l > 0.0 ? l : 0.0;
        ub[p] = base - 2.0 * (est - half) + rot_err + slack;
    }
    free(t);
    free(qr);
    free(uq);
}

/* Bounds on ||q - o||^2 from the RaBitQ estimator, FP64, for the objects of
 * list l (same inputs and 4-bit query as oracle_sign_bounds).  In RaBitQ's
 * notation, with unit vectors o_r = r / ||r|| (r = P u, u = o - c_l),
 * q_r = q' / ||q'|| and the quantised unit vector o_bar = s / sqrt(d):
 *   <o_bar, o_r> = <s, r> / (sqrt(d) ||r||) = alpha sqrt(d) / ||r||;
 *   estimator   <o_r, q_r> ~ <o_bar, q_r> / <o_bar, o_r>;
 *   error bound |estimate - <o_r, q_r>| <= sqrt((1 - <o_bar, o_r>^2) / <o_bar, o_r>^2)
 *                                          * epsilon_0 / sqrt(d - 1)
 * with high probability over the random rotation.  Since alpha is the mean
 * |r_i|, r - alpha s is orthogonal to s and ||r||^2 = e^2 + d alpha^2 (e =
 * ||r - alpha s||), so <o_bar, o_r> and ||r|| come from the stored factors;
 * q_r is replaced by the 4-bit query q~.  Under the random rotation <s, q' - q~> behaves like a sum
 * of d terms of random sign, standard deviation ||q' - q~|| = eta, so its
 * share of the error is taken at the same confidence, epsilon_0 eta (the
 * worst case is sqrt(d) eta).  The estimate of <q', r> = ||q'|| ||r|| <o_r, q_r>
 * then gives
 *   <q', r> in ||r||^2 / (d alpha) <s, q~>
 *              +- ( ||q'|| ||r|| sqrt(1 / <o_bar, o_r>^2 - 1) epsilon_0 / sqrt(d - 1)
 *                   + ||r||^2 / (d alpha) epsilon_0 eta ).
 * The distance then follows as in oracle_sign_bounds.  An object with
 * alpha = 0 (o at its centroid) keeps the hard bound. */
void oracle_sign_bounds_rq(const float* q, int32_t d, const float* centroid, const float* rot, double eps,
                           const uint32_t* codes, const double* fac, int64_t n, double eps0,
                           double* lb, double* ub) {
    const int32_t W = d / 32;
    double* t = (double*)malloc(sizeof(double) * (size_t)d);
    double* qr = (double*)malloc(sizeof(double) * (size_t)d);
    int32_t* uq = (int32_t*)malloc(sizeof(int32_t) * (size_t)d);
    double tn2 = 0.0;
    for (int32_t i = 0; i < d; ++i) { t[i] = (double)q[i] - (double)centroid[i]; tn2 += t[i] * t[i]; }
    double lo = INFINITY, hi = -INFINITY, qn2 = 0.0;
    for (int32_t i = 0; i < d; ++i) {
        double a = 0.0;
        for (int32_t j = 0; j < d; ++j) a += (double)rot[(size_t)i * d + j] * t[j];
        qr[i] = a;
        qn2 += a * a;
        if (a < lo) lo = a;
        if (a > hi) hi = a;
    }
    const double delta = (hi - lo) / 15.0;
    double eta2 = 0.0;
    int64_t usum = 0;
    for (int32_t i = 0; i < d; ++i) {
        int32_t ui = 0;
        if (delta > 0.0) {
            double v = nearbyint((qr[i] - lo) / delta);
            ui = v < 0.0 ? 0 : (v > 15.0 ? 15 : (int32_t)v);
        }
        uq[i] = ui;
        usum += ui;
        const double diff = qr[i] - (lo + delta * ui);
        eta2 += diff * diff;
    }
    const double eta = sqrt(eta2), qn = sqrt(qn2), tn = sqrt(tn2), sd = sqrt((double)d);
    const double tail = eps0 / sqrt((double)(d > 1 ? d - 1 : 1));
    for (int64_t p = 0; p < n; ++p) {
        const uint32_t* cw = codes + (size_t)p * W;
        int64_t ub_sum = 0;
        for (int32_t i = 0; i < d; ++i)
            if ((cw[i / 32] >> (i % 32)) & 1u) ub_sum += uq[i];
        const double alpha = fac[p * 4 + 0], e = fac[p * 4 + 1], un2 = fac[p * 4 + 2], pc = fac[p * 4 + 3];
        const double X = lo * (2.0 * pc - d) + delta * (2.0 * (double)ub_sum - (double)usum);   /* <s, q~> */
        const double rn = sqrt(e * e + (double)d * alpha * alpha);    /* ||r|| */
        double est, half;
        if (alpha > 0.0 && rn > 0.0) {
            const double ip_bar = alpha * sd / rn;                     /* <o_bar, o_r> */
            double spread = (1.0 - ip_bar * ip_bar) / (ip_bar * ip_bar);
            if (spread < 0.0) spread = 0.0;
            const double kappa = rn * rn / ((double)d * alpha);        /* ||r||^2 / (d alpha) */
            est = kappa * X;
            half = qn * rn * sqrt(spread) * tail + kappa * eps0 * eta;
        } else {
            est = alpha * X;
            half = qn * e + fabs(alpha) * eta * sd;
        }
        const double rot_err = 2.0 * eps * tn * sqrt(un2);
        const double base = tn2 + un2;
        const double slack = 1e-12 * (base + 2.0 * fabs(est) + 2.0 * half + rot_err);
        double l = base - 2.0 * (est + half) - rot_err - slack;
        lb[p] = l > 0.0 ? l : 0.0;
        ub[p] = base - 2.0 * (est - half) + rot_err + slack;
    }
    free(t);
    free(qr);
    free(uq);
}

/* ---- binary heaps over (key, index) for Algorithm 2 ---- */
typedef struct { double key; int64_t i; } hitem;
static int hless(hitem a, hitem b) { return a.key < b.key || (a.key == b.key && a.i < b.i); }
/* max-heap when mx = 1, min-heap when mx = 0 */
static int hbefore(hitem a, hitem b, int mx) { return mx ? hless(b, a) : hless(a, b); }
static void hpush(hitem* h, int64_t* n, hitem x, int mx) {
    int64_t i = (*n)++;
    h[i] = x;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (!hbefore(h[i], h[p], mx)) break;
        hitem t = h[i]; h[i] = h[p]; h[p] = t;
        i = p;
    }
}
static hitem hpop(hitem* h, int64_t* n, int mx) {
    hitem top = h[0];
    h[0] = h[--(*n)];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, b = i;
        if (l < *n && hbefore(h[l], h[b], mx)) b = l;
        if (r < *n && hbefore(h[r], h[b], mx)) b = r;
        if (b == i) break;
        hitem t = h[i]; h[i] = h[b]; h[b] = t;
        i = b;
    }
    return top;
}

/* Algorithm 2 (minimal re-ranking of a bounded method) over n objects with
 * bounds [lb, ub] and exact distances ex (evaluated only when re-ranked).
 * H_u is a max-heap on ub of at most k objects; H_l a min-heap on lb.  After
 * the collection phase, the object with the smaller lower bound among the
 * two tops is re-ranked (its bounds collapse to its exact distance) while the
 * top upper bound of H_u exceeds the top lower bound of H_l.  Ties in keys
 * go to the smaller index.  Writes the result (indices into the arrays, at
 * most k) to out_idx and returns the number of exact distances computed. */
int64_t oracle_alg2(const double* lb, const double* ub, const double* ex, int64_t n, int32_t k,
                    int64_t* out_idx, int64_t* out_n) {
    hitem* hu = (hitem*)malloc(sizeof(hitem) * (size_t)(k + 2));
    hitem* hl = (hitem*)malloc(sizeof(hitem) * (size_t)(n + 2));
    double* cl = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));   /* current lb */
    double* cu = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));   /* current ub */
    char* vis = (char*)calloc((size_t)(n > 0 ? n : 1), 1);
    int64_t nu = 0, nl = 0, reranked = 0;
    for (int64_t i = 0; i < n; ++i) { cl[i] = lb[i]; cu[i] = ub[i]; }
    for (int64_t i = 0; i < n; ++i) {
        const double top = nu < k ? INFINITY : hu[0].key;
        if (cu[i] < top) {
            hitem x = {cu[i], i};
            hpush(hu, &nu, x, 1);
            if (nu > k) {
                hitem m = hpop(hu, &nu, 1);
                hitem y = {cl[m.i], m.i};
                hpush(hl, &nl, y, 0);
            }
        } else if (cl[i] < top) {
            hitem y = {cl[i], i};
            hpush(hl, &nl, y, 0);
        }
    }
    for (;;) {
        const double utop = nu < k ? INFINITY : hu[0].key;
        const double ltop = nl > 0 ? hl[0].key : INFINITY;
        if (!(utop > ltop)) break;
        /* the top of H_u with the larger upper bound, or the top of H_l */
        int from_u = nu > 0 && !vis[hu[0].i] && cl[hu[0].i] < ltop;
        int64_t o;
        if (from_u) o = hpop(hu, &nu, 1).i;
        else o = hpop(hl, &nl, 0).i;
        if (vis[o]) continue;
        vis[o] = 1;
        ++reranked;
        cl[o] = cu[o] = ex[o];
        hitem x = {ex[o], o};
        hpush(hu, &nu, x, 1);
        if (nu > k) {
            hitem m = hpop(hu, &nu, 1);
            if (!vis[m.i]) {
                hitem y = {cl[m.i], m.i};
                hpush(hl, &nl, y, 0);
            }
        }
    }
    *out_n = nu;
    for (int64_t i = 0; i < nu; ++i) out_idx[i] = hu[i].i;
    free(hu); free(hl); free(cl); free(cu); free(vis);
    return reranked;
}

/* Observation 1: objects whose bounds enclose Dist_k, the distance of the
 * k-th object in (exact, index) order. */
int64_t oracle_obs1_count(const double* lb, const double* ub, const double* ex, int64_t n, int32_t k) {
    if (n <= k || k <= 0) return 0;
    dkey* a = (dkey*)malloc(sizeof(dkey) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) { a[i].s = ex[i]; a[i].id = i; }
    qsort(a, (size_t)n, sizeof(dkey), cmp_dkey);
    const double dk = a[k - 1].s;
    free(a);
    int64_t c = 0;
    for (int64_t i = 0; i < n; ++i) c += (lb[i] <= dk && dk <= ub[i]) ? 1 : 0;
    return c;
}

/* The one-shot classification of the bounded re-rank: U_k = k-th smallest
 * ub, S = {lb <= U_k}, L = (k+1)-th smallest lb over S; certainly in
 * (ub < L), to decide (the rest of S).  Returns |S| and writes |in|, |R|. */
int64_t oracle_oneshot(const double* lb, const double* ub, int64_t n, int32_t k, int64_t* n_in,
                       int64_t* n_r) {
    if (n <= k) { *n_in = n; *n_r = 0; return n; }
    double* v = (double*)malloc(sizeof(double) * (size_t)n);
    memcpy(v, ub, sizeof(double) * (size_t)n);
    qsort(v, (size_t)n, sizeof(double), cmp_double);
    const double uk = v[k - 1];
    int64_t ns = 0;
    for (int64_t i = 0; i < n; ++i)
        if (lb[i] <= uk) v[ns++] = lb[i];
    if (ns <= k) { free(v); *n_in = ns; *n_r = 0; return ns; }
    qsort(v, (size_t)ns, sizeof(double), cmp_double);
    const double l1 = v[k];
    int64_t in = 0;
    for (int64_t i = 0; i < n; ++i)
        if (lb[i] <= uk && ub[i] < l1) ++in;
    free(v);
    *n_in = in;
    *n_r = ns - in;
    return ns;
}

/* The bounded re-rank with exact returned distances, in two rounds (the
 * batched form of Algorithm 3's marginal re-ranking):
 *   1. U_k = k-th smallest ub; S = {lb <= U_k} (every member of the top-k).
 *   2. B = the ceil(first * k) members of S with the smallest interval
 *      centre (lb + ub) / 2 (index breaking ties), all of S when it is not
 *      larger; re-rank B; U' = the k-th smallest exact distance in B, an
 *      upper bound of Dist_k (any k objects have a k-th smallest >= Dist_k).
 *   3. S' = {o in S \ B : lb_o <= U'}; re-rank S'.
 *   4. Result: the k smallest (exact, index) of B u S'.
 * Every object outside B u S' has lb > U' >= Dist_k, so it is not among the
 * top k.  The centres pick, among objects whose intervals all reach below
 * U_k, the likeliest members first, so U' lands near Dist_k and S' stays
 * small.  Writes the result indices (sorted) and returns the number of exact
 * distances computed (|B| + |S'|). */
int64_t oracle_rounds(const double* lb, const double* ub, const double* ex, int64_t n, int32_t k, double first,
                      int64_t* out_idx, int64_t* out_n) {
    dkey* a = (dkey*)malloc(sizeof(dkey) * (size_t)(n > 0 ? n : 1));
    char* re = (char*)calloc((size_t)(n > 0 ? n : 1), 1);
    int64_t count = 0;
    if (n <= k) {
        for (int64_t i = 0; i < n; ++i) re[i] = 1;
        count = n;
    } else {
        for (int64_t i = 0; i < n; ++i) { a[i].s = ub[i]; a[i].id = i; }
        qsort(a, (size_t)n, sizeof(dkey), cmp_dkey);
        const double uk = a[k - 1].s;
        int64_t ns = 0;                                    /* S, ordered by (centre, index) */
        for (int64_t i = 0; i < n; ++i)
            if (lb[i] <= uk) { a[ns].s = 0.5 * (lb[i] + ub[i]); a[ns].id = i; ++ns; }
        qsort(a, (size_t)ns, sizeof(dkey), cmp_dkey);
        int64_t nb = (int64_t)ceil(first * (double)k);
        if (nb > ns) nb = ns;
        double* eb = (double*)malloc(sizeof(double) * (size_t)(nb > 0 ? nb : 1));
        for (int64_t j = 0; j < nb; ++j) { re[a[j].id] = 1; eb[j] = ex[a[j].id]; }
        qsort(eb, (size_t)nb, sizeof(double), cmp_double);
        const double up = eb[(k < nb ? k : nb) - 1];
        free(eb);
        count = nb;
        for (int64_t i = 0; i < n; ++i) {
            if (!re[i] && lb[i] <= uk && lb[i] <= up) { re[i] = 1; ++count; }
        }
    }
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i)
        if (re[i]) { a[m].s = ex[i]; a[m].id = i; ++m; }
    qsort(a, (size_t)m, sizeof(dkey), cmp_dkey);
    *out_n = m < k ? m : k;
    for (int64_t i = 0; i < *out_n; ++i) out_idx[i] = a[i].id;
    free(a);
    free(re);
    return count;
}
