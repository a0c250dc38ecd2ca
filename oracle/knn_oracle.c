/*
 * knn_oracle.c -- plain, slow, double-precision CPU oracle for the adaptive
 * k-NN method (LeJeune, Baraniuk, Heckel, AISTATS 2019).
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the CPU
 * baseline of the benchmark; never by the product path. Shares no code with
 * the CUDA library.
 *
 * Pieces and where they come from:
 *   - Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw,
 *     "Parallel random numbers: as easy as 1, 2, 3", SC'11), written from the
 *     published round function.
 *   - coordinate draw: uniform index in [0, m) with replacement (Section 4,
 *     sampled estimator).
 *   - alpha(u): footnote form (Section 4), Lemma form (Lemma "probound",
 *     Section 6) and the experiment form with C_alpha (Section 5).
 *   - brute force: all distances then sort (Section 3).
 *   - batched rounds: every undecided point gets the same number of new
 *     samples per round; the elimination/acceptance rules are the batched
 *     form of the LUCB indices (Eq. d_ind) and of the termination argument
 *     (Eq. termination and the first paragraph of the proof of Theorem 1).
 *   - sequential: Algorithm 1 as printed (two arms per iteration).
 *   - block samples (not in the paper): with block g > 1 a sample is one of
 *     M = ceil(m/g) blocks of g consecutive coordinates, drawn uniformly with
 *     replacement, and its value the block's sum of squared differences. The
 *     block sum over g (times 1/span^2) lies in [0, 1], so the sampled
 *     estimator of Section 4 and its bounds apply with u = blocks drawn; its
 *     mean over all M blocks is d^2/(M g), the same for every point up to the
 *     factor d^2, and after M samples the estimate is exact (Algorithm 1's
 *     cap at T = m, with M in place of m).
 */
#include "knn_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- Philox */

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    /* Multipliers and Weyl key increments of Philox4x32 (SC'11, Table 2):
     * each round multiplies words 0 and 2, xors the high halves of the
     * 64-bit products with the other words and the round key, and the key
     * advances between rounds. */
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * c0, p1 = (uint64_t)M1 * c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0, n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1, n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Block `blk` of a (query, point) pair's stream: Philox4x32-10 at counter
 * (blk, point, query low word, query high word), key (seed low word, seed
 * high word). */
static void pair_block(uint64_t seed, uint64_t qid, uint64_t point, uint32_t blk, uint64_t mask_p,
                       uint64_t mask_q, uint32_t out[4]) {
    const uint64_t qf = qid & mask_q;
    uint32_t ctr[4] = {blk, (uint32_t)(point & mask_p), (uint32_t)qf, (uint32_t)(qf >> 32)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, out);
}

/* The s-th draw of a (query, point) pair: word s mod 4 of block s / 4,
 * scaled to [0, m) by floor(word * m / 2^32). */
int32_t orc_coordinate(uint64_t seed, uint64_t qid, uint64_t point, uint64_t s, int32_t m,
                       uint64_t mask_p, uint64_t mask_q) {
    uint32_t out[4];
    pair_block(seed, qid, point, (uint32_t)(s >> 2), mask_p, mask_q, out);
    uint32_t word = out[s & 3];
    return (int32_t)(((uint64_t)word * (uint64_t)(uint32_t)m) >> 32);
}

/* MurmurHash3's 32-bit finaliser (Appleby, public domain): the round
 * function of the permutation below. */
static uint32_t fmix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x85EBCA6Bu;
    x ^= x >> 13;
    x *= 0xC2B2AE35u;
    x ^= x >> 16;
    return x;
}

/* Eight Feistel rounds on the 2h-bit value x with round keys k[0..7]. */
static uint32_t feistel8(uint32_t x, int h, const uint32_t k[8]) {
    const uint32_t mask = (1u << h) - 1u;
    uint32_t L = x >> h, R = x & mask;
    for (int r = 0; r < 8; ++r) {
        uint32_t nL = R;
        uint32_t nR = L ^ (fmix32(R ^ k[r]) & mask);
        L = nL;
        R = nR;
    }
    return (L << h) | R;
}

int32_t orc_coordinate_wor(uint64_t seed, uint64_t qid, uint64_t point, uint64_t s, int32_t m,
                           uint64_t mask_p, uint64_t mask_q) {
    /* round keys: the two last blocks of the pair's stream */
    uint32_t k[8];
    pair_block(seed, qid, point, 0xFFFFFFFEu, mask_p, mask_q, k);
    pair_block(seed, qid, point, 0xFFFFFFFFu, mask_p, mask_q, k + 4);
    int bits = 0;
    while (((uint64_t)1 << bits) < (uint64_t)m) ++bits;  /* ceil(log2 m) */
    int h = (bits + 1) / 2;
    if (h < 1) h = 1;
    /* cycle walking: s < m lies on a cycle of the permutation of [0, 4^h),
     * so the walk meets a value below m again */
    uint32_t x = (uint32_t)s;
    do {
        x = feistel8(x, h, k);
    } while (x >= (uint32_t)m);
    return (int32_t)x;
}

/* ----------------------------------------------------------------- alpha */

double orc_alpha(int32_t form, double c_alpha, int64_t u, int64_t n, double delta) {
    double uu = (double)u;
    double dprime = delta / (double)n;
    if (form == ORC_BOUND_FOOTNOTE) {
        /* beta(u, delta') = log(1/delta') + 3 log log(1/delta') + 1.5 log(1 + log u) */
        double beta = log(1.0 / dprime) + 3.0 * log(log(1.0 / dprime)) + 1.5 * log(1.0 + log(uu));
        return sqrt(2.0 * beta / uu);
    }
    if (form == ORC_BOUND_LEMMA) {
        /* beta(t, delta') = 2 log(125 log(1.12 t) / delta') */
        double beta = 2.0 * log(125.0 * log(1.12 * uu) / dprime);
        return sqrt(2.0 * beta / uu);
    }
    /* Section 5: sqrt(C_alpha log(1 + (1 + log u) n / delta) / u) */
    return sqrt(c_alpha * log(1.0 + (1.0 + log(uu)) * (double)n / delta) / uu);
}

/* ------------------------------------------------------------- storage */

/* bfloat16: keep the top 16 bits of the float, rounding to nearest with
 * ties to even (NaN is left as is). */
float orc_round_bf16(float x) {
    uint32_t u;
    memcpy(&u, &x, 4);
    if ((u & 0x7F800000u) == 0x7F800000u && (u & 0x007FFFFFu)) return x;
    u = (u + 0x7FFFu + ((u >> 16) & 1u)) & 0xFFFF0000u;
    float y;
    memcpy(&y, &u, 4);
    return y;
}

/* FP8 e4m3 (the variant without infinities): 3 fraction bits, normal
 * exponents -6..8, subnormal spacing 2^-9, largest finite 448; round to
 * nearest, ties to even, saturating at 448. */
float orc_round_e4m3(float x) {
    double a = fabs((double)x);
    if (a == 0.0 || a != a) return x;
    int ex;
    frexp(a, &ex);               /* a = f 2^ex, f in [0.5, 1): binade exponent ex - 1 */
    int e = ex - 1;
    if (e < -6) e = -6;          /* subnormal range shares the quantum of 2^-6 */
    double quantum = ldexp(1.0, e - 3);
    double r = rint(a / quantum) * quantum;   /* default rounding: ties to even */
    if (r > 448.0) r = 448.0;
    return (float)(x < 0 ? -r : r);
}

double orc_quantize(int32_t storage, const float* X, int64_t n, int32_t m, float* out, float* scale) {
    double emax = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        const float* xr = X + (size_t)i * (size_t)m;
        float* o = out + (size_t)i * (size_t)m;
        if (storage == ORC_STORE_BF16) {
            for (int32_t j = 0; j < m; ++j) o[j] = orc_round_bf16(xr[j]);
        } else if (storage == ORC_STORE_FP8) {
            float mx = 0.0f;
            for (int32_t j = 0; j < m; ++j) if (fabsf(xr[j]) > mx) mx = fabsf(xr[j]);
            volatile float s = mx > 0.0f ? mx / 448.0f : 1.0f;
            if (scale) scale[i] = s;
            for (int32_t j = 0; j < m; ++j) {
                volatile float t = xr[j] / s;
                float v = orc_round_e4m3(t);
                o[j] = (float)((double)s * (double)v);
            }
        } else {
            for (int32_t j = 0; j < m; ++j) o[j] = xr[j];
        }
        for (int32_t j = 0; j < m; ++j) {
            double d = fabs((double)o[j] - (double)xr[j]);
            if (d > emax) emax = d;
        }
    }
    return emax;
}

/* ----------------------------------------------------------- brute force */

typedef struct { double v; int64_t i; } vi_t;

static int cmp_vi(const void* a, const void* b) {
    const vi_t* x = (const vi_t*)a;
    const vi_t* y = (const vi_t*)b;
    if (x->v < y->v) return -1;
    if (x->v > y->v) return 1;
    return (x->i > y->i) - (x->i < y->i);
}

static double sqdist(const float* x, const float* q, int32_t m) {
    double s = 0.0;
    for (int32_t j = 0; j < m; ++j) {
        double d = (double)x[j] - (double)q[j];
        s += d * d;
    }
    return s;
}

/* l1 distance (the generalisation named in Section 3). */
static double l1dist(const float* x, const float* q, int32_t m) {
    double s = 0.0;
    for (int32_t j = 0; j < m; ++j) s += fabs((double)x[j] - (double)q[j]);
    return s;
}

static double dist_of(int32_t metric, const float* x, const float* q, int32_t m) {
    return metric == ORC_METRIC_L1 ? l1dist(x, q, m) : sqdist(x, q, m);
}

/* One coordinate's contribution: (x - q)^2, or |x - q| for l1. */
static double term_of(int32_t metric, double d) { return metric == ORC_METRIC_L1 ? fabs(d) : d * d; }

void orc_exact_knn_metric(const float* X, int64_t n, int32_t m, const float* q, int32_t k, int32_t metric,
                          int64_t* idx, double* dist) {
    vi_t* a = (vi_t*)malloc(sizeof(vi_t) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        a[i].v = dist_of(metric, X + (size_t)i * (size_t)m, q, m);
        a[i].i = i;
    }
    qsort(a, (size_t)n, sizeof(vi_t), cmp_vi);
    for (int32_t t = 0; t < k; ++t) {
        idx[t] = t < n ? a[t].i : -1;
        if (dist) dist[t] = t < n ? a[t].v : INFINITY;
    }
    free(a);
}

void orc_exact_knn(const float* X, int64_t n, int32_t m, const float* q, int32_t k,
                   int64_t* idx, double* dist) {
    orc_exact_knn_metric(X, n, m, q, k, ORC_METRIC_L2SQ, idx, dist);
}

void orc_exact_knn_batch_metric(const float* X, int64_t n, int32_t m, const float* Q, int32_t nq,
                                int32_t k, int32_t metric, int64_t* idx, double* dist, int32_t threads) {
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int32_t qi = 0; qi < nq; ++qi)
        orc_exact_knn_metric(X, n, m, Q + (size_t)qi * (size_t)m, k, metric, idx + (size_t)qi * (size_t)k,
                             dist ? dist + (size_t)qi * (size_t)k : NULL);
}

void orc_exact_knn_batch(const float* X, int64_t n, int32_t m, const float* Q, int32_t nq,
                         int32_t k, int64_t* idx, double* dist, int32_t threads) {
    orc_exact_knn_batch_metric(X, n, m, Q, nq, k, ORC_METRIC_L2SQ, idx, dist, threads);
}

int32_t orc_max_threads(void) {
#ifdef _OPENMP
    return (int32_t)omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------- batched rounds */

/* A bound value together with the magnitude (estimate + width) of the pair
 * it belongs to; the magnitude scales the near-threshold band. */
typedef struct { double v; double mag; } vm_t;

static int cmp_vm(const void* a, const void* b) {
    const vm_t* x = (const vm_t*)a;
    const vm_t* y = (const vm_t*)b;
    if (x->v < y->v) return -1;
    if (x->v > y->v) return 1;
    return (x->mag < y->mag) - (x->mag > y->mag); /* larger magnitude first among ties */
}

/* Decision that a log entry implies for round r: ACTIVE, ELIMINATED or
 * ACCEPTED, or -1 when the entry says the pair was already gone. */
static int logged_decision(int32_t code, int32_t r) {
    int32_t rc = code >> 2, kind = code & 3;
    if (rc > r) return ORC_ACTIVE;
    if (rc == r) return kind;
    return -1;
}

static int64_t round_samples(const orc_adaptive_params* p, int32_t r, int64_t Tcur) {
    if (r == 0) return p->B0;
    if (p->grow) return Tcur > p->B ? Tcur : p->B;
    return p->B;
}

/* One query. X is the FP32 data (it fixes the span), G the values the
 * samples are read from (X itself, or its dequantised BF16/FP8 copy whose
 * elements differ from X by at most emax). */
static int32_t adaptive_core(const float* X, const float* G, double emax, int64_t n, int32_t m, const float* q,
                             const orc_adaptive_params* p, const int32_t* replay,
                             int64_t* out_idx, int32_t* code, double* S, int32_t* T,
                             orc_adaptive_stats* st) {
    const int32_t k = p->k, h = p->h;
    const int64_t kh = (int64_t)k + h;
    if (k < 1 || h < 0 || n < k || m < 1 || !(p->delta > 0.0 && p->delta < 1.0) || p->B0 < 1 || p->B < 1 ||
        p->block < 0 || (p->sampling != ORC_SAMPLE_WITH && p->sampling != ORC_SAMPLE_WITHOUT) ||
        (p->sampling == ORC_SAMPLE_WITHOUT && p->block > 1))
        return 1;
    /* g coordinates per sample, M samples make the exact distance */
    const int32_t g = p->block > 1 ? p->block : 1;
    const int32_t M = (int32_t)(((int64_t)m + g - 1) / g);
    memset(st, 0, sizeof(*st));
    for (int64_t t = 0; t < kh; ++t) out_idx[t] = -1;

    if (n <= kh) { /* every point is a candidate: nothing to estimate */
        for (int64_t i = 0; i < n; ++i) {
            out_idx[i] = i;
            if (code) code[i] = ORC_ACTIVE;
            if (S) S[i] = 0.0;
            if (T) T[i] = 0;
        }
        st->count = (int32_t)n;
        st->term = 0;
        return 0;
    }

    /* Affine normalisation of Section 3 (||x||_inf <= 1/2): with
     * span = max - min over the data and the query, every sample
     * (x_ij - x_j)^2 / span^2 lies in [0, 1]; bounds are used in raw units
     * scaled by span^2. */
    double lo = q[0], hi = q[0];
    for (int32_t j = 0; j < m; ++j) {
        if (q[j] < lo) lo = q[j];
        if (q[j] > hi) hi = q[j];
    }
    for (size_t e = 0; e < (size_t)n * (size_t)m; ++e) {
        if (X[e] < lo) lo = X[e];
        if (X[e] > hi) hi = X[e];
    }
    const double span = hi - lo;
    /* A stored copy moves each sample by at most
     * |xt - x| |xt + x - 2q| <= emax (2 span + emax), so its distances lie
     * within eps of the true ones, and its samples within [0, (span + 2 emax)^2]:
     * the width of the sampled bounds grows accordingly. The exact cap reads
     * the FP32 data, so exact distances keep width 0.
     * For l1 a sample |x - q| lies in [0, span] (normalised by span, not
     * span^2), and a copy moves it by at most emax, within [0, span + emax].
     * (eps is the round-0 copy term; later rounds may use a smaller one.) */
    const int32_t metric = p->metric;
    const double spanw = metric == ORC_METRIC_L1 ? span + emax : span + 2.0 * emax;
    const double span2 = metric == ORC_METRIC_L1 ? spanw : spanw * spanw;
    const double eps = metric == ORC_METRIC_L1 ? emax : emax * (2.0 * span + emax);

    unsigned char* status = (unsigned char*)malloc((size_t)n);
    double* Sx = (double*)malloc(sizeof(double) * (size_t)n);
    int32_t* Tx = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    int32_t* cx = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    double* dh = (double*)malloc(sizeof(double) * (size_t)n); /* frozen estimate */
    double* ub = (double*)malloc(sizeof(double) * (size_t)n); /* frozen UCB */
    double* lb = (double*)malloc(sizeof(double) * (size_t)n); /* frozen LCB */
    double* wd = (double*)malloc(sizeof(double) * (size_t)n); /* frozen width */
    unsigned char* newst = (unsigned char*)malloc((size_t)n);
    vm_t* su = (vm_t*)malloc(sizeof(vm_t) * (size_t)n);
    vm_t* sl = (vm_t*)malloc(sizeof(vm_t) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) { status[i] = ORC_ACTIVE; Sx[i] = 0.0; Tx[i] = 0; cx[i] = 0; }

    int64_t nact = n, nacc = 0, evals = 0;
    double min_elim = INFINITY, min_elim_mag = 0.0;
    int64_t Tcur = 0;
    int32_t r = 0, term = 0;
    for (;;) {
        int64_t Br = round_samples(p, r, Tcur);
        int exact = (Tcur + Br >= M);
        int64_t Tn = exact ? M : Tcur + Br;
        /* Sample step (Algorithm 1 update, batched): every active point
         * gets draws Tcur .. Tn-1, or its exact distance when the count
         * would reach M (Algorithm 1 computes the distance exactly once all
         * m coordinates would be sampled; M = m for single coordinates). */
        for (int64_t i = 0; i < n; ++i) {
            if (status[i] != ORC_ACTIVE) continue;
            const float* xi = G + (size_t)i * (size_t)m;
            if (exact) { /* the exact distance is taken on the FP32 data itself */
                Sx[i] = dist_of(metric, X + (size_t)i * (size_t)m, q, m);
            } else {
                for (int64_t t = Tcur; t < Tn; ++t) {
                    /* draw t picks block b: coordinates b*g .. min(b*g + g, m) - 1
                     * (without replacement g = 1 and b is the pair's t-th
                     * coordinate of its permutation) */
                    int32_t b = p->sampling == ORC_SAMPLE_WITHOUT
                                    ? orc_coordinate_wor(p->seed, p->qid, (uint64_t)i, (uint64_t)t, m, p->mask_p,
                                                         p->mask_q)
                                    : orc_coordinate(p->seed, p->qid, (uint64_t)i, (uint64_t)t, M, p->mask_p, p->mask_q);
                    int32_t j1 = (b + 1) * g < m ? (b + 1) * g : m;
                    for (int32_t j = b * g; j < j1; ++j) Sx[i] += term_of(metric, (double)xi[j] - (double)q[j]);
                }
            }
            Tx[i] = (int32_t)Tn;
        }
        evals += nact * (exact ? (int64_t)m : Br * g);
        /* estimate: mean per coordinate of the sampled blocks (S / (T g)) */
        const double Tg = (double)Tn * (double)g;
        /* A copy's sample differs from the data's by at most e (2 |xt - q| + e),
         * so its mean over the sampled coordinates by at most e (2 mean|xt - q|
         * + e) <= e (2 sqrt(d_i) + e), d_i the copy's estimate (the mean of
         * |z| is at most the square root of the mean of z^2). In every round
         * the width takes the largest estimate among the points it decides,
         * when that is below the span form. */
        double eps_r = eps;
        if (!exact && emax > 0.0 && metric != ORC_METRIC_L1) {
            double dmax = 0.0;
            for (int64_t i = 0; i < n; ++i)
                if (status[i] == ORC_ACTIVE && Sx[i] / Tg > dmax) dmax = Sx[i] / Tg;
            const double e2 = emax * (2.0 * sqrt(dmax) + emax);
            if (e2 < eps_r) eps_r = e2;
        }
        const double w = exact ? 0.0 : span2 * orc_alpha(p->bound, p->c_alpha, Tn, n, p->delta) + eps_r;

        /* Bounds of the non-eliminated points: current ones for active
         * points, frozen ones for accepted points. */
        int64_t cnt = 0;
        for (int64_t i = 0; i < n; ++i) {
            if (status[i] == ORC_ACTIVE) {
                double d = Sx[i] / Tg;
                su[cnt].v = d + w; su[cnt].mag = d + w;
                sl[cnt].v = d - w; sl[cnt].mag = d + w;
                ++cnt;
            } else if (status[i] == ORC_ACCEPTED) {
                su[cnt].v = ub[i]; su[cnt].mag = dh[i] + wd[i];
                sl[cnt].v = lb[i]; sl[cnt].mag = dh[i] + wd[i];
                ++cnt;
            }
        }
        qsort(su, (size_t)cnt, sizeof(vm_t), cmp_vm);
        qsort(sl, (size_t)cnt, sizeof(vm_t), cmp_vm);
        /* tau_U: k-th smallest UCB (the batched q1 of Eq. d_ind);
         * tau_L: (k+1)-th smallest LCB, or a smaller frozen LCB of an
         * eliminated point (the batched q2). */
        const double tauU = su[k - 1].v, tauU_mag = su[k - 1].mag;
        double tauL = sl[k].v, tauL_mag = sl[k].mag;
        if (min_elim < tauL) { tauL = min_elim; tauL_mag = min_elim_mag; }

        /* Decide: a point whose LCB exceeds tau_U has k points certainly
         * closer, so it is not among the k nearest; a point whose UCB is
         * below tau_L is closer than n-k points, so it is among them. */
        double round_min = INFINITY, round_min_mag = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            newst[i] = status[i];
            if (status[i] != ORC_ACTIVE) continue;
            double d = Sx[i] / Tg;
            double U = d + w, L = d - w, mag = d + w;
            int o = (L > tauU) ? ORC_ELIMINATED : ((U < tauL) ? ORC_ACCEPTED : ORC_ACTIVE);
            if (replay) {
                int nearU = fabs(L - tauU) <= p->tol * (mag + tauU_mag);
                int nearL = fabs(U - tauL) <= p->tol * (mag + tauL_mag);
                int nr = nearU || nearL;
                if (nr) st->near++;
                int g = logged_decision(replay[i], r);
                if (g < 0) {
                    st->log_inconsistent++;
                } else if (g != o) {
                    if (nr) st->near_disagree++; else st->mismatch++;
                    o = g;
                }
            }
            if (o == ORC_ELIMINATED) {
                newst[i] = ORC_ELIMINATED;
                cx[i] = 4 * r + ORC_ELIMINATED;
                dh[i] = d; lb[i] = L; ub[i] = U; wd[i] = w;
                if (L < round_min) { round_min = L; round_min_mag = mag; }
            } else if (o == ORC_ACCEPTED) {
                newst[i] = ORC_ACCEPTED;
                cx[i] = 4 * r + ORC_ACCEPTED;
                dh[i] = d; lb[i] = L; ub[i] = U; wd[i] = w;
            }
        }
        for (int64_t i = 0; i < n; ++i) {
            if (status[i] == ORC_ACTIVE && newst[i] != ORC_ACTIVE) {
                --nact;
                if (newst[i] == ORC_ACCEPTED) ++nacc;
            }
            status[i] = newst[i];
        }
        if (round_min < min_elim) { min_elim = round_min; min_elim_mag = round_min_mag; }
        Tcur = Tn;
        /* Termination (batched form of Eq. termination). */
        if (nact + nacc <= kh) term = 1;
        else if (nacc >= k) term = 2;
        else if (exact) term = 3;
        if (term) break;
        ++r;
    }
    for (int64_t i = 0; i < n; ++i)
        if (status[i] == ORC_ACTIVE) { cx[i] = 4 * r + ORC_ACTIVE; dh[i] = Sx[i] / ((double)Tx[i] * g); }
    if (replay)
        for (int64_t i = 0; i < n; ++i)
            if ((replay[i] >> 2) > r || ((replay[i] & 3) == ORC_ACTIVE && (replay[i] >> 2) != r))
                st->log_inconsistent++;

    /* Output: accepted points by (estimate, index), then active points by
     * (estimate, index), at most k+h (the set S-hat of Algorithm 1). */
    vi_t* acc = (vi_t*)malloc(sizeof(vi_t) * (size_t)(nacc > 0 ? nacc : 1));
    vi_t* act = (vi_t*)malloc(sizeof(vi_t) * (size_t)(nact > 0 ? nact : 1));
    int64_t na = 0, nb = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (status[i] == ORC_ACCEPTED) { acc[na].v = dh[i]; acc[na].i = i; ++na; }
        else if (status[i] == ORC_ACTIVE) { act[nb].v = dh[i]; act[nb].i = i; ++nb; }
    }
    qsort(acc, (size_t)na, sizeof(vi_t), cmp_vi);
    qsort(act, (size_t)nb, sizeof(vi_t), cmp_vi);
    int64_t c = 0;
    for (int64_t t = 0; t < na && c < kh; ++t) out_idx[c++] = acc[t].i;
    for (int64_t t = 0; t < nb && c < kh; ++t) out_idx[c++] = act[t].i;

    st->evals = evals;
    st->rounds = r + 1;
    st->count = (int32_t)c;
    st->term = term;
    if (code) memcpy(code, cx, sizeof(int32_t) * (size_t)n);
    if (S) memcpy(S, Sx, sizeof(double) * (size_t)n);
    if (T) memcpy(T, Tx, sizeof(int32_t) * (size_t)n);
    free(acc); free(act);
    free(status); free(Sx); free(Tx); free(cx); free(dh); free(ub); free(lb); free(wd);
    free(newst); free(su); free(sl);
    return 0;
}

int32_t orc_adaptive(const float* X, int64_t n, int32_t m, const float* q,
                     const orc_adaptive_params* p, const int32_t* replay,
                     int64_t* out_idx, int32_t* code, double* S, int32_t* T,
                     orc_adaptive_stats* st) {
    if (p->storage == ORC_STORE_F32)
        return adaptive_core(X, X, 0.0, n, m, q, p, replay, out_idx, code, S, T, st);
    float* G = (float*)malloc(sizeof(float) * (size_t)n * (size_t)m);
    double emax = orc_quantize(p->storage, X, n, m, G, NULL);
    int32_t rc = adaptive_core(X, G, emax, n, m, q, p, replay, out_idx, code, S, T, st);
    free(G);
    return rc;
}

int32_t orc_adaptive_batch(const float* X, int64_t n, int32_t m, const float* Q, int32_t nq,
                           const orc_adaptive_params* p, const int32_t* replay,
                           int64_t* out_idx, int32_t* codes, double* S, int32_t* T,
                           orc_adaptive_stats* st, int32_t threads) {
    const int64_t kh = (int64_t)p->k + p->h;
    const float* G = X;
    float* Gq = NULL;
    double emax = 0.0;
    if (p->storage != ORC_STORE_F32) {
        Gq = (float*)malloc(sizeof(float) * (size_t)n * (size_t)m);
        emax = orc_quantize(p->storage, X, n, m, Gq, NULL);
        G = Gq;
    }
    int32_t bad = 0;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(dynamic, 1) reduction(|: bad)
#endif
    for (int32_t qi = 0; qi < nq; ++qi) {
        orc_adaptive_params pq = *p;
        pq.qid = p->qid + (uint64_t)qi;
        size_t off = (size_t)qi * (size_t)n;
        bad |= adaptive_core(X, G, emax, n, m, Q + (size_t)qi * (size_t)m, &pq,
                             replay ? replay + off : NULL, out_idx + (size_t)qi * (size_t)kh,
                             codes ? codes + off : NULL, S ? S + off : NULL, T ? T + off : NULL, st + qi);
    }
    free(Gq);
    return bad;
}

/* ---------------------------------------------------- Algorithm 1 as printed */

int32_t orc_sequential(const float* X, int64_t n, int32_t m, const float* q,
                       const orc_adaptive_params* p, int64_t max_iter,
                       int64_t* out_idx, int64_t* out_evals, int64_t* out_iters) {
    const int32_t k = p->k, h = p->h;
    const int64_t kh = (int64_t)k + h;
    if (k < 1 || h < 0 || n < k || m < 1 || !(p->delta > 0.0 && p->delta < 1.0)) return 1;
    for (int64_t t = 0; t < kh; ++t) out_idx[t] = -1;
    *out_evals = 0;
    *out_iters = 0;
    if (n <= kh) {
        for (int64_t i = 0; i < n; ++i) out_idx[i] = i;
        return 0;
    }
    double lo = q[0], hi = q[0];
    for (int32_t j = 0; j < m; ++j) { if (q[j] < lo) lo = q[j]; if (q[j] > hi) hi = q[j]; }
    for (size_t e = 0; e < (size_t)n * (size_t)m; ++e) { if (X[e] < lo) lo = X[e]; if (X[e] > hi) hi = X[e]; }
    const double span2 = (hi - lo) * (hi - lo);

    double* sum = (double*)malloc(sizeof(double) * (size_t)n);
    double* est = (double*)malloc(sizeof(double) * (size_t)n);
    double* al = (double*)malloc(sizeof(double) * (size_t)n);
    int64_t* Tn = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    int64_t* perm = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    int64_t evals = 0;

    /* Initialisation: one sample per point. */
    for (int64_t i = 0; i < n; ++i) {
        const float* xi = X + (size_t)i * (size_t)m;
        if (m == 1) { /* one sample is the whole distance */
            sum[i] = sqdist(xi, q, m); Tn[i] = 1; est[i] = sum[i]; al[i] = 0.0; evals += 1;
        } else {
            int32_t j = orc_coordinate(p->seed, p->qid, (uint64_t)i, 0, m, p->mask_p, p->mask_q);
            double d = (double)xi[j] - (double)q[j];
            sum[i] = d * d; Tn[i] = 1; est[i] = sum[i];
            al[i] = span2 * orc_alpha(p->bound, p->c_alpha, 1, n, p->delta);
            evals += 1;
        }
        perm[i] = i;
    }
    /* Sort the permutation by (estimate, index); insertion sort keeps it
     * ordered cheaply as only two estimates change per iteration. */
    for (int64_t a = 1; a < n; ++a) {
        int64_t v = perm[a], b = a - 1;
        while (b >= 0 && (est[perm[b]] > est[v] || (est[perm[b]] == est[v] && perm[b] > v))) {
            perm[b + 1] = perm[b]; --b;
        }
        perm[b + 1] = v;
    }
    int64_t it = 0;
    for (; it < max_iter; ++it) {
        /* q1: largest UCB among the k smallest estimates. */
        int64_t q1 = perm[0];
        for (int64_t a = 0; a < k; ++a) {
            int64_t i = perm[a];
            if (est[i] + al[i] > est[q1] + al[q1]) q1 = i;
        }
        /* q2: smallest LCB among ranks k+h+1 .. n. */
        int64_t q2 = perm[kh];
        for (int64_t a = kh; a < n; ++a) {
            int64_t i = perm[a];
            if (est[i] - al[i] < est[q2] - al[q2]) q2 = i;
        }
        if (est[q1] + al[q1] <= est[q2] - al[q2]) break; /* Eq. termination */
        /* b2: largest width among q2 and the middle ranks k+1 .. k+h (Eq. blowbupdef). */
        int64_t b2 = q2;
        for (int64_t a = k; a < kh; ++a) {
            int64_t i = perm[a];
            if (al[i] > al[b2]) b2 = i;
        }
        int64_t upd[2] = {q1, b2};
        for (int u = 0; u < 2; ++u) {
            int64_t l = upd[u];
            if (Tn[l] >= m) continue; /* already exact */
            const float* xl = X + (size_t)l * (size_t)m;
            int32_t j = orc_coordinate(p->seed, p->qid, (uint64_t)l, (uint64_t)Tn[l], m, p->mask_p, p->mask_q);
            double d = (double)xl[j] - (double)q[j];
            sum[l] += d * d;
            Tn[l] += 1;
            evals += 1;
            if (Tn[l] == m) {
                est[l] = sqdist(xl, q, m) / (double)m;
                al[l] = 0.0;
                evals += m;
            } else {
                est[l] = sum[l] / (double)Tn[l];
                al[l] = span2 * orc_alpha(p->bound, p->c_alpha, Tn[l], n, p->delta);
            }
        }
        /* Restore the order (insertion sort on a nearly sorted array). */
        for (int64_t a = 1; a < n; ++a) {
            int64_t v = perm[a], b = a - 1;
            while (b >= 0 && (est[perm[b]] > est[v] || (est[perm[b]] == est[v] && perm[b] > v))) {
                perm[b + 1] = perm[b]; --b;
            }
            perm[b + 1] = v;
        }
    }
    for (int64_t t = 0; t < kh; ++t) out_idx[t] = perm[t];
    *out_evals = evals;
    *out_iters = it;
    free(sum); free(est); free(al); free(Tn); free(perm);
    return it >= max_iter ? 2 : 0;
}

/* ----------------------------------------- Algorithm 1 with the seven heaps */

/* The same algorithm as orc_sequential, with the data structures of Section
 * 4.1 (Figure "heaps"): the points are split by their rank in the (estimate,
 * index) order into the close set (ranks 1..k), the middle set (k+1..k+h)
 * and the far set (the rest). Close keeps a max-heap on the estimate and a
 * max-heap on the UCB (q1 is its top); middle a min- and a max-heap on the
 * estimate and a max-heap on the width (candidates for b2); far a min-heap
 * on the estimate and a min-heap on the LCB (q2 is its top). An iteration
 * costs O(log n): the two updated points leave their heaps, are re-inserted,
 * and the sets are repaired by swapping boundary elements. Ties follow the
 * rank order, as in the scan version. */

enum { HC_EST = 0, HC_UCB, HM_EMIN, HM_EMAX, HM_AL, HF_EST, HF_LCB, NHEAP };

typedef struct {
    const double* est;
    const double* al;
    int64_t* a[NHEAP];
    int64_t* pos[NHEAP];
    int64_t size[NHEAP];
} heaps_t;

static int rank_lt(const heaps_t* H, int64_t i, int64_t j) {
    return H->est[i] < H->est[j] || (H->est[i] == H->est[j] && i < j);
}

/* 1 if i belongs above j in heap t */
static int heap_before(const heaps_t* H, int t, int64_t i, int64_t j) {
    const double* e = H->est;
    const double* a = H->al;
    switch (t) {
    case HC_EST: case HM_EMAX: return rank_lt(H, j, i);
    case HM_EMIN: case HF_EST: return rank_lt(H, i, j);
    case HC_UCB: {
        double ui = e[i] + a[i], uj = e[j] + a[j];
        return ui > uj || (ui == uj && rank_lt(H, i, j));
    }
    case HM_AL: return a[i] > a[j] || (a[i] == a[j] && rank_lt(H, i, j));
    default: { /* HF_LCB */
        double li = e[i] - a[i], lj = e[j] - a[j];
        return li < lj || (li == lj && rank_lt(H, i, j));
    }
    }
}

static void heap_swap(heaps_t* H, int t, int64_t x, int64_t y) {
    int64_t* a = H->a[t];
    int64_t v = a[x];
    a[x] = a[y]; a[y] = v;
    H->pos[t][a[x]] = x;
    H->pos[t][a[y]] = y;
}

static void heap_sift(heaps_t* H, int t, int64_t x) {
    int64_t* a = H->a[t];
    while (x > 0 && heap_before(H, t, a[x], a[(x - 1) / 2])) {
        heap_swap(H, t, x, (x - 1) / 2);
        x = (x - 1) / 2;
    }
    for (;;) {
        int64_t l = 2 * x + 1, r = l + 1, b = x;
        if (l < H->size[t] && heap_before(H, t, a[l], a[b])) b = l;
        if (r < H->size[t] && heap_before(H, t, a[r], a[b])) b = r;
        if (b == x) break;
        heap_swap(H, t, x, b);
        x = b;
    }
}

static void heap_push(heaps_t* H, int t, int64_t i) {
    int64_t x = H->size[t]++;
    H->a[t][x] = i;
    H->pos[t][i] = x;
    heap_sift(H, t, x);
}

static void heap_remove(heaps_t* H, int t, int64_t i) {
    int64_t x = H->pos[t][i], last = --H->size[t];
    if (x != last) {
        heap_swap(H, t, x, last);
        H->pos[t][i] = -1;
        heap_sift(H, t, x);
    } else {
        H->pos[t][i] = -1;
    }
}

static const int set_heaps[3][3] = {{HC_EST, HC_UCB, -1}, {HM_EMIN, HM_EMAX, HM_AL}, {HF_EST, HF_LCB, -1}};

static void set_insert(heaps_t* H, unsigned char* set, int s, int64_t i) {
    set[i] = (unsigned char)s;
    for (int u = 0; u < 3; ++u)
        if (set_heaps[s][u] >= 0) heap_push(H, set_heaps[s][u], i);
}

static void set_remove(heaps_t* H, const unsigned char* set, int64_t i) {
    for (int u = 0; u < 3; ++u)
        if (set_heaps[set[i]][u] >= 0) heap_remove(H, set_heaps[set[i]][u], i);
}

/* Restores close < middle < far in the (estimate, index) order by swapping
 * the offending boundary elements. */
static void sets_repair(heaps_t* H, unsigned char* set, int32_t h) {
    for (;;) {
        int changed = 0;
        if (h > 0) {
            int64_t c = H->a[HC_EST][0], mm = H->a[HM_EMIN][0];
            if (rank_lt(H, mm, c)) {
                set_remove(H, set, c); set_remove(H, set, mm);
                set_insert(H, set, 1, c); set_insert(H, set, 0, mm);
                changed = 1;
            }
            int64_t mx = H->a[HM_EMAX][0], f = H->a[HF_EST][0];
            if (rank_lt(H, f, mx)) {
                set_remove(H, set, mx); set_remove(H, set, f);
                set_insert(H, set, 2, mx); set_insert(H, set, 1, f);
                changed = 1;
            }
        } else {
            int64_t c = H->a[HC_EST][0], f = H->a[HF_EST][0];
            if (rank_lt(H, f, c)) {
                set_remove(H, set, c); set_remove(H, set, f);
                set_insert(H, set, 2, c); set_insert(H, set, 0, f);
                changed = 1;
            }
        }
        if (!changed) break;
    }
}

static int cmp_rank_pair(const void* x, const void* y) {
    const vi_t* a = (const vi_t*)x;
    const vi_t* b = (const vi_t*)y;
    if (a->v < b->v) return -1;
    if (a->v > b->v) return 1;
    return (a->i > b->i) - (a->i < b->i);
}

int32_t orc_sequential_heaps(const float* X, int64_t n, int32_t m, const float* q,
                             const orc_adaptive_params* p, int64_t max_iter,
                             int64_t* out_idx, int64_t* out_evals, int64_t* out_iters) {
    const int32_t k = p->k, h = p->h;
    const int64_t kh = (int64_t)k + h;
    if (k < 1 || h < 0 || n < k || m < 1 || !(p->delta > 0.0 && p->delta < 1.0)) return 1;
    for (int64_t t = 0; t < kh; ++t) out_idx[t] = -1;
    *out_evals = 0;
    *out_iters = 0;
    if (n <= kh) {
        for (int64_t i = 0; i < n; ++i) out_idx[i] = i;
        return 0;
    }
    double lo = q[0], hi = q[0];
    for (int32_t j = 0; j < m; ++j) { if (q[j] < lo) lo = q[j]; if (q[j] > hi) hi = q[j]; }
    for (size_t e = 0; e < (size_t)n * (size_t)m; ++e) { if (X[e] < lo) lo = X[e]; if (X[e] > hi) hi = X[e]; }
    const double span2 = (hi - lo) * (hi - lo);

    double* sum = (double*)malloc(sizeof(double) * (size_t)n);
    double* est = (double*)malloc(sizeof(double) * (size_t)n);
    double* al = (double*)malloc(sizeof(double) * (size_t)n);
    int64_t* Tn = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    unsigned char* set = (unsigned char*)malloc((size_t)n);
    vi_t* order = (vi_t*)malloc(sizeof(vi_t) * (size_t)n);
    heaps_t H;
    H.est = est;
    H.al = al;
    for (int t = 0; t < NHEAP; ++t) {
        H.a[t] = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
        H.pos[t] = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
        H.size[t] = 0;
        for (int64_t i = 0; i < n; ++i) H.pos[t][i] = -1;
    }
    int64_t evals = 0;
    /* Initialisation: one sample per point (as the scan version). */
    for (int64_t i = 0; i < n; ++i) {
        const float* xi = X + (size_t)i * (size_t)m;
        if (m == 1) {
            sum[i] = sqdist(xi, q, m); Tn[i] = 1; est[i] = sum[i]; al[i] = 0.0; evals += 1;
        } else {
            int32_t j = orc_coordinate(p->seed, p->qid, (uint64_t)i, 0, m, p->mask_p, p->mask_q);
            double d = (double)xi[j] - (double)q[j];
            sum[i] = d * d; Tn[i] = 1; est[i] = sum[i];
            al[i] = span2 * orc_alpha(p->bound, p->c_alpha, 1, n, p->delta);
            evals += 1;
        }
        order[i].v = est[i];
        order[i].i = i;
    }
    qsort(order, (size_t)n, sizeof(vi_t), cmp_rank_pair);
    for (int64_t r = 0; r < n; ++r) set_insert(&H, set, r < k ? 0 : (r < kh ? 1 : 2), order[r].i);
    int64_t it = 0;
    for (; it < max_iter; ++it) {
        const int64_t q1 = H.a[HC_UCB][0], q2 = H.a[HF_LCB][0];
        if (est[q1] + al[q1] <= est[q2] - al[q2]) break; /* Eq. termination */
        int64_t b2 = q2;
        if (h > 0) {
            const int64_t c = H.a[HM_AL][0];
            if (al[c] > al[q2]) b2 = c;
        }
        const int64_t upd[2] = {q1, b2};
        for (int u = 0; u < 2; ++u) {
            const int64_t l = upd[u];
            if (Tn[l] >= m) continue;
            const int s = set[l];
            set_remove(&H, set, l);
            const float* xl = X + (size_t)l * (size_t)m;
            int32_t j = orc_coordinate(p->seed, p->qid, (uint64_t)l, (uint64_t)Tn[l], m, p->mask_p, p->mask_q);
            double d = (double)xl[j] - (double)q[j];
            sum[l] += d * d;
            Tn[l] += 1;
            evals += 1;
            if (Tn[l] == m) {
                est[l] = sqdist(xl, q, m) / (double)m;
                al[l] = 0.0;
                evals += m;
            } else {
                est[l] = sum[l] / (double)Tn[l];
                al[l] = span2 * orc_alpha(p->bound, p->c_alpha, Tn[l], n, p->delta);
            }
            set_insert(&H, set, s, l);
        }
        sets_repair(&H, set, h);
    }
    int64_t cnt = 0;
    for (int64_t i = 0; i < n; ++i)
        if (set[i] != 2) { order[cnt].v = est[i]; order[cnt].i = i; ++cnt; }
    qsort(order, (size_t)cnt, sizeof(vi_t), cmp_rank_pair);
    for (int64_t t = 0; t < cnt && t < kh; ++t) out_idx[t] = order[t].i;
    *out_evals = evals;
    *out_iters = it;
    for (int t = 0; t < NHEAP; ++t) { free(H.a[t]); free(H.pos[t]); }
    free(sum); free(est); free(al); free(Tn); free(set); free(order);
    return it >= max_iter ? 2 : 0;
}
