/*
 * knn_oracle.h -- plain CPU oracle for the adaptive k-NN method of
 * LeJeune, Baraniuk and Heckel, "Adaptive Estimation for Approximate
 * k-Nearest-Neighbor Computations" (AISTATS 2019).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path links, loads or calls
 * this code: only the tests, the package's smoke check and the CPU-baseline leg
 * of the benchmark do. It shares no source with the CUDA library.
 *
 * All arithmetic is double precision; inputs are float32 arrays read as-is.
 */
#ifndef KNN_ORACLE_H
#define KNN_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Confidence-bound forms (Section 4): footnote form, Lemma form, and the
 * experiment form of Section 5 with a free constant C_alpha. */
enum { ORC_BOUND_FOOTNOTE = 0, ORC_BOUND_LEMMA = 1, ORC_BOUND_EXP = 2 };

/* Per-point decision kinds written to the decision codes (code = 4*round + kind). */
enum { ORC_ACTIVE = 0, ORC_ELIMINATED = 1, ORC_ACCEPTED = 2 };

/* Philox4x32 with 10 rounds (Salmon et al., SC'11): out = philox(ctr, key). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Index in [0, m) of the s-th coordinate drawn (0-based) for point `point` of
 * query `qid`. Uniform with replacement (Section 4, sampled estimator): word
 * s mod 4 of Philox4x32-10 at counter (s / 4, point & mask_p, low and high
 * words of qid & mask_q), key (low and high words of seed), scaled to [0, m)
 * by floor(word * m / 2^32). */
int32_t orc_coordinate(uint64_t seed, uint64_t qid, uint64_t point, uint64_t s, int32_t m,
                       uint64_t mask_p, uint64_t mask_q);

/* Without replacement (footnote to Section 4: a cipher on [m] makes the
 * estimate exact after m draws). The s-th draw (0-based, s < m) of a pair is
 * pi(s), pi a permutation of [0, m) keyed per (seed, point, query):
 *   round keys k_0..k_7 = the words of blocks 2^32 - 2 and 2^32 - 1 of the
 *   pair's Philox4x32-10 stream (counter and key as for orc_coordinate, in
 *   that order); a balanced Feistel network (Luby and Rackoff) of 8 rounds
 *   on 2h bits (4 rounds leave consecutive draws visibly correlated on
 *   small domains),
 *   h = max(1, ceil(ceil(log2 m) / 2)): with x = (L, R), L the high h bits,
 *   a round maps (L, R) to (R, L xor (F(k_r, R) mod 2^h)), where
 *   F(k, R) = fmix32(R xor k), fmix32 the 32-bit finaliser of MurmurHash3;
 *   extended to [0, m) by cycle walking (Black and Rogaway): the network is
 *   applied again until the value is below m. */
int32_t orc_coordinate_wor(uint64_t seed, uint64_t qid, uint64_t point, uint64_t s, int32_t m,
                           uint64_t mask_p, uint64_t mask_q);

/* alpha(u) in normalised units ([0,1]-bounded samples). */
double orc_alpha(int32_t form, double c_alpha, int64_t u, int64_t n, double delta);

/* Brute force (Section 3): the k nearest points of q by squared l2 distance,
 * ties broken by the smaller index. idx[k], dist[k] (squared distances). */
void orc_exact_knn(const float* X, int64_t n, int32_t m, const float* q, int32_t k,
                   int64_t* idx, double* dist);
/* The same under a metric (ORC_METRIC_*); dist holds that metric's values. */
void orc_exact_knn_metric(const float* X, int64_t n, int32_t m, const float* q, int32_t k, int32_t metric,
                          int64_t* idx, double* dist);

typedef struct {
    int32_t k, h;
    int32_t bound;        /* ORC_BOUND_* */
    double c_alpha;       /* EXP form only */
    double delta;
    int32_t B0, B, grow;  /* round schedule: B_0 = B0; later B_r = B, or max(B, T) if grow */
    uint64_t seed, qid, mask_p, mask_q;
    double tol;           /* relative width of the near-threshold band used in replay */
    int32_t storage;      /* ORC_STORE_*: the values the samples are taken from */
    int32_t block;        /* coordinates per sample: 0 or 1 is the paper's one coordinate; g > 1 draws
                           * one of ceil(m/g) blocks of g consecutive coordinates (the last may be
                           * shorter) and adds the block's sum of squared differences */
    int32_t metric;       /* ORC_METRIC_*: squared l2 (the paper's), or l1 (Section 3's generalisation):
                           * samples |x_j - q_j|, normalised by span instead of span^2 */
    int32_t sampling;     /* ORC_SAMPLE_*: with replacement (Section 4), or without (single coordinates:
                           * a pair's draws follow orc_coordinate_wor's permutation) */
} orc_adaptive_params;

enum { ORC_SAMPLE_WITH = 0, ORC_SAMPLE_WITHOUT = 1 };

enum { ORC_METRIC_L2SQ = 0, ORC_METRIC_L1 = 1 };

/* Storage of the gathered copy: FP32 itself, BF16 (round to nearest even),
 * or FP8 e4m3 with a per-row scale max|x_i| / 448. */
enum { ORC_STORE_F32 = 0, ORC_STORE_BF16 = 1, ORC_STORE_FP8 = 2 };

/* Dequantised copies: out = bf16(x) as float; or, per row, s = max|x|/448
 * (1 if the row is zero) and out = fl32(s * e4m3(fl32(x / s))). Returns the
 * largest |out - x| (exact). scale may be NULL. */
double orc_quantize(int32_t storage, const float* X, int64_t n, int32_t m, float* out, float* scale);
float orc_round_bf16(float x);
float orc_round_e4m3(float x);

typedef struct {
    int64_t evals;        /* coordinate evaluations: samples drawn x block + m per exact distance */
    int32_t rounds;
    int32_t count;        /* candidates returned (<= k+h) */
    int32_t term;         /* 1: size <= k+h; 2: >= k accepted; 3: exact round; 0: n <= k+h */
    int64_t near;         /* decisions whose test lies in the near-threshold band */
    int64_t near_disagree;/* of those, decisions where the replayed log differs */
    int64_t mismatch;     /* decisions outside the band where the replayed log differs */
    int64_t log_inconsistent; /* log entries that cannot be reached (wrong round) */
} orc_adaptive_stats;

/* Batched adaptive rounds for one query (hot-path rules, see knn_oracle.c).
 * Outputs: out_idx[k+h] (-1 padded), code[n] (4*round + kind), S[n] (sum of
 * sampled squared differences, or the exact squared distance), T[n] (samples;
 * blocks with block > 1, ceil(m/block) once exact).
 * If `replay` is non-NULL it holds another implementation's codes for the
 * same query; the oracle then adopts that decision wherever the two disagree
 * and counts the disagreement as near-band or mismatch. */
int32_t orc_adaptive(const float* X, int64_t n, int32_t m, const float* q,
                     const orc_adaptive_params* p, const int32_t* replay,
                     int64_t* out_idx, int32_t* code, double* S, int32_t* T,
                     orc_adaptive_stats* st);

/* Many queries, OpenMP over queries. q is nq x m; out_idx nq x (k+h);
 * codes/S/T may be NULL (else nq x n). qid of query i is p->qid + i. */
int32_t orc_adaptive_batch(const float* X, int64_t n, int32_t m, const float* Q, int32_t nq,
                           const orc_adaptive_params* p, const int32_t* replay,
                           int64_t* out_idx, int32_t* codes, double* S, int32_t* T,
                           orc_adaptive_stats* st, int32_t threads);

/* Algorithm 1 as printed (two arms per iteration, LUCB indices q1, b2),
 * with O(n) scans in place of the seven heaps. out_idx[k+h]. Pinned at its
 * two closed-form limits (wide bounds: every distance exact; vanishing
 * bounds: no iteration) and by Theorem 1's containment; the iteration
 * counts in between are fixed by nothing in the paper (parity unpinned
 * there). */
int32_t orc_sequential(const float* X, int64_t n, int32_t m, const float* q,
                       const orc_adaptive_params* p, int64_t max_iter,
                       int64_t* out_idx, int64_t* out_evals, int64_t* out_iters);

/* Algorithm 1 with the seven heaps of Section 4.1 (Figure "heaps"): the same
 * iterations, samples and output as orc_sequential, O(log n) per iteration. */
int32_t orc_sequential_heaps(const float* X, int64_t n, int32_t m, const float* q,
                             const orc_adaptive_params* p, int64_t max_iter,
                             int64_t* out_idx, int64_t* out_evals, int64_t* out_iters);

/* Brute force for many queries (OpenMP). idx/dist are nq x k. */
void orc_exact_knn_batch(const float* X, int64_t n, int32_t m, const float* Q, int32_t nq,
                         int32_t k, int64_t* idx, double* dist, int32_t threads);
void orc_exact_knn_batch_metric(const float* X, int64_t n, int32_t m, const float* Q, int32_t nq,
                                int32_t k, int32_t metric, int64_t* idx, double* dist, int32_t threads);

int32_t orc_max_threads(void);

#ifdef __cplusplus
}
#endif
#endif
