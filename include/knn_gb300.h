/*
 * knn_gb300.h -- C ABI of the GB300 (sm_103a) adaptive k-nearest-neighbour
 * library.
 *
 * Method: LeJeune, Baraniuk, Heckel, "Adaptive Estimation for Approximate
 * k-Nearest-Neighbor Computations" (AISTATS 2019). Given points X (n x m) and a
 * query x, return a set of size at most k+h that contains the k nearest
 * neighbours of x in squared l2 distance (Section 3), by estimating the
 * normalised distances d_i = ||x - x_i||^2 / m from uniformly sampled
 * coordinates (Section 4) and discarding points whose confidence intervals
 * separate them from the k closest (Algorithm 1, Eq. d_ind, Eq. termination).
 *
 * Conventions shared by every entry point
 *   - All array arguments are DEVICE pointers unless stated; the caller owns
 *     them. Matrices are row-major and densely packed (row stride = m).
 *   - Every call is asynchronous on `stream` (a cudaStream_t, NULL = legacy
 *     default stream). Argument errors are detected on the host before any
 *     launch and returned; launch failures return KNN_ECUDA. Nothing is
 *     thrown across the ABI. knn_last_error() gives a message for the last
 *     failing call on the calling thread.
 *   - `workspace` is device scratch of at least the size the matching
 *     *_workspace_size function returns (256-byte aligned). If `workspace` is
 *     NULL the library allocates it stream-ordered (cudaMallocAsync) and frees
 *     it stream-ordered after the work.
 *   - Limits: 1 <= m <= 16384, 1 <= k, k + h <= 1024, n < 2^31.
 */
#ifndef KNN_GB300_H
#define KNN_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    KNN_OK = 0,
    KNN_EINVAL = 1,      /* invalid argument (sizes, delta, options, alignment) */
    KNN_ENOMEM = 2,      /* workspace too small, or allocation failed */
    KNN_ECUDA = 3,       /* a CUDA runtime call or launch failed */
    KNN_EUNSUPPORTED = 4 /* the device is not sm_103 / feature not built */
} knn_status;

/* Confidence-bound forms alpha(u) (normalised units):
 *   FOOTNOTE  sqrt(2 beta(u, delta/n) / u), beta = log(1/d') + 3 log log(1/d') + 1.5 log(1 + log u)
 *             (Section 4, footnote to the definition of alpha; needs delta/n < 1/e)
 *   LEMMA     sqrt(2 beta / u), beta = 2 log(125 log(1.12 u) / d'), d' = delta/n
 *             (Lemma "probound", Section 6)
 *   EXP       sqrt(C_alpha log(1 + (1 + log u) n / delta) / u)   (Section 5)       */
typedef enum { KNN_BOUND_FOOTNOTE = 0, KNN_BOUND_LEMMA = 1, KNN_BOUND_EXP = 2 } knn_bound;

/* Element type of the copy of the data the adaptive rounds gather from. */
typedef enum {
    KNN_STORE_F32 = 0,   /* the FP32 data itself */
    KNN_STORE_BF16 = 1,  /* bfloat16, round to nearest even */
    KNN_STORE_FP8 = 2    /* FP8 e4m3, per-row scale s_i = max_j |x_ij| / 448 (1 for a zero row) */
} knn_storage;

/* Distance of the method: squared l2 (the paper's), or l1. */
typedef enum { KNN_METRIC_L2SQ = 0, KNN_METRIC_L1 = 1 } knn_metric;

/* How a pair's coordinates are drawn: uniformly with replacement (Section 4,
 * the default), or without replacement (the footnote to Section 4: a cipher on
 * [m]): the pair's s-th draw is pi(s), pi a permutation of [0, m) keyed per
 * (seed, point, query) -- an 8-round balanced Feistel network on 2h bits
 * (4^h >= m, h >= 1) whose round keys are the words of blocks 2^32 - 2 and
 * 2^32 - 1 of the pair's Philox4x32-10 stream (counter and key as for the
 * draws with replacement), round function fmix32(R xor k_r) mod 2^h (MurmurHash3's
 * finaliser), cycle-walked onto [0, m). The bounds are unchanged (Hoeffding's
 * inequality holds for sampling without replacement). */
typedef enum { KNN_SAMPLE_WITH = 0, KNN_SAMPLE_WITHOUT = 1 } knn_sampling;

/* Options of knn_adaptive. Fill with knn_opts_default() and change fields. */
typedef struct {
    int32_t h;          /* extra set size: returned set has at most k+h points; -1 means h = k */
    int32_t bound;      /* knn_bound */
    double c_alpha;     /* C_alpha of the EXP form */
    int32_t B0;         /* coordinates sampled per point in round 0 (>= 1) */
    int32_t B;          /* coordinates per point in later rounds (>= 1) */
    int32_t grow;       /* 0: B per round; 1: max(B, T) per round (T doubles) */
    uint64_t qid_base;  /* query i of the batch draws coordinates with query id qid_base + i */
    uint64_t mask_p;    /* point field mask of the Philox counter (all ones: independent draws) */
    uint64_t mask_q;    /* query field mask of the Philox counter (all ones: independent draws) */
    int32_t threads;    /* threads per query (CTA) of the round-loop kernel: 0 (default 512), 256, 512, 1024 */
    int32_t max_ctas;   /* cap on resident CTAs of the round-loop kernel (0: all that fit) */
    int32_t block;      /* coordinates per sample, 0..64. 0 or 1: single coordinates (the paper's
                         * estimator). g > 1: block samples (not in the paper): a draw picks one of
                         * M = ceil(m/g) blocks of g consecutive coordinates (the last may be
                         * shorter), uniformly with replacement, and adds the block's sum of
                         * squared differences; B0 and B count blocks, the estimate is
                         * S / (T g), alpha takes u = T blocks (a block sum over g lies in
                         * [0, span^2], so the bounds of Section 4 hold), the distance is exact
                         * once T + B_r >= M, and out_evals counts g per block drawn. With
                         * g x element size = 32 bytes a draw reads one DRAM sector. */
    int32_t metric;     /* knn_metric: KNN_METRIC_L2SQ (default, the paper's squared l2) or KNN_METRIC_L1
                         * (the l1 distance Section 3 names as a generalisation): samples |x_j - q_j|,
                         * which lie in [0, span], so bounds are d^ -/+ span alpha(T); a stored copy
                         * with element error e moves a sample by at most e (width (span + e) alpha + e);
                         * the exact cap takes sum_j |x_j - q_j| on the FP32 data */
    int32_t sampling;   /* knn_sampling: KNN_SAMPLE_WITH (default) or KNN_SAMPLE_WITHOUT (single
                         * coordinates, the FP32 data; not with shared-coordinate copies, block
                         * samples, stored copies or knn_adaptive_noalloc: KNN_EINVAL) */
    int32_t r0_tensor;  /* 1: under shared coordinates (dataset calls with knn_dataset_share's copies,
                         * B0 <= 64, single coordinates, squared l2) round 0 is a tcgen05 contraction:
                         * every pair's sum over the shared columns J is formed as
                         * ||x_J - mu||^2 + ||q_J - mu||^2 - 2 (x_J - mu).(q_J - mu) with the centred
                         * values split into three BF16 parts (FP32 accumulation in tensor memory),
                         * mu a fixed centre; that sum (within a few units of FP32 roundoff of
                         * (||x_J - mu||^2 + ||q_J - mu||^2), not of the sum itself) decides which
                         * points the round-0 filter drops, and every kept point's sum is taken
                         * again sample by sample before the round's decisions. 0 (default): the
                         * sums are taken sample by sample for every point. Ignored elsewhere. */
    int32_t query_order; /* 1 (default): dataset calls take the queries of a batch in a locality order
                          * (a SimHash of each query: 16 signs of projections of the query minus the
                          * batch mean), so queries near one another run at the same time and the rows
                          * they keep active stay in L2; 0: batch order. Only the schedule changes: a
                          * query's draws, decisions and result depend on its id, not its turn. */
    int32_t row_pass;   /* 1 (default): per-pair draws over the FP32 data (storage KNN_STORE_F32, single
                         * coordinates, with replacement) take row passes: from a round r >= 2 whose
                         * active points nearly all survived the round before (at least 3/4 of them), or
                         * from a round drawing at least m/8 coordinates per point, and with at most
                         * 8192 points active, a warp reads each active point's row once and forms the
                         * sums of that round and of up to 5 later ones (up to the exact distance) from
                         * it, each in the order that round's own gather uses; the later rounds read
                         * their sums back. Results are the same bit for bit; draws of rounds a point
                         * no longer reaches are computed and dropped (not counted in out_evals).
                         * 0: every round gathers its own draws. */
} knn_opts;

void knn_opts_default(knn_opts* opts);

/* Bytes of device scratch knn_adaptive needs for these sizes/options. */
size_t knn_adaptive_workspace_size(int64_t n, int32_t m, int32_t nq, int32_t k, const knn_opts* opts);

/*
 * knn_adaptive -- the batched adaptive rounds (the hot path).
 *
 * For every query q (row q of Q, nq x m) independently:
 *   round r draws B_r new coordinates j ~ U[0, m) for every still-active
 *   point i (Philox4x32-10, key (low and high words of seed), counter
 *   (s/4, i & mask_p, low and high words of (qid_base+q) & mask_q), word
 *   s mod 4 scaled by floor(w m / 2^32), s = 0,1,2,... the point's sample
 *   number); sums (X[i,j] - Q[q,j])^2 into a
 *   running FP32 sum S_i (Kahan-compensated), or computes the exact distance
 *   once T + B_r >= m (Algorithm 1's exact-evaluation step at T = m);
 *   with span = max(X, Q[q]) - min(X, Q[q]) (the normalisation of Section 3)
 *   forms UCB/LCB = S_i/T -/+ span^2 alpha(T);
 *   tau_U = k-th smallest UCB over non-eliminated points, tau_L = min((k+1)-th
 *   smallest LCB over them, smallest LCB of an eliminated point);
 *   eliminates i if LCB_i > tau_U, accepts i if UCB_i < tau_L;
 *   stops when active+accepted <= k+h, accepted >= k, or after an exact round.
 *   Output: accepted points by (estimate, index), then active points by
 *   (estimate, index), at most k+h.
 *
 * X:        n x m float32 (device).           Q: nq x m float32 (device).
 * delta:    in (0,1); FOOTNOTE additionally needs delta/n < 1/e.
 * out_idx:  nq x (k+h) int64, -1 padded (device, required).
 * out_count:nq int32 candidates returned (device, required).
 * out_evals:nq int64 coordinate evaluations: samples drawn (x block) + m per exact
 *           distance (device, required).
 * out_rounds: nq int32 rounds run (device, may be NULL).
 * log_code: nq x n int32 decision log, 4*round + kind (kind 0 still active at
 *           the end, 1 eliminated, 2 accepted) (device, may be NULL).
 * log_S:    nq x n float32 sum S_i at the point's decision (device, may be NULL;
 *           only written when log_code is given).
 * Non-finite data give out_count = 0 for the affected queries.
 */
knn_status knn_adaptive(const float* X, int64_t n, int32_t m, const float* Q, int32_t nq,
                        int32_t k, double delta, uint64_t seed, const knn_opts* opts,
                        int64_t* out_idx, int32_t* out_count, int64_t* out_evals,
                        int32_t* out_rounds, int32_t* log_code, float* log_S,
                        void* workspace, size_t workspace_bytes, void* stream);

/*
 * knn_adaptive_noalloc -- knn_adaptive for callers that cannot allocate device
 * memory. (The paper has no counterpart: this is a deployment variant.)
 *
 * Some callers cannot call cudaMalloc: code running inside a host framework
 * that has already reserved all device memory in its own pool, plugins whose
 * host forbids outside allocations, or latency-critical paths that must not
 * risk an allocation failing or stalling. This entry point allocates nothing:
 * it runs the same round-loop kernel as knn_adaptive, with the same
 * arguments and outputs (all caller-owned), and takes its scratch from a
 * fixed array of knn_adaptive_noalloc_scratch_bytes() bytes (64 MiB) that
 * every GPU which loads the library holds until the process exits.
 *
 * - The scratch needs about 24 n bytes per query processed at a time; the
 *   call runs as many queries at once as fit (fewer than knn_adaptive when n
 *   is large) and returns KNN_EINVAL with a message when even one query's
 *   lists exceed the array (n above roughly 2.7 million).
 * - The first call on each device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current; make that first call
 *   before any stream capture. The address is cached with the id of the
 *   CUDA context it was found in, and looked up again when the current
 *   context differs (after cudaDeviceReset or a recreated primary context
 *   the module loads again and the array may move); after such a reset, make
 *   one call again before capturing.
 * - Every call shares the one array and starts by resetting the parts that
 *   must start fresh. Calls whose work overlaps on the GPU (on different
 *   streams or from different threads without ordering) race on the array
 *   and give wrong results; order them on one stream.
 * - Single coordinates only: opts->block above 1 returns KNN_EINVAL.
 */
size_t knn_adaptive_noalloc_scratch_bytes(void);
knn_status knn_adaptive_noalloc(const float* X, int64_t n, int32_t m, const float* Q, int32_t nq,
                                int32_t k, double delta, uint64_t seed, const knn_opts* opts,
                                int64_t* out_idx, int32_t* out_count, int64_t* out_evals,
                                int32_t* out_rounds, int32_t* log_code, float* log_S, void* stream);

/*
 * Datasets: a resident copy of X with everything the rounds need precomputed
 * once -- the data range (finite values; non-finite data flagged) and, on
 * request, BF16 and FP8 copies with their largest element error e.
 * (Mixed-precision storage is not in the paper; it cuts gather bytes. The
 * bounds stay valid: a sample of a copy differs from the data's sample by at
 * most eps = e (2 span + e), so the width of a sampled interval becomes
 * (span + 2e)^2 alpha(T) + eps. The exact cap always reads the FP32 data, so
 * exact distances stay exact (width 0). The returned candidates are then
 * reranked on the FP32 data.)
 *
 * knn_dataset_create: X is the caller's n x m FP32 device matrix and must
 *   stay alive and unchanged while the dataset is used (FP32 rounds and
 *   reranks read it). `copies` is a bit mask of (1 << KNN_STORE_BF16),
 *   (1 << KNN_STORE_FP8) and KNN_COPY_SCREEN (the operand of the
 *   tensor-core screen of knn_exact_ds). Allocates the copies with cudaMalloc, builds them
 *   on `stream` and waits for them. *out receives the handle.
 * knn_dataset_destroy: frees the copies (waits for the device first).
 * knn_dataset_error: largest |copy - X| of a copy (host value; 0 for F32).
 * knn_adaptive_ds: knn_adaptive over the dataset, gathering from the chosen
 *   copy (same outputs, same workspace size as knn_adaptive).
 */
typedef struct knn_dataset knn_dataset;
/* Operands of knn_exact_ds's tensor-core screens (see there): BF16 hi/lo
 * split (KNN_SCREEN_BF16X3), FP16 scaled by a power of two (KNN_SCREEN_F16),
 * single BF16 (KNN_SCREEN_BF16). */
enum { KNN_COPY_SCREEN = 1 << 3, KNN_COPY_SCREEN_F16 = 1 << 4, KNN_COPY_SCREEN_BF16 = 1 << 5 };
knn_status knn_dataset_create(const float* X, int64_t n, int32_t m, int32_t copies, void* stream,
                              knn_dataset** out);
knn_status knn_dataset_destroy(knn_dataset* ds);
knn_status knn_dataset_error(const knn_dataset* ds, int32_t storage, float* out_error);
knn_status knn_adaptive_ds(const knn_dataset* ds, int32_t storage, const float* Q, int32_t nq,
                           int32_t k, double delta, uint64_t seed, const knn_opts* opts,
                           int64_t* out_idx, int32_t* out_count, int64_t* out_evals,
                           int32_t* out_rounds, int32_t* log_code, float* log_S,
                           void* workspace, size_t workspace_bytes, void* stream);

/*
 * knn_dataset_share -- shared coordinates. With both Philox counter masks of
 * the options zero (mask_p = mask_q = 0) every (query, point) pair of a seed
 * draws the same coordinate sequence j_0, j_1, ..., so a point's first T draws
 * are the first T columns of a copy whose column t is column j_t of the data.
 * This builds that copy for `seed` and each storage in `copies` (bit mask of
 * 1 << KNN_STORE_*; BF16/FP8 need those copies in the dataset), rows padded to
 * a multiple of 8, and waits for it. knn_adaptive_ds(_multi) then reads
 * contiguous row prefixes instead of drawing and gathering, with the same
 * results bit for bit. (Each point's samples are still uniform draws with
 * replacement, as Lemma "probound" needs; points share them, which the
 * per-point union bound allows.) A later call with another seed replaces the
 * copies.
 */
knn_status knn_dataset_share(knn_dataset* ds, uint64_t seed, int32_t copies, void* stream);

/*
 * knn_adaptive_ds_multi -- one launch over a mixed batch: query q uses its
 * own k = k_per_query[q] (1 <= k <= k_max) and its own Philox query id
 * query_ids[q] (both device arrays), so a query's draws, decisions and
 * result do not depend on which batch or position it runs in. h is
 * opts->h, or each query's own k when opts->h < 0. out_idx rows are
 * k_max + h_max long (h_max = opts->h, or k_max), -1 padded. No decision
 * log. Workspace: knn_adaptive_ds_multi_workspace_size.
 * (Batching of requests with different k is a serving need; the paper
 * treats one query at a time.)
 */
size_t knn_adaptive_ds_multi_workspace_size(const knn_dataset* ds, int32_t nq, int32_t k_max, const knn_opts* opts);
knn_status knn_adaptive_ds_multi(const knn_dataset* ds, int32_t storage, const float* Q, int32_t nq,
                                 const int32_t* k_per_query, int32_t k_max, const uint64_t* query_ids,
                                 double delta, uint64_t seed, const knn_opts* opts,
                                 int64_t* out_idx, int32_t* out_count, int64_t* out_evals, int32_t* out_rounds,
                                 void* workspace, size_t workspace_bytes, void* stream);

/*
 * knn_rerank -- exact distances of candidate points, then top-k.
 *
 * For each query q, returns the k candidates c = cand[q, t] (t < ncand;
 * entries < 0 are skipped; the valid entries of a row must be distinct: a
 * repeated index is ranked twice) with the smallest d = sum_j (X[c,j] -
 * Q[q,j])^2 by (d, index) (Section 3's brute force restricted to the
 * candidates; the last step of returning the k nearest from the set S-hat).
 * Every candidate's distance is taken in FP32 (relative error at most
 * gamma_(m+2)); only the candidates whose FP32 distance lies within that
 * error of the k-th one are recomputed in FP64 and ranked, which gives the
 * same result as ranking every candidate in FP64. A row whose first entry is
 * -2 ranks every point instead.
 * out_idx: nq x k int64 (-1 padded when fewer valid candidates);
 * out_dist: nq x k float64 squared distances (+inf padded).
 * ncand <= 4096. No workspace.
 */
knn_status knn_rerank(const float* X, int64_t n, int32_t m, const float* Q, int32_t nq,
                      const int64_t* cand, int32_t ncand, int32_t k,
                      int64_t* out_idx, double* out_dist, void* stream);

/* knn_rerank under a distance (knn_metric): with KNN_METRIC_L1 the FP64
 * distances are sum_j |X[c,j] - Q[q,j]| and out_dist holds them. */
knn_status knn_rerank_metric(const float* X, int64_t n, int32_t m, const float* Q, int32_t nq,
                             const int64_t* cand, int32_t ncand, int32_t k, int32_t metric,
                             int64_t* out_idx, double* out_dist, void* stream);

/*
 * knn_exact -- the naive exact method (Section 3: all distances, then
 * select): a screening pass computes ||x_i||^2 - 2 x_i.q + ||q||^2 for every
 * pair, keeps every point whose screened value is within the screen's
 * proven rounding bound of the k-th smallest, and knn_rerank's FP64 step
 * picks the exact k nearest among them.
 * out_idx: nq x k int64; out_dist: nq x k float64.
 */
size_t knn_exact_workspace_size(int64_t n, int32_t m, int32_t nq, int32_t k);
knn_status knn_exact(const float* X, int64_t n, int32_t m, const float* Q, int32_t nq, int32_t k,
                     int64_t* out_idx, double* out_dist,
                     void* workspace, size_t workspace_bytes, void* stream);

/* knn_exact under the l1 distance (the generalisation Section 3 names): FP32
 * SIMT distances of every pair (each within a relative error (m+2) 2^-24 of
 * the exact one; l1 has no product form for a tensor-core screen), every
 * point within that margin of the k-th kept, FP64 l1 rerank. Same arguments,
 * workspace (knn_exact_workspace_size) and outputs as knn_exact; out_dist
 * holds l1 distances. */
knn_status knn_exact_l1(const float* X, int64_t n, int32_t m, const float* Q, int32_t nq, int32_t k,
                        int64_t* out_idx, double* out_dist, void* workspace, size_t workspace_bytes,
                        void* stream);

/*
 * knn_exact_ds -- the naive exact method over a resident dataset, with a
 * choice of screen:
 *   KNN_SCREEN_F32     the FP32 SIMT screen of knn_exact;
 *   KNN_SCREEN_F16     a tcgen05 tensor-core GEMM of the centred data and
 *                      queries, each scaled by a power of two and rounded to
 *                      FP16 (FP32 accumulation in tensor memory); needs
 *                      KNN_COPY_SCREEN_F16;
 *   KNN_SCREEN_BF16    the same GEMM on values rounded to BF16; needs
 *                      KNN_COPY_SCREEN_BF16;
 *   KNN_SCREEN_BF16X3  the same GEMM on the centred data split into BF16
 *                      hi + lo parts (three products per pair); needs
 *                      KNN_COPY_SCREEN.
 * The tensor-core screens (sm_10x devices) select inside the GEMM: a first
 * pass over a subset of the points bounds each query's k-th screened value
 * from above, a second pass appends every pair within twice the screen's
 * proven error bound of that bound to the query's candidate list (no n x nq
 * matrix is written); the FP32 screen writes the matrix and selects. All
 * keep every true k-nearest point and rank the candidates as knn_rerank does,
 * so the result is exact: the k nearest by (distance, index). A query whose
 * candidates overflow the list is ranked over every point.
 */
enum { KNN_SCREEN_F32 = 0, KNN_SCREEN_BF16X3 = 1, KNN_SCREEN_F16 = 2, KNN_SCREEN_BF16 = 3 };
size_t knn_exact_ds_workspace_size(const knn_dataset* ds, int32_t screen, int32_t nq);
knn_status knn_exact_ds(const knn_dataset* ds, int32_t screen, const float* Q, int32_t nq, int32_t k,
                        int64_t* out_idx, double* out_dist, void* workspace, size_t workspace_bytes, void* stream);

/* Failure detection, a test hook (no counterpart in the paper): the
 * tensor-core kernels' pipeline waits give up after `tries` polls of their
 * barrier (tries < 0 restores the default, about a second). A wait that gives
 * up records a code read by knn_device_status; its call's outputs are then
 * invalid. With 0 every such wait gives up at once, before any copy or
 * matrix multiply is issued. Applies to calls made after it. */
knn_status knn_debug_wait_limit(int64_t tries);

/* Library status of the current device: 0, or a nonzero code recorded by a
 * kernel that gave up a bounded wait (the call's outputs are then invalid).
 * Waits for the device, then clears the status. */
knn_status knn_device_status(int32_t* out);

/* Clock totals of the phases of the adaptive round-loop kernel, summed over
 * its CTAs (SM clock cycles seen by each CTA's first thread between phase
 * boundaries; tracing, not part of the method). out: 16 host uint64_t:
 *   [0] setup  [1] sampled gathers  [2] exact rows  [3] select
 *   [4] thresholds  [5] decide + compact  [6] output (per query)
 * for the rounds after round 0, and [8..13] phases 0-5 of round 0 ([9] is the
 * round-0 filter when the point-major pass ran). reset != 0 zeroes the totals
 * after reading. Waits for the device. Only a library compiled with
 * KNN_PHASE_TIMING records them (a separate build: the timing adds a barrier
 * per query and atomics by one thread); any other returns KNN_EUNSUPPORTED. */
knn_status knn_phase_clocks(uint64_t* out, int32_t reset);

/* Kernel timing of knn_adaptive_ds(_multi) calls (measurement; no
 * counterpart in the paper). knn_kernel_timing(1) makes later calls record
 * CUDA events on their stream around the point-major round-0 pass and the
 * round-loop kernel (do not enable it while capturing a CUDA graph);
 * knn_kernel_timing(0) stops. knn_kernel_times waits for the last recorded
 * event and writes out_ms[0] = total milliseconds of the round-0 passes and
 * out_ms[1] = of the round-loop kernels, over every call since the last
 * reset (2 host doubles); reset != 0 starts a new total. */
knn_status knn_kernel_timing(int32_t enable);
knn_status knn_kernel_times(double* out_ms, int32_t reset);

/* Rate of the coordinate generator (measurement; no counterpart in the
 * paper): ctas CTAs of 1024 threads each evaluate iters Philox4x32-10 blocks
 * with the kernels' own generator function and write one word per thread to
 * out (device, ctas * 1024 uint32, caller-owned). Time it on `stream` to
 * measure the blocks per second this GPU sustains; every draw of the
 * per-pair estimator costs a quarter of a block. KNN_EINVAL on iters < 0,
 * ctas < 1 or a null out. */
knn_status knn_philox_blocks(int64_t iters, int32_t ctas, uint32_t* out, void* stream);

/* Message of the last failing call on this thread ("" if none). */
const char* knn_last_error(void);

/* Library version string. */
const char* knn_version(void);

#ifdef __cplusplus
}
#endif
#endif
