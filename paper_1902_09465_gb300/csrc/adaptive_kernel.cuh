// adaptive_kernel.cuh -- the batched adaptive rounds of the k-NN method of
// LeJeune, Baraniuk and Heckel (AISTATS 2019), as one persistent kernel,
// templated on the element type of the gathered copy (FP32, BF16, FP8 e4m3
// with per-row scale).
//
// One CTA owns one query at a time and runs all of its rounds; CTAs take the
// next query from a device work queue, so queries of uneven difficulty share
// the GPU without host round trips. Per round and query:
//   gather    every active point draws B_r coordinates (Philox4x32-10) and
//             adds the squared differences to its FP32 Kahan sum S, or takes
//             its exact distance once the count would reach m (Algorithm 1);
//             the same pass histograms the new sums (bits 31..20 of the key);
//   select    the k+1 smallest sums among active points (radix select that
//             finishes in shared memory);
//   bounds    UCB/LCB = S/T +- span^2 alpha(T) (Section 4, footnote and
//             Lemma forms, or the Section 5 form with C_alpha);
//   decide    tau_U = k-th smallest UCB over active and accepted points,
//             tau_L = min((k+1)-th smallest LCB, smallest eliminated LCB);
//             LCB > tau_U eliminates, UCB < tau_L accepts (the batched form
//             of Eq. d_ind and Eq. termination);
//   compact   order-preserving prefix-sum compaction of the survivors into the
//             other half of the CTA's ping-pong buffers.
// Active points of a query all carry the same sample count T, so T is a
// per-round scalar, and the per-point state is (id, S, Kahan term).
//
// Variants, each a template argument: the element type wraps the copy
// for shared coordinates (Perm: row prefixes of a column-permuted copy),
// block samples (Blk: one of ceil(m/g) blocks of g coordinates per draw) or
// draws without replacement (Wor: each pair's keyed permutation of [0, m)); a
// bool selects the l1 distance (|x - q| terms, span-scaled widths). Round 0
// of a dataset call comes from a point-major pass (round0_kernel for per-pair
// draws, round0_shared_kernel for shared coordinates) that writes the
// round-0 sums and per-tile minima; the round loop then drops the provably
// eliminated points in one streaming pass (round0_filter) before its first
// select.
#pragma once

#include <cuda_fp8.h>

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <type_traits>

#include "knn_common.cuh"
#include "knn_internal.h"

namespace knn {

struct AdaptiveArgs {
  const float* X;       // the FP32 data, row-major n x m (exact rounds read it)
  const void* G;        // gathered copy: float, bf16 bits or e4m3 bytes, row-major n x m
  const float* gscale;  // per-row scale of an FP8 copy (else unused)
  const float* emax;    // largest |copy - data| of a stored copy (device scalar; null for FP32)
  const float* Q;
  int64_t n;
  int32_t m;
  int32_t nq;
  int32_t k, h;         // k (the largest k when kq is given) and h; see h_per_k
  const int32_t* kq;    // per-query k (device, may be null: every query uses k)
  const uint64_t* qids; // per-query id of the Philox counter (device, may be null: qid_base + q)
  int32_t h_per_k;      // 1: each query uses h = its k; 0: every query uses h
  int32_t out_stride;   // row length of out_idx
  int32_t bound;
  float a_c0, a_c1, c_alpha;  // host-precomputed constants of alpha(u)
  int32_t B0, B, grow;
  uint64_t seed, qid_base, mask_p, mask_q;
  PhiloxKeys rk;        // round keys of seed (philox_keys)
  const uint32_t* xrange;  // ordered keys of min(X), max(X) over finite values; [2] non-finite flag
  int32_t* ws_ids;
  float* ws_S;
  float* ws_C;
  int32_t* ws_acc_id;
  float* ws_acc_d;
  float* ws_acc_U;
  float* ws_acc_L;
  int32_t acc_cap;
  int32_t* queue;
  int64_t* out_idx;
  int32_t* out_count;
  int64_t* out_evals;
  int32_t* out_rounds;
  int32_t* log_code;
  float* log_S;
  int32_t vec;  // rows of X start on 16-byte boundaries: exact rows use 16-byte loads
  int32_t g;    // coordinates per sample (1: single coordinates; > 1: blocks of g consecutive ones)
  int32_t Mb;   // samples that make a distance exact: ceil(m / g)
  int32_t gvec; // a block is 32 bytes of the copy on 16-byte aligned rows: two 16-byte loads
  int32_t l1;   // 1: l1 distance (samples |x - q|); 0: squared l2 (samples (x - q)^2)
  int32_t qvec; // query rows start on 16-byte boundaries (m % 4 == 0 and Q aligned): 16-byte loads
  const float* R0;      // round-0 sums [nq][n] precomputed by round0_kernel (null: round 0 samples in place)
  const float* R0min;   // smallest round-0 sum of each tile of points [nq][r0tiles] (null: no filter)
  int32_t r0tiles;      // tiles per query in R0min
  const int32_t* jperm; // shared-coordinate copies: column of draw t (t < m), for Perm element types
  int32_t mp;           // row pitch of a shared-coordinate copy (m rounded up to 8)
  unsigned long long* phase_clk;  // per-phase clock totals [16] (libraries built with phase timing; else null)
  int32_t wor_h;        // draws without replacement: half width h of the Feistel network (4^h >= m)
  const int32_t* qorder = nullptr;  // order in which CTAs take the queries (null: batch order)
  int32_t r0_resum = 0; // the round-0 sums came from the tensor-core contraction: the points the
                        // round-0 filter keeps get their sums again, sample by sample
  float* ws_F = nullptr;  // row passes: later rounds' sums by pass slot, [kFuseRounds][fuse_cap] per CTA,
                          // then each active slot's pass slot, [2][fuse_cap] (int32)
  int32_t fuse_cap = 0;   // slots a row pass may cover (0: no row passes)
};

// Row passes (per-pair draws over the FP32 data): once the active points
// mostly survive from one round to the next, or a round draws at least m/8
// coordinates per point, a warp reads each active point's row once into
// shared memory and takes the sums of up to kFuseRounds rounds from it (the
// remaining ones up to the exact distance when they fit), each in the order
// its own round's gather would use. Later rounds read their sums back.
constexpr int kFuseRounds = 6;
constexpr int kFuseParts = kFuseRounds * 32;  // per-warp partial sums (virtual lanes of every round)
constexpr int kFuseCap = 8192;

// Phase timing (compiled in only with KNN_PHASE_TIMING): thread 0 of each CTA
// adds the SM clocks spent since the previous boundary to phase i of
// phase_clk; phases of round 0 go to i + 8 (the output phase stays at 6).
#ifdef KNN_PHASE_TIMING
#define KNN_PHASE_START long long phase_t0_ = clock64()
#define KNN_PHASE(i)                                                                                 \
  do {                                                                                               \
    if (threadIdx.x == 0 && a.phase_clk) {                                                           \
      const long long t_ = clock64();                                                                \
      atomicAdd(a.phase_clk + (i) + ((r) == 0 && (i) != 6 ? 8 : 0), (unsigned long long)(t_ - phase_t0_)); \
      phase_t0_ = t_;                                                                                \
    }                                                                                                \
  } while (0)
#define KNN_PHASE_SYNC(i) \
  do {                    \
    __syncthreads();      \
    KNN_PHASE(i);         \
  } while (0)
#else
#define KNN_PHASE_START \
  do {                  \
  } while (0)
#define KNN_PHASE(i) \
  do {               \
  } while (0)
#define KNN_PHASE_SYNC(i) \
  do {                    \
  } while (0)
#endif

// Element access of the gathered copy. A stored BF16 value is the top half of
// the FP32 word; an FP8 e4m3 value is converted exactly and multiplied by its
// row's scale with one FP32 rounding (__fmul_rn, never fused into the
// following subtraction): fl32(s * value) is the dequantised value the error
// bound is measured on.
struct ElemF32 {
  using T = float;
  static constexpr int kStorage = KNN_STORE_F32;
  static constexpr bool kScaled = false;
  static constexpr bool kPerm = false;
  static constexpr bool kBlk = false;
  static constexpr bool kWor = false;
  __device__ static __forceinline__ float load(const T* p) { return __ldg(p); }
  __device__ static __forceinline__ float conv(T v) { return v; }
};
struct ElemBF16 {
  using T = uint16_t;
  static constexpr int kStorage = KNN_STORE_BF16;
  static constexpr bool kScaled = false;
  static constexpr bool kPerm = false;
  static constexpr bool kBlk = false;
  static constexpr bool kWor = false;
  __device__ static __forceinline__ float conv(T v) { return __uint_as_float((uint32_t)v << 16); }
  __device__ static __forceinline__ float load(const T* p) { return conv(__ldg(p)); }
};
struct ElemFP8 {
  using T = uint8_t;
  static constexpr int kStorage = KNN_STORE_FP8;
  static constexpr bool kScaled = true;
  static constexpr bool kPerm = false;
  static constexpr bool kBlk = false;
  static constexpr bool kWor = false;
  __device__ static __forceinline__ float conv(T v) {
    __nv_fp8_e4m3 f;
    f.__x = v;
    return static_cast<float>(f);
  }
  __device__ static __forceinline__ float load(const T* p) { return conv(__ldg(p)); }
};

constexpr int kIPT = 4;  // consecutive slots per thread in the decide pass

template <int NT>
struct AdaptiveShared {
  BlockScratch<NT> bs;
  SelectShared ss;
  int q;
  int nacc_add;
  int bad;
  float tauU, tauL;
  // the rounds of a row pass: samples [f_T[i], f_Tn[i]); the last one exact
  // if f_exact; sampled round i has virtual lanes f_uoff[i] .. f_uoff[i+1]-1
  int f_nr, f_exact;
  int f_T[kFuseRounds], f_Tn[kFuseRounds], f_uoff[kFuseRounds + 1];
  int4 f_unit[kFuseParts];  // virtual lane u: (T, Tn, G, v) of its round
};

// Shared coordinates (both counter masks zero): every pair draws the same
// coordinate sequence j_0, j_1, ... for a seed, so a point's first T draws are
// the first T columns of a copy whose column t holds column j_t of the data.
// Rounds then read contiguous row prefixes instead of drawing and gathering.
template <class Base>
struct Perm : Base {
  static constexpr bool kPerm = true;
};

// Block samples (g > 1 coordinates per draw) over a stored copy: the same
// round loop with gather_blocks in place of gather_sampled.
template <class Base>
struct Blk : Base {
  static constexpr bool kBlk = true;
};

// Draws without replacement (single coordinates): a pair's s-th draw is the
// s-th value of its keyed permutation of [0, m) (wor_coordinate) in place of
// a uniform word scaled to [0, m).
template <class Base>
struct Wor : Base {
  static constexpr bool kWor = true;
};

// MurmurHash3's 32-bit finaliser (Appleby, public domain): the round function
// of the keyed permutation.
__device__ __forceinline__ uint32_t fmix32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x85EBCA6Bu;
  x ^= x >> 13;
  x *= 0xC2B2AE35u;
  x ^= x >> 16;
  return x;
}

// Draw s (< m) of a pair sampled without replacement (the footnote to
// Section 4: a cipher on [m]): a balanced Feistel network of 8 rounds on 2h
// bits (L the high h bits; a round maps (L, R) to (R, L ^ (fmix32(R ^ k_r) mod
// 2^h))) keyed by the eight words of the last two Philox blocks of the pair's
// stream (k),
// extended to [0, m) by cycle walking (apply it again until the value is
// below m). From s < m the walk returns below m within one cycle of the
// permutation of [0, 4^h); the walk is capped at 4^h steps all the same.
__device__ __forceinline__ int wor_coordinate(const Draws8& k, uint32_t s, uint32_t m, int h) {
  const uint32_t mask = (1u << h) - 1u;
  const uint32_t cap = 1u << (2 * h);
  uint32_t x = s;
  for (uint32_t step = 0; step < cap; ++step) {
    uint32_t L = x >> h, R = x & mask;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const uint32_t nR = L ^ (fmix32(R ^ philox_word(k, r)) & mask);
      L = R;
      R = nR;
    }
    x = (L << h) | R;
    if (x < m) return (int)x;
  }
  return 0;
}

// 8 consecutive elements of a shared-coordinate row (16-byte aligned blocks
// for FP32 and BF16, 8-byte for FP8), converted to FP32.
template <class E>
__device__ __forceinline__ void load8(const typename E::T* p, float* x) {
  if constexpr (sizeof(typename E::T) == 4) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(p));
    const float4 b = __ldg(reinterpret_cast<const float4*>(p) + 1);
    x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
    x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
  } else if constexpr (sizeof(typename E::T) == 2) {
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(p));
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = E::conv((typename E::T)(w[i >> 1] >> (16 * (i & 1))));
  } else {
    const uint2 v = __ldg(reinterpret_cast<const uint2*>(p));
    const uint32_t w[2] = {v.x, v.y};
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = E::conv((typename E::T)(w[i >> 2] >> (8 * (i & 3))));
  }
}

// alpha(u) in normalised units. c0/c1 carry the delta- and n-dependent
// constants computed on the host in double precision.
__device__ __forceinline__ float alpha_of(const AdaptiveArgs& a, int64_t u) {
  const float uu = (float)u;
  const float lu = logf(uu);
  if (a.bound == KNN_BOUND_FOOTNOTE) {
    // beta = log(1/d') + 3 log log(1/d') + 1.5 log(1 + log u)
    const float beta = a.a_c0 + 1.5f * logf(1.0f + lu);
    return sqrtf(2.0f * beta / uu);
  }
  if (a.bound == KNN_BOUND_LEMMA) {
    // beta = 2 log(125 log(1.12 u) / d') = 2 (log(125/d') + log log(1.12 u))
    const float beta = 2.0f * (a.a_c0 + logf(logf(1.12f * uu)));
    return sqrtf(2.0f * beta / uu);
  }
  // sqrt(C log(1 + (1 + log u) n / delta) / u), c1 = n / delta
  return sqrtf(a.c_alpha * log1pf((1.0f + lu) * a.a_c1) / uu);
}

// One coordinate's term added to a partial sum: (x - q)^2 (squared l2, one
// fused multiply-add) or |x - q| (l1). The metric is a template argument of
// every gather; the round loop picks the instantiation once per call site.
template <bool L1>
__device__ __forceinline__ float add_term(float d, float part) {
  if constexpr (L1)
    return part + fabsf(d);
  else
    return fmaf(d, d, part);
}

// Value of rank `kth` (1-based) in the union of the ascending array A[0..na)
// and the unordered array Bv[0..nb). Every thread gets the result.
template <int NT>
__device__ float kth_of_union(const float* A, int na, const float* Bv, int nb, int kth, float* out) {
  for (int t = threadIdx.x; t < na + nb; t += NT) {
    const float v = t < na ? A[t] : Bv[t - na];
    int lo = 0, hi = na;  // lower bound of v in A
    while (lo < hi) {
      int mid = (lo + hi) >> 1;
      if (A[mid] < v) lo = mid + 1; else hi = mid;
    }
    int lt = lo;
    hi = na;  // upper bound of v in A
    while (lo < hi) {
      int mid = (lo + hi) >> 1;
      if (A[mid] <= v) lo = mid + 1; else hi = mid;
    }
    int le = lo;
    for (int b = 0; b < nb; ++b) {
      const float x = Bv[b];
      lt += x < v;
      le += x <= v;
    }
    if (lt < kth && kth <= le) *out = v;
  }
  __syncthreads();
  const float r = *out;
  __syncthreads();
  return r;
}

// Sampled gather: slots [0, nact) of the active list, samples T .. Tn-1.
// G lanes share a point (G = blocks of 8 draws this round, rounded up to a
// power of two, at most 32); each lane walks its blocks of its points as one
// flat sequence of items and computes the next item's Philox blocks while the
// current item's 8 loads are in flight (software pipelining over items).
template <int NT, class E, bool L1>
__device__ __forceinline__ void gather_sampled(const AdaptiveArgs& a, uint64_t qid, int r, int nact, int64_t T, int64_t Tn,
                                               const float* qs, const int32_t* idc, float* Sc, float* Cc,
                                               uint32_t* hist, bool ids_given = false) {
  using Tp = typename E::T;
  const int m = a.m;
  const uint64_t blo = (uint64_t)T >> 3, bhi = (uint64_t)(Tn - 1) >> 3;
  const int nblk = (int)(bhi - blo + 1);
  int G = 1;
  while (G < nblk && G < 32) G <<= 1;
  const int lg = __ffs(G) - 1;
  if constexpr (E::kPerm) {
    // shared coordinates: row prefixes of the permuted copy; qs here holds the
    // query permuted the same way. Same lanes, order and reduction as below.
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int grp = lane >> lg, gl = lane & (G - 1);
    const int ppw = 32 >> lg;
    for (int base = warp * ppw; base < nact; base += (NT / 32) * ppw) {
      const int sidx = base + grp;
      float part = 0.0f;
      if (sidx < nact) {
        const int id = (r == 0 && !ids_given) ? sidx : idc[sidx];
        const Tp* xr = static_cast<const Tp*>(a.G) + (size_t)id * (size_t)a.mp;
        const float sc = E::kScaled ? __ldg(a.gscale + id) : 1.0f;
        for (uint64_t b = blo + gl; b <= bhi; b += G) {
          float x[8];
          load8<E>(xr + 8 * b, x);
#pragma unroll
          for (int w = 0; w < 8; ++w) {
            const int64_t s = (int64_t)(8 * b) + w;
            if (s >= T && s < Tn) {
              const float d = (E::kScaled ? __fmul_rn(x[w], sc) : x[w]) - qs[s];
              part = add_term<L1>(d, part);
            }
          }
        }
      }
#pragma unroll
      for (int o = 16; o; o >>= 1)
        if (o < G) part += __shfl_xor_sync(0xffffffffu, part, o);
      if (sidx < nact && gl == 0) {
        float S;
        if (r == 0) {
          S = part;
        } else {
          const float S0 = Sc[sidx], c0 = Cc[sidx];
          const float y = part - c0;
          const float tt = S0 + y;
          Cc[sidx] = (tt - S0) - y;
          S = tt;
        }
        Sc[sidx] = S;
        atomicAdd(&hist[f2key(S) >> 20], 1u);
      }
    }
    return;
  }
  const int nbl = (nblk + G - 1) / G;  // blocks per lane per point
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane >> lg, gl = lane & (G - 1);
  const int ppw = 32 >> lg;
  const int pstride = (NT / 32) * ppw;
  const uint64_t qfield = qid & a.mask_q;
  const Tp* G0 = static_cast<const Tp*>(a.G);
  // items of this lane: t = pair_iter * nbl + j, point slot warp*ppw + grp + pair_iter*pstride, block blo + gl + j*G
  const int first = warp * ppw;
  const int npairs = first < nact ? (nact - first + pstride - 1) / pstride : 0;  // warp-uniform
  const int nitems = npairs * nbl;
  if (nitems == 0) return;
  // item state: slot, point id, block, and its Philox output
  auto item = [&](int t, int& sidx, int& id, uint64_t& b, bool& has) {
    const int pi = t / nbl, j = t - pi * nbl;
    sidx = first + grp + pi * pstride;
    b = blo + (uint64_t)(gl + j * G);
    has = sidx < nact && b <= bhi;
    id = has ? ((r == 0) ? sidx : idc[sidx]) : 0;
  };
  int sidx, id;
  uint64_t b;
  bool has;
  const int Ti = (int)T, Tni = (int)Tn;
  item(0, sidx, id, b, has);
  // (without replacement one item per pair: the last two blocks of its stream, the round keys)
  Draws8 ph = has ? pair_draws8(E::kWor ? kWorKeyItem : (uint32_t)b, (uint64_t)id & a.mask_p, qfield, a.rk)
                  : Draws8{};
  float part = 0.0f;
  for (int t = 0; t < nitems; ++t) {
    // issue the current item's loads
    float xv[8];
    int jj[8];
    const Tp* xr = G0 + (size_t)id * (size_t)m;
    const int s0 = (int)(b << 3);  // sampled rounds have Tn < m
    // draws of the item inside [T, Tn): bit w for draw s0 + w
    uint32_t okm = 0;
    if (has) {
      if (s0 >= Ti && s0 + 8 <= Tni) {
        okm = 0xFFu;
      } else {
#pragma unroll
        for (int w = 0; w < 8; ++w) okm |= (uint32_t)(s0 + w >= Ti && s0 + w < Tni) << w;
      }
    }
    if (!E::kWor && okm == 0xFFu) {
#pragma unroll
      for (int w = 0; w < 8; ++w) {
        jj[w] = (int)__umulhi(philox_word(ph, w), (uint32_t)m);
        xv[w] = E::load(xr + jj[w]);
      }
    } else {
#pragma unroll
      for (int w = 0; w < 8; ++w) {
        const bool ok = (okm >> w) & 1u;
        if constexpr (E::kWor)
          jj[w] = ok ? wor_coordinate(ph, (uint32_t)(s0 + w), (uint32_t)m, a.wor_h) : 0;
        else
          jj[w] = (int)__umulhi(philox_word(ph, w), (uint32_t)m);
        xv[w] = ok ? E::load(xr + jj[w]) : 0.0f;
      }
    }
    const float sc = (E::kScaled && has) ? __ldg(a.gscale + id) : 1.0f;
    const int cur_sidx = sidx;
    const uint32_t cur_okm = okm;
    // the next item's Philox while the loads are in flight
    if (t + 1 < nitems) {
      item(t + 1, sidx, id, b, has);
      if (has) ph = pair_draws8(E::kWor ? kWorKeyItem : (uint32_t)b, (uint64_t)id & a.mask_p, qfield, a.rk);
    }
    // consume
    if (cur_okm == 0xFFu) {
#pragma unroll
      for (int w = 0; w < 8; ++w) {
        const float d = (E::kScaled ? __fmul_rn(xv[w], sc) : xv[w]) - qs[jj[w]];
        part = add_term<L1>(d, part);
      }
    } else if (cur_okm) {
#pragma unroll
      for (int w = 0; w < 8; ++w) {
        if ((cur_okm >> w) & 1u) {
          const float d = (E::kScaled ? __fmul_rn(xv[w], sc) : xv[w]) - qs[jj[w]];
          part = add_term<L1>(d, part);
        }
      }
    }
    if ((t + 1) % nbl == 0) {  // last block of this point: combine the G lanes and store
#pragma unroll
      for (int o = 16; o; o >>= 1)
        if (o < G) part += __shfl_xor_sync(0xffffffffu, part, o);
      const int ps = first + grp + (t / nbl) * pstride;
      if (ps < nact && gl == 0) {
        float S;
        if (r == 0) {
          S = part;
        } else {
          // Kahan-compensated running sum
          const float S0 = Sc[ps], c0 = Cc[ps];
          const float y = part - c0;
          const float tt = S0 + y;
          Cc[ps] = (tt - S0) - y;
          S = tt;
        }
        Sc[ps] = S;
        atomicAdd(&hist[f2key(S) >> 20], 1u);
      }
      part = 0.0f;
    }
    (void)cur_sidx;
  }
}

// Sum of squared differences over one 32-byte block of the copy (two 16-byte
// words, elements in memory order) against the FP32 query values qb, added
// to part in coordinate order.
template <class E, bool L1>
__device__ __forceinline__ float block_sum32(const uint4 v0, const uint4 v1, const float* qb, float sc, float part) {
  constexpr int per = 4 / (int)sizeof(typename E::T);  // elements per 32-bit word
  const uint32_t wv[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
  for (int c4 = 0; c4 < 8 * per; c4 += 4) {
    const float4 q4 = *reinterpret_cast<const float4*>(qb + c4);
    const float qv[4] = {q4.x, q4.y, q4.z, q4.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int c = c4 + e;
      const uint32_t word = wv[c / per];
      float x;
      if constexpr (per == 1)
        x = __uint_as_float(word);
      else if constexpr (per == 2)
        x = E::conv((typename E::T)(word >> (16 * (c & 1))));
      else
        x = E::conv((typename E::T)(word >> (8 * (c & 3))));
      if constexpr (E::kScaled) x = __fmul_rn(x, sc);
      const float d = x - qv[e];
      part = add_term<L1>(d, part);
    }
  }
  return part;
}

// Block samples (g > 1 coordinates per draw): draw s of a pair picks block
// jb = floor(word_s * Mb / 2^32) and adds the squared differences of its
// coordinates jb*g .. min(jb*g + g, m) - 1 in order. Lanes, items (one
// two Philox blocks, 8 draws) and the reduction are those of gather_sampled. A
// 32-byte block on 16-byte aligned rows (gvec) is two 16-byte loads, F draws
// in flight per lane; a ragged last block is read element by element.
template <int NT, class E, bool L1>
__device__ __forceinline__ void gather_blocks(const AdaptiveArgs& a, uint64_t qid, int r, int nact, int64_t T, int64_t Tn,
                                              const float* qs, const int32_t* idc, float* Sc, float* Cc,
                                              uint32_t* hist) {
  using Tp = typename E::T;
  constexpr int F = 2;
  const int m = a.m, g = a.g;
  const uint32_t Mb = (uint32_t)a.Mb;
  const uint64_t blo = (uint64_t)T >> 3, bhi = (uint64_t)(Tn - 1) >> 3;
  const int nblk = (int)(bhi - blo + 1);
  int G = 1;
  while (G < nblk && G < 32) G <<= 1;
  const int lg = __ffs(G) - 1;
  const int nbl = (nblk + G - 1) / G;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane >> lg, gl = lane & (G - 1);
  const int ppw = 32 >> lg;
  const int pstride = (NT / 32) * ppw;
  const uint64_t qfield = qid & a.mask_q;
  const Tp* G0 = static_cast<const Tp*>(a.G);
  const int first = warp * ppw;
  const int npairs = first < nact ? (nact - first + pstride - 1) / pstride : 0;  // warp-uniform
  const int nitems = npairs * nbl;
  float part = 0.0f;
  for (int t = 0; t < nitems; ++t) {
    const int pi = t / nbl, jt = t - pi * nbl;
    const int sidx = first + grp + pi * pstride;
    const uint64_t b = blo + (uint64_t)(gl + jt * G);
    if (sidx < nact && b <= bhi) {
      const int id = (r == 0) ? sidx : idc[sidx];
      const Draws8 ph = pair_draws8((uint32_t)b, (uint64_t)id & a.mask_p, qfield, a.rk);
      const Tp* xr = G0 + (size_t)id * (size_t)m;
      const float sc = E::kScaled ? __ldg(a.gscale + id) : 1.0f;
      const int64_t s0 = (int64_t)(b << 3);
#pragma unroll
      for (int w0 = 0; w0 < 8; w0 += F) {
        uint4 v[F][2];
        int cb[F];
        bool ok[F], full[F];
#pragma unroll
        for (int f = 0; f < F; ++f) {
          const int64_t s = s0 + w0 + f;
          ok[f] = s >= T && s < Tn;
          cb[f] = (int)__umulhi(philox_word(ph, w0 + f), Mb) * g;
          full[f] = a.gvec && cb[f] + g <= m;
          if (ok[f] && full[f]) {
            const uint4* p = reinterpret_cast<const uint4*>(xr + cb[f]);
            v[f][0] = __ldg(p);
            v[f][1] = __ldg(p + 1);
          }
        }
#pragma unroll
        for (int f = 0; f < F; ++f) {
          if (!ok[f]) continue;
          if (full[f]) {
            part = block_sum32<E, L1>(v[f][0], v[f][1], qs + cb[f], sc, part);
          } else {
            const int c1 = min(cb[f] + g, m);
            for (int c = cb[f]; c < c1; ++c) {
              float x = E::load(xr + c);
              if (E::kScaled) x = __fmul_rn(x, sc);
              const float d = x - qs[c];
              part = add_term<L1>(d, part);
            }
          }
        }
      }
    }
    if ((t + 1) % nbl == 0) {  // last block of this point: combine the G lanes and store
#pragma unroll
      for (int o = 16; o; o >>= 1)
        if (o < G) part += __shfl_xor_sync(0xffffffffu, part, o);
      if (sidx < nact && gl == 0) {
        float S;
        if (r == 0) {
          S = part;
        } else {
          const float S0 = Sc[sidx], c0 = Cc[sidx];
          const float y = part - c0;
          const float tt = S0 + y;
          Cc[sidx] = (tt - S0) - y;
          S = tt;
        }
        Sc[sidx] = S;
        atomicAdd(&hist[f2key(S) >> 20], 1u);
      }
      part = 0.0f;
    }
  }
}

// Exact round: one warp per active point, the full FP32 row of the data
// (16-byte loads when rows are 16-byte aligned).
template <int NT, bool L1>
__device__ __forceinline__ void gather_exact(const AdaptiveArgs& a, int r, int nact, const float* qs,
                                             const int32_t* idc, float* Sc, uint32_t* hist) {
  const int m = a.m;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // two rows per warp at a time, their loads interleaved (each row's sum in
  // the same order as one row alone)
  for (int s0 = 2 * warp; s0 < nact; s0 += 2 * (NT / 32)) {
    const bool two = s0 + 1 < nact;
    const int ida = (r == 0) ? s0 : idc[s0];
    const int idb = two ? ((r == 0) ? s0 + 1 : idc[s0 + 1]) : ida;
    const float* xa = a.X + (size_t)ida * (size_t)m;
    const float* xb = a.X + (size_t)idb * (size_t)m;
    float pa = 0.0f, pb = 0.0f;
    if (a.vec) {
#pragma unroll 4
      for (int j = lane * 4; j < m; j += 128) {
        const float4 x4 = __ldg(reinterpret_cast<const float4*>(xa + j));
        const float4 y4 = __ldg(reinterpret_cast<const float4*>(xb + j));
        const float4 q4 = *reinterpret_cast<const float4*>(qs + j);
        pa = add_term<L1>(x4.x - q4.x, pa);
        pb = add_term<L1>(y4.x - q4.x, pb);
        pa = add_term<L1>(x4.y - q4.y, pa);
        pb = add_term<L1>(y4.y - q4.y, pb);
        pa = add_term<L1>(x4.z - q4.z, pa);
        pb = add_term<L1>(y4.z - q4.z, pb);
        pa = add_term<L1>(x4.w - q4.w, pa);
        pb = add_term<L1>(y4.w - q4.w, pb);
      }
    } else {
#pragma unroll 4
      for (int j = lane; j < m; j += 32) {
        const float qj = qs[j];
        pa = add_term<L1>(__ldg(xa + j) - qj, pa);
        pb = add_term<L1>(__ldg(xb + j) - qj, pb);
      }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      pa += __shfl_xor_sync(0xffffffffu, pa, o);
      pb += __shfl_xor_sync(0xffffffffu, pb, o);
    }
    if (lane == 0) {
      Sc[s0] = pa;
      atomicAdd(&hist[f2key(pa) >> 20], 1u);
      if (two) {
        Sc[s0 + 1] = pb;
        atomicAdd(&hist[f2key(pb) >> 20], 1u);
      }
    }
  }
}

// Row pass (per-pair draws over the FP32 data): a warp takes one active
// point at a time, reads its row once (its differences to the query go to
// shared memory) and forms the sums of the pass's rounds from it. A sampled round's sum is that of
// gather_sampled: virtual lane v of the round's G sums its blocks v, v + G,
// ... in turn (8 draws each, in draw order) and the G partial sums go through
// the same butterfly; an exact round's sum is that of gather_exact (lane
// order of its loads, then the full butterfly). The first round updates the
// running sums like a gather; round i > 0 goes to F[(i-1) cap + slot].
template <int NT, bool L1>
__device__ __forceinline__ void gather_fused(const AdaptiveArgs& a, const AdaptiveShared<NT>& sh, uint64_t qid, int nact,
                                          const float* qs, const int32_t* idc, float* Sc, float* Cc,
                                          uint32_t* hist, float* rows, float* F) {
  const int m = a.m;
  const int mpad = (m + 3) & ~3;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* row = rows + (size_t)warp * (size_t)(mpad + kFuseParts);
  float* P = row + mpad;
  const int nr = sh.f_nr;
  const int nsamp = sh.f_exact ? nr - 1 : nr;  // sampled rounds
  const int nunits = sh.f_uoff[nsamp];
  const uint64_t qfield = qid & a.mask_q;
  const int cap = a.fuse_cap;
  int id_next = warp < nact ? idc[warp] : 0;  // point ids one step ahead
  for (int s = warp; s < nact; s += NT / 32) {
    // the row's differences to the query, x_j - q_j (each draw then takes one
    // shared-memory read; the same FP32 subtraction every gather performs)
    const int id = id_next;
    if (s + NT / 32 < nact) id_next = idc[s + NT / 32];
    const float* xr = a.X + (size_t)id * (size_t)m;
    if (a.vec) {
      for (int j4 = lane; j4 < (m >> 2); j4 += 32) {
        const float4 x4 = ld_stream4(reinterpret_cast<const float4*>(xr) + j4);
        const float4 q4 = reinterpret_cast<const float4*>(qs)[j4];
        reinterpret_cast<float4*>(row)[j4] = make_float4(x4.x - q4.x, x4.y - q4.y, x4.z - q4.z, x4.w - q4.w);
      }
    } else {
      for (int j = lane; j < m; j += 32) row[j] = ld_stream(xr + j) - qs[j];
    }
    __syncwarp();
    const uint64_t pfield = (uint64_t)id & a.mask_p;
    for (int u = lane; u < nunits; u += 32) {
      const int4 ud = sh.f_unit[u];
      const int T = ud.x, Tn = ud.y, G = ud.z, v = ud.w;
      const int bhi = (Tn - 1) >> 3;
      float part = 0.0f;
      for (int b = (T >> 3) + v; b <= bhi; b += G) {
        const Draws8 ph = pair_draws8((uint32_t)b, pfield, qfield, a.rk);
        if (8 * b >= T && 8 * b + 8 <= Tn) {  // the whole block is in the round
#pragma unroll
          for (int w = 0; w < 8; ++w) part = add_term<L1>(row[__umulhi(philox_word(ph, w), (uint32_t)m)], part);
        } else {
#pragma unroll
          for (int w = 0; w < 8; ++w) {
            const int sv = 8 * b + w;
            if (sv >= T && sv < Tn) part = add_term<L1>(row[__umulhi(philox_word(ph, w), (uint32_t)m)], part);
          }
        }
      }
      P[u] = part;
    }
    __syncwarp();
    // every round's sum: lane v < G holds virtual lane v's partial of a sampled
    // round, every lane its share of the exact round; the butterflies of all
    // rounds run side by side (a round adds over offsets below its G only)
    float x[kFuseRounds];
    int Gr[kFuseRounds];
#pragma unroll
    for (int i = 0; i < kFuseRounds; ++i) {
      x[i] = 0.0f;
      Gr[i] = 0;
      if (i < nsamp) {
        Gr[i] = sh.f_uoff[i + 1] - sh.f_uoff[i];
        if (lane < Gr[i]) x[i] = P[sh.f_uoff[i] + lane];
      } else if (i == nsamp && i < nr) {  // the exact round
        Gr[i] = 32;
        float e = 0.0f;
        if (a.vec) {
          for (int j = lane * 4; j < m; j += 128) {
            const float4 d4 = *reinterpret_cast<const float4*>(row + j);
            e = add_term<L1>(d4.x, e);
            e = add_term<L1>(d4.y, e);
            e = add_term<L1>(d4.z, e);
            e = add_term<L1>(d4.w, e);
          }
        } else {
          for (int j = lane; j < m; j += 32) e = add_term<L1>(row[j], e);
        }
        x[i] = e;
      }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
#pragma unroll
      for (int i = 0; i < kFuseRounds; ++i) {
        if (i < nr) {
          const float y = __shfl_xor_sync(0xffffffffu, x[i], o);
          if (o < Gr[i]) x[i] += y;
        }
      }
    }
    if (lane == 0) {
      {  // this round: Kahan-compensated running sum, as a gather updates it
        const float S0 = Sc[s], c0 = Cc[s];
        const float y = x[0] - c0;
        const float tt = S0 + y;
        Cc[s] = (tt - S0) - y;
        Sc[s] = tt;
        atomicAdd(&hist[f2key(tt) >> 20], 1u);
      }
#pragma unroll
      for (int i = 1; i < kFuseRounds; ++i)
        if (i < nr) F[(size_t)(i - 1) * (size_t)cap + s] = x[i];
    }
    __syncwarp();
  }
}

// A round whose sums a row pass formed (read through each slot's pass slot):
// the running sums take them as a gather would (exact rounds replace them).
template <int NT>
__device__ __forceinline__ void gather_from_pass(int nact, bool exact, const float* Fc, const int32_t* fslot,
                                                 float* Sc, float* Cc, uint32_t* hist) {
  for (int s = threadIdx.x; s < nact; s += NT) {
    const float x = Fc[fslot[s]];
    float S;
    if (exact) {
      S = x;
    } else {
      const float S0 = Sc[s], c0 = Cc[s];
      const float y = x - c0;
      S = S0 + y;
      Cc[s] = (S - S0) - y;
    }
    Sc[s] = S;
    atomicAdd(&hist[f2key(S) >> 20], 1u);
  }
}

// Round 0 from the point-major pass, with tile minima. tau_U' = (k-th
// smallest tile minimum)/T + w is at least tau_U (the k smallest tile minima
// are sums of k distinct points), so a point whose LCB exceeds tau_U' is
// eliminated whatever the other sums are. One streaming pass drops those
// points (logged; their smallest LCB joins min_elim) and keeps the others in
// index order (idA/SA); the round then runs on the kept points alone. The k
// smallest sums are always kept, so tau_U is unchanged, and the (k+1)-th
// smallest LCB over all points is the smaller of the kept points' (k+1)-th
// and the dropped points' smallest. hist holds zeros on entry and the level-1
// counts of the kept keys on exit; stI/stS are staging space of n entries.
template <int NT>
__device__ int round0_filter(const AdaptiveArgs& a, int q, int64_t n, int k, float w, float Tf, uint32_t* hist,
                             uint32_t* buf, AdaptiveShared<NT>& sh, int32_t* idA, float* SA, int32_t* stI,
                             float* stS, int32_t* lcode, float* lS, float* min_elim) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float* mq = a.R0min + (size_t)q * (size_t)a.r0tiles;
  const int nt = a.r0tiles;
  for (int i = tid; i < nt; i += NT) atomicAdd(&hist[f2key(mq[i]) >> 20], 1u);
  __syncthreads();
  select_smallest<NT>([&](int i) { return f2key(mq[i]); }, nt, k, hist, buf, sh.ss, sh.bs);
  const float tU = key2f(buf[k - 1]) / Tf + w;  // the UCB of that sum, formed as the thresholds form it
  // The LCB fl(fl(S / T) - w) does not decrease with S, so the dropped sums
  // are those above one float Sc: found once by bisection on the bit
  // patterns of non-negative floats, it turns the test into one comparison.
  uint32_t lo = 0u, hi = 0x7F800000u;  // L(0) <= tU (kept), L(+inf) > tU (dropped)
  while (hi - lo > 1u) {
    const uint32_t mid = lo + ((hi - lo) >> 1);
    if (__uint_as_float(mid) / Tf - w > tU) hi = mid; else lo = mid;
  }
  const float Sc = __uint_as_float(lo);
  for (int i = tid; i < kHistBins; i += NT) hist[i] = 0;
  __syncthreads();
  // warp w scans its own contiguous segment, several loads in flight per
  // lane; the kept points are staged in index order (ballots or a warp scan
  // inside the warp, the warps' counts across them)
  constexpr int U = 8;
  constexpr int NW = NT / 32;
  const float* R0q = a.R0 + (size_t)q * (size_t)n;
  // 16-byte loads when the rows of sums are 16-byte aligned: segments of a
  // multiple of 128 sums, four per lane and load, U4 loads in flight
  const bool vec4 = (n & 3) == 0 && ((reinterpret_cast<uintptr_t>(a.R0) & 15) == 0);
  const int64_t seg = vec4 ? ((n + NW - 1) / NW + 127) & ~(int64_t)127 : ((n + NW - 1) / NW + 31) & ~(int64_t)31;
  const int64_t s0 = (int64_t)warp * seg, s1 = min(n, s0 + seg);
  int cnt = 0;
  float mn = INFINITY;  // smallest dropped sum
  auto drop = [&](int64_t i, float v) {  // LCB > tU
    mn = fminf(mn, v);
    if (lcode) {
      lcode[i] = 1;  // eliminated in round 0
      if (lS) lS[i] = v;
    }
  };
  if (vec4) {
    constexpr int U4 = 4;
    for (int64_t base = s0; base < s1; base += 128 * U4) {
      float4 v[U4];
#pragma unroll
      for (int u = 0; u < U4; ++u) {
        const int64_t i = base + u * 128 + 4 * lane;  // s1 is a multiple of 4: a float4 is in or out
        v[u] = i < s1 ? __ldcs(reinterpret_cast<const float4*>(R0q + i)) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < U4; ++u) {
        const int64_t i = base + u * 128 + 4 * lane;
        const float vv[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
        uint32_t km = 0;
        if (i < s1) {
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            if (vv[c] > Sc) drop(i + c, vv[c]); else km |= 1u << c;
          }
        }
        // kept sums of lower lanes come first (index order: lane, then c)
        const int kc = __popc(km);
        int incl = kc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int t = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += t;
        }
        int pos = cnt + incl - kc;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          if (km & (1u << c)) {
            stI[s0 + pos] = (int32_t)(i + c);
            stS[s0 + pos] = vv[c];
            atomicAdd(&hist[f2key(vv[c]) >> 20], 1u);
            ++pos;
          }
        }
        cnt += __shfl_sync(0xffffffffu, incl, 31);
      }
    }
  } else {
    for (int64_t base = s0; base < s1; base += 32 * U) {
      float v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t i = base + u * 32 + lane;
        v[u] = i < s1 ? __ldcs(R0q + i) : 0.0f;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t i = base + u * 32 + lane;
        bool keep = false;
        if (i < s1) {
          if (v[u] > Sc) drop(i, v[u]); else keep = true;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (keep) {
          const int pos = cnt + __popc(bal & ((1u << lane) - 1u));
          stI[s0 + pos] = (int32_t)i;
          stS[s0 + pos] = v[u];
          atomicAdd(&hist[f2key(v[u]) >> 20], 1u);
        }
        cnt += __popc(bal);
      }
    }
  }
  int total;
  const int off = block_exclusive_scan<NT>(lane == 0 ? cnt : 0, sh.bs, &total);  // barriers order the staging
  const int woff = __shfl_sync(0xffffffffu, off, 0);
  for (int t = lane; t < cnt; t += 32) {
    idA[woff + t] = stI[s0 + t];
    SA[woff + t] = stS[s0 + t];
  }
  mn = block_min<NT>(mn, sh.bs);
  if (mn < INFINITY) *min_elim = fminf(*min_elim, mn / Tf - w);  // the smallest dropped LCB
  return total;
}

template <int NT, class E, bool L1>
__global__ void __launch_bounds__(NT, 1024 / NT) adaptive_rounds_kernel(AdaptiveArgs a) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  __shared__ AdaptiveShared<NT> sh;
  const int m = a.m;
  const int mpad = (m + 3) & ~3;
  float* qs = reinterpret_cast<float*>(smem_raw);
  uint32_t* hist = reinterpret_cast<uint32_t*>(qs + mpad);
  uint32_t* buf = hist + kHistBins;
  float* actU = reinterpret_cast<float*>(buf + kSelCap);
  float* actL = actU + (kMaxKH + 4);
  int32_t* oid = reinterpret_cast<int32_t*>(actL + (kMaxKH + 4));
  float* qsp = reinterpret_cast<float*>(oid + kMaxKH);  // permuted query (shared coordinates only)
  float* frows = qsp + (E::kPerm ? ((m + 7) & ~7) : 0);  // row passes: a row and partials per warp
  constexpr bool kRowPass = std::is_same<E, ElemF32>::value;
  float* tmpS = actU;                              // reused in the output phase
  int32_t* tmpI = reinterpret_cast<int32_t*>(actL);

  const int tid = threadIdx.x;
  const int64_t n = a.n;
  const size_t slot = blockIdx.x;
  // ping-pong halves: buffer b of this CTA starts at base + b * n
  int32_t* const ids0 = a.ws_ids + slot * 2 * (size_t)n;
  float* const S0 = a.ws_S + slot * 2 * (size_t)n;
  float* const C0 = a.ws_C + slot * 2 * (size_t)n;
  int32_t* acc_id = a.ws_acc_id + slot * (size_t)a.acc_cap;
  float* acc_d = a.ws_acc_d + slot * (size_t)a.acc_cap;
  float* acc_U = a.ws_acc_U + slot * (size_t)a.acc_cap;
  float* acc_L = a.ws_acc_L + slot * (size_t)a.acc_cap;
  // row passes: sums of later rounds per active slot, ping-pong like the slots
  // row passes: round c's sums by pass slot (the slot a point had in the pass
  // round), and each active slot's pass slot, ping-pong like the slots
  float* const F0 = a.ws_F ? a.ws_F + slot * (kFuseRounds + 2) * (size_t)a.fuse_cap : nullptr;
  auto Fcol = [&](int c) { return F0 + (size_t)c * (size_t)a.fuse_cap; };
  auto Fslot = [&](int b) { return reinterpret_cast<int32_t*>(F0 + (size_t)(kFuseRounds + b) * (size_t)a.fuse_cap); };
  KNN_PHASE_START;

  for (;;) {
    if (tid == 0) sh.q = atomicAdd(a.queue, 1);
    __syncthreads();
    if (sh.q >= a.nq) break;
    const int q = a.qorder ? a.qorder[sh.q] : sh.q;
    // this query's k, h and counter id (a mixed batch gives each query its own)
    const int k = a.kq ? max(1, min(a.kq[q], a.k)) : a.k;
    const int kh = k + (a.h_per_k ? k : a.h);
    const uint64_t qid = a.qids ? a.qids[q] : a.qid_base + (uint64_t)q;
    const int stride = a.out_stride;
    int64_t* oidx = a.out_idx + (size_t)q * stride;
    int32_t* lcode = a.log_code ? a.log_code + (size_t)q * (size_t)n : nullptr;
    float* lS = a.log_S ? a.log_S + (size_t)q * (size_t)n : nullptr;

    // ---- query row into shared memory; span of the normalisation (Section 3)
    const float* qr = a.Q + (size_t)q * m;
    float qmin = FLT_MAX, qmax = -FLT_MAX;
    int bad = 0;
    for (int j = tid; j < m; j += NT) {
      const float v = qr[j];
      qs[j] = v;
      bad |= !isfinite(v);
      qmin = fminf(qmin, v);
      qmax = fmaxf(qmax, v);
    }
    for (int j = m + tid; j < mpad; j += NT) qs[j] = 0.0f;
    bad = __syncthreads_or(bad);
    if constexpr (E::kPerm) {
      for (int t = tid; t < a.mp; t += NT) qsp[t] = t < m ? qs[a.jperm[t]] : 0.0f;
      __syncthreads();
    }
    qmin = block_min<NT>(qmin, sh.bs);
    qmax = block_max<NT>(qmax, sh.bs);
    const float xmin = key2f(a.xrange[0]), xmax = key2f(a.xrange[1]);
    bad |= a.xrange[2] != 0u;  // non-finite data (flagged by the range pass)
    const float span = fmaxf(xmax, qmax) - fminf(xmin, qmin);
    // A stored copy moves each sample by at most e (2 span + e), e its largest
    // element error: the copy's samples lie in [0, (span + 2e)^2] and its
    // distances within eps of the data's, so the width of sampled bounds
    // grows by eps. Exact rounds read the FP32 data and keep width 0.
    // (l1: a sample |x - q| lies in [0, span], normalised by span; a copy
    // moves it by at most e, within [0, span + e])
    float spanw = span, eps = 0.0f, ecopy = 0.0f;
    if (E::kStorage != KNN_STORE_F32) {
      const float e = *a.emax;
      ecopy = e;
      spanw = a.l1 ? span + e : span + 2.0f * e;
      eps = a.l1 ? e : e * (2.0f * span + e);
    }
    const float span2 = a.l1 ? spanw : spanw * spanw;
    if (bad || !isfinite(span2)) {
      for (int t = tid; t < stride; t += NT) oidx[t] = -1;
      if (tid == 0) {
        a.out_count[q] = 0;
        a.out_evals[q] = 0;
        if (a.out_rounds) a.out_rounds[q] = 0;
      }
      __syncthreads();
      continue;
    }
    if (n <= kh) {  // every point is a candidate
      for (int t = tid; t < stride; t += NT) oidx[t] = t < n ? t : -1;
      if (lcode)
        for (int64_t i = tid; i < n; i += NT) {
          lcode[i] = 0;
          if (lS) lS[i] = 0.0f;
        }
      if (tid == 0) {
        a.out_count[q] = (int32_t)n;
        a.out_evals[q] = 0;
        if (a.out_rounds) a.out_rounds[q] = 0;
      }
      __syncthreads();
      continue;
    }

    int nact = (int)n, nacc = 0, cur = 0, r = 0, term = 0;
    int fcols = 0, fnext = 0, nact_prev = 0;  // rounds held in F, the next one's column; active points at
                                               // the previous round's start
    int64_t T = 0, evals = 0;
    float min_elim = INFINITY;
    for (;;) {
      const int64_t Br = (r == 0) ? a.B0 : (a.grow ? (T > a.B ? T : (int64_t)a.B) : (int64_t)a.B);
      const bool exact = T + Br >= a.Mb;  // Mb = m for single coordinates
      const int64_t Tn = exact ? a.Mb : T + Br;
      const int32_t* idc = ids0 + (size_t)cur * n;
      const bool pre = (r == 0) && a.R0 && !exact;  // round-0 sums computed point-major beforehand
      // with tile minima, round 0 first drops the points they already prove eliminated
      const bool flt = pre && a.R0min && a.r0tiles >= k;
      float* Sc = pre && !flt ? const_cast<float*>(a.R0) + (size_t)q * (size_t)n : S0 + (size_t)cur * n;
      float* Cc = C0 + (size_t)cur * n;
      evals += (int64_t)nact * (exact ? (int64_t)m : Br * a.g);
      float w = exact ? 0.0f : span2 * alpha_of(a, Tn) + eps;
      const float Tf = (float)(Tn * a.g);  // estimate = S / (T g): mean per coordinate
      // A copy's term shrinks to e (2 sqrt(d_max) + e), d_max the largest
      // estimate among the points this round decides: a copy moves a sample by
      // at most e (2 |x~ - q| + e), and the mean of |x~ - q| is at most the
      // square root of the mean of (x~ - q)^2.
      const bool shrink = !L1 && E::kStorage != KNN_STORE_F32 && !exact && ecopy > 0.0f;
      auto copy_width = [&](float mx) {
        const float e2 = ecopy * (2.0f * sqrtf(mx / Tf) + ecopy);
        if (e2 < eps) w = span2 * alpha_of(a, Tn) + e2;
      };
      if (flt && shrink) {  // the filter needs the width first: d_max over every round-0 sum
        const float* R0q = a.R0 + (size_t)q * (size_t)n;
        float mx = 0.0f;
        for (int64_t i = tid; i < n; i += NT) mx = fmaxf(mx, R0q[i]);
        copy_width(block_max<NT>(mx, sh.bs));
      }
      // a row pass from this round: after a round that kept at least 3/4 of its
      // points, or for a round drawing m/8 coordinates or more per point
      bool fuse_now = false;
      if constexpr (kRowPass) {
        fuse_now = a.fuse_cap > 0 && fcols == 0 && r >= 1 && !exact && nact <= a.fuse_cap && a.G == a.X &&
                   ((r >= 2 && 4 * (int64_t)nact >= 3 * (int64_t)nact_prev) || 8 * Br >= m);
        if (fuse_now && tid == 0) {
          int64_t Ti = T;
          int nr = 0, u = 0, ex = 0;
          sh.f_uoff[0] = 0;
          while (nr < kFuseRounds) {
            const int64_t Bi = a.grow ? (Ti > a.B ? Ti : (int64_t)a.B) : (int64_t)a.B;
            const bool xi = Ti + Bi >= a.Mb;
            const int64_t Tni = xi ? a.Mb : Ti + Bi;
            sh.f_T[nr] = (int)Ti;
            sh.f_Tn[nr] = (int)Tni;
            if (!xi) {
              const int nb = (int)(((Tni - 1) >> 3) - (Ti >> 3) + 1);
              int G = 1;
              while (G < nb && G < 32) G <<= 1;
              for (int v = 0; v < G; ++v) sh.f_unit[u + v] = make_int4((int)Ti, (int)Tni, G, v);
              u += G;
            }
            sh.f_uoff[++nr] = u;
            Ti = Tni;
            if (xi) {
              ex = 1;
              break;
            }
          }
          sh.f_nr = nr;
          sh.f_exact = ex;
        }
      }
      for (int i = tid; i < kHistBins; i += NT) hist[i] = 0;
      __syncthreads();
      KNN_PHASE(0);  // setup
      // slots' sums of later rounds to carry through this round's compaction
      // a pass slot to carry through this round's compaction: the pass round
      // gives each slot its own; later rounds carry them while F holds rounds
      const int fcarry = fuse_now ? 1 : (fcols > 1 ? 2 : 0);
      if (flt) {
        nact = round0_filter<NT>(a, q, n, k, w, Tf, hist, buf, sh, ids0 + (size_t)cur * n, Sc,
                                 ids0 + (size_t)(cur ^ 1) * n, S0 + (size_t)(cur ^ 1) * n, lcode, lS, &min_elim);
        if constexpr (E::kPerm) {
          if (a.r0_resum) {
            // the contraction's sums only chose the points the filter keeps:
            // their sums again, sample by sample, before the round's decisions
            for (int i = tid; i < kHistBins; i += NT) hist[i] = 0;
            __syncthreads();
            gather_sampled<NT, E, L1>(a, qid, 0, nact, 0, Tn, qsp, idc, Sc, Cc, hist, true);
          }
        }
      }
      else if (kRowPass && fcols > 0)  // a row pass formed this round's sums
        gather_from_pass<NT>(nact, exact, Fcol(fnext), Fslot(cur), Sc, Cc, hist);
      else if (kRowPass && fuse_now)
        gather_fused<NT, L1>(a, sh, qid, nact, qs, idc, Sc, Cc, hist, frows, Fcol(0));
      else if (exact)  // the exact cap reads the FP32 data whatever copy the samples use
        gather_exact<NT, L1>(a, r, nact, qs, idc, Sc, hist);
      else if (pre)
        for (int i = tid; i < nact; i += NT) atomicAdd(&hist[f2key(Sc[i]) >> 20], 1u);
      else if constexpr (E::kBlk)
        gather_blocks<NT, E, L1>(a, qid, r, nact, T, Tn, qs, idc, Sc, Cc, hist);
      else
        gather_sampled<NT, E, L1>(a, qid, r, nact, T, Tn, E::kPerm ? qsp : qs, idc, Sc, Cc, hist);
      __syncthreads();
      if (exact) KNN_PHASE(2); else KNN_PHASE(1);  // exact rows / sampled gathers (round 0: the filter)
      const bool ident = (r == 0) && !flt;  // slot s holds point s
      if (shrink && !flt) {  // every point of the round has its sum in Sc
        float mx = 0.0f;
        for (int i = tid; i < nact; i += NT) mx = fmaxf(mx, Sc[i]);
        copy_width(block_max<NT>(mx, sh.bs));
      }

      // ---- thresholds
      const int kk = min(k + 1, nact);
      select_smallest<NT>([&](int i) { return f2key(Sc[i]); }, nact, kk, hist, buf, sh.ss, sh.bs);
      for (int j = tid; j < kk; j += NT) {
        const float d = key2f(buf[j]) / Tf;
        actU[j] = d + w;
        actL[j] = d - w;
      }
      if (tid == 0) sh.nacc_add = 0;
      __syncthreads();
      KNN_PHASE(3);  // select
      const float tauU = kth_of_union<NT>(actU, min(k, nact), acc_U, nacc, k, &sh.tauU);
      // (after the round-0 filter the kept points can number k: the (k+1)-th
      // smallest LCB is then that of a dropped point, min_elim)
      const float tauL = nact + nacc > k ? fminf(kth_of_union<NT>(actL, kk, acc_L, nacc, k + 1, &sh.tauL), min_elim)
                                         : min_elim;

      KNN_PHASE(4);  // thresholds
      // ---- decide + compact (order-preserving)
      int32_t* idn = ids0 + (size_t)(cur ^ 1) * n;
      float* Sn = S0 + (size_t)(cur ^ 1) * n;
      float* Cn = C0 + (size_t)(cur ^ 1) * n;
      float rmin = INFINITY;
      int out_base = 0;
      for (int cb = 0; cb < nact; cb += NT * kIPT) {
        int myid[kIPT];
        float myS[kIPT], myC[kIPT];
        bool keep[kIPT];
        int cnt = 0;
#pragma unroll
        for (int e = 0; e < kIPT; ++e) {
          const int s = cb + tid * kIPT + e;
          keep[e] = false;
          myid[e] = 0;
          myS[e] = 0.0f;
          myC[e] = 0.0f;
          if (s < nact) {
            const int id = ident ? s : idc[s];
            const float S = Sc[s];
            const float c = (r == 0 || exact) ? 0.0f : Cc[s];
            const float d = S / Tf;
            const float U = d + w, L = d - w;
            if (L > tauU) {
              rmin = fminf(rmin, L);
              if (lcode) {
                lcode[id] = 4 * r + 1;
                if (lS) lS[id] = S;
              }
            } else if (U < tauL) {
              const int sl = nacc + atomicAdd(&sh.nacc_add, 1);
              if (sl < a.acc_cap) {
                acc_id[sl] = id;
                acc_d[sl] = d;
                acc_U[sl] = U;
                acc_L[sl] = L;
              }
              if (lcode) {
                lcode[id] = 4 * r + 2;
                if (lS) lS[id] = S;
              }
            } else {
              keep[e] = true;
              ++cnt;
            }
            myid[e] = id;
            myS[e] = S;
            myC[e] = c;
          }
        }
        int total;
        int pos = out_base + block_exclusive_scan<NT>(cnt, sh.bs, &total);
#pragma unroll
        for (int e = 0; e < kIPT; ++e) {
          if (keep[e]) {
            idn[pos] = myid[e];
            Sn[pos] = myS[e];
            Cn[pos] = myC[e];
            if constexpr (kRowPass) {
              if (fcarry) {
                const int sl = cb + tid * kIPT + e;
                Fslot(cur ^ 1)[pos] = fcarry == 1 ? sl : Fslot(cur)[sl];
              }
            }
            ++pos;
          }
        }
        out_base += total;
      }
      rmin = block_min<NT>(rmin, sh.bs);  // also orders sh.nacc_add
      KNN_PHASE(5);  // decide + compact
      nacc = min(nacc + sh.nacc_add, a.acc_cap);
      nact_prev = nact;
      nact = out_base;
      if (fuse_now) {
        fcols = sh.f_nr - 1;
        fnext = 0;
      } else if (fcols > 0) {
        --fcols;
        ++fnext;
      }
      min_elim = fminf(min_elim, rmin);
      T = Tn;
      cur ^= 1;
      if (nact + nacc <= kh) term = 1;
      else if (nacc >= k) term = 2;
      else if (exact) term = 3;
      if (term) break;
      ++r;
      __syncthreads();
    }

    // ---- output: accepted by (estimate, index), then active by (estimate, index)
    const int32_t* idf = ids0 + (size_t)cur * n;
    const float* Sf = S0 + (size_t)cur * n;
    const int nacc_o = min(nacc, kh);
    const int rem = kh - nacc_o;
    const int nact_o = min(nact, rem);
    for (int i = tid; i < nacc; i += NT) {
      const float di = acc_d[i];
      const int ii = acc_id[i];
      int rank = 0;
      for (int j = 0; j < nacc; ++j) {
        const float dj = acc_d[j];
        rank += (dj < di) || (dj == di && acc_id[j] < ii);
      }
      if (rank < kh) oid[rank] = ii;
    }
    if (nact_o > 0) {
      if (nact <= rem) {
        for (int i = tid; i < nact; i += NT) {
          tmpS[i] = Sf[i];
          tmpI[i] = idf[i];
        }
      } else {
        for (int i = tid; i < kHistBins; i += NT) hist[i] = 0;
        __syncthreads();
        for (int i = tid; i < nact; i += NT) atomicAdd(&hist[f2key(Sf[i]) >> 20], 1u);
        __syncthreads();
        select_smallest<NT>([&](int i) { return f2key(Sf[i]); }, nact, rem, hist, buf, sh.ss, sh.bs);
        const uint32_t kstar = buf[rem - 1];
        int nless = 0;  // keys of buf below kstar (buf is ascending)
        {
          int lo = 0, hi = rem;
          while (lo < hi) {
            int mid = (lo + hi) >> 1;
            if (buf[mid] < kstar) lo = mid + 1; else hi = mid;
          }
          nless = lo;
        }
        const int need_ties = rem - nless;
        if (tid == 0) sh.ss.cnt = 0;
        __syncthreads();
        int tie_base = 0;
        for (int cb = 0; cb < nact; cb += NT) {
          const int s = cb + tid;
          uint32_t key = 0xFFFFFFFFu;
          if (s < nact) key = f2key(Sf[s]);
          const bool less = s < nact && key < kstar;
          const bool tie = s < nact && key == kstar;
          if (less) {
            const int p = atomicAdd(&sh.ss.cnt, 1);
            tmpS[p] = Sf[s];
            tmpI[p] = idf[s];
          }
          int total;
          const int tr = tie_base + block_exclusive_scan<NT>(tie ? 1 : 0, sh.bs, &total);
          if (tie && tr < need_ties) {
            tmpS[nless + tr] = Sf[s];
            tmpI[nless + tr] = idf[s];
          }
          tie_base += total;
        }
      }
      __syncthreads();
      for (int i = tid; i < nact_o; i += NT) {
        const float si = tmpS[i];
        const int ii = tmpI[i];
        int rank = 0;
        for (int j = 0; j < nact_o; ++j) {
          const float sj = tmpS[j];
          rank += (sj < si) || (sj == si && tmpI[j] < ii);
        }
        oid[nacc_o + rank] = ii;
      }
    }
    __syncthreads();
    const int count = nacc_o + nact_o;
    for (int t = tid; t < stride; t += NT) oidx[t] = t < count ? (int64_t)oid[t] : -1;
    if (lcode)
      for (int i = tid; i < nact; i += NT) {
        lcode[idf[i]] = 4 * r + 0;
        if (lS) lS[idf[i]] = Sf[i];
      }
    KNN_PHASE_SYNC(6);  // output
    if (tid == 0) {
      a.out_count[q] = count;
      a.out_evals[q] = evals;
      if (a.out_rounds) a.out_rounds[q] = r + 1;
    }
    __syncthreads();
  }
}

// ---- locality order of a batch's queries
// Queries close to one another keep most of the same points active after
// round 0, so running them at the same time lets those rows stay in L2. The
// key is a SimHash of the query: the signs of 16 projections of the query
// minus the batch's mean onto fixed +-1 directions (bit of a hash of
// (direction, column)); ties by index. Only the schedule changes: a query's
// draws, decisions and result depend on its id, not on when it runs.
constexpr int kOrderMax = 16384;  // queries ordered at once (larger chunks keep the batch order)

// Column sums of the batch (mean zeroed first): 32 slices of rows in parallel.
static __global__ void query_mean_kernel(const float* __restrict__ Q, int nq, int m, float* __restrict__ mean) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  float s = 0.0f;
  for (int q = blockIdx.y; q < nq; q += gridDim.y) s += __ldg(Q + (size_t)q * m + j);
  atomicAdd(&mean[j], s);
}

static __global__ void query_code_kernel(const float* __restrict__ Q, int nq, int m, const float* __restrict__ mean,
                                         uint64_t* __restrict__ keys) {
  const int q = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (q >= nq) return;
  const float inv_nq = 1.0f / (float)nq;
  float acc[16];
#pragma unroll
  for (int b = 0; b < 16; ++b) acc[b] = 0.0f;
  for (int j = lane; j < m; j += 32) {
    const float v = __ldg(Q + (size_t)q * m + j) - mean[j] * inv_nq;
    const uint32_t h = fmix32((uint32_t)j * 0x9E3779B9u + 0x7F4A7C15u);
#pragma unroll
    for (int b = 0; b < 16; ++b) acc[b] += ((h >> b) & 1u) ? v : -v;
  }
  uint32_t code = 0;
#pragma unroll
  for (int b = 0; b < 16; ++b) {
    float t = acc[b];
#pragma unroll
    for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    code |= (t > 0.0f ? 1u : 0u) << b;
  }
  if (lane == 0) keys[q] = ((uint64_t)code << 32) | (uint32_t)q;
}

// One CTA: bitonic sort of the keys in shared memory, the query order out.
static __global__ void __launch_bounds__(1024) query_order_kernel(const uint64_t* __restrict__ keys, int nq,
                                                                   int32_t* __restrict__ order) {
  extern __shared__ uint64_t sk[];
  int P = 2;
  while (P < nq) P <<= 1;
  for (int i = threadIdx.x; i < P; i += blockDim.x) sk[i] = i < nq ? keys[i] : ~0ull;
  __syncthreads();
  for (int size = 2; size <= P; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < (P >> 1); i += blockDim.x) {
        const int lo = 2 * i - (i & (stride - 1)), hi = lo + stride;
        const bool up = (lo & size) == 0;
        const uint64_t a = sk[lo], b = sk[hi];
        if ((b < a) == up) {
          sk[lo] = b;
          sk[hi] = a;
        }
      }
      __syncthreads();
    }
  for (int i = threadIdx.x; i < nq; i += blockDim.x) order[i] = (int32_t)(uint32_t)sk[i];
}

static inline size_t query_order_scratch(int32_t m, int32_t nq) {
  return ((size_t)m * 4 + 255) / 256 * 256 + ((size_t)nq * 8 + 255) / 256 * 256 + ((size_t)nq * 4 + 255) / 256 * 256;
}

// The chunk's order into `order` (nq entries) from scratch of query_order_scratch bytes.
static inline knn_status launch_query_order(const float* Q, int nq, int m, uint8_t* scratch, int32_t* order,
                                            cudaStream_t stream) {
  float* mean = reinterpret_cast<float*>(scratch);
  uint64_t* keys = reinterpret_cast<uint64_t*>(scratch + ((size_t)m * 4 + 255) / 256 * 256);
  knn_status s0 = cuda_check(cudaMemsetAsync(mean, 0, (size_t)m * 4, stream), "memset(query mean)");
  if (s0 != KNN_OK) return s0;
  query_mean_kernel<<<dim3((m + 255) / 256, 32), 256, 0, stream>>>(Q, nq, m, mean);
  query_code_kernel<<<(nq * 32 + 255) / 256, 256, 0, stream>>>(Q, nq, m, mean, keys);
  int P = 2;
  while (P < nq) P <<= 1;
  const size_t smem = (size_t)P * 8;
  knn_status s = cuda_check(
      cudaFuncSetAttribute(query_order_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
      "cudaFuncSetAttribute(query order)");
  if (s != KNN_OK) return s;
  query_order_kernel<<<1, 1024, smem, stream>>>(keys, nq, order);
  return cuda_check(cudaGetLastError(), "query order kernels");
}

// Round 0 for every query of a batch, point-major: a CTA stages a tile of
// rows of the gathered copy in shared memory (dequantised to FP32) and
// computes the round-0 sums of all queries for those rows, so the copy
// streams from DRAM once per batch instead of being sampled at random per
// query. Draws, lane grouping (G lanes per point, one block of 8 draws each)
// and the shuffle reduction are those of gather_sampled, so the sums are the
// same bit for bit. Needs B0 <= 256 (at most 32 blocks).
constexpr int kR0Threads = 1024;
constexpr int kR0MaxRows = 32;
constexpr size_t kR0SmemBudget = 110 * 1024;

// Rows a CTA stages: as many as 110 KB hold, at most 32; with round-0 blocks
// spread over two or more lanes per point (B0 > 8: warp steps of 16 points or
// fewer) 48 rows where they fit in 150 KB, so each query row fetched into L1
// serves more pairs (measured 2.12 -> 2.01 ms at B0 = 16, m = 784; 48 rows
// would leave a half-empty step at B0 <= 8).
constexpr int kR0WideRows = 48;
constexpr size_t kR0WideBudget = 150 * 1024;

static inline int round0_rows(int m, int B0) {
  if (B0 > 8 && (size_t)kR0WideRows * (size_t)m * 4 <= kR0WideBudget) return kR0WideRows;
  const int r = (int)(kR0SmemBudget / ((size_t)m * 4));
  return r < 1 ? 1 : (r > kR0MaxRows ? kR0MaxRows : r);
}

template <class E, bool L1>
__global__ void __launch_bounds__(kR0Threads) round0_kernel(AdaptiveArgs a, int rows_per_cta, float* R0,
                                                            float* R0min) {
  extern __shared__ __align__(16) float rows[];
  using Tp = typename E::T;
  const int m = a.m;
  const int64_t n = a.n;
  const int64_t p0 = (int64_t)blockIdx.x * rows_per_cta;
  const int np = (int)((n - p0) < rows_per_cta ? (n - p0) : rows_per_cta);
  const Tp* G0 = static_cast<const Tp*>(a.G);
  if constexpr (std::is_same<Tp, float>::value && !E::kScaled) {
    // the tile's rows are one contiguous run of the data, read once
    const float* src = static_cast<const float*>(a.G) + (size_t)p0 * m;
    const int cnt = np * m;
    if (a.vec) {  // m % 4 == 0 and 16-byte aligned rows
      for (int e = threadIdx.x; e < (cnt >> 2); e += kR0Threads)
        reinterpret_cast<float4*>(rows)[e] = ld_stream4(reinterpret_cast<const float4*>(src) + e);
    } else {
      for (int e = threadIdx.x; e < cnt; e += kR0Threads) rows[e] = ld_stream(src + e);
    }
  } else {
    for (int e = threadIdx.x; e < np * m; e += kR0Threads) {
      const int pi = e / m, j = e - pi * m;
      const float x = E::load(G0 + (size_t)(p0 + pi) * m + j);
      rows[e] = E::kScaled ? __fmul_rn(x, __ldg(a.gscale + p0 + pi)) : x;
    }
  }
  __syncthreads();
  const int nblk = (a.B0 + 7) >> 3;
  int G = 1;
  while (G < nblk && G < 32) G <<= 1;
  const int lg = __ffs(G) - 1;
  const int ppw = 32 >> lg;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane >> lg, gl = lane & (G - 1);
  for (int q = warp; q < a.nq; q += kR0Threads / 32) {
    const uint64_t qid = a.qids ? a.qids[q] : a.qid_base + (uint64_t)q;
    const uint64_t qfield = qid & a.mask_q;
    const float* qr = a.Q + (size_t)q * m;
    float tmin = INFINITY;  // smallest sum of this CTA's rows for query q
    for (int base = 0; base < np; base += ppw) {
      const int pi = base + grp;
      float part = 0.0f;
      if (pi < np && gl < nblk) {
        const uint64_t id = (uint64_t)(p0 + pi);
        const Draws8 ph = pair_draws8(E::kWor ? kWorKeyItem : (uint32_t)gl, id & a.mask_p, qfield, a.rk);
        const float* xr = rows + (size_t)pi * m;
        if constexpr (!E::kBlk) {
          if (!E::kWor && gl * 8 + 8 <= a.B0) {  // the whole block is in round 0
#pragma unroll
            for (int w = 0; w < 8; ++w) {
              const int j = (int)__umulhi(philox_word(ph, w), (uint32_t)m);
              part = add_term<L1>(xr[j] - __ldg(qr + j), part);
            }
          } else {
#pragma unroll
            for (int w = 0; w < 8; ++w) {
              if (gl * 8 + w < a.B0) {  // B0 < m: the draw index is below m
                const int j = E::kWor ? wor_coordinate(ph, (uint32_t)(gl * 8 + w), (uint32_t)m, a.wor_h)
                                      : (int)__umulhi(philox_word(ph, w), (uint32_t)m);
                const float d = xr[j] - __ldg(qr + j);
                part = add_term<L1>(d, part);
              }
            }
          }
        } else {  // block samples, in gather_blocks' order
          const bool vec4 = a.qvec && (a.g & 3) == 0;  // staged rows and query rows 16-byte aligned
          for (int w = 0; w < 8; ++w) {
            if (gl * 8 + w < a.B0) {
              const int c0 = (int)__umulhi(philox_word(ph, w), (uint32_t)a.Mb) * a.g;
              const int c1 = min(c0 + a.g, m);
              if (vec4 && c1 - c0 == a.g) {
                for (int c = c0; c < c1; c += 4) {
                  const float4 x4 = *reinterpret_cast<const float4*>(xr + c);
                  const float4 q4 = __ldg(reinterpret_cast<const float4*>(qr + c));
                  part = add_term<L1>(x4.x - q4.x, part);
                  part = add_term<L1>(x4.y - q4.y, part);
                  part = add_term<L1>(x4.z - q4.z, part);
                  part = add_term<L1>(x4.w - q4.w, part);
                }
              } else {
                for (int c = c0; c < c1; ++c) {
                  const float d = xr[c] - __ldg(qr + c);
                  part = add_term<L1>(d, part);
                }
              }
            }
          }
        }
      }
#pragma unroll
      for (int o = 16; o; o >>= 1)
        if (o < G) part += __shfl_xor_sync(0xffffffffu, part, o);
      if (pi < np && gl == 0) {
        R0[(size_t)q * (size_t)n + p0 + pi] = part;
        tmin = fminf(tmin, part);
      }
    }
    if (R0min) {
#pragma unroll
      for (int o = 16; o; o >>= 1) tmin = fminf(tmin, __shfl_xor_sync(0xffffffffu, tmin, o));
      if (lane == 0) R0min[(size_t)q * gridDim.x + blockIdx.x] = tmin;
    }
  }
}

// Round 0 under shared coordinates: a point's first B0 draws are the first
// B0 columns of its permuted row, so one thread per point reads them once and
// forms the round-0 sum with every query of the chunk (their permuted values
// staged in shared memory). The sum follows the round-loop kernel's order:
// each block of 8 draws in sequence into its own partial, then the partials
// combined as the lane butterfly of the round loop combines them (G lanes,
// G the power of two at or above the number of blocks). NB blocks of 8 at
// most: B0 <= 8 NB.
constexpr int kR0SharedThreads = 256;

template <int NB>
struct R0SharedCfg {
  static constexpr int kQueries = NB <= 2 ? 256 : (NB <= 4 ? 128 : 64);  // queries staged at a time (16 KB)
};

// The chunk's query values at the first W permuted columns (zero past B0),
// row-major [nq][W], so the round-0 pass stages them with plain loads.
static __global__ void permute_query_columns_kernel(const float* __restrict__ Q, int m, int nq,
                                                    const int32_t* __restrict__ jperm, int B0, int W,
                                                    float* __restrict__ Qp) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)nq * W) return;
  const int q = (int)(e / W), t = (int)(e - (int64_t)q * W);
  Qp[e] = t < B0 ? __ldg(Q + (size_t)q * m + jperm[t]) : 0.0f;
}

// One point's round-0 sum against one staged query row v4 (the round loop's
// order: blocks of 8 draws into partials, then the lane butterfly over G).
template <int NB, bool L1>
__device__ __forceinline__ float r0_shared_sum(const float* x, const float4* v4, int nfull, int rem, int G) {
  float p[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    p[b] = 0.0f;
    if (b < nfull || (b == nfull && rem)) {  // uniform over the grid
      const float4 va = v4[2 * b], vb = v4[2 * b + 1];
      const float vv[8] = {va.x, va.y, va.z, va.w, vb.x, vb.y, vb.z, vb.w};
      if (b < nfull) {
#pragma unroll
        for (int w = 0; w < 8; ++w) {
          const float d = x[8 * b + w] - vv[w];
          p[b] = add_term<L1>(d, p[b]);
        }
      } else {
#pragma unroll
        for (int w = 0; w < 8; ++w)
          if (w < rem) {
            const float d = x[8 * b + w] - vv[w];
            p[b] = add_term<L1>(d, p[b]);
          }
      }
    }
  }
#pragma unroll
  for (int o = NB / 2; o; o >>= 1)
    if (o < G) {
#pragma unroll
      for (int j = 0; j < o; ++j) p[j] += p[j + o];
    }
  return p[0];
}

template <class E, int NB, bool L1>
__global__ void __launch_bounds__(kR0SharedThreads) round0_shared_kernel(AdaptiveArgs a, const float* Qp, float* R0,
                                                                         float* R0min) {
  // grid: x = tiles of kR0SharedThreads points, y = slices of kQ queries
  constexpr int W = 8 * NB;
  constexpr int kQ = R0SharedCfg<NB>::kQueries;
  __shared__ __align__(16) float qv[kQ * W];
  using Tp = typename E::T;
  const int64_t n = a.n;
  const int B0 = a.B0;
  const int nfull = B0 >> 3, rem = B0 & 7;
  const int nblk = nfull + (rem ? 1 : 0);
  int G = 1;
  while (G < nblk) G <<= 1;
  const int64_t i = (int64_t)blockIdx.x * kR0SharedThreads + threadIdx.x;
  const int q0 = (int)blockIdx.y * kQ;
  const int qc = min(kQ, a.nq - q0);
  {
    const float4* src = reinterpret_cast<const float4*>(Qp + (size_t)q0 * W);
    float4* dst = reinterpret_cast<float4*>(qv);
    for (int e = threadIdx.x; e < qc * W / 4; e += kR0SharedThreads) dst[e] = __ldg(src + e);
  }
  float x[W];
#pragma unroll
  for (int t = 0; t < W; ++t) x[t] = 0.0f;
  if (i < n) {
    const Tp* xr = static_cast<const Tp*>(a.G) + (size_t)i * (size_t)a.mp;
    const float sc = E::kScaled ? __ldg(a.gscale + i) : 1.0f;
#pragma unroll
    for (int b = 0; b < NB; ++b)
      if (b < nblk) load8<E>(xr + 8 * b, x + 8 * b);
#pragma unroll
    for (int t = 0; t < W; ++t) x[t] = E::kScaled ? __fmul_rn(x[t], sc) : x[t];
  }
  __syncthreads();
  if (((int64_t)blockIdx.x * kR0SharedThreads + (threadIdx.x & ~31)) >= n) return;  // warp-uniform
  const float4* v4 = reinterpret_cast<const float4*>(qv);
  auto store = [&](int qq, float S) {
    const int qg = q0 + qq;
    if (i < n) R0[(size_t)qg * (size_t)n + i] = S;
    if (R0min) {  // smallest sum of the warp's 32 points
      float t = i < n ? S : INFINITY;
#pragma unroll
      for (int o = 16; o; o >>= 1) t = fminf(t, __shfl_xor_sync(0xffffffffu, t, o));
      if ((threadIdx.x & 31) == 0) R0min[(size_t)qg * (size_t)a.r0tiles + (size_t)(i >> 5)] = t;
    }
  };
  int qq = 0;
  for (; qq + 1 < qc; qq += 2) {  // two queries at a time: independent chains
    const float S0 = r0_shared_sum<NB, L1>(x, v4 + (size_t)qq * (W / 4), nfull, rem, G);
    const float S1 = r0_shared_sum<NB, L1>(x, v4 + (size_t)(qq + 1) * (W / 4), nfull, rem, G);
    store(qq, S0);
    store(qq + 1, S1);
  }
  if (qq < qc) store(qq, r0_shared_sum<NB, L1>(x, v4 + (size_t)qq * (W / 4), nfull, rem, G));
}

// Range of the finite data as ordered keys, xr[0] = min, xr[1] = max, and
// xr[2] = 1 if any element is NaN or infinite.
static __global__ void minmax_kernel(const float* __restrict__ X, size_t count, uint32_t* xr) {
  uint32_t lo = 0xFFFFFFFFu, hi = 0u, bad = 0u;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
    const float v = __ldg(X + i);
    if (isfinite(v)) {
      const uint32_t key = f2key(v);
      lo = min(lo, key);
      hi = max(hi, key);
    } else {
      bad = 1u;
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&xr[0], lo);
    atomicMax(&xr[1], hi);
    if (bad) atomicOr(&xr[2], 1u);
  }
}

// --------------------------------------------------------------- host side

constexpr int kAdaptiveNT = 512;  // default threads per CTA (256 is the other choice)

// Dynamic shared memory of the round loop: query row, histogram, select
// buffer, accepted lists, the permuted query (shared coordinates) and, with
// row passes, one row and kFuseParts partial sums per warp.
static size_t adaptive_smem_bytes(int m, bool perm = false, int fuse_threads = 0) {
  const size_t mpad = (size_t)((m + 3) & ~3);
  const size_t mp = (size_t)((m + 7) & ~7);
  return mpad * 4 + (size_t)kHistBins * 4 + (size_t)kSelCap * 4 + 2 * (size_t)(kMaxKH + 4) * 4 +
         (size_t)kMaxKH * 4 + (perm ? mp * 4 : 0) + (size_t)(fuse_threads / 32) * (mpad + kFuseParts) * 4;
}

struct AdaptivePlan {
  int grid = 0;
  int threads = kAdaptiveNT;
  int acc_cap = 0;
  size_t smem = 0;
  int fuse_cap = 0;  // slots a row pass may cover (0: none)
};

// The round-loop kernel instantiated for a thread count (256, 512 or 1024;
// all keep 64 registers per thread: 8, 16 or 32 warps per query) and a metric.
template <class E, bool L1>
static void* rounds_kernel_for_metric(int threads) {
  if (threads == 256) return reinterpret_cast<void*>(adaptive_rounds_kernel<256, E, L1>);
  if (threads == 1024) return reinterpret_cast<void*>(adaptive_rounds_kernel<1024, E, L1>);
  return reinterpret_cast<void*>(adaptive_rounds_kernel<512, E, L1>);
}

template <class E>
static void* rounds_kernel_for(int threads, bool l1) {
  return l1 ? rounds_kernel_for_metric<E, true>(threads) : rounds_kernel_for_metric<E, false>(threads);
}

template <class E>
static knn_status plan_adaptive(int64_t n, int32_t m, int32_t nq, int32_t k, const knn_opts* o, AdaptivePlan* p) {
  DeviceInfo di;
  knn_status s = device_info(&di);
  if (s != KNN_OK) return s;
  p->threads = (o && (o->threads == 256 || o->threads == 1024)) ? o->threads : kAdaptiveNT;
  p->smem = adaptive_smem_bytes(m, E::kPerm);
  p->fuse_cap = 0;
  if (std::is_same<E, ElemF32>::value && o && o->row_pass) {  // row passes: per-pair draws of the FP32 data
    const size_t f = adaptive_smem_bytes(m, false, p->threads);
    if (f + 1024 <= di.smem_optin) {
      p->smem = f;
      p->fuse_cap = (int)std::min<int64_t>(n, kFuseCap);
    }
  }
  const void* fn = rounds_kernel_for<E>(p->threads, o && o->metric == KNN_METRIC_L1);
  s = cuda_check(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->smem),
                 "cudaFuncSetAttribute(adaptive)");
  if (s != KNN_OK) return s;
  int per_sm = 0;
  s = cuda_check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, p->threads, p->smem),
                 "occupancy(adaptive)");
  if (s != KNN_OK) return s;
  if (per_sm < 1) {
    set_error("adaptive kernel does not fit on an SM");
    return KNN_EUNSUPPORTED;
  }
  int grid = per_sm * di.sms;
  if (o && o->max_ctas > 0 && o->max_ctas < grid) grid = o->max_ctas;
  if (grid > nq) grid = nq;
  if (grid < 1) grid = 1;
  p->grid = grid;
  p->acc_cap = 2 * k + 2;
  return KNN_OK;
}

template <class E, bool L1>
static void launch_rounds_metric(const AdaptivePlan& p, const AdaptiveArgs& a, cudaStream_t stream) {
  if (p.threads == 256)
    adaptive_rounds_kernel<256, E, L1><<<p.grid, 256, p.smem, stream>>>(a);
  else if (p.threads == 1024)
    adaptive_rounds_kernel<1024, E, L1><<<p.grid, 1024, p.smem, stream>>>(a);
  else
    adaptive_rounds_kernel<512, E, L1><<<p.grid, 512, p.smem, stream>>>(a);
}

template <class E>
static knn_status launch_rounds(const AdaptivePlan& p, const AdaptiveArgs& a, cudaStream_t stream) {
  // the plan may come from another element type of the same layout (draws
  // without replacement share the per-pair plan): the launched kernel gets its
  // own shared-memory limit
  const knn_status s = cuda_check(cudaFuncSetAttribute(rounds_kernel_for<E>(p.threads, a.l1),
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem),
                                  "cudaFuncSetAttribute(adaptive)");
  if (s != KNN_OK) return s;
  if (a.l1)
    launch_rounds_metric<E, true>(p, a, stream);
  else
    launch_rounds_metric<E, false>(p, a, stream);
  return cuda_check(cudaGetLastError(), "adaptive_rounds_kernel launch");
}

struct AdaptiveCarve {
  uint32_t* xrange;
  int32_t* queue;
  int32_t* ids;
  float* S;
  float* C;
  int32_t* acc_id;
  float* acc_d;
  float* acc_U;
  float* acc_L;
  float* F;
};

static size_t carve_adaptive(Carve& cv, int64_t n, const AdaptivePlan& p, AdaptiveCarve* out) {
  AdaptiveCarve c;
  c.xrange = cv.take<uint32_t>(3);
  c.queue = cv.take<int32_t>(1);
  const size_t per = (size_t)p.grid * 2 * (size_t)n;
  c.ids = cv.take<int32_t>(per);
  c.S = cv.take<float>(per);
  c.C = cv.take<float>(per);
  const size_t acc = (size_t)p.grid * (size_t)p.acc_cap;
  c.acc_id = cv.take<int32_t>(acc);
  c.acc_d = cv.take<float>(acc);
  c.acc_U = cv.take<float>(acc);
  c.acc_L = cv.take<float>(acc);
  c.F = p.fuse_cap ? cv.take<float>((size_t)p.grid * (kFuseRounds + 2) * (size_t)p.fuse_cap) : nullptr;
  if (out) *out = c;
  return cv.off;
}

// Round-0 sums of a chunk of queries (the point-major round-0 pass), at
// most kR0BufferBytes: the query chunk is sized to fit.
constexpr size_t kR0BufferBytes = size_t(1) << 30;

static inline int32_t block_count(int32_t m, const knn_opts& o) {
  const int32_t g = o.block > 1 ? o.block : 1;
  return (m + g - 1) / g;
}

static inline bool round0_applies(int32_t m, const knn_opts& o) { return o.B0 < block_count(m, o) && o.B0 <= 256; }

// Block samples of a launch (after a.m and a.G are set): g coordinates per
// draw, ceil(m/g) draws to the exact distance, and whether a block is one
// 32-byte run of the copy on 16-byte aligned rows.
template <class E>
static inline void set_blocks(AdaptiveArgs& a, const knn_opts& o) {
  a.l1 = o.metric == KNN_METRIC_L1 ? 1 : 0;  // (the metric and the query alignment ride along)
  a.qvec = (a.m % 4 == 0 && ((uintptr_t)a.Q & 15) == 0) ? 1 : 0;
  const size_t elem = sizeof(typename E::T);
  const int32_t g = (E::kBlk && o.block > 1) ? o.block : 1;
  a.g = g;
  a.Mb = (a.m + g - 1) / g;
  a.gvec = (g > 1 && (size_t)g * elem == 32 && ((size_t)a.m * elem) % 16 == 0 && ((uintptr_t)a.G & 15) == 0) ? 1 : 0;
  int bits = 0;  // ceil(log2 m)
  while ((1 << bits) < a.m) ++bits;
  a.wor_h = E::kWor ? std::max(1, (bits + 1) / 2) : 0;
}

// Queries per chunk: as many as the buffer holds, but never fewer than the
// round-loop kernel's resident CTAs (a smaller chunk would leave SMs idle).
static inline int round0_chunk(int64_t n, int32_t nq, int grid) {
  const int64_t c = std::max<int64_t>((int64_t)(kR0BufferBytes / (4 * (size_t)n)), grid);
  return (int)std::max<int64_t>(1, std::min<int64_t>(nq, c));
}

static knn_status validate(int64_t n, int32_t m, int32_t nq, int32_t k, double delta, const knn_opts& o) {
  if (n < 1 || n >= (int64_t)1 << 31) return set_error("n must be in [1, 2^31)"), KNN_EINVAL;
  if (m < 1 || m > kMaxM) return set_error("m must be in [1, 16384]"), KNN_EINVAL;
  if (nq < 0) return set_error("nq must be >= 0"), KNN_EINVAL;
  if (k < 1 || k > n) return set_error("k must be in [1, n]"), KNN_EINVAL;
  if (o.h < 0 || (int64_t)k + o.h > kMaxKH) return set_error("need h >= 0 and k + h <= 1024"), KNN_EINVAL;
  if (!(delta > 0.0 && delta < 1.0)) return set_error("delta must be in (0, 1)"), KNN_EINVAL;
  if (o.bound < 0 || o.bound > 2) return set_error("unknown bound form"), KNN_EINVAL;
  if (o.bound == KNN_BOUND_FOOTNOTE && !(delta / (double)n < std::exp(-1.0)))
    return set_error("footnote bound needs delta/n < 1/e"), KNN_EINVAL;
  if (o.bound == KNN_BOUND_EXP && !(o.c_alpha > 0.0)) return set_error("c_alpha must be > 0"), KNN_EINVAL;
  if (o.B0 < 1 || o.B < 1) return set_error("B0 and B must be >= 1"), KNN_EINVAL;
  if (o.threads != 0 && o.threads != 256 && o.threads != 512 && o.threads != 1024)
    return set_error("threads must be 0, 256, 512 or 1024"), KNN_EINVAL;
  if (o.grow != 0 && o.grow != 1) return set_error("grow must be 0 or 1"), KNN_EINVAL;
  if (o.block < 0 || o.block > 64) return set_error("block must be in [0, 64]"), KNN_EINVAL;
  if (o.metric != KNN_METRIC_L2SQ && o.metric != KNN_METRIC_L1) return set_error("unknown metric"), KNN_EINVAL;
  if (o.sampling != KNN_SAMPLE_WITH && o.sampling != KNN_SAMPLE_WITHOUT)
    return set_error("unknown sampling"), KNN_EINVAL;
  if (o.sampling == KNN_SAMPLE_WITHOUT && o.block > 1)
    return set_error("sampling without replacement takes single coordinates (block 0 or 1)"), KNN_EINVAL;
  return KNN_OK;
}

static knn_opts resolve(const knn_opts* opts, int32_t k) {
  knn_opts o;
  knn_opts_default(&o);
  if (opts) o = *opts;
  if (o.h < 0) o.h = k;
  return o;
}

}  // namespace knn
