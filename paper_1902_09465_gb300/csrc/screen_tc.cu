// screen_tc.cu -- the naive exact method (Section 3: every distance, then
// select) as a tcgen05 tensor-core GEMM with the selection fused into its
// epilogue, followed by an FP32 refine and an FP64 rerank of near ties
// (rerank.cu).
//
// Distances are translation invariant, so the data is centred on its column
// mean mu once (xc = x - mu) and the screened distance of a pair is
//   D~ = fl(||xc||^2 + ||qc||^2 + c2 * acc),   acc ~ sum_j xc^_j qc^_j,
// acc accumulated in FP32 in tensor memory over 16-bit operands xc^, qc^ of
// one of three kinds:
//   F16     xc and qc scaled by powers of two (max |.| in [2^14, 2^15)) and
//           rounded to FP16 (u = 2^-11): K = m, c2 = -2 / (scales);
//   BF16    rounded to BF16 (u = 2^-8): K = m, c2 = -2;
//   BF16X3  split xc = hi + lo + r (|r| <= 2^-18 |xc|), the concatenated rows
//           [hi | hi | lo] . [qhi | qlo | qhi]: K = 3m, c2 = -2.
// |D~ - d| <= E_q, a bound from the operand rounding, the FP32 accumulation
// and the norms' FP32 sums (exact_tc below).
//
// Two passes of one persistent kernel avoid writing the nq x n matrix:
//   pass 1  every s-th tile of 128 points: the smallest D~ of each group of 32
//           points, per query (group minima come from distinct points, so the
//           k-th smallest of them bounds the k-th smallest D~ from above);
//   cut     tau_q = that k-th smallest, cut_q = tau_q + 2 E_q (screen_cut_kernel);
//   pass 2  every tile: each pair with D~ <= cut_q joins the query's candidate
//           list (atomic append; a full list marks the query for a full scan).
// Every true k-nearest point j is kept: k points have D~ <= tau_q, so the
// k-th true distance is at most tau_q + E_q, and d_j <= that gives
// D~_j <= d_j + E_q <= cut_q.
//
// Kernel layout: one CTA per SM, persistent over tiles of 128 points x 256
// queries, 10 warps. Warp 0 lane 0 issues TMA loads (128-byte swizzle, 64
// K-elements per stage, 4 stages); warp 1 lane 0 issues tcgen05.mma (M = 128,
// N = 256, K = 16, FP32 accumulator in TMEM) into one of two accumulators of
// 256 columns, so the epilogue of one tile overlaps the MMAs of the next;
// warps 2-9 read the accumulator (tcgen05.ld 32x32b; two warps per TMEM lane
// quarter, 128 columns each) and run the pass's epilogue. Every mbarrier wait
// is bounded: a wait that gives up records a code in the library status
// word, the CTA waits for its TMA copies and MMAs in flight and frees its
// tensor memory before it exits.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <mutex>
#include <string>

#include "knn_common.cuh"
#include "knn_internal.h"

namespace knn {

knn_status launch_refine(const float* X, int64_t n, int32_t m, const float* Q, int32_t nq, const int64_t* cand,
                         int32_t ncand, const int32_t* cnt, int32_t k, int64_t* out_idx, double* out_dist,
                         cudaStream_t stream, int32_t metric, const float* cand_d = nullptr,
                         const float* eq = nullptr);

constexpr int kTcM = 128, kTcN = 256, kTcK = 64, kTcStages = 4, kTcThreads = 320;
constexpr int kTcABytes = kTcM * kTcK * 2;  // 16 KB
constexpr int kTcBBytes = kTcN * kTcK * 2;  // 32 KB
constexpr int kTcCols = 2 * kTcN;           // two accumulators of 256 FP32 columns
constexpr int kScreenCap = 2048;            // candidate slots per query
constexpr int kStage = 8;                   // pairs of a query column staged per tile in shared memory
constexpr uint32_t kSpinDefault = 1u << 26;
constexpr int kStatusTimeout = 0x5C7C;      // recorded when a bounded wait gives up

// Tries of the pipeline waits (a test hook; see knn_debug_wait_limit).
static std::atomic<uint32_t> g_wait_limit{kSpinDefault};

enum ScreenKind { kKindF16 = 0, kKindBF16 = 1, kKindBF16x3 = 2 };

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for the phase of `parity` to complete; false after `limit` tries.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint32_t limit) {
  for (uint32_t i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::
          "r"(dst),
      "l"(map), "r"(bar), "r"(c0), "r"(c1)
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major tile written by TMA with the
// 128-byte swizzle: rows of 128 bytes, groups of 8 rows 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_kmajor_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address (16-byte units)
  d |= (uint64_t)1 << 16;                     // leading byte offset (unused with this swizzle)
  d |= (uint64_t)(1024 >> 4) << 32;           // stride byte offset: 8-row group pitch
  d |= (uint64_t)1 << 46;                     // descriptor version of tcgen05
  d |= (uint64_t)2 << 61;                     // 128-byte swizzle
  return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), A and
// B types at bits 7-9 and 10-12 (0 = F16, 1 = BF16), both K-major, N >> 3 at
// bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_f16kind(bool bf16) {
  return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) | ((uint32_t)(kTcN >> 3) << 17) |
         ((uint32_t)(kTcM >> 4) << 24);
}

__device__ __forceinline__ void umma_f16kind(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                             uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
// Barrier of the 256 epilogue threads (named barrier 1).
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

// OR of a predicate over the 256 epilogue threads (named barrier 1).
__device__ __forceinline__ bool epi_any(bool p) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.or.pred q, 1, 256, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)p)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ void tmem_ld_x32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Minimum over the 32 lanes of each of 16 values: halve the set per step
// (lanes of the upper half keep the upper values), 16 shuffles in all. On
// return the lane pair (2c, 2c + 1) holds the minimum of value c.
__device__ __forceinline__ float warp_min16(float (&v)[16], int lane) {
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const bool up = lane & 16;
    const float keep = up ? v[j + 8] : v[j], send = up ? v[j] : v[j + 8];
    v[j] = fminf(keep, __shfl_xor_sync(0xffffffffu, send, 16));
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const bool up = lane & 8;
    const float keep = up ? v[j + 4] : v[j], send = up ? v[j] : v[j + 4];
    v[j] = fminf(keep, __shfl_xor_sync(0xffffffffu, send, 8));
  }
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const bool up = lane & 4;
    const float keep = up ? v[j + 2] : v[j], send = up ? v[j] : v[j + 2];
    v[j] = fminf(keep, __shfl_xor_sync(0xffffffffu, send, 4));
  }
  {
    const bool up = lane & 2;
    const float keep = up ? v[1] : v[0], send = up ? v[0] : v[1];
    v[0] = fminf(keep, __shfl_xor_sync(0xffffffffu, send, 2));
  }
  return fminf(v[0], __shfl_xor_sync(0xffffffffu, v[0], 1));
}

struct ScreenArgs {
  int64_t n;          // points
  int nq;             // queries
  int nk;             // K blocks of 64 elements per row
  int nqt;            // query tiles (256 queries each)
  int stride;         // point tiles visited: every stride-th (pass 1), every one (pass 2)
  int ntiles;         // tiles of this pass: ceil(point tiles / stride) x nqt
  int pass;           // 1: group minima, 2: candidate lists
  uint32_t idesc;     // MMA instruction descriptor (operand type)
  uint32_t limit;     // tries of a pipeline wait before it gives up
  const float* xn;    // [n] ||xc||^2 (FP32)
  const float* qn;    // [nq] ||qc||^2 (FP32)
  const float* c2;    // device scalar: -2 / (product of the operand scales)
  float* gmin;        // pass 1: [nq][nunits] smallest D~ of each group of 32 points
  int nunits;         // groups per query in pass 1: 4 per visited point tile
  const float* cut;   // pass 2: [nq] cut_q
  int* cnt;           // pass 2: [nq] candidates appended (may exceed cap)
  int64_t* cand;      // pass 2: [nq][cap] candidate points
  float* cand_d;      // pass 2: [nq][cap] their screened values D~
  int cap;
  int* status;        // library status word
  int ksteps;         // MMAs (K = 16 each) per stage: 4, or fewer when the operands' columns end earlier
  int8_t akb[8];      // pass 3: K block of A and of B loaded by stage kb (part products of split operands)
  int8_t bkb[8];
  float* r0;          // pass 3: [nq][n] the round-0 sums (gmin takes the group minima)
};

__global__ void __launch_bounds__(kTcThreads, 1)
    screen_tc_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                     const ScreenArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;
  uint8_t* sB = smem + kTcStages * kTcABytes;
  // barriers: full[S], empty[S], acc_full[2], acc_empty[2], drain
  uint64_t* bars = reinterpret_cast<uint64_t*>(sB + kTcStages * kTcBBytes);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kTcStages + 5);
  volatile int* err = reinterpret_cast<volatile int*>(tmem_slot + 1);
  int* scnt = reinterpret_cast<int*>(tmem_slot + 4);                 // [256] staged pairs per column (pass 2)
  uint8_t* srow = reinterpret_cast<uint8_t*>(scnt + kTcN);           // [256][kStage] their rows in the tile
  float2* colv = reinterpret_cast<float2*>(srow + kTcN * kStage);    // [256] per-column constants of the tile
  float* sval = reinterpret_cast<float*>(colv + kTcN);                // [256][kStage] their screened values
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + kTcStages);
  const uint32_t accf0 = smem_u32(bars + 2 * kTcStages), acce0 = smem_u32(bars + 2 * kTcStages + 2);
  const uint32_t drain = smem_u32(bars + 2 * kTcStages + 4);

  if (threadIdx.x == 0) {
    for (int s = 0; s < kTcStages; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accf0 + 8 * b, 1);
      mbar_init(acce0 + 8 * b, 256);  // every epilogue thread arrives once per tile
    }
    mbar_init(drain, 1);
    *err = 0;
    for (int c = 0; c < kTcN; ++c) scnt[c] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTcCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  uint32_t issued = 0;  // k-block loads the producer issued (for the clean-up)
  if (warp == 0) {
    if (lane == 0) {  // TMA producer
      uint32_t it = 0;
      for (int t = blockIdx.x; t < a.ntiles && !*err; t += gridDim.x) {
        const int p0 = (t / a.nqt) * a.stride * kTcM, q0 = (t % a.nqt) * kTcN;
        for (int kb = 0; kb < a.nk; ++kb, ++it) {
          const int s = it % kTcStages;
          const uint32_t ph = (it / kTcStages) & 1u;
          if (!mbar_wait(empty0 + 8 * s, ph ^ 1u, a.limit)) {
            *err = 1;
            break;
          }
          mbar_expect_tx(full0 + 8 * s, kTcABytes + kTcBBytes);
          const int ka = a.pass == 3 ? a.akb[kb] : kb, kbb = a.pass == 3 ? a.bkb[kb] : kb;
          tma_load_2d(smem_u32(sA + s * kTcABytes), &mapA, full0 + 8 * s, ka * kTcK, p0);
          tma_load_2d(smem_u32(sB + s * kTcBBytes), &mapB, full0 + 8 * s, kbb * kTcK, q0);
          issued = it + 1;
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      uint32_t it = 0, tc = 0;
      for (int t = blockIdx.x; t < a.ntiles && !*err; t += gridDim.x, ++tc) {
        const int buf = tc & 1;
        if (!mbar_wait(acce0 + 8 * buf, ((tc >> 1) & 1u) ^ 1u, a.limit)) {
          *err = 1;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(buf * kTcN);
        bool ok = true;
        for (int kb = 0; kb < a.nk; ++kb, ++it) {
          const int s = it % kTcStages;
          const uint32_t ph = (it / kTcStages) & 1u;
          if (!mbar_wait(full0 + 8 * s, ph, a.limit)) {
            *err = 1;
            ok = false;
            break;
          }
          tc_fence_after();
          const uint64_t ad = sw128_kmajor_desc(smem_u32(sA + s * kTcABytes));
          const uint64_t bd = sw128_kmajor_desc(smem_u32(sB + s * kTcBBytes));
          for (int ks = 0; ks < a.ksteps; ++ks)  // 16 elements = 32 bytes per step along K
            umma_f16kind(d, ad + 2 * ks, bd + 2 * ks, a.idesc, (kb | ks) != 0);
          umma_commit(empty0 + 8 * s);
        }
        if (!ok) break;
        umma_commit(accf0 + 8 * buf);
      }
      // every MMA this thread issued completes before the tensor memory is freed
      umma_commit(drain);
      mbar_wait(drain, 0, kSpinDefault);
    }
    __syncwarp();
  } else {  // epilogue: warps 2-9; warp w reads TMEM lanes 32 (w % 4) .. + 31, columns 128 ((w - 2) / 4) .. + 127
    const int quarter = warp & 3;
    const int half = (warp - 2) >> 2;
    const int row = quarter * 32 + lane;
    const int et = threadIdx.x - 64;  // 0..255: the column this thread stages and flushes
    const float c2 = *a.c2;
    uint32_t tc = 0;
    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x, ++tc) {
      const int buf = tc & 1;
      const bool ok = !*err && mbar_wait(accf0 + 8 * buf, (tc >> 1) & 1u, a.limit);
      // the epilogue warps take the same decision, so that none of them waits
      // at a named barrier that another has left
      if (epi_any(!ok)) {
        *err = 1;
        break;
      }
      tc_fence_after();
      const int pt_vis = t / a.nqt;
      const int64_t p0 = (int64_t)pt_vis * a.stride * kTcM;
      const int q0 = (t % a.nqt) * kTcN;
      const int64_t p = p0 + row;
      const float xv = p < a.n ? __ldg(a.xn + p) : INFINITY;
      {  // the tile's per-column constants: ||qc||^2 and the cut (-inf: no query)
        const int q = q0 + et;
        colv[et] = q < a.nq ? make_float2(__ldg(a.qn + q), a.pass == 2 ? __ldg(a.cut + q) : 0.0f)
                            : make_float2(0.0f, -INFINITY);  // (passes 1 and 3: 0 marks a query)
      }
      epi_sync();
      const uint32_t taddr =
          tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(buf * kTcN) + (uint32_t)(half * (kTcN / 2));
      for (int c0 = 0; c0 < kTcN / 2; c0 += 32) {
        float v[32];
        tmem_ld_x32(taddr + (uint32_t)c0, v);
        const int cb = half * (kTcN / 2) + c0;  // tile column of v[0]
        if (a.pass != 2) {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const float2 cv = colv[cb + j];
            v[j] = cv.y == -INFINITY ? INFINITY : fmaf(c2, v[j], xv + cv.x);
          }
          if (a.pass == 3 && p < a.n) {  // round-0 sums: a sum of squares is never below 0
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              v[j] = fmaxf(v[j], 0.0f);
              const int q = q0 + cb + j;
              if (q < a.nq) a.r0[(size_t)q * a.n + p] = v[j];
            }
          }
          const float mn0 = warp_min16(*reinterpret_cast<float(*)[16]>(v), lane);
          const float mn1 = warp_min16(*reinterpret_cast<float(*)[16]>(v + 16), lane);
          if ((lane & 1) == 0) {
            const size_t unit = (size_t)pt_vis * 4 + quarter;
            const int qa = q0 + cb + (lane >> 1), qb = qa + 16;
            if (unit < (size_t)a.nunits) {  // (round 0: groups past the last point are not stored)
              if (qa < a.nq) a.gmin[(size_t)qa * a.nunits + unit] = mn0;
              if (qb < a.nq) a.gmin[(size_t)qb * a.nunits + unit] = mn1;
            }
          }
        } else {
          uint32_t hit = 0;
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const float2 cv = colv[cb + j];
            v[j] = fmaf(c2, v[j], xv + cv.x);
            hit |= (v[j] <= cv.y ? 1u : 0u) << j;
          }
          if (p >= a.n) hit = 0;
          if (__any_sync(0xffffffffu, hit != 0)) {
            // stage passing pairs per column in shared memory (a global atomic
            // per pair here would stall the warp for its round trip)
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              if (!((hit >> j) & 1u)) continue;
              const int c = cb + j;
              const int slot = atomicAdd(&scnt[c], 1);
              if (slot < kStage) {
                srow[c * kStage + slot] = (uint8_t)row;
                sval[c * kStage + slot] = v[j];
              } else {  // a crowded column: straight to the global list
                const int q = q0 + c;
                const int pos = atomicAdd(a.cnt + q, 1);
                if (pos < a.cap) {
                  a.cand[(size_t)q * a.cap + pos] = p;
                  a.cand_d[(size_t)q * a.cap + pos] = v[j];
                }
              }
            }
          }
        }
      }
      tc_fence_before();
      mbar_arrive(acce0 + 8 * buf);  // the accumulator is free for the next tile's MMAs
      if (a.pass == 2) {
        // flush: one global reservation per column with staged pairs
        epi_sync();
        const int cnt_c = min(scnt[et], kStage);
        if (cnt_c > 0) {
          const int q = q0 + et;
          const int base = atomicAdd(a.cnt + q, cnt_c);
          for (int i = 0; i < cnt_c; ++i)
            if (base + i < a.cap) {
              a.cand[(size_t)q * a.cap + base + i] = p0 + srow[et * kStage + i];
              a.cand_d[(size_t)q * a.cap + base + i] = sval[et * kStage + i];
            }
        }
        scnt[et] = 0;  // (the next tile stages after its own barrier)
      }
    }
  }

  __syncthreads();
  if (*err) {
    if (threadIdx.x == 0) atomicExch(a.status, kStatusTimeout);
    // the copies this CTA issued land before its shared memory is released
    if (warp == 0 && lane == 0)
      for (uint32_t it = (issued > kTcStages ? issued - kTcStages : 0); it < issued; ++it)
        mbar_wait(full0 + 8 * (it % kTcStages), (it / kTcStages) & 1u, kSpinDefault);
  }
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols));
  }
}

// ---- pass 1 -> pass 2: the cut of each query

// cut_q = tau_q + 2 E_q (plus a few units of roundoff), tau_q the k-th
// smallest group minimum of pass 1; +inf when there are fewer than k groups.
// Also stores E_q (for the ranking) and zeroes the query's candidate count
// for pass 2.
constexpr int kCutNT = 256;

__global__ void __launch_bounds__(kCutNT) screen_cut_kernel(const float* __restrict__ gmin, int nunits, int k, int m,
                                                            const float* __restrict__ qn,
                                                            const unsigned* __restrict__ xn_max_bits,
                                                            float c_cross, float c_square, float* __restrict__ cut,
                                                            float* __restrict__ eq, int* __restrict__ cnt) {
  __shared__ uint32_t hist[kHistBins];
  __shared__ uint32_t buf[kSelCap];
  __shared__ BlockScratch<kCutNT> bs;
  __shared__ SelectShared ss;
  const int q = blockIdx.x;
  float tau = INFINITY;
  if (nunits >= k) {
    const float* g = gmin + (size_t)q * nunits;
    for (int i = threadIdx.x; i < kHistBins; i += kCutNT) hist[i] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < nunits; i += kCutNT) atomicAdd(&hist[f2key(g[i]) >> 20], 1u);
    __syncthreads();
    select_smallest<kCutNT>([&](int i) { return f2key(g[i]); }, nunits, k, hist, buf, ss, bs);
    tau = key2f(buf[k - 1]);
  }
  if (threadIdx.x == 0) {
    // FP32 arithmetic on non-negative terms: a few units of roundoff,
    // covered by the factor 1.001 (the coefficients carry their own margins)
    const float u = 1.0f / 16777216.0f;
    const float gm = (float)(m + 2) * u / (1.0f - (float)(m + 2) * u);  // the norms' FP32 sums
    const float xmax = sqrtf(__uint_as_float(*xn_max_bits) * (1.0f + gm));
    const float qq = sqrtf(qn[q] * (1.0f + gm));
    const float E = 1.001f * (c_cross * xmax * qq + c_square * (xmax + qq) * (xmax + qq));
    float c = INFINITY;
    if (isfinite(tau)) {
      const float x = tau + 2.0f * E;
      c = x + 8.0f * u * fabsf(x) + 1e-30f;
    }
    cut[q] = c;
    eq[q] = E * (1.0f + 8.0f * u);
    cnt[q] = 0;
  }
}

// ---- operands

// Column sums of X (any fixed vector works as the centre; this one keeps the
// centred values small).
static __global__ void column_sums_kernel(const float* __restrict__ X, int64_t n, int m, float* __restrict__ sums) {
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    float s = 0.0f;
    for (int64_t i = blockIdx.x; i < n; i += gridDim.x) s += __ldg(X + (size_t)i * m + j);
    atomicAdd(&sums[j], s);
  }
}
static __global__ void scale_kernel(float* v, int m, float f) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) v[j] *= f;
}

// Largest |x - mu| over rows (float bits of a non-negative value, atomicMax).
static __global__ void centred_absmax_kernel(const float* __restrict__ X, int64_t rows, int m,
                                             const float* __restrict__ mu, unsigned* max_bits) {
  unsigned mx = 0;
  const size_t count = (size_t)rows * (size_t)m;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x)
    mx = max(mx, __float_as_uint(fabsf(__ldg(X + e) - mu[e % m])));
#pragma unroll
  for (int o = 16; o; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) atomicMax(max_bits, mx);
}

// Power-of-two exponent that brings the largest |value| M into [2^14, 2^15)
// (FP16's largest finite value is 65504): 0 for M = 0.
__device__ __forceinline__ int f16_exponent(unsigned max_bits) {
  const float M = __uint_as_float(max_bits);
  if (!(M > 0.0f) || !isfinite(M)) return 0;
  return max(-120, min(120, 14 - ilogbf(M)));
}

// -2 / (product of the operand scales): the coefficient of the accumulator in
// the screened distance.
static __global__ void screen_coeff_kernel(int kind, const unsigned* xmax_bits, const unsigned* qmax_bits,
                                           float* c2) {
  if (kind == kKindF16)
    *c2 = ldexpf(-2.0f, -(f16_exponent(*xmax_bits) + f16_exponent(*qmax_bits)));
  else
    *c2 = -2.0f;
}

// Rows of a screen operand from x - mu, each part Kp wide and zero padded:
//   F16:    [fp16(2^e (x - mu))], e from the largest |x - mu| of the side;
//   BF16:   [bf16(x - mu)];
//   BF16X3: [hi | hi | lo] (data side) or [hi | lo | hi] (query side).
// norms[r] = ||x - mu||^2 (FP32), max_bits their largest value.
static __global__ void split_rows_kernel(int kind, const float* __restrict__ X, int64_t rows, int64_t rows_pad, int m,
                                         int Kp, const float* __restrict__ mu, bool query_side,
                                         const unsigned* __restrict__ absmax_bits, uint16_t* __restrict__ out,
                                         float* __restrict__ norms, unsigned* max_bits) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int parts = kind == kKindBF16x3 ? 3 : 1;
  const int e = kind == kKindF16 ? f16_exponent(*absmax_bits) : 0;
  unsigned mx = 0;
  for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < rows_pad; r += warps) {
    uint16_t* o = out + (size_t)r * parts * Kp;
    float s = 0.0f;
    for (int j = lane; j < Kp; j += 32) {
      float xc = 0.0f;
      if (r < rows && j < m) {
        xc = __ldg(X + (size_t)r * m + j) - mu[j];
        s = fmaf(xc, xc, s);
      }
      if (kind == kKindF16) {
        o[j] = __half_as_ushort(__float2half_rn(ldexpf(xc, e)));
      } else {
        const __nv_bfloat16 h = __float2bfloat16_rn(xc);
        const uint16_t hb = __bfloat16_as_ushort(h);
        o[j] = hb;
        if (kind == kKindBF16x3) {
          const uint16_t lb = __bfloat16_as_ushort(__float2bfloat16_rn(xc - __bfloat162float(h)));
          o[Kp + j] = query_side ? lb : hb;
          o[2 * Kp + j] = query_side ? hb : lb;
        }
      }
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0 && r < rows) {
      norms[r] = s;
      mx = max(mx, __float_as_uint(s));
    }
  }
  if (lane == 0 && max_bits) atomicMax(max_bits, mx);
}

// ---- host

using EncodeTiled = PFN_cuTensorMapEncodeTiled_v12000;

static knn_status get_encoder(EncodeTiled* out) {
  static std::mutex mu;
  static EncodeTiled fn = nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    knn_status s =
        cuda_check(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q),
                   "cudaGetDriverEntryPointByVersion(cuTensorMapEncodeTiled)");
    if (s != KNN_OK) return s;
    if (q != cudaDriverEntryPointSuccess || !p) {
      set_error("cuTensorMapEncodeTiled is not available");
      return KNN_EUNSUPPORTED;
    }
    fn = reinterpret_cast<EncodeTiled>(p);
  }
  *out = fn;
  return KNN_OK;
}

// 2-D 16-bit tensor map over rows x Kt (row pitch Kt elements), box 64 x
// box_rows, 128-byte swizzle. Every tile the kernel loads lies inside rows.
static knn_status make_map(CUtensorMap* map, const void* base, int64_t rows, int Kt, int box_rows, bool bf16) {
  EncodeTiled enc;
  knn_status s = get_encoder(&enc);
  if (s != KNN_OK) return s;
  cuuint64_t dims[2] = {(cuuint64_t)Kt, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)Kt * 2};
  cuuint32_t box[2] = {(cuuint32_t)kTcK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
                   const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return KNN_ECUDA;
  }
  return KNN_OK;
}

static size_t screen_smem_bytes() {
  return 1024 + (size_t)kTcStages * (kTcABytes + kTcBBytes) + (2 * kTcStages + 5) * 8 + 16 + kTcN * 4 +
         kTcN * kStage + kTcN * 8 + kTcN * kStage * 4;
}

static int kind_of_screen(int32_t screen) {
  return screen == KNN_SCREEN_F16 ? kKindF16 : (screen == KNN_SCREEN_BF16 ? kKindBF16 : kKindBF16x3);
}
static int parts_of(int kind) { return kind == kKindBF16x3 ? 3 : 1; }

static uint16_t* operand_of(const knn_dataset* ds, int kind) {
  return kind == kKindF16 ? ds->screen16 : (kind == kKindBF16 ? ds->screenb : ds->screenA);
}

// Builds the dataset's screen operands named in `copies` (KNN_COPY_SCREEN*;
// called by knn_dataset_create): the column mean, the centred norms and
// their largest value once, then each operand.
knn_status build_screen_operand(knn_dataset* ds, int32_t copies, cudaStream_t stream) {
  const int64_t n = ds->n;
  const int m = ds->m;
  ds->Kp = (m + kTcK - 1) / kTcK * kTcK;
  const size_t rows_pad = (size_t)((n + kTcM - 1) / kTcM) * kTcM;
  knn_status s = cuda_check(cudaMalloc(&ds->mu, (size_t)m * 4), "cudaMalloc(mu)");
  if (s == KNN_OK) s = cuda_check(cudaMalloc(&ds->xcn, (size_t)n * 4), "cudaMalloc(norms)");
  if (s == KNN_OK) s = cuda_check(cudaMalloc(&ds->xcn_max, 8), "cudaMalloc(norm max)");
  if (s == KNN_OK) s = cuda_check(cudaMemsetAsync(ds->mu, 0, (size_t)m * 4, stream), "memset");
  if (s == KNN_OK) s = cuda_check(cudaMemsetAsync(ds->xcn_max, 0, 8, stream), "memset");
  DeviceInfo di;
  if (s == KNN_OK) s = device_info(&di);
  if (s != KNN_OK) return s;
  column_sums_kernel<<<di.sms * 4, 256, 0, stream>>>(ds->X, n, m, ds->mu);
  scale_kernel<<<(m + 255) / 256, 256, 0, stream>>>(ds->mu, m, 1.0f / (float)n);
  // xcn_max[1]: largest |x - mu| (the FP16 operand's scale)
  centred_absmax_kernel<<<di.sms * 8, 256, 0, stream>>>(ds->X, n, m, ds->mu, ds->xcn_max + 1);
  s = cuda_check(cudaGetLastError(), "screen operand kernels");
  struct Want {
    int32_t flag;
    int kind;
    uint16_t** dst;
  } wants[3] = {{KNN_COPY_SCREEN, kKindBF16x3, &ds->screenA},
                {KNN_COPY_SCREEN_F16, kKindF16, &ds->screen16},
                {KNN_COPY_SCREEN_BF16, kKindBF16, &ds->screenb}};
  bool norms = false;
  for (const Want& w : wants) {
    if (s != KNN_OK || !(copies & w.flag)) continue;
    s = cuda_check(cudaMalloc(w.dst, rows_pad * parts_of(w.kind) * (size_t)ds->Kp * 2), "cudaMalloc(screen operand)");
    if (s != KNN_OK) break;
    split_rows_kernel<<<di.sms * 8, 256, 0, stream>>>(w.kind, ds->X, n, (int64_t)rows_pad, m, ds->Kp, ds->mu, false,
                                                       ds->xcn_max + 1, *w.dst, ds->xcn,
                                                       norms ? nullptr : ds->xcn_max);
    norms = true;
    s = cuda_check(cudaGetLastError(), "screen operand kernels");
  }
  return s;
}

struct TcCarve {
  uint16_t* B;
  float* qn;
  unsigned* qmax;  // [1] largest |q - mu| of the batch
  float* c2;
  float* gmin;
  float* cut;
  float* eq;
  int* cnt;
  int64_t* cand;
  float* cand_d;
};

static size_t carve_tc(Carve& cv, int64_t n, int32_t nq, int Kt, TcCarve* out) {
  TcCarve c;
  const size_t nq_pad = (size_t)((nq + kTcN - 1) / kTcN) * kTcN;
  const size_t npt = (size_t)((n + kTcM - 1) / kTcM);
  c.B = cv.take<uint16_t>(nq_pad * (size_t)Kt);
  c.qn = cv.take<float>(nq_pad);
  c.qmax = cv.take<unsigned>(1);
  c.c2 = cv.take<float>(1);
  c.gmin = cv.take<float>((size_t)nq * 4 * npt);
  c.cut = cv.take<float>((size_t)nq);
  c.eq = cv.take<float>((size_t)nq);
  c.cnt = cv.take<int>((size_t)nq);
  c.cand = cv.take<int64_t>((size_t)nq * kScreenCap);
  c.cand_d = cv.take<float>((size_t)nq * kScreenCap);
  if (out) *out = c;
  return cv.off;
}

size_t exact_tc_workspace(int64_t n, int32_t m, int32_t nq, int32_t screen) {
  Carve cv;
  const int Kp = (m + kTcK - 1) / kTcK * kTcK;
  return carve_tc(cv, n, nq, parts_of(kind_of_screen(screen)) * Kp, nullptr) + 256;
}

// Point tiles skipped between the tiles pass 1 visits: the k-th smallest of
// the visited groups' minima then lies near the (s k)-th smallest screened
// value, so about s k points (plus the screen's margin) become candidates.
static int pass1_stride(int64_t npt, int k) {
  int s = std::max(1, std::min(16, 128 / k));
  while (s > 1 && 4 * ((npt + s - 1) / s) < 4 * (int64_t)k) --s;
  return s;
}

knn_status exact_tc(const knn_dataset* ds, int32_t screen, const float* Q, int32_t nq, int32_t k, int64_t* out_idx,
                    double* out_dist, void* workspace, size_t workspace_bytes, cudaStream_t stream) {
  const int kind = kind_of_screen(screen);
  const uint16_t* A = operand_of(ds, kind);
  if (!A) {
    set_error("knn_exact_ds: the dataset was created without this screen's operand (KNN_COPY_SCREEN*)");
    return KNN_EINVAL;
  }
  DeviceInfo di;
  knn_status s = device_info(&di);
  if (s != KNN_OK) return s;
  if (di.major != 10) {
    set_error("the tensor-core screen needs an sm_10x device");
    return KNN_EUNSUPPORTED;
  }
  const int64_t n = ds->n;
  const int m = ds->m, Kp = ds->Kp, Kt = parts_of(kind) * Kp;
  const size_t need = exact_tc_workspace(n, m, nq, screen);
  Workspace ws;
  s = ws.acquire(workspace, workspace_bytes, need, stream);
  if (s != KNN_OK) return s;
  Carve cv;
  cv.base = reinterpret_cast<uint8_t*>(((uintptr_t)ws.ptr + 255) & ~uintptr_t(255));
  TcCarve c;
  carve_tc(cv, n, nq, Kt, &c);
  const int64_t nq_pad = (int64_t)((nq + kTcN - 1) / kTcN) * kTcN;
  const int64_t npt = (n + kTcM - 1) / kTcM;
  const int nqt = (int)(nq_pad / kTcN);

  // query operand, norms and the accumulator's coefficient
  s = cuda_check(cudaMemsetAsync(c.qmax, 0, 4, stream), "memset");
  if (s == KNN_OK) {
    if (kind == kKindF16)
      centred_absmax_kernel<<<(int)std::min<int64_t>(((int64_t)nq * m + 255) / 256, (int64_t)di.sms * 8), 256, 0,
                              stream>>>(Q, nq, m, ds->mu, c.qmax);
    split_rows_kernel<<<(int)std::min<int64_t>((nq_pad + 7) / 8, (int64_t)di.sms * 8), 256, 0, stream>>>(
        kind, Q, nq, nq_pad, m, Kp, ds->mu, true, c.qmax, c.B, c.qn, nullptr);
    screen_coeff_kernel<<<1, 1, 0, stream>>>(kind, ds->xcn_max + 1, c.qmax, c.c2);
    s = cuda_check(cudaGetLastError(), "query operand kernels");
  }
  CUtensorMap mapA, mapB;
  const bool bf16 = kind != kKindF16;
  if (s == KNN_OK) s = make_map(&mapA, A, npt * kTcM, Kt, kTcM, bf16);
  if (s == KNN_OK) s = make_map(&mapB, c.B, nq_pad, Kt, kTcN, bf16);
  int* status = nullptr;
  if (s == KNN_OK) s = device_status_ptr(&status);
  const size_t smem = screen_smem_bytes();
  if (s == KNN_OK)
    s = cuda_check(cudaFuncSetAttribute(screen_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                   "cudaFuncSetAttribute(screen_tc)");
  ScreenArgs a{};
  a.n = n;
  a.nq = nq;
  a.nk = Kt / kTcK;
  a.nqt = nqt;
  a.idesc = idesc_f16kind(bf16);
  a.limit = g_wait_limit.load();
  a.xn = ds->xcn;
  a.qn = c.qn;
  a.c2 = c.c2;
  a.gmin = c.gmin;
  a.cut = c.cut;
  a.cnt = c.cnt;
  a.cand = c.cand;
  a.cand_d = c.cand_d;
  a.cap = kScreenCap;
  a.status = status;
  a.ksteps = kTcK / 16;

  // pass 1: group minima over every s-th point tile (skipped when every
  // point fits the candidate list: the cut is then +inf)
  const bool pass1 = n > kScreenCap;
  const int stride = pass1 ? pass1_stride(npt, k) : 1;
  const int64_t nvis = (npt + stride - 1) / stride;
  a.nunits = pass1 ? (int)(4 * nvis) : 0;
  if (s == KNN_OK && pass1) {
    a.pass = 1;
    a.stride = stride;
    a.ntiles = (int)(nvis * nqt);
    screen_tc_kernel<<<std::min(a.ntiles, di.sms), kTcThreads, smem, stream>>>(mapA, mapB, a);
    s = cuda_check(cudaGetLastError(), "screen_tc_kernel launch (pass 1)");
  }
  if (s == KNN_OK) {
    // Error bound of a screened value (u = 2^-24): the operands' rounding
    // (F16: (2 u16 + u16^2) sum|xc qc|, u16 = 2^-11, plus the subnormal
    // spacing of the scaled values, below 2^-30 ||xc|| ||qc||; BF16: u16 =
    // 2^-8; BF16x3: the split residuals, 3.1 2^-18 sum|xc qc|), the FP32
    // tensor-core accumulation over Kt terms ((Kt + 16) 2^-22 sum|terms|:
    // two units of the last place per term, covering truncating adders), and
    // the norms' FP32 sums (gamma_m) with the final additions (a few units of
    // (||xc|| + ||qc||)^2); sum|xc qc| <= ||xc|| ||qc||. A factor 1.5 covers
    // second-order terms.
    const double u = 1.0 / 16777216.0;
    const double gacc = (double)(Kt + 16) * 4.0 * u;
    double prod;
    if (kind == kKindF16) prod = 2.0 * std::ldexp(1.0, -11) + std::ldexp(1.0, -22) + std::ldexp(1.0, -30);
    else if (kind == kKindBF16) prod = 2.0 * std::ldexp(1.0, -8) + std::ldexp(1.0, -16);
    else prod = 3.1 * 64.0 * u;
    const double gm = (double)(m + 2) * u / (1.0 - (double)(m + 2) * u);
    const double c_cross = 1.5 * 2.0 * (gacc + prod) * 1.01;
    const double c_square = 1.5 * (gm + 6.0 * u);
    screen_cut_kernel<<<nq, kCutNT, 0, stream>>>(c.gmin, a.nunits, k, m, c.qn, ds->xcn_max, (float)c_cross,
                                                 (float)c_square, c.cut, c.eq, c.cnt);
    s = cuda_check(cudaGetLastError(), "screen_cut_kernel launch");
  }
  if (s == KNN_OK) {  // pass 2: candidates
    a.pass = 2;
    a.stride = 1;
    a.ntiles = (int)(npt * nqt);
    screen_tc_kernel<<<std::min(a.ntiles, di.sms), kTcThreads, smem, stream>>>(mapA, mapB, a);
    s = cuda_check(cudaGetLastError(), "screen_tc_kernel launch (pass 2)");
  }
  if (s == KNN_OK)
    s = launch_refine(ds->X, n, m, Q, nq, c.cand, kScreenCap, c.cnt, k, out_idx, out_dist, stream, KNN_METRIC_L2SQ,
                      c.cand_d, c.eq);
  ws.release();
  return s;
}

// ---- round 0 under shared coordinates as a tensor-core contraction

constexpr int kR0Cols = 64;  // permuted columns held by the operand (B0 <= 64)

// Three BF16 parts of an FP32 value: v = hi + mid + lo exactly for normal v
// (each part takes the next 8 significant bits, rounded to nearest).
__device__ __forceinline__ void split3(float v, uint16_t* h, uint16_t* m, uint16_t* l) {
  const __nv_bfloat16 a = __float2bfloat16_rn(v);
  const float r1 = v - __bfloat162float(a);
  const __nv_bfloat16 b = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(b);
  *h = __bfloat16_as_ushort(a);
  *m = __bfloat16_as_ushort(b);
  *l = __bfloat16_as_ushort(__float2bfloat16_rn(r2));
}

// Centre of the operand: the mean of each of the first 64 permuted columns
// of the FP32 data (any fixed vector works; this one keeps the centred
// values, and the cancellation in ||xc||^2 + ||qc||^2 - 2 xc.qc, small).
static __global__ void r0_centre_kernel(const float* __restrict__ X, int64_t n, int m,
                                        const int32_t* __restrict__ jperm, int cols, float* __restrict__ mu) {
  const int t = threadIdx.x;
  if (t >= cols) return;
  const int j = jperm[t];
  float s = 0.0f;
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) s += __ldg(X + (size_t)i * m + j);
  atomicAdd(&mu[t], s);
}

// Operand rows [hi | mid | lo] (64 columns each) of v - mu, v the value of the
// gathered copy at permuted column t (dequantised for FP8), zero past m and
// for padding rows.
template <int Storage>
static __global__ void r0_operand_kernel(const void* __restrict__ G, const float* __restrict__ scale8, int64_t n,
                                         int64_t rows_pad, int m, int mp, const float* __restrict__ mu,
                                         uint16_t* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows_pad * kR0Cols) return;
  const int64_t i = e / kR0Cols;
  const int t = (int)(e - i * kR0Cols);
  float v = 0.0f;
  if (i < n && t < m) {
    float x;
    if (Storage == KNN_STORE_F32) {
      x = __ldg(static_cast<const float*>(G) + (size_t)i * mp + t);
    } else if (Storage == KNN_STORE_BF16) {
      x = __uint_as_float((uint32_t)__ldg(static_cast<const uint16_t*>(G) + (size_t)i * mp + t) << 16);
    } else {
      __nv_fp8_e4m3 f;
      f.__x = __ldg(static_cast<const uint8_t*>(G) + (size_t)i * mp + t);
      x = __fmul_rn(static_cast<float>(f), __ldg(scale8 + i));
    }
    v = x - mu[t];
  }
  uint16_t h, md, l;
  split3(v, &h, &md, &l);
  uint16_t* o = out + (size_t)i * 3 * kR0Cols;
  o[t] = h;
  o[kR0Cols + t] = md;
  o[2 * kR0Cols + t] = l;
}

knn_status build_round0_operand(knn_dataset* ds, int storage, cudaStream_t stream) {
  const int64_t n = ds->n;
  const int64_t rows_pad = (n + kTcM - 1) / kTcM * kTcM;
  knn_status s = KNN_OK;
  if (!ds->r0mu) {
    s = cuda_check(cudaMalloc(&ds->r0mu, kR0Cols * 4), "cudaMalloc(round-0 centre)");
    if (s == KNN_OK) s = cuda_check(cudaMemsetAsync(ds->r0mu, 0, kR0Cols * 4, stream), "memset");
    if (s != KNN_OK) return s;
    DeviceInfo di;
    s = device_info(&di);
    if (s != KNN_OK) return s;
    const int cols = std::min(kR0Cols, ds->m);
    r0_centre_kernel<<<di.sms * 4, kR0Cols, 0, stream>>>(ds->X, n, ds->m, ds->jperm, cols, ds->r0mu);
    scale_kernel<<<1, kR0Cols, 0, stream>>>(ds->r0mu, kR0Cols, 1.0f / (float)n);
    s = cuda_check(cudaGetLastError(), "round-0 centre");
    if (s != KNN_OK) return s;
  }
  if (!ds->r0op[storage])
    s = cuda_check(cudaMalloc(&ds->r0op[storage], (size_t)rows_pad * 3 * kR0Cols * 2), "cudaMalloc(round-0 operand)");
  if (s != KNN_OK) return s;
  const int64_t count = rows_pad * kR0Cols;
  const unsigned blocks = (unsigned)((count + 255) / 256);
  if (storage == KNN_STORE_F32)
    r0_operand_kernel<KNN_STORE_F32><<<blocks, 256, 0, stream>>>(ds->p32, ds->scale8, n, rows_pad, ds->m, ds->mp,
                                                                 ds->r0mu, ds->r0op[storage]);
  else if (storage == KNN_STORE_BF16)
    r0_operand_kernel<KNN_STORE_BF16><<<blocks, 256, 0, stream>>>(ds->pb, ds->scale8, n, rows_pad, ds->m, ds->mp,
                                                                  ds->r0mu, ds->r0op[storage]);
  else
    r0_operand_kernel<KNN_STORE_FP8><<<blocks, 256, 0, stream>>>(ds->p8, ds->scale8, n, rows_pad, ds->m, ds->mp,
                                                                 ds->r0mu, ds->r0op[storage]);
  return cuda_check(cudaGetLastError(), "round-0 operand");
}

// Query side: rows [hi | mid | lo] of q_(jperm t) - mu_t for t < B0 (zero past
// B0 and for padding rows), and ||qc||^2 over those B0 columns (FP32, the
// parts summed back exactly).
static __global__ void r0_query_kernel(const float* __restrict__ Q, int nq, int64_t nq_pad, int m,
                                       const int32_t* __restrict__ jperm, const float* __restrict__ mu, int B0,
                                       uint16_t* __restrict__ out, float* __restrict__ qn) {
  const int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (q >= nq_pad) return;
  float sq = 0.0f;
  for (int t = lane; t < kR0Cols; t += 32) {
    float v = 0.0f;
    if (q < nq && t < B0) v = __ldg(Q + (size_t)q * m + jperm[t]) - mu[t];
    uint16_t h, md, l;
    split3(v, &h, &md, &l);
    uint16_t* o = out + (size_t)q * 3 * kR0Cols;
    o[t] = h;
    o[kR0Cols + t] = md;
    o[2 * kR0Cols + t] = l;
    sq = fmaf(v, v, sq);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
  if (lane == 0 && q < nq) qn[q] = sq;
}

// ||xc||^2 over the first B0 permuted columns of each point, from its parts.
static __global__ void r0_point_norms_kernel(const uint16_t* __restrict__ op, int64_t n, int B0,
                                             float* __restrict__ xn) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint16_t* o = op + (size_t)i * 3 * kR0Cols;
  float s = 0.0f;
  for (int t = 0; t < B0; ++t) {
    const float v = (__uint_as_float((uint32_t)o[t] << 16) + __uint_as_float((uint32_t)o[kR0Cols + t] << 16)) +
                    __uint_as_float((uint32_t)o[2 * kR0Cols + t] << 16);
    s = fmaf(v, v, s);
  }
  xn[i] = s;
}

static __global__ void fill_kernel(float* p, float v) { *p = v; }

struct R0Carve {
  uint16_t* B;
  float* qn;
  float* xn;
  float* c2;
};

static size_t carve_r0(Carve& cv, int64_t n, int32_t nq, R0Carve* out) {
  R0Carve c;
  const size_t nq_pad = (size_t)((nq + kTcN - 1) / kTcN) * kTcN;
  c.B = cv.take<uint16_t>(nq_pad * 3 * kR0Cols);
  c.qn = cv.take<float>(nq_pad);
  c.xn = cv.take<float>((size_t)n);
  c.c2 = cv.take<float>(1);
  if (out) *out = c;
  return cv.off;
}

size_t round0_tc_scratch(int64_t n, int32_t nq) {
  Carve cv;
  return carve_r0(cv, n, nq, nullptr) + 256;
}

knn_status round0_tc(const knn_dataset* ds, int storage, const float* Q, int32_t nq, int32_t B0, float* R0,
                     float* R0min, int32_t r0tiles, void* scratch, cudaStream_t stream) {
  const uint16_t* A = ds->r0op[storage];
  if (!A || !ds->r0mu) return set_error("round0_tc: no round-0 operand for this storage"), KNN_EINVAL;
  if (B0 < 1 || B0 > kR0Cols) return set_error("round0_tc: needs 1 <= B0 <= 64"), KNN_EINVAL;
  DeviceInfo di;
  knn_status s = device_info(&di);
  if (s != KNN_OK) return s;
  const int64_t n = ds->n;
  const int64_t npt = (n + kTcM - 1) / kTcM;
  const int64_t nq_pad = (int64_t)((nq + kTcN - 1) / kTcN) * kTcN;
  Carve cv;
  cv.base = reinterpret_cast<uint8_t*>(((uintptr_t)scratch + 255) & ~uintptr_t(255));
  R0Carve c;
  carve_r0(cv, n, nq, &c);
  r0_query_kernel<<<(unsigned)((nq_pad + 7) / 8), 256, 0, stream>>>(Q, nq, nq_pad, ds->m, ds->jperm, ds->r0mu, B0,
                                                                    c.B, c.qn);
  r0_point_norms_kernel<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(A, n, B0, c.xn);
  fill_kernel<<<1, 1, 0, stream>>>(c.c2, -2.0f);
  s = cuda_check(cudaGetLastError(), "round-0 operand kernels");
  CUtensorMap mapA, mapB;
  if (s == KNN_OK) s = make_map(&mapA, A, npt * kTcM, 3 * kR0Cols, kTcM, true);
  if (s == KNN_OK) s = make_map(&mapB, c.B, nq_pad, 3 * kR0Cols, kTcN, true);
  int* status = nullptr;
  if (s == KNN_OK) s = device_status_ptr(&status);
  const size_t smem = screen_smem_bytes();
  if (s == KNN_OK)
    s = cuda_check(cudaFuncSetAttribute(screen_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                   "cudaFuncSetAttribute(screen_tc)");
  if (s != KNN_OK) return s;
  ScreenArgs a{};
  a.n = n;
  a.nq = nq;
  // xc.qc from the parts: hi.hi, hi.mid, hi.lo, mid.hi, mid.mid, lo.hi (the
  // three dropped products are below 2^-26 |xc| |qc| together)
  const int8_t akb[6] = {0, 0, 0, 1, 1, 2}, bkb[6] = {0, 1, 2, 0, 1, 0};
  a.nk = 6;
  for (int i = 0; i < 6; ++i) {
    a.akb[i] = akb[i];
    a.bkb[i] = bkb[i];
  }
  a.ksteps = (B0 + 15) / 16;
  a.nqt = (int)(nq_pad / kTcN);
  a.stride = 1;
  a.ntiles = (int)(npt * a.nqt);
  a.pass = 3;
  a.idesc = idesc_f16kind(true);
  a.limit = g_wait_limit.load();
  a.xn = c.xn;
  a.qn = c.qn;
  a.c2 = c.c2;
  a.gmin = R0min;
  a.nunits = r0tiles;
  a.r0 = R0;
  a.status = status;
  screen_tc_kernel<<<std::min(a.ntiles, di.sms), kTcThreads, smem, stream>>>(mapA, mapB, a);
  return cuda_check(cudaGetLastError(), "screen_tc_kernel launch (round 0)");
}

}  // namespace knn

// Tries of the tensor-core kernels' pipeline waits before they give up.
extern "C" knn_status knn_debug_wait_limit(int64_t tries) {
  knn::clear_error();
  knn::g_wait_limit.store(tries < 0 ? knn::kSpinDefault : (uint32_t)std::min<int64_t>(tries, 0xFFFFFFFFll));
  return KNN_OK;
}
