// screen_tc.cu -- the naive exact method's screen as a tcgen05 tensor-core
// GEMM (Section 3: all distances, then select; the select and the FP64 rerank
// are in exact.cu and rerank.cu).
//
// Distances are translation invariant, so the data is centred on its column
// mean mu once (xc = x - mu) and each centred value is split into two BF16
// parts, xc = hi + lo + r with |r| <= 2^-18 |xc|. One BF16 GEMM over the
// concatenated rows [hi | hi | lo] . [qhi | qlo | qhi] then gives
// hi.qhi + hi.qlo + lo.qhi, the product of the centred vectors up to
// 3.1 * 2^-18 sum|xc||qc| plus the accumulation error; the screened distance
// is ||xc||^2 + ||qc||^2 - 2 xc.qc and its error bound is applied by the
// select kernel.
//
// GEMM: one CTA per 128-point x 256-query tile, 128 threads, two CTAs per
// SM (about 97 KB of shared memory and 256 TMEM columns each, so one CTA's
// epilogue overlaps the other's main loop). Warp 0 lane 0 issues TMA loads
// (128-byte swizzle, 64 K-elements per stage, 2 stages),
// warp 1 lane 0 issues tcgen05.mma (M=128, N=256, K=16, BF16 x BF16 -> FP32
// in TMEM) and commits each stage back to the producer; all four warps then
// read their 32 TMEM lanes (tcgen05.ld 32x32b) and write the screened values.
// Every mbarrier wait is bounded; a wait that gives up records an error in
// the library status word and the CTA still frees its TMEM before it exits.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <mutex>
#include <string>

#include "knn_common.cuh"
#include "knn_internal.h"

namespace knn {

knn_status launch_rerank(const float* X, int64_t n, int32_t m, const float* Q, int32_t nq, const int64_t* cand,
                         int32_t ncand, int32_t k, int64_t* out_idx, double* out_dist, cudaStream_t stream,
                         int32_t metric = KNN_METRIC_L2SQ);
knn_status launch_screen_select(float* D, int64_t n, int32_t nq, int32_t m, int32_t k, const float* qn,
                                const unsigned* xn_max_bits, double c_cross, double c_square, const float* X,
                                const float* Q, int64_t* cand,
                                cudaStream_t stream);
constexpr int kExactCandTc = 2048;

constexpr int kTcM = 128, kTcN = 256, kTcK = 64, kTcStages = 2, kTcThreads = 128;
constexpr int kTcABytes = kTcM * kTcK * 2;  // 16 KB
constexpr int kTcBBytes = kTcN * kTcK * 2;  // 32 KB
constexpr uint32_t kSpinLimit = 1u << 26;
constexpr int kStatusTimeout = 0x5C7C;      // recorded when a bounded wait gives up

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
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
// Waits for the phase of `parity` to complete; false after kSpinLimit tries.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (uint32_t i = 0; i < kSpinLimit; ++i)
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

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N = 256, M = 128.
constexpr uint32_t kIdescBf16 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                                ((uint32_t)(kTcM >> 4) << 24);

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(kIdescBf16), "r"(accum)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tmem_ld_x16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__global__ void __launch_bounds__(kTcThreads, 2)
    screen_tc_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int64_t n,
                     int nq, int Kt, const float* __restrict__ xn, const float* __restrict__ qn, float* __restrict__ D,
                     int* status) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;
  uint8_t* sB = smem + kTcStages * kTcABytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sB + kTcStages * kTcBBytes);  // full[S], empty[S], done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kTcStages + 1);
  int* cta_err = reinterpret_cast<int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q0 = blockIdx.x * kTcN;
  const int64_t p0 = (int64_t)blockIdx.y * kTcM;
  const int nk = Kt / kTcK;
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + kTcStages), done = smem_u32(bars + 2 * kTcStages);

  if (threadIdx.x == 0) {
    for (int s = 0; s < kTcStages; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(done, 1);
    *cta_err = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTcN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  int issued = 0;
  if (warp == 0 && lane == 0) {  // TMA producer
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % kTcStages;
      const uint32_t ph = (uint32_t)(kb / kTcStages) & 1u;
      if (!mbar_wait(empty0 + 8 * s, ph ^ 1u)) {
        *cta_err = 1;
        break;
      }
      mbar_expect_tx(full0 + 8 * s, kTcABytes + kTcBBytes);
      tma_load_2d(smem_u32(sA + s * kTcABytes), &mapA, full0 + 8 * s, kb * kTcK, (int)p0);
      tma_load_2d(smem_u32(sB + s * kTcBBytes), &mapB, full0 + 8 * s, kb * kTcK, q0);
      issued = kb + 1;
    }
  } else if (warp == 1 && lane == 0) {  // MMA issuer
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % kTcStages;
      const uint32_t ph = (uint32_t)(kb / kTcStages) & 1u;
      if (!mbar_wait(full0 + 8 * s, ph)) {
        *cta_err = 1;
        break;
      }
      tc_fence_after();
      const uint64_t ad = sw128_kmajor_desc(smem_u32(sA + s * kTcABytes));
      const uint64_t bd = sw128_kmajor_desc(smem_u32(sB + s * kTcBBytes));
#pragma unroll
      for (int ks = 0; ks < kTcK / 16; ++ks)  // 16 BF16 = 32 bytes per step along K
        umma_bf16(tmem, ad + 2 * ks, bd + 2 * ks, (kb | ks) != 0);
      umma_commit(empty0 + 8 * s);
    }
    umma_commit(done);
  }
  __syncwarp();

  // ---- epilogue: lanes of TMEM are the tile's 128 points, columns its queries
  const bool ok = mbar_wait(done, 0);
  tc_fence_after();
  const int row = warp * 32 + lane;
  const int64_t p = p0 + row;
  const float xv = (p < n) ? xn[p] : 0.0f;
  for (int c0 = 0; c0 < kTcN; c0 += 16) {
    float v[16];
    tmem_ld_x16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
    if (ok && p < n) {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int q = q0 + c0 + j;
        if (q < nq) D[(size_t)q * n + p] = (xv + qn[q]) - 2.0f * v[j];
      }
    }
  }
  if (!ok) *cta_err = 1;
  tc_fence_before();
  __syncthreads();
  if (*cta_err) {
    if (threadIdx.x == 0) atomicExch(status, kStatusTimeout);
    // let the copies this CTA issued land before its shared memory is released
    if (warp == 0 && lane == 0)
      for (int kb = (issued > kTcStages ? issued - kTcStages : 0); kb < issued; ++kb)
        mbar_wait(full0 + 8 * (kb % kTcStages), (uint32_t)(kb / kTcStages) & 1u);
  }
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcN));
  }
}

// ---- operand preparation

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

// Rows of the screen operand: [hi | hi | lo] (dataset side, second = false)
// or [hi | lo | hi] (query side, second = true) of x - mu, each Kp wide and
// zero padded; norms[r] = ||x - mu||^2 (FP32), max_bits its largest value.
static __global__ void split_rows_kernel(const float* __restrict__ X, int64_t rows, int64_t rows_pad, int m, int Kp,
                                         const float* __restrict__ mu, bool query_side, uint16_t* __restrict__ out,
                                         float* __restrict__ norms, unsigned* max_bits) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  unsigned mx = 0;
  for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < rows_pad; r += warps) {
    uint16_t* o = out + (size_t)r * 3 * Kp;
    float s = 0.0f;
    for (int j = lane; j < Kp; j += 32) {
      uint16_t hb = 0, lb = 0;
      if (r < rows && j < m) {
        const float xc = __ldg(X + (size_t)r * m + j) - mu[j];
        const __nv_bfloat16 h = __float2bfloat16_rn(xc);
        const float hf = __bfloat162float(h);
        const __nv_bfloat16 l = __float2bfloat16_rn(xc - hf);
        hb = __bfloat16_as_ushort(h);
        lb = __bfloat16_as_ushort(l);
        s = fmaf(xc, xc, s);
      }
      o[j] = hb;
      o[Kp + j] = query_side ? lb : hb;
      o[2 * Kp + j] = query_side ? hb : lb;
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

// 2-D BF16 tensor map over rows x Kt (row pitch Kt elements), box 64 x box_rows,
// 128-byte swizzle; rows beyond the tensor read as zero.
static knn_status make_map(CUtensorMap* map, const void* base, int64_t rows, int Kt, int box_rows) {
  EncodeTiled enc;
  knn_status s = get_encoder(&enc);
  if (s != KNN_OK) return s;
  cuuint64_t dims[2] = {(cuuint64_t)Kt, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)Kt * 2};
  cuuint32_t box[2] = {(cuuint32_t)kTcK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return KNN_ECUDA;
  }
  return KNN_OK;
}

static size_t screen_smem_bytes() {
  return 1024 + (size_t)kTcStages * (kTcABytes + kTcBBytes) + (2 * kTcStages + 1) * 8 + 16;
}

// Builds the dataset's screen operand (called by knn_dataset_create).
knn_status build_screen_operand(knn_dataset* ds, cudaStream_t stream) {
  const int64_t n = ds->n;
  const int m = ds->m;
  ds->Kp = (m + kTcK - 1) / kTcK * kTcK;
  const size_t rows_pad = (size_t)((n + kTcM - 1) / kTcM) * kTcM;
  knn_status s = cuda_check(cudaMalloc(&ds->screenA, rows_pad * 3 * (size_t)ds->Kp * 2), "cudaMalloc(screen operand)");
  if (s == KNN_OK) s = cuda_check(cudaMalloc(&ds->mu, (size_t)m * 4), "cudaMalloc(mu)");
  if (s == KNN_OK) s = cuda_check(cudaMalloc(&ds->xcn, (size_t)n * 4), "cudaMalloc(norms)");
  if (s == KNN_OK) s = cuda_check(cudaMalloc(&ds->xcn_max, 4), "cudaMalloc(norm max)");
  if (s == KNN_OK) s = cuda_check(cudaMemsetAsync(ds->mu, 0, (size_t)m * 4, stream), "memset");
  if (s == KNN_OK) s = cuda_check(cudaMemsetAsync(ds->xcn_max, 0, 4, stream), "memset");
  if (s != KNN_OK) return s;
  DeviceInfo di;
  s = device_info(&di);
  if (s != KNN_OK) return s;
  column_sums_kernel<<<di.sms * 4, 256, 0, stream>>>(ds->X, n, m, ds->mu);
  scale_kernel<<<(m + 255) / 256, 256, 0, stream>>>(ds->mu, m, 1.0f / (float)n);
  split_rows_kernel<<<di.sms * 8, 256, 0, stream>>>(ds->X, n, (int64_t)rows_pad, m, ds->Kp, ds->mu, false,
                                                     ds->screenA, ds->xcn, ds->xcn_max);
  return cuda_check(cudaGetLastError(), "screen operand kernels");
}

struct TcCarve {
  uint16_t* B;
  float* qn;
  float* D;
  int64_t* cand;
};

static size_t carve_tc(Carve& cv, int64_t n, int32_t nq, int Kp, TcCarve* out) {
  TcCarve c;
  const size_t nq_pad = (size_t)((nq + kTcN - 1) / kTcN) * kTcN;
  c.B = cv.take<uint16_t>(nq_pad * 3 * (size_t)Kp);
  c.qn = cv.take<float>(nq_pad);
  c.D = cv.take<float>((size_t)nq * (size_t)n);
  c.cand = cv.take<int64_t>((size_t)nq * kExactCandTc);
  if (out) *out = c;
  return cv.off;
}

size_t exact_tc_workspace(int64_t n, int32_t m, int32_t nq) {
  Carve cv;
  return carve_tc(cv, n, nq, (m + kTcK - 1) / kTcK * kTcK, nullptr) + 256;
}

knn_status exact_tc(const knn_dataset* ds, const float* Q, int32_t nq, int32_t k, int64_t* out_idx,
                    double* out_dist, void* workspace, size_t workspace_bytes, cudaStream_t stream) {
  if (!ds->screenA) {
    set_error("knn_exact_ds: the dataset was created without the tensor-core screen operand");
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
  const int m = ds->m, Kp = ds->Kp, Kt = 3 * Kp;
  const size_t need = exact_tc_workspace(n, m, nq);
  Workspace ws;
  s = ws.acquire(workspace, workspace_bytes, need, stream);
  if (s != KNN_OK) return s;
  Carve cv;
  cv.base = reinterpret_cast<uint8_t*>(((uintptr_t)ws.ptr + 255) & ~uintptr_t(255));
  TcCarve c;
  carve_tc(cv, n, nq, Kp, &c);
  const int64_t nq_pad = (int64_t)((nq + kTcN - 1) / kTcN) * kTcN;
  split_rows_kernel<<<(int)std::min<int64_t>((nq_pad + 7) / 8, (int64_t)di.sms * 8), 256, 0, stream>>>(
      Q, nq, nq_pad, m, Kp, ds->mu, true, c.B, c.qn, nullptr);
  s = cuda_check(cudaGetLastError(), "query split kernel");
  CUtensorMap mapA, mapB;
  if (s == KNN_OK) s = make_map(&mapA, ds->screenA, (n + kTcM - 1) / kTcM * kTcM, Kt, kTcM);
  if (s == KNN_OK) s = make_map(&mapB, c.B, nq_pad, Kt, kTcN);
  int* status = nullptr;
  if (s == KNN_OK) s = device_status_ptr(&status);
  if (s == KNN_OK) {
    const size_t smem = screen_smem_bytes();
    s = cuda_check(cudaFuncSetAttribute(screen_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                   "cudaFuncSetAttribute(screen_tc)");
    if (s == KNN_OK) {
      dim3 grid((unsigned)(nq_pad / kTcN), (unsigned)((n + kTcM - 1) / kTcM));
      screen_tc_kernel<<<grid, kTcThreads, smem, stream>>>(mapA, mapB, n, nq, Kt, ds->xcn, c.qn, c.D, status);
      s = cuda_check(cudaGetLastError(), "screen_tc_kernel launch");
    }
  }
  if (s == KNN_OK) {
    // Error bound of a screened value (u = 2^-24): the K-concatenated product
    // misses at most 3.1 * 2^-18 sum|xc||qc| from the split, and its FP32
    // tensor-core accumulation over Kt terms is bounded by (Kt + 16) 2^-22
    // sum|terms| (two units of the last place per term, covering truncating
    // adders); sum|xc||qc| <= ||xc|| ||qc||. The centred norms are FP32 sums
    // over m terms (gamma_m), and the final additions and the centring cost a
    // few units of roundoff of (||xc|| + ||qc||)^2. A factor 1.5 covers
    // second-order terms.
    const double u = 1.0 / 16777216.0;
    const double gacc = (double)(Kt + 16) * 4.0 * u;
    const double gm = (double)(m + 2) * u / (1.0 - (double)(m + 2) * u);
    const double c_cross = 1.5 * 2.0 * (gacc + 3.1 * 64.0 * u) * 1.01;
    const double c_square = 1.5 * (gm + 6.0 * u);
    s = launch_screen_select(c.D, n, nq, m, k, c.qn, ds->xcn_max, c_cross, c_square, ds->X, Q, c.cand, stream);
  }
  if (s == KNN_OK) s = launch_rerank(ds->X, n, m, Q, nq, c.cand, kExactCandTc, k, out_idx, out_dist, stream);
  ws.release();
  return s;
}

}  // namespace knn
