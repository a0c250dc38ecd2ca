// exact.cu -- the naive exact k-NN method the paper compares against
// (Section 3: compute all distances, then select), as
//   screen   D~[q,i] = ||x_i||^2 + ||q||^2 - 2 x_i.q  (a GEMM, FP32 here)
//   select   per query, the k-th smallest screened value tau~ and every
//            point with D~ <= tau~ + 2E_q, E_q a proven bound on the screen's
//            rounding error for that query
//   rerank   exact FP64 distances of those candidates, top-k by (d, index).
// The candidate rule is exact: k points have D~ <= tau~, so the k-th true
// distance is at most tau~ + E_q, and every true k-nearest point j has
// D~_j <= d_j + E_q <= tau~ + 2 E_q.
#include <cfloat>
#include <cmath>

#include "knn_common.cuh"
#include "knn_internal.h"

namespace knn {

knn_status launch_rerank(const float* X, int64_t n, int32_t m, const float* Q, int32_t nq, const int64_t* cand,
                         int32_t ncand, int32_t k, int64_t* out_idx, double* out_dist, cudaStream_t stream,
                         int32_t metric = KNN_METRIC_L2SQ);
size_t exact_tc_workspace(int64_t n, int32_t m, int32_t nq, int32_t screen);
knn_status exact_tc(const knn_dataset* ds, int32_t screen, const float* Q, int32_t nq, int32_t k, int64_t* out_idx,
                    double* out_dist, void* workspace, size_t workspace_bytes, cudaStream_t stream);

constexpr int kExactCand = 2048;  // candidate slots per query before falling back to a full scan

// Squared norms of rows (FP32, one warp per row) and the largest of them.
__global__ void row_norms_kernel(const float* __restrict__ A, int64_t rows, int m, float* __restrict__ out,
                                 unsigned* max_bits) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  unsigned mx = 0;
  for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < rows; r += warps) {
    const float* ar = A + (size_t)r * m;
    float s = 0.0f;
    for (int j = lane; j < m; j += 32) {
      const float v = __ldg(ar + j);
      s = fmaf(v, v, s);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      out[r] = s;
      mx = max(mx, __float_as_uint(s));
    }
  }
  if (lane == 0 && max_bits) atomicMax(max_bits, mx);
}

// FP32 SIMT screen: D[q*n + i] = xn[i] + qn[q] - 2 sum_j X[i,j] Q[q,j]
// (L1: D[q*n + i] = sum_j |X[i,j] - Q[q,j]|, each term and the sum in FP32,
// in coordinate order). 128 x 128 tile (points x queries), k-step 8, 256
// threads with 8 x 8 outputs each, double-buffered shared memory.
constexpr int kBM = 128, kBN = 128, kBK = 8;

template <bool L1>
__global__ void __launch_bounds__(256) screen_sgemm_kernel(const float* __restrict__ X, const float* __restrict__ Q,
                                                           int64_t n, int nq, int m, const float* __restrict__ xn,
                                                           const float* __restrict__ qn, float* __restrict__ D) {
  __shared__ __align__(16) float As[2][kBK][kBM];
  __shared__ __align__(16) float Bs[2][kBK][kBN];
  const int tid = threadIdx.x;
  const int64_t p0 = (int64_t)blockIdx.x * kBM;
  const int q0 = blockIdx.y * kBN;
  // loader: each thread brings 4 consecutive k of one row of each operand
  const int lrow = tid >> 1, lk = (tid & 1) * 4;
  const int64_t arow = p0 + lrow;
  const int brow = q0 + lrow;
  const bool aok = arow < n, bok = brow < nq;
  const float* ap = X + (size_t)(aok ? arow : 0) * m;
  const float* bp = Q + (size_t)(bok ? brow : 0) * m;
  const int tp = tid & 15, tq = tid >> 4;
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;

  auto load = [&](int kb, float ra[4], float rb[4]) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int kk = kb + lk + e;
      ra[e] = (aok && kk < m) ? __ldg(ap + kk) : 0.0f;
      rb[e] = (bok && kk < m) ? __ldg(bp + kk) : 0.0f;
    }
  };
  float ra[4], rb[4];
  load(0, ra, rb);
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    As[0][lk + e][lrow] = ra[e];
    Bs[0][lk + e][lrow] = rb[e];
  }
  __syncthreads();
  int buf = 0;
  for (int kb = 0; kb < m; kb += kBK) {
    const bool more = kb + kBK < m;
    if (more) load(kb + kBK, ra, rb);
#pragma unroll
    for (int kk = 0; kk < kBK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][tp * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + tp * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tq * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 + tq * 4]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if constexpr (L1)
            acc[i][j] += fabsf(av[i] - bv[j]);
          else
            acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
    }
    if (more) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        As[buf ^ 1][lk + e][lrow] = ra[e];
        Bs[buf ^ 1][lk + e][lrow] = rb[e];
      }
    }
    __syncthreads();
    buf ^= 1;
  }
  // epilogue: point i = p0 + {tp*4 + e, 64 + tp*4 + e}, query q = q0 + {tq*4 + e, 64 + tq*4 + e}
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int q = q0 + (j < 4 ? tq * 4 + j : 64 + tq * 4 + (j - 4));
    if (q >= nq) continue;
    float* drow = D + (size_t)q * n;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int64_t p = p0 + (i < 4 ? tp * 4 + i : 64 + tp * 4 + (i - 4));
      if (p >= n) continue;
      if constexpr (L1)
        drow[p] = acc[i][j];
      else
        drow[p] = (xn[p] + qn[q]) - 2.0f * acc[i][j];
    }
  }
}

// Per query: k-th smallest screened value, then every point within 2 E_q of
// it into cand[q, 0..kExactCand) (-1 padded). E_q is the screen's error bound
// for the query: c_cross ||x||max ||q|| + c_square (||x||max + ||q||)^2,
// with the norms of the vectors the screen multiplied (FP32 sums, inflated by
// their own rounding bound). When that window holds more points than the
// list (clustered data: the bound scales with the norms, not with the
// distances), a second screen takes the window's distances directly in FP32,
// sum of (x_j - q_j)^2, whose error is at most rel = gamma_(m+4) times the
// distance itself: with tau32 the k-th smallest of them, every point whose
// distance is at most the k-th true one has d32 <= tau32 (1 + rel)/(1 - rel).
// A row that still does not fit is marked -2 (rerank then scans every point).
constexpr int kSelNT = 512;

__global__ void __launch_bounds__(kSelNT) screen_select_kernel(float* __restrict__ D, int64_t n, int m, int k,
                                                               const float* __restrict__ qn,
                                                               const unsigned* __restrict__ xn_max_bits,
                                                               float c_cross, float c_square,
                                                               const float* __restrict__ X,
                                                               const float* __restrict__ Q,
                                                               int64_t* __restrict__ cand) {
  __shared__ uint32_t hist[kHistBins];
  __shared__ uint32_t buf[kSelCap];
  __shared__ BlockScratch<kSelNT> bs;
  __shared__ SelectShared ss;
  __shared__ int cnt;
  const int q = blockIdx.x;
  float* dr = D + (size_t)q * n;
  for (int i = threadIdx.x; i < kHistBins; i += kSelNT) hist[i] = 0;
  __syncthreads();
  for (int64_t i = threadIdx.x; i < n; i += kSelNT) atomicAdd(&hist[f2key(__ldg(dr + i)) >> 20], 1u);
  __syncthreads();
  select_smallest<kSelNT>([&](int i) { return f2key(__ldg(dr + i)); }, (int)n, k, hist, buf, ss, bs);
  const float tau = key2f(buf[k - 1]);
  const float u = 1.0f / 16777216.0f;
  float thr;
  const bool relative = c_cross < 0.0f;  // screened values within a relative error -c_cross of the distances
  if (relative) {
    const float r = -c_cross;
    thr = tau * ((1.0f + r) / (1.0f - r)) * (1.0f + 4.0f * u);
  } else {
    // FP32 arithmetic on non-negative terms: a few units of roundoff, covered
    // by the factor 1.001 (the coefficients carry their own margins)
    const float gm = (float)(m + 2) * u / (1.0f - (float)(m + 2) * u);
    const float xmax = sqrtf(__uint_as_float(*xn_max_bits) * (1.0f + gm));
    const float qq = sqrtf(qn[q] * (1.0f + gm));
    const float E = 1.001f * (c_cross * xmax * qq + c_square * (xmax + qq) * (xmax + qq));
    thr = (tau + 2.0f * E) * (1.0f + 4.0f * u);
  }
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  int64_t* cr = cand + (size_t)q * kExactCand;
  for (int64_t i = threadIdx.x; i < n; i += kSelNT) {
    if (__ldg(dr + i) <= thr) {
      const int p = atomicAdd(&cnt, 1);
      if (p < kExactCand) cr[p] = i;
    }
  }
  __syncthreads();
  int c = cnt;
  if (c > kExactCand && !relative) {
    // second screen: direct FP32 distances of the window, one warp per point
    // (the screened row is scratch: window points get d32, the others +inf)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float* qr = Q + (size_t)q * m;
    for (int i = threadIdx.x; i < kHistBins; i += kSelNT) hist[i] = 0;
    __syncthreads();
    for (int64_t base = (int64_t)warp * 32; base < n; base += (int64_t)(kSelNT / 32) * 32) {
      const int64_t i = base + lane;
      const bool win = i < n && dr[i] <= thr;
      unsigned bal = __ballot_sync(0xffffffffu, win);
      if (i < n && !win) {
        dr[i] = INFINITY;
        atomicAdd(&hist[f2key(INFINITY) >> 20], 1u);
      }
      while (bal) {
        const int src = __ffs(bal) - 1;
        bal &= bal - 1;
        const float* xr = X + (size_t)(base + src) * m;
        float acc = 0.0f;
        for (int j = lane; j < m; j += 32) {
          const float t = __ldg(xr + j) - __ldg(qr + j);
          acc = fmaf(t, t, acc);
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == src) {
          dr[i] = acc;
          atomicAdd(&hist[f2key(acc) >> 20], 1u);
        }
      }
    }
    __syncthreads();
    select_smallest<kSelNT>([&](int i) { return f2key(dr[i]); }, (int)n, k, hist, buf, ss, bs);
    const float tau32 = key2f(buf[k - 1]);
    const float rel = (float)(m + 4) * u / (1.0f - (float)(m + 4) * u);
    const float thr2 = tau32 * ((1.0f + rel) / (1.0f - rel)) * (1.0f + 4.0f * u);
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    for (int64_t i = threadIdx.x; i < n; i += kSelNT) {
      if (dr[i] <= thr2) {
        const int p = atomicAdd(&cnt, 1);
        if (p < kExactCand) cr[p] = i;
      }
    }
    __syncthreads();
    c = cnt;
  }
  if (c > kExactCand) {
    for (int t = threadIdx.x; t < kExactCand; t += kSelNT) cr[t] = t == 0 ? -2 : -1;
  } else {
    for (int t = c + threadIdx.x; t < kExactCand; t += kSelNT) cr[t] = -1;
  }
}

knn_status launch_screen_select(float* D, int64_t n, int32_t nq, int32_t m, int32_t k, const float* qn,
                                const unsigned* xn_max_bits, double c_cross, double c_square, const float* X,
                                const float* Q, int64_t* cand, cudaStream_t stream) {
  screen_select_kernel<<<nq, kSelNT, 0, stream>>>(D, n, m, k, qn, xn_max_bits, (float)c_cross, (float)c_square, X,
                                                  Q, cand);
  return cuda_check(cudaGetLastError(), "screen_select_kernel launch");
}

// SIMT screen bound: the dot product and both norms are length-m FP32 sums
// (gamma_m times the sum of magnitudes), plus two final roundings, all
// bounded by (||x|| + ||q||)^2; a factor 2 covers second-order terms.
static double simt_c_square(int m) {
  const double u = 1.0 / 16777216.0;
  const double gm = (double)(m + 2) * u / (1.0 - (double)(m + 2) * u);
  return 2.0 * (gm + 4.0 * u);
}

struct ExactCarve {
  float* xn;
  float* qn;
  unsigned* xmax;
  float* D;
  int64_t* cand;
};

static size_t carve_exact(Carve& cv, int64_t n, int32_t nq, ExactCarve* out) {
  ExactCarve c;
  c.xn = cv.take<float>((size_t)n);
  c.qn = cv.take<float>((size_t)nq);
  c.xmax = cv.take<unsigned>(1);
  c.D = cv.take<float>((size_t)nq * (size_t)n);
  c.cand = cv.take<int64_t>((size_t)nq * kExactCand);
  if (out) *out = c;
  return cv.off;
}

}  // namespace knn

using namespace knn;

extern "C" size_t knn_exact_workspace_size(int64_t n, int32_t m, int32_t nq, int32_t k) {
  (void)m;
  (void)k;
  Carve cv;
  return carve_exact(cv, n, nq, nullptr) + 256;
}

extern "C" knn_status knn_exact(const float* X, int64_t n, int32_t m, const float* Q, int32_t nq, int32_t k,
                                int64_t* out_idx, double* out_dist, void* workspace, size_t workspace_bytes,
                                void* stream_) {
  clear_error();
  if (n < 1 || n >= (int64_t)1 << 31 || m < 1 || m > kMaxM || nq < 0 || k < 1 || k > n || k > kMaxKH) {
    set_error("knn_exact: need 1 <= n < 2^31, 1 <= m <= 16384, 1 <= k <= min(n, 1024)");
    return KNN_EINVAL;
  }
  if (nq == 0) return KNN_OK;
  if (!X || !Q || !out_idx || !out_dist) {
    set_error("knn_exact: null pointer");
    return KNN_EINVAL;
  }
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  Carve measure;
  const size_t need = carve_exact(measure, n, nq, nullptr) + 256;
  Workspace ws;
  knn_status s = ws.acquire(workspace, workspace_bytes, need, stream);
  if (s != KNN_OK) return s;
  Carve cv;
  cv.base = reinterpret_cast<uint8_t*>(((uintptr_t)ws.ptr + 255) & ~uintptr_t(255));
  ExactCarve c;
  carve_exact(cv, n, nq, &c);
  DeviceInfo di;
  device_info(&di);
  s = cuda_check(cudaMemsetAsync(c.xmax, 0, 4, stream), "memset");
  if (s == KNN_OK) {
    row_norms_kernel<<<di.sms * 8, 256, 0, stream>>>(X, n, m, c.xn, c.xmax);
    row_norms_kernel<<<(nq + 7) / 8, 256, 0, stream>>>(Q, nq, m, c.qn, nullptr);
    dim3 grid((unsigned)((n + kBM - 1) / kBM), (unsigned)((nq + kBN - 1) / kBN));
    screen_sgemm_kernel<false><<<grid, 256, 0, stream>>>(X, Q, n, nq, m, c.xn, c.qn, c.D);
    s = cuda_check(cudaGetLastError(), "exact kernels launch");
    if (s == KNN_OK)
      s = launch_screen_select(c.D, n, nq, m, k, c.qn, c.xmax, 0.0, simt_c_square(m), X, Q, c.cand, stream);
  }
  if (s == KNN_OK) s = launch_rerank(X, n, m, Q, nq, c.cand, kExactCand, k, out_idx, out_dist, stream);
  ws.release();
  return s;
}

extern "C" size_t knn_exact_ds_workspace_size(const knn_dataset* ds, int32_t screen, int32_t nq) {
  if (!ds) return 0;
  if (screen == KNN_SCREEN_BF16X3 || screen == KNN_SCREEN_F16 || screen == KNN_SCREEN_BF16)
    return exact_tc_workspace(ds->n, ds->m, nq, screen);
  return knn_exact_workspace_size(ds->n, ds->m, nq, 1);
}

extern "C" knn_status knn_exact_ds(const knn_dataset* ds, int32_t screen, const float* Q, int32_t nq, int32_t k,
                                   int64_t* out_idx, double* out_dist, void* workspace, size_t workspace_bytes,
                                   void* stream_) {
  clear_error();
  if (!ds) return set_error("knn_exact_ds: null dataset"), KNN_EINVAL;
  if (k < 1 || k > ds->n || k > kMaxKH || nq < 0)
    return set_error("knn_exact_ds: need 1 <= k <= min(n, 1024), nq >= 0"), KNN_EINVAL;
  if (screen != KNN_SCREEN_F32 && screen != KNN_SCREEN_BF16X3 && screen != KNN_SCREEN_F16 && screen != KNN_SCREEN_BF16)
    return set_error("knn_exact_ds: unknown screen"), KNN_EINVAL;
  if (nq == 0) return KNN_OK;
  if (!Q || !out_idx || !out_dist) return set_error("knn_exact_ds: null pointer"), KNN_EINVAL;
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  if (screen != KNN_SCREEN_F32)
    return exact_tc(ds, screen, Q, nq, k, out_idx, out_dist, workspace, workspace_bytes, stream);
  return knn_exact(ds->X, ds->n, ds->m, Q, nq, k, out_idx, out_dist, workspace, workspace_bytes, stream_);
}

// The naive exact method under the l1 distance: FP32 SIMT distances of every
// pair (no product form exists for l1), each within a relative error
// gamma_(m+2) of the exact distance; select within that margin; FP64 l1
// rerank of the candidates.
extern "C" knn_status knn_exact_l1(const float* X, int64_t n, int32_t m, const float* Q, int32_t nq, int32_t k,
                                   int64_t* out_idx, double* out_dist, void* workspace, size_t workspace_bytes,
                                   void* stream_) {
  clear_error();
  if (n < 1 || n >= (int64_t)1 << 31 || m < 1 || m > kMaxM || nq < 0 || k < 1 || k > n || k > kMaxKH) {
    set_error("knn_exact_l1: need 1 <= n < 2^31, 1 <= m <= 16384, 1 <= k <= min(n, 1024)");
    return KNN_EINVAL;
  }
  if (nq == 0) return KNN_OK;
  if (!X || !Q || !out_idx || !out_dist) {
    set_error("knn_exact_l1: null pointer");
    return KNN_EINVAL;
  }
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  Carve measure;
  const size_t need = carve_exact(measure, n, nq, nullptr) + 256;
  Workspace ws;
  knn_status s = ws.acquire(workspace, workspace_bytes, need, stream);
  if (s != KNN_OK) return s;
  Carve cv;
  cv.base = reinterpret_cast<uint8_t*>(((uintptr_t)ws.ptr + 255) & ~uintptr_t(255));
  ExactCarve c;
  carve_exact(cv, n, nq, &c);
  const double u = 1.0 / 16777216.0;
  const double rel = (double)(m + 2) * u / (1.0 - (double)(m + 2) * u);
  dim3 grid((unsigned)((n + kBM - 1) / kBM), (unsigned)((nq + kBN - 1) / kBN));
  screen_sgemm_kernel<true><<<grid, 256, 0, stream>>>(X, Q, n, nq, m, nullptr, nullptr, c.D);
  s = cuda_check(cudaGetLastError(), "l1 screen launch");
  if (s == KNN_OK)
    s = launch_screen_select(c.D, n, nq, m, k, c.qn, c.xmax, -rel, 0.0, X, Q, c.cand, stream);
  if (s == KNN_OK) s = launch_rerank(X, n, m, Q, nq, c.cand, kExactCand, k, out_idx, out_dist, stream, KNN_METRIC_L1);
  ws.release();
  return s;
}
