// rerank.cu -- exact FP64 distances of candidate points and top-k selection
// (the brute force of Section 3 restricted to a candidate set, e.g. the set
// S-hat returned by the adaptive rounds). The only double-precision
// arithmetic of the library.
#include <cfloat>
#include <cmath>

#include "knn_common.cuh"
#include "knn_internal.h"

namespace knn {

constexpr int kRerankNT = 256;
constexpr int kRerankCap = 4096;  // candidates sorted at once

// Keys are (bits of a non-negative double, index); +inf bits mark no point.
__device__ __forceinline__ bool pair_less(uint64_t ka, int64_t ia, uint64_t kb, int64_t ib) {
  return ka < kb || (ka == kb && ia < ib);
}

template <int NT>
__device__ void bitonic_sort_pairs(uint64_t* key, int64_t* idx, int P) {
  for (int size = 2; size <= P; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < (P >> 1); i += NT) {
        const int lo = 2 * i - (i & (stride - 1));
        const int hi = lo + stride;
        const bool up = (lo & size) == 0;
        const uint64_t ka = key[lo], kb = key[hi];
        const int64_t ia = idx[lo], ib = idx[hi];
        if (pair_less(kb, ib, ka, ia) == up) {
          key[lo] = kb;
          key[hi] = ka;
          idx[lo] = ib;
          idx[hi] = ia;
        }
      }
      __syncthreads();
    }
  }
}

// Squared l2 distance (or l1 distance) of one row in FP64, one warp.
__device__ __forceinline__ double row_dist64(const float* xr, const float* qs, int m, int lane, bool l1) {
  double s = 0.0;
  for (int j = lane; j < m; j += 32) {
    const double d = (double)__ldg(xr + j) - (double)qs[j];
    s = l1 ? s + fabs(d) : fma(d, d, s);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// One CTA per query. cand[q*ncand + t]: candidate indices (< 0 skipped). A
// row whose first entry is -2 asks for every point (used when a screen
// could not bound its candidate set); the points are then taken in chunks
// and merged with the running top-k.
template <int NT>
__global__ void __launch_bounds__(NT) rerank_kernel(const float* __restrict__ X, int64_t n, int m,
                                                    const float* __restrict__ Q, const int64_t* __restrict__ cand,
                                                    int ncand, int k, int64_t* out_idx, double* out_dist,
                                                    int l1) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  uint64_t* key = reinterpret_cast<uint64_t*>(smem_raw);
  int64_t* idx = reinterpret_cast<int64_t*>(key + kRerankCap);
  float* qs = reinterpret_cast<float*>(idx + kRerankCap);
  const int q = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t kInf = 0x7FF0000000000000ULL;
  for (int j = threadIdx.x; j < m; j += NT) qs[j] = Q[(size_t)q * m + j];
  const int64_t* cr = cand + (size_t)q * ncand;
  const bool full = ncand > 0 && cr[0] == -2;
  __syncthreads();
  if (!full) {
    const int P = next_pow2(ncand < 2 ? 2 : ncand);
    for (int t = threadIdx.x; t < P; t += NT) {
      key[t] = kInf;
      idx[t] = INT64_MAX;
    }
    __syncthreads();
    for (int t = warp; t < ncand; t += NT / 32) {
      const int64_t c = cr[t];
      if (c < 0 || c >= n) continue;
      const double d = row_dist64(X + (size_t)c * m, qs, m, lane, l1 != 0);
      if (lane == 0) {
        key[t] = (uint64_t)__double_as_longlong(d);
        idx[t] = c;
      }
    }
    __syncthreads();
    bitonic_sort_pairs<NT>(key, idx, P);
  } else {
    // running top-k in [0, k), next chunk of points in [k, kRerankCap)
    for (int t = threadIdx.x; t < kRerankCap; t += NT) {
      key[t] = kInf;
      idx[t] = INT64_MAX;
    }
    __syncthreads();
    const int chunk = kRerankCap - k;
    for (int64_t base = 0; base < n; base += chunk) {
      for (int t = k + threadIdx.x; t < kRerankCap; t += NT) {
        key[t] = kInf;
        idx[t] = INT64_MAX;
      }
      __syncthreads();
      for (int t = warp; t < chunk; t += NT / 32) {
        const int64_t c = base + t;
        if (c >= n) break;
        const double d = row_dist64(X + (size_t)c * m, qs, m, lane, l1 != 0);
        if (lane == 0) {
          key[k + t] = (uint64_t)__double_as_longlong(d);
          idx[k + t] = c;
        }
      }
      __syncthreads();
      bitonic_sort_pairs<NT>(key, idx, kRerankCap);
    }
  }
  for (int t = threadIdx.x; t < k; t += NT) {
    const bool ok = key[t] != kInf;
    out_idx[(size_t)q * k + t] = ok ? idx[t] : -1;
    out_dist[(size_t)q * k + t] = ok ? __longlong_as_double((long long)key[t]) : INFINITY;
  }
}

knn_status launch_rerank(const float* X, int64_t n, int32_t m, const float* Q, int32_t nq, const int64_t* cand,
                         int32_t ncand, int32_t k, int64_t* out_idx, double* out_dist, cudaStream_t stream,
                         int32_t metric) {
  const size_t smem = (size_t)kRerankCap * 16 + (size_t)m * 4;
  knn_status s = cuda_check(
      cudaFuncSetAttribute(rerank_kernel<kRerankNT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
      "cudaFuncSetAttribute(rerank)");
  if (s != KNN_OK) return s;
  rerank_kernel<kRerankNT><<<nq, kRerankNT, smem, stream>>>(X, n, m, Q, cand, ncand, k, out_idx, out_dist,
                                                            metric == KNN_METRIC_L1 ? 1 : 0);
  return cuda_check(cudaGetLastError(), "rerank_kernel launch");
}

}  // namespace knn

extern "C" knn_status knn_rerank(const float* X, int64_t n, int32_t m, const float* Q, int32_t nq,
                                 const int64_t* cand, int32_t ncand, int32_t k, int64_t* out_idx, double* out_dist,
                                 void* stream) {
  return knn_rerank_metric(X, n, m, Q, nq, cand, ncand, k, KNN_METRIC_L2SQ, out_idx, out_dist, stream);
}

extern "C" knn_status knn_rerank_metric(const float* X, int64_t n, int32_t m, const float* Q, int32_t nq,
                                        const int64_t* cand, int32_t ncand, int32_t k, int32_t metric,
                                        int64_t* out_idx, double* out_dist, void* stream) {
  knn::clear_error();
  if (metric != KNN_METRIC_L2SQ && metric != KNN_METRIC_L1) {
    knn::set_error("knn_rerank_metric: unknown metric");
    return KNN_EINVAL;
  }
  if (n < 1 || m < 1 || m > knn::kMaxM || nq < 0 || k < 1 || k > knn::kMaxKH || ncand < 1 ||
      ncand > knn::kRerankCap) {
    knn::set_error("knn_rerank: need n >= 1, 1 <= m <= 16384, 1 <= k <= 1024, 1 <= ncand <= 4096");
    return KNN_EINVAL;
  }
  if (nq == 0) return KNN_OK;
  if (!X || !Q || !cand || !out_idx || !out_dist) {
    knn::set_error("knn_rerank: null pointer");
    return KNN_EINVAL;
  }
  return knn::launch_rerank(X, n, m, Q, nq, cand, ncand, k, out_idx, out_dist, static_cast<cudaStream_t>(stream),
                            metric);
}
