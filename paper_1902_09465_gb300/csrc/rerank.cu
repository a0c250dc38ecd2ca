// rerank.cu -- exact k nearest of candidate points (the brute force of
// Section 3 restricted to a candidate set, e.g. the set S-hat returned by the
// adaptive rounds, or the candidates of the exact method's screen): FP32
// distances of every candidate, FP64 only for those the FP32 error bound
// cannot separate from the k-th. The only double-precision arithmetic of the
// library.
#include <cfloat>
#include <cmath>

#include "knn_common.cuh"
#include "knn_internal.h"

namespace knn {

constexpr int kRerankNT = 512;
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

// FP32 distance of one row, one warp: squared l2 or l1, each term and the
// sum in FP32 (within a relative error gamma_(m+2) of the exact distance:
// one rounding for the difference, one for the square, m - 1 additions).
__device__ __forceinline__ float row_dist32(const float* xr, const float* qs, int m, int lane, bool l1, bool vec) {
  float s = 0.0f;
  if (vec) {
    for (int j = lane * 4; j < m; j += 128) {
      const float4 x4 = __ldg(reinterpret_cast<const float4*>(xr + j));
      const float4 q4 = *reinterpret_cast<const float4*>(qs + j);
      const float d0 = x4.x - q4.x, d1 = x4.y - q4.y, d2 = x4.z - q4.z, d3 = x4.w - q4.w;
      if (l1) {
        s += fabsf(d0);
        s += fabsf(d1);
        s += fabsf(d2);
        s += fabsf(d3);
      } else {
        s = fmaf(d0, d0, s);
        s = fmaf(d1, d1, s);
        s = fmaf(d2, d2, s);
        s = fmaf(d3, d3, s);
      }
    }
  } else {
    for (int j = lane; j < m; j += 32) {
      const float d = __ldg(xr + j) - qs[j];
      s = l1 ? s + fabsf(d) : fmaf(d, d, s);
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

template <int NT>
__device__ void bitonic_sort_u64(uint64_t* key, int P) {
  for (int size = 2; size <= P; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < (P >> 1); i += NT) {
        const int lo = 2 * i - (i & (stride - 1));
        const int hi = lo + stride;
        const bool up = (lo & size) == 0;
        const uint64_t a = key[lo], b = key[hi];
        if ((b < a) == up) {
          key[lo] = b;
          key[hi] = a;
        }
      }
      __syncthreads();
    }
  }
}

// One CTA per query: the exact k nearest of a candidate list by (distance,
// index). Candidates: cand[q*ncand + t] for t < ncand (entries < 0 skipped),
// or t < cnt[q] when counts are given.
//   1. FP32 distance d32 of every candidate (relative error <= rel);
//   2. tau32 = the k-th smallest d32; every candidate whose distance is at
//      most the k-th true one has d32 <= tau32 (1 + rel) / (1 - rel) (k
//      candidates have d <= tau32 / (1 - rel));
//   3. FP64 distances of that window only, top-k by (d64, index).
// A list that overflowed (cnt[q] > ncand, or a first entry of -2) asks for
// every point instead: points stream in index order, FP64 only for those
// whose d32 can still reach the running k-th distance, merged with the
// running top-k chunk by chunk.
template <int NT>
__global__ void __launch_bounds__(NT) refine_kernel(const float* __restrict__ X, int64_t n, int m,
                                                    const float* __restrict__ Q, const int64_t* __restrict__ cand,
                                                    int ncand, const int32_t* __restrict__ cnt, int k,
                                                    int64_t* out_idx, double* out_dist, int l1, int vec, int cap,
                                                    const float* __restrict__ cand_d, const float* __restrict__ eq) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  uint64_t* key = reinterpret_cast<uint64_t*>(smem_raw);
  int64_t* idx = reinterpret_cast<int64_t*>(key + cap);
  uint64_t* k32 = reinterpret_cast<uint64_t*>(idx + cap);
  float* qs = reinterpret_cast<float*>(k32 + cap);
  __shared__ int s_cnt;
  const int q = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t kInf = 0x7FF0000000000000ULL;
  const float u = 1.0f / 16777216.0f;
  const float rel = (float)(m + 2) * u / (1.0f - (float)(m + 2) * u);
  for (int j = threadIdx.x; j < m; j += NT) qs[j] = Q[(size_t)q * m + j];
  const int64_t* cr = cand + (size_t)q * ncand;
  const int c = cnt ? min(cnt[q], ncand + 1) : ncand;
  const bool full = c > ncand || (ncand > 0 && c > 0 && cr[0] == -2);
  __syncthreads();
  if (!full) {
    int P = next_pow2(c < 2 ? 2 : c);
    if (cand_d) {
      // 0. a screen's candidates with their screened values D~ (|D~ - d| <=
      // E_q): FP32 distances of the k smallest by D~ bound the k-th distance,
      // d_(k) <= D*/(1 - rel) with D* their largest d32, and every true
      // k-nearest point j has D~_j <= d_j + E_q <= D*/(1 - rel) + E_q; only
      // the candidates below that need their FP32 distance.
      float* d32s = reinterpret_cast<float*>(key);  // scratch until step 3
      for (int t = threadIdx.x; t < P; t += NT)
        k32[t] = t < c ? ((uint64_t)f2key(cand_d[(size_t)q * ncand + t]) << 32) | (uint32_t)t : ~0ull;
      __syncthreads();
      bitonic_sort_u64<NT>(k32, P);
      const int kk = min(k, c);
      float dmax = 0.0f;
      for (int t = warp; t < kk; t += NT / 32) {
        const int64_t id = cr[(uint32_t)k32[t]];
        const float d = row_dist32(X + (size_t)id * m, qs, m, lane, l1 != 0, vec != 0);
        if (lane == 0) d32s[t] = d;
        dmax = fmaxf(dmax, d);
      }
      if (lane != 0) dmax = 0.0f;
      __shared__ float s_dmax;
      if (threadIdx.x == 0) s_dmax = 0.0f;
      __syncthreads();
      if (lane == 0) atomicMax(reinterpret_cast<unsigned*>(&s_dmax), __float_as_uint(dmax));
      __syncthreads();
      const float cut2 = (s_dmax / (1.0f - rel) * (1.0f + 4.0f * u) + eq[q]) * (1.0f + 4.0f * u);
      int w2 = 0;
      for (int b = 0; b < c; b += NT)
        w2 += __syncthreads_count(b + threadIdx.x < c && key2f((uint32_t)(k32[b + threadIdx.x] >> 32)) <= cut2);
      w2 = max(w2, kk);
      for (int t = kk + warp; t < w2; t += NT / 32) {
        const int64_t id = cr[(uint32_t)k32[t]];
        const float d = row_dist32(X + (size_t)id * m, qs, m, lane, l1 != 0, vec != 0);
        if (lane == 0) d32s[t] = d;
      }
      __syncthreads();
      // 1. keyed (d32 bits, slot) for the step below
      uint64_t nk[8];
      const int P2 = next_pow2(w2 < 2 ? 2 : w2);
      int e = 0;
      for (int t = threadIdx.x; t < P2; t += NT, ++e)
        nk[e] = t < w2 && !isnan(d32s[t]) ? ((uint64_t)f2key(d32s[t]) << 32) | (uint32_t)k32[t] : ~0ull;
      __syncthreads();
      e = 0;
      for (int t = threadIdx.x; t < P2; t += NT, ++e) k32[t] = nk[e];
      __syncthreads();
      P = P2;
    } else {
      // 1. FP32 distances, keyed (d32 bits, slot)
      for (int t = threadIdx.x; t < P; t += NT) k32[t] = ~0ull;
      __syncthreads();
      for (int t = warp; t < c; t += NT / 32) {
        const int64_t id = cr[t];
        if (id < 0 || id >= n) continue;
        const float d = row_dist32(X + (size_t)id * m, qs, m, lane, l1 != 0, vec != 0);
        if (lane == 0 && !isnan(d)) k32[t] = ((uint64_t)f2key(d) << 32) | (uint32_t)t;
      }
      __syncthreads();
    }
    bitonic_sort_u64<NT>(k32, P);
    // 2. the window: a prefix of the sorted keys
    int v = 0;
    for (int b = 0; b < P; b += NT) v += __syncthreads_count(b + threadIdx.x < P && k32[b + threadIdx.x] != ~0ull);
    const int kk = min(k, v);
    int w = 0;
    if (kk > 0) {
      const float tau = key2f((uint32_t)(k32[kk - 1] >> 32));
      const float thr = tau * ((1.0f + rel) / (1.0f - rel)) * (1.0f + 4.0f * u);
      for (int b = 0; b < v; b += NT)
        w += __syncthreads_count(b + threadIdx.x < v && key2f((uint32_t)(k32[b + threadIdx.x] >> 32)) <= thr);
    }
    // 3. FP64 distances of the window
    const int P2 = next_pow2(w < 2 ? 2 : w);
    for (int t = threadIdx.x; t < P2; t += NT) {
      key[t] = kInf;
      idx[t] = INT64_MAX;
    }
    __syncthreads();
    for (int t = warp; t < w; t += NT / 32) {
      const int64_t id = cr[(uint32_t)k32[t]];
      const double d = row_dist64(X + (size_t)id * m, qs, m, lane, l1 != 0);
      if (lane == 0) {
        key[t] = (uint64_t)__double_as_longlong(d);
        idx[t] = id;
      }
    }
    __syncthreads();
    bitonic_sort_pairs<NT>(key, idx, P2);
  } else {
    // running top-k in [0, k), the chunk's admitted points after it
    for (int t = threadIdx.x; t < cap; t += NT) {
      key[t] = kInf;
      idx[t] = INT64_MAX;
    }
    __syncthreads();
    const int chunk = cap - k;
    float thr32 = INFINITY;
    for (int64_t base = 0; base < n; base += chunk) {
      if (threadIdx.x == 0) s_cnt = 0;
      __syncthreads();
      for (int t = warp; t < chunk; t += NT / 32) {
        const int64_t id = base + t;
        if (id >= n) break;
        const float d32 = row_dist32(X + (size_t)id * m, qs, m, lane, l1 != 0, vec != 0);
        if (d32 <= thr32) {  // warp-uniform
          const double d = row_dist64(X + (size_t)id * m, qs, m, lane, l1 != 0);
          if (lane == 0) {
            const int p = atomicAdd(&s_cnt, 1);
            key[k + p] = (uint64_t)__double_as_longlong(d);
            idx[k + p] = id;
          }
        }
      }
      __syncthreads();
      const int used = k + s_cnt;
      const int P = next_pow2(used < 2 ? 2 : used);
      for (int t = used + threadIdx.x; t < P; t += NT) {
        key[t] = kInf;
        idx[t] = INT64_MAX;
      }
      __syncthreads();
      bitonic_sort_pairs<NT>(key, idx, P);
      // a later point (larger index) enters only with a smaller distance:
      // d32 <= d (1 + rel) <= d64_k (1 + rel)
      if (key[k - 1] != kInf)
        thr32 = __double2float_ru(__longlong_as_double((long long)key[k - 1]) * (1.0 + (double)rel) * (1.0 + 1e-9));
      for (int t = k + threadIdx.x; t < P; t += NT) {
        key[t] = kInf;
        idx[t] = INT64_MAX;
      }
      __syncthreads();
    }
  }
  for (int t = threadIdx.x; t < k; t += NT) {
    const bool ok = key[t] != kInf;
    out_idx[(size_t)q * k + t] = ok ? idx[t] : -1;
    out_dist[(size_t)q * k + t] = ok ? __longlong_as_double((long long)key[t]) : INFINITY;
  }
}

knn_status launch_refine(const float* X, int64_t n, int32_t m, const float* Q, int32_t nq, const int64_t* cand,
                         int32_t ncand, const int32_t* cnt, int32_t k, int64_t* out_idx, double* out_dist,
                         cudaStream_t stream, int32_t metric, const float* cand_d, const float* eq) {
  // sort capacity: every candidate, and room for a chunk of points beside the
  // running top-k when a list asks for every point
  int cap = 2;
  while (cap < ncand || cap < 2 * k + 256) cap <<= 1;
  const size_t smem = (size_t)cap * 24 + (size_t)m * 4;
  knn_status s = cuda_check(
      cudaFuncSetAttribute(refine_kernel<kRerankNT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
      "cudaFuncSetAttribute(refine)");
  if (s != KNN_OK) return s;
  const int vec = (m % 4 == 0) && (((uintptr_t)X & 15) == 0);
  refine_kernel<kRerankNT><<<nq, kRerankNT, smem, stream>>>(X, n, m, Q, cand, ncand, cnt, k, out_idx, out_dist,
                                                            metric == KNN_METRIC_L1 ? 1 : 0, vec, cap, cand_d,
                                                            eq);
  return cuda_check(cudaGetLastError(), "refine_kernel launch");
}

knn_status launch_rerank(const float* X, int64_t n, int32_t m, const float* Q, int32_t nq, const int64_t* cand,
                         int32_t ncand, int32_t k, int64_t* out_idx, double* out_dist, cudaStream_t stream,
                         int32_t metric) {
  return launch_refine(X, n, m, Q, nq, cand, ncand, nullptr, k, out_idx, out_dist, stream, metric, nullptr, nullptr);
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
