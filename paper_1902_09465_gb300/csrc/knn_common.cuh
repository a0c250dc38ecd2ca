// knn_common.cuh -- device helpers shared by the kernels of the library:
// the Philox4x32-10 generator, order-preserving float keys, block-wide scans
// and reductions, a shared-memory bitonic sort and a three-level radix select
// of the smallest keys.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace knn {

constexpr int kMaxM = 16384;     // largest dimension m
constexpr int kMaxKH = 1024;     // largest k + h
constexpr int kSelCap = 4096;    // keys a select may finish on in shared memory
constexpr int kHistBins = 4096;  // level-1 bins (key bits 31..20)

// ----------------------------------------------------------------- Philox
// Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11): the round
// multiplies words 0 and 2 by fixed odd constants, xors the high halves of
// the 64-bit products with the other words and the round key, and bumps the
// key by the Weyl constants between rounds. 32-bit products are native.
__device__ __forceinline__ uint4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                               uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += W0;
      k1 += W1;
    }
    const uint32_t hi0 = __umulhi(M0, c0), lo0 = M0 * c0;
    const uint32_t hi1 = __umulhi(M1, c2), lo1 = M1 * c2;
    c0 = hi1 ^ c1 ^ k0;
    c1 = lo1;
    c2 = hi0 ^ c3 ^ k1;
    c3 = lo0;
  }
  return make_uint4(c0, c1, c2, c3);
}

// Draws 8i .. 8i + 7 of a (query, point) pair: the words of blocks 2i and
// 2i + 1 of its stream -- Philox4x32-10 at counter (block, point field, low
// and high words of the query field), key (low and high words of the seed).
struct Draws8 {
  uint32_t w[8];
};

__device__ __forceinline__ Draws8 pair_draws8(uint32_t item, uint64_t point_field, uint64_t query_field,
                                              uint64_t seed) {
  const uint32_t p = (uint32_t)point_field, ql = (uint32_t)query_field, qh = (uint32_t)(query_field >> 32);
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  const uint4 a = philox4x32_10(2u * item, p, ql, qh, k0, k1);
  const uint4 b = philox4x32_10(2u * item + 1u, p, ql, qh, k0, k1);
  Draws8 d;
  d.w[0] = a.x;
  d.w[1] = a.y;
  d.w[2] = a.z;
  d.w[3] = a.w;
  d.w[4] = b.x;
  d.w[5] = b.y;
  d.w[6] = b.z;
  d.w[7] = b.w;
  return d;
}

// The ten round keys of a seed, (k0 + r W0, k1 + r W1) for r = 0 .. 9, held
// in a kernel's parameters: the rounds then read them as constant operands
// instead of adding the Weyl increments per call.
struct PhiloxKeys {
  uint32_t k[20];
};

__host__ __device__ inline PhiloxKeys philox_keys(uint64_t seed) {
  PhiloxKeys K;
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    K.k[2 * r] = k0;
    K.k[2 * r + 1] = k1;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return K;
}

// philox4x32_10 with the round keys given
__device__ __forceinline__ uint4 philox4x32_10_rk(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                  const PhiloxKeys& K) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(M0, c0), lo0 = M0 * c0;
    const uint32_t hi1 = __umulhi(M1, c2), lo1 = M1 * c2;
    c0 = hi1 ^ c1 ^ K.k[2 * r];
    c1 = lo1;
    c2 = hi0 ^ c3 ^ K.k[2 * r + 1];
    c3 = lo0;
  }
  return make_uint4(c0, c1, c2, c3);
}

// pair_draws8 with the seed's round keys given
__device__ __forceinline__ Draws8 pair_draws8(uint32_t item, uint64_t point_field, uint64_t query_field,
                                              const PhiloxKeys& K) {
  const uint32_t p = (uint32_t)point_field, ql = (uint32_t)query_field, qh = (uint32_t)(query_field >> 32);
  const uint4 a = philox4x32_10_rk(2u * item, p, ql, qh, K);
  const uint4 b = philox4x32_10_rk(2u * item + 1u, p, ql, qh, K);
  Draws8 d;
  d.w[0] = a.x;
  d.w[1] = a.y;
  d.w[2] = a.z;
  d.w[3] = a.w;
  d.w[4] = b.x;
  d.w[5] = b.y;
  d.w[6] = b.z;
  d.w[7] = b.w;
  return d;
}

// Item whose two blocks are the last of a pair's stream (blocks 2^32 - 2 and
// 2^32 - 1): the round keys of the draws without replacement.
constexpr uint32_t kWorKeyItem = 0x7FFFFFFFu;

__device__ __forceinline__ uint32_t philox_word(const Draws8& d, int w) { return d.w[w]; }

// ------------------------------------------------------- streaming loads
// Read-only loads that do not allocate in L1: rows read once (staged in
// shared memory) leave L1 to the data that is reused.
__device__ __forceinline__ float4 ld_stream4(const float4* p) {
  float4 v;
  asm("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
      : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
      : "l"(p));
  return v;
}
__device__ __forceinline__ float ld_stream(const float* p) {
  float v;
  asm("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}

// ------------------------------------------------------------------- keys
// Unsigned keys whose integer order is the float order (-0 < +0; NaN sorts
// above +inf with the sign bit clear, below -inf with it set).
__device__ __forceinline__ uint32_t f2key(float f) {
  uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float key2f(uint32_t k) {
  uint32_t u = (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
  return __uint_as_float(u);
}

// --------------------------------------------------------- block helpers
template <int NT>
struct BlockScratch {
  int warp[NT / 32 + 1];
  float wf[NT / 32 + 1];
  int bcast[4];
};

// Exclusive prefix sum of v over the block; *total gets the sum. All threads
// must call it. Uses two barriers.
template <int NT>
__device__ __forceinline__ int block_exclusive_scan(int v, BlockScratch<NT>& s, int* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s.warp[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int t = lane < NT / 32 ? s.warp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < NT / 32) s.warp[lane] = t;  // inclusive prefix of warp totals
  }
  __syncthreads();
  const int before = wid ? s.warp[wid - 1] : 0;
  *total = s.warp[NT / 32 - 1];
  __syncthreads();  // s.warp is reused by the next call
  return before + x - v;
}

template <int NT>
__device__ __forceinline__ float block_min(float v, BlockScratch<NT>& s) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (lane == 0) s.wf[wid] = v;
  __syncthreads();
  float r = s.wf[0];
#pragma unroll
  for (int i = 1; i < NT / 32; ++i) r = fminf(r, s.wf[i]);
  __syncthreads();
  return r;
}

template <int NT>
__device__ __forceinline__ float block_max(float v, BlockScratch<NT>& s) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (lane == 0) s.wf[wid] = v;
  __syncthreads();
  float r = s.wf[0];
#pragma unroll
  for (int i = 1; i < NT / 32; ++i) r = fmaxf(r, s.wf[i]);
  __syncthreads();
  return r;
}

__device__ __forceinline__ int next_pow2(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

// Ascending bitonic sort of buf[0..cnt) in shared memory (padded with the
// largest key up to a power of two, which must fit in the buffer).
template <int NT>
__device__ void bitonic_sort_keys(uint32_t* buf, int cnt) {
  if (cnt <= 32) {  // one warp, in registers: no block barrier per stage
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      uint32_t v = lane < cnt ? buf[lane] : 0xFFFFFFFFu;
#pragma unroll
      for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
          const uint32_t o = __shfl_xor_sync(0xffffffffu, v, stride);
          const bool lower = (lane & stride) == 0, up = (lane & size) == 0;
          v = (lower == up) ? min(v, o) : max(v, o);
        }
      }
      buf[lane] = v;
    }
    __syncthreads();
    return;
  }
  const int P = next_pow2(cnt < 2 ? 2 : cnt);
  for (int i = cnt + threadIdx.x; i < P; i += NT) buf[i] = 0xFFFFFFFFu;
  __syncthreads();
  for (int size = 2; size <= P; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < (P >> 1); i += NT) {
        const int lo = 2 * i - (i & (stride - 1));
        const int hi = lo + stride;
        const bool up = (lo & size) == 0;
        const uint32_t a = buf[lo], b = buf[hi];
        if ((a > b) == up) {
          buf[lo] = b;
          buf[hi] = a;
        }
      }
      __syncthreads();
    }
  }
}

// -------------------------------------------------------- radix select
// Shared state of select_smallest.
struct SelectShared {
  int cnt;
  int bin;
  int below;
  int inbin;
};

// Finds the bin of hist[0..nbins) that holds the rank-th key (0-based) among
// keys counted there, and the count of keys in lower bins.
template <int NT>
__device__ void find_bin(const uint32_t* hist, int nbins, int rank, SelectShared& ss, BlockScratch<NT>& bs) {
  const int per = (nbins + NT - 1) / NT;
  const int b0 = threadIdx.x * per;
  int local = 0;
  for (int b = b0; b < b0 + per && b < nbins; ++b) local += (int)hist[b];
  int total;
  int pre = block_exclusive_scan<NT>(local, bs, &total);
  if (rank >= pre && rank < pre + local) {
    int acc = pre;
    for (int b = b0; b < b0 + per && b < nbins; ++b) {
      int c = (int)hist[b];
      if (rank < acc + c) {
        ss.bin = b;
        ss.below = acc;
        ss.inbin = c;
        break;
      }
      acc += c;
    }
  }
  __syncthreads();
}

// The kk smallest of N keys get(0..N-1), ascending, into buf[0..kk)
// (1 <= kk <= N, kk <= kSelCap). On entry hist[0..kHistBins) must hold the
// counts of key >> 20 over the N keys; it is overwritten. Up to three levels
// of histogram (bits 31..20, 19..10, 9..0); the keys are finished in shared
// memory as soon as the candidates fit, and every level costs one pass.
template <int NT, class Get>
__device__ void select_smallest(Get get, int N, int kk, uint32_t* hist, uint32_t* buf, SelectShared& ss,
                                BlockScratch<NT>& bs) {
  const int rank = kk - 1;
  find_bin<NT>(hist, kHistBins, rank, ss, bs);
  const uint32_t b1 = (uint32_t)ss.bin;
  int below = ss.below, inbin = ss.inbin;
  int shift = 20;
  uint32_t prefix = b1;
  // finish in shared memory once the candidates fit; for small kk go on to
  // finer levels until one warp can sort them (a histogram level costs a few
  // barriers, a block-wide sort of thousands of keys dozens)
  const int cap = kk <= 32 ? 32 : kSelCap;
  bool done = below + inbin <= cap;
  if (!done) {
    // level 2: bits 19..10 of keys in bin b1
    for (int i = threadIdx.x; i < 1024; i += NT) hist[i] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < N; i += NT) {
      uint32_t key = get(i);
      if ((key >> 20) == b1) atomicAdd(&hist[(key >> 10) & 1023u], 1u);
    }
    __syncthreads();
    find_bin<NT>(hist, 1024, rank - below, ss, bs);
    const uint32_t b2 = (uint32_t)ss.bin;
    below += ss.below;
    inbin = ss.inbin;
    shift = 10;
    prefix = (b1 << 10) | b2;
    done = below + inbin <= cap;
    if (!done) {
      // level 3: bits 9..0 of keys with prefix (b1, b2); fixes the key exactly
      for (int i = threadIdx.x; i < 1024; i += NT) hist[i] = 0;
      __syncthreads();
      for (int i = threadIdx.x; i < N; i += NT) {
        uint32_t key = get(i);
        if ((key >> 10) == prefix) atomicAdd(&hist[key & 1023u], 1u);
      }
      __syncthreads();
      find_bin<NT>(hist, 1024, rank - below, ss, bs);
      const uint32_t kstar = (prefix << 10) | (uint32_t)ss.bin;
      below += ss.below;  // keys strictly below kstar: below < kk
      if (threadIdx.x == 0) ss.cnt = 0;
      __syncthreads();
      for (int i = threadIdx.x; i < N; i += NT) {
        uint32_t key = get(i);
        if (key < kstar) buf[atomicAdd(&ss.cnt, 1)] = key;
      }
      __syncthreads();
      bitonic_sort_keys<NT>(buf, below);  // pads past `below`; the ties are written after
      for (int i = below + threadIdx.x; i < kk; i += NT) buf[i] = kstar;
      __syncthreads();
      return;
    }
  }
  if (threadIdx.x == 0) ss.cnt = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < N; i += NT) {
    uint32_t key = get(i);
    if ((key >> shift) <= prefix) buf[atomicAdd(&ss.cnt, 1)] = key;
  }
  __syncthreads();
  bitonic_sort_keys<NT>(buf, below + inbin);
}

}  // namespace knn
