// dataset.cu -- resident datasets: the data range computed once, BF16 and
// FP8-e4m3 (per-row scale) copies with their largest element error, and the
// adaptive rounds over a chosen copy (knn_adaptive_ds).
#include <cuda_bf16.h>

#include <string>

#include "adaptive_kernel.cuh"

namespace knn {

knn_status build_screen_operand(knn_dataset* ds, cudaStream_t stream);

// BF16 copy (round to nearest even) and its largest element error.
static __global__ void quantize_bf16_kernel(const float* __restrict__ X, size_t count, uint16_t* __restrict__ out,
                                            unsigned* emax_bits) {
  float e = 0.0f;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
    const float x = __ldg(X + i);
    const __nv_bfloat16 b = __float2bfloat16_rn(x);
    const uint16_t bits = __bfloat16_as_ushort(b);
    out[i] = bits;
    const float d = fabsf(__uint_as_float((uint32_t)bits << 16) - x);
    if (isfinite(x)) e = fmaxf(e, d);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) e = fmaxf(e, __shfl_xor_sync(0xffffffffu, e, o));
  if ((threadIdx.x & 31) == 0) atomicMax(emax_bits, __float_as_uint(e));
}

// FP8 e4m3 copy, one warp per row: s = max|x| / 448 (1 for a zero row),
// value = e4m3(x / s) rounded to nearest even and saturated at 448; the
// dequantised value is s * value in FP32.
static __global__ void quantize_fp8_kernel(const float* __restrict__ X, int64_t n, int m, uint8_t* __restrict__ out,
                                           float* __restrict__ scale, unsigned* emax_bits) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  float e = 0.0f;
  for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < n; r += warps) {
    const float* xr = X + (size_t)r * m;
    float mx = 0.0f;
    for (int j = lane; j < m; j += 32) mx = fmaxf(mx, fabsf(__ldg(xr + j)));
#pragma unroll
    for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const float s = mx > 0.0f ? mx / 448.0f : 1.0f;
    if (lane == 0) scale[r] = s;
    for (int j = lane; j < m; j += 32) {
      const float x = __ldg(xr + j);
      const __nv_fp8_storage_t v = __nv_cvt_float_to_fp8(x / s, __NV_SATFINITE, __NV_E4M3);
      out[(size_t)r * m + j] = v;
      __nv_fp8_e4m3 f;
      f.__x = v;
      // the dequantised value is fl32(s * value): __fmul_rn keeps it from
      // being fused into the subtraction
      const float d = fabsf(__fmul_rn(s, static_cast<float>(f)) - x);
      if (isfinite(x)) e = fmaxf(e, d);
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) e = fmaxf(e, __shfl_xor_sync(0xffffffffu, e, o));
  if (lane == 0) atomicMax(emax_bits, __float_as_uint(e));
}

// Column of draw t under shared coordinates: Philox4x64-10 with key
// (seed, 0) and counter (t / 8, 0, 0, 0), word t mod 8 scaled to [0, m).
static __global__ void shared_columns_kernel(uint64_t seed, int m, int32_t* jperm) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m) return;
  const Philox4x64 ph = philox4x64_10((uint64_t)t >> 3, 0, 0, 0, seed, 0);
  jperm[t] = (int32_t)__umulhi(philox_word(ph, t & 7), (uint32_t)m);
}

// Permuted copy: out[i, t] = src[i, jperm[t]] for t < m, zero up to mp.
template <class T>
static __global__ void permute_rows_kernel(const T* __restrict__ src, int64_t n, int m, int mp,
                                           const int32_t* __restrict__ jperm, T* __restrict__ out) {
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    const T* sr = src + (size_t)i * m;
    T* orow = out + (size_t)i * mp;
    for (int t = threadIdx.x; t < mp; t += blockDim.x) orow[t] = t < m ? sr[jperm[t]] : T(0);
  }
}

}  // namespace knn

using namespace knn;

extern "C" knn_status knn_dataset_create(const float* X, int64_t n, int32_t m, int32_t copies, void* stream_,
                                         knn_dataset** out) {
  clear_error();
  if (!out || !X) return set_error("knn_dataset_create: null pointer"), KNN_EINVAL;
  *out = nullptr;
  if (n < 1 || n >= (int64_t)1 << 31 || m < 1 || m > kMaxM)
    return set_error("knn_dataset_create: need 1 <= n < 2^31 and 1 <= m <= 16384"), KNN_EINVAL;
  if (copies & ~((1 << KNN_STORE_BF16) | (1 << KNN_STORE_FP8) | KNN_COPY_SCREEN))
    return set_error("knn_dataset_create: copies must be a mask of BF16, FP8 and the screen operand"), KNN_EINVAL;
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  knn_dataset* ds = new knn_dataset();
  ds->X = X;
  ds->n = n;
  ds->m = m;
  ds->copies = copies;
  knn_status s = cuda_check(cudaGetDevice(&ds->device), "cudaGetDevice");
  const size_t count = (size_t)n * (size_t)m;
  if (s == KNN_OK) s = cuda_check(cudaMalloc(&ds->range, 3 * sizeof(uint32_t)), "cudaMalloc(range)");
  if (s == KNN_OK) s = cuda_check(cudaMalloc(&ds->emax, 3 * sizeof(unsigned)), "cudaMalloc(emax)");
  if (s == KNN_OK && (copies & (1 << KNN_STORE_BF16)))
    s = cuda_check(cudaMalloc(&ds->xb, count * sizeof(uint16_t)), "cudaMalloc(bf16 copy)");
  if (s == KNN_OK && (copies & (1 << KNN_STORE_FP8))) {
    s = cuda_check(cudaMalloc(&ds->x8, count), "cudaMalloc(fp8 copy)");
    if (s == KNN_OK) s = cuda_check(cudaMalloc(&ds->scale8, (size_t)n * sizeof(float)), "cudaMalloc(fp8 scale)");
  }
  if (s == KNN_OK) s = cuda_check(cudaMemsetAsync(ds->range, 0xFF, 4, stream), "memset");
  if (s == KNN_OK) s = cuda_check(cudaMemsetAsync(ds->range + 1, 0x00, 8, stream), "memset");
  if (s == KNN_OK) s = cuda_check(cudaMemsetAsync(ds->emax, 0x00, 12, stream), "memset");
  DeviceInfo di;
  if (s == KNN_OK) s = device_info(&di);
  if (s == KNN_OK) {
    const int blocks = (int)std::max<size_t>(1, std::min<size_t>((count + 255) / 256, (size_t)di.sms * 8));
    minmax_kernel<<<blocks, 256, 0, stream>>>(X, count, ds->range);
    if (ds->xb) quantize_bf16_kernel<<<blocks, 256, 0, stream>>>(X, count, ds->xb, ds->emax + KNN_STORE_BF16);
    if (ds->x8)
      quantize_fp8_kernel<<<di.sms * 8, 256, 0, stream>>>(X, n, m, ds->x8, ds->scale8, ds->emax + KNN_STORE_FP8);
    s = cuda_check(cudaGetLastError(), "dataset kernels launch");
  }
  if (s == KNN_OK && (copies & KNN_COPY_SCREEN)) s = build_screen_operand(ds, stream);
  if (s == KNN_OK) s = cuda_check(cudaStreamSynchronize(stream), "dataset build");
  if (s == KNN_OK) {
    unsigned bits[3];
    s = cuda_check(cudaMemcpy(bits, ds->emax, sizeof(bits), cudaMemcpyDeviceToHost), "read copy errors");
    for (int i = 0; i < 3 && s == KNN_OK; ++i) memcpy(&ds->emax_host[i], &bits[i], 4);
  }
  if (s != KNN_OK) {
    knn_dataset_destroy(ds);
    return s;
  }
  *out = ds;
  return KNN_OK;
}

extern "C" knn_status knn_dataset_destroy(knn_dataset* ds) {
  if (!ds) return KNN_OK;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(ds->device);
  cudaDeviceSynchronize();
  cudaFree(ds->range);
  cudaFree(ds->emax);
  cudaFree(ds->xb);
  cudaFree(ds->x8);
  cudaFree(ds->scale8);
  cudaFree(ds->screenA);
  cudaFree(ds->mu);
  cudaFree(ds->xcn);
  cudaFree(ds->xcn_max);
  cudaFree(ds->jperm);
  cudaFree(ds->p32);
  cudaFree(ds->pb);
  cudaFree(ds->p8);
  cudaSetDevice(cur);
  delete ds;
  return KNN_OK;
}

extern "C" knn_status knn_dataset_error(const knn_dataset* ds, int32_t storage, float* out_error) {
  clear_error();
  if (!ds || !out_error || storage < 0 || storage > 2)
    return set_error("knn_dataset_error: bad arguments"), KNN_EINVAL;
  *out_error = ds->emax_host[storage];
  return KNN_OK;
}

// Per-query k and counter ids of a mixed batch (null: one k, ids qid_base + q).
struct MixedBatch {
  const int32_t* kq = nullptr;
  const uint64_t* qids = nullptr;
  int32_t h_per_k = 0;
  int32_t out_stride = 0;
};

template <class E>
static knn_status adaptive_ds_launch(const knn_dataset* ds, const float* Q, int32_t nq, int32_t k, double delta,
                                     uint64_t seed, const knn_opts& o, int64_t* out_idx, int32_t* out_count,
                                     int64_t* out_evals, int32_t* out_rounds, int32_t* log_code, float* log_S,
                                     void* workspace, size_t workspace_bytes, cudaStream_t stream,
                                     const MixedBatch* mix = nullptr) {
  const int64_t n = ds->n;
  const int32_t m = ds->m;
  // round 0 point-major: the shared form for B0 <= 64, the staged-rows pass otherwise
  const bool r0 = E::kPerm ? (o.B0 < m && o.B0 <= 64) : round0_applies(m, o);
  AdaptivePlan p;
  knn_status s = plan_adaptive<E>(n, m, nq, k, &o, &p);
  if (s != KNN_OK) return s;
  const int chunk = r0 ? round0_chunk(n, nq, p.grid) : nq;
  // round-0 tile minima: per CTA of the staged-rows pass, per warp of the shared pass
  const int rows = round0_rows(m);
  const int tiles = !r0 ? 0 : (int)(E::kPerm ? (n + 31) / 32 : (n + rows - 1) / rows);
  Carve measure;
  carve_adaptive(measure, n, p, nullptr);
  const int qpw = E::kPerm && r0 ? (o.B0 <= 16 ? 16 : (o.B0 <= 32 ? 32 : 64)) : 0;  // staged by round 0
  if (r0) {
    measure.take<float>((size_t)chunk * (size_t)n);
    measure.take<float>((size_t)chunk * (size_t)tiles);
    measure.take<float>((size_t)chunk * (size_t)qpw);
  }
  const size_t need = measure.off + 256;
  Workspace ws;
  s = ws.acquire(workspace, workspace_bytes, need, stream);
  if (s != KNN_OK) return s;
  Carve cv;
  cv.base = reinterpret_cast<uint8_t*>(((uintptr_t)ws.ptr + 255) & ~uintptr_t(255));
  AdaptiveCarve c;
  carve_adaptive(cv, n, p, &c);
  float* r0buf = r0 ? cv.take<float>((size_t)chunk * (size_t)n) : nullptr;
  float* r0min = r0 ? cv.take<float>((size_t)chunk * (size_t)tiles) : nullptr;
  float* qperm = qpw ? cv.take<float>((size_t)chunk * (size_t)qpw) : nullptr;
  AdaptiveArgs a;
  const void* G = ds->X;
  if (E::kStorage == KNN_STORE_BF16) G = ds->xb;
  if (E::kStorage == KNN_STORE_FP8) G = ds->x8;
  if (E::kPerm) G = E::kStorage == KNN_STORE_BF16 ? (const void*)ds->pb
                    : (E::kStorage == KNN_STORE_FP8 ? (const void*)ds->p8 : (const void*)ds->p32);
  a.X = ds->X;
  a.G = G;
  a.gscale = ds->scale8;
  a.emax = E::kStorage == KNN_STORE_F32 ? nullptr : reinterpret_cast<const float*>(ds->emax + E::kStorage);
  a.Q = Q;
  a.n = n;
  a.m = m;
  a.nq = nq;
  a.k = k;
  a.h = o.h;
  a.kq = mix ? mix->kq : nullptr;
  a.qids = mix ? mix->qids : nullptr;
  a.h_per_k = mix ? mix->h_per_k : 0;
  a.out_stride = mix ? mix->out_stride : k + o.h;
  a.bound = o.bound;
  const double dprime = delta / (double)n;
  a.a_c0 = 0.0f;
  a.a_c1 = 0.0f;
  if (o.bound == KNN_BOUND_FOOTNOTE)
    a.a_c0 = (float)(std::log(1.0 / dprime) + 3.0 * std::log(std::log(1.0 / dprime)));
  else if (o.bound == KNN_BOUND_LEMMA)
    a.a_c0 = (float)std::log(125.0 / dprime);
  else
    a.a_c1 = (float)((double)n / delta);
  a.c_alpha = (float)o.c_alpha;
  a.B0 = o.B0;
  a.B = o.B;
  a.grow = o.grow;
  a.seed = seed;
  a.qid_base = o.qid_base;
  a.mask_p = o.mask_p;
  a.mask_q = o.mask_q;
  a.xrange = ds->range;
  a.ws_ids = c.ids;
  a.ws_S = c.S;
  a.ws_C = c.C;
  a.ws_acc_id = c.acc_id;
  a.ws_acc_d = c.acc_d;
  a.ws_acc_U = c.acc_U;
  a.ws_acc_L = c.acc_L;
  a.acc_cap = p.acc_cap;
  a.queue = c.queue;
  a.out_idx = out_idx;
  a.out_count = out_count;
  a.out_evals = out_evals;
  a.out_rounds = out_rounds;
  a.log_code = log_code;
  a.log_S = log_code ? log_S : nullptr;
  a.vec = (m % 4 == 0) && (((uintptr_t)ds->X & 15) == 0);
  set_blocks<E>(a, o);
  a.R0 = r0buf;
  a.R0min = r0min;
  a.r0tiles = tiles;
  a.jperm = ds->jperm;
  a.mp = ds->mp;
  if (r0 && !E::kPerm) {
    s = cuda_check(cudaFuncSetAttribute(round0_kernel<E>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)((size_t)rows * m * 4)),
                   "cudaFuncSetAttribute(round0)");
    if (s != KNN_OK) {
      ws.release();
      return s;
    }
  }
  // queries in chunks whose round-0 sums fit the buffer: round 0 point-major,
  // then the remaining rounds of the chunk's queries
  for (int32_t q0 = 0; q0 < nq && s == KNN_OK; q0 += chunk) {
    AdaptiveArgs ac = a;
    ac.nq = std::min(chunk, nq - q0);
    ac.Q = Q + (size_t)q0 * m;
    ac.out_idx = out_idx + (size_t)q0 * a.out_stride;
    ac.out_count = out_count + q0;
    ac.out_evals = out_evals + q0;
    ac.out_rounds = out_rounds ? out_rounds + q0 : nullptr;
    ac.log_code = log_code ? log_code + (size_t)q0 * n : nullptr;
    ac.log_S = a.log_S ? a.log_S + (size_t)q0 * n : nullptr;
    ac.kq = a.kq ? a.kq + q0 : nullptr;
    ac.qids = a.qids ? a.qids + q0 : nullptr;
    ac.qid_base = a.qid_base + (uint64_t)q0;
    s = cuda_check(cudaMemsetAsync(c.queue, 0, 4, stream), "memset(queue)");
    if (s == KNN_OK && r0) {
      if constexpr (E::kPerm) {
        const unsigned blocks = (unsigned)((n + kR0SharedThreads - 1) / kR0SharedThreads);
        const int64_t cnt = (int64_t)ac.nq * qpw;
        permute_query_columns_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, stream>>>(ac.Q, m, ac.nq, ds->jperm,
                                                                                         o.B0, qpw, qperm);
        s = cuda_check(cudaGetLastError(), "permute_query_columns_kernel launch");
        if (s != KNN_OK) break;
        if (o.B0 <= 16) {
          const dim3 grid(blocks, (unsigned)((ac.nq + R0SharedCfg<2>::kQueries - 1) / R0SharedCfg<2>::kQueries));
          round0_shared_kernel<E, 2><<<grid, kR0SharedThreads, 0, stream>>>(ac, qperm, r0buf, r0min);
        } else if (o.B0 <= 32) {
          const dim3 grid(blocks, (unsigned)((ac.nq + R0SharedCfg<4>::kQueries - 1) / R0SharedCfg<4>::kQueries));
          round0_shared_kernel<E, 4><<<grid, kR0SharedThreads, 0, stream>>>(ac, qperm, r0buf, r0min);
        } else {
          const dim3 grid(blocks, (unsigned)((ac.nq + R0SharedCfg<8>::kQueries - 1) / R0SharedCfg<8>::kQueries));
          round0_shared_kernel<E, 8><<<grid, kR0SharedThreads, 0, stream>>>(ac, qperm, r0buf, r0min);
        }
        s = cuda_check(cudaGetLastError(), "round0_shared_kernel launch");
      } else {
        const unsigned blocks = (unsigned)((n + rows - 1) / rows);
        round0_kernel<E><<<blocks, kR0Threads, (size_t)rows * m * 4, stream>>>(ac, rows, r0buf, r0min);
        s = cuda_check(cudaGetLastError(), "round0_kernel launch");
      }
    }
    if (s == KNN_OK) s = launch_rounds<E>(p, ac, stream);
  }
  ws.release();
  return s;
}

// Element type of the launch: the shared-coordinate copy when both counter
// masks are zero and the dataset holds that copy for this seed, else the
// stored copy with per-pair draws.
static knn_status dispatch_ds(const knn_dataset* ds, int32_t storage, const float* Q, int32_t nq, int32_t k,
                              double delta, uint64_t seed, const knn_opts& o, int64_t* out_idx, int32_t* out_count,
                              int64_t* out_evals, int32_t* out_rounds, int32_t* log_code, float* log_S,
                              void* workspace, size_t workspace_bytes, cudaStream_t stream, const MixedBatch* mix) {
  // (shared-coordinate copies hold single coordinates: block samples draw per pair)
  const bool shared = o.mask_p == 0 && o.mask_q == 0 && o.block <= 1 && ((ds->share_ready >> storage) & 1) &&
                      ds->share_seed == seed;
#define KNN_DS_LAUNCH(E)                                                                                        \
  return adaptive_ds_launch<E>(ds, Q, nq, k, delta, seed, o, out_idx, out_count, out_evals, out_rounds, log_code, \
                               log_S, workspace, workspace_bytes, stream, mix)
  if (shared) {
    if (storage == KNN_STORE_BF16) KNN_DS_LAUNCH(Perm<ElemBF16>);
    if (storage == KNN_STORE_FP8) KNN_DS_LAUNCH(Perm<ElemFP8>);
    KNN_DS_LAUNCH(Perm<ElemF32>);
  }
  if (o.block > 1) {
    if (storage == KNN_STORE_BF16) KNN_DS_LAUNCH(Blk<ElemBF16>);
    if (storage == KNN_STORE_FP8) KNN_DS_LAUNCH(Blk<ElemFP8>);
    KNN_DS_LAUNCH(Blk<ElemF32>);
  }
  if (storage == KNN_STORE_BF16) KNN_DS_LAUNCH(ElemBF16);
  if (storage == KNN_STORE_FP8) KNN_DS_LAUNCH(ElemFP8);
  KNN_DS_LAUNCH(ElemF32);
#undef KNN_DS_LAUNCH
}

extern "C" knn_status knn_adaptive_ds(const knn_dataset* ds, int32_t storage, const float* Q, int32_t nq, int32_t k,
                                      double delta, uint64_t seed, const knn_opts* opts, int64_t* out_idx,
                                      int32_t* out_count, int64_t* out_evals, int32_t* out_rounds, int32_t* log_code,
                                      float* log_S, void* workspace, size_t workspace_bytes, void* stream_) {
  clear_error();
  if (!ds) return set_error("knn_adaptive_ds: null dataset"), KNN_EINVAL;
  const knn_opts o = resolve(opts, k);
  knn_status s = validate(ds->n, ds->m, nq, k, delta, o);
  if (s != KNN_OK) return s;
  if (storage < 0 || storage > 2) return set_error("unknown storage"), KNN_EINVAL;
  if ((storage == KNN_STORE_BF16 && !ds->xb) || (storage == KNN_STORE_FP8 && !ds->x8))
    return set_error("knn_adaptive_ds: the dataset was created without that copy"), KNN_EINVAL;
  if (nq == 0) return KNN_OK;
  if (!Q || !out_idx || !out_count || !out_evals)
    return set_error("Q, out_idx, out_count and out_evals are required"), KNN_EINVAL;
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  return dispatch_ds(ds, storage, Q, nq, k, delta, seed, o, out_idx, out_count, out_evals, out_rounds, log_code,
                     log_S, workspace, workspace_bytes, stream, nullptr);
}

extern "C" size_t knn_adaptive_ds_multi_workspace_size(const knn_dataset* ds, int32_t nq, int32_t k_max,
                                                       const knn_opts* opts) {
  if (!ds) return 0;
  return knn_adaptive_workspace_size(ds->n, ds->m, nq, k_max, opts);
}

extern "C" knn_status knn_adaptive_ds_multi(const knn_dataset* ds, int32_t storage, const float* Q, int32_t nq,
                                            const int32_t* k_per_query, int32_t k_max, const uint64_t* query_ids,
                                            double delta, uint64_t seed, const knn_opts* opts, int64_t* out_idx,
                                            int32_t* out_count, int64_t* out_evals, int32_t* out_rounds,
                                            void* workspace, size_t workspace_bytes, void* stream_) {
  clear_error();
  if (!ds) return set_error("knn_adaptive_ds_multi: null dataset"), KNN_EINVAL;
  knn_opts raw;
  knn_opts_default(&raw);
  if (opts) raw = *opts;
  const knn_opts o = resolve(opts, k_max);  // h resolved for the largest k: the bound on k + h
  knn_status s = validate(ds->n, ds->m, nq, k_max, delta, o);
  if (s != KNN_OK) return s;
  if (storage < 0 || storage > 2) return set_error("unknown storage"), KNN_EINVAL;
  if ((storage == KNN_STORE_BF16 && !ds->xb) || (storage == KNN_STORE_FP8 && !ds->x8))
    return set_error("knn_adaptive_ds_multi: the dataset was created without that copy"), KNN_EINVAL;
  if (nq == 0) return KNN_OK;
  if (!Q || !k_per_query || !query_ids || !out_idx || !out_count || !out_evals)
    return set_error("knn_adaptive_ds_multi: Q, k_per_query, query_ids and the outputs are required"), KNN_EINVAL;
  MixedBatch mix;
  mix.kq = k_per_query;
  mix.qids = query_ids;
  mix.h_per_k = raw.h < 0 ? 1 : 0;
  mix.out_stride = k_max + o.h;
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  return dispatch_ds(ds, storage, Q, nq, k_max, delta, seed, o, out_idx, out_count, out_evals, out_rounds, nullptr,
                     nullptr, workspace, workspace_bytes, stream, &mix);
}

extern "C" knn_status knn_dataset_share(knn_dataset* ds, uint64_t seed, int32_t copies, void* stream_) {
  clear_error();
  if (!ds) return set_error("knn_dataset_share: null dataset"), KNN_EINVAL;
  if (copies & ~((1 << KNN_STORE_F32) | (1 << KNN_STORE_BF16) | (1 << KNN_STORE_FP8)))
    return set_error("knn_dataset_share: copies must be a mask of F32, BF16 and FP8"), KNN_EINVAL;
  if (((copies >> KNN_STORE_BF16) & 1) && !ds->xb)
    return set_error("knn_dataset_share: the dataset has no BF16 copy"), KNN_EINVAL;
  if (((copies >> KNN_STORE_FP8) & 1) && !ds->x8)
    return set_error("knn_dataset_share: the dataset has no FP8 copy"), KNN_EINVAL;
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  const int64_t n = ds->n;
  const int m = ds->m;
  ds->mp = (m + 7) & ~7;
  const size_t cnt = (size_t)n * (size_t)ds->mp;
  knn_status s = KNN_OK;
  if (!ds->jperm) s = cuda_check(cudaMalloc(&ds->jperm, (size_t)m * 4), "cudaMalloc(columns)");
  if (s == KNN_OK && ((copies >> KNN_STORE_F32) & 1) && !ds->p32)
    s = cuda_check(cudaMalloc(&ds->p32, cnt * 4), "cudaMalloc(shared F32 copy)");
  if (s == KNN_OK && ((copies >> KNN_STORE_BF16) & 1) && !ds->pb)
    s = cuda_check(cudaMalloc(&ds->pb, cnt * 2), "cudaMalloc(shared BF16 copy)");
  if (s == KNN_OK && ((copies >> KNN_STORE_FP8) & 1) && !ds->p8)
    s = cuda_check(cudaMalloc(&ds->p8, cnt), "cudaMalloc(shared FP8 copy)");
  if (s != KNN_OK) return s;
  ds->share_ready = 0;
  shared_columns_kernel<<<(m + 255) / 256, 256, 0, stream>>>(seed, m, ds->jperm);
  DeviceInfo di;
  s = device_info(&di);
  if (s != KNN_OK) return s;
  const int blocks = (int)std::min<int64_t>(n, (int64_t)di.sms * 16);
  if ((copies >> KNN_STORE_F32) & 1) permute_rows_kernel<float><<<blocks, 256, 0, stream>>>(ds->X, n, m, ds->mp, ds->jperm, ds->p32);
  if ((copies >> KNN_STORE_BF16) & 1) permute_rows_kernel<uint16_t><<<blocks, 256, 0, stream>>>(ds->xb, n, m, ds->mp, ds->jperm, ds->pb);
  if ((copies >> KNN_STORE_FP8) & 1) permute_rows_kernel<uint8_t><<<blocks, 256, 0, stream>>>(ds->x8, n, m, ds->mp, ds->jperm, ds->p8);
  s = cuda_check(cudaGetLastError(), "shared-coordinate kernels");
  if (s == KNN_OK) s = cuda_check(cudaStreamSynchronize(stream), "shared-coordinate build");
  if (s == KNN_OK) {
    ds->share_seed = seed;
    ds->share_ready = copies;
  }
  return s;
}
