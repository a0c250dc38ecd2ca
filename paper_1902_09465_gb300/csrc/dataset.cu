// dataset.cu -- resident datasets: the data range computed once, BF16 and
// FP8-e4m3 (per-row scale) copies with their largest element error, and the
// adaptive rounds over a chosen copy (knn_adaptive_ds).
#include <cuda_bf16.h>

#include <string>

#include "dataset_launch.cuh"

namespace knn {
// instantiated in the ds_launch_*.cu translation units
extern template KNN_DS_LAUNCH_DECL(ElemF32);
extern template KNN_DS_LAUNCH_DECL(Perm<ElemF32>);
extern template KNN_DS_LAUNCH_DECL(Blk<ElemF32>);
extern template KNN_DS_LAUNCH_DECL(Wor<ElemF32>);
extern template KNN_DS_LAUNCH_DECL(ElemBF16);
extern template KNN_DS_LAUNCH_DECL(Perm<ElemBF16>);
extern template KNN_DS_LAUNCH_DECL(Blk<ElemBF16>);
extern template KNN_DS_LAUNCH_DECL(ElemFP8);
extern template KNN_DS_LAUNCH_DECL(Perm<ElemFP8>);
extern template KNN_DS_LAUNCH_DECL(Blk<ElemFP8>);
}  // namespace knn

namespace knn {

knn_status build_screen_operand(knn_dataset* ds, int32_t copies, cudaStream_t stream);

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

// Column of draw t under shared coordinates: word t mod 4 of Philox4x32-10
// at counter (t / 4, 0, 0, 0), key (seed words), scaled to [0, m).
static __global__ void shared_columns_kernel(uint64_t seed, int m, int32_t* jperm) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m) return;
  const Draws8 ph = pair_draws8((uint32_t)(t >> 3), 0, 0, seed);
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
  const int32_t screens = KNN_COPY_SCREEN | KNN_COPY_SCREEN_F16 | KNN_COPY_SCREEN_BF16;
  if (copies & ~((1 << KNN_STORE_BF16) | (1 << KNN_STORE_FP8) | screens))
    return set_error("knn_dataset_create: copies must be a mask of BF16, FP8 and the screen operands"), KNN_EINVAL;
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
  if (s == KNN_OK && (copies & screens)) s = build_screen_operand(ds, copies, stream);
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
  cudaFree(ds->screen16);
  cudaFree(ds->screenb);
  cudaFree(ds->mu);
  cudaFree(ds->xcn);
  cudaFree(ds->xcn_max);
  cudaFree(ds->jperm);
  cudaFree(ds->p32);
  cudaFree(ds->pb);
  cudaFree(ds->p8);
  cudaFree(ds->r0mu);
  for (int st = 0; st < 3; ++st) cudaFree(ds->r0op[st]);
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

// Element type of the launch: the shared-coordinate copy when both counter
// masks are zero and the dataset holds that copy for this seed, else the
// stored copy with per-pair draws.
static knn_status dispatch_ds(const knn_dataset* ds, int32_t storage, const float* Q, int32_t nq, int32_t k,
                              double delta, uint64_t seed, const knn_opts& o, int64_t* out_idx, int32_t* out_count,
                              int64_t* out_evals, int32_t* out_rounds, int32_t* log_code, float* log_S,
                              void* workspace, size_t workspace_bytes, cudaStream_t stream, const MixedBatch* mix) {
  // (shared-coordinate copies hold single coordinates: block samples draw per pair)
  const bool shared = o.mask_p == 0 && o.mask_q == 0 && o.block <= 1 && o.sampling == KNN_SAMPLE_WITH &&
                      ((ds->share_ready >> storage) & 1) && ds->share_seed == seed;
#define KNN_DS_LAUNCH(E)                                                                                        \
  return adaptive_ds_launch<E>(ds, Q, nq, k, delta, seed, o, out_idx, out_count, out_evals, out_rounds, log_code, \
                               log_S, workspace, workspace_bytes, stream, mix)
  if (shared) {
    if (storage == KNN_STORE_BF16) KNN_DS_LAUNCH(Perm<ElemBF16>);
    if (storage == KNN_STORE_FP8) KNN_DS_LAUNCH(Perm<ElemFP8>);
    KNN_DS_LAUNCH(Perm<ElemF32>);
  }
  if (o.sampling == KNN_SAMPLE_WITHOUT) {
    if (storage != KNN_STORE_F32)
      return set_error("sampling without replacement gathers from the FP32 data (storage F32)"), KNN_EINVAL;
    KNN_DS_LAUNCH(Wor<ElemF32>);
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
  // the round-0 contraction's operands (centre recomputed for this seed's columns)
  cudaFree(ds->r0mu);
  ds->r0mu = nullptr;
  for (int st = 0; st < 3 && s == KNN_OK; ++st)
    if ((copies >> st) & 1) s = build_round0_operand(ds, st, stream);
  if (s == KNN_OK) s = cuda_check(cudaStreamSynchronize(stream), "shared-coordinate build");
  if (s == KNN_OK) {
    ds->share_seed = seed;
    ds->share_ready = copies;
  }
  return s;
}
