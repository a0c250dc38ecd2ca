// adaptive.cu -- C-ABI entry points of the adaptive rounds over an FP32
// matrix: knn_adaptive (workspace from the caller or stream-ordered) and
// knn_adaptive_noalloc (scratch in a fixed device array). The kernel itself
// is in adaptive_kernel.cuh.
#include <mutex>
#include <string>

#include "adaptive_kernel.cuh"

using namespace knn;

extern "C" void knn_opts_default(knn_opts* o) {
  if (!o) return;
  o->h = -1;
  o->bound = KNN_BOUND_FOOTNOTE;
  o->c_alpha = 1.0;
  o->B0 = 16;
  o->B = 16;
  o->grow = 0;
  o->qid_base = 0;
  o->mask_p = ~0ULL;
  o->mask_q = ~0ULL;
  o->threads = 0;
  o->max_ctas = 0;
  o->block = 1;
  o->metric = KNN_METRIC_L2SQ;
  o->sampling = KNN_SAMPLE_WITH;
  o->r0_tensor = 0;
  o->query_order = 1;
  o->row_pass = 1;
}

extern "C" size_t knn_adaptive_workspace_size(int64_t n, int32_t m, int32_t nq, int32_t k, const knn_opts* opts) {
  const knn_opts o = resolve(opts, k);
  AdaptivePlan p;
  const knn_status ps = o.block > 1 ? plan_adaptive<Blk<ElemF32>>(n, m, nq, k, &o, &p)
                                    : plan_adaptive<ElemF32>(n, m, nq, k, &o, &p);
  if (ps != KNN_OK) return 0;
  Carve cv;
  carve_adaptive(cv, n, p, nullptr);
  if (round0_applies(m, o) || (o.block <= 1 && o.B0 < m && o.B0 <= 64)) {  // dataset paths only
    const size_t chunk = (size_t)round0_chunk(n, nq, p.grid);
    cv.take<float>(chunk * (size_t)n);                                      // round-0 sums
    const int64_t rows = round0_rows(m, o.B0);
    cv.take<float>(chunk * (size_t)std::max<int64_t>((n + rows - 1) / rows, (n + 31) / 32));  // their tile minima
    cv.take<float>(chunk * 64);                                             // permuted query columns
    if (o.r0_tensor && o.B0 <= 64) cv.take<uint8_t>(round0_tc_scratch(n, (int32_t)chunk));  // tensor-core round 0
  }
  {  // the locality order of a chunk (dataset paths: chunks of round0_chunk queries, or the whole batch)
    const size_t chunk = nq <= kOrderMax ? (size_t)nq : (size_t)round0_chunk(n, nq, p.grid);
    if (o.query_order && chunk >= 2 && chunk <= (size_t)kOrderMax)
      cv.take<uint8_t>(query_order_scratch(m, (int32_t)chunk));
  }
  return cv.off + 256;
}

extern "C" knn_status knn_adaptive(const float* X, int64_t n, int32_t m, const float* Q, int32_t nq, int32_t k,
                                   double delta, uint64_t seed, const knn_opts* opts, int64_t* out_idx,
                                   int32_t* out_count, int64_t* out_evals, int32_t* out_rounds, int32_t* log_code,
                                   float* log_S, void* workspace, size_t workspace_bytes, void* stream_) {
  clear_error();
  const knn_opts o = resolve(opts, k);
  knn_status s = validate(n, m, nq, k, delta, o);
  if (s != KNN_OK) return s;
  if (nq == 0) return KNN_OK;
  if (!X || !Q || !out_idx || !out_count || !out_evals) {
    set_error("X, Q, out_idx, out_count and out_evals are required");
    return KNN_EINVAL;
  }
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  AdaptivePlan p;
  s = o.block > 1 ? plan_adaptive<Blk<ElemF32>>(n, m, nq, k, &o, &p) : plan_adaptive<ElemF32>(n, m, nq, k, &o, &p);
  if (s != KNN_OK) return s;
  Carve measure;
  const size_t need = carve_adaptive(measure, n, p, nullptr) + 256;
  Workspace ws;
  s = ws.acquire(workspace, workspace_bytes, need, stream);
  if (s != KNN_OK) return s;
  Carve cv;
  cv.base = reinterpret_cast<uint8_t*>(((uintptr_t)ws.ptr + 255) & ~uintptr_t(255));
  AdaptiveCarve c;
  carve_adaptive(cv, n, p, &c);

  // span: min/max of the data (keys), then the rounds
  s = cuda_check(cudaMemsetAsync(c.xrange, 0xFF, 4, stream), "memset(range)");
  if (s == KNN_OK) s = cuda_check(cudaMemsetAsync(c.xrange + 1, 0x00, 8, stream), "memset(range)");
  if (s == KNN_OK) s = cuda_check(cudaMemsetAsync(c.queue, 0, 4, stream), "memset(queue)");
  if (s != KNN_OK) {
    ws.release();
    return s;
  }
  {
    DeviceInfo di;
    device_info(&di);
    const size_t count = (size_t)n * (size_t)m;
    int blocks = (int)std::min<size_t>((count + 255) / 256, (size_t)di.sms * 8);
    if (blocks < 1) blocks = 1;
    minmax_kernel<<<blocks, 256, 0, stream>>>(X, count, c.xrange);
    s = cuda_check(cudaGetLastError(), "minmax_kernel launch");
    if (s != KNN_OK) {
      ws.release();
      return s;
    }
  }

  AdaptiveArgs a;
  a.X = X;
  a.G = X;
  a.gscale = nullptr;
  a.emax = nullptr;
  a.Q = Q;
  a.n = n;
  a.m = m;
  a.nq = nq;
  a.k = k;
  a.h = o.h;
  a.kq = nullptr;
  a.qids = nullptr;
  a.h_per_k = 0;
  a.out_stride = k + o.h;
  a.R0 = nullptr;
  a.R0min = nullptr;
  a.r0tiles = 0;
  a.jperm = nullptr;
  a.mp = 0;
  a.phase_clk = phase_clocks_ptr();
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
  a.rk = philox_keys(seed);
  a.qid_base = o.qid_base;
  a.mask_p = o.mask_p;
  a.mask_q = o.mask_q;
  a.xrange = c.xrange;
  a.ws_ids = c.ids;
  a.ws_S = c.S;
  a.ws_C = c.C;
  a.ws_acc_id = c.acc_id;
  a.ws_acc_d = c.acc_d;
  a.ws_acc_U = c.acc_U;
  a.ws_acc_L = c.acc_L;
  a.acc_cap = p.acc_cap;
  a.ws_F = c.F;
  a.fuse_cap = p.fuse_cap;
  a.queue = c.queue;
  a.out_idx = out_idx;
  a.out_count = out_count;
  a.out_evals = out_evals;
  a.out_rounds = out_rounds;
  a.log_code = log_code;
  a.log_S = log_code ? log_S : nullptr;
  a.vec = (m % 4 == 0) && (((uintptr_t)X & 15) == 0);
  if (o.block > 1) {
    set_blocks<Blk<ElemF32>>(a, o);
    s = launch_rounds<Blk<ElemF32>>(p, a, stream);
  } else if (o.sampling == KNN_SAMPLE_WITHOUT) {
    set_blocks<Wor<ElemF32>>(a, o);
    s = launch_rounds<Wor<ElemF32>>(p, a, stream);
  } else {
    set_blocks<ElemF32>(a, o);
    s = launch_rounds<ElemF32>(p, a, stream);
  }
  ws.release();
  return s;
}

// ------------------------------------------------- entry without allocation
// knn_adaptive_noalloc runs the same round-loop kernel as knn_adaptive but
// takes its scratch (data range, work-queue counter, the per-CTA active lists
// and accepted lists) from this fixed array instead of a workspace. Every GPU
// that loads the library holds the array until the process exits.
namespace knn {

constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;  // 64 MiB
static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocScratchBytes];

static SymbolSlot g_noalloc_slots[64];  // device address of the array, per device and context

// In host code the array's name is only a host-side stand-in; the device
// address is looked up with the device current, once per CUDA context.
static knn_status noalloc_address(void** out) {
  return symbol_address(reinterpret_cast<const void*>(&g_noalloc_scratch), g_noalloc_slots, out,
                        "cudaGetSymbolAddress(no-alloc scratch)");
}

}  // namespace knn

extern "C" size_t knn_adaptive_noalloc_scratch_bytes(void) { return knn::kNoAllocScratchBytes; }

extern "C" knn_status knn_adaptive_noalloc(const float* X, int64_t n, int32_t m, const float* Q, int32_t nq,
                                           int32_t k, double delta, uint64_t seed, const knn_opts* opts,
                                           int64_t* out_idx, int32_t* out_count, int64_t* out_evals,
                                           int32_t* out_rounds, int32_t* log_code, float* log_S, void* stream_) {
  clear_error();
  const knn_opts o = resolve(opts, k);
  knn_status s = validate(n, m, nq, k, delta, o);
  if (s != KNN_OK) return s;
  if (o.block > 1) return set_error("knn_adaptive_noalloc takes single coordinates (block 0 or 1)"), KNN_EINVAL;
  if (o.sampling != KNN_SAMPLE_WITH)
    return set_error("knn_adaptive_noalloc draws with replacement only"), KNN_EINVAL;
  if (nq == 0) return KNN_OK;
  if (!X || !Q || !out_idx || !out_count || !out_evals) {
    set_error("X, Q, out_idx, out_count and out_evals are required");
    return KNN_EINVAL;
  }
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  AdaptivePlan p;
  s = plan_adaptive<ElemF32>(n, m, nq, k, &o, &p);
  if (s != KNN_OK) return s;
  // as many resident CTAs as the fixed scratch holds (each needs 24 n bytes)
  for (;;) {
    Carve measure;
    if (carve_adaptive(measure, n, p, nullptr) <= kNoAllocScratchBytes) break;
    if (p.grid == 1) {
      Carve one;
      set_error("knn_adaptive_noalloc: n = " + std::to_string(n) + " needs " +
                std::to_string(carve_adaptive(one, n, p, nullptr)) + " bytes of scratch for one query at a time; " +
                "the fixed scratch is " + std::to_string(kNoAllocScratchBytes) + " bytes");
      return KNN_EINVAL;
    }
    p.grid = p.grid > 8 ? p.grid - p.grid / 8 : p.grid - 1;
  }
  void* base = nullptr;
  s = noalloc_address(&base);
  if (s != KNN_OK) return s;
  Carve cv;
  cv.base = static_cast<uint8_t*>(base);  // the array is 256-byte aligned
  AdaptiveCarve c;
  carve_adaptive(cv, n, p, &c);

  // the array keeps the previous call's contents: reset what must start fresh
  s = cuda_check(cudaMemsetAsync(c.xrange, 0xFF, 4, stream), "memset(range)");
  if (s == KNN_OK) s = cuda_check(cudaMemsetAsync(c.xrange + 1, 0x00, 8, stream), "memset(range)");
  if (s == KNN_OK) s = cuda_check(cudaMemsetAsync(c.queue, 0, 4, stream), "memset(queue)");
  if (s != KNN_OK) return s;
  {
    DeviceInfo di;
    device_info(&di);
    const size_t count = (size_t)n * (size_t)m;
    int blocks = (int)std::min<size_t>((count + 255) / 256, (size_t)di.sms * 8);
    if (blocks < 1) blocks = 1;
    minmax_kernel<<<blocks, 256, 0, stream>>>(X, count, c.xrange);
    s = cuda_check(cudaGetLastError(), "minmax_kernel launch");
    if (s != KNN_OK) return s;
  }
  AdaptiveArgs a;
  a.X = X;
  a.G = X;
  a.gscale = nullptr;
  a.emax = nullptr;
  a.Q = Q;
  a.n = n;
  a.m = m;
  a.nq = nq;
  a.k = k;
  a.h = o.h;
  a.kq = nullptr;
  a.qids = nullptr;
  a.h_per_k = 0;
  a.out_stride = k + o.h;
  a.R0 = nullptr;
  a.R0min = nullptr;
  a.r0tiles = 0;
  a.jperm = nullptr;
  a.mp = 0;
  a.phase_clk = phase_clocks_ptr();
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
  a.rk = philox_keys(seed);
  a.qid_base = o.qid_base;
  a.mask_p = o.mask_p;
  a.mask_q = o.mask_q;
  a.xrange = c.xrange;
  a.ws_ids = c.ids;
  a.ws_S = c.S;
  a.ws_C = c.C;
  a.ws_acc_id = c.acc_id;
  a.ws_acc_d = c.acc_d;
  a.ws_acc_U = c.acc_U;
  a.ws_acc_L = c.acc_L;
  a.acc_cap = p.acc_cap;
  a.ws_F = c.F;
  a.fuse_cap = p.fuse_cap;
  a.queue = c.queue;
  a.out_idx = out_idx;
  a.out_count = out_count;
  a.out_evals = out_evals;
  a.out_rounds = out_rounds;
  a.log_code = log_code;
  a.log_S = log_code ? log_S : nullptr;
  a.vec = (m % 4 == 0) && (((uintptr_t)X & 15) == 0);
  set_blocks<ElemF32>(a, o);
  return launch_rounds<ElemF32>(p, a, stream);
}

// --------------------------------------------------------- generator rate
namespace knn {
// Each thread evaluates `iters` Philox4x32-10 blocks with the round loop's
// generator (counter: block index, thread, two fixed words; the round keys of
// a fixed seed) and writes the XOR of their words, so that none is dropped.
static __global__ void __launch_bounds__(1024) philox_blocks_kernel(PhiloxKeys K, int64_t iters, uint32_t* out) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t acc = 0;
  for (int64_t i = 0; i < iters; ++i) {
    const uint4 w = philox4x32_10_rk((uint32_t)i, t, 0x9E3779B9u, 0x7F4A7C15u, K);
    acc += w.x ^ w.y ^ w.z ^ w.w;
  }
  out[t] = acc;
}
}  // namespace knn

extern "C" knn_status knn_philox_blocks(int64_t iters, int32_t ctas, uint32_t* out, void* stream) {
  knn::clear_error();
  if (iters < 0 || ctas < 1 || !out) return knn::set_error("knn_philox_blocks: bad arguments"), KNN_EINVAL;
  knn::philox_blocks_kernel<<<ctas, 1024, 0, static_cast<cudaStream_t>(stream)>>>(knn::philox_keys(0x243F6A8885A308D3ull),
                                                                                   iters, out);
  return knn::cuda_check(cudaGetLastError(), "philox_blocks_kernel launch");
}
