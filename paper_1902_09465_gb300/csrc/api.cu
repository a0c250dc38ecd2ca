// api.cu -- host runtime of the C ABI: error messages, device queries and
// stream-ordered workspaces.
#include <cuda.h>

#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "knn_internal.h"

namespace knn {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }
void clear_error() { g_last_error.clear(); }

knn_status cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return KNN_OK;
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return KNN_ECUDA;
}

knn_status device_info(DeviceInfo* di) {
  static std::mutex mu;
  static DeviceInfo cache[64];
  static bool have[64] = {};
  int dev = 0;
  knn_status s = cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
  if (s != KNN_OK) return s;
  if (dev < 0 || dev >= 64) {
    set_error("device ordinal out of range");
    return KNN_EUNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (!have[dev]) {
    DeviceInfo d;
    d.device = dev;
    s = cuda_check(cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev), "sm count");
    if (s == KNN_OK) s = cuda_check(cudaDeviceGetAttribute(&d.major, cudaDevAttrComputeCapabilityMajor, dev), "cc");
    if (s == KNN_OK) s = cuda_check(cudaDeviceGetAttribute(&d.minor, cudaDevAttrComputeCapabilityMinor, dev), "cc");
    int optin = 0;
    if (s == KNN_OK)
      s = cuda_check(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev), "smem optin");
    if (s != KNN_OK) return s;
    d.smem_optin = (size_t)optin;
    cache[dev] = d;
    have[dev] = true;
  }
  *di = cache[dev];
  return KNN_OK;
}

knn_status Workspace::acquire(void* user, size_t user_bytes, size_t need, cudaStream_t s) {
  stream = s;
  if (user) {
    if (user_bytes < need) {
      set_error("workspace too small: need " + std::to_string(need) + " bytes, got " + std::to_string(user_bytes));
      return KNN_ENOMEM;
    }
    ptr = user;
    owned = false;
    return KNN_OK;
  }
  cudaError_t e = cudaMallocAsync(&ptr, need, s);
  if (e != cudaSuccess) {
    set_error(std::string("cudaMallocAsync(workspace): ") + cudaGetErrorString(e));
    ptr = nullptr;
    return KNN_ENOMEM;
  }
  owned = true;
  return KNN_OK;
}

void Workspace::release() {
  if (owned && ptr) cudaFreeAsync(ptr, stream);
  ptr = nullptr;
  owned = false;
}

// Status word per device (see knn_device_status).
static __device__ int g_device_status;

// Unique id of the calling thread's current context (cuCtxGetId, resolved
// through the runtime so the library needs no link-time driver dependency).
static knn_status current_context_id(unsigned long long* id) {
  using GetCurrent = CUresult (*)(CUcontext*);
  using GetId = CUresult (*)(CUcontext, unsigned long long*);
  static std::once_flag once;
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrent>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetId>(f);
  });
  if (!get_current || !get_id) {
    set_error("cuCtxGetCurrent / cuCtxGetId unavailable from the driver");
    return KNN_ECUDA;
  }
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS) return set_error("cuCtxGetCurrent failed"), KNN_ECUDA;
  if (!ctx) {
    // no context current yet: cudaSetDevice initialises the device's primary
    // context and makes it current
    int dev = 0;
    knn_status s = cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
    if (s == KNN_OK) s = cuda_check(cudaSetDevice(dev), "cudaSetDevice");
    if (s != KNN_OK) return s;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return set_error("no current CUDA context"), KNN_ECUDA;
  }
  if (get_id(ctx, id) != CUDA_SUCCESS) return set_error("cuCtxGetId failed"), KNN_ECUDA;
  return KNN_OK;
}

knn_status symbol_address(const void* symbol, SymbolSlot (&slots)[64], void** out, const char* what) {
  static std::mutex mu;
  int dev = 0;
  knn_status s = cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
  if (s != KNN_OK) return s;
  if (dev < 0 || dev >= 64) {
    set_error("device ordinal out of range");
    return KNN_EUNSUPPORTED;
  }
  unsigned long long ctx = 0;
  s = current_context_id(&ctx);
  if (s != KNN_OK) return s;
  std::lock_guard<std::mutex> lock(mu);
  if (!slots[dev].addr || slots[dev].ctx != ctx) {
    void* p = nullptr;
    s = cuda_check(cudaGetSymbolAddress(&p, symbol), what);
    if (s != KNN_OK) return s;
    slots[dev].addr = p;
    slots[dev].ctx = ctx;
  }
  *out = slots[dev].addr;
  return KNN_OK;
}

knn_status device_status_ptr(int** out) {
  static SymbolSlot slots[64];
  void* p = nullptr;
  knn_status s = symbol_address(reinterpret_cast<const void*>(&g_device_status), slots, &p,
                                "cudaGetSymbolAddress(status)");
  if (s != KNN_OK) return s;
  *out = static_cast<int*>(p);
  return KNN_OK;
}

#ifdef KNN_PHASE_TIMING
// Phase clock totals of the round-loop kernel (see knn_phase_clocks).
static __device__ unsigned long long g_phase_clk[16];

unsigned long long* phase_clocks_ptr() {
  void* p = nullptr;
  return cudaGetSymbolAddress(&p, g_phase_clk) == cudaSuccess ? static_cast<unsigned long long*>(p) : nullptr;
}
#else
unsigned long long* phase_clocks_ptr() { return nullptr; }
#endif

// Events of the marks of the last timed call(s), host side.
static std::mutex g_timing_mu;
static bool g_timing = false;
static std::vector<std::pair<cudaEvent_t, int>> g_marks;  // (event, kind) in stream order
static std::vector<cudaEvent_t> g_event_pool;

bool kernel_timing_on() { return g_timing; }

void kernel_mark(cudaStream_t stream, int kind) {
  std::lock_guard<std::mutex> lock(g_timing_mu);
  if (!g_timing) return;
  cudaEvent_t ev;
  if (g_event_pool.empty()) {
    if (cudaEventCreate(&ev) != cudaSuccess) return;
  } else {
    ev = g_event_pool.back();
    g_event_pool.pop_back();
  }
  if (cudaEventRecord(ev, stream) != cudaSuccess) {
    g_event_pool.push_back(ev);
    return;
  }
  g_marks.emplace_back(ev, kind);
}

}  // namespace knn

extern "C" knn_status knn_kernel_timing(int32_t enable) {
  knn::clear_error();
  std::lock_guard<std::mutex> lock(knn::g_timing_mu);
  knn::g_timing = enable != 0;
  return KNN_OK;
}

extern "C" knn_status knn_kernel_times(double* out_ms, int32_t reset) {
  knn::clear_error();
  if (!out_ms) return knn::set_error("knn_kernel_times: null pointer"), KNN_EINVAL;
  std::lock_guard<std::mutex> lock(knn::g_timing_mu);
  out_ms[0] = out_ms[1] = 0.0;
  auto& mk = knn::g_marks;
  knn_status s = KNN_OK;
  if (!mk.empty()) s = knn::cuda_check(cudaEventSynchronize(mk.back().first), "cudaEventSynchronize");
  for (size_t i = 0; s == KNN_OK && i + 1 < mk.size(); ++i) {
    if (mk[i].second > 1) continue;
    float ms = 0.0f;
    s = knn::cuda_check(cudaEventElapsedTime(&ms, mk[i].first, mk[i + 1].first), "cudaEventElapsedTime");
    out_ms[mk[i].second] += ms;
  }
  if (reset) {
    for (auto& e : mk) knn::g_event_pool.push_back(e.first);
    mk.clear();
  }
  return s;
}

extern "C" knn_status knn_phase_clocks(uint64_t* out, int32_t reset) {
  knn::clear_error();
  if (!out) return knn::set_error("knn_phase_clocks: null pointer"), KNN_EINVAL;
  unsigned long long* p = knn::phase_clocks_ptr();
  if (!p) return knn::set_error("knn_phase_clocks: library built without phase timing"), KNN_EUNSUPPORTED;
  unsigned long long v[16];
  knn_status s = knn::cuda_check(cudaMemcpy(v, p, sizeof(v), cudaMemcpyDeviceToHost), "read phase clocks");
  if (s == KNN_OK && reset) s = knn::cuda_check(cudaMemset(p, 0, sizeof(v)), "clear phase clocks");
  for (int i = 0; i < 16; ++i) out[i] = (uint64_t)v[i];
  return s;
}

extern "C" knn_status knn_device_status(int32_t* out) {
  knn::clear_error();
  if (!out) return knn::set_error("knn_device_status: null pointer"), KNN_EINVAL;
  int* p = nullptr;
  knn_status s = knn::device_status_ptr(&p);
  if (s != KNN_OK) return s;
  int v = 0;
  s = knn::cuda_check(cudaMemcpy(&v, p, sizeof(int), cudaMemcpyDeviceToHost), "read status");
  if (s == KNN_OK && v != 0) s = knn::cuda_check(cudaMemset(p, 0, sizeof(int)), "clear status");
  *out = v;
  return s;
}

extern "C" const char* knn_last_error(void) { return knn::g_last_error.c_str(); }

extern "C" const char* knn_version(void) { return "knn_gb300 0.1 (sm_103a)"; }
