// api.cu -- host runtime of the C ABI: error messages, device queries and
// stream-ordered workspaces.
#include <mutex>
#include <string>

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

knn_status device_status_ptr(int** out) {
  static std::mutex mu;
  static int* addr[64] = {};
  int dev = 0;
  knn_status s = cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
  if (s != KNN_OK) return s;
  if (dev < 0 || dev >= 64) {
    set_error("device ordinal out of range");
    return KNN_EUNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    s = cuda_check(cudaGetSymbolAddress(&p, g_device_status), "cudaGetSymbolAddress(status)");
    if (s != KNN_OK) return s;
    addr[dev] = static_cast<int*>(p);
  }
  *out = addr[dev];
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

}  // namespace knn

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
