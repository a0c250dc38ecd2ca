// knn_internal.h -- host-side helpers shared by the library's translation
// units: error reporting, workspace carving and device queries.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>

#include "../../include/knn_gb300.h"

namespace knn {

void set_error(const std::string& msg);
void clear_error();

// Returns KNN_ECUDA and records the message if `e` is an error.
knn_status cuda_check(cudaError_t e, const char* what);

// Bump allocator over a caller-provided device buffer (256-byte aligned
// pieces). With base == nullptr it only measures.
struct Carve {
  uint8_t* base = nullptr;
  size_t off = 0;
  template <class T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

struct DeviceInfo {
  int device = 0;
  int sms = 0;
  int major = 0, minor = 0;
  size_t smem_optin = 0;
};
knn_status device_info(DeviceInfo* di);

// Stream-ordered workspace: either the caller's buffer or an allocation
// released on the same stream by release().
struct Workspace {
  void* ptr = nullptr;
  bool owned = false;
  cudaStream_t stream = nullptr;
  knn_status acquire(void* user, size_t user_bytes, size_t need, cudaStream_t s);
  void release();
};

// Device address of a __device__ variable of this library (`symbol` is the
// host-side stand-in the variable's name gives in host code) in the current
// CUDA context. The address is cached per device together with the context's
// unique id, and looked up again when that context changed (after a
// cudaDeviceReset, or a primary context released and created again, the
// module loads anew and the variable may move). The first call in a context
// does the lookup; later calls only compare ids.
struct SymbolSlot {
  unsigned long long ctx = 0;
  void* addr = nullptr;
};
knn_status symbol_address(const void* symbol, SymbolSlot (&slots)[64], void** out, const char* what);

// Round 0 under shared coordinates as a tcgen05 contraction (screen_tc.cu):
// writes R0[q * n + i] = sum_{t < B0} (x_it - q_t)^2 over the first B0
// permuted columns (as ||xc||^2 + ||qc||^2 - 2 xc.qc of centred values, FP32)
// and R0min[q * r0tiles + i / 32] = the smallest sum of each group of 32
// points, for the nq queries of Q (the chunk).
knn_status round0_tc(const knn_dataset* ds, int storage, const float* Q, int32_t nq, int32_t B0, float* R0,
                     float* R0min, int32_t r0tiles, void* scratch, cudaStream_t stream);
size_t round0_tc_scratch(int64_t n, int32_t nq);
knn_status build_round0_operand(knn_dataset* ds, int storage, cudaStream_t stream);

// Library status word of the current device: kernels that give up a bounded
// wait record a code here (read and cleared by knn_device_status).
knn_status device_status_ptr(int** out);

// Device address of the round-loop phase clock totals of the current device
// (16 counters) in a library built with KNN_PHASE_TIMING; null otherwise.
unsigned long long* phase_clocks_ptr();

// Kernel timing of the adaptive calls (knn_kernel_timing): when enabled,
// kernel_mark(stream, kind) records a CUDA event on the stream; the time from
// one mark to the next is charged to the earlier mark's kind (0: round-0 pass,
// 1: round loop, 2: end of a call).
bool kernel_timing_on();
void kernel_mark(cudaStream_t stream, int kind);

}  // namespace knn

// A resident dataset (see knn_dataset_create).
struct knn_dataset {
  const float* X = nullptr;
  int64_t n = 0;
  int32_t m = 0;
  int32_t copies = 0;
  int device = 0;
  uint32_t* range = nullptr;  // [3]: min key, max key (finite values), non-finite flag
  uint16_t* xb = nullptr;     // BF16 copy
  uint8_t* x8 = nullptr;      // FP8 e4m3 copy
  float* scale8 = nullptr;    // FP8 per-row scale
  unsigned* emax = nullptr;   // [3]: largest |copy - X| per storage, as float bits
  float emax_host[3] = {0.0f, 0.0f, 0.0f};
  // tensor-core screen operands of x - mu, each part Kp wide: BF16x3 rows
  // [hi | hi | lo], single FP16 rows (scaled by a power of two), single BF16 rows
  int32_t Kp = 0;
  uint16_t* screenA = nullptr;
  uint16_t* screen16 = nullptr;
  uint16_t* screenb = nullptr;
  float* mu = nullptr;        // column means
  float* xcn = nullptr;       // ||x_i - mu||^2
  unsigned* xcn_max = nullptr;  // [2]: largest ||x_i - mu||^2, largest |x_ij - mu_j| (float bits)
  // shared-coordinate copies for one seed: column t holds column jperm[t]
  uint64_t share_seed = 0;
  int32_t share_ready = 0;    // bit s set: the copy of storage s is built
  int32_t mp = 0;             // row pitch (m rounded up to 8)
  int32_t* jperm = nullptr;
  float* p32 = nullptr;
  uint16_t* pb = nullptr;
  uint8_t* p8 = nullptr;
  // tensor-core operand of the shared round 0, per storage: the first 64
  // permuted columns minus r0mu, split into three BF16 parts [hi | mid | lo]
  float* r0mu = nullptr;
  uint16_t* r0op[3] = {nullptr, nullptr, nullptr};
};
