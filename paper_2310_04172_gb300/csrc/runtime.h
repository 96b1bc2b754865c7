// Host runtime pieces shared by the C-ABI translation units: error
// reporting, per-device state, per-(device, stream) workspace, phase timing,
// and the map object.
#pragma once

#include <cstdarg>
#include <cstdint>

#include "mcl_internal.h"

namespace mcl {

mcl_status fail(mcl_status s, const char* fmt, ...);
mcl_status cuda_fail(cudaError_t e, const char* what);

#define MCL_CUDA(call)                                        \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return ::mcl::cuda_fail(e_, #call); \
  } while (0)

constexpr int64_t kMaxCount = 2147483647LL;

struct DeviceState {
  unsigned* status = nullptr;
  int sms = 0;
};

mcl_status device_state(int* dev_out, DeviceState* out);
mcl_status workspace(cudaStream_t s, size_t bytes, void** out);

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
inline bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }
inline bool finite_pos(float v) { return v == v && v > 0.f && v < 3.4e38f; }

// Brackets the work enqueued in its scope with CUDA events while profiling is on.
class PhaseScope {
 public:
  PhaseScope(int phase, cudaStream_t s, int kernels = 1);
  ~PhaseScope();

 private:
  int phase_, kernels_;
  cudaStream_t s_;
  cudaEvent_t a_ = nullptr, b_ = nullptr;
};

// Launch shape and workspace layout of one sensor update.
struct Plan {
  SensorShape sh;
  int K, nblk, blocks_per_sm, sms;
  bool spatial;
  long long n_items;
  size_t off_mats, off_scan, off_partial, off_logw, off_stats, off_ostats, off_est, off_key,
      off_rank, off_hist, total;
};

mcl_status check_params(const mcl_sensor_params* p);
mcl_status make_plan(mcl_map_t m, int64_t P, int64_t N, const mcl_sensor_params* p, Plan* pl);
mcl_status check_device(mcl_map_t m);

}  // namespace mcl

struct mcl_map_s {
  int device = 0;
  int kind = 0, dtype = 0;
  mcl::MapView view{};
  void* d_values = nullptr;
  uint2* d_table = nullptr;
  int64_t bytes = 0, n_bricks = 0, capacity = 0;
  int max_probe = 0;
};

