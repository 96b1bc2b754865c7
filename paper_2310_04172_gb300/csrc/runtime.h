// Host runtime pieces shared by the C-ABI translation units: error
// reporting, per-device state, per-(device, stream) workspace, phase timing,
// and the map object.
#pragma once

#include <cstdarg>
#include <cstdint>
#include <vector>

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

// Maps whose sessions can share one batched sensor launch (same kernel kind,
// layout, storage type, geometry and kind of values), and the per-session
// map fields of a batch table entry (mcl_batch.cpp).
bool same_geometry(const mcl_map_s* a, const mcl_map_s* b);
void session_map(const mcl_map_s* m, BatchSession* t);

// Batched side launches (mcl_side.cpp): the session table and the block
// prefix of every launch kind, written into one host buffer of
// side_table_bytes(n) bytes whose device copy lives at d.
struct SideTables {
  const SideSeg* segs = nullptr;  // device
  SegBlocks b[kSideLaunches];
};
size_t side_table_bytes(int n);
void side_tables(const std::vector<SideSeg>& segs, char* h, char* d, SideTables* out);
mcl_status enqueue_side(const SideTables& t, int kind, cudaStream_t s);
int side_launch_count(const SideTables& t);  // launch kinds with work

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
  int sweep;  // particle blocks per sweep of the item order (nblk: chunk-major)
  bool spatial;
  bool dynamic;  // items handed out by a device counter (item order 3)
  long long n_items;
  size_t off_mats, off_scan, off_partial, off_logw, off_stats, off_ostats, off_est, off_key,
      off_rank, off_hist, off_queue, total;
};

// Enqueues one sensor update (pose matrices, scan packing, sensor kernel,
// log-weights, normalisation with the optional fused estimate) on s, with the
// plan's workspace at ws. Arguments must already be validated.
mcl_status enqueue_sensor(mcl_map_t m, const float* particles, int64_t P, const float* scan,
                          int64_t N, const mcl_sensor_params* p, float* logw, float* w,
                          mcl_estimate* est, const Plan& pl, char* ws, unsigned* status,
                          cudaStream_t s);

// While one is alive on a thread, PhaseScope records nothing on that thread
// (work enqueued into a stream that is being captured into a graph).
class NoProfileScope {
 public:
  NoProfileScope();
  ~NoProfileScope();

 private:
  bool prev_;
};

// Resampling offset r in [0, 1) of a filter step: the SplitMix64 finaliser of
// (seed, step) as a counter hash, 53 bits.
inline double resample_offset(uint64_t seed, uint64_t step) {
  uint64_t z = seed ^ (step * 0x9E3779B97F4A7C15ull);
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * 0x1.0p-53;
}

mcl_status check_params(const mcl_sensor_params* p);
mcl_status make_plan(mcl_map_t m, int64_t P, int64_t N, const mcl_sensor_params* p, Plan* pl);
mcl_status check_device(mcl_map_t m);

}  // namespace mcl

struct mcl_map_s {
  int device = 0;
  int kind = 0, dtype = 0;
  mcl::MapView view{};
  void* d_values = nullptr;
  uint2* d_table = nullptr;     // hash index
  uint32_t* d_grid = nullptr;   // grid index (allocation; view.grid = d_grid + grid_front)
  int64_t grid_cells = 0;       // cells allocated, guard cells included
  int64_t grid_front = 0;       // guard cells in front of cell (0, 0, 0)
  bool dense_tiles = false;     // DENSE: values in 8 x 4 tiles (kKindDenseTiles)
  int64_t bytes = 0, n_bricks = 0, capacity = 0;
  int max_probe = 0;
  float score_sigma = 0.f;    // > 0: values are scores for this sigma
  float score_outside = 0.f;  // score map: value read where nothing is stored
};

namespace mcl {

// Kernel kind of a map: dense (linear or in tiles), brick with the hash
// index (layout chosen at run time) or brick with the grid index.
inline int kernel_kind(const mcl_map_s* m) {
  if (m->d_grid) return kKindBrickGrid;
  return m->kind == MCL_MAP_DENSE && m->dense_tiles ? kKindDenseTiles : m->kind;
}

// Item order of a batched sensor launch (ItemSeg). Without interleaving,
// session by session, each in its own sweeps. With it (dynamic item order):
// a session alone on its map keeps its own sweeps; sessions that read the
// same map values are interleaved sweep by sweep, in
// R rounds with R about their items / slots (at most max_rounds), each
// session's sweep cut to ceil(blocks / R), so that round r covers the same
// fraction of every such session's spatial order and the items in flight read
// one region of the map for all of them, as one session's sweep does (4
// sessions of 250,000 particles on one building: 8.35 DRAM bytes per
// evaluation session by session). sweeps: the sweep of each session.
struct SegSession {
  const void* values;
  int nblk, K, sweep;
};
long long item_segments(const std::vector<SegSession>& s, long long slots, bool interleave, int max_rounds,
                        std::vector<int>* sweeps, std::vector<ItemSeg>* segs);
constexpr int kBatchMaxRounds = 1024;   // batches (tables built once)
constexpr int kServerMaxRounds = 256;   // serving steps (tables in a fixed slot buffer)

// Ring count of the 4-ring x 8-point patch staging (SensorShape::rings)
// for a scan of N points that the caller says holds `rings` rings, ring
// after ring: `rings` when it divides N, is a multiple of 4 and N / rings
// one of 8, else 0 (the points staged in the order given). The rule
// make_plan applies to the scan size it plans for; a serving step applies it
// to each submitted scan's own size.
inline int patch_rings(int64_t N, int rings) {
  return rings > 0 && N % rings == 0 && rings % 4 == 0 && (N / rings) % 8 == 0 ? rings : 0;
}

// SUM mode: the kernel forms each point's p_hit without its constant as
// 2^(v^2 cs) with the hardware base-2 exponential, v the stored value in
// storage units: cs = -log2(e) / (2 sigma^2), times scale^2 for int16
// values (FP64, one FP32 rounding).
inline float sum_exponent_constant(double sigma, bool q16, double scale) {
  return (float)(-1.4426950408889634 / (2.0 * sigma * sigma) * (q16 ? scale * scale : 1.0));
}

// Kernel mode and the value read where nothing is stored (storage units)
// of a sensor update on map m with the caller's mode.
inline int kernel_mode(const mcl_map_s* m, int mode) { return m->score_sigma > 0.f ? kModeScore : mode; }
inline float outside_raw(const mcl_map_s* m) {
  if (m->score_sigma > 0.f) return m->score_outside;
  return m->dtype == MCL_I16 ? 32767.0f : m->view.tau;
}
// The values a read takes where nothing is stored (SensorArgs::vout, vnear)
// for the kernel mode a->mode and neglect flag a->neglect on map m.
inline void set_fills(const mcl_map_s* m, SensorArgs* a) {
  a->vout = outside_raw(m);
  if (!a->neglect) a->vnear = a->vout;
  else a->vnear = a->mode == MCL_SUM ? __builtin_huge_valf() : 0.0f;
}
// EINVAL unless the parameters fit the map (a score map needs SUM, its own
// sigma and the nearest-voxel read).
mcl_status check_map_params(mcl_map_t m, const mcl_sensor_params* p);

}  // namespace mcl
