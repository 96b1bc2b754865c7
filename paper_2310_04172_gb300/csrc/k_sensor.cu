// Sensor update kernel (Sec. III, Eq. 3; Sec. V-B), GB300 design.
//
// The paper evaluates one particle per thread and loops over all scan points.
// Here a persistent grid walks work items (point chunk c, block of `ppi`
// particles) strided by the grid size. The CTA holds the chunk's scan points in
// shared memory, staged with one bulk asynchronous copy (cp.async.bulk,
// completion on an mbarrier) and re-staged only when the item's chunk changes;
// that is the only CTA-wide barrier. A group of G lanes owns one particle: lane
// l of the group takes points l, l + G, l + 2G, ... of the chunk, so
// neighbouring lanes read neighbouring scan points (neighbouring azimuths of
// one ring) and their map gathers fall in the same or adjacent sectors. Each
// lane keeps U look-ups in flight per step (brick-index entries first, then
// the values). Per-point terms are summed in FP32 per lane in point order, then
// over the group with a fixed xor-shuffle tree; lane 0 of the group writes the
// particle's chunk sum to partial[c * P + p]. The summation order depends only
// on (chunk, G).
//
// LOGPROD accumulates d^2 (the score -d^2 / (2 sigma^2) is applied once per
// particle when the chunks are added); SUM accumulates exp(-d^2 / (2 sigma^2))
// (Eq. 3 without its constant, applied at the end). For int16 maps the terms
// use the stored integer q (d = q * scale): LOGPROD accumulates q^2 and the
// chunk sum is multiplied by scale^2 once; SUM folds scale^2 into the exponent
// constant. A point without a stored value reads +tau (q = 32767 for int16).
#include <algorithm>
#include <map>
#include <mutex>

#include "mcl_internal.h"

namespace mcl {

#define MCL_SENSOR_UNIT(d, k) void* sensor_kernel_##d##_##k(int mode, const SensorShape& sh, bool batch);
#define MCL_SENSOR_UNITS(d)                                                                   \
  MCL_SENSOR_UNIT(d, dense) MCL_SENSOR_UNIT(d, hash) MCL_SENSOR_UNIT(d, block4) MCL_SENSOR_UNIT(d, grid) \
  MCL_SENSOR_UNIT(d, tiles)
MCL_SENSOR_UNITS(f32)
MCL_SENSOR_UNITS(f16)
MCL_SENSOR_UNITS(i16)
#undef MCL_SENSOR_UNITS
#undef MCL_SENSOR_UNIT

namespace {

// Kernel for (map kind, brick layout, storage type, mode, shape), or NULL.
void* pick(int kind, int layout, int dtype, int mode, const SensorShape& sh, bool batch = false) {
#define MCL_PICK(d)                                                                     \
  if (kind == MCL_MAP_DENSE) return sensor_kernel_##d##_dense(mode, sh, batch);         \
  if (kind == kKindDenseTiles) return sensor_kernel_##d##_tiles(mode, sh, batch);       \
  if (kind == kKindBrickGrid) return sensor_kernel_##d##_grid(mode, sh, batch);         \
  if (kind == MCL_MAP_BRICK && layout == MCL_LAYOUT_BLOCK4)                             \
    return sensor_kernel_##d##_block4(mode, sh, batch);                                 \
  if (kind == MCL_MAP_BRICK) return sensor_kernel_##d##_hash(mode, sh, batch);          \
  return nullptr;
  if (dtype == MCL_F32) { MCL_PICK(f32) }
  if (dtype == MCL_F16) { MCL_PICK(f16) }
  if (dtype == MCL_I16) { MCL_PICK(i16) }
#undef MCL_PICK
  return nullptr;
}

// Shared memory / L1 split of the SM's unified array. The kernel needs `smem`
// bytes per CTA; whatever the carveout leaves is L1, which holds the brick
// index and (trilinear read) the corner values. The carveout is sized for the
// resident CTAs, at most kL1Blocks of them, instead of the largest shared
// configuration: 176.9 -> 134.0 ms for the 1M x 65,536 building (nearest, 4
// CTAs; 128.0 ms at 5), 599 -> 559 ms (trilinear), 2.36 -> 2.08 ms for the
// dense hall (which gives up one of its six CTAs for it). The hash-index kernels keep all the CTAs
// their registers allow (6: 4 CTAs and a larger L1 measured 259 against
// 211 ms): their probe loop needs the warps more than the L1. Chosen once
// per (kernel, shape).
#ifndef MCL_L1_BLOCKS
#define MCL_L1_BLOCKS 5
#endif
constexpr int kL1Blocks = MCL_L1_BLOCKS;

int l1_blocks(int kind) { return kind == MCL_MAP_BRICK ? 1 << 30 : kL1Blocks; }

struct CarveKey {
  void* f;
  int smem, threads;
  bool operator<(const CarveKey& o) const {
    return f != o.f ? f < o.f : smem != o.smem ? smem < o.smem : threads < o.threads;
  }
};
std::mutex g_carve_mu;
std::map<CarveKey, int> g_carve;  // kernel -> carveout percent

cudaError_t prepare(void* f, int smem, int threads, int max_blocks) {
  cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  int pct = -1;
  {
    std::lock_guard<std::mutex> lk(g_carve_mu);
    auto it = g_carve.find(CarveKey{f, smem, threads});
    if (it != g_carve.end()) pct = it->second;
  }
  if (pct < 0) {
    e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
    int bps = 0, dev = 0, per_sm = 0, reserved = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, f, threads, smem);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    if (e != cudaSuccess) return e;
    const long long need = (long long)std::min(bps, max_blocks) * (smem + reserved);
    pct = per_sm > 0 && bps > 0 ? (int)std::min<long long>(100, (100 * need + per_sm - 1) / per_sm) : 100;
    std::lock_guard<std::mutex> lk(g_carve_mu);
    g_carve[CarveKey{f, smem, threads}] = pct;
  }
  return cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
}

}  // namespace

// staged scan chunk | mbarrier (16 B) | per-group pose rows (up to 32 groups
// x 6 float4)
int sensor_smem_bytes(const SensorShape& sh) {
  return scan_layout(sh).smem_bytes() + 16 + 32 * 6 * (int)sizeof(float4);
}

cudaError_t sensor_occupancy(int kind, int layout, int dtype, int mode, const SensorShape& sh,
                             int* blocks_per_sm) {
  void* f = pick(kind, layout, dtype, mode, sh);
  if (!f) return cudaErrorInvalidValue;
  const int smem = sensor_smem_bytes(sh);
  cudaError_t e = prepare(f, smem, sh.threads, l1_blocks(kind));
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, f, sh.threads, smem);
}

cudaError_t launch_sensor(int kind, int layout, int dtype, const SensorArgs& a,
                          const SensorShape& sh, cudaStream_t s) {
  void* f = pick(kind, layout, dtype, a.mode, sh);
  if (!f) return cudaErrorInvalidValue;
  const int smem = sensor_smem_bytes(sh);
  cudaError_t e = prepare(f, smem, sh.threads, l1_blocks(kind));
  if (e != cudaSuccess) return e;
  void* args[] = {const_cast<SensorArgs*>(&a)};
  return cudaLaunchKernel(f, dim3(sh.grid), dim3(sh.threads), args, (size_t)smem, s);
}

cudaError_t sensor_batch_occupancy(int kind, int layout, int dtype, int mode, const SensorShape& sh,
                                   int* blocks_per_sm) {
  void* f = pick(kind, layout, dtype, mode, sh, true);
  if (!f) return cudaErrorInvalidValue;
  const int smem = sensor_smem_bytes(sh);
  cudaError_t e = prepare(f, smem, sh.threads, l1_blocks(kind));
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, f, sh.threads, smem);
}

cudaError_t launch_sensor_batch(int kind, int layout, int dtype, const BatchArgs& b,
                                const SensorShape& sh, cudaStream_t s) {
  void* f = pick(kind, layout, dtype, b.base.mode, sh, true);
  if (!f) return cudaErrorInvalidValue;
  const int smem = sensor_smem_bytes(sh);
  cudaError_t e = prepare(f, smem, sh.threads, l1_blocks(kind));
  if (e != cudaSuccess) return e;
  void* args[] = {const_cast<BatchArgs*>(&b)};
  return cudaLaunchKernel(f, dim3(sh.grid), dim3(sh.threads), args, (size_t)smem, s);
}

}  // namespace mcl
