// Host runtime behind the C ABI of include/mcl.h: argument checks, map upload
// (dense grid or 16^3 bricks with an open-addressing hash of brick cells),
// per-(device, stream) workspace, launch planning, per-phase event timing.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include <cuda_fp16.h>
#include <nvtx3/nvToolsExt.h>

#include "runtime.h"

namespace mcl {

namespace {
thread_local std::string g_err;
}  // namespace

mcl_status fail(mcl_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

mcl_status cuda_fail(cudaError_t e, const char* what) {
  cudaGetLastError();  // clear a sticky-free error so the next call starts clean
  if (e == cudaErrorMemoryAllocation) return fail(MCL_ENOMEM, "%s: out of device memory", what);
  return fail(MCL_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

namespace {
std::mutex g_mu;
std::map<int, DeviceState> g_dev;
std::map<std::pair<int, uintptr_t>, std::pair<void*, size_t>> g_ws;
}  // namespace

mcl_status device_state(int* dev_out, DeviceState* out) {
  int dev = 0;
  MCL_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_mu);
  DeviceState& st = g_dev[dev];
  if (!st.status) {
    unsigned* p = nullptr;
    MCL_CUDA(cudaMalloc(&p, sizeof(unsigned)));
    MCL_CUDA(cudaMemset(p, 0, sizeof(unsigned)));
    MCL_CUDA(cudaDeviceGetAttribute(&st.sms, cudaDevAttrMultiProcessorCount, dev));
    st.status = p;
  }
  *out = st;
  if (dev_out) *dev_out = dev;
  return MCL_OK;
}

// Scratch of at least `bytes` for (current device, stream). Grows by freeing
// the old buffer after the stream drained and allocating a larger one.
mcl_status workspace(cudaStream_t s, size_t bytes, void** out) {
  int dev = 0;
  MCL_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_mu);
  auto& slot = g_ws[{dev, (uintptr_t)s}];
  if (slot.second < bytes) {
    if (slot.first) {
      MCL_CUDA(cudaStreamSynchronize(s));
      MCL_CUDA(cudaFree(slot.first));
      slot = {nullptr, 0};
    }
    size_t want = std::max(bytes, (size_t)1 << 20);
    void* p = nullptr;
    MCL_CUDA(cudaMalloc(&p, want));
    slot = {p, want};
  }
  *out = slot.first;
  return MCL_OK;
}

// ---------------------------------------------------------------- profiling
namespace {
struct PhaseEvents {
  int phase, kernels;
  cudaEvent_t a, b;
};
bool g_prof_on = false;
std::vector<PhaseEvents> g_prof;
std::vector<cudaEvent_t> g_event_pool;
}  // namespace

static cudaEvent_t take_event() {
  if (!g_event_pool.empty()) {
    cudaEvent_t e = g_event_pool.back();
    g_event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

thread_local bool t_no_profile = false;

NoProfileScope::NoProfileScope() : prev_(t_no_profile) { t_no_profile = true; }
NoProfileScope::~NoProfileScope() { t_no_profile = prev_; }

// NVTX range names of the phases (seen by nsys / ncu range filters; the
// calls cost nothing when no tool is attached).
const char* const kPhaseRange[] = {"mcl.pose",      "mcl.pack",     "mcl.sensor", "mcl.reduce",
                                   "mcl.normalise", "mcl.resample", "mcl.motion", "mcl.other"};

PhaseScope::PhaseScope(int ph, cudaStream_t st, int nk) : phase_(ph), kernels_(nk), s_(st) {
  nvtxRangePushA(kPhaseRange[ph >= 0 && ph < MCL_NUM_PHASES ? ph : MCL_PHASE_OTHER]);
  if (t_no_profile) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_prof_on) return;
  a_ = take_event();
  b_ = take_event();
  cudaEventRecord(a_, s_);
}

PhaseScope::~PhaseScope() {
  nvtxRangePop();
  if (!a_) return;
  cudaEventRecord(b_, s_);
  std::lock_guard<std::mutex> lk(g_mu);
  g_prof.push_back({phase_, kernels_, a_, b_});
}

}  // namespace mcl

using namespace mcl;

extern "C" {

const char* mcl_last_error(void) { return g_err.c_str(); }

int32_t mcl_version(void) { return 200; }

mcl_status mcl_sync(mcl_stream_t stream) {
  cudaStream_t s = (cudaStream_t)stream;
  MCL_CUDA(cudaStreamSynchronize(s));
  DeviceState st;
  mcl_status rc = device_state(nullptr, &st);
  if (rc) return rc;
  unsigned v = 0;
  MCL_CUDA(cudaMemcpy(&v, st.status, sizeof v, cudaMemcpyDeviceToHost));
  if (v) {
    MCL_CUDA(cudaMemset(st.status, 0, sizeof v));
    return fail(MCL_EINTERNAL, "device status word 0x%x (%s%s)", v,
                (v & kDevErrTimeout) ? "bounded wait ran out " : "",
                (v & kDevErrIndex) ? "index check failed" : "");
  }
  return MCL_OK;
}

mcl_status mcl_selftest_wait(double* waited_s, mcl_stream_t stream) {
  cudaStream_t s = (cudaStream_t)stream;
  MCL_CUDA(cudaStreamSynchronize(s));
  DeviceState st;
  if (mcl_status rc = device_state(nullptr, &st)) return rc;
  unsigned v = 0;
  MCL_CUDA(cudaMemcpy(&v, st.status, sizeof v, cudaMemcpyDeviceToHost));
  if (v) return fail(MCL_EINTERNAL, "selftest_wait: status word already 0x%x", v);
  unsigned long long* d_ns = nullptr;
  MCL_CUDA(cudaMalloc(&d_ns, sizeof(unsigned long long)));
  unsigned long long ns = 0;
  cudaError_t e = launch_wait_selftest(st.status, d_ns, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaMemcpy(&ns, d_ns, sizeof ns, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&v, st.status, sizeof v, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(st.status, 0, sizeof v);
  cudaFree(d_ns);
  MCL_CUDA(e);
  if (waited_s) *waited_s = (double)ns * 1e-9;
  if (!(v & kDevErrTimeout)) return fail(MCL_EINTERNAL, "selftest_wait: the timeout was not recorded");
  return MCL_OK;
}

// ---------------------------------------------------------------- maps
mcl_status mcl_map_create(const mcl_map_desc* d, const void* host_values, mcl_map_t* out) {
  if (!d || !out) return fail(MCL_EINVAL, "map_create: NULL desc or out");
  *out = nullptr;
  if (d->struct_size < sizeof(mcl_map_desc))
    return fail(MCL_EINVAL, "map_create: struct_size %u < %zu", d->struct_size, sizeof(mcl_map_desc));
  if (d->kind != MCL_MAP_DENSE && d->kind != MCL_MAP_BRICK)
    return fail(MCL_EINVAL, "map_create: kind %d", d->kind);
  if (d->dtype < MCL_F32 || d->dtype > MCL_I16) return fail(MCL_EINVAL, "map_create: dtype %d", d->dtype);
  if (!finite_pos(d->voxel) || !finite_pos(d->truncation))
    return fail(MCL_EINVAL, "map_create: voxel and truncation must be finite and > 0");
  for (int k = 0; k < 3; ++k) {
    if (!std::isfinite(d->origin[k])) return fail(MCL_EINVAL, "map_create: origin not finite");
    if (d->dims[k] <= 0 || d->dims[k] > (1 << 23))
      return fail(MCL_EINVAL, "map_create: dims[%d] = %lld outside [1, 2^23]", k, (long long)d->dims[k]);
  }
  if (d->kind == MCL_MAP_BRICK && d->device_layout != MCL_LAYOUT_LINEAR &&
      d->device_layout != MCL_LAYOUT_BLOCK4)
    return fail(MCL_EINVAL, "map_create: device_layout %d", d->device_layout);
  if (d->kind == MCL_MAP_DENSE && d->device_layout != MCL_LAYOUT_LINEAR)
    return fail(MCL_EINVAL, "map_create: dense maps are stored linearly");
  if (d->index < MCL_INDEX_AUTO || d->index > MCL_INDEX_GRID)
    return fail(MCL_EINVAL, "map_create: index %d", d->index);
  if (d->kind == MCL_MAP_BRICK && d->index == MCL_INDEX_GRID && d->device_layout != MCL_LAYOUT_LINEAR)
    return fail(MCL_EINVAL, "map_create: the grid index is built for the linear layout only");
  if (d->kind == MCL_MAP_BRICK && d->index == MCL_INDEX_GRID && d->n_bricks > kGridMaxBricks)
    return fail(MCL_EINVAL, "map_create: the grid index addresses at most 2^20 bricks (%lld given)",
                (long long)d->n_bricks);
  float inv = d->inv_voxel == 0.f ? (float)(1.0 / (double)d->voxel) : d->inv_voxel;
  if (!finite_pos(inv)) return fail(MCL_EINVAL, "map_create: inv_voxel must be finite and > 0");
  const size_t es = d->dtype == MCL_F32 ? 4 : 2;

  int dev = 0;
  MCL_CUDA(cudaGetDevice(&dev));
  mcl_map_s* m = new mcl_map_s();
  m->device = dev;
  m->kind = d->kind;
  m->dtype = d->dtype;
  MapView& v = m->view;
  v.ox = d->origin[0];
  v.oy = d->origin[1];
  v.oz = d->origin[2];
  v.inv = inv;
  v.nx = (int)d->dims[0];
  v.ny = (int)d->dims[1];
  v.nz = (int)d->dims[2];
  v.fnx = (float)v.nx;
  v.fny = (float)v.ny;
  v.fnz = (float)v.nz;
  v.tau = d->truncation;
  v.scale = (float)((double)d->truncation / 32767.0);
  v.layout = d->kind == MCL_MAP_BRICK ? d->device_layout : MCL_LAYOUT_LINEAR;

  auto cleanup = [&](mcl_status s) {
    if (m->d_values) cudaFree(m->d_values);
    if (m->d_table) cudaFree(m->d_table);
    if (m->d_grid) cudaFree(m->d_grid);
    delete m;
    return s;
  };

  if (d->kind == MCL_MAP_DENSE) {
    const int64_t nx = d->dims[0], ny = d->dims[1], nz = d->dims[2];
    // grids in 8 x 4 tiles: the VLP-16 hall step 1.835 -> 1.706 ms (FP32),
    // 1.861 -> 1.806 ms (FP16)
    m->dense_tiles = MCL_DENSE_TILES != 0;
    if (nx * ny * nz > kMaxCount) return cleanup(fail(MCL_EINVAL, "map_create: dense grid above 2^31 - 1 voxels"));
    const int64_t stored = dense_stored(nx, ny, nz, m->dense_tiles);  // with the tiles' padding
    if (stored > kMaxCount)
      return cleanup(fail(MCL_EINVAL, "map_create: dense grid above 2^31 - 1 values after padding to 8 x 4 tiles"));
    if (!host_values) return cleanup(fail(MCL_EINVAL, "map_create: NULL values"));
    v.ntx = (uint32_t)((nx + 7) / 8);
    v.nty = (uint32_t)((ny + 3) / 4);
    v.tcy = 8u * v.ntx - 8u;
    v.tsz = 32u * v.ntx * v.nty;
    cudaError_t e = cudaMalloc(&m->d_values, (size_t)stored * es);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "map_create values"));
    if (!m->dense_tiles) {
      e = cudaMemcpy(m->d_values, host_values, (size_t)stored * es, cudaMemcpyHostToDevice);
      if (e != cudaSuccess) return cleanup(cuda_fail(e, "map_create upload"));
    } else {
      e = cudaMemset(m->d_values, 0, (size_t)stored * es);
      // upload through a staging buffer of whole z layers (about 64 MB) and move
      // each voxel to its place in the tiles on the device
      const int64_t layer = nx * ny;
      const int64_t per = std::max<int64_t>(1, std::min<int64_t>(nz, (64ll << 20) / std::max<int64_t>(1, layer * (int64_t)es)));
      void* stage = nullptr;
      if (e == cudaSuccess) e = cudaMalloc(&stage, (size_t)(per * layer) * es);
      for (int64_t z0 = 0; z0 < nz && e == cudaSuccess; z0 += per) {
        const int64_t cnt = std::min(per, nz - z0);
        e = cudaMemcpy(stage, (const char*)host_values + (size_t)(z0 * layer) * es, (size_t)(cnt * layer) * es,
                       cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
          e = launch_dense_to_tiles(stage, m->d_values, (int)nx, (int)ny, (int)z0, (int)cnt, v.ntx, v.nty,
                                    (int)es, nullptr);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
      }
      if (stage) cudaFree(stage);
      if (e != cudaSuccess) return cleanup(cuda_fail(e, "map_create upload"));
    }
    m->bytes = stored * (int64_t)es;
  } else {
    for (int k = 0; k < 3; ++k)
      if (d->dims[k] % kBrick) return cleanup(fail(MCL_EINVAL, "map_create: dims must be multiples of 16"));
    const uint64_t nbx = (uint64_t)d->dims[0] / kBrick, nby = (uint64_t)d->dims[1] / kBrick,
                   nbz = (uint64_t)d->dims[2] / kBrick;
    if (nbx * nby * nbz > 0xFFFFFFFEull) return cleanup(fail(MCL_EINVAL, "map_create: too many brick cells"));
    const int64_t nb = d->n_bricks;
    if (nb < 0 || nb > (1LL << 29)) return cleanup(fail(MCL_EINVAL, "map_create: n_bricks %lld", (long long)nb));
    if (nb > 0 && (!host_values || !d->brick_coords))
      return cleanup(fail(MCL_EINVAL, "map_create: NULL brick values or coordinates"));
    int bits = 1;
    while ((1LL << bits) < std::max<int64_t>(2, 4 * nb)) ++bits;
    const int64_t cap = 1LL << bits;
    std::vector<uint2> table((size_t)cap, make_uint2(kEmptyKey, 0u));
    const int shift = 32 - bits;
    int max_probe = 1;
    for (int64_t b = 0; b < nb; ++b) {
      const int32_t* c = d->brick_coords + 3 * b;
      if (c[0] < 0 || c[1] < 0 || c[2] < 0 || (uint64_t)c[0] >= nbx || (uint64_t)c[1] >= nby ||
          (uint64_t)c[2] >= nbz)
        return cleanup(fail(MCL_EINVAL, "map_create: brick %lld coordinates out of range", (long long)b));
      const uint32_t key = (uint32_t)(((uint64_t)c[2] * nby + (uint64_t)c[1]) * nbx + (uint64_t)c[0]);
      uint32_t h = brick_hash(key, shift);
      int probe = 1;
      while (table[h].x != kEmptyKey) {
        if (table[h].x == key)
          return cleanup(fail(MCL_EINVAL, "map_create: brick %lld duplicated", (long long)b));
        h = (h + 1) & (uint32_t)(cap - 1);
        ++probe;
      }
      table[h] = make_uint2(key, (uint32_t)b);
      max_probe = std::max(max_probe, probe);
    }
    // The cell grid with a guard layer: one more cell along each axis (cell
    // nb) and gsz + gsy + 1 cells in front, all empty. Every cell coordinate
    // in [-1, nb] then has its own cell (a guard one outside the map), so a
    // voxel index clamped to n, or a trilinear corner at -1 or n, reads "no
    // brick" without an inside test.
    const uint64_t gsy = nbx + 1, gsz = (nbx + 1) * (nby + 1), front = gsz + gsy + 1;
    const uint64_t cells = front + gsz * (nbz + 1);
    if (d->index == MCL_INDEX_GRID && cells > 0x7FFFFFFFull)
      return cleanup(fail(MCL_EINVAL, "map_create: %llu grid cells exceed signed 32-bit keys; use the hash index",
                          (unsigned long long)cells));
    const bool grid = d->index == MCL_INDEX_GRID ||
                      (d->index == MCL_INDEX_AUTO && v.layout == MCL_LAYOUT_LINEAR &&
                       cells * sizeof(uint32_t) <= (512ull << 20) && nb <= kGridMaxBricks);
    const size_t vbytes = (size_t)nb * kBrickVoxels * es;
    cudaError_t e = cudaMalloc(&m->d_values, std::max(vbytes, (size_t)256));
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "map_create values"));
    if (vbytes && v.layout == MCL_LAYOUT_LINEAR && !grid) {
      e = cudaMemcpy(m->d_values, host_values, vbytes, cudaMemcpyHostToDevice);
      if (e != cudaSuccess) return cleanup(cuda_fail(e, "map_create upload"));
    } else if (vbytes) {
      // upload through a staging buffer and reorder each brick on the device:
      // 4x4x4 blocks, or (cell grid) rotated by the brick's cell coordinates
      const int64_t per = std::min<int64_t>(nb, 1 << 16);
      const size_t brick_bytes = (size_t)kBrickVoxels * es;
      void* stage = nullptr;
      int32_t* dcoords = nullptr;
      e = cudaMalloc(&stage, (size_t)per * brick_bytes);
      if (e == cudaSuccess && grid) e = cudaMalloc((void**)&dcoords, (size_t)per * 3 * sizeof(int32_t));
      for (int64_t b0 = 0; b0 < nb && e == cudaSuccess; b0 += per) {
        const int64_t cnt = std::min(per, nb - b0);
        e = cudaMemcpy(stage, (const char*)host_values + (size_t)b0 * brick_bytes,
                       (size_t)cnt * brick_bytes, cudaMemcpyHostToDevice);
        char* dst = (char*)m->d_values + (size_t)b0 * brick_bytes;
        if (e == cudaSuccess && grid)
          e = cudaMemcpy(dcoords, d->brick_coords + 3 * b0, (size_t)cnt * 3 * sizeof(int32_t),
                         cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
          e = grid ? launch_brick_to_skew(stage, dst, dcoords, cnt, (int)es, nullptr)
                   : launch_brick_to_block4(stage, dst, cnt, (int)es, nullptr);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
      }
      if (stage) cudaFree(stage);
      if (dcoords) cudaFree(dcoords);
      if (e != cudaSuccess) return cleanup(cuda_fail(e, grid ? "map_create skewed layout" : "map_create block layout"));
    }
    v.nbx = (uint32_t)nbx;
    v.nby = (uint32_t)nby;
    v.gsy = (uint32_t)gsy;
    v.gsz = (uint32_t)gsz;
    v.n_slots = (uint32_t)nb;
    m->n_bricks = nb;
    if (grid) {
      // coarse level as a dense array: brick cell -> slot * 4096, the index of
      // the brick's first value (the duplicates and ranges were checked while
      // the hash was filled above; at most 2^20 bricks, so it fits)
      std::vector<uint32_t> cell_slot((size_t)cells, kNoSlot);
      for (int64_t b = 0; b < nb; ++b) {
        const int32_t* c = d->brick_coords + 3 * b;
        cell_slot[front + (uint64_t)c[2] * gsz + (uint64_t)c[1] * gsy + (uint64_t)c[0]] =
            (uint32_t)b * (uint32_t)kBrickVoxels;
      }
      e = cudaMalloc((void**)&m->d_grid, (size_t)cells * sizeof(uint32_t));
      if (e != cudaSuccess) return cleanup(cuda_fail(e, "map_create grid index"));
      e = cudaMemcpy(m->d_grid, cell_slot.data(), (size_t)cells * sizeof(uint32_t), cudaMemcpyHostToDevice);
      if (e != cudaSuccess) return cleanup(cuda_fail(e, "map_create grid upload"));
      v.grid = m->d_grid + front;
      m->grid_cells = (int64_t)cells;
      m->grid_front = (int64_t)front;
      m->bytes = (int64_t)vbytes + (int64_t)cells * (int64_t)sizeof(uint32_t);
    } else {
      e = cudaMalloc(&m->d_table, (size_t)cap * sizeof(uint2));
      if (e != cudaSuccess) return cleanup(cuda_fail(e, "map_create table"));
      e = cudaMemcpy(m->d_table, table.data(), (size_t)cap * sizeof(uint2), cudaMemcpyHostToDevice);
      if (e != cudaSuccess) return cleanup(cuda_fail(e, "map_create table upload"));
      v.table = m->d_table;
      v.hash_mask = (uint32_t)(cap - 1);
      v.hash_shift = shift;
      v.max_probe = max_probe;
      m->capacity = cap;
      m->max_probe = max_probe;
      m->bytes = (int64_t)vbytes + cap * (int64_t)sizeof(uint2);
    }
  }
  v.values = m->d_values;
  *out = m;
  return MCL_OK;
}

mcl_status mcl_map_create_score(mcl_map_t src, float sigma, int32_t dtype, mcl_map_t* out) {
  if (!src || !out) return fail(MCL_EINVAL, "map_create_score: NULL source or out");
  *out = nullptr;
  if (!finite_pos(sigma)) return fail(MCL_EINVAL, "map_create_score: sigma must be finite and > 0");
  if (dtype != MCL_F16 && dtype != MCL_F32) return fail(MCL_EINVAL, "map_create_score: dtype %d", dtype);
  if (src->score_sigma > 0.f) return fail(MCL_EINVAL, "map_create_score: the source is a score map");
  if (mcl_status rc = check_device(src)) return rc;
  const int64_t n = src->kind == MCL_MAP_DENSE
                        ? dense_stored(src->view.nx, src->view.ny, src->view.nz, src->dense_tiles)
                        : src->n_bricks * (int64_t)kBrickVoxels;
  const size_t es = dtype == MCL_F32 ? 4 : 2;
  mcl_map_s* m = new mcl_map_s(*src);
  m->dtype = dtype;
  m->d_values = nullptr;
  m->d_table = nullptr;
  m->d_grid = nullptr;
  auto cleanup = [&](mcl_status st) {
    if (m->d_values) cudaFree(m->d_values);
    if (m->d_table) cudaFree(m->d_table);
    if (m->d_grid) cudaFree(m->d_grid);
    delete m;
    return st;
  };
  cudaError_t e = cudaMalloc(&m->d_values, std::max((size_t)n * es, (size_t)256));
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "map_create_score values"));
  const double tau = (double)src->view.tau;
  e = launch_score_values(src->d_values, src->dtype, n, tau, (double)sigma, m->d_values, dtype, nullptr);
  if (e == cudaSuccess && src->d_table) {
    e = cudaMalloc((void**)&m->d_table, (size_t)src->capacity * sizeof(uint2));
    if (e == cudaSuccess)
      e = cudaMemcpy(m->d_table, src->d_table, (size_t)src->capacity * sizeof(uint2),
                     cudaMemcpyDeviceToDevice);
  }
  if (e == cudaSuccess && src->d_grid) {
    e = cudaMalloc((void**)&m->d_grid, (size_t)src->grid_cells * sizeof(uint32_t));
    if (e == cudaSuccess)
      e = cudaMemcpy(m->d_grid, src->d_grid, (size_t)src->grid_cells * sizeof(uint32_t),
                     cudaMemcpyDeviceToDevice);
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "map_create_score"));
  // The score of +tau, computed the same way (FP64, one rounding).
  const double eo = std::exp(-(tau * tau) / (2.0 * (double)sigma * (double)sigma));
  m->score_outside = dtype == MCL_F16 ? __half2float(__double2half(eo)) : (float)eo;
  m->score_sigma = sigma;
  m->view.values = m->d_values;
  m->view.table = m->d_table;
  m->view.grid = m->d_grid ? m->d_grid + m->grid_front : nullptr;
  m->view.tau = m->score_outside;  // what a look-up reads where nothing is stored
  m->bytes = (int64_t)n * (int64_t)es + (m->d_table ? m->capacity * (int64_t)sizeof(uint2) : 0) +
             (m->d_grid ? m->grid_cells * (int64_t)sizeof(uint32_t) : 0);
  *out = m;
  return MCL_OK;
}

mcl_status mcl_map_destroy(mcl_map_t m) {
  if (!m) return MCL_OK;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(m->device);
  cudaDeviceSynchronize();
  if (m->d_values) cudaFree(m->d_values);
  if (m->d_table) cudaFree(m->d_table);
  if (m->d_grid) cudaFree(m->d_grid);
  cudaSetDevice(cur);
  delete m;
  return MCL_OK;
}

mcl_status mcl_map_get_info(mcl_map_t m, mcl_map_info* out) {
  if (!m || !out) return fail(MCL_EINVAL, "map_get_info: NULL argument");
  if (out->struct_size < sizeof(mcl_map_info)) return fail(MCL_EINVAL, "map_get_info: struct_size");
  out->device_bytes = m->bytes;
  out->n_bricks = m->n_bricks;
  out->hash_capacity = m->capacity;
  out->hash_max_probe = m->max_probe;
  out->device = m->device;
  out->score_sigma = m->score_sigma;
  out->score_outside = m->score_outside;
  out->index = m->kind == MCL_MAP_BRICK ? (m->d_grid ? MCL_INDEX_GRID : MCL_INDEX_HASH) : 0;
  out->reserved = 0;
  out->index_bytes = m->d_grid ? m->grid_cells * (int64_t)sizeof(uint32_t)
                               : m->capacity * (int64_t)sizeof(uint2);
  return MCL_OK;
}

}  // extern "C"

namespace mcl {

mcl_status check_device(mcl_map_t m) {
  int dev = 0;
  MCL_CUDA(cudaGetDevice(&dev));
  if (dev != m->device) return fail(MCL_EINVAL, "map lives on device %d, current device is %d", m->device, dev);
  return MCL_OK;
}

}  // namespace mcl

extern "C" {

mcl_status mcl_map_lookup(mcl_map_t m, const float* pts, int64_t N, int64_t* out_index,
                          float* out_value, mcl_stream_t stream) {
  if (!m || !pts) return fail(MCL_EINVAL, "map_lookup: NULL map or points");
  if (N < 1 || N > kMaxCount) return fail(MCL_EINVAL, "map_lookup: N = %lld", (long long)N);
  if (!aligned(pts, 4) || !aligned(out_index, 8) || !aligned(out_value, 4))
    return fail(MCL_EINVAL, "map_lookup: misaligned pointer");
  if (mcl_status rc = check_device(m)) return rc;
  PhaseScope ps(MCL_PHASE_OTHER, (cudaStream_t)stream);
  MCL_CUDA(launch_map_lookup(kernel_kind(m), m->dtype, m->view, pts, (int)N, (long long*)out_index,
                             out_value, (cudaStream_t)stream));
  return MCL_OK;
}

// ---------------------------------------------------------------- sensor update
}  // extern "C"

namespace mcl {

mcl_status check_params(const mcl_sensor_params* p) {
  if (!p) return fail(MCL_EINVAL, "sensor params: NULL");
  if (p->struct_size < sizeof(mcl_sensor_params)) return fail(MCL_EINVAL, "sensor params: struct_size");
  if (!finite_pos(p->sigma_hit)) return fail(MCL_EINVAL, "sensor params: sigma_hit must be finite and > 0");
  if (p->mode != MCL_LOGPROD && p->mode != MCL_SUM) return fail(MCL_EINVAL, "sensor params: mode %d", p->mode);
  if (p->flags & ~(MCL_NEGLECT_OUTSIDE | MCL_TRILINEAR))
    return fail(MCL_EINVAL, "sensor params: unknown flags 0x%x", p->flags);
  if ((p->flags & MCL_TRILINEAR) && p->lanes_per_particle != 0 && p->lanes_per_particle != 32)
    return fail(MCL_EINVAL, "sensor params: the trilinear read needs 32 lanes per particle");
  const int c = p->points_per_chunk;
  if (c != 0 && (c < 32 || c > 8192 || c % 32))
    return fail(MCL_EINVAL, "sensor params: points_per_chunk %d", c);
  const int g = p->lanes_per_particle;
  if (g != 0 && g != 8 && g != 16 && g != 32) return fail(MCL_EINVAL, "sensor params: lanes_per_particle %d", g);
  if (p->particles_per_item < 0 || p->particles_per_item > 4096)
    return fail(MCL_EINVAL, "sensor params: particles_per_item %d", p->particles_per_item);
  if (p->unroll != 0 && p->unroll != 2 && p->unroll != 4 && p->unroll != 8)
    return fail(MCL_EINVAL, "sensor params: unroll %d", p->unroll);
  if (p->pipeline < 0 || p->pipeline > 2) return fail(MCL_EINVAL, "sensor params: pipeline %d", p->pipeline);
  if (p->particle_order < 0 || p->particle_order > 2)
    return fail(MCL_EINVAL, "sensor params: particle_order %d", p->particle_order);
  if (p->item_order < 0 || p->item_order > 3)
    return fail(MCL_EINVAL, "sensor params: item_order %d", p->item_order);
  if (p->scan_rings < 0) return fail(MCL_EINVAL, "sensor params: scan_rings %d", p->scan_rings);
  return MCL_OK;
}

mcl_status check_map_params(mcl_map_t m, const mcl_sensor_params* p) {
  if (m->score_sigma > 0.f) {
    if (p->mode != MCL_SUM) return fail(MCL_EINVAL, "score map: mode must be MCL_SUM");
    if (p->sigma_hit != m->score_sigma)
      return fail(MCL_EINVAL, "score map: sigma_hit %g differs from the map's %g", p->sigma_hit, m->score_sigma);
    if (p->flags & MCL_TRILINEAR) return fail(MCL_EINVAL, "score map: no trilinear read");
    if (p->pipeline == 2) return fail(MCL_EINVAL, "score map: no pipelined loop");
  }
  return MCL_OK;
}

// Particles are evaluated in spatial order unless told otherwise (or too few
// to matter).
constexpr int64_t kSpatialOrderMinParticles = 4096;

mcl_status make_plan(mcl_map_t m, int64_t P, int64_t N, const mcl_sensor_params* p, Plan* pl) {
  *pl = Plan{};  // every field below is set from (m, P, N, p) or stays zero
  DeviceState st;
  if (mcl_status rc = device_state(nullptr, &st)) return rc;
  SensorShape& sh = pl->sh;
  // Brick maps: map larger than L2, where the sweep item order pays
  // (measured on GB300: 1M x 65,536 int16 bricks 184.2 -> 177.4 ms static,
  // 130.3 -> 113.8 ms handed out dynamically; the trilinear read 545.0 ->
  // 460.8 ms dynamically, 584.4 ms static; slower for the L2-resident dense
  // hall).
  const bool brick_nearest = m->kind == MCL_MAP_BRICK && !(p->flags & MCL_TRILINEAR);
  sh.chunk = p->points_per_chunk ? p->points_per_chunk : 2048;
  sh.lanes = p->lanes_per_particle ? p->lanes_per_particle : 32;
  // particles per item: 64 for the hash index (4-deep loop), else 128 (the
  // 8-deep cell-grid kernel: 96.4 against 97.0 ms with 64)
  sh.ppi = p->particles_per_item ? p->particles_per_item
                                 : (brick_nearest && m->d_grid == nullptr ? 64 : 128);
  // Eight look-ups in flight per lane (64 registers, 4 CTAs per SM) for the
  // nearest read of the cell-grid brick map and of dense maps: the packed
  // pair stage re-reads the pose rows half as often as with four (1M x
  // 65,536 int16 building: 97.0 against 102.6 ms at 5 CTAs; 50,000 x 28,800
  // dense FP32 hall: 1.74 against 1.97 ms); four for the hash index.
  const bool nearest = !(p->flags & MCL_TRILINEAR);
  const bool deep = nearest && (m->kind == MCL_MAP_DENSE || m->d_grid != nullptr);
  sh.unroll = p->unroll ? p->unroll : (deep ? 8 : 4);
  sh.pipeline = p->pipeline == 2 ? 1 : 0;
  // unroll and pipeline are hints: lane groups narrower than a warp run the
  // plain 4-deep loop, and the pipelined loop exists for 2 or 4 look-ups.
  if (sh.lanes < 32) {
    sh.unroll = 4;
    sh.pipeline = 0;
  } else if (sh.unroll == 8) {
    sh.pipeline = 0;
  }
  if (mcl_status rc = check_map_params(m, p)) return rc;
  if (m->score_sigma > 0.f) sh.pipeline = 0;
  sh.interp = (p->flags & MCL_TRILINEAR) ? 1 : 0;
  if (sh.interp) {  // two points per lane per step, no pipelining
    sh.unroll = 2;
    sh.pipeline = 0;
  }
  sh.threads = 256;
  // scan staged in 4-ring x 8-point patches when the caller gives its ring
  // structure and it fits (85.6 -> 83.9 ms for the OS0-64 building)
  if (p->scan_rings > 0 && N % p->scan_rings == 0 && p->scan_rings % 4 == 0 && (N / p->scan_rings) % 8 == 0) {
    sh.rings = p->scan_rings;
    sh.az = (int)(N / p->scan_rings);
  }
  int bps = 0;
  MCL_CUDA(sensor_occupancy(kernel_kind(m), m->view.layout, m->dtype, kernel_mode(m, p->mode), sh, &bps));
  if (bps < 1) return fail(MCL_EINVAL, "sensor plan: launch shape does not fit on an SM");
  pl->spatial = p->particle_order == 2 || (p->particle_order == 0 && P >= kSpatialOrderMinParticles);
  pl->K = (int)((N + sh.chunk - 1) / sh.chunk);
  const long long slots = (long long)st.sms * bps;
  if (!p->particles_per_item) {
    // Small sets: shrink the particle block (not below one particle per lane
    // group of the CTA) until every resident CTA has an item; the block size
    // changes no result.
    const int groups = (sh.threads / 32) * (32 / sh.lanes);
    const long long per = ((long long)P * pl->K + slots - 1) / slots;
    while (sh.ppi > groups && sh.ppi / 2 >= per) sh.ppi /= 2;
  }
  pl->nblk = (int)((P + sh.ppi - 1) / sh.ppi);
  pl->n_items = (long long)pl->K * pl->nblk;
  pl->blocks_per_sm = bps;
  pl->sms = st.sms;
  sh.grid = (int)std::min<long long>(pl->n_items, slots);
  // Item order. Sweeps: slots / K particle blocks at a time through all K
  // chunks, on a grid of sweep * K CTAs, so that every CTA keeps its chunk
  // (no re-staging) and the CTAs resident together work on few particles,
  // whose map neighbourhoods (in spatial order) overlap in L2. Needs at
  // least one CTA per chunk; auto takes it for nearest reads of brick maps
  // from two items per slot on.
  pl->sweep = pl->nblk;
  pl->dynamic = false;
  const bool auto_sweeps = p->item_order == 0 && m->kind == MCL_MAP_BRICK && pl->n_items >= 2 * slots;
  const bool sweeps = p->item_order == 2;
  if ((p->item_order == 3 || auto_sweeps) && pl->K > 1 && slots >= pl->K) {
    // Dynamic sweeps: the same numbering, items handed out in order by a
    // device counter to whichever CTA is free, so the items in flight stay
    // within about one sweep whatever the cost of each chunk (with static
    // striding the CTAs of cheap chunks run ahead of the others, the CTAs in
    // flight spread over many sweeps and the map reads of different
    // particles no longer meet in L2: 9.75 against 6.06 DRAM bytes per
    // evaluation at 200,000 x 65,536).
    pl->sweep = (int)std::min<long long>(pl->nblk, std::max<long long>(1, slots / pl->K));
    pl->dynamic = true;
  } else if (sweeps && pl->K > 1 && slots >= pl->K) {
    pl->sweep = (int)std::min<long long>(pl->nblk, slots / pl->K);
    sh.grid = (int)std::min<long long>(pl->n_items, (long long)pl->sweep * pl->K);
  }
  size_t o = 0;
  pl->off_mats = o;
  o = align256(o + (size_t)P * 3 * sizeof(float4));
  pl->off_scan = o;
  o = align256(o + scan_layout(sh).total_bytes((int)N));
  pl->off_partial = o;
  o = align256(o + (size_t)pl->K * (size_t)P * sizeof(float));
  pl->off_logw = o;
  o = align256(o + (size_t)P * sizeof(float));
  pl->off_stats = o;
  o = align256(o + (size_t)normalise_blocks((int)P) * sizeof(float2));
  pl->off_ostats = o;
  o = align256(o + 2 * sizeof(float));
  pl->off_est = o;
  o = align256(o + (size_t)normalise_blocks((int)P) * sizeof(EstPartial));
  pl->off_key = o;
  o = align256(o + (pl->spatial ? (size_t)P * sizeof(uint32_t) : 0));
  pl->off_rank = o;
  o = align256(o + (pl->spatial ? (size_t)P * sizeof(int) : 0));
  pl->off_hist = o;
  o = align256(o + (pl->spatial ? order_hist_bytes() : 0));
  pl->off_queue = o;
  o = align256(o + sizeof(unsigned long long));
  pl->total = o;
  return MCL_OK;
}

}  // namespace mcl

extern "C" {

mcl_status mcl_sensor_plan_get(mcl_map_t m, int64_t P, int64_t N, const mcl_sensor_params* p,
                               mcl_sensor_plan* out) {
  if (!m || !out) return fail(MCL_EINVAL, "sensor_plan: NULL argument");
  if (out->struct_size < sizeof(mcl_sensor_plan)) return fail(MCL_EINVAL, "sensor_plan: struct_size");
  if (P < 1 || P > kMaxCount || N < 1 || N > kMaxCount) return fail(MCL_EINVAL, "sensor_plan: sizes");
  if (mcl_status rc = check_params(p)) return rc;
  if (mcl_status rc = check_device(m)) return rc;
  Plan pl;
  if (mcl_status rc = make_plan(m, P, N, p, &pl)) return rc;
  out->points_per_chunk = pl.sh.chunk;
  out->lanes_per_particle = pl.sh.lanes;
  out->particles_per_item = pl.sh.ppi;
  out->unroll = pl.sh.unroll;
  out->pipeline = pl.sh.pipeline ? 2 : 1;
  out->particle_order = pl.spatial ? 2 : 1;
  out->threads = pl.sh.threads;
  out->grid = pl.sh.grid;
  out->blocks_per_sm = pl.blocks_per_sm;
  out->num_sms = pl.sms;
  out->n_items = pl.n_items;
  out->workspace_bytes = (int64_t)pl.total;
  out->item_order = pl.dynamic ? 3 : pl.sweep < pl.nblk ? 2 : 1;
  out->blocks_per_sweep = pl.sweep;
  return MCL_OK;
}

}  // extern "C"

namespace mcl {
namespace {

mcl_status sensor_update(mcl_map_t m, const float* particles, int64_t P, const float* scan,
                         int64_t N, const mcl_sensor_params* p, float* logw, float* w,
                         mcl_estimate* est, cudaStream_t s) {
  if (!m || !particles || !scan) return fail(MCL_EINVAL, "sensor_update: NULL map, particles or scan");
  if (P < 1 || P > kMaxCount) return fail(MCL_EINVAL, "sensor_update: P = %lld", (long long)P);
  if (N < 1 || N > kMaxCount) return fail(MCL_EINVAL, "sensor_update: N = %lld", (long long)N);
  if (!logw && !w) return fail(MCL_EINVAL, "sensor_update: both outputs NULL");
  if (!aligned(particles, 4) || !aligned(scan, 4) || !aligned(logw, 4) || !aligned(w, 4))
    return fail(MCL_EINVAL, "sensor_update: pointers need 4-byte alignment");
  if (mcl_status rc = check_params(p)) return rc;
  if (mcl_status rc = check_device(m)) return rc;
  DeviceState st;
  if (mcl_status rc = device_state(nullptr, &st)) return rc;
  Plan pl;
  if (mcl_status rc = make_plan(m, P, N, p, &pl)) return rc;
  char* ws = nullptr;
  if (mcl_status rc = workspace(s, pl.total, (void**)&ws)) return rc;
  return enqueue_sensor(m, particles, P, scan, N, p, logw, w, est, pl, ws, st.status, s);
}

}  // namespace

mcl_status enqueue_sensor(mcl_map_t m, const float* particles, int64_t P, const float* scan,
                          int64_t N, const mcl_sensor_params* p, float* logw, float* w,
                          mcl_estimate* est, const Plan& pl, char* ws, unsigned* status,
                          cudaStream_t s) {
  float4* mats = (float4*)(ws + pl.off_mats);
  void* packed = ws + pl.off_scan;
  float* partial = (float*)(ws + pl.off_partial);
  float* L = logw ? logw : (float*)(ws + pl.off_logw);
  float2* bstats = (float2*)(ws + pl.off_stats);
  float* ostats = (float*)(ws + pl.off_ostats);
  int* rank = pl.spatial ? (int*)(ws + pl.off_rank) : nullptr;
  {
    // the pose phase also packs the scan (one launch for both)
    PhaseScope ps(MCL_PHASE_POSE, s, pl.spatial ? 5 : 1);
    if (pl.spatial)
      MCL_CUDA(launch_particle_order(particles, (int)P, m->view, (uint32_t*)(ws + pl.off_key),
                                     (uint32_t*)(ws + pl.off_hist), rank, s));
    MCL_CUDA(launch_pose_and_pack(particles, (int)P, mats, rank, sensor_frame(m->view, pl.sh.interp != 0),
                                  scan, (int)N, scan_layout(pl.sh), packed, s));
  }
  const double sig = (double)p->sigma_hit;
  SensorArgs a;
  a.map = m->view;
  a.mats = mats;
  a.scan = (const float4*)packed;
  a.layout = scan_layout(pl.sh);
  a.partial = partial;
  a.status = status;
  a.P = (int)P;
  a.N = (int)N;
  a.chunk = pl.sh.chunk;
  a.K = pl.K;
  a.ppi = pl.sh.ppi;
  a.nblk = pl.nblk;
  a.sweep = pl.sweep;
  a.n_items = pl.n_items;
  a.mode = kernel_mode(m, p->mode);
  a.neglect = (p->flags & MCL_NEGLECT_OUTSIDE) ? 1 : 0;
  const float c = (float)(-0.5 / (sig * sig));
  const bool q16 = m->dtype == MCL_I16;
  const double scale = (double)m->view.scale;
  set_fills(m, &a);
  a.cs = sum_exponent_constant(sig, q16, scale);
  a.store_scale = (q16 && p->mode == MCL_LOGPROD) ? (float)(scale * scale) : 1.0f;
  if (pl.dynamic) {
    a.queue = (unsigned long long*)(ws + pl.off_queue);
    MCL_CUDA(cudaMemsetAsync(a.queue, 0, sizeof(unsigned long long), s));
  }
  {
    PhaseScope ps(MCL_PHASE_SENSOR, s);
    MCL_CUDA(launch_sensor(kernel_kind(m), m->view.layout, m->dtype, a, pl.sh, s));
  }
  const float k = (float)(1.0 / std::sqrt(2.0 * 3.141592653589793 * sig * sig));
  const int nb = normalise_blocks((int)P);
  {
    PhaseScope ps(MCL_PHASE_REDUCE, s);
    MCL_CUDA(launch_finish_and_normalise(partial, rank, (int)P, pl.K, p->mode, c, k, L, nullptr,
                                         bstats, nb, nullptr, s));
  }
  if (w) {
    PhaseScope ps(MCL_PHASE_NORMALISE, s);
    MCL_CUDA(launch_normalise_from_stats(L, (int)P, w, bstats, nb, ostats, particles,
                                         (EstPartial*)(ws + pl.off_est), est, s));
  }
  return MCL_OK;
}

}  // namespace mcl

extern "C" {

mcl_status mcl_sensor_update(mcl_map_t m, const float* particles, int64_t P, const float* scan,
                             int64_t N, const mcl_sensor_params* p, float* logw, float* w,
                             mcl_stream_t stream) {
  return sensor_update(m, particles, P, scan, N, p, logw, w, nullptr, (cudaStream_t)stream);
}

mcl_status mcl_sensor_update_estimate(mcl_map_t m, const float* particles, int64_t P,
                                      const float* scan, int64_t N, const mcl_sensor_params* p,
                                      float* logw, float* w, mcl_estimate* out,
                                      mcl_stream_t stream) {
  if (!w || !out) return fail(MCL_EINVAL, "sensor_update_estimate: NULL w or out");
  if (!aligned(out, 8)) return fail(MCL_EINVAL, "sensor_update_estimate: out needs 8-byte alignment");
  return sensor_update(m, particles, P, scan, N, p, logw, w, out, (cudaStream_t)stream);
}

mcl_status mcl_pose_estimate(const float* particles, const float* w, int64_t P, mcl_estimate* out,
                             mcl_stream_t stream) {
  if (!particles || !w || !out) return fail(MCL_EINVAL, "pose_estimate: NULL pointer");
  if (P < 1 || P > kMaxCount) return fail(MCL_EINVAL, "pose_estimate: P = %lld", (long long)P);
  if (!aligned(particles, 4) || !aligned(w, 4) || !aligned(out, 8))
    return fail(MCL_EINVAL, "pose_estimate: misaligned pointer");
  cudaStream_t s = (cudaStream_t)stream;
  void* ws = nullptr;
  if (mcl_status rc = workspace(s, (size_t)normalise_blocks((int)P) * sizeof(EstPartial), &ws)) return rc;
  PhaseScope ps(MCL_PHASE_NORMALISE, s);
  MCL_CUDA(launch_pose_estimate(particles, w, (int)P, (EstPartial*)ws, out, s));
  return MCL_OK;
}

mcl_status mcl_normalise(const float* logw, int64_t P, float* w, float* out_stats, mcl_stream_t stream) {
  if (!logw || !w) return fail(MCL_EINVAL, "normalise: NULL logw or w");
  if (P < 1 || P > kMaxCount) return fail(MCL_EINVAL, "normalise: P = %lld", (long long)P);
  if (!aligned(logw, 4) || !aligned(w, 4) || !aligned(out_stats, 4))
    return fail(MCL_EINVAL, "normalise: misaligned pointer");
  cudaStream_t s = (cudaStream_t)stream;
  const int nb = normalise_blocks((int)P);
  void* ws = nullptr;
  if (mcl_status rc = workspace(s, (size_t)nb * sizeof(float2), &ws)) return rc;
  PhaseScope ps(MCL_PHASE_NORMALISE, s);
  MCL_CUDA(launch_normalise(logw, (int)P, w, (float2*)ws, nb, out_stats, s));
  return MCL_OK;
}

mcl_status mcl_pose_to_matrix(const float* particles, int64_t P, float* out_mat, mcl_stream_t stream) {
  if (!particles || !out_mat) return fail(MCL_EINVAL, "pose_to_matrix: NULL pointer");
  if (P < 1 || P > kMaxCount) return fail(MCL_EINVAL, "pose_to_matrix: P = %lld", (long long)P);
  if (!aligned(particles, 4) || !aligned(out_mat, 16))
    return fail(MCL_EINVAL, "pose_to_matrix: particles need 4-byte, out_mat 16-byte alignment");
  PhaseScope ps(MCL_PHASE_POSE, (cudaStream_t)stream);
  MCL_CUDA(launch_pose_to_matrix(particles, (int)P, (float4*)out_mat, nullptr, (cudaStream_t)stream));
  return MCL_OK;
}

// ---------------------------------------------------------------- resampling
mcl_status mcl_resample(const float* w, int64_t P, double r, int32_t* idx, const float* pin,
                        float* pout, mcl_stream_t stream) {
  if (!w || !idx) return fail(MCL_EINVAL, "resample: NULL w or idx");
  if (P < 1 || P > kMaxCount) return fail(MCL_EINVAL, "resample: P = %lld", (long long)P);
  if (!(r >= 0.0 && r < 1.0)) return fail(MCL_EINVAL, "resample: r must lie in [0, 1)");
  if (pin && !pout) return fail(MCL_EINVAL, "resample: particles_out NULL");
  if (pin && pin == pout) return fail(MCL_EINVAL, "resample: particles_in and particles_out alias");
  if (!aligned(w, 4) || !aligned(idx, 4) || !aligned(pin, 4) || !aligned(pout, 4))
    return fail(MCL_EINVAL, "resample: misaligned pointer");
  cudaStream_t s = (cudaStream_t)stream;
  const int nt = resample_tiles((int)P);
  const size_t o_cum = 0, o_tot = align256((size_t)P * 8), o_last = align256(o_tot + (size_t)(nt + 1) * 8),
               total = align256(o_last + (size_t)(nt + 1) * 8);
  char* ws = nullptr;
  if (mcl_status rc = workspace(s, total, (void**)&ws)) return rc;
  PhaseScope ps(MCL_PHASE_RESAMPLE, s, resample_kernels((int)P));
  MCL_CUDA(launch_resample(w, (int)P, r, idx, pin, pout, (double*)(ws + o_cum), (double*)(ws + o_tot),
                           (long long*)(ws + o_last), s));
  return MCL_OK;
}

mcl_status mcl_resample_noalloc(const float* w, int64_t P, double r, int32_t* idx, const float* pin,
                                float* pout, mcl_stream_t stream) {
  if (!w || !idx) return fail(MCL_EINVAL, "resample_noalloc: NULL w or idx");
  if (P < 1 || P > kStaticMaxParticles)
    return fail(MCL_EINVAL, "resample_noalloc: P = %lld outside [1, %d] (static scratch limit)",
                (long long)P, kStaticMaxParticles);
  if (!(r >= 0.0 && r < 1.0)) return fail(MCL_EINVAL, "resample_noalloc: r must lie in [0, 1)");
  if (pin && !pout) return fail(MCL_EINVAL, "resample_noalloc: particles_out NULL");
  if (pin && pin == pout) return fail(MCL_EINVAL, "resample_noalloc: particles_in and particles_out alias");
  if (!aligned(w, 4) || !aligned(idx, 4) || !aligned(pin, 4) || !aligned(pout, 4))
    return fail(MCL_EINVAL, "resample_noalloc: misaligned pointer");
  // the scope records pooled events only; it allocates no device memory
  PhaseScope ps(MCL_PHASE_RESAMPLE, (cudaStream_t)stream, resample_kernels((int)P));
  MCL_CUDA(launch_resample_static(w, (int)P, r, idx, pin, pout, (cudaStream_t)stream));
  return MCL_OK;
}

// ---------------------------------------------------------------- motion
mcl_status mcl_motion_update(float* particles, int64_t P, const float delta[6], const float sigma[6],
                             uint64_t seed, uint64_t step, mcl_stream_t stream) {
  if (!particles || !delta || !sigma) return fail(MCL_EINVAL, "motion_update: NULL pointer");
  if (P < 1 || P > kMaxCount) return fail(MCL_EINVAL, "motion_update: P = %lld", (long long)P);
  if (!aligned(particles, 4)) return fail(MCL_EINVAL, "motion_update: misaligned particles");
  for (int k = 0; k < 6; ++k) {
    if (!std::isfinite(delta[k])) return fail(MCL_EINVAL, "motion_update: delta not finite");
    if (!std::isfinite(sigma[k]) || sigma[k] < 0.f) return fail(MCL_EINVAL, "motion_update: sigma");
  }
  PhaseScope ps(MCL_PHASE_MOTION, (cudaStream_t)stream);
  MCL_CUDA(launch_motion(particles, (int)P, delta, sigma, seed, step, (cudaStream_t)stream));
  return MCL_OK;
}

// ---------------------------------------------------------------- gather roofline
mcl_status mcl_gather_bench(const void* buf, int64_t n_elems, int32_t elem_bytes, int32_t blocks,
                            int32_t iters, uint64_t seed, mcl_stream_t stream) {
  if (!buf || n_elems < 1) return fail(MCL_EINVAL, "gather_bench: empty buffer");
  if (elem_bytes != 2 && elem_bytes != 4) return fail(MCL_EINVAL, "gather_bench: elem_bytes %d", elem_bytes);
  if (blocks < 1 || iters < 1) return fail(MCL_EINVAL, "gather_bench: blocks and iters must be >= 1");
  if (!aligned(buf, (size_t)elem_bytes)) return fail(MCL_EINVAL, "gather_bench: misaligned buffer");
  cudaStream_t s = (cudaStream_t)stream;
  void* ws = nullptr;
  if (mcl_status rc = workspace(s, (size_t)blocks * sizeof(float), &ws)) return rc;
  PhaseScope ps(MCL_PHASE_OTHER, s);
  MCL_CUDA(launch_gather_bench(buf, n_elems, elem_bytes, blocks, iters, seed, (float*)ws, s));
  return MCL_OK;
}

// ---------------------------------------------------------------- runtime
mcl_status mcl_workspace_release(mcl_stream_t stream) {
  int dev = 0;
  MCL_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_ws.find({dev, (uintptr_t)stream});
  if (it == g_ws.end()) return MCL_OK;
  MCL_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  if (it->second.first) MCL_CUDA(cudaFree(it->second.first));
  g_ws.erase(it);
  return MCL_OK;
}

mcl_status mcl_profile_begin(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& pe : g_prof) {
    g_event_pool.push_back(pe.a);
    g_event_pool.push_back(pe.b);
  }
  g_prof.clear();
  g_prof_on = true;
  return MCL_OK;
}

mcl_status mcl_profile_end(mcl_profile* out) {
  std::vector<PhaseEvents> recs;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    g_prof_on = false;
    recs.swap(g_prof);
  }
  if (out && out->struct_size < sizeof(mcl_profile)) return fail(MCL_EINVAL, "profile_end: struct_size");
  if (out) {
    for (int k = 0; k < MCL_NUM_PHASES; ++k) {
      out->launches[k] = 0;
      out->ms[k] = 0.0;
    }
  }
  mcl_status rc = MCL_OK;
  for (auto& pe : recs) {
    cudaError_t e = cudaEventSynchronize(pe.b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, pe.a, pe.b);
    if (e != cudaSuccess && rc == MCL_OK) rc = cuda_fail(e, "profile_end");
    if (out && pe.phase >= 0 && pe.phase < MCL_NUM_PHASES) {
      out->launches[pe.phase] += pe.kernels;
      out->ms[pe.phase] += ms;
    }
  }
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& pe : recs) {
    g_event_pool.push_back(pe.a);
    g_event_pool.push_back(pe.b);
  }
  return rc;
}

}  // extern "C"
