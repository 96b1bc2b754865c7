// Spatial processing order of the particles (a GB300 locality device; the
// paper evaluates particles in the order given, Sec. V-B).
//
// Particles are bucketed by position into a 64 x 64 x 64 grid over the map's
// extent, buckets ordered along a Morton (Z-order) curve, and each particle
// gets a slot rank[p] in that order (counting sort: histogram, one-block
// exclusive scan, scatter). The sensor kernel then works on the particles slot
// by slot, so the CTAs running at the same time hold particles that are close
// in space and read the same map bricks from L2. Each particle's result
// depends only on its own pose, never on its slot, so the order within a
// bucket (decided by atomics) changes nothing downstream.
#include "mcl_internal.h"

namespace mcl {
namespace {

constexpr int kOrderBits = 6;                         // cells per axis = 64
constexpr int kOrderBuckets = 1 << (3 * kOrderBits);  // 262144
constexpr int kScanThreads = 1024;

__device__ __forceinline__ uint32_t spread3(uint32_t v) {
  uint32_t r = 0;
#pragma unroll
  for (int b = 0; b < kOrderBits; ++b) r |= ((v >> b) & 1u) << (3 * b);
  return r;
}

__device__ __forceinline__ uint32_t cell_of(float x, float o, float s) {
  const float u = (x - o) * s;
  // NaN and everything below the extent go to cell 0, everything above to 63
  return u >= 1.0f ? (uint32_t)fminf(u, (float)((1 << kOrderBits) - 1)) : 0u;
}

__global__ void k_order_keys(const float* __restrict__ poses, int P, float3 o, float3 s,
                             uint32_t* __restrict__ key, uint32_t* __restrict__ hist) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const float* q = poses + 6 * (size_t)p;
  const uint32_t k = spread3(cell_of(q[0], o.x, s.x)) | (spread3(cell_of(q[1], o.y, s.y)) << 1) |
                     (spread3(cell_of(q[2], o.z, s.z)) << 2);
  key[p] = k;
  atomicAdd(hist + k, 1u);
}

// One block: exclusive prefix of the bucket counts, in place.
__global__ void __launch_bounds__(kScanThreads) k_order_scan(uint32_t* __restrict__ hist) {
  constexpr int per = kOrderBuckets / kScanThreads;
  __shared__ uint32_t warp_tot[32];
  uint32_t* mine = hist + threadIdx.x * per;
  uint32_t local = 0;
  for (int i = 0; i < per; ++i) local += mine[i];
  // inclusive scan of the per-thread totals
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = local;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += v;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t t = warp_tot[lane];
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t v = __shfl_up_sync(0xffffffffu, t, off);
      if (lane >= off) t += v;
    }
    warp_tot[lane] = t;
  }
  __syncthreads();
  uint32_t run = incl - local + (warp > 0 ? warp_tot[warp - 1] : 0u);
  for (int i = 0; i < per; ++i) {
    const uint32_t c = mine[i];
    mine[i] = run;
    run += c;
  }
}

__global__ void k_order_scatter(const uint32_t* __restrict__ key, int P,
                                uint32_t* __restrict__ cursor, int* __restrict__ rank) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  rank[p] = (int)atomicAdd(cursor + key[p], 1u);
}

}  // namespace

size_t order_hist_bytes() { return (size_t)kOrderBuckets * sizeof(uint32_t); }

cudaError_t launch_particle_order(const float* poses, int P, const MapView& m, uint32_t* key,
                                  uint32_t* hist, int* rank, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(hist, 0, order_hist_bytes(), s);
  if (e != cudaSuccess) return e;
  const float cells = (float)(1 << kOrderBits);
  const float ex = m.fnx / m.inv, ey = m.fny / m.inv, ez = m.fnz / m.inv;  // extent in metres
  const float3 o = make_float3(m.ox, m.oy, m.oz);
  const float3 sc = make_float3(cells / ex, cells / ey, cells / ez);
  const int g = (P + 255) / 256;
  k_order_keys<<<g, 256, 0, s>>>(poses, P, o, sc, key, hist);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_order_scan<<<1, kScanThreads, 0, s>>>(hist);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_order_scatter<<<g, 256, 0, s>>>(key, P, hist, rank);
  return cudaGetLastError();
}

}  // namespace mcl
