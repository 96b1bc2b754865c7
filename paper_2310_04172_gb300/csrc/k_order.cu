// Spatial processing order of the particles (a GB300 locality device; the
// paper evaluates particles in the order given, Sec. V-B).
//
// Particles are bucketed by position into cubic cells, 64 along the longest
// axis of the map's extent (fewer along the others), buckets ordered along a
// Morton (Z-order) curve, and each particle
// gets a slot rank[p] in that order (counting sort: histogram, exclusive
// scan of the bucket counts in tiles of 1024 plus a scan of the tile totals,
// scatter). The sensor kernel then works on the particles slot
// by slot, so the CTAs running at the same time hold particles that are close
// in space and read the same map bricks from L2. Each particle's result
// depends only on its own pose, never on its slot, so the order within a
// bucket (decided by atomics) changes nothing downstream.
#include "mcl_internal.h"

namespace mcl {
namespace {

// MCL_ORDER_YAW_BITS: the low bits of a bucket number are the particle's
// yaw bin (2^bits bins over the full turn) and the cells are coarser, so
// that within a cell the particles facing the same way come together.
#ifndef MCL_ORDER_YAW_BITS
#define MCL_ORDER_YAW_BITS 0
#endif
constexpr int kYawBits = MCL_ORDER_YAW_BITS;
static_assert(kYawBits % 3 == 0 && kYawBits < 18, "yaw bits replace whole Morton levels");
constexpr int kOrderBits = 6 - kYawBits / 3;          // cells per axis = 2^kOrderBits
constexpr int kOrderBuckets = 1 << 18;                // 262144
constexpr int kScanTile = 1024;                          // buckets per scan block
constexpr int kScanTiles = kOrderBuckets / kScanTile;  // 256

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

__device__ __forceinline__ void order_key(const float* __restrict__ poses, int p, float3 o, float3 s,
                                          uint32_t* __restrict__ key, uint32_t* __restrict__ hist) {
  const float* q = poses + 6 * (size_t)p;
  uint32_t k = spread3(cell_of(q[0], o.x, s.x)) | (spread3(cell_of(q[1], o.y, s.y)) << 1) |
               (spread3(cell_of(q[2], o.z, s.z)) << 2);
  if constexpr (kYawBits > 0) {
    const float t = q[5] * 0.15915494f;  // turns
    const float f = t - floorf(t);       // [0, 1]; NaN and inf give NaN
    const uint32_t yb = f >= 0.f ? min((uint32_t)(f * (float)(1 << kYawBits)), (1u << kYawBits) - 1u) : 0u;
    k = (k << kYawBits) | yb;
  }
  key[p] = k;
  atomicAdd(hist + k, 1u);
}

__global__ void k_order_keys(const float* __restrict__ poses, int P, float3 o, float3 s,
                             uint32_t* __restrict__ key, uint32_t* __restrict__ hist) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < P) order_key(poses, p, o, s, key, hist);
}

// Inclusive scan over a block of 1024 threads (warp shuffles, then the warp
// totals); returns this thread's inclusive prefix and the block total.
__device__ __forceinline__ uint32_t block_incl_scan(uint32_t v, uint32_t* warp_tot, uint32_t& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t u = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += u;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int nw = (int)(blockDim.x >> 5);
    uint32_t t = lane < nw ? warp_tot[lane] : 0u;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t u = __shfl_up_sync(0xffffffffu, t, off);
      if (lane >= off) t += u;
    }
    warp_tot[lane] = t;
  }
  __syncthreads();
  total = warp_tot[(blockDim.x >> 5) - 1];
  return incl + (warp > 0 ? warp_tot[warp - 1] : 0u);
}

// Tile b: exclusive prefix of its 1024 bucket counts in place (coalesced),
// its total to tile_off[b].
__device__ __forceinline__ void scan_tile(uint32_t* __restrict__ hist, uint32_t* __restrict__ tile_off,
                                          int b) {
  __shared__ uint32_t warp_tot[32];
  const size_t i = (size_t)b * kScanTile + threadIdx.x;
  const uint32_t v = hist[i];
  uint32_t total;
  const uint32_t incl = block_incl_scan(v, warp_tot, total);
  hist[i] = incl - v;
  if (threadIdx.x == 0) tile_off[b] = total;
}

__global__ void __launch_bounds__(kScanTile) k_order_scan_tiles(uint32_t* __restrict__ hist,
                                                                 uint32_t* __restrict__ tile_off) {
  scan_tile(hist, tile_off, blockIdx.x);
}

// Exclusive prefix of the tile totals in place (one block of kScanTiles).
__device__ __forceinline__ void scan_totals(uint32_t* __restrict__ tile_off) {
  __shared__ uint32_t warp_tot[32];
  const uint32_t v = tile_off[threadIdx.x];
  uint32_t total;
  const uint32_t incl = block_incl_scan(v, warp_tot, total);
  tile_off[threadIdx.x] = incl - v;
}

__global__ void __launch_bounds__(kScanTiles) k_order_scan_totals(uint32_t* __restrict__ tile_off) {
  scan_totals(tile_off);
}

__device__ __forceinline__ void order_rank(const uint32_t* __restrict__ key, int p,
                                           uint32_t* __restrict__ cursor,
                                           const uint32_t* __restrict__ tile_off, int* __restrict__ rank) {
  const uint32_t k = key[p];
  rank[p] = (int)(__ldg(tile_off + k / kScanTile) + atomicAdd(cursor + k, 1u));
}

__global__ void k_order_scatter(const uint32_t* __restrict__ key, int P,
                                uint32_t* __restrict__ cursor, const uint32_t* __restrict__ tile_off,
                                int* __restrict__ rank) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < P) order_rank(key, p, cursor, tile_off, rank);
}

// ---------------------------------------------------------------- batched forms
// One launch of each step for every session with a spatial order (segments
// of blocks per session, see SegBlocks); the same arithmetic as above.
constexpr int kZeroPerBlock = kSideThreads * 4;  // histogram entries a zeroing block clears

__global__ void __launch_bounds__(kSideThreads) k_order_zero_b(const SideSeg* __restrict__ segs, SegBlocks b) {
  const int s = seg_of(b.first, b.n, blockIdx.x);
  const int j = blockIdx.x - __ldg(b.first + s);
  uint4* h = reinterpret_cast<uint4*>(segs[s].hist) + (size_t)j * kSideThreads + threadIdx.x;
  *h = make_uint4(0u, 0u, 0u, 0u);
}

__global__ void __launch_bounds__(kSideThreads) k_order_keys_b(const SideSeg* __restrict__ segs, SegBlocks b) {
  const int s = seg_of(b.first, b.n, blockIdx.x);
  const SideSeg& g = segs[s];
  const int p = (blockIdx.x - __ldg(b.first + s)) * kSideThreads + threadIdx.x;
  if (p < g.P) order_key(g.particles, p, g.order_o, g.order_s, g.key, g.hist);
}

__global__ void __launch_bounds__(kScanTile) k_order_scan_tiles_b(const SideSeg* __restrict__ segs, SegBlocks b) {
  const int s = seg_of(b.first, b.n, blockIdx.x);
  scan_tile(segs[s].hist, segs[s].hist + kOrderBuckets, blockIdx.x - __ldg(b.first + s));
}

__global__ void __launch_bounds__(kScanTiles) k_order_scan_totals_b(const SideSeg* __restrict__ segs, SegBlocks b) {
  const int s = seg_of(b.first, b.n, blockIdx.x);
  scan_totals(segs[s].hist + kOrderBuckets);
}

__global__ void __launch_bounds__(kSideThreads) k_order_scatter_b(const SideSeg* __restrict__ segs, SegBlocks b) {
  const int s = seg_of(b.first, b.n, blockIdx.x);
  const SideSeg& g = segs[s];
  const int p = (blockIdx.x - __ldg(b.first + s)) * kSideThreads + threadIdx.x;
  if (p < g.P) order_rank(g.key, p, g.hist, g.hist + kOrderBuckets, g.rank);
}

}  // namespace

// bucket counts / cursors, then the tile offsets
size_t order_hist_bytes() { return (size_t)(kOrderBuckets + kScanTiles) * sizeof(uint32_t); }

void order_grid(const MapView& m, float3* o, float3* sc) {
  const float cells = (float)(1 << kOrderBits);
  const float ex = m.fnx / m.inv, ey = m.fny / m.inv, ez = m.fnz / m.inv;  // extent in metres
  *o = make_float3(m.ox, m.oy, m.oz);
  // cubic cells, 64 along the longest axis: a run of buckets on the curve
  // then covers a compact block of space rather than a flat slab
  const float emax = fmaxf(ex, fmaxf(ey, ez));
  *sc = make_float3(cells / emax, cells / emax, cells / emax);
}

cudaError_t launch_particle_order(const float* poses, int P, const MapView& m, uint32_t* key,
                                  uint32_t* hist, int* rank, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(hist, 0, (size_t)kOrderBuckets * sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  float3 o, sc;
  order_grid(m, &o, &sc);
  const int g = (P + 255) / 256;
  k_order_keys<<<g, 256, 0, s>>>(poses, P, o, sc, key, hist);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  uint32_t* tile_off = hist + kOrderBuckets;
  k_order_scan_tiles<<<kScanTiles, kScanTile, 0, s>>>(hist, tile_off);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_order_scan_totals<<<1, kScanTiles, 0, s>>>(tile_off);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_order_scatter<<<g, 256, 0, s>>>(key, P, hist, tile_off, rank);
  return cudaGetLastError();
}

int side_blocks_order(int kind, const SideSeg& g) {
  if (!g.rank) return 0;
  switch (kind) {
    case kSideOrderZero: return kOrderBuckets / kZeroPerBlock;
    case kSideOrderKeys:
    case kSideOrderScatter: return (g.P + kSideThreads - 1) / kSideThreads;
    case kSideOrderTiles: return kScanTiles;
    case kSideOrderTotals: return 1;
    default: return 0;
  }
}

cudaError_t launch_side_order(int kind, const SideSeg* segs, const SegBlocks& b, cudaStream_t s) {
  if (b.blocks == 0) return cudaSuccess;
  switch (kind) {
    case kSideOrderZero: k_order_zero_b<<<b.blocks, kSideThreads, 0, s>>>(segs, b); break;
    case kSideOrderKeys: k_order_keys_b<<<b.blocks, kSideThreads, 0, s>>>(segs, b); break;
    case kSideOrderTiles: k_order_scan_tiles_b<<<b.blocks, kScanTile, 0, s>>>(segs, b); break;
    case kSideOrderTotals: k_order_scan_totals_b<<<b.blocks, kScanTiles, 0, s>>>(segs, b); break;
    case kSideOrderScatter: k_order_scatter_b<<<b.blocks, kSideThreads, 0, s>>>(segs, b); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace mcl
