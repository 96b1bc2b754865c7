// Systematic resampling (Sec. III: a new particle set drawn from the current
// one in proportion to the weights), exact and order-independent.
//
// Weights are quantised to integer multiples of 2^-52 (q = rint(w 2^52) 2^-52,
// exact in FP64 for any FP32 w). For normalised weights every partial sum of
// q stays below 2 and is therefore exact in FP64, so the prefix sum C is the
// same bit for bit whatever the summation order: tiles of 4096 scan locally,
// one block scans the tile totals, and each output j finds
// min{p : C_p > t_j}, t_j = ((j + r) / P) S, by a binary search over tile ends
// and then inside the tile. Sets of at most one tile take one fused launch.
#include <algorithm>
#include <mutex>

#include "mcl_internal.h"

namespace mcl {
namespace {

constexpr int kRT = 1024, kRI = 4, kTile = kRT * kRI;

__device__ __forceinline__ double warp_incl_scan(double v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const double o = __shfl_up_sync(0xffffffffu, v, off);
    if (lane >= off) v = __dadd_rn(v, o);
  }
  return v;
}

// Inclusive block scan of one double per thread (values exact, so the
// association order does not change the result). Returns the inclusive value;
// *total gets the block total.
__device__ __forceinline__ double block_incl_scan(double v, double* sh, double* total) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  double incl = warp_incl_scan(v);
  __syncthreads();
  if (lane == 31) sh[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    double t = lane < nw ? sh[lane] : 0.0;
    t = warp_incl_scan(t);
    sh[lane] = t;
  }
  __syncthreads();
  if (warp > 0) incl = __dadd_rn(incl, sh[warp - 1]);
  *total = sh[nw - 1];
  return incl;
}

__device__ __forceinline__ long long block_max_ll(long long v, long long* sh) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const long long o = __shfl_xor_sync(0xffffffffu, v, off);
    v = o > v ? o : v;
  }
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  v = lane < nw ? sh[lane] : -1;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const long long o = __shfl_xor_sync(0xffffffffu, v, off);
    v = o > v ? o : v;
  }
  return v;
}

__device__ __forceinline__ void tile_scan(const float* __restrict__ w, int P, double* __restrict__ cum,
                                          double* __restrict__ tile_total,
                                          long long* __restrict__ tile_last, int blk) {
  __shared__ double sh[32];
  __shared__ long long shl[32];
  const long long base = (long long)blk * kTile + (long long)threadIdx.x * kRI;
  double run = 0.0, q[kRI];
  long long last = -1;
#pragma unroll
  for (int i = 0; i < kRI; ++i) {
    const long long p = base + i;
    double v = 0.0;
    if (p < P) {
      v = __dmul_rn(rint(__dmul_rn((double)w[p], 0x1.0p52)), 0x1.0p-52);
      if (v > 0.0) last = p;
    }
    run = __dadd_rn(run, v);
    q[i] = run;
  }
  double total;
  const double incl = block_incl_scan(run, sh, &total);
  const double excl = __dsub_rn(incl, run);
#pragma unroll
  for (int i = 0; i < kRI; ++i)
    if (base + i < P) cum[base + i] = __dadd_rn(excl, q[i]);
  last = block_max_ll(last, shl);
  if (threadIdx.x == 0) {
    tile_total[blk] = total;
    tile_last[blk] = last;
  }
}

__global__ void __launch_bounds__(kRT) k_tile_scan(const float* __restrict__ w, int P,
                                                   double* __restrict__ cum,
                                                   double* __restrict__ tile_total,
                                                   long long* __restrict__ tile_last) {
  tile_scan(w, P, cum, tile_total, tile_last, blockIdx.x);
}

// One block: tile totals -> exclusive tile offsets (in place); entry ntiles
// receives the grand total S and the last index with a positive weight.
__device__ __forceinline__ void tile_offsets(double* __restrict__ tile_total,
                                             long long* __restrict__ tile_last, int ntiles) {
  __shared__ double sh[32];
  __shared__ long long shl[32];
  double carry = 0.0;
  long long last = -1;
  for (int b = 0; b < ntiles; b += kRT) {
    const int i = b + threadIdx.x;
    const double v = i < ntiles ? tile_total[i] : 0.0;
    const long long l = i < ntiles ? tile_last[i] : -1;
    double total;
    const double incl = block_incl_scan(v, sh, &total);
    if (i < ntiles) tile_total[i] = __dadd_rn(carry, __dsub_rn(incl, v));
    carry = __dadd_rn(carry, total);
    const long long lm = block_max_ll(l, shl);
    last = lm > last ? lm : last;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    tile_total[ntiles] = carry;
    tile_last[ntiles] = last;
  }
}

__global__ void __launch_bounds__(kRT) k_tile_offsets(double* __restrict__ tile_total,
                                                      long long* __restrict__ tile_last,
                                                      int ntiles) {
  tile_offsets(tile_total, tile_last, ntiles);
}

// Draw j of the systematic scheme (target t_j, search over the tile ends,
// then inside the tile) and the gather of its particle.
__device__ __forceinline__ void systematic_one(const double* __restrict__ cum,
                                               const double* __restrict__ tile_off,
                                               const long long* __restrict__ tile_last, int P,
                                               int ntiles, double r, int32_t* __restrict__ idx,
                                               const float* __restrict__ pin,
                                               float* __restrict__ pout, int j) {
  const double S = tile_off[ntiles];
  int res;
  if (!(S > 0.0)) {
    res = j;  // all weights zero: identity
  } else {
    const double t = __dmul_rn(__ddiv_rn(__dadd_rn((double)j, r), (double)P), S);
    int lo = 0, hi = ntiles;  // first tile whose end C exceeds t
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (tile_off[mid + 1] > t) hi = mid; else lo = mid + 1;
    }
    if (lo == ntiles) {
      res = (int)tile_last[ntiles];
    } else {
      const double off = tile_off[lo];
      int a = lo * kTile, b = min(P, a + kTile);
      while (a < b) {
        const int mid = (a + b) >> 1;
        if (__dadd_rn(off, cum[mid]) > t) b = mid; else a = mid + 1;
      }
      res = a;
    }
  }
  idx[j] = res;
  if (pin) {
    const float* src = pin + 6 * (size_t)res;
    float* dst = pout + 6 * (size_t)j;
#pragma unroll
    for (int k = 0; k < 6; ++k) dst[k] = src[k];
  }
}

__global__ void k_systematic(const double* __restrict__ cum, const double* __restrict__ tile_off,
                             const long long* __restrict__ tile_last, int P, int ntiles, double r,
                             const double* __restrict__ r_dev, int32_t* __restrict__ idx,
                             const float* __restrict__ pin, float* __restrict__ pout) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= P) return;
  if (r_dev) r = *r_dev;
  systematic_one(cum, tile_off, tile_last, P, ntiles, r, idx, pin, pout, j);
}

// ---------------------------------------------------------------- batched forms
// The three-launch path for every session at once (segments of blocks,
// SegBlocks); for a set of at most one tile it draws the same indices as the
// fused small-set kernel (same quantised weights, exact prefix, targets and
// search).
__global__ void __launch_bounds__(kRT) k_tile_scan_b(const SideSeg* __restrict__ segs, SegBlocks b) {
  const int s = seg_of(b.first, b.n, blockIdx.x);
  const SideSeg& g = segs[s];
  tile_scan(g.w, g.P, g.cum, g.tile_total, g.tile_last, blockIdx.x - __ldg(b.first + s));
}

__global__ void __launch_bounds__(kRT) k_tile_offsets_b(const SideSeg* __restrict__ segs, SegBlocks b) {
  const int s = seg_of(b.first, b.n, blockIdx.x);
  const SideSeg& g = segs[s];
  tile_offsets(g.tile_total, g.tile_last, (g.P + kTile - 1) / kTile);
}

__global__ void __launch_bounds__(256) k_systematic_b(const SideSeg* __restrict__ segs, SegBlocks b) {
  const int s = seg_of(b.first, b.n, blockIdx.x);
  const SideSeg& g = segs[s];
  const int j = (blockIdx.x - __ldg(b.first + s)) * 256 + threadIdx.x;
  if (j >= g.P) return;
  systematic_one(g.cum, g.tile_total, g.tile_last, g.P, (g.P + kTile - 1) / kTile, *g.r, g.idx,
                 g.pin, g.pout, j);
}

// Sets of at most one tile in one launch: the same quantised weights, the
// same exact prefix (kept in shared memory), the same targets and search, so
// the same indices as the three-launch path. Every block forms the whole
// prefix (exact, so the same bits in every block and for any block size) and
// then serves its own contiguous slice of the targets: the FP64 division and
// search of each target run on several SMs instead of one (FP64 issue per SM
// is slow on this part).
__global__ void __launch_bounds__(kRT) k_systematic_small(const float* __restrict__ w, int P,
                                                          double r, const double* __restrict__ r_dev,
                                                          int32_t* __restrict__ idx,
                                                          const float* __restrict__ pin,
                                                          float* __restrict__ pout) {
  __shared__ double cs[kTile];
  __shared__ double sh[32];
  __shared__ long long shl[32];
  const int base = threadIdx.x * kRI;
  double run = 0.0, q[kRI];
  long long last = -1;
#pragma unroll
  for (int i = 0; i < kRI; ++i) {
    const int p = base + i;
    double v = 0.0;
    if (p < P) {
      v = __dmul_rn(rint(__dmul_rn((double)w[p], 0x1.0p52)), 0x1.0p-52);
      if (v > 0.0) last = p;
    }
    run = __dadd_rn(run, v);
    q[i] = run;
  }
  double S;
  const double incl = block_incl_scan(run, sh, &S);
  const double excl = __dsub_rn(incl, run);
#pragma unroll
  for (int i = 0; i < kRI; ++i)
    if (base + i < P) cs[base + i] = __dadd_rn(excl, q[i]);
  last = block_max_ll(last, shl);
  __syncthreads();
  if (r_dev) r = *r_dev;
  const int slice = (P + gridDim.x - 1) / gridDim.x;
  const int j_end = min(P, (int)(blockIdx.x + 1) * slice);
  for (int j = blockIdx.x * slice + threadIdx.x; j < j_end; j += blockDim.x) {
    int res;
    if (!(S > 0.0)) {
      res = j;  // all weights zero: identity
    } else {
      const double t = __dmul_rn(__ddiv_rn(__dadd_rn((double)j, r), (double)P), S);
      int a = 0, b = P;
      while (a < b) {
        const int mid = (a + b) >> 1;
        if (cs[mid] > t) b = mid; else a = mid + 1;
      }
      res = a < P ? a : (int)last;
    }
    idx[j] = res;
    if (pin) {
      const float* src = pin + 6 * (size_t)res;
      float* dst = pout + 6 * (size_t)j;
#pragma unroll
      for (int k = 0; k < 6; ++k) dst[k] = src[k];
    }
  }
}

}  // namespace

int resample_tiles(int P) { return (P + kTile - 1) / kTile; }
int resample_kernels(int P) { return P <= kTile ? 1 : 3; }

// ---------------------------------------------------------------- static scratch
// Scratch for the allocation-free entry point (mcl_resample_noalloc), for
// callers that may not allocate device memory: the FP64 prefix C (one double
// per particle) and the tile totals and last-positive indices (one entry per
// tile plus the grand total), for at most kStaticMaxParticles particles. It is
// a file-scope device array, so every GPU that loads the library holds it
// (about 8.4 MB) until the process exits. Every call overwrites all of it that
// it reads (k_tile_scan writes C and the tile entries, k_tile_offsets the
// offsets and totals), so nothing has to start at zero; but all calls on a
// device share it, and calls whose work overlaps on the GPU race.
constexpr int kStaticTiles = (kStaticMaxParticles + kTile - 1) / kTile;
constexpr size_t kStaticBytes =
    (size_t)kStaticMaxParticles * sizeof(double) + 2 * (size_t)(kStaticTiles + 1) * sizeof(double);
static __device__ __align__(256) unsigned char g_resample_scratch[kStaticBytes];

namespace {
std::mutex g_static_mu;
void* g_static_ptr[kMaxDevices] = {};  // device address of the array, per device
}  // namespace

cudaError_t launch_resample_static(const float* w, int P, double r, int32_t* idx,
                                   const float* particles_in, float* particles_out, cudaStream_t s) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  void* base = nullptr;
  {
    // Once per device, with that device current: the host-side name of the
    // array is only a stand-in, its device address comes from the runtime.
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_resample_scratch);
      if (e != cudaSuccess) return e;
      g_static_ptr[dev] = p;
    }
    base = g_static_ptr[dev];
  }
  double* cum = static_cast<double*>(base);
  double* tile_total = cum + kStaticMaxParticles;
  long long* tile_last = reinterpret_cast<long long*>(tile_total + (kStaticTiles + 1));
  return launch_resample(w, P, r, idx, particles_in, particles_out, cum, tile_total, tile_last, s);
}

int side_blocks_resample(int kind, const SideSeg& g) {
  if (!g.idx) return 0;
  switch (kind) {
    case kSideTileScan: return (g.P + kTile - 1) / kTile;
    case kSideTileOffsets: return 1;
    case kSideSystematic: return (g.P + 255) / 256;
    default: return 0;
  }
}

cudaError_t launch_side_resample(int kind, const SideSeg* segs, const SegBlocks& b, cudaStream_t s) {
  if (b.blocks == 0) return cudaSuccess;
  switch (kind) {
    case kSideTileScan: k_tile_scan_b<<<b.blocks, kRT, 0, s>>>(segs, b); break;
    case kSideTileOffsets: k_tile_offsets_b<<<b.blocks, kRT, 0, s>>>(segs, b); break;
    case kSideSystematic: k_systematic_b<<<b.blocks, 256, 0, s>>>(segs, b); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_resample(const float* w, int P, double r, int32_t* idx,
                            const float* particles_in, float* particles_out, double* cum,
                            double* tile_total, long long* tile_last, cudaStream_t s,
                            const double* r_dev) {
  if (P <= kTile) {
    // threads: kRI weights each, whole warps; blocks: about 128 targets each
    const int threads = std::min(kRT, ((P + kRI - 1) / kRI + 31) / 32 * 32);
    const int blocks = std::min(32, (P + 127) / 128);
    k_systematic_small<<<blocks, threads, 0, s>>>(w, P, r, r_dev, idx, particles_in, particles_out);
    return cudaGetLastError();
  }
  const int ntiles = resample_tiles(P);
  k_tile_scan<<<ntiles, kRT, 0, s>>>(w, P, cum, tile_total, tile_last);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_tile_offsets<<<1, kRT, 0, s>>>(tile_total, tile_last, ntiles);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_systematic<<<(P + 255) / 256, 256, 0, s>>>(cum, tile_total, tile_last, P, ntiles, r, r_dev,
                                               idx, particles_in, particles_out);
  return cudaGetLastError();
}

}  // namespace mcl
