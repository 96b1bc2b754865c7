// Internal declarations of the GB300 MCL library: the device view of a map,
// the index and look-up rule, kernel launchers and the host runtime pieces.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "mcl.h"

namespace mcl {

constexpr int kBrick = 16;
constexpr int kBrickVoxels = kBrick * kBrick * kBrick;
// Bricks the cell-grid index addresses: the grid kernels form value indices
// slot * 4096 + offset in 32 bits (one instruction fewer per value read than
// 64-bit indices: 177.1 -> 175.7 ms for the 1M x 65,536 building, 676 -> 594
// ms for its trilinear read), so slot * 4096 must stay below 2^32.
constexpr int64_t kGridMaxBricks = int64_t(1) << 20;
constexpr uint32_t kEmptyKey = 0xFFFFFFFFu;
constexpr uint32_t kNoSlot = 0xFFFFFFFFu;
constexpr int kKindBrickBlock4 = 2;  // internal kind: brick map stored in 4x4x4 blocks
constexpr int kModeScore = 2;        // internal mode: SUM on a score map (stored values are scores)
constexpr int kKindBrickGrid = 3;    // internal kind: brick map (linear layout) with the cell grid index
constexpr int kKindDenseTiles = 4;   // internal kind: dense map stored in 8 x 4 tiles (dense_index)
__host__ __device__ constexpr bool is_dense(int kind) { return kind == MCL_MAP_DENSE || kind == kKindDenseTiles; }

// Bits of the per-device status word that kernels set instead of faulting.
enum : unsigned { kDevErrTimeout = 1u, kDevErrIndex = 2u };

// Debug builds (-DMCL_DEBUG_BOUNDS=1) check every brick slot a kernel is about
// to read against the number of stored bricks; a bad one sets kDevErrIndex in
// the status word (mcl_sync reports MCL_EINTERNAL) and reads nothing.
#ifndef MCL_DEBUG_BOUNDS
#define MCL_DEBUG_BOUNDS 0
#endif

// Device view of a TSDF map (Sec. III). Passed by value to the kernels.
struct MapView {
  const void* values;   // dense grid or brick-major values
  const uint2* table;   // BRICK, hash index: open-addressing hash (key, slot), capacity 2^bits
  const uint32_t* grid; // BRICK, grid index: slot of each brick cell (kNoSlot if none), cell
                        // (cx, cy, cz) at cz * gsz + cy * gsy + cx for every cx in [-1, nbx],
                        // cy in [-1, nby], cz in [-1, nbz] (guard cells outside the map)
  uint32_t n_slots;     // BRICK: bricks stored (slots are below this)
  float ox, oy, oz;     // grid corner
  float inv;            // 1 / voxel as used by the index rule
  float fnx, fny, fnz;  // dims as FP32 for the inside test
  int nx, ny, nz;
  uint32_t nbx, nby;    // BRICK: brick grid size (x, y)
  uint32_t gsy, gsz;    // BRICK, grid index: cell strides nbx + 1 and (nbx + 1)(nby + 1)
  uint32_t ntx, nty;    // DENSE, tiled: tiles along x and y (dense_index)
  uint32_t tcy, tsz;    // DENSE, tiled: 8 ntx - 8 and 32 ntx nty (dense_index)
  uint32_t hash_mask;   // capacity - 1
  int hash_shift;       // 32 - bits
  int max_probe;        // longest probe sequence of a stored key (>= 1)
  float tau;            // truncation: value read where nothing is stored
  float scale;          // I16: tau / 32767 in FP32
  int layout;           // BRICK: MCL_LAYOUT_LINEAR or MCL_LAYOUT_BLOCK4
};

// Dense maps (kKindDenseTiles) are stored in tiles of 8 x 4 x 1 voxels
// (x-fastest rows of 8 in a tile, tiles x-fastest: ntx = ceil(nx / 8) by
// nty = ceil(ny / 4) per z layer), so a 128-byte line holds an 8 x 4 patch
// instead of 32 voxels of one row. A warp's gathers (neighbouring points of
// one ring, on walls facing x or y) then touch fewer lines: 7.9 -> 4.2 per
// request in a model of the VLP-16 hall, and the L1's requests to L2, which
// bound that L2-resident case, fall with them. Index of voxel (ix, iy, iz),
// at most 2^31 - 1 values after padding:
#ifndef MCL_DENSE_TILES
#define MCL_DENSE_TILES 1  // 0: every dense map linear
#endif
// ((iz nty + (iy >> 2)) ntx + (ix >> 3)) 32 + (iy & 3) 8 + (ix & 7), written
// as ix + 3 (ix & ~7) + 8 iy + (iy & ~3)(8 ntx - 8) + iz (32 ntx nty) so that
// it takes two masks, three multiply-adds and one shift-add (tcy, tsz:
// the two strides, precomputed).
template <bool TILES>
__host__ __device__ inline uint32_t dense_index(uint32_t ix, uint32_t iy, uint32_t iz, uint32_t nx,
                                                uint32_t ny, uint32_t tcy, uint32_t tsz) {
  if constexpr (TILES) {
    return iz * tsz + ((iy & ~3u) * tcy + (ix + 3u * (ix & ~7u)) + (iy << 3));
  } else {
    return (iz * ny + iy) * nx + ix;
  }
}
// Values a dense map holds on the device (with the tiles' padding).
inline int64_t dense_stored(int64_t nx, int64_t ny, int64_t nz, bool tiles) {
  return tiles ? ((nx + 7) / 8 * 8) * ((ny + 3) / 4 * 4) * nz : nx * ny * nz;
}

// Fibonacci hashing of a brick-cell key (Knuth, TAOCP vol. 3, 6.4).
__host__ __device__ inline uint32_t brick_hash(uint32_t key, int shift) {
  return (key * 0x9E3779B1u) >> shift;
}

#ifdef __CUDACC__

// Voxel containing a world point (the map query): u = (x - o) * inv in two FP32
// roundings per axis, inside iff 0 <= u < n on all axes (NaN is outside),
// i = floor(u). Returns false outside the grid.
__device__ __forceinline__ bool voxel_of(const MapView& m, float x, float y, float z, int& ix,
                                         int& iy, int& iz) {
  float ux = __fmul_rn(__fsub_rn(x, m.ox), m.inv);
  float uy = __fmul_rn(__fsub_rn(y, m.oy), m.inv);
  float uz = __fmul_rn(__fsub_rn(z, m.oz), m.inv);
  bool in = (ux >= 0.f) & (ux < m.fnx) & (uy >= 0.f) & (uy < m.fny) & (uz >= 0.f) & (uz < m.fnz);
  ix = (int)ux;
  iy = (int)uy;
  iz = (int)uz;
  return in;
}

template <int DTYPE>
__device__ __forceinline__ float load_value(const MapView& m, size_t i) {
  if constexpr (DTYPE == MCL_F32) {
    return __ldg(static_cast<const float*>(m.values) + i);
  } else if constexpr (DTYPE == MCL_F16) {
    return __half2float(__ldg(static_cast<const __half*>(m.values) + i));
  } else {
    return (float)__ldg(static_cast<const short*>(m.values) + i) * m.scale;
  }
}

// In-brick offset of local voxel (lx, ly, lz) in the 4x4x4-block layout:
// block-major (block index z, y, x), each block z-major.
__host__ __device__ inline uint32_t block4_local(uint32_t lx, uint32_t ly, uint32_t lz) {
  return ((lz >> 2) << 10) | ((ly >> 2) << 8) | ((lx >> 2) << 6) | ((lz & 3u) << 4) |
         ((ly & 3u) << 2) | (lx & 3u);
}

// Cell-grid maps keep each brick's values rotated by the brick's cell
// coordinates: voxel (ix, iy, iz) sits at skew_local(ix, iy, iz) =
// (ix + 16 iy + 256 iz) mod 4096 of its brick, that is at lx + 16 ((ly + bx)
// mod 16) + 256 ((lz + by + carry) mod 16), a bijection of the brick's 4096
// places, and the grid holds slot * 4096 (or kNoSlot). The value index of a
// voxel is then grid[cell] | skew_local: two shift-adds of the voxel index
// and one OR whichever the brick, and a trilinear corner's offset is the
// lower corner's plus cx + 16 cy + 256 cz, mod 4096, across brick faces too.
#ifndef MCL_GRID_SKEW
#define MCL_GRID_SKEW 1
#endif
__host__ __device__ inline uint32_t skew_local(uint32_t ix, uint32_t iy, uint32_t iz) {
#if MCL_GRID_SKEW
  return (ix + (iy << 4) + (iz << 8)) & (uint32_t)(kBrickVoxels - 1);
#else
  return ((iz & 15u) << 8) | ((iy & 15u) << 4) | (ix & 15u);
#endif
}

// Brick-cell key (hash index; GRID: the cell's place in the padded grid) and
// in-brick offset of a voxel (GRID: skew_local).
template <bool GRID>
__device__ __forceinline__ void brick_key(const MapView& m, int ix, int iy, int iz, uint32_t& key,
                                          uint32_t& local) {
  if constexpr (GRID)
    key = (uint32_t)(iz >> 4) * m.gsz + (uint32_t)(iy >> 4) * m.gsy + (uint32_t)(ix >> 4);
  else
    key = ((uint32_t)(iz >> 4) * m.nby + (uint32_t)(iy >> 4)) * m.nbx + (uint32_t)(ix >> 4);
  const uint32_t lx = (uint32_t)ix & 15u, ly = (uint32_t)iy & 15u, lz = (uint32_t)iz & 15u;
  if constexpr (GRID)
    local = skew_local((uint32_t)ix, (uint32_t)iy, (uint32_t)iz);
  else
    local = m.layout == MCL_LAYOUT_BLOCK4 ? block4_local(lx, ly, lz) : ((lz * kBrick + ly) * kBrick + lx);
}

// Continue a probe sequence after a first entry that did not match. Bounded by
// the longest stored probe sequence, so an absent key ends without an EMPTY.
__device__ __forceinline__ uint32_t probe_rest(const MapView& m, uint32_t key, uint32_t h) {
  for (int it = 1; it < m.max_probe; ++it) {
    h = (h + 1) & m.hash_mask;
    uint2 e = __ldg(m.table + h);
    if (e.x == key) return e.y;
    if (e.x == kEmptyKey) return kNoSlot;
  }
  return kNoSlot;
}

// Full single-point look-up (used by the map query kernel).
template <int KIND, int DTYPE>
__device__ __forceinline__ bool lookup(const MapView& m, float x, float y, float z, float& d,
                                       long long& linear) {
  int ix, iy, iz;
  linear = -1;
  d = m.tau;
  if (!voxel_of(m, x, y, z, ix, iy, iz)) return false;
  linear = ((long long)iz * m.ny + iy) * m.nx + ix;
  if constexpr (is_dense(KIND)) {
    d = load_value<DTYPE>(m, dense_index<KIND == kKindDenseTiles>((uint32_t)ix, (uint32_t)iy, (uint32_t)iz,
                                                                  (uint32_t)m.nx, (uint32_t)m.ny, m.tcy, m.tsz));
    return true;
  } else {
    uint32_t key, local, slot;
    brick_key<KIND == kKindBrickGrid>(m, ix, iy, iz, key, local);
    if constexpr (KIND == kKindBrickGrid) {
      slot = __ldg(m.grid + key);
    } else {
      uint32_t h = brick_hash(key, m.hash_shift);
      uint2 e = __ldg(m.table + h);
      slot = e.x == key ? e.y : (e.x == kEmptyKey ? kNoSlot : probe_rest(m, key, h));
    }
    if (slot == kNoSlot) return false;
    if constexpr (KIND == kKindBrickGrid)
      d = load_value<DTYPE>(m, (size_t)(slot | local));  // slot: index of the brick's first value
    else
      d = load_value<DTYPE>(m, (size_t)slot * kBrickVoxels + local);
    return true;
  }
}

#endif  // __CUDACC__

// ---------------------------------------------------------------- launchers
// Packed scan of one sensor update, chunk by chunk (a1), in pairs: a lane
// group of G lanes takes points l, l + G, l + 2G, ... of a chunk, two per
// step of its loop, so pair (s, l) of a chunk holds points
// s 2G + l and s 2G + G + l as XY = (x0, x1, y0, y1) (one float4) in a first
// array and Z = (z0, z1) (one float2) in a second right after it: the lane
// reads its two points with two shared loads and has each coordinate of the
// two in one register pair for the packed FP32x2 instructions. A chunk of cnt
// points holds pairs(cnt) = ceil(cnt / 2G) G pairs (24 bytes each; points past
// cnt are zero) and starts at byte c * full_pairs() * 24. Both reads (nearest
// and trilinear) use it; pair_g = 0 packs one float4 (x, y, z, 0) per point.
struct ScanLayout {
  int chunk;   // points per chunk
  int pair_g;  // G of the pair layout, 0: one float4 per point
  int rings;   // > 0: the scan is `rings` rings of `az` points, ring-major, staged in patches
  int az;      // (source), else in the order given
  // Scan point staged at place j: with rings, patches of 4 rings x 8
  // neighbouring points, patch after patch along the rings, band of 4 rings
  // after band, so that the 32 lanes of a warp take one 4 x 8 patch (the
  // pair partner the next one) and their gathers share more sectors.
  __host__ __device__ int source(int j) const {
    if (rings <= 0) return j;
    const int band = j / (4 * az), t = j - band * 4 * az, u = t & 31;
    return (band * 4 + (u >> 3)) * az + (t >> 5) * 8 + (u & 7);
  }
  __host__ __device__ int pairs(int cnt) const { return (cnt + 2 * pair_g - 1) / (2 * pair_g) * pair_g; }
  __host__ __device__ int full_pairs() const { return pairs(chunk); }
  __host__ __device__ size_t chunk_offset(int c) const {
    return pair_g ? (size_t)c * (size_t)full_pairs() * 24 : (size_t)c * (size_t)chunk * 16;
  }
  __host__ __device__ uint32_t chunk_bytes(int cnt) const {
    return pair_g ? (uint32_t)pairs(cnt) * 24u : (uint32_t)cnt * 16u;
  }
  __host__ __device__ int smem_bytes() const { return pair_g ? full_pairs() * 24 : chunk * 16; }
  __host__ __device__ size_t total_bytes(int N) const {
    const size_t K = ((size_t)N + chunk - 1) / chunk;
    return pair_g ? K * (size_t)full_pairs() * 24 : (size_t)N * 16;
  }
};

struct SensorShape {
  int chunk;      // points per chunk (fixes the summation order)
  int lanes;      // lanes per particle (fixes the summation order)
  int ppi;        // particles per work item
  int unroll;     // points per lane per loop step
  int pipeline;   // 1: next step's index look-ups overlap this step's gathers
  int interp;     // 1: trilinear read (MCL_TRILINEAR)
  int threads;    // threads per CTA
  int grid;       // CTAs (persistent)
  int rings, az;  // scan staged in 4 x 8 patches of `rings` rings of `az` points (0: as given)
};

// Scan layout of a launch shape: pairs of the shape's lane groups (the
// nearest and the trilinear read).
inline ScanLayout scan_layout(const SensorShape& sh) {
  return ScanLayout{sh.chunk, sh.lanes, sh.rings, sh.az};
}

struct SensorArgs {
  MapView map;
  const float4* mats;  // P x 3 rows [R_i0 R_i1 R_i2 t_i]
  const float4* scan;  // packed scan (layout)
  ScanLayout layout;
  float* partial;      // K x P chunk partial sums (chunk-major)
  unsigned* status;
  int P, N, chunk, K, ppi, nblk;
  int sweep;           // particle blocks per sweep (nblk: chunk-major order)
  long long n_items;
  int mode, neglect;
  float vout;          // value read where nothing is stored, in storage units (tau, or 32767 for I16)
  // What the nearest read takes where nothing is stored: vout, or with
  // MCL_NEGLECT_OUTSIDE a value whose term is exactly zero (0 for LOGPROD and
  // score maps, +inf for SUM: exp(-inf) = 0), so that no per-point test of
  // the flag is needed and the sums keep their bits.
  float vnear;
  float cs;            // SUM exponent constant, base 2, in storage units (sum_exponent_constant)
  float store_scale;   // chunk sum -> real units: scale^2 for I16 in LOGPROD (sum of q^2), else 1
  // Dynamic item order: a device counter (zero at launch) hands out the items
  // in order, one at a time per CTA; NULL: static striding over the grid.
  unsigned long long* queue = nullptr;
};

// Pose rows -> [R | t]; with rank, particle p's matrix goes to slot rank[p].
// Batched sensor update: sessions sharing one map and score constants.
struct BatchSession {
  const float4* mats;  // P x 3 rows
  const float4* scan;  // packed scan (the group's layout)
  float* partial;      // K x P chunk sums
  int P, N, nblk, K, sweep;
  int ppi;             // particles per block of this session (its plan may shrink it)
  // this session's map: values and brick index (geometry and score constants
  // are the group's, in BatchArgs::base.map)
  const void* values;
  const uint2* table;
  const uint32_t* grid;
  uint32_t n_slots, hash_mask;
  int hash_shift, max_probe;
};

// ---------------------------------------------------------------- batched side kernels
struct EstPartial;
// One session of a batched step as the side kernels read it (a device table):
// the spatial order, pose rows and scan packing, log-weights, normalisation
// with the optional estimate, and systematic resampling of every session run
// as one launch each, whatever the number of sessions.
// Frame of the sensor kernel's pose rows. Rows [R' | t'] with
// R' = R inv and t' = (t - o) inv - shift, evaluated in FP64 in that order
// (R from the FP64 pose rotation, t, o and inv as FP32 numbers) and rounded
// to FP32 once per entry: R' z + t' is then the scan point's index-rule
// coordinate u along each axis (shift 0: nearest voxel) or f = u - 1/2
// (shift 1/2: trilinear read) directly, with three FP32 fma per axis. The
// identity frame (o = 0, inv = 1, shift = 0) gives the plain [R | t].
struct RowFrame {
  float ox, oy, oz, inv, shift;
};
__host__ __device__ inline RowFrame identity_frame() { return RowFrame{0.f, 0.f, 0.f, 1.f, 0.f}; }
inline RowFrame sensor_frame(const MapView& m, bool trilinear) {
  return RowFrame{m.ox, m.oy, m.oz, m.inv, trilinear ? 0.5f : 0.f};
}

struct SideSeg {
  float* mpart;            // motion update of these P x 6 poses first (NULL: none)
  float mdelta[6], msig[6];
  unsigned long long mseed, mstep;
  const float* particles;  // P x 6
  const float* scan;       // N x 3
  int P, N;
  uint32_t* key;           // spatial order: key, histogram (then cursors), rank; rank NULL: none
  uint32_t* hist;
  int* rank;
  float3 order_o, order_s; // cell-grid origin and scale of the spatial order
  float4* mats;            // P x 3 pose rows
  RowFrame frame;          // their frame
  void* packed;            // packed scan
  ScanLayout layout;
  const float* partial;    // K x P chunk sums
  int K, mode;             // kernel mode as the user gave it (MCL_LOGPROD or MCL_SUM)
  float c, k;              // score constants of the log-weights
  float* logw;
  float* w;                // NULL: log-weights only
  float2* stats;           // normalisation blocks
  int nb;
  float* ostats;           // (M, S)
  EstPartial* est_part;    // NULL: no estimate
  mcl_estimate* est;
  int32_t* idx;            // NULL: no resampling
  const float* pin;        // particles gathered by the draw (NULL: indices only)
  float* pout;
  double* cum;
  double* tile_total;
  long long* tile_last;
  const double* r;         // resampling offset, read when the kernel runs
};

// Blocks of one batched launch: segment s owns blocks [first[s], first[s + 1]).
struct SegBlocks {
  const int* first;  // device, n + 1 entries
  int n;
  int blocks;        // first[n]
};

// Kinds of batched side launch (one block layout each).
enum SideLaunch : int {
  kSideMotion = 0,     // motion update
  kSideOrderZero,      // zero the spatial-order histograms
  kSideOrderKeys,      // bucket keys and counts
  kSideOrderTiles,     // exclusive scan of the counts, tile by tile
  kSideOrderTotals,    // exclusive scan of the tile totals
  kSideOrderScatter,   // ranks
  kSidePosePack,       // pose rows and packed scan
  kSideStats,          // log-weights and block statistics
  kSideNormalise,      // weights (and estimate partials)
  kSideEstimate,       // estimate of each session
  kSideTileScan,       // resampling: prefix tiles
  kSideTileOffsets,    // resampling: tile offsets
  kSideSystematic,     // resampling: the draw
  kSideLaunches
};

// Segment of block b: the last s with first[s] <= b (empty segments skipped).
#ifdef __CUDACC__
__device__ __forceinline__ int seg_of(const int* __restrict__ first, int n, int b) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(first + mid) <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}
#endif
// The spatial order's cell grid of a map: origin and scale (cells per metre).
void order_grid(const MapView& m, float3* o, float3* s);
// Per-file parts of the batched side launches.
int side_blocks_order(int kind, const SideSeg& g);
cudaError_t launch_side_order(int kind, const SideSeg* segs, const SegBlocks& b, cudaStream_t s);
int side_blocks_pose(const SideSeg& g);
cudaError_t launch_side_pose(const SideSeg* segs, const SegBlocks& b, cudaStream_t s);
int side_blocks_normalise(int kind, const SideSeg& g);
cudaError_t launch_side_normalise(int kind, const SideSeg* segs, const SegBlocks& b, cudaStream_t s);
int side_blocks_resample(int kind, const SideSeg& g);
cudaError_t launch_side_resample(int kind, const SideSeg* segs, const SegBlocks& b, cudaStream_t s);
int side_blocks_motion(const SideSeg& g);
cudaError_t launch_side_motion(const SideSeg* segs, const SegBlocks& b, cudaStream_t s);

// Blocks session `g` needs in side launch `kind` (threads per block fixed per kind).
int side_blocks(int kind, const SideSeg& g);
constexpr int kSideThreads = 256;  // of the per-particle side launches
cudaError_t launch_side(int kind, const SideSeg* segs, const SegBlocks& b, cudaStream_t s);

// A run of consecutive items of one session in a batched launch's item order:
// items [begin, next segment's begin) are the session's local items local0, ...
struct ItemSeg {
  long long begin;
  long long local0;
  int session;  // index into BatchArgs::sessions (-1: the closing entry)
  int pad;
};

struct BatchArgs {
  SensorArgs base;                 // map, score constants, chunk, ppi, status
  const BatchSession* sessions;    // device table
  const ItemSeg* segs;             // device, n_segs + 1 entries (the last: begin = n_items)
  int n_segs;
  long long n_items;
};

cudaError_t launch_sensor_batch(int kind, int layout, int dtype, const BatchArgs& b,
                                const SensorShape& sh, cudaStream_t s);
cudaError_t sensor_batch_occupancy(int kind, int layout, int dtype, int mode, const SensorShape& sh,
                                   int* blocks_per_sm);

cudaError_t launch_pose_to_matrix(const float* poses, int P, float4* mats, const int* rank,
                                  cudaStream_t s);

// Spatial processing order (slot rank[p] of particle p), see k_order.cu.
size_t order_hist_bytes();
cudaError_t launch_particle_order(const float* poses, int P, const MapView& m, uint32_t* key,
                                  uint32_t* hist, int* rank, cudaStream_t s);
// Pose matrices in the frame f (as launch_pose_to_matrix for the identity
// frame) and scan packing (N x 3 -> the layout) in one launch.
cudaError_t launch_pose_and_pack(const float* poses, int P, float4* mats, const int* rank,
                                 const RowFrame& f, const float* scan, int N,
                                 const ScanLayout& layout, void* packed, cudaStream_t s);
cudaError_t launch_sensor(int kind, int layout, int dtype, const SensorArgs& a,
                          const SensorShape& sh, cudaStream_t s);
int sensor_smem_bytes(const SensorShape& sh);
cudaError_t sensor_occupancy(int kind, int layout, int dtype, int mode, const SensorShape& sh,
                             int* blocks_per_sm);

// Map upload helper: z layers [z0, z0 + nzs) of an x-fastest dense grid
// (src, nx * ny values per layer) -> their places in the stored grid (dst,
// dense_index).
cudaError_t launch_dense_to_tiles(const void* src, void* dst, int nx, int ny, int z0, int nzs,
                                  uint32_t ntx, uint32_t nty, int elem_bytes, cudaStream_t s);
// Map upload helper: x-fastest bricks (src) -> 4x4x4-block layout (dst).
cudaError_t launch_brick_to_block4(const void* src, void* dst, long long n_bricks, int elem_bytes,
                                   cudaStream_t s);
// Map upload helper: x-fastest bricks (src) at cell coordinates coords
// (device, 3 int32 per brick) -> the cell grid's skewed layout (skew_local).
cudaError_t launch_brick_to_skew(const void* src, void* dst, const int32_t* coords,
                                 long long n_bricks, int elem_bytes, cudaStream_t s);

// Score map values: s = exp(-d^2 / (2 sigma^2)) of n stored values (src of
// src_dtype, int16 scaled by tau / 32767), FP64, rounded once to dst_dtype
// (MCL_F16 or MCL_F32).
cudaError_t launch_score_values(const void* src, int src_dtype, long long n, double tau,
                                double sigma, void* dst, int dst_dtype, cudaStream_t s);

// Finishing pass: L_p from the chunk partials, then block max / sum-exp.
// With rank, particle p's chunk sums sit in slot rank[p] of partial.
cudaError_t launch_finish_and_normalise(const float* partial, const int* rank, int P, int K,
                                        int mode, float c, float k, float* logw, float* w,
                                        float2* block_stats, int nblocks, float* out_stats,
                                        cudaStream_t s);
cudaError_t launch_normalise(const float* logw, int P, float* w, float2* block_stats, int nblocks,
                             float* out_stats, cudaStream_t s);
int normalise_blocks(int P);

// Pose estimate (k_normalise.cu): per-block FP64 sums of the weighted pose
// terms and the block's largest weight, then one block that combines them.
constexpr int kEstSums = 18;  // W, sum w^2, 6 x sum w s_k, 10 x sum w q_i q_j (i <= j)
struct EstPartial {
  double v[kEstSums];
  float best_w;
  int best_p;
};
// Normalisation from block statistics already computed for logw (by
// launch_finish_and_normalise); with est, the estimate of the weighted
// particles (P x 6, original order) is accumulated in the same pass.
cudaError_t launch_normalise_from_stats(const float* logw, int P, float* w,
                                        const float2* block_stats, int nblocks, float* out_stats,
                                        const float* particles, EstPartial* part,
                                        mcl_estimate* est, cudaStream_t s);
// Estimate from given weights (same blocks and order as the fused pass).
cudaError_t launch_pose_estimate(const float* particles, const float* w, int P, EstPartial* part,
                                 mcl_estimate* est, cudaStream_t s);

cudaError_t launch_map_lookup(int kind, int dtype, const MapView& m, const float* pts, int N,
                              long long* out_index, float* out_value, cudaStream_t s);

// Resampling scratch: C (P doubles), per-tile totals and last positive index.
int resample_tiles(int P);
int resample_kernels(int P);  // launches of one resampling call
// r_dev (device, optional) overrides r: the offset is read when the kernel runs.
cudaError_t launch_resample(const float* w, int P, double r, int32_t* idx,
                            const float* particles_in, float* particles_out, double* cum,
                            double* tile_total, long long* tile_last, cudaStream_t s,
                            const double* r_dev = nullptr);

// Resampling with scratch in a static device array (no allocation), for at
// most kStaticMaxParticles particles.
constexpr int kStaticMaxParticles = 1 << 20;
constexpr int kMaxDevices = 64;
cudaError_t launch_resample_static(const float* w, int P, double r, int32_t* idx,
                                   const float* particles_in, float* particles_out, cudaStream_t s);

// Inputs of one filter step read from device memory when the kernels run,
// so that a captured graph replays with each step's values.
struct StepIn {
  float delta[6];           // odometry increment
  int motion;               // 0: no motion update this step
  int pad;
  unsigned long long step;  // motion-noise counter
  double r;                 // resampling offset
};

// With in, delta and step come from in (read at run time) and the update is
// skipped when in->motion is 0.
cudaError_t launch_motion(float* particles, int P, const float delta[6], const float sigma[6],
                          uint64_t seed, uint64_t step, cudaStream_t s,
                          const StepIn* in = nullptr);

// One CTA waits on a barrier phase nothing completes (k_diag.cu).
cudaError_t launch_wait_selftest(unsigned* status, unsigned long long* waited_ns, cudaStream_t s);

cudaError_t launch_gather_bench(const void* buf, long long n_elems, int elem_bytes, int blocks,
                                int iters, unsigned long long seed, float* sink, cudaStream_t s);

}  // namespace mcl
