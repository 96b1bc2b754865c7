// Per-particle pose matrices, scan packing and the map query kernel.
#include <algorithm>

#include "mcl_internal.h"

namespace mcl {
namespace {

// [R | t] rows from (x, y, z, roll, pitch, yaw) (Sec. III, Eq. 2). The
// rotation R = Rz(yaw) Ry(pitch) Rx(roll) is evaluated in FP64 in a fixed
// order with every product and sum rounded on its own (no contraction), and
// each entry is rounded to FP32 once:
//   a = cy*sp, b = sy*sp
//   [ cy*cp   a*sr - sy*cr   a*cr + sy*sr ]
//   [ sy*cp   b*sr + cy*cr   b*cr - cy*sr ]
//   [ -sp     cp*sr          cp*cr        ]
// In the frame f (RowFrame) each entry is then R_ij * inv and each
// translation (t_i - o_i) * inv - shift, still in FP64, before the one
// rounding; the identity frame changes no bit.
__device__ __forceinline__ float frame_t(float t, float o, double inv, double shift) {
  return __double2float_rn(__dsub_rn(__dmul_rn(__dsub_rn((double)t, (double)o), inv), shift));
}

__device__ __forceinline__ void pose_to_matrix(const float* __restrict__ poses, int p,
                                               float4* __restrict__ mats, const int* __restrict__ rank,
                                               const RowFrame& f) {
  const float* s = poses + 6 * (size_t)p;
  const float x = s[0], y = s[1], z = s[2];
  const double roll = (double)s[3], pitch = (double)s[4], yaw = (double)s[5];
  double cr, sr, cp, sp, cy, sy;  // one shared range reduction per angle
  sincos(roll, &sr, &cr);
  sincos(pitch, &sp, &cp);
  sincos(yaw, &sy, &cy);
  const double a = __dmul_rn(cy, sp), b = __dmul_rn(sy, sp);
  const double r00 = __dmul_rn(cy, cp);
  const double r01 = __dsub_rn(__dmul_rn(a, sr), __dmul_rn(sy, cr));
  const double r02 = __dadd_rn(__dmul_rn(a, cr), __dmul_rn(sy, sr));
  const double r10 = __dmul_rn(sy, cp);
  const double r11 = __dadd_rn(__dmul_rn(b, sr), __dmul_rn(cy, cr));
  const double r12 = __dsub_rn(__dmul_rn(b, cr), __dmul_rn(cy, sr));
  const double r20 = -sp;
  const double r21 = __dmul_rn(cp, sr);
  const double r22 = __dmul_rn(cp, cr);
  const double inv = (double)f.inv, sh = (double)f.shift;
  auto e = [inv](double r) { return __double2float_rn(__dmul_rn(r, inv)); };
  float4* o = mats + 3 * (size_t)(rank ? rank[p] : p);
  o[0] = make_float4(e(r00), e(r01), e(r02), frame_t(x, f.ox, inv, sh));
  o[1] = make_float4(e(r10), e(r11), e(r12), frame_t(y, f.oy, inv, sh));
  o[2] = make_float4(e(r20), e(r21), e(r22), frame_t(z, f.oz, inv, sh));
}

// N x 3 scan rows -> N float4 (x, y, z, 0): 16-byte records that a bulk copy
// can move and a lane can read with one 128-bit shared-memory load.
__device__ __forceinline__ void scan_pack(const float* __restrict__ scan, int j, const ScanLayout& L,
                                          float4* __restrict__ packed) {
  const float* q = scan + 3 * (size_t)L.source(j);
  packed[j] = make_float4(q[0], q[1], q[2], 0.f);
}

__global__ void k_pose_to_matrix(const float* __restrict__ poses, int P, float4* __restrict__ mats,
                                 const int* __restrict__ rank) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < P) pose_to_matrix(poses, p, mats, rank, identity_frame());
}

// Pair t of the pair layout (ScanLayout): chunk c = t / full_pairs, pair
// (s, l) = divmod(t % full_pairs, G) of points s 2G + l and s 2G + G + l of
// the chunk (zeros past its end).
__device__ __forceinline__ void scan_pack_pair(const float* __restrict__ scan, int N,
                                               const ScanLayout L, int t,
                                               unsigned char* __restrict__ packed) {
  const int fp = L.full_pairs();
  const int c = t / fp, pi = t - c * fp;
  const int cnt = min(L.chunk, N - c * L.chunk);
  const int np = L.pairs(cnt);
  if (pi >= np) return;  // beyond this (last) chunk's pairs
  const int G = L.pair_g;
  const int s = pi / G, l = pi - s * G;
  const int i0 = s * 2 * G + l, i1 = i0 + G;
  float a[3] = {0.f, 0.f, 0.f}, b[3] = {0.f, 0.f, 0.f};
  if (i0 < cnt) {
    const float* q = scan + 3 * (size_t)L.source(c * L.chunk + i0);
    a[0] = q[0]; a[1] = q[1]; a[2] = q[2];
  }
  if (i1 < cnt) {
    const float* q = scan + 3 * (size_t)L.source(c * L.chunk + i1);
    b[0] = q[0]; b[1] = q[1]; b[2] = q[2];
  }
  unsigned char* base = packed + L.chunk_offset(c);
  reinterpret_cast<float4*>(base)[pi] = make_float4(a[0], b[0], a[1], b[1]);
  reinterpret_cast<float2*>(base + (size_t)np * 16)[pi] = make_float2(a[2], b[2]);
}

// Pose matrices and scan packing of one sensor update in one launch: blocks
// [0, pose_blocks) take particles, the rest take scan points or pairs (the
// two are independent; one launch instead of two matters for small updates,
// where each launch costs about as much as its work).
__global__ void k_pose_and_pack(const float* __restrict__ poses, int P, float4* __restrict__ mats,
                                const int* __restrict__ rank, const RowFrame f, int pose_blocks,
                                const float* __restrict__ scan, int N, const ScanLayout L,
                                void* __restrict__ packed) {
  if ((int)blockIdx.x < pose_blocks) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < P) pose_to_matrix(poses, p, mats, rank, f);
  } else {
    const int j = (blockIdx.x - pose_blocks) * blockDim.x + threadIdx.x;
    if (L.pair_g == 0) {
      if (j < N) scan_pack(scan, j, L, static_cast<float4*>(packed));
    } else {
      const int K = (N + L.chunk - 1) / L.chunk;
      if (j < K * L.full_pairs()) scan_pack_pair(scan, N, L, j, static_cast<unsigned char*>(packed));
    }
  }
}

// Scan units of the packing: pairs of the pair layout, else points.
__host__ __device__ inline long long pack_units(int N, const ScanLayout& L) {
  return L.pair_g ? (long long)((N + L.chunk - 1) / L.chunk) * L.full_pairs() : (long long)N;
}

// Batched form: per session, pose blocks then packing blocks of kSideThreads.
__global__ void __launch_bounds__(kSideThreads) k_pose_and_pack_b(const SideSeg* __restrict__ segs, SegBlocks b) {
  const int s = seg_of(b.first, b.n, blockIdx.x);
  const SideSeg& g = segs[s];
  const int j = blockIdx.x - __ldg(b.first + s);
  const int pb = (g.P + kSideThreads - 1) / kSideThreads;
  if (j < pb) {
    const int p = j * kSideThreads + threadIdx.x;
    if (p < g.P) pose_to_matrix(g.particles, p, g.mats, g.rank, g.frame);
  } else {
    const int t = (j - pb) * kSideThreads + threadIdx.x;
    const ScanLayout L = g.layout;
    if (t < pack_units(g.N, L)) {
      if (L.pair_g == 0) scan_pack(g.scan, t, L, static_cast<float4*>(g.packed));
      else scan_pack_pair(g.scan, g.N, L, t, static_cast<unsigned char*>(g.packed));
    }
  }
}

template <int KIND, int DTYPE>
__global__ void k_map_lookup(const MapView m, const float* __restrict__ pts, int N,
                             long long* __restrict__ out_index, float* __restrict__ out_value) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  const float* q = pts + 3 * (size_t)j;
  float d;
  long long linear;
  lookup<KIND, DTYPE>(m, q[0], q[1], q[2], d, linear);
  if (out_index) out_index[j] = linear;
  if (out_value) out_value[j] = d;
}

template <typename T>
__global__ void k_brick_to_block4(const T* __restrict__ src, T* __restrict__ dst, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const long long b = i >> 12;
  const uint32_t l = (uint32_t)i & 4095u;
  dst[(b << 12) + block4_local(l & 15u, (l >> 4) & 15u, l >> 8)] = src[i];
}

// Value l of brick b (x-fastest) moves to skew_local of its voxel: local
// (lx, ly, lz) plus 16 times the brick's cell coordinates.
template <typename T>
__global__ void k_brick_to_skew(const T* __restrict__ src, T* __restrict__ dst,
                                const int32_t* __restrict__ coords, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const long long b = i >> 12;
  const uint32_t l = (uint32_t)i & 4095u;
  const uint32_t ix = (uint32_t)coords[3 * b] * 16u + (l & 15u);
  const uint32_t iy = (uint32_t)coords[3 * b + 1] * 16u + ((l >> 4) & 15u);
  const uint32_t iz = (uint32_t)coords[3 * b + 2] * 16u + (l >> 8);
  dst[(b << 12) + skew_local(ix, iy, iz)] = src[i];
}

// Voxel i of layers [z0, z0 + nzs) (x-fastest in src) to dense_index.
template <typename T>
__global__ void k_dense_to_tiles(const T* __restrict__ src, T* __restrict__ dst, int nx, int ny,
                                 int z0, long long n, uint32_t ntx, uint32_t nty) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const long long layer = (long long)nx * ny;
  const uint32_t iz = (uint32_t)(z0 + i / layer);
  const uint32_t r = (uint32_t)(i % layer);
  const uint32_t iy = r / (uint32_t)nx, ix = r - iy * (uint32_t)nx;
  dst[dense_index<true>(ix, iy, iz, (uint32_t)nx, (uint32_t)ny, 8u * ntx - 8u, 32u * ntx * nty)] = src[i];
}

inline int blocks_for(long long n, int t) { return (int)((n + t - 1) / t); }

// Score map values (Sec. III: the exponential of Eq. 3 evaluated once per map
// entry): s = exp(-d^2 / (2 sigma^2)) in FP64, rounded once to the output type.
template <int SRC>
__global__ void k_score_values(const void* __restrict__ src, long long n, double tau, double sigma,
                               void* __restrict__ dst, int dst_f16) {
  const double c = 2.0 * sigma * sigma;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double d;
    if constexpr (SRC == MCL_F32) d = (double)static_cast<const float*>(src)[i];
    else if constexpr (SRC == MCL_F16) d = (double)__half2float(static_cast<const __half*>(src)[i]);
    else d = (double)static_cast<const short*>(src)[i] * (tau / 32767.0);
    const double e = exp(-(d * d) / c);
    if (dst_f16) static_cast<__half*>(dst)[i] = __double2half(e);  // round to nearest even
    else static_cast<float*>(dst)[i] = __double2float_rn(e);
  }
}

}  // namespace

// FP64 trigonometry per particle: small sets use small blocks so that they
// spread over many SMs instead of loading a few (FP64 issue per SM is slow)
inline int pose_threads(int P) {
  int threads = 256;
  while (threads > 32 && (P + threads - 1) / threads < 2 * 152) threads >>= 1;
  return threads;
}

cudaError_t launch_pose_to_matrix(const float* poses, int P, float4* mats, const int* rank,
                                  cudaStream_t s) {
  const int threads = pose_threads(P);
  k_pose_to_matrix<<<blocks_for(P, threads), threads, 0, s>>>(poses, P, mats, rank);
  return cudaGetLastError();
}

cudaError_t launch_pose_and_pack(const float* poses, int P, float4* mats, const int* rank,
                                 const RowFrame& f, const float* scan, int N,
                                 const ScanLayout& layout, void* packed, cudaStream_t s) {
  const int threads = pose_threads(P);
  const long long units = pack_units(N, layout);
  const int pb = blocks_for(P, threads), sb = blocks_for(units, threads);
  k_pose_and_pack<<<pb + sb, threads, 0, s>>>(poses, P, mats, rank, f, pb, scan, N, layout, packed);
  return cudaGetLastError();
}

int side_blocks_pose(const SideSeg& g) {
  return blocks_for(g.P, kSideThreads) + blocks_for(pack_units(g.N, g.layout), kSideThreads);
}

cudaError_t launch_side_pose(const SideSeg* segs, const SegBlocks& b, cudaStream_t s) {
  if (b.blocks == 0) return cudaSuccess;
  k_pose_and_pack_b<<<b.blocks, kSideThreads, 0, s>>>(segs, b);
  return cudaGetLastError();
}

cudaError_t launch_brick_to_block4(const void* src, void* dst, long long n_bricks, int elem_bytes,
                                   cudaStream_t s) {
  const long long n = n_bricks * kBrickVoxels;
  if (n <= 0) return cudaSuccess;
  if (elem_bytes == 2)
    k_brick_to_block4<<<blocks_for(n, 256), 256, 0, s>>>((const short*)src, (short*)dst, n);
  else
    k_brick_to_block4<<<blocks_for(n, 256), 256, 0, s>>>((const float*)src, (float*)dst, n);
  return cudaGetLastError();
}

cudaError_t launch_dense_to_tiles(const void* src, void* dst, int nx, int ny, int z0, int nzs,
                                  uint32_t ntx, uint32_t nty, int elem_bytes, cudaStream_t s) {
  const long long n = (long long)nx * ny * nzs;
  if (n <= 0) return cudaSuccess;
  if (elem_bytes == 2)
    k_dense_to_tiles<<<blocks_for(n, 256), 256, 0, s>>>((const short*)src, (short*)dst, nx, ny, z0, n,
                                                         ntx, nty);
  else
    k_dense_to_tiles<<<blocks_for(n, 256), 256, 0, s>>>((const float*)src, (float*)dst, nx, ny, z0, n,
                                                         ntx, nty);
  return cudaGetLastError();
}

cudaError_t launch_brick_to_skew(const void* src, void* dst, const int32_t* coords,
                                 long long n_bricks, int elem_bytes, cudaStream_t s) {
  const long long n = n_bricks * kBrickVoxels;
  if (n <= 0) return cudaSuccess;
  if (elem_bytes == 2)
    k_brick_to_skew<<<blocks_for(n, 256), 256, 0, s>>>((const short*)src, (short*)dst, coords, n);
  else
    k_brick_to_skew<<<blocks_for(n, 256), 256, 0, s>>>((const float*)src, (float*)dst, coords, n);
  return cudaGetLastError();
}

cudaError_t launch_score_values(const void* src, int src_dtype, long long n, double tau,
                                double sigma, void* dst, int dst_dtype, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int g = (int)std::min<long long>(blocks_for(n, 256), 152LL * 64);
  const int f16 = dst_dtype == MCL_F16;
  if (src_dtype == MCL_F32) k_score_values<MCL_F32><<<g, 256, 0, s>>>(src, n, tau, sigma, dst, f16);
  else if (src_dtype == MCL_F16) k_score_values<MCL_F16><<<g, 256, 0, s>>>(src, n, tau, sigma, dst, f16);
  else k_score_values<MCL_I16><<<g, 256, 0, s>>>(src, n, tau, sigma, dst, f16);
  return cudaGetLastError();
}

cudaError_t launch_map_lookup(int kind, int dtype, const MapView& m, const float* pts, int N,
                              long long* out_index, float* out_value, cudaStream_t s) {
  const int g = blocks_for(N, 256);
#define MCL_LOOKUP_CASE(K, D) \
  if (kind == K && dtype == D) { k_map_lookup<K, D><<<g, 256, 0, s>>>(m, pts, N, out_index, out_value); return cudaGetLastError(); }
  MCL_LOOKUP_CASE(MCL_MAP_DENSE, MCL_F32)
  MCL_LOOKUP_CASE(MCL_MAP_DENSE, MCL_F16)
  MCL_LOOKUP_CASE(MCL_MAP_DENSE, MCL_I16)
  MCL_LOOKUP_CASE(kKindDenseTiles, MCL_F32)
  MCL_LOOKUP_CASE(kKindDenseTiles, MCL_F16)
  MCL_LOOKUP_CASE(kKindDenseTiles, MCL_I16)
  MCL_LOOKUP_CASE(MCL_MAP_BRICK, MCL_F32)
  MCL_LOOKUP_CASE(MCL_MAP_BRICK, MCL_F16)
  MCL_LOOKUP_CASE(MCL_MAP_BRICK, MCL_I16)
  MCL_LOOKUP_CASE(kKindBrickGrid, MCL_F32)
  MCL_LOOKUP_CASE(kKindBrickGrid, MCL_F16)
  MCL_LOOKUP_CASE(kKindBrickGrid, MCL_I16)
#undef MCL_LOOKUP_CASE
  return cudaErrorInvalidValue;
}

}  // namespace mcl
