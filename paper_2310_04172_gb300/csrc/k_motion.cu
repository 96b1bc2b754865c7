// Motion update (Sec. III: the motion model is applied to each particle; the
// odometry comes from dead reckoning or an IMU, Sec. IV). The paper does not
// specify the model; this library applies a body-frame increment with
// per-component Gaussian noise:
//   u = delta + sigma * n,   t' = t + R(s) u_t,   R' = R(s) R(u_r),
// with n six standard normals from Philox4x32-10 (Salmon, Moraes, Dror,
// Shaw, SC'11; counter (b, particle, step_lo, step_hi), key = seed) and the
// Box-Muller transform, all in FP64, the result rounded to FP32.
#include "mcl_internal.h"

namespace mcl {
namespace {

// Up to this many particles the six-warp kernel: 6 warps per 32 particles
// fill at most 960 warps, about the GPU's 608 sub-partitions and a half.
constexpr int kMotionSmallMax = 5120;

struct MotionArgs {
  float delta[6];
  float sigma[6];
};

// Philox4x32 bijection, 10 rounds: per round the two multipliers act on
// counter words 0 and 2, high halves are mixed into the other words with the
// round key, and the key advances by the Weyl increments.
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
    const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

// The steps of one particle's update, shared by both kernels below so that
// they give the same bits. Every FP64 operation is written out (no
// contraction), in the oracle's order.

// Normals n[2b], n[2b+1] of particle i: Philox block b, Box-Muller.
__device__ __forceinline__ void normal_pair(uint32_t b, int i, uint64_t step, uint64_t seed,
                                            double& n0, double& n1) {
  uint32_t c[4] = {b, (uint32_t)i, (uint32_t)step, (uint32_t)(step >> 32)};
  philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  const uint64_t hi = ((((uint64_t)c[0]) << 32) | c[1]) >> 11;
  const uint64_t lo = ((((uint64_t)c[2]) << 32) | c[3]) >> 11;
  const double u1 = __dmul_rn(__dadd_rn((double)hi, 0.5), 0x1.0p-53);
  const double u2 = __dmul_rn((double)lo, 0x1.0p-53);
  const double rho = sqrt(__dmul_rn(-2.0, log(u1)));
  double sn, cs;
  sincos(__dmul_rn(6.283185307179586, u2), &sn, &cs);
  n0 = __dmul_rn(rho, cs);
  n1 = __dmul_rn(rho, sn);
}

// Rotation Rz(yaw) Ry(pitch) Rx(roll) (row-major 3 x 3) from the sines and
// cosines of the three angles.
__device__ __forceinline__ void rpy_from(double sr, double cr, double sp, double cp, double sy,
                                         double cy, double R[9]) {
  const double a = __dmul_rn(cy, sp), b = __dmul_rn(sy, sp);
  R[0] = __dmul_rn(cy, cp);
  R[1] = __dsub_rn(__dmul_rn(a, sr), __dmul_rn(sy, cr));
  R[2] = __dadd_rn(__dmul_rn(a, cr), __dmul_rn(sy, sr));
  R[3] = __dmul_rn(sy, cp);
  R[4] = __dadd_rn(__dmul_rn(b, sr), __dmul_rn(cy, cr));
  R[5] = __dsub_rn(__dmul_rn(b, cr), __dmul_rn(cy, sr));
  R[6] = -sp;
  R[7] = __dmul_rn(cp, sr);
  R[8] = __dmul_rn(cp, cr);
}

// x0 y0 + x1 y1 + x2 y2, left to right, each operation rounded.
__device__ __forceinline__ double dot3(double x0, double x1, double x2, double y0, double y1,
                                       double y2) {
  return __dadd_rn(__dadd_rn(__dmul_rn(x0, y0), __dmul_rn(x1, y1)), __dmul_rn(x2, y2));
}

// t' = t + A u_t and R' = A B.
__device__ __forceinline__ void compose(const double A[9], const double B[9], const float* s,
                                        const double u[3], double t[3], double Rn[9]) {
#pragma unroll
  for (int r = 0; r < 3; ++r) t[r] = __dadd_rn((double)s[r], dot3(A[3 * r], A[3 * r + 1], A[3 * r + 2], u[0], u[1], u[2]));
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      Rn[3 * r + c] = dot3(A[3 * r], A[3 * r + 1], A[3 * r + 2], B[c], B[3 + c], B[6 + c]);
}

// ZYX Euler angles of R' (yaw wrapped into [-pi, pi)): angle k of 0, 1, 2.
__device__ __forceinline__ double euler_angle(const double Rn[9], int k) {
  if (k == 0) return atan2(Rn[7], Rn[8]);
  if (k == 1) return asin(fmin(1.0, fmax(-1.0, -Rn[6])));
  const double yaw = atan2(Rn[3], Rn[0]);
  return yaw >= 3.141592653589793 ? -3.141592653589793 : yaw;
}

// One thread per particle.
// Motion update of particle i (one thread).
__device__ __forceinline__ void motion_one(float* __restrict__ poses, int i, const MotionArgs& a,
                                           uint64_t seed, uint64_t step) {
  double n[6];
#pragma unroll
  for (uint32_t b = 0; b < 3; ++b) normal_pair(b, i, step, seed, n[2 * b], n[2 * b + 1]);
  double u[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) u[k] = __dadd_rn((double)a.delta[k], __dmul_rn((double)a.sigma[k], n[k]));
  float* s = poses + 6 * (size_t)i;
  double sc[6][2];  // sin, cos of the pose angles (0-2) and of the rotation increment (3-5)
#pragma unroll
  for (int k = 0; k < 3; ++k) sincos((double)s[3 + k], &sc[k][0], &sc[k][1]);
#pragma unroll
  for (int k = 0; k < 3; ++k) sincos(u[3 + k], &sc[3 + k][0], &sc[3 + k][1]);
  double A[9], B[9], t[3], Rn[9];
  rpy_from(sc[0][0], sc[0][1], sc[1][0], sc[1][1], sc[2][0], sc[2][1], A);
  rpy_from(sc[3][0], sc[3][1], sc[4][0], sc[4][1], sc[5][0], sc[5][1], B);
  compose(A, B, s, u, t, Rn);
  double ang[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) ang[k] = euler_angle(Rn, k);
#pragma unroll
  for (int k = 0; k < 3; ++k) s[k] = (float)t[k];
#pragma unroll
  for (int k = 0; k < 3; ++k) s[3 + k] = (float)ang[k];
}

__global__ void k_motion(float* __restrict__ poses, int P, MotionArgs a, uint64_t seed,
                         uint64_t step, const StepIn* __restrict__ in) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  if (in) {
    if (!in->motion) return;
    step = in->step;
#pragma unroll
    for (int k = 0; k < 6; ++k) a.delta[k] = in->delta[k];
  }
  motion_one(poses, i, a, seed, step);
}

// Batched form: every session with a motion update (SideSeg::mpart), one
// thread per particle, the same arithmetic as k_motion.
__global__ void __launch_bounds__(kSideThreads) k_motion_b(const SideSeg* __restrict__ segs, SegBlocks b) {
  const int s = seg_of(b.first, b.n, blockIdx.x);
  const SideSeg& g = segs[s];
  const int i = (blockIdx.x - __ldg(b.first + s)) * kSideThreads + threadIdx.x;
  if (i >= g.P) return;
  MotionArgs a;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    a.delta[k] = g.mdelta[k];
    a.sigma[k] = g.msig[k];
  }
  motion_one(g.mpart, i, a, g.mseed, g.mstep);
}

// Small sets: FP64 issue is slow on this part (a warp instruction holds its
// SM sub-partition's FP64 pipe for many cycles whatever the number of active
// lanes), so one warp per 32 particles is bound by the length of the
// per-particle FP64 stream. Here six warps share 32 particles (lane l of
// every warp serves particle 32 b + l) and run its independent pieces side by
// side: the three normal pairs and the three sines/cosines of the pose
// angles; then the sines/cosines of the three rotation increments; then the
// composition (one warp); then the three angles. Same helpers, same bits as
// k_motion.
constexpr int kSmallWarps = 6;

__global__ void __launch_bounds__(32 * kSmallWarps) k_motion_small(float* __restrict__ poses, int P,
                                                                   MotionArgs a, uint64_t seed,
                                                                   uint64_t step,
                                                                   const StepIn* __restrict__ in) {
  __shared__ double sh_n[6][32];      // normals
  __shared__ double sh_sc[6][2][32];  // sin, cos: pose angles 0-2, increments 3-5
  __shared__ double sh_r[9][32];      // R'
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * 32 + lane;
  const bool live = i < P;
  if (in) {
    if (!in->motion) return;  // uniform over the grid
    step = in->step;
#pragma unroll
    for (int k = 0; k < 6; ++k) a.delta[k] = in->delta[k];
  }
  float* s = poses + 6 * (size_t)(live ? i : 0);
  if (live) {
    if (warp < 3) {
      normal_pair((uint32_t)warp, i, step, seed, sh_n[2 * warp][lane], sh_n[2 * warp + 1][lane]);
    } else {
      const int k = warp - 3;
      sincos((double)s[3 + k], &sh_sc[k][0][lane], &sh_sc[k][1][lane]);
    }
  }
  __syncthreads();
  if (live && warp < 3) {
    const int k = 3 + warp;
    const double uk = __dadd_rn((double)a.delta[k], __dmul_rn((double)a.sigma[k], sh_n[k][lane]));
    sincos(uk, &sh_sc[k][0][lane], &sh_sc[k][1][lane]);
  }
  __syncthreads();
  if (live && warp == 0) {
    double u[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) u[k] = __dadd_rn((double)a.delta[k], __dmul_rn((double)a.sigma[k], sh_n[k][lane]));
    double A[9], B[9], t[3], Rn[9];
    rpy_from(sh_sc[0][0][lane], sh_sc[0][1][lane], sh_sc[1][0][lane], sh_sc[1][1][lane],
             sh_sc[2][0][lane], sh_sc[2][1][lane], A);
    rpy_from(sh_sc[3][0][lane], sh_sc[3][1][lane], sh_sc[4][0][lane], sh_sc[4][1][lane],
             sh_sc[5][0][lane], sh_sc[5][1][lane], B);
    compose(A, B, s, u, t, Rn);
#pragma unroll
    for (int k = 0; k < 9; ++k) sh_r[k][lane] = Rn[k];
#pragma unroll
    for (int k = 0; k < 3; ++k) s[k] = (float)t[k];
  }
  __syncthreads();
  if (live && warp < 3) {
    double Rn[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) Rn[k] = sh_r[k][lane];
    s[3 + warp] = (float)euler_angle(Rn, warp);
  }
}

}  // namespace

cudaError_t launch_motion(float* particles, int P, const float delta[6], const float sigma[6],
                          uint64_t seed, uint64_t step, cudaStream_t s, const StepIn* in) {
  MotionArgs a;
  for (int k = 0; k < 6; ++k) {
    a.delta[k] = delta ? delta[k] : 0.f;
    a.sigma[k] = sigma[k];
  }
  if (P <= kMotionSmallMax) {
    k_motion_small<<<(P + 31) / 32, 32 * kSmallWarps, 0, s>>>(particles, P, a, seed, step, in);
    return cudaGetLastError();
  }
  // FP64-heavy per particle: mid-size sets use small blocks so that they
  // still spread over many SMs (one block of 256 would load a single SM).
  int threads = 256;
  while (threads > 32 && (P + threads - 1) / threads < 2 * 152) threads >>= 1;
  k_motion<<<(P + threads - 1) / threads, threads, 0, s>>>(particles, P, a, seed, step, in);
  return cudaGetLastError();
}

int side_blocks_motion(const SideSeg& g) { return g.mpart ? (g.P + kSideThreads - 1) / kSideThreads : 0; }

cudaError_t launch_side_motion(const SideSeg* segs, const SegBlocks& b, cudaStream_t s) {
  if (b.blocks == 0) return cudaSuccess;
  k_motion_b<<<b.blocks, kSideThreads, 0, s>>>(segs, b);
  return cudaGetLastError();
}

}  // namespace mcl
