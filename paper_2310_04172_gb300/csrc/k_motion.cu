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

// Rotation Rz(yaw) Ry(pitch) Rx(roll) in FP64 (row-major 3 x 3).
__device__ __forceinline__ void rpy(double roll, double pitch, double yaw, double R[9]) {
  double cr, sr, cp, sp, cy, sy;  // one shared range reduction per angle
  sincos(roll, &sr, &cr);
  sincos(pitch, &sp, &cp);
  sincos(yaw, &sy, &cy);
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
  double n[6];
#pragma unroll
  for (uint32_t b = 0; b < 3; ++b) {
    uint32_t c[4] = {b, (uint32_t)i, (uint32_t)step, (uint32_t)(step >> 32)};
    philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    const uint64_t hi = ((((uint64_t)c[0]) << 32) | c[1]) >> 11;
    const uint64_t lo = ((((uint64_t)c[2]) << 32) | c[3]) >> 11;
    const double u1 = __dmul_rn(__dadd_rn((double)hi, 0.5), 0x1.0p-53);
    const double u2 = __dmul_rn((double)lo, 0x1.0p-53);
    const double rho = sqrt(__dmul_rn(-2.0, log(u1)));
    double sn, cs;
    sincos(__dmul_rn(6.283185307179586, u2), &sn, &cs);
    n[2 * b] = __dmul_rn(rho, cs);
    n[2 * b + 1] = __dmul_rn(rho, sn);
  }
  double u[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) u[k] = __dadd_rn((double)a.delta[k], __dmul_rn((double)a.sigma[k], n[k]));
  float* s = poses + 6 * (size_t)i;
  double A[9], B[9], Rn[9];
  rpy((double)s[3], (double)s[4], (double)s[5], A);
  rpy(u[3], u[4], u[5], B);
  double t[3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
    t[r] = (double)s[r] + (A[3 * r] * u[0] + A[3 * r + 1] * u[1] + A[3 * r + 2] * u[2]);
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c2 = 0; c2 < 3; ++c2)
      Rn[3 * r + c2] = A[3 * r] * B[c2] + A[3 * r + 1] * B[3 + c2] + A[3 * r + 2] * B[6 + c2];
  const double sp = fmin(1.0, fmax(-1.0, -Rn[6]));
  const double roll = atan2(Rn[7], Rn[8]), pitch = asin(sp);
  double yaw = atan2(Rn[3], Rn[0]);
  if (yaw >= 3.141592653589793) yaw = -3.141592653589793;
  s[0] = (float)t[0];
  s[1] = (float)t[1];
  s[2] = (float)t[2];
  s[3] = (float)roll;
  s[4] = (float)pitch;
  s[5] = (float)yaw;
}

}  // namespace

cudaError_t launch_motion(float* particles, int P, const float delta[6], const float sigma[6],
                          uint64_t seed, uint64_t step, cudaStream_t s, const StepIn* in) {
  MotionArgs a;
  for (int k = 0; k < 6; ++k) {
    a.delta[k] = delta ? delta[k] : 0.f;
    a.sigma[k] = sigma[k];
  }
  // FP64-heavy per particle: small sets use small blocks so that they still
  // spread over many SMs (one block of 256 would load a single SM).
  int threads = 256;
  while (threads > 32 && (P + threads - 1) / threads < 2 * 152) threads >>= 1;
  k_motion<<<(P + threads - 1) / threads, threads, 0, s>>>(particles, P, a, seed, step, in);
  return cudaGetLastError();
}

}  // namespace mcl
