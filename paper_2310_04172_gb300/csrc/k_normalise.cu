// Particle log-weights from chunk partials, and normalisation (Sec. V-A: the
// weights are summed for normalisation; Sec. V-B: a GPU reduction).
//
// The paper reduces with repeated pairwise-halving launches. Here two
// launches suffice: each of up to 1024 blocks of 256 threads owns a contiguous particle range
// and writes its (max, sum exp(L - max)); every block of the second launch
// combines all block pairs in the same fixed order (so all blocks agree on M
// and S bit for bit) and writes w = exp(L - M) / S for its range. FP32
// throughout; max-subtracted so nothing overflows.
#include <cfloat>
#include <climits>

#include "mcl_internal.h"

namespace mcl {
namespace {

// 256 threads per block: small particle sets still spread over several SMs,
// which matters for the FP64 sums of the estimate (FP64 throughput per SM is
// low on this part).
constexpr int kT = 256;

__device__ __forceinline__ float block_max(float v, float* sh) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, off));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  v = lane < (int)(blockDim.x >> 5) ? sh[lane] : -INFINITY;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, off));
  return v;
}

// Fixed pairwise tree: xor shuffles inside each warp, then over warp totals.
__device__ __forceinline__ float block_sum(float v, float* sh) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = __fadd_rn(v, __shfl_xor_sync(0xffffffffu, v, off));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  v = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.f;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = __fadd_rn(v, __shfl_xor_sync(0xffffffffu, v, off));
  return v;
}

// One block per contiguous particle range. With `partial`, L_p is first
// assembled from the K chunk sums in chunk order: LOGPROD L = c * sum(d^2),
// SUM L = log(k * sum exp(c d^2)).
__device__ __forceinline__ void block_stats(const float* __restrict__ partial,
                                            const int* __restrict__ rank, int P, int K, int mode,
                                            float c, float k, float* __restrict__ logw,
                                            float2* __restrict__ stats, int range, int blk) {
  __shared__ float sh[32];
  const int start = blk * range, end = min(P, start + range);
  float m = -INFINITY;
  for (int p = start + threadIdx.x; p < end; p += blockDim.x) {
    float L;
    if (partial) {
      float s = 0.f;
      const size_t slot = rank ? (size_t)rank[p] : (size_t)p;
      for (int q = 0; q < K; ++q) s = __fadd_rn(s, partial[(size_t)q * P + slot]);
      L = mode == MCL_LOGPROD ? __fmul_rn(c, s) : logf(__fmul_rn(k, s));
      logw[p] = L;
    } else {
      L = logw[p];
    }
    m = fmaxf(m, L);
  }
  m = block_max(m, sh);
  float s = 0.f;
  if (m > -INFINITY)
    for (int p = start + threadIdx.x; p < end; p += blockDim.x) s = __fadd_rn(s, expf(__fsub_rn(logw[p], m)));
  s = block_sum(s, sh);
  if (threadIdx.x == 0) stats[blk] = make_float2(m, m > -INFINITY ? s : 0.f);
}

__global__ void __launch_bounds__(kT) k_block_stats(const float* __restrict__ partial,
                                                    const int* __restrict__ rank, int P, int K,
                                                    int mode, float c, float k,
                                                    float* __restrict__ logw,
                                                    float2* __restrict__ stats, int range) {
  block_stats(partial, rank, P, K, mode, c, k, logw, stats, range, blockIdx.x);
}

// ---------------------------------------------------------------- pose estimate
// Per-particle terms of the estimate: W, sum w^2, sum w s_k, sum w q_i q_j.
// The quaternion of R(s) = Rz(yaw) Ry(pitch) Rx(roll) is the product of the
// three half-angle quaternions, evaluated in FP32; the sums are FP64.
struct EstAcc {
  double v[kEstSums];
  float bw;
  int bp;
};

__device__ __forceinline__ void est_init(EstAcc& a) {
#pragma unroll
  for (int i = 0; i < kEstSums; ++i) a.v[i] = 0.0;
  a.bw = -INFINITY;
  a.bp = INT_MAX;
}

// (w, p) beats (bw, bp): larger weight, or equal weight and lower index.
__device__ __forceinline__ void est_best(EstAcc& a, float w, int p) {
  if (w > a.bw || (w == a.bw && p < a.bp)) {
    a.bw = w;
    a.bp = p;
  }
}

__device__ __forceinline__ void est_add(EstAcc& a, const float* __restrict__ particles, float w,
                                        int p) {
  const float* s = particles + (size_t)p * 6;
  float sv[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) sv[k] = __ldg(s + k);
  float sr, cr, sp, cp, sy, cy;
  sincosf(0.5f * sv[3], &sr, &cr);
  sincosf(0.5f * sv[4], &sp, &cp);
  sincosf(0.5f * sv[5], &sy, &cy);
  const float q[4] = {cy * cp * cr + sy * sp * sr, cy * cp * sr - sy * sp * cr,
                      cy * sp * cr + sy * cp * sr, sy * cp * cr - cy * sp * sr};
  const double wd = (double)w;
  a.v[0] += wd;
  a.v[1] = fma(wd, wd, a.v[1]);
#pragma unroll
  for (int k = 0; k < 6; ++k) a.v[2 + k] = fma(wd, (double)sv[k], a.v[2 + k]);
  int o = 8;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const double wq = wd * (double)q[i];
#pragma unroll
    for (int j = i; j < 4; ++j) {
      a.v[o] = fma(wq, (double)q[j], a.v[o]);
      ++o;
    }
  }
  est_best(a, w, p);
}

__device__ __forceinline__ void est_best_warp(EstAcc& a) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const float ow = __shfl_xor_sync(0xffffffffu, a.bw, off);
    const int op = __shfl_xor_sync(0xffffffffu, a.bp, off);
    est_best(a, ow, op);
  }
}

// Block reduction of the estimate terms (blockDim.x == kT; the result is
// thread 0's). Every thread's sums go to shared memory; thread k + 18 g
// (g < 8 warps) adds term k of warp g's 32 threads in thread order, then
// thread k adds the 8 warp totals in warp order. A fixed order, and far fewer
// FP64 warp instructions than a shuffle tree over all 18 terms in every lane
// (FP64 issue is slow on this part: this reduction dominated the estimate
// for small particle sets). The best weight is reduced with shuffles.
struct EstShared {
  double v[kT][kEstSums];
  double warp[kT / 32][kEstSums];
  float bw[kT / 32];
  int bp[kT / 32];
};

__device__ void est_block_reduce(EstAcc& a, EstShared& sh) {
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  __syncthreads();  // sh may still be read by a previous use
#pragma unroll
  for (int k = 0; k < kEstSums; ++k) sh.v[t][k] = a.v[k];
  est_best_warp(a);
  if (lane == 0) {
    sh.bw[warp] = a.bw;
    sh.bp[warp] = a.bp;
  }
  __syncthreads();
  if (t < kEstSums * (kT / 32)) {
    const int k = t % kEstSums, g = t / kEstSums;
    double s = 0.0;
#pragma unroll 8
    for (int i = 0; i < 32; ++i) s += sh.v[g * 32 + i][k];
    sh.warp[g][k] = s;
  }
  __syncthreads();
  if (t < kEstSums) {
    double s = 0.0;
#pragma unroll
    for (int g = 0; g < kT / 32; ++g) s += sh.warp[g][t];
    sh.v[0][t] = s;
  }
  __syncthreads();
  if (t == 0) {
#pragma unroll
    for (int k = 0; k < kEstSums; ++k) a.v[k] = sh.v[0][k];
    for (int g = 0; g < kT / 32; ++g) est_best(a, sh.bw[g], sh.bp[g]);
  }
}

__device__ __forceinline__ void est_store(const EstAcc& a, EstPartial* out) {
#pragma unroll
  for (int i = 0; i < kEstSums; ++i) out->v[i] = a.v[i];
  out->best_w = a.bw;
  out->best_p = a.bp;
}

template <bool EST>
__device__ __forceinline__ void normalise_block(const float* __restrict__ logw, int P,
                                                float* __restrict__ w,
                                                const float2* __restrict__ stats, int nb, int range,
                                                float* __restrict__ out_stats,
                                                const float* __restrict__ particles,
                                                EstPartial* __restrict__ part, int blk) {
  __shared__ float sh[32];
  float m = -INFINITY;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) m = fmaxf(m, stats[i].x);
  const float M = block_max(m, sh);
  const bool degenerate = !(M > -INFINITY) || !(M < INFINITY);
  float s = 0.f;
  if (!degenerate)
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
      const float2 st = stats[i];
      if (st.x > -INFINITY) s = __fadd_rn(s, __fmul_rn(st.y, expf(__fsub_rn(st.x, M))));
    }
  const float S = block_sum(s, sh);
  const int start = blk * range, end = min(P, start + range);
  const float uni = 1.0f / (float)P;
  EstAcc acc;
  if (EST) est_init(acc);
  for (int p = start + threadIdx.x; p < end; p += blockDim.x) {
    const float wp = degenerate ? uni : __fdiv_rn(expf(__fsub_rn(logw[p], M)), S);
    w[p] = wp;
    if (EST) est_add(acc, particles, wp, p);
  }
  if (out_stats && blk == 0 && threadIdx.x == 0) {
    out_stats[0] = M;
    out_stats[1] = degenerate ? 0.f : S;
  }
  if constexpr (EST) {
    __shared__ EstShared esh;
    est_block_reduce(acc, esh);
    if (threadIdx.x == 0) est_store(acc, part + blk);
  }
}

template <bool EST>
__global__ void __launch_bounds__(kT) k_normalise(const float* __restrict__ logw, int P,
                                                  float* __restrict__ w,
                                                  const float2* __restrict__ stats, int nb,
                                                  int range, float* __restrict__ out_stats,
                                                  const float* __restrict__ particles,
                                                  EstPartial* __restrict__ part) {
  normalise_block<EST>(logw, P, w, stats, nb, range, out_stats, particles, part, blockIdx.x);
}

// The same per-block terms from weights in memory (same ranges, same order).
__global__ void __launch_bounds__(kT) k_estimate_blocks(const float* __restrict__ particles,
                                                        const float* __restrict__ w, int P,
                                                        int range, EstPartial* __restrict__ part) {
  __shared__ EstShared esh;
  EstAcc acc;
  est_init(acc);
  const int start = blockIdx.x * range, end = min(P, start + range);
  for (int p = start + threadIdx.x; p < end; p += blockDim.x) est_add(acc, particles, w[p], p);
  est_block_reduce(acc, esh);
  if (threadIdx.x == 0) est_store(acc, part + blockIdx.x);
}

// Cyclic Jacobi rotations on a symmetric 4 x 4 matrix in FP32: A becomes
// diagonal (the eigenvalues), V collects the rotations (columns = unit
// eigenvectors). FP32 because this runs on one thread, where the long
// latency of FP64 arithmetic on this part would dominate the whole estimate;
// the FP64 polish below restores the precision.
__device__ void jacobi4f(float A[4][4], float V[4][4]) {
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) V[i][j] = i == j ? 1.f : 0.f;
  for (int sweep = 0; sweep < 10; ++sweep) {
    float off = 0.f, all = 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        all += A[i][j] * A[i][j];
        if (i != j) off += A[i][j] * A[i][j];
      }
    if (!(off > 1e-14f * all)) break;
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int q = p + 1; q < 4; ++q) {
        const float apq = A[p][q];
        if (apq == 0.f) continue;
        const float theta = (A[q][q] - A[p][p]) / (2.f * apq);
        const float t = (theta >= 0.f ? 1.f : -1.f) / (fabsf(theta) + sqrtf(theta * theta + 1.f));
        const float c = rsqrtf(t * t + 1.f), s = t * c;
#pragma unroll
        for (int k = 0; k < 4; ++k) {  // A <- A J
          const float akp = A[k][p], akq = A[k][q];
          A[k][p] = c * akp - s * akq;
          A[k][q] = s * akp + c * akq;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {  // A <- J^T A
          const float apk = A[p][k], aqk = A[q][k];
          A[p][k] = c * apk - s * aqk;
          A[q][k] = s * apk + c * aqk;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {  // V <- V J
          const float vkp = V[k][p], vkq = V[k][q];
          V[k][p] = c * vkp - s * vkq;
          V[k][q] = s * vkp + c * vkq;
        }
      }
  }
}

// One block of kT threads: partials are combined in a fixed order (thread
// i takes i, i + kT, ..., then the block reduction), then thread 0 solves the
// 4 x 4 eigenproblem.
constexpr int kTF = kT;

__device__ __forceinline__ void estimate_final(const EstPartial* __restrict__ part, int nb,
                                               const float* __restrict__ particles,
                                               mcl_estimate* __restrict__ out) {
  __shared__ EstShared esh;
  EstAcc acc;
  est_init(acc);
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    const EstPartial& e = part[i];
#pragma unroll
    for (int k = 0; k < kEstSums; ++k) acc.v[k] += e.v[k];
    est_best(acc, e.best_w, e.best_p);
  }
  est_block_reduce(acc, esh);
  // The 16 quotients sum / W (6 mean pose terms, 10 second moments) on 16
  // lanes at once: an FP64 division is a dozen FP64 instructions, and one
  // thread doing all of them in turn dominated this kernel.
  __shared__ double quot[kEstSums - 2];
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < kEstSums; ++k) esh.v[0][k] = acc.v[k];
  }
  __syncthreads();
  if (threadIdx.x < kEstSums - 2) quot[threadIdx.x] = esh.v[0][2 + threadIdx.x] / esh.v[0][0];
  __syncthreads();
  if (threadIdx.x != 0) return;
  const double W = acc.v[0], W2 = acc.v[1];
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  out->weight_sum = W;
  out->n_eff = W2 > 0.0 ? W * W / W2 : 0.0;
  for (int k = 0; k < 6; ++k) out->mean_pose[k] = quot[k];
  double A[4][4];
  bool finite = W != 0.0;
  {
    int o = 6;
    for (int i = 0; i < 4; ++i)
      for (int j = i; j < 4; ++j) {
        const double qij = quot[o++];
        finite = finite && isfinite(qij);
        A[i][j] = qij;
        A[j][i] = qij;
      }
  }
  if (finite) {
    // Dominant eigenvector of Q: FP32 Jacobi, then two FP64 power steps
    // v <- Q v / |Q v| (each shrinks the error by lambda_2 / lambda_1).
    float Af[4][4], Vf[4][4];
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) Af[i][j] = (float)A[i][j];
    jacobi4f(Af, Vf);
    int b = 0;
    for (int i = 1; i < 4; ++i)
      if (Af[i][i] > Af[b][b]) b = i;
    double q[4] = {Vf[0][b], Vf[1][b], Vf[2][b], Vf[3][b]};
    for (int it = 0; it < 2; ++it) {
      double y[4];
      for (int i = 0; i < 4; ++i) y[i] = A[i][0] * q[0] + A[i][1] * q[1] + A[i][2] * q[2] + A[i][3] * q[3];
      const double inv = rsqrt(y[0] * y[0] + y[1] * y[1] + y[2] * y[2] + y[3] * y[3]);
      for (int i = 0; i < 4; ++i) q[i] = y[i] * inv;
    }
    int f = 0;
    while (f < 3 && q[f] == 0.0) ++f;
    if (q[f] < 0.0)
      for (int i = 0; i < 4; ++i) q[i] = -q[i];
    double lam = 0.0;
    for (int i = 0; i < 4; ++i)
      lam += q[i] * (A[i][0] * q[0] + A[i][1] * q[1] + A[i][2] * q[2] + A[i][3] * q[3]);
    const double r21 = 2.0 * (q[2] * q[3] + q[0] * q[1]);
    const double r22 = 1.0 - 2.0 * (q[1] * q[1] + q[2] * q[2]);
    const double r20 = 2.0 * (q[1] * q[3] - q[0] * q[2]);
    const double r10 = 2.0 * (q[1] * q[2] + q[0] * q[3]);
    const double r00 = 1.0 - 2.0 * (q[2] * q[2] + q[3] * q[3]);
    for (int i = 0; i < 4; ++i) out->quat[i] = q[i];
    // angles in FP32 (about 1e-7 rad): FP64 transcendentals on one thread
    // would dominate the whole estimate on this part
    out->rpy[0] = (double)atan2f((float)r21, (float)r22);
    out->rpy[1] = (double)asinf(fminf(1.f, fmaxf(-1.f, (float)-r20)));
    out->rpy[2] = (double)atan2f((float)r10, (float)r00);
    out->concentration = lam;
  } else {
    for (int i = 0; i < 4; ++i) out->quat[i] = nan;
    for (int i = 0; i < 3; ++i) out->rpy[i] = nan;
    out->concentration = nan;
  }
  if (acc.bp != INT_MAX) {
    out->argmax = acc.bp;
    for (int k = 0; k < 6; ++k) out->best_pose[k] = particles[(size_t)acc.bp * 6 + k];
    out->best_w = acc.bw;
  } else {
    out->argmax = -1;
    for (int k = 0; k < 6; ++k) out->best_pose[k] = __int_as_float(0x7fc00000);
    out->best_w = __int_as_float(0x7fc00000);
  }
  out->reserved = 0;
}

__global__ void __launch_bounds__(kTF) k_estimate_final(const EstPartial* __restrict__ part, int nb,
                                                        const float* __restrict__ particles,
                                                        mcl_estimate* __restrict__ out) {
  estimate_final(part, nb, particles, out);
}

inline __host__ __device__ int range_of(int P, int nb) { return (P + nb - 1) / nb; }

// ---------------------------------------------------------------- batched forms
// One launch of each pass for every session (segments of blocks, SegBlocks):
// the same blocks, ranges and order as the single-session launches, so the
// same bits.
__global__ void __launch_bounds__(kT) k_block_stats_b(const SideSeg* __restrict__ segs, SegBlocks b) {
  const int s = seg_of(b.first, b.n, blockIdx.x);
  const SideSeg& g = segs[s];
  block_stats(g.partial, g.rank, g.P, g.K, g.mode, g.c, g.k, g.logw, g.stats, range_of(g.P, g.nb),
              blockIdx.x - __ldg(b.first + s));
}

__global__ void __launch_bounds__(kT) k_normalise_b(const SideSeg* __restrict__ segs, SegBlocks b) {
  const int s = seg_of(b.first, b.n, blockIdx.x);
  const SideSeg& g = segs[s];
  const int j = blockIdx.x - __ldg(b.first + s);
  if (g.est_part)
    normalise_block<true>(g.logw, g.P, g.w, g.stats, g.nb, range_of(g.P, g.nb), g.ostats,
                          g.particles, g.est_part, j);
  else
    normalise_block<false>(g.logw, g.P, g.w, g.stats, g.nb, range_of(g.P, g.nb), g.ostats, nullptr,
                           nullptr, j);
}

__global__ void __launch_bounds__(kTF) k_estimate_final_b(const SideSeg* __restrict__ segs, SegBlocks b) {
  const int s = seg_of(b.first, b.n, blockIdx.x);
  const SideSeg& g = segs[s];
  estimate_final(g.est_part, g.nb, g.particles, g.est);
}

}  // namespace

int side_blocks_normalise(int kind, const SideSeg& g) {
  switch (kind) {
    case kSideStats: return g.nb;
    case kSideNormalise: return g.w ? g.nb : 0;
    case kSideEstimate: return g.w && g.est_part ? 1 : 0;
    default: return 0;
  }
}

cudaError_t launch_side_normalise(int kind, const SideSeg* segs, const SegBlocks& b, cudaStream_t s) {
  if (b.blocks == 0) return cudaSuccess;
  switch (kind) {
    case kSideStats: k_block_stats_b<<<b.blocks, kT, 0, s>>>(segs, b); break;
    case kSideNormalise: k_normalise_b<<<b.blocks, kT, 0, s>>>(segs, b); break;
    case kSideEstimate: k_estimate_final_b<<<b.blocks, kTF, 0, s>>>(segs, b); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

int normalise_blocks(int P) {
  const int b = (P + kT - 1) / kT;
  return b < 1024 ? b : 1024;
}

cudaError_t launch_finish_and_normalise(const float* partial, const int* rank, int P, int K,
                                        int mode, float c, float k, float* logw, float* w,
                                        float2* block_stats, int nblocks, float* out_stats,
                                        cudaStream_t s) {
  const int range = range_of(P, nblocks);
  k_block_stats<<<nblocks, kT, 0, s>>>(partial, rank, P, K, mode, c, k, logw, block_stats, range);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !w) return e;
  return launch_normalise_from_stats(logw, P, w, block_stats, nblocks, out_stats, nullptr, nullptr,
                                     nullptr, s);
}

cudaError_t launch_normalise_from_stats(const float* logw, int P, float* w,
                                        const float2* block_stats, int nblocks, float* out_stats,
                                        const float* particles, EstPartial* part,
                                        mcl_estimate* est, cudaStream_t s) {
  const int range = range_of(P, nblocks);
  if (!est) {
    k_normalise<false><<<nblocks, kT, 0, s>>>(logw, P, w, block_stats, nblocks, range, out_stats,
                                              nullptr, nullptr);
    return cudaGetLastError();
  }
  k_normalise<true><<<nblocks, kT, 0, s>>>(logw, P, w, block_stats, nblocks, range, out_stats,
                                           particles, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_estimate_final<<<1, kTF, 0, s>>>(part, nblocks, particles, est);
  return cudaGetLastError();
}

cudaError_t launch_pose_estimate(const float* particles, const float* w, int P, EstPartial* part,
                                 mcl_estimate* est, cudaStream_t s) {
  const int nb = normalise_blocks(P);
  k_estimate_blocks<<<nb, kT, 0, s>>>(particles, w, P, range_of(P, nb), part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_estimate_final<<<1, kTF, 0, s>>>(part, nb, particles, est);
  return cudaGetLastError();
}

cudaError_t launch_normalise(const float* logw, int P, float* w, float2* block_stats, int nblocks,
                             float* out_stats, cudaStream_t s) {
  return launch_finish_and_normalise(nullptr, nullptr, P, 0, MCL_LOGPROD, 0.f, 0.f,
                                     const_cast<float*>(logw), w, block_stats, nblocks, out_stats, s);
}

}  // namespace mcl
