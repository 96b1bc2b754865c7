// Particle log-weights from chunk partials, and normalisation (Sec. V-A: the
// weights are summed for normalisation; Sec. V-B: a GPU reduction).
//
// The paper reduces with repeated pairwise-halving launches. Here two
// launches suffice: each of up to 1024 blocks owns a contiguous particle range
// and writes its (max, sum exp(L - max)); every block of the second launch
// combines all block pairs in the same fixed order (so all blocks agree on M
// and S bit for bit) and writes w = exp(L - M) / S for its range. FP32
// throughout; max-subtracted so nothing overflows.
#include <cfloat>

#include "mcl_internal.h"

namespace mcl {
namespace {

constexpr int kT = 1024;

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
__global__ void __launch_bounds__(kT) k_block_stats(const float* __restrict__ partial,
                                                    const int* __restrict__ rank, int P, int K,
                                                    int mode, float c, float k,
                                                    float* __restrict__ logw,
                                                    float2* __restrict__ stats, int range) {
  __shared__ float sh[32];
  const int start = blockIdx.x * range, end = min(P, start + range);
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
  if (threadIdx.x == 0) stats[blockIdx.x] = make_float2(m, m > -INFINITY ? s : 0.f);
}

__global__ void __launch_bounds__(kT) k_normalise(const float* __restrict__ logw, int P,
                                                  float* __restrict__ w,
                                                  const float2* __restrict__ stats, int nb,
                                                  int range, float* __restrict__ out_stats) {
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
  const int start = blockIdx.x * range, end = min(P, start + range);
  const float uni = 1.0f / (float)P;
  for (int p = start + threadIdx.x; p < end; p += blockDim.x)
    w[p] = degenerate ? uni : __fdiv_rn(expf(__fsub_rn(logw[p], M)), S);
  if (out_stats && blockIdx.x == 0 && threadIdx.x == 0) {
    out_stats[0] = M;
    out_stats[1] = degenerate ? 0.f : S;
  }
}

inline int range_of(int P, int nb) { return (P + nb - 1) / nb; }

}  // namespace

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
  k_normalise<<<nblocks, kT, 0, s>>>(logw, P, w, block_stats, nblocks, range, out_stats);
  return cudaGetLastError();
}

cudaError_t launch_normalise(const float* logw, int P, float* w, float2* block_stats, int nblocks,
                             float* out_stats, cudaStream_t s) {
  return launch_finish_and_normalise(nullptr, nullptr, P, 0, MCL_LOGPROD, 0.f, 0.f,
                                     const_cast<float*>(logw), w, block_stats, nblocks, out_stats, s);
}

}  // namespace mcl
