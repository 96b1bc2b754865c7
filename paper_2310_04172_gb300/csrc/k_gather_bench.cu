// Gather roofline microbenchmark: uniform-random reads of 2- or 4-byte
// elements over a caller buffer. Its gathers/s at a given footprint is the
// ceiling for the TSDF look-ups of the sensor update (Sec. VI-C: the map
// look-ups are random accesses and bound the kernel), measured on this GPU.
//
// Every thread draws indices from its own counter-based stream (a 64-bit
// multiply-xorshift mix of (seed, thread, i)), keeps U loads in flight and
// folds the values into one sink word per thread block so nothing is
// optimised away.
#include "mcl_internal.h"

namespace mcl {
namespace {

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 33)) * 0xFF51AFD7ED558CCDull;
  z = (z ^ (z >> 33)) * 0xC4CEB9FE1A85EC53ull;
  return z ^ (z >> 33);
}

template <typename T, int U>
__global__ void __launch_bounds__(256) k_gather(const T* __restrict__ buf, uint64_t n, int iters,
                                                uint64_t seed, float* __restrict__ sink) {
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t state = mix64(seed ^ (tid * 0x9E3779B97F4A7C15ull));
  float acc = 0.f;
  for (int it = 0; it < iters; ++it) {
    T v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      state = mix64(state + 0x9E3779B97F4A7C15ull);
      const uint64_t i = __umul64hi(state, n);  // uniform in [0, n)
      v[u] = __ldg(buf + i);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) acc += (float)v[u];
  }
  acc += __shfl_xor_sync(0xffffffffu, acc, 16);
  if ((threadIdx.x & 31) == 0 && acc == 1234.5f) sink[blockIdx.x] = acc;  // practically never
}

}  // namespace

cudaError_t launch_gather_bench(const void* buf, long long n_elems, int elem_bytes, int blocks,
                                int iters, unsigned long long seed, float* sink, cudaStream_t s) {
  if (elem_bytes == 2)
    k_gather<short, 8><<<blocks, 256, 0, s>>>((const short*)buf, (uint64_t)n_elems, iters, seed, sink);
  else if (elem_bytes == 4)
    k_gather<float, 8><<<blocks, 256, 0, s>>>((const float*)buf, (uint64_t)n_elems, iters, seed, sink);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace mcl
