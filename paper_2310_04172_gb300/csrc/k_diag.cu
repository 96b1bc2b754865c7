// Self-test of the failure path of the bounded waits: one CTA waits on an
// mbarrier phase that nothing completes (no copy is issued, nothing
// arrives); the wait must give up after its time limit, record the timeout
// in the device status word and let the kernel return, leaving the context
// usable.
#include "k_sensor_impl.cuh"

namespace mcl {
namespace {

__global__ void k_wait_selftest(unsigned* __restrict__ status,
                                unsigned long long* __restrict__ waited_ns) {
  __shared__ __align__(8) unsigned long long bar;
  const uint32_t b = sensor::smem_addr(&bar);
  sensor::init_barrier(b);
  const uint64_t t0 = sensor::global_ns();
  const bool ok = sensor::mbar_wait_bounded(b, 0u);
  __syncthreads();
  if (threadIdx.x == 0) {
    if (!ok) atomicOr(status, kDevErrTimeout);
    *waited_ns = sensor::global_ns() - t0;
  }
}

}  // namespace

cudaError_t launch_wait_selftest(unsigned* status, unsigned long long* waited_ns, cudaStream_t s) {
  k_wait_selftest<<<1, 32, 0, s>>>(status, waited_ns);
  return cudaGetLastError();
}

}  // namespace mcl
