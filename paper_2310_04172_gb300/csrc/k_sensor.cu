// Sensor update kernel (Sec. III, Eq. 3; Sec. V-B), GB300 design.
//
// The paper evaluates one particle per thread and loops over all scan points.
// Here a persistent grid walks work items (point chunk c, block of `ppi`
// particles). For each item the CTA holds the chunk's scan points in shared
// memory, staged once with a bulk asynchronous copy (cp.async.bulk, completion
// on an mbarrier); the chunk is re-staged only when the item's chunk changes.
// A group of G lanes owns one particle: lane l of the group takes points
// l, l + G, l + 2G, ... of the chunk, so neighbouring lanes read neighbouring
// scan points (neighbouring azimuths of one ring) and their map gathers fall
// in the same or adjacent sectors. Each lane issues U independent look-ups
// per step to keep several gathers in flight. Per-point scores are summed in
// FP32 per lane in point order, then reduced over the group with a fixed
// xor-shuffle tree; the chunk sum of each particle is written to
// partial[c * P + p]. The summation order depends only on (chunk, G).
//
// LOGPROD accumulates d^2 (the score -d^2 / (2 sigma^2) is applied once per
// particle when the chunks are added); SUM accumulates exp(-d^2 / (2 sigma^2))
// (Eq. 3 without its constant, applied at the end).
#include "mcl_internal.h"

namespace mcl {
namespace {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on an mbarrier phase: gives up after about a second.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  for (int i = 0; i < (1 << 22); ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if (i >= 32) __nanosleep(256);
  }
  return false;
}

__device__ __forceinline__ void bulk_copy_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                              uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

template <int KIND, int DTYPE, int G, int U>
__global__ void __launch_bounds__(256) k_sensor(const SensorArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  float4* sscan = reinterpret_cast<float4*>(smem);
  float* sout = reinterpret_cast<float*>(smem + (size_t)a.chunk * sizeof(float4));
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + (size_t)a.chunk * sizeof(float4) +
                                              (((size_t)a.ppi * sizeof(float) + 15) & ~(size_t)15));
  const uint32_t bar_s = smem_addr(bar);
  const MapView& m = a.map;

  constexpr int GPW = 32 / G;  // groups per warp
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gid = lane / G, glane = lane % G;
  const int ngroups = (blockDim.x >> 5) * GPW;

  if (threadIdx.x == 0) {
    mbar_init(bar_s, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  int loaded = -1;
  uint32_t parity = 0;
  for (long long item = blockIdx.x; item < a.n_items; item += gridDim.x) {
    const int c = (int)(item / a.nblk);
    const int p0 = (int)(item % a.nblk) * a.ppi;
    const int pn = min(a.ppi, a.P - p0);
    const int j0 = c * a.chunk;
    const int cnt = min(a.chunk, a.N - j0);

    __syncthreads();  // previous item's sout and scan reads are done
    if (c != loaded) {
      if (threadIdx.x == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        const uint32_t bytes = (uint32_t)cnt * (uint32_t)sizeof(float4);
        mbar_expect_tx(bar_s, bytes);
        bulk_copy_g2s(smem_addr(sscan), a.scan + j0, bytes, bar_s);
      }
      const bool ok = mbar_wait_bounded(bar_s, parity);
      parity ^= 1u;
      if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) {
          atomicOr(a.status, kDevErrTimeout);
          mbar_wait_bounded(bar_s, parity ^ 1u);  // let an in-flight copy land
        }
        return;
      }
      loaded = c;
    }

    for (int i0 = warp * GPW; i0 < pn; i0 += ngroups) {
      const int i = i0 + gid;
      const bool gvalid = i < pn;
      const size_t p = (size_t)p0 + (gvalid ? i : 0);
      const float4 r0 = __ldg(a.mats + 3 * p), r1 = __ldg(a.mats + 3 * p + 1),
                   r2 = __ldg(a.mats + 3 * p + 2);
      float acc = 0.f;
      for (int base = 0; base < cnt; base += G * U) {
        float dv[U];
        bool use[U];
        if constexpr (KIND == MCL_MAP_DENSE) {
          uint32_t idx[U];
          bool in[U];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int j = base + u * G + glane;
            const bool v = gvalid && j < cnt;
            const float4 z = sscan[v ? j : 0];
            float x, y, w;
            transform_point(r0, r1, r2, z, x, y, w);
            int ix, iy, iz;
            const bool inside = voxel_of(m, x, y, w, ix, iy, iz);
            in[u] = v && inside;
            use[u] = v && (inside || !a.neglect);
            idx[u] = ((uint32_t)iz * (uint32_t)m.ny + (uint32_t)iy) * (uint32_t)m.nx + (uint32_t)ix;
          }
#pragma unroll
          for (int u = 0; u < U; ++u) dv[u] = in[u] ? load_value<DTYPE>(m, idx[u]) : m.tau;
        } else {
          uint32_t key[U], loc[U];
          uint2 e[U];
          bool in[U], v[U];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int j = base + u * G + glane;
            v[u] = gvalid && j < cnt;
            const float4 z = sscan[v[u] ? j : 0];
            float x, y, w;
            transform_point(r0, r1, r2, z, x, y, w);
            int ix, iy, iz;
            in[u] = v[u] && voxel_of(m, x, y, w, ix, iy, iz);
            brick_key(m, ix, iy, iz, key[u], loc[u]);
          }
#pragma unroll
          for (int u = 0; u < U; ++u)
            e[u] = in[u] ? __ldg(m.table + brick_hash(key[u], m.hash_shift))
                         : make_uint2(kEmptyKey, 0u);
#pragma unroll
          for (int u = 0; u < U; ++u) {
            uint32_t slot = kNoSlot;
            if (in[u]) {
              if (e[u].x == key[u]) slot = e[u].y;
              else if (e[u].x != kEmptyKey) slot = probe_rest(m, key[u], brick_hash(key[u], m.hash_shift));
            }
            const bool st = slot != kNoSlot;
            dv[u] = st ? load_value<DTYPE>(m, (size_t)slot * kBrickVoxels + loc[u]) : m.tau;
            use[u] = v[u] && (st || !a.neglect);
          }
        }
        if (a.mode == MCL_LOGPROD) {
#pragma unroll
          for (int u = 0; u < U; ++u)
            if (use[u]) acc = fmaf(dv[u], dv[u], acc);
        } else {
#pragma unroll
          for (int u = 0; u < U; ++u)
            if (use[u]) acc = __fadd_rn(acc, expf(__fmul_rn(__fmul_rn(dv[u], dv[u]), a.c)));
        }
      }
#pragma unroll
      for (int off = G / 2; off > 0; off >>= 1)
        acc = __fadd_rn(acc, __shfl_xor_sync(0xffffffffu, acc, off));
      if (glane == 0 && gvalid) sout[i] = acc;
    }
    __syncthreads();
    float* dst = a.partial + (size_t)c * a.P + p0;
    for (int i = threadIdx.x; i < pn; i += blockDim.x) dst[i] = sout[i];
  }
}

template <int KIND, int DTYPE, int G, int U>
void* kernel_ptr() {
  return reinterpret_cast<void*>(&k_sensor<KIND, DTYPE, G, U>);
}

template <int KIND, int DTYPE>
void* pick_gu(int G, int U) {
  if (G == 32) return U == 2 ? kernel_ptr<KIND, DTYPE, 32, 2>() : kernel_ptr<KIND, DTYPE, 32, 4>();
  if (G == 16) return U == 2 ? kernel_ptr<KIND, DTYPE, 16, 2>() : kernel_ptr<KIND, DTYPE, 16, 4>();
  if (G == 8) return U == 2 ? kernel_ptr<KIND, DTYPE, 8, 2>() : kernel_ptr<KIND, DTYPE, 8, 4>();
  return nullptr;
}

void* pick(int kind, int dtype, int G, int U) {
  if (U != 2 && U != 4) return nullptr;
  if (kind == MCL_MAP_DENSE) {
    if (dtype == MCL_F32) return pick_gu<MCL_MAP_DENSE, MCL_F32>(G, U);
    if (dtype == MCL_F16) return pick_gu<MCL_MAP_DENSE, MCL_F16>(G, U);
    if (dtype == MCL_I16) return pick_gu<MCL_MAP_DENSE, MCL_I16>(G, U);
  } else if (kind == MCL_MAP_BRICK) {
    if (dtype == MCL_F32) return pick_gu<MCL_MAP_BRICK, MCL_F32>(G, U);
    if (dtype == MCL_F16) return pick_gu<MCL_MAP_BRICK, MCL_F16>(G, U);
    if (dtype == MCL_I16) return pick_gu<MCL_MAP_BRICK, MCL_I16>(G, U);
  }
  return nullptr;
}

}  // namespace

int sensor_smem_bytes(const SensorShape& sh) {
  return sh.chunk * (int)sizeof(float4) + ((sh.ppi * (int)sizeof(float) + 15) & ~15) + 16;
}

cudaError_t sensor_occupancy(int kind, int dtype, const SensorShape& sh, int* blocks_per_sm) {
  void* f = pick(kind, dtype, sh.lanes, sh.unroll);
  if (!f) return cudaErrorInvalidValue;
  const int smem = sensor_smem_bytes(sh);
  cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, f, sh.threads, smem);
}

cudaError_t launch_sensor(int kind, int dtype, const SensorArgs& a, const SensorShape& sh,
                          cudaStream_t s) {
  void* f = pick(kind, dtype, sh.lanes, sh.unroll);
  if (!f) return cudaErrorInvalidValue;
  const int smem = sensor_smem_bytes(sh);
  cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  void* args[] = {const_cast<SensorArgs*>(&a)};
  return cudaLaunchKernel(f, dim3(sh.grid), dim3(sh.threads), args, (size_t)smem, s);
}

}  // namespace mcl
