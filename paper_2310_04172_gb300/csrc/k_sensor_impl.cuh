// Sensor update kernel (Sec. III, Eq. 3; Sec. V-B), GB300 design.
//
// The paper evaluates one particle per thread and loops over all scan points.
// Here a persistent grid walks work items (point chunk c, block of `ppi`
// particles) strided by the grid size. The CTA holds the chunk's scan points in
// shared memory, staged with one bulk asynchronous copy (cp.async.bulk,
// completion on an mbarrier) and re-staged only when the item's chunk changes;
// that is the only CTA-wide barrier. A group of G lanes owns one particle: lane
// l of the group takes points l, l + G, l + 2G, ... of the chunk, so
// neighbouring lanes read neighbouring scan points (neighbouring azimuths of
// one ring) and their map gathers fall in the same or adjacent sectors. Each
// lane keeps U look-ups in flight per step (brick-index entries first, then
// the values). Per-point terms are summed in FP32 per lane in point order, then
// over the group with a fixed xor-shuffle tree; lane 0 of the group writes the
// particle's chunk sum to partial[c * P + p]. The summation order depends only
// on (chunk, G).
//
// LOGPROD accumulates d^2 (the score -d^2 / (2 sigma^2) is applied once per
// particle when the chunks are added); SUM accumulates exp(-d^2 / (2 sigma^2))
// (Eq. 3 without its constant, applied at the end). For int16 maps the terms
// use the stored integer q (d = q * scale): LOGPROD accumulates q^2 and the
// chunk sum is multiplied by scale^2 once; SUM folds scale^2 into the exponent
// constant. A point without a stored value reads +tau (q = 32767 for int16).
#pragma once

#include "mcl_internal.h"

namespace mcl {
namespace sensor {


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

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// How long a CTA waits for its own bulk copy before it gives up.
constexpr uint64_t kWaitLimitNs = 1000000000ull;  // 1 s

// Bounded wait on an mbarrier phase: gives up after about a second of wall
// time (globaltimer), whatever each try_wait's own suspension is, with an
// iteration cap as a backstop.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (int i = 0; i < (1 << 26); ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > kWaitLimitNs) return false;
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

// What the accumulation works on: FP32 / FP16 values as floats; int16 as
// the stored integer q converted to float (LOGPROD sums q^2 and the chunk sum
// is scaled by scale^2 once; SUM folds scale^2 into the exponent constant).
// Sums are FP32. (Exact 64-bit integer sums of q^2, one wide multiply-add per
// point instead of a conversion and an FMA, measured slower: 107.9 against
// 102.8 ms for 1M x 65,536; so did predicating the gathers inside their own
// load instruction, which made the kernel spill.)
template <int DTYPE, int MODE>
struct Raw {
  using value = float;
  using acc = float;
};

#ifndef MCL_VALUE_LOAD_HINT
#define MCL_VALUE_LOAD_HINT 1
#endif

// Read-only 16/32-bit gathers of map values. Hint 1 (default): do not
// allocate in L1 (the values have little reuse there; the brick index and
// the scan keep L1): 184.5 ms against 189.9 ms with plain read-only loads for
// 1M x 65,536. Hints 2 and 3 add an L2 evict-first / evict-last policy.
__device__ __forceinline__ unsigned short ld_u16(const void* p) {
  unsigned short v;
#if MCL_VALUE_LOAD_HINT == 1
  asm volatile("ld.global.nc.L1::no_allocate.u16 %0, [%1];" : "=h"(v) : "l"(p));
#elif MCL_VALUE_LOAD_HINT == 2 || MCL_VALUE_LOAD_HINT == 3
  uint64_t pol;
#if MCL_VALUE_LOAD_HINT == 2
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
#else
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
#endif
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.u16 %0, [%1], %2;" : "=h"(v) : "l"(p), "l"(pol));
#else
  v = __ldg(static_cast<const unsigned short*>(p));
#endif
  return v;
}

__device__ __forceinline__ float ld_f32(const void* p) {
  float v;
#if MCL_VALUE_LOAD_HINT == 1
  asm volatile("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
#elif MCL_VALUE_LOAD_HINT == 2 || MCL_VALUE_LOAD_HINT == 3
  uint64_t pol;
#if MCL_VALUE_LOAD_HINT == 2
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
#else
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
#endif
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
#else
  v = __ldg(static_cast<const float*>(p));
#endif
  return v;
}

template <int DTYPE, int MODE>
__device__ __forceinline__ typename Raw<DTYPE, MODE>::value load_raw(const void* values, size_t i) {
  if constexpr (DTYPE == MCL_F32) {
    return ld_f32(static_cast<const float*>(values) + i);
  } else if constexpr (DTYPE == MCL_F16) {
    return __half2float(__ushort_as_half(ld_u16(static_cast<const __half*>(values) + i)));
  } else {
    return (float)(short)ld_u16(static_cast<const short*>(values) + i);
  }
}

// The same through L1: the trilinear read's eight corners share L1 lines.
template <int DTYPE, int MODE>
__device__ __forceinline__ typename Raw<DTYPE, MODE>::value load_raw_l1(const void* values, size_t i) {
  if constexpr (DTYPE == MCL_F32) {
    return __ldg(static_cast<const float*>(values) + i);
  } else if constexpr (DTYPE == MCL_F16) {
    return __half2float(__ldg(static_cast<const __half*>(values) + i));
  } else {
    return (float)__ldg(static_cast<const short*>(values) + i);
  }
}

// Value the nearest read takes where nothing is stored, in the same units
// (its term is exactly zero under MCL_NEGLECT_OUTSIDE).
template <int DTYPE, int MODE>
__device__ __forceinline__ typename Raw<DTYPE, MODE>::value outside_value(const SensorArgs& a) {
  return a.vnear;
}

// Index of a brick value. Cell-grid kind: `slot` is the grid entry, the
// index of the brick's first value (slot * 4096, at most kGridMaxBricks
// bricks, so 32 bits), and `local` the skewed offset (skew_local); 64-bit
// slot * 4096 + local otherwise.
template <int KIND>
__device__ __forceinline__ size_t value_index(uint32_t slot, uint32_t local) {
  if constexpr (KIND == kKindBrickGrid) return (size_t)(slot | local);
  else return (size_t)slot * kBrickVoxels + local;
}

// Slot number of a slot as a kernel holds it (cell grid: the grid entry).
template <int KIND>
__device__ __forceinline__ uint32_t slot_number(uint32_t slot) {
  if constexpr (KIND == kKindBrickGrid) return slot / (uint32_t)kBrickVoxels;
  else return slot;
}

// In-brick offset: linear x-fastest, or 4x4x4 blocks (block-major, each block
// z-major) so that a 32-byte sector of int16 values is a 4 x 4 patch in x, y.
template <int KIND>
__device__ __forceinline__ uint32_t brick_local(int ix, int iy, int iz) {
  const uint32_t lx = (uint32_t)ix & 15u, ly = (uint32_t)iy & 15u, lz = (uint32_t)iz & 15u;
  if constexpr (KIND == kKindBrickBlock4) {
    return ((lz >> 2) << 10) | ((ly >> 2) << 8) | ((lx >> 2) << 6) | ((lz & 3u) << 4) |
           ((ly & 3u) << 2) | (lx & 3u);
  } else {
    return (lz << 8) | (ly << 4) | lx;
  }
}

// Stage A of one step of U points per lane: load the points, transform them,
// find their voxels and issue the first index look-up (brick maps: the cell
// grid's slot or the first hash entry; dense maps: the value itself). FULL:
// every point index is inside the chunk and the group is valid (no bounds
// predicates).
template <int KIND, int DTYPE, int MODE, int U>
struct Pending {
  uint32_t key[U], loc[U];  // BRICK: brick-cell key, in-brick offset; DENSE: key = linear index
  uint2 e[U];               // BRICK: first hash entry (EMPTY where not in[u]); grid: .y = slot
  typename Raw<DTYPE, MODE>::value dv[U];  // DENSE: value
  bool in[U], v[U];
};

// The particle's [R | t] rows live in shared memory (one slot per lane group,
// each entry duplicated into both halves of a pair for the packed
// instructions) and are re-read every step, so they do not hold registers
// across the gathers (with the pose rows in registers the kernel needed 5
// resident CTAs per SM instead of 6: 243 against 239 ms for 1M x 65,536).
__device__ __forceinline__ float4 lds_volatile(const float4* p) {
  float4 v;
  asm volatile("ld.volatile.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"((uint32_t)__cvta_generic_to_shared(p)));
  return v;
}

// Stage A on the pair layout (ScanLayout): the lane's points j and j + G of a
// step come as one XY float4 and one Z float2, so each coordinate of the two
// sits in one register pair and the transform and the floor run as packed
// FP32x2 instructions (IEEE per element: the same bits as the scalar fmaf
// chain). The pose rows are in the map's index frame (RowFrame), so the fma
// chain gives the index coordinate u itself: no origin or scale step per
// point (the frame costs three FP32x2 operations per pair and axis less:
// 93.5 against 87.0 ms for 1M x 65,536). The floor comes from a
// round-down add of 2^23: for 0 <= u < 2^23 the sum's bits are 0x4B000000 +
// floor(u) exactly, and every other u (negative, >= 2^23, +-inf, NaN) leaves
// bits - 0x4B000000 >= 2^23 as an unsigned number, so one unsigned compare
// with n (at most 2^23) is the rule 0 <= u < n, NaN outside. rows: the
// group's six float4 of duplicated pose entries (pair_rows).
constexpr uint32_t kFloorBits = 0x4B000000u;  // bits of 2^23

// Cell-grid kind: instead of the inside test, each index is clamped to n
// (unsigned min), which sends every point outside the grid to a guard cell
// of the padded cell grid that holds no brick, so it reads the outside value
// exactly as the test would give, and the cell look-up needs no predicate.
#ifndef MCL_GRID_CLAMP
#define MCL_GRID_CLAMP 1
#endif

template <int KIND, int DTYPE, int MODE, int G, int U, bool FULL>
__device__ __forceinline__ void stage_a_pairs(const SensorArgs& a, const float4* __restrict__ sxy,
                                              const float2* __restrict__ sz, int base, int glane,
                                              int cnt, bool gvalid, const float4* rows,
                                              Pending<KIND, DTYPE, MODE, U>& s) {
  static_assert(U % 2 == 0, "points come in pairs");
  const MapView& m = a.map;
  // the rows once per step: re-reading them for every pair of the step frees
  // their 24 registers (no spills at 64) but measured 104.1 against 97.0 ms
  const float4 q0 = lds_volatile(rows), q1 = lds_volatile(rows + 1), q2 = lds_volatile(rows + 2),
               q3 = lds_volatile(rows + 3), q4 = lds_volatile(rows + 4), q5 = lds_volatile(rows + 5);
  const float2 two23 = make_float2(8388608.f, 8388608.f);
#pragma unroll
  for (int k = 0; k < U / 2; ++k) {
    const int j0 = base + 2 * k * G + glane;
    s.v[2 * k] = FULL || (gvalid && j0 < cnt);
    s.v[2 * k + 1] = FULL || (gvalid && j0 + G < cnt);
    const int pi = (base / (2 * G) + k) * G + glane;
    const float4 xy = sxy[pi];
    const float2 zz = sz[pi];
    const float2 zx = make_float2(xy.x, xy.y), zy = make_float2(xy.z, xy.w);
    // u_i = fma(R'_i0, z0, fma(R'_i1, z1, fma(R'_i2, z2, t'_i))) for both points
    // (rows in the map's index frame, RowFrame)
    const float2 X = __ffma2_rn(make_float2(q0.x, q0.y), zx,
                                __ffma2_rn(make_float2(q0.z, q0.w), zy,
                                           __ffma2_rn(make_float2(q1.x, q1.y), zz, make_float2(q1.z, q1.w))));
    const float2 Y = __ffma2_rn(make_float2(q2.x, q2.y), zx,
                                __ffma2_rn(make_float2(q2.z, q2.w), zy,
                                           __ffma2_rn(make_float2(q3.x, q3.y), zz, make_float2(q3.z, q3.w))));
    const float2 W = __ffma2_rn(make_float2(q4.x, q4.y), zx,
                                __ffma2_rn(make_float2(q4.z, q4.w), zy,
                                           __ffma2_rn(make_float2(q5.x, q5.y), zz, make_float2(q5.z, q5.w))));
    // floor via the round-down add of 2^23
    const float2 fx = __fadd2_rd(X, two23), fy = __fadd2_rd(Y, two23), fz = __fadd2_rd(W, two23);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int u = 2 * k + h;
      uint32_t ix = __float_as_uint(h ? fx.y : fx.x) - kFloorBits;
      uint32_t iy = __float_as_uint(h ? fy.y : fy.x) - kFloorBits;
      uint32_t iz = __float_as_uint(h ? fz.y : fz.x) - kFloorBits;
      if constexpr (KIND == kKindBrickGrid && MCL_GRID_CLAMP) {
        ix = min(ix, (uint32_t)m.nx);
        iy = min(iy, (uint32_t)m.ny);
        iz = min(iz, (uint32_t)m.nz);
        s.in[u] = s.v[u];
      } else {
        s.in[u] = s.v[u] && (ix < (uint32_t)m.nx) && (iy < (uint32_t)m.ny) && (iz < (uint32_t)m.nz);
      }
      if constexpr (is_dense(KIND)) {
        s.key[u] = dense_index<KIND == kKindDenseTiles>(ix, iy, iz, (uint32_t)m.nx, (uint32_t)m.ny, m.tcy, m.tsz);
      } else if constexpr (KIND == kKindBrickGrid) {
        s.key[u] = (iz >> 4) * m.gsz + (iy >> 4) * m.gsy + (ix >> 4);
        s.loc[u] = skew_local(ix, iy, iz);
      } else {
        s.key[u] = ((iz >> 4) * m.nby + (iy >> 4)) * m.nbx + (ix >> 4);
        s.loc[u] = brick_local<KIND>((int)ix, (int)iy, (int)iz);
      }
    }
  }
#pragma unroll
  for (int u = 0; u < U; ++u) {
    if constexpr (is_dense(KIND)) {
      s.dv[u] = s.in[u] ? load_raw<DTYPE, MODE>(m.values, s.key[u]) : outside_value<DTYPE, MODE>(a);
    } else if constexpr (KIND == kKindBrickGrid) {
      s.e[u].y = s.in[u] ? __ldg(m.grid + s.key[u]) : kNoSlot;
    } else {
      s.e[u] = s.in[u] ? __ldg(m.table + brick_hash(s.key[u], m.hash_shift))
                       : make_uint2(kEmptyKey, 0u);
    }
  }
}

// Stage B: resolve the brick slot (further probes if the first entry was
// another key) and issue the value gathers; outputs the values and which
// points count.
template <int KIND, int DTYPE, int MODE, int U>
__device__ __forceinline__ void stage_b(const SensorArgs& a, const Pending<KIND, DTYPE, MODE, U>& s,
                                        typename Raw<DTYPE, MODE>::value* dv, bool* use) {
  const MapView& m = a.map;
#pragma unroll
  for (int u = 0; u < U; ++u) {
    if constexpr (is_dense(KIND)) {
      dv[u] = s.dv[u];
      use[u] = s.v[u];
    } else {
      uint32_t slot = kNoSlot;
      if constexpr (KIND == kKindBrickGrid) {
        slot = s.e[u].y;  // kNoSlot outside the grid or in an empty cell
      } else if (s.in[u]) {
        if (s.e[u].x == s.key[u]) slot = s.e[u].y;
        else if (s.e[u].x != kEmptyKey)
          slot = probe_rest(m, s.key[u], brick_hash(s.key[u], m.hash_shift));
      }
#if MCL_DEBUG_BOUNDS
      if (slot != kNoSlot && slot_number<KIND>(slot) >= m.n_slots) {
        atomicOr(a.status, kDevErrIndex);
        slot = kNoSlot;
      }
#endif
      const bool st = slot != kNoSlot;
      dv[u] = st ? load_raw<DTYPE, MODE>(m.values, value_index<KIND>(slot, s.loc[u]))
                 : outside_value<DTYPE, MODE>(a);
      use[u] = s.v[u];
    }
  }
}

// 2^x by the hardware approximation (PTX ex2.approx.f32: relative error of a
// few units in the last place, subnormal results kept, 2^-inf = 0): the SUM
// mode's per-point exp(-d^2 / (2 sigma^2)) as 2^(d^2 cs), cs carrying log2(e)
// (SUM on the TSDF for 1M x 65,536: 94.8 ms against 97.3 ms with expf).
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

template <int DTYPE, int MODE, int U>
__device__ __forceinline__ void accumulate(const SensorArgs& a,
                                           const typename Raw<DTYPE, MODE>::value* dv,
                                           const bool* use, typename Raw<DTYPE, MODE>::acc& acc) {
  if constexpr (MODE == MCL_LOGPROD) {
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (use[u]) acc = fmaf(dv[u], dv[u], acc);
  } else if constexpr (MODE == kModeScore) {
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (use[u]) acc = __fadd_rn(acc, dv[u]);
  } else {
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (use[u]) acc = __fadd_rn(acc, ex2_approx(__fmul_rn(__fmul_rn(dv[u], dv[u]), a.cs)));
  }
}

// All points [0, end) of one particle's chunk, end a multiple of G*U, without
// bounds checks. PIPE: stage A of step i+1 is issued before the gathers of
// step i are consumed, so the index look-ups of the next step overlap the
// value gathers of this one (the per-point order of the sum is unchanged).
template <int KIND, int DTYPE, int MODE, int G, int U, bool PIPE>
__device__ __forceinline__ void eval_full(const SensorArgs& a, const float4* __restrict__ sxy,
                                          const float2* __restrict__ sz, int end, int glane,
                                          const float4* rows, typename Raw<DTYPE, MODE>::acc& acc) {
  constexpr int STEP = G * U;
  using V = typename Raw<DTYPE, MODE>::value;
  if (end <= 0) return;
  Pending<KIND, DTYPE, MODE, U> s;
  if constexpr (PIPE) {
    stage_a_pairs<KIND, DTYPE, MODE, G, U, true>(a, sxy, sz, 0, glane, end, true, rows, s);
    for (int base = 0; base < end; base += STEP) {
      V dv[U];
      bool use[U];
      stage_b<KIND, DTYPE, MODE, U>(a, s, dv, use);
      if (base + STEP < end)
        stage_a_pairs<KIND, DTYPE, MODE, G, U, true>(a, sxy, sz, base + STEP, glane, end, true, rows, s);
      accumulate<DTYPE, MODE, U>(a, dv, use, acc);
    }
  } else {
    for (int base = 0; base < end; base += STEP) {
      V dv[U];
      bool use[U];
      stage_a_pairs<KIND, DTYPE, MODE, G, U, true>(a, sxy, sz, base, glane, end, true, rows, s);
      stage_b<KIND, DTYPE, MODE, U>(a, s, dv, use);
      accumulate<DTYPE, MODE, U>(a, dv, use, acc);
    }
  }
}

// One bounds-checked step (chunk tails, partly valid groups).
template <int KIND, int DTYPE, int MODE, int G, int U>
__device__ __forceinline__ void eval_checked(const SensorArgs& a, const float4* __restrict__ sxy,
                                             const float2* __restrict__ sz, int base, int glane,
                                             int cnt, bool gvalid, const float4* rows,
                                             typename Raw<DTYPE, MODE>::acc& acc) {
  Pending<KIND, DTYPE, MODE, U> s;
  typename Raw<DTYPE, MODE>::value dv[U];
  bool use[U];
  stage_a_pairs<KIND, DTYPE, MODE, G, U, false>(a, sxy, sz, base, glane, cnt, gvalid, rows, s);
  stage_b<KIND, DTYPE, MODE, U>(a, s, dv, use);
  accumulate<DTYPE, MODE, U>(a, dv, use, acc);
}

// ---------------------------------------------------------------- trilinear read
// MCL_TRILINEAR (Sec. III: a pseudo-continuous value by interpolation). The
// stored value of voxel i is the SDF at its centre o + (i + 1/2) r, so with
// f = u - 1/2 (FP32; the pose rows in the index frame with shift 1/2,
// RowFrame), the eight centres around the point are i0 + {0, 1} per axis,
// i0 = floor(f), with weights
// a = f - i0 and 1 - a. A corner outside the grid or in no brick reads the
// same value as an unstored voxel. The point counts as stored if any corner
// is. Interpolation in FP32: along x for the four (y, z) corner pairs, then
// y, then z, each step fma(a, v1 - v0, v0). (Skipping the look-ups of bricks
// beyond the first that no lane of the warp needs, decided by warp votes,
// needs the whole warp on this path for every point: 595 against 459 ms for
// 1M x 65,536, the early return for points outside the grid matters more; a
// per-lane loop over only the crossed bricks diverges: 506 ms.)
template <int KIND, int DTYPE, int MODE>
__device__ __forceinline__ float tri_read(const SensorArgs& a, float fx, float fy, float fz,
                                          bool& stored) {
  const MapView& m = a.map;
  stored = false;
  // Some corner is inside iff -1 <= f < n on every axis (NaN fails).
  if (!((fx >= -1.f) & (fx < m.fnx) & (fy >= -1.f) & (fy < m.fny) & (fz >= -1.f) & (fz < m.fnz)))
    return a.vout;
  const float flx = floorf(fx), fly = floorf(fy), flz = floorf(fz);
  const int x0 = (int)flx, y0 = (int)fly, z0 = (int)flz;
  const float ax = __fsub_rn(fx, flx), ay = __fsub_rn(fy, fly), az = __fsub_rn(fz, flz);
  const bool inx[2] = {x0 >= 0, x0 + 1 < m.nx};
  const bool iny[2] = {y0 >= 0, y0 + 1 < m.ny};
  const bool inz[2] = {z0 >= 0, z0 + 1 < m.nz};
  float v[8];
  if constexpr (is_dense(KIND)) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int cx = c & 1, cy = (c >> 1) & 1, cz = c >> 2;
      const bool in = inx[cx] & iny[cy] & inz[cz];
      const uint32_t lin = dense_index<KIND == kKindDenseTiles>(
          (uint32_t)(x0 + cx), (uint32_t)(y0 + cy), (uint32_t)(z0 + cz), (uint32_t)m.nx, (uint32_t)m.ny,
          m.tcy, m.tsz);
      v[c] = in ? load_raw_l1<DTYPE, MODE>(m.values, lin) : a.vout;
      stored |= in;
    }
  } else if constexpr (KIND == kKindBrickGrid || KIND == MCL_MAP_BRICK) {
    // Linear bricks. Along each axis the two corners share a brick unless
    // the lower one sits on the brick's last voxel (s = 1; always so for
    // i0 = -1). Corner c therefore lies in brick b0 + (c_x s_x, c_y s_y,
    // c_z s_z): at most 2^(s_x + s_y + s_z) distinct bricks, one for 82 % of
    // the points of the building scan. Hash index: a brick is looked up only
    // if a corner inside the grid lies in it; a corner outside the grid maps
    // to a brick that was not looked up, so its slot is empty. Cell grid: the
    // cells at -1 and nb along each axis are guard cells that hold no brick,
    // so every brick a corner lies in is looked up as it is. Brick keys are
    // formed in 32-bit arithmetic, which wraps consistently for i0 = -1; a
    // cell-grid key is then a signed offset from cell (0, 0, 0) (down to the
    // first front guard cell) and is sign-extended before it meets the pointer.
    const uint32_t sx = (x0 & 15) == 15, sy = (y0 & 15) == 15, sz = (z0 & 15) == 15;
    constexpr bool kGuard = KIND == kKindBrickGrid && MCL_GRID_CLAMP;
    const uint32_t nbx = KIND == kKindBrickGrid ? m.gsy : m.nbx,
                   nbxy = KIND == kKindBrickGrid ? m.gsz : m.nbx * m.nby;
    const uint32_t k0 = (uint32_t)(z0 >> 4) * nbxy + (uint32_t)(y0 >> 4) * nbx + (uint32_t)(x0 >> 4);
    const bool ux[2] = {kGuard || inx[0], (sx != 0) && (kGuard || inx[1])};
    const bool uy[2] = {kGuard || iny[0], (sy != 0) && (kGuard || iny[1])};
    const bool uz[2] = {kGuard || inz[0], (sz != 0) && (kGuard || inz[1])};
    uint32_t b[8];  // slot of brick b0 + (q & 1, (q >> 1) & 1, q >> 2)
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int qx = q & 1, qy = (q >> 1) & 1, qz = q >> 2;
      const bool need = ux[qx] & uy[qy] & uz[qz];
      const uint32_t key = k0 + (uint32_t)qx + (uint32_t)qy * nbx + (uint32_t)qz * nbxy;
      if constexpr (KIND == kKindBrickGrid) {
        b[q] = need ? __ldg(m.grid + (int32_t)key) : kNoSlot;
      } else {
        b[q] = kNoSlot;
        if (need) {
          const uint32_t h = brick_hash(key, m.hash_shift);
          const uint2 e = __ldg(m.table + h);
          b[q] = e.x == key ? e.y : (e.x == kEmptyKey ? kNoSlot : probe_rest(m, key, h));
        }
      }
    }
    uint32_t slot[8];
    slot[0] = b[0];
    slot[1] = sx ? b[1] : b[0];
    slot[2] = sy ? b[2] : b[0];
    slot[3] = sx ? (sy ? b[3] : b[1]) : slot[2];
    slot[4] = sz ? b[4] : b[0];
    slot[5] = sz ? (sx ? b[5] : b[4]) : slot[1];
    slot[6] = sz ? (sy ? b[6] : b[4]) : slot[2];
    slot[7] = sz ? (sx ? (sy ? b[7] : b[5]) : (sy ? b[6] : b[4])) : slot[3];
    // in-brick offsets. Linear bricks: one step up along an axis is +1 / +16 /
    // +256, or back to 0 on that axis when the corner crosses into the next
    // brick. Cell grid (skewed bricks, skew_local): +1 / +16 / +256 mod 4096
    // whether or not the corner crosses.
    constexpr bool kSkew = KIND == kKindBrickGrid && MCL_GRID_SKEW;
    const int base = kSkew ? (int)skew_local((uint32_t)x0, (uint32_t)y0, (uint32_t)z0)
                           : (((z0 & 15) << 8) | ((y0 & 15) << 4) | (x0 & 15));
    const int ox = !kSkew && sx ? -15 : 1, oy = !kSkew && sy ? -240 : 16, oz = !kSkew && sz ? -3840 : 256;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int cx = c & 1, cy = (c >> 1) & 1, cz = c >> 2;
#if MCL_DEBUG_BOUNDS
      if (slot[c] != kNoSlot && slot_number<KIND>(slot[c]) >= m.n_slots) {
        atomicOr(a.status, kDevErrIndex);
        slot[c] = kNoSlot;
      }
#endif
      const bool st = slot[c] != kNoSlot;
      int off = base + (cx ? ox : 0) + (cy ? oy : 0) + (cz ? oz : 0);
      if constexpr (kSkew) off &= kBrickVoxels - 1;
      v[c] = st ? load_raw_l1<DTYPE, MODE>(m.values, value_index<KIND>(slot[c], (uint32_t)off))
                : a.vout;
      stored |= st;
    }
  } else {
    uint32_t key[8], slot[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int cx = c & 1, cy = (c >> 1) & 1, cz = c >> 2;
      key[c] = ((uint32_t)((z0 + cz) >> 4) * m.nby + (uint32_t)((y0 + cy) >> 4)) * m.nbx +
               (uint32_t)((x0 + cx) >> 4);
    }
    // One probe per distinct brick: a corner reuses the slot of a neighbouring
    // corner (lower along x, else y, else z) in the same brick.
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int cx = c & 1, cy = (c >> 1) & 1, cz = c >> 2;
      const bool in = inx[cx] & iny[cy] & inz[cz];
      slot[c] = kNoSlot;
      if (!in) continue;
      int r = -1;
      if (cx && (inx[0] & iny[cy] & inz[cz]) && key[c ^ 1] == key[c]) r = c ^ 1;
      else if (cy && (inx[cx] & iny[0] & inz[cz]) && key[c ^ 2] == key[c]) r = c ^ 2;
      else if (cz && (inx[cx] & iny[cy] & inz[0]) && key[c ^ 4] == key[c]) r = c ^ 4;
      if (r >= 0) {
        slot[c] = slot[r];
      } else {  // 4x4x4-block bricks have the hash index only
        const uint32_t h = brick_hash(key[c], m.hash_shift);
        const uint2 e = __ldg(m.table + h);
        slot[c] = e.x == key[c] ? e.y : (e.x == kEmptyKey ? kNoSlot : probe_rest(m, key[c], h));
      }
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int cx = c & 1, cy = (c >> 1) & 1, cz = c >> 2;
#if MCL_DEBUG_BOUNDS
      if (slot[c] != kNoSlot && slot_number<KIND>(slot[c]) >= m.n_slots) {
        atomicOr(a.status, kDevErrIndex);
        slot[c] = kNoSlot;
      }
#endif
      const bool st = slot[c] != kNoSlot;
      v[c] = st ? load_raw_l1<DTYPE, MODE>(m.values, (size_t)slot[c] * kBrickVoxels +
                                                     brick_local<KIND>(x0 + cx, y0 + cy, z0 + cz))
                : a.vout;
      stored |= st;
    }
  }
  const float c00 = fmaf(ax, __fsub_rn(v[1], v[0]), v[0]);
  const float c10 = fmaf(ax, __fsub_rn(v[3], v[2]), v[2]);
  const float c01 = fmaf(ax, __fsub_rn(v[5], v[4]), v[4]);
  const float c11 = fmaf(ax, __fsub_rn(v[7], v[6]), v[6]);
  const float c0 = fmaf(ay, __fsub_rn(c10, c00), c00);
  const float c1 = fmaf(ay, __fsub_rn(c11, c01), c01);
  return fmaf(az, __fsub_rn(c1, c0), c0);
}

// One particle's points of the staged chunk with the trilinear read: lane
// glane takes points glane, glane + G, ... in order (the summation order of
// the nearest-voxel path), one pair (j, j + G) of the pair layout per loop
// step. The transform runs as packed FP32x2 instructions (the same bits as
// the scalar fma chain); with the rows in the index frame with shift 1/2
// (RowFrame) it gives f = u - 1/2 directly. rows: the group's duplicated
// pose entries, as for the nearest read.
template <int KIND, int DTYPE, int MODE, int G>
__device__ __forceinline__ void eval_tri(const SensorArgs& a, const float4* __restrict__ sxy,
                                         const float2* __restrict__ sz, int glane, int cnt,
                                         const float4* rows, float& acc) {
  for (int j = glane; j < cnt; j += 2 * G) {
    // the rows are re-read each step: they hold no registers across the corner reads
    const float4 q0 = lds_volatile(rows), q1 = lds_volatile(rows + 1), q2 = lds_volatile(rows + 2),
                 q3 = lds_volatile(rows + 3), q4 = lds_volatile(rows + 4), q5 = lds_volatile(rows + 5);
    const int pi = (j - glane) / (2 * G) * G + glane;
    const float4 xy = sxy[pi];
    const float2 zz = sz[pi];
    const float2 zx = make_float2(xy.x, xy.y), zy = make_float2(xy.z, xy.w);
    const float2 X = __ffma2_rn(make_float2(q0.x, q0.y), zx,
                                __ffma2_rn(make_float2(q0.z, q0.w), zy,
                                           __ffma2_rn(make_float2(q1.x, q1.y), zz, make_float2(q1.z, q1.w))));
    const float2 Y = __ffma2_rn(make_float2(q2.x, q2.y), zx,
                                __ffma2_rn(make_float2(q2.z, q2.w), zy,
                                           __ffma2_rn(make_float2(q3.x, q3.y), zz, make_float2(q3.z, q3.w))));
    const float2 W = __ffma2_rn(make_float2(q4.x, q4.y), zx,
                                __ffma2_rn(make_float2(q4.z, q4.w), zy,
                                           __ffma2_rn(make_float2(q5.x, q5.y), zz, make_float2(q5.z, q5.w))));
    const float2 fx = X, fy = Y, fz = W;  // rows in the frame of f = u - 1/2
    float d[2];
    bool use[2], st;
    d[0] = tri_read<KIND, DTYPE, MODE>(a, fx.x, fy.x, fz.x, st);
    use[0] = st || !a.neglect;
    if (j + G < cnt) {
      d[1] = tri_read<KIND, DTYPE, MODE>(a, fx.y, fy.y, fz.y, st);
      use[1] = st || !a.neglect;
    } else {
      d[1] = 0.f;
      use[1] = false;
    }
    accumulate<DTYPE, MODE, 2>(a, d, use, acc);
  }
}

// Resident CTAs per SM the register allocation is held to (measured on the
// 1M x 65,536 building step): with the hash index 6 for the 2- and 4-deep
// loops (40 registers; 5 or 4 were slower); with the cell-grid index 5 for
// the 4-deep loop of the single-session kernel (48 registers; packed pair
// stage, dynamic sweeps: 102.6 ms against 105.9 at 4 and 108.1 at 6) and 4
// for the batched one; 4 for the 8-deep loop (64 registers: 97.0 ms, the
// default of the cell-grid kernel, against 103.7 at 5 and 106.9 at 3); 5 for
// the trilinear read (48 registers without spills once the guard cells took
// the inside tests out: 363.9 against 369.1 ms at 4; with the earlier
// crossing-bit walk 4 was best, 596 ms against 613 at 5), 4 for its batched
// form (which would spill about 100 bytes at 48 registers).
#ifndef MCL_SENSOR_MIN_BLOCKS
#define MCL_SENSOR_MIN_BLOCKS 6
#endif
#ifndef MCL_SENSOR_MIN_BLOCKS_GRID
#define MCL_SENSOR_MIN_BLOCKS_GRID 5
#endif
#ifndef MCL_BATCH_MIN_BLOCKS_GRID
#define MCL_BATCH_MIN_BLOCKS_GRID 4
#endif
#ifndef MCL_TRI_MIN_BLOCKS
#define MCL_TRI_MIN_BLOCKS 5
#endif
#ifndef MCL_TRI_BATCH_MIN_BLOCKS
#define MCL_TRI_BATCH_MIN_BLOCKS 4
#endif
#ifndef MCL_U8_MIN_BLOCKS
#define MCL_U8_MIN_BLOCKS 4
#endif

template <int KIND, int U, bool TRI = false, bool BATCH = false>
struct MinBlocks {
  static constexpr int value = TRI ? (BATCH ? MCL_TRI_BATCH_MIN_BLOCKS : MCL_TRI_MIN_BLOCKS)
                               : U == 8 ? MCL_U8_MIN_BLOCKS
                               : KIND == kKindBrickGrid
                                   ? (BATCH ? MCL_BATCH_MIN_BLOCKS_GRID : MCL_SENSOR_MIN_BLOCKS_GRID)
                                   : MCL_SENSOR_MIN_BLOCKS;
};

// Stage one chunk of the packed scan (`bytes` from `src`) into shared memory
// with one bulk copy; every thread of the CTA calls this. Returns false (after
// recording the error and letting an in-flight copy land) if the bounded wait
// ran out.
__device__ __forceinline__ bool stage_chunk(void* sdst, uint32_t bar_s, const void* src,
                                            uint32_t bytes, uint32_t& parity, unsigned* status) {
  __syncthreads();  // every group is done with the previous chunk
  if (threadIdx.x == 0) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(bar_s, bytes);
    bulk_copy_g2s(smem_addr(sdst), src, bytes, bar_s);
  }
  const bool ok = mbar_wait_bounded(bar_s, parity);
  parity ^= 1u;
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0) {
      atomicOr(status, kDevErrTimeout);
      mbar_wait_bounded(bar_s, parity ^ 1u);
    }
    return false;
  }
  return true;
}

// Particles [p0, p0 + pn) of one session against the staged chunk c (cnt
// points at sscan, in the layout of a.layout): each lane group takes a
// particle, sums its chunk terms and writes the chunk sum to
// partial[c * P + p]. The group's slot of smat holds its particle's pose
// rows: six float4 of duplicated entries (R_i0, R_i0, R_i1, R_i1), (R_i2,
// R_i2, t_i, t_i) per row i for the packed nearest read, the three rows as
// they are for the trilinear read.
template <int KIND, int DTYPE, int MODE, int G, int U, bool PIPE, bool TRI>
__device__ __forceinline__ void process_block(const SensorArgs& a, const unsigned char* sscan,
                                              float4* smat, const float4* __restrict__ mats,
                                              float* __restrict__ partial, int P, int c, int p0,
                                              int pn, int cnt, int* pnext = nullptr) {
  constexpr int GPW = 32 / G;  // groups per warp
  constexpr int STEP = G * U;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gid = lane / G, glane = lane % G;
  const int ngroups = (blockDim.x >> 5) * GPW;
  const int full_end = (cnt / STEP) * STEP;
  const float4* sxy = reinterpret_cast<const float4*>(sscan);
  const float2* sz = reinterpret_cast<const float2*>(sscan + (size_t)a.layout.pairs(cnt) * 16);
  // pnext (shared, zero at the item's start): the warps take the item's
  // particles from this counter, GPW at a time, so a warp that drew cheap
  // particles takes more and the item's closing barrier waits less; NULL:
  // warp w takes particles w GPW, w GPW + ngroups, ...
  int i0 = warp * GPW;
  if (pnext) {
    if (lane == 0) i0 = atomicAdd(pnext, GPW);
    i0 = __shfl_sync(0xffffffffu, i0, 0);
  }
  for (; i0 < pn;) {
    const int i = i0 + gid;
    const bool gvalid = i < pn;  // (whole-warp groups: always, as i0 < pn)
    const size_t p = (size_t)p0 + (gvalid ? i : 0);
    float4* rows = smat + 6 * (warp * GPW + gid);
    if (glane < 6) {
      const float4 r = __ldg(mats + 3 * p + (glane >> 1));
      rows[glane] = (glane & 1) ? make_float4(r.z, r.z, r.w, r.w) : make_float4(r.x, r.x, r.y, r.y);
    }
    __syncwarp();
    typename Raw<DTYPE, MODE>::acc acc = 0;
    if constexpr (TRI) {
      static_assert(G == 32, "the trilinear read uses whole-warp groups");
      eval_tri<KIND, DTYPE, MODE, G>(a, sxy, sz, glane, cnt, rows, acc);
    } else {
      int base = 0;
      if (G == 32 || __all_sync(0xffffffffu, gvalid)) {
        eval_full<KIND, DTYPE, MODE, G, U, PIPE>(a, sxy, sz, full_end, glane, rows, acc);
        base = full_end;
      }
      for (; base < cnt; base += STEP)
        eval_checked<KIND, DTYPE, MODE, G, U>(a, sxy, sz, base, glane, cnt, gvalid, rows, acc);
    }
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1)
      acc = __fadd_rn(acc, __shfl_xor_sync(0xffffffffu, acc, off));
    if (glane == 0 && gvalid) partial[(size_t)c * P + p] = __fmul_rn(acc, a.store_scale);
    __syncwarp();  // every lane read the rows before the next particle's are written
    if (pnext) {
      if (lane == 0) i0 = atomicAdd(pnext, GPW);
      i0 = __shfl_sync(0xffffffffu, i0, 0);
    } else {
      i0 += ngroups;
    }
  }
}

__device__ __forceinline__ void init_barrier(uint32_t bar_s) {
  if (threadIdx.x == 0) {
    mbar_init(bar_s, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
}

// Item -> (chunk c, particle block blk). Items are numbered sweep by sweep:
// a sweep is `sweep` consecutive particle blocks (fewer in the last) times
// all K chunks, chunk-major within the sweep. sweep = nblk numbers all items
// chunk-major; a small sweep keeps the particles that resident CTAs work on
// at the same time few and (in spatial order) close together. Every item
// writes only its own partial sums, so the order changes no result.
__device__ __forceinline__ void item_coords(long long item, int nblk, int K, int sweep, int& c,
                                            int& blk) {
  const long long per = (long long)sweep * K;
  const long long s = item / per;
  const int b0 = (int)s * sweep;
  const int bs = min(sweep, nblk - b0);
  const long long r = item - s * per;
  c = (int)(r / bs);
  blk = b0 + (int)(r % bs);
}

// One session: items (chunk c, particle block) strided over a persistent grid.
template <int KIND, int DTYPE, int MODE, int G, int U, bool PIPE, bool TRI>
__global__ void __launch_bounds__(256, (MinBlocks<KIND, U, TRI>::value)) k_sensor(const SensorArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int sbytes = a.layout.smem_bytes();
  const uint32_t bar_s = smem_addr(smem + sbytes);
  float4* smat = reinterpret_cast<float4*>(smem + sbytes + 16);
  init_barrier(bar_s);
  int loaded = -1;
  uint32_t parity = 0;
  if (a.queue) {
    // Dynamic order: thread 0 takes the next item from the device counter one
    // item ahead; the barrier at the top of each step publishes it and is the
    // point where every warp is done with the previous item.
    // The item's particles go to the warps through a shared counter, one per
    // item parity: counter (k + 1) & 1 is reset during item k, when no warp
    // uses it any more (all passed the barrier that closed item k - 1).
    __shared__ long long s_next[2];
    __shared__ int s_pnext[2];
    if (threadIdx.x == 0) {
      s_next[0] = (long long)atomicAdd(a.queue, 1ull);
      s_pnext[0] = 0;
    }
    for (int k = 0;; ++k) {
      __syncthreads();
      const long long item = s_next[k & 1];
      if (item >= a.n_items) break;
      if (threadIdx.x == 0) {
        s_next[(k + 1) & 1] = (long long)atomicAdd(a.queue, 1ull);
        s_pnext[(k + 1) & 1] = 0;
      }
      int c, blk;
      item_coords(item, a.nblk, a.K, a.sweep, c, blk);
      const int p0 = blk * a.ppi;
      const int pn = min(a.ppi, a.P - p0);
      const int cnt = min(a.chunk, a.N - c * a.chunk);
      if (c != loaded) {
        if (!stage_chunk(smem, bar_s, reinterpret_cast<const unsigned char*>(a.scan) +
                                          a.layout.chunk_offset(c),
                         a.layout.chunk_bytes(cnt), parity, a.status))
          return;
        loaded = c;
      }
      process_block<KIND, DTYPE, MODE, G, U, PIPE, TRI>(a, smem, smat, a.mats, a.partial, a.P, c, p0,
                                                        pn, cnt, &s_pnext[k & 1]);
    }
    return;
  }
  for (long long item = blockIdx.x; item < a.n_items; item += gridDim.x) {
    int c, blk;
    item_coords(item, a.nblk, a.K, a.sweep, c, blk);
    const int p0 = blk * a.ppi;
    const int pn = min(a.ppi, a.P - p0);
    const int cnt = min(a.chunk, a.N - c * a.chunk);
    if (c != loaded) {  // uniform over the CTA: every thread walks the same items
      if (!stage_chunk(smem, bar_s, reinterpret_cast<const unsigned char*>(a.scan) +
                                        a.layout.chunk_offset(c),
                       a.layout.chunk_bytes(cnt), parity, a.status))
        return;
      loaded = c;
    }
    process_block<KIND, DTYPE, MODE, G, U, PIPE, TRI>(a, smem, smat, a.mats, a.partial, a.P, c, p0,
                                                      pn, cnt);
  }
}

// Many sessions whose maps share kind, storage type, geometry and score
// constants: items (session, chunk, particle block) of uneven sizes, listed as
// segments of consecutive items of one session (each session's items in its
// own sweep order; sessions on one map interleaved sweep by sweep, see
// item_segments). A device counter hands them out in
// order when b.base.queue is set (as in k_sensor), else they are strided over
// the grid. Each session reads its own map (values and brick index from its
// table entry; the rest of the view is the group's) and gets the results the
// single-session kernel gives.
template <int KIND, int DTYPE, int MODE, int G, int U, bool PIPE, bool TRI>
__device__ __forceinline__ bool batch_item(const BatchArgs& b, long long item, unsigned char* smem,
                                           uint32_t bar_s, float4* smat, long long& loaded,
                                           uint32_t& parity, int* pnext) {
  const SensorArgs& a = b.base;
  int lo = 0, hi = b.n_segs - 1;  // segment that holds `item`
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(&b.segs[mid].begin) <= item) lo = mid; else hi = mid - 1;
  }
  const int ses = __ldg(&b.segs[lo].session);
  const BatchSession& S = b.sessions[ses];
  const long long local = __ldg(&b.segs[lo].local0) + (item - __ldg(&b.segs[lo].begin));
  int c, blk;
  item_coords(local, S.nblk, S.K, S.sweep, c, blk);
  const int ppi = S.ppi, P = S.P;
  const int p0 = blk * ppi;
  const int pn = min(ppi, P - p0);
  const int cnt = min(a.chunk, S.N - c * a.chunk);
  const long long key = ((long long)ses << 32) | (unsigned)c;
  if (key != loaded) {
    if (!stage_chunk(smem, bar_s, reinterpret_cast<const unsigned char*>(S.scan) +
                                      a.layout.chunk_offset(c),
                     a.layout.chunk_bytes(cnt), parity, a.status))
      return false;
    loaded = key;
  }
  SensorArgs as = a;  // the group's arguments with this session's map
  as.map.values = S.values;
  as.map.grid = S.grid;
  as.map.table = S.table;
  as.map.n_slots = S.n_slots;
  as.map.hash_mask = S.hash_mask;
  as.map.hash_shift = S.hash_shift;
  as.map.max_probe = S.max_probe;
  process_block<KIND, DTYPE, MODE, G, U, PIPE, TRI>(as, smem, smat, S.mats, S.partial, P, c, p0, pn,
                                                    cnt, pnext);
  return true;
}

template <int KIND, int DTYPE, int MODE, int G, int U, bool PIPE, bool TRI>
__global__ void __launch_bounds__(256, (MinBlocks<KIND, U, TRI, true>::value)) k_sensor_batch(const BatchArgs b) {
  const SensorArgs& a = b.base;
  extern __shared__ __align__(128) unsigned char smem[];
  const int sbytes = a.layout.smem_bytes();
  const uint32_t bar_s = smem_addr(smem + sbytes);
  float4* smat = reinterpret_cast<float4*>(smem + sbytes + 16);
  init_barrier(bar_s);
  long long loaded = -1;
  uint32_t parity = 0;
  if (a.queue) {  // dynamic order, as in k_sensor
    __shared__ long long s_next[2];
    __shared__ int s_pnext[2];
    if (threadIdx.x == 0) {
      s_next[0] = (long long)atomicAdd(a.queue, 1ull);
      s_pnext[0] = 0;
    }
    for (int k = 0;; ++k) {
      __syncthreads();
      const long long item = s_next[k & 1];
      if (item >= b.n_items) break;
      if (threadIdx.x == 0) {
        s_next[(k + 1) & 1] = (long long)atomicAdd(a.queue, 1ull);
        s_pnext[(k + 1) & 1] = 0;
      }
      if (!batch_item<KIND, DTYPE, MODE, G, U, PIPE, TRI>(b, item, smem, bar_s, smat, loaded, parity,
                                                          &s_pnext[k & 1]))
        return;
    }
    return;
  }
  for (long long item = blockIdx.x; item < b.n_items; item += gridDim.x)
    if (!batch_item<KIND, DTYPE, MODE, G, U, PIPE, TRI>(b, item, smem, bar_s, smat, loaded, parity,
                                                        nullptr))
      return;
}

template <int KIND, int DTYPE, int MODE, int G, int U, bool PIPE, bool TRI = false>
void* kernel_ptr(bool batch) {
  return batch ? reinterpret_cast<void*>(&k_sensor_batch<KIND, DTYPE, MODE, G, U, PIPE, TRI>)
               : reinterpret_cast<void*>(&k_sensor<KIND, DTYPE, MODE, G, U, PIPE, TRI>);
}

// Kernel for one storage type, or NULL for an unsupported shape. Shapes:
// G = 32 with U = 2 or 4 (plain or pipelined) or U = 8 (plain); G = 16 or 8
// with U = 4 (plain); the trilinear read with G = 32.
template <int KIND, int DTYPE, int MODE>
void* pick_shape(const SensorShape& sh, bool batch) {
  if (sh.interp) return sh.lanes == 32 ? kernel_ptr<KIND, DTYPE, MODE, 32, 2, false, true>(batch) : nullptr;
  const bool pipe = sh.pipeline != 0;
  if (sh.lanes == 32) {
    if (sh.unroll == 2) return pipe ? kernel_ptr<KIND, DTYPE, MODE, 32, 2, true>(batch)
                                    : kernel_ptr<KIND, DTYPE, MODE, 32, 2, false>(batch);
    if (sh.unroll == 4) return pipe ? kernel_ptr<KIND, DTYPE, MODE, 32, 4, true>(batch)
                                    : kernel_ptr<KIND, DTYPE, MODE, 32, 4, false>(batch);
    if (sh.unroll == 8 && !pipe) return kernel_ptr<KIND, DTYPE, MODE, 32, 8, false>(batch);
    return nullptr;
  }
  if (pipe || sh.unroll != 4) return nullptr;
  if (sh.lanes == 16) return kernel_ptr<KIND, DTYPE, MODE, 16, 4, false>(batch);
  if (sh.lanes == 8) return kernel_ptr<KIND, DTYPE, MODE, 8, 4, false>(batch);
  return nullptr;
}

// Score maps (FP16 or FP32 values that are already scores): the plain
// shapes, nearest-voxel read only.
template <int KIND, int DTYPE>
void* pick_score_shape(const SensorShape& sh, bool batch) {
  if (sh.interp || sh.pipeline) return nullptr;
  if (sh.lanes == 32) {
    if (sh.unroll == 2) return kernel_ptr<KIND, DTYPE, kModeScore, 32, 2, false>(batch);
    if (sh.unroll == 4) return kernel_ptr<KIND, DTYPE, kModeScore, 32, 4, false>(batch);
    if (sh.unroll == 8) return kernel_ptr<KIND, DTYPE, kModeScore, 32, 8, false>(batch);
    return nullptr;
  }
  if (sh.unroll != 4) return nullptr;
  if (sh.lanes == 16) return kernel_ptr<KIND, DTYPE, kModeScore, 16, 4, false>(batch);
  if (sh.lanes == 8) return kernel_ptr<KIND, DTYPE, kModeScore, 8, 4, false>(batch);
  return nullptr;
}

// Kernel of one map kind and storage type for a score mode and shape, or NULL.
template <int KIND, int DTYPE>
void* pick_kind(int mode, const SensorShape& sh, bool batch) {
  if (mode == kModeScore) {
    if constexpr (DTYPE == MCL_I16) return nullptr;
    else return pick_score_shape<KIND, DTYPE>(sh, batch);
  }
  return mode == MCL_LOGPROD ? pick_shape<KIND, DTYPE, MCL_LOGPROD>(sh, batch)
                             : pick_shape<KIND, DTYPE, MCL_SUM>(sh, batch);
}

}  // namespace sensor
}  // namespace mcl
