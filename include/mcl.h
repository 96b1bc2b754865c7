/*
 * mcl.h - C ABI of the GB300 library for the 6D Monte Carlo Localization
 * sensor update in TSDF maps (Eisoldt, Mock, Porrmann, Wiemann, "Towards 6D
 * MCL for LiDARs in 3D TSDF Maps on Embedded Systems with GPUs").
 *
 * Conventions for every call:
 *  - The return value is an mcl_status; MCL_OK is 0. On failure,
 *    mcl_last_error() returns a message for the calling thread. Nothing
 *    throws across this boundary.
 *  - Array arguments marked (device) are caller-owned CUDA device pointers
 *    on the current device; (host) are caller-owned host pointers. The
 *    library never frees caller memory and keeps no reference to it after
 *    the call returns (device arrays are read or written by work enqueued on
 *    `stream`, so they must stay valid until that work completes).
 *  - `stream` is a cudaStream_t (NULL = legacy default stream). Calls are
 *    asynchronous with respect to the host unless stated otherwise; errors of
 *    the device work itself are reported by mcl_sync() or by a later call.
 *  - Poses are FP32 rows (x, y, z, roll, pitch, yaw): the state
 *    s = (x, y, z, phi, psi, theta) of Sec. III, Eq. 2, with
 *    R = Rz(yaw) Ry(pitch) Rx(roll) mapping the sensor frame to the map frame.
 *  - Scan points are FP32 rows (x, y, z) in the sensor frame.
 *  - Scratch memory: the compute calls keep a library-owned device workspace
 *    per (device, stream); it grows with cudaMalloc on first use at a larger
 *    size, so call once with the largest sizes before capturing a stream
 *    into a CUDA graph.
 */
#ifndef MCL_H_
#define MCL_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t mcl_status;
#define MCL_OK 0
#define MCL_EINVAL 1      /* bad argument: size, pointer, alignment, value */
#define MCL_ENOMEM 2      /* device or host allocation failed / over budget */
#define MCL_EBUSY 3       /* no free slot (serving) */
#define MCL_ETIMEDOUT 4   /* wait ran out of time */
#define MCL_ECUDA 5       /* a CUDA runtime call failed */
#define MCL_EINTERNAL 6   /* a kernel reported an internal error (status word) */

typedef void* mcl_stream_t; /* cudaStream_t */

/* Thread-local message of the last failed call on this thread ("" if none). */
const char* mcl_last_error(void);

/* Library version as an integer (major * 10000 + minor * 100 + patch). */
int32_t mcl_version(void);

/* Waits for `stream`, then reports any CUDA error and any internal error a
 * kernel of this library recorded in its device status word (a bounded wait
 * that ran out, an index check that failed); the status word is cleared. */
mcl_status mcl_sync(mcl_stream_t stream);

/* Self-test of the library's failure path (the paper has no counterpart):
 * launches one CTA that waits, with the same bounded wait the sensor kernel
 * uses for its scan copies, on a barrier phase that nothing completes. The
 * wait gives up after about one second, the kernel records the timeout in
 * the device status word and returns; this call waits for it (synchronous),
 * checks that the timeout was recorded, clears the status word and writes
 * the time the kernel waited to waited_s (host, may be NULL). MCL_OK if the
 * failure path worked; MCL_EINTERNAL if the timeout was not recorded. */
mcl_status mcl_selftest_wait(double* waited_s, mcl_stream_t stream);

/* ------------------------------------------------------------------ maps */

enum { MCL_MAP_DENSE = 0, MCL_MAP_BRICK = 1 };
enum { MCL_F32 = 0, MCL_F16 = 1, MCL_I16 = 2 };
enum { MCL_LAYOUT_LINEAR = 0, MCL_LAYOUT_BLOCK4 = 1 };
enum { MCL_INDEX_AUTO = 0, MCL_INDEX_HASH = 1, MCL_INDEX_GRID = 2 };

/* TSDF map description (Sec. III: a TSDF volume; the sparse form keeps fine
 * blocks only where values lie within the truncation distance, every other
 * cell reads the truncation value).
 *
 * Voxel (ix, iy, iz) covers [o + i r, o + (i + 1) r) on each axis. A point
 * falls in voxel i_k = floor(u_k), inside iff 0 <= u_k < dims_k on every
 * axis, with u_k its index coordinate in FP32:
 *  - a world point x (mcl_map_lookup): u_k = (x_k - o_k) * inv_voxel in two
 *    FP32 roundings;
 *  - a scan point z seen from a particle (the sensor update): the pose rows
 *    [R | t] are taken into the map's index frame, R'_kj = R_kj * inv_voxel
 *    and t'_k = (t_k - o_k) * inv_voxel, each evaluated in FP64 (R from the
 *    FP64 rotation of mcl_pose_to_matrix) and rounded to FP32 once, then
 *    u_k = fma(R'_k0, z_0, fma(R'_k1, z_1, fma(R'_k2, z_2, t'_k))) in FP32.
 * dims_k lie in [1, 2^23] (the kernels take floor(u) from the bits of a
 * round-down u + 2^23, exact below 2^23); larger dims are EINVAL.
 * Values are the signed distance at the voxel centre, clamped to
 * [-truncation, truncation], stored as FP32, FP16 or scaled int16
 * (q stands for q * truncation / 32767).
 *
 * DENSE: values[(iz * dims[1] + iy) * dims[0] + ix], at most 2^31 voxels.
 * BRICK: 16^3 bricks; dims multiples of 16; brick b (coordinates
 *        brick_coords[3b..3b+2] = (bx, by, bz) in brick units) holds
 *        values[b * 4096 + (lz * 16 + ly) * 16 + lx]; a voxel in no listed
 *        brick reads +truncation. At most 2^31 - 1 bricks and 2^32 - 2
 *        brick cells; duplicated or out-of-range coordinates are EINVAL.
 * inv_voxel = 0 lets the library use (float)(1.0 / voxel).
 * device_layout (BRICK) chooses how the library stores each brick on the
 * device: MCL_LAYOUT_LINEAR keeps the x-fastest order, MCL_LAYOUT_BLOCK4
 * stores 4x4x4 blocks (block-major, each block z-major) so that neighbouring
 * voxels in x and y share memory sectors. host_values are always x-fastest;
 * results do not depend on the layout.
 * index (BRICK) chooses how a brick cell finds its brick (the coarse level
 * of Sec. III's coarse/fine split): MCL_INDEX_GRID keeps a dense array of
 * one 32-bit slot per brick cell (4 bytes x cells; neighbouring cells are
 * neighbours in memory), MCL_INDEX_HASH an open-addressing hash table of
 * 8-byte entries, at least 4 per brick (for sparse maps of a huge extent).
 * MCL_INDEX_AUTO takes the grid for the linear layout when it needs at most
 * 512 MB and the map has at most 2^20 bricks, else the hash. The grid is
 * only built with MCL_LAYOUT_LINEAR and for at most 2^20 bricks (its kernels
 * address values with 32-bit indices); MCL_INDEX_GRID beyond that is EINVAL.
 * Results do not depend on the index.
 * Device storage the library chooses (no result depends on it): with the
 * grid index, each brick's values are rotated by its cell coordinates (voxel
 * (ix, iy, iz) at (ix + 16 iy + 256 iz) mod 4096 of its brick) and the grid
 * is padded by one empty cell per axis; dense grids are stored in tiles of
 * 8 x 4 x 1 voxels, padded to whole tiles (device_bytes of mcl_map_info
 * counts the padding). */
typedef struct mcl_map_desc {
  uint32_t struct_size; /* sizeof(mcl_map_desc) */
  int32_t kind;         /* MCL_MAP_DENSE or MCL_MAP_BRICK */
  int32_t dtype;        /* MCL_F32, MCL_F16 or MCL_I16 */
  float origin[3];      /* map-frame coordinates of the grid corner (m) */
  float voxel;          /* voxel edge r (m), > 0 */
  float inv_voxel;      /* 1 / r as used by the index rule, or 0 */
  float truncation;     /* tau (m), > 0 */
  int64_t dims[3];      /* grid size in voxels (x, y, z) */
  int64_t n_bricks;     /* BRICK: number of bricks */
  const int32_t* brick_coords; /* BRICK: (host) n_bricks x 3 int32 */
  int32_t device_layout;       /* BRICK: MCL_LAYOUT_LINEAR or MCL_LAYOUT_BLOCK4 */
  int32_t index;               /* BRICK: MCL_INDEX_AUTO (0), MCL_INDEX_HASH or MCL_INDEX_GRID */
} mcl_map_desc;

typedef struct mcl_map_s* mcl_map_t;

/* Uploads a map to the current device. `host_values` (host) holds the values
 * in the layout above and the dtype given. The map owns its device memory.
 * EINVAL for a bad description, ENOMEM if the device is out of memory. */
mcl_status mcl_map_create(const mcl_map_desc* desc, const void* host_values, mcl_map_t* out);

/* Frees the map's device memory (synchronises the device first). NULL is a no-op. */
mcl_status mcl_map_destroy(mcl_map_t map);

typedef struct mcl_map_info {
  uint32_t struct_size;
  int64_t device_bytes;   /* values + index bytes held on the device */
  int64_t n_bricks;       /* BRICK: bricks stored; DENSE: 0 */
  int64_t hash_capacity;  /* BRICK with the hash index: table entries (power of two) */
  int32_t hash_max_probe; /* BRICK with the hash index: longest probe sequence of a stored brick */
  int32_t device;         /* CUDA device that holds the map */
  float score_sigma;      /* > 0: a score map made for this sigma (mcl_map_create_score) */
  float score_outside;    /* score map: the score read where nothing is stored */
  int32_t index;          /* BRICK: MCL_INDEX_HASH or MCL_INDEX_GRID; DENSE: 0 */
  int32_t reserved;
  int64_t index_bytes;    /* BRICK: device bytes of the brick index */
} mcl_map_info;

mcl_status mcl_map_get_info(mcl_map_t map, mcl_map_info* out);

/* Score map (Sec. III: all entries of the map can be computed before the
 * scans, so the exponential of Eq. 3 is not evaluated per point). Makes, on
 * the source map's device, a map of the same kind, grid and bricks whose
 * values are the scores s = exp(-d^2 / (2 sigma^2)) of the source's values d
 * (dequantised; computed in FP64 and rounded once, to nearest even, to
 * dtype MCL_F16 or MCL_F32); a point where nothing is stored reads the score
 * of +truncation. A sensor update on a score map must use mode MCL_SUM, the
 * same sigma_hit (bit for bit) and no MCL_TRILINEAR; it sums the stored
 * scores: L = log(k * sum s), k the constant of Eq. 3. mcl_map_lookup on a
 * score map returns the scores. EINVAL: sigma not finite and > 0, another
 * dtype, a score map as source. The new map owns its memory. */
mcl_status mcl_map_create_score(mcl_map_t src, float sigma_hit, int32_t dtype, mcl_map_t* out);

/* Map query at N world points (device, N x 3 FP32): out_index (device, N
 * int64) gets the linear voxel index (iz * dims[1] + iy) * dims[0] + ix or -1
 * outside the grid; out_value (device, N FP32) the value read there,
 * dequantised, +truncation outside the grid or in a voxel of no brick. Either
 * output may be NULL. Uses the world-point index rule (Sec. III look-up). */
mcl_status mcl_map_lookup(mcl_map_t map, const float* points, int64_t N, int64_t* out_index,
                          float* out_value, mcl_stream_t stream);

/* ------------------------------------------------------------------ sensor update */

enum { MCL_LOGPROD = 0, MCL_SUM = 1 };
#define MCL_NEGLECT_OUTSIDE 1u /* points without a stored value are left out */
#define MCL_TRILINEAR 2u       /* read the TSDF by trilinear interpolation (see below) */

/* Sensor-model parameters (Sec. III, Eq. 3).
 * mode LOGPROD: per-point score -d^2 / (2 sigma^2) (log of Eq. 3 without its
 *   constant), particle log-weight L = sum of scores (product of p_hit).
 * mode SUM: per-point score p_hit of Eq. 3, L = log(sum of p_hit).
 * A point outside the grid or in a voxel of no brick reads d = +truncation
 * (Sec. III clamping), or with MCL_NEGLECT_OUTSIDE contributes nothing.
 * MCL_TRILINEAR (Sec. III: a pseudo-continuous value by interpolation)
 * replaces the containing voxel's value by the trilinear interpolation of the
 * eight voxel centres around the point: with f = u - 1/2, formed like u of
 * the sensor update's index rule with t'_k = (t_k - o_k) * inv_voxel - 1/2
 * (FP64, one FP32 rounding), corners i0 + {0, 1} per axis, i0 = floor(f), weights
 * a = f - i0 and 1 - a; a corner outside the grid or in no brick reads
 * +truncation, and the point counts as stored (for MCL_NEGLECT_OUTSIDE) if
 * any corner is. Interpolated in FP32 along x, then y, then z. Needs
 * lanes_per_particle 0 or 32; unroll and pipeline are ignored.
 * points_per_chunk and lanes_per_particle fix the FP32 summation order
 * (points of one particle are split in chunks of points_per_chunk, each
 * summed by lanes_per_particle lanes and a shuffle tree, chunks added in
 * order); 0 selects the defaults 2048 and 32. Results are bit-reproducible
 * for equal (points_per_chunk, lanes_per_particle, scan_rings). */
typedef struct mcl_sensor_params {
  uint32_t struct_size;       /* sizeof(mcl_sensor_params) */
  float sigma_hit;            /* sigma of Eq. 3 (m), > 0 */
  int32_t mode;               /* MCL_LOGPROD or MCL_SUM */
  uint32_t flags;             /* MCL_NEGLECT_OUTSIDE or 0 */
  int32_t points_per_chunk;   /* 0 or a multiple of 32 in [32, 8192] */
  int32_t lanes_per_particle; /* 0, 8, 16 or 32 */
  int32_t particles_per_item; /* launch shape hint, 0 = auto (no effect on results) */
  int32_t unroll;             /* 0 (auto), 2, 4 or 8: look-ups in flight per lane (hint; lane
                                 groups narrower than 32 always use 4; no effect on results) */
  int32_t pipeline;           /* 0 (auto), 1 off, 2 on: overlap the next step's index look-ups
                                 with this step's gathers (hint; only for unroll 2 or 4 with
                                 32 lanes; no effect on results) */
  int32_t particle_order;     /* 0 (auto), 1 as given, 2 spatial (Morton-ordered buckets over
                                 the map extent): the order particles are evaluated in;
                                 no effect on results */
  int32_t item_order;         /* 0 (auto), 1 chunk-major, 2 sweeps, 3 dynamic sweeps: the
                                 order of the (point chunk, particle block) work items.
                                 Sweeps walk a few particle blocks through every chunk at a
                                 time, so the CTAs working at the same time read the map
                                 around few (spatially ordered) particles; in 2 each
                                 resident CTA keeps one chunk (static striding), in 3 a
                                 device counter hands the items out in order to whichever
                                 CTA is free (which re-stages its item's chunk), so the
                                 items in flight stay within about one sweep whatever each
                                 chunk costs. Auto takes 3 for the nearest read of a brick
                                 map once there are at least two items per resident CTA,
                                 else 1. No effect on results */
  int32_t scan_rings;         /* 0: the scan's points are staged in the order given. R > 0:
                                 the scan is R rings of N / R points each, ring after ring;
                                 the library stages it in patches of 4 rings x 8 neighbouring
                                 points, so that the 32 lanes of a warp take one 4 x 8 patch
                                 and their gathers share more DRAM sectors. It pays where
                                 the particles are spread over the map (global
                                 localisation, DRAM-bound: 86.0 -> 84.1 ms for 1M uniform
                                 particles x 64 rings x 1,024 points) and costs where they
                                 have converged (tracking, served from L1 and L2: the
                                 patch spans more cache lines than a run along one ring;
                                 +4 % on int16 bricks, up to 1.9x on a dense FP16 map).
                                 Applied when R divides N, R is a multiple of 4 and N / R
                                 of 8, else the order given. Sets the order points are
                                 summed in, like points_per_chunk; < 0 is EINVAL */
} mcl_sensor_params;

/* Sensor update of P particles (device, P x 6 FP32) against one scan
 * (device, N x 3 FP32): every scan point is moved into the map frame by
 * each particle's pose, the TSDF is read at the voxel that contains it, the
 * score is summed per particle (Sec. III, Eq. 3; Sec. V-B). Writes the
 * log-weights to logw (device, P FP32) and, if w is not NULL, the normalised
 * weights w_p = exp(L_p - M) / sum_q exp(L_q - M), M = max L (device, P FP32).
 * logw may be NULL if w is not. Pointers need 4-byte alignment.
 * EINVAL: P or N outside [1, 2^31 - 1], sigma not finite and > 0, bad
 * params, both outputs NULL. Non-finite pose values are not checked: their
 * points fall outside the grid. */
mcl_status mcl_sensor_update(mcl_map_t map, const float* particles, int64_t P, const float* scan,
                             int64_t N, const mcl_sensor_params* params, float* logw, float* w,
                             mcl_stream_t stream);

/* Normalisation alone (Sec. V-A: weights summed for normalisation): w_p =
 * exp(L_p - M) / S with M = max L, S = sum exp(L - M) in FP32, reduced in a
 * fixed order. If M is not finite (no particle scored) every w_p = 1 / P.
 * out_stats (device, 2 FP32, may be NULL) gets (M, S); S = 0 flags that
 * degenerate case. */
mcl_status mcl_normalise(const float* logw, int64_t P, float* w, float* out_stats,
                         mcl_stream_t stream);

/* Pose estimate of a weighted particle set (Sec. III: the pose is the
 * weighted average of the particles or the particle with the highest weight;
 * Sec. V: after the weights, the weighted sum of the poses). Written to
 * device memory by mcl_pose_estimate and mcl_sensor_update_estimate; sums in
 * FP64 in a fixed order (bit-reproducible), quaternions of the particles in
 * FP32. With W = sum of w_p:
 *   mean_pose     sum w_p s_p / W, each of the six pose components as a
 *                 number (the literal weighted average: its angles are
 *                 meaningful only while the particles' angles stay away from
 *                 the +-pi wrap);
 *   quat          (w, x, y, z): unit eigenvector of the largest eigenvalue of
 *                 Q = sum w_p q_p q_p^T / W, q_p the quaternion of R(s_p) -
 *                 the rotation R minimising sum w_p ||R - R(s_p)||_F^2 (no
 *                 wrap problem); sign: first non-zero component positive;
 *   rpy           that rotation as (roll, pitch, yaw), R = Rz Ry Rx (from the
 *                 FP64 quaternion, angles evaluated in FP32);
 *   concentration that eigenvalue, in [1/4, 1]: 1 iff all weighted
 *                 rotations coincide;
 *   n_eff         W^2 / sum w_p^2 (0 if W = 0);
 *   argmax        lowest p with the largest w_p (NaN weights ignored; -1 if
 *                 all are NaN), best_pose its row, best_w its weight.
 * W = 0 (or non-finite sums) gives NaN means, quat, rpy and concentration. */
typedef struct mcl_estimate {
  double weight_sum;
  double n_eff;
  double mean_pose[6];
  double quat[4];
  double rpy[3];
  double concentration;
  int64_t argmax;
  float best_pose[6];
  float best_w;
  int32_t reserved;
} mcl_estimate;

/* Estimate from given weights: particles (device, P x 6 FP32), w (device, P
 * FP32, normalised or not), out (device, one mcl_estimate, 8-byte aligned).
 * EINVAL: P outside [1, 2^31 - 1], a NULL pointer, misalignment. */
mcl_status mcl_pose_estimate(const float* particles, const float* w, int64_t P, mcl_estimate* out,
                             mcl_stream_t stream);

/* mcl_sensor_update with the pose estimate fused into the normalisation
 * pass (the estimate of the normalised weights it writes, identical bit for
 * bit to mcl_pose_estimate on those weights). w and out are required. */
mcl_status mcl_sensor_update_estimate(mcl_map_t map, const float* particles, int64_t P,
                                      const float* scan, int64_t N,
                                      const mcl_sensor_params* params, float* logw, float* w,
                                      mcl_estimate* out, mcl_stream_t stream);

/* Pose rows -> [R | t] (device, P x 12 FP32, rows [R_i0 R_i1 R_i2 t_i]):
 * R = Rz(yaw) Ry(pitch) Rx(roll) evaluated in FP64 in the fixed order
 * a = cy*sp, b = sy*sp, R = [[cy*cp, a*sr - sy*cr, a*cr + sy*sr],
 * [sy*cp, b*sr + cy*cr, b*cr - cy*sr], [-sp, cp*sr, cp*cr]], each entry
 * rounded to FP32. The sensor update takes its rows from the same FP64
 * rotation, in the map's index frame (see the map description). */
mcl_status mcl_pose_to_matrix(const float* particles, int64_t P, float* out_mat,
                              mcl_stream_t stream);

/* Launch plan the sensor update would use for these sizes on the current
 * device (no work is enqueued). workspace_bytes is the scratch the call
 * needs; points_per_chunk, lanes_per_particle and scan_rings fix the
 * summation order. */
typedef struct mcl_sensor_plan {
  uint32_t struct_size;
  int32_t points_per_chunk, lanes_per_particle, particles_per_item, unroll, pipeline;
  int32_t particle_order;   /* 1 as given, 2 spatial */
  int32_t threads, grid, blocks_per_sm, num_sms;
  int64_t n_items;          /* (chunk, particle block) work items */
  int64_t workspace_bytes;  /* library scratch for one call */
  int32_t item_order;       /* 1 chunk-major, 2 sweeps, 3 dynamic sweeps */
  int32_t blocks_per_sweep; /* particle blocks per sweep (all blocks: chunk-major) */
} mcl_sensor_plan;

mcl_status mcl_sensor_plan_get(mcl_map_t map, int64_t P, int64_t N,
                               const mcl_sensor_params* params, mcl_sensor_plan* out);

/* ------------------------------------------------------------------ autotuner */

/* Autotuner of the launch shape (the paper has none; the shape is a GB300
 * choice). Times candidates with CUDA events on the caller's particles (the
 * first max_particles of them) and scan, by coordinate descent from base's
 * shape (0 fields: the library's defaults) over particles per item, unroll,
 * pipeline, particle order and item order, and with tune_summation = 1 also
 * over points_per_chunk in {1024, 2048, 4096} and lanes_per_particle in
 * {32, 16} (32 only for MCL_TRILINEAR; those two fix the FP32 summation
 * order: keep a tuned pair fixed for a session). The winner is appended to the JSON-lines cache at
 * cache_path (NULL: $MCL_TUNE_CACHE) when use_cache = 1, keyed by GPU name,
 * map kind, layout, storage type, score mode (a score map's own), flags,
 * whether base's scan_rings applies to N, and the power-of-two buckets of P
 * and N; a later call with the same key returns it without timing. Synchronous:
 * returns after timing. Allocates a scratch buffer of max_particles floats. */
typedef struct mcl_tune_params {
  uint32_t struct_size;
  int32_t max_particles;   /* 0 = 65536 */
  int32_t repeats;         /* timed runs per candidate, best kept; 0 = 3 */
  int32_t use_cache;       /* 1: read and append the cache file */
  int32_t tune_summation;  /* 1: also tune points_per_chunk and lanes_per_particle */
  const char* cache_path;
} mcl_tune_params;

typedef struct mcl_tune_result {
  uint32_t struct_size;
  mcl_sensor_params best;  /* base with the tuned fields filled in */
  double best_ms;          /* per call on the timing subset */
  double default_ms;       /* the base shape on the same subset */
  int32_t candidates;      /* shapes timed (0 when served from the cache) */
  int32_t from_cache;
} mcl_tune_result;

mcl_status mcl_autotune(mcl_map_t map, const float* particles, int64_t P, const float* scan,
                        int64_t N, const mcl_sensor_params* base, const mcl_tune_params* tune,
                        mcl_tune_result* out, mcl_stream_t stream);

/* ------------------------------------------------------------------ resampling */

/* Systematic resampling (Sec. III: a new set drawn from the old one in
 * proportion to the weights) with offset r in [0, 1):
 *   q_p = rint(w_p * 2^52) * 2^-52, C_p = q_0 + ... + q_p (FP64, exact while
 *   the total stays below 2, i.e. for normalised weights), S = C_{P-1},
 *   t_j = ((j + r) / P) * S, idx_j = min{p : C_p > t_j}, else the last p
 *   with q_p > 0. All-zero weights give idx_j = j.
 * w (device, P FP32, >= 0), idx (device, P int32). If particles_in is not
 * NULL, particles_out[j] = particles_in[idx_j] (device, P x 6 FP32; must not
 * alias). EINVAL: P outside [1, 2^31 - 1], r outside [0, 1), idx NULL. */
mcl_status mcl_resample(const float* w, int64_t P, double r, int32_t* idx,
                        const float* particles_in, float* particles_out, mcl_stream_t stream);

/* Allocation-free variant of mcl_resample (the paper has no counterpart; it
 * exists for callers that may not allocate device memory: real-time control
 * loops that forbid allocation after start-up, since cudaMalloc and cudaFree
 * can block and cudaFree synchronises the device, and plug-ins whose host
 * application owns every device allocation). Same arguments, results and
 * errors as mcl_resample (indices identical bit for bit), but its scratch is
 * a fixed static device array inside the library, so P is limited to
 * [1, 1048576] (2^20; larger P is EINVAL) and every GPU that loads the
 * library holds that array (about 8.4 MB) until the process exits. Calls
 * allocate nothing. The first call on each device looks up the array's
 * device address with that device current; make that first call before
 * capturing a stream into a graph. All calls on a device share the one
 * array: calls whose work overlaps on the GPU (different streams, or
 * different host threads) race and give wrong indices; serialise them. */
mcl_status mcl_resample_noalloc(const float* w, int64_t P, double r, int32_t* idx,
                                const float* particles_in, float* particles_out,
                                mcl_stream_t stream);

/* ------------------------------------------------------------------ motion update */

/* Motion update (Sec. III: the motion model is applied to every particle).
 * Increment u = delta + sigma * n per particle, n six standard normals from
 * Philox4x32-10 (key = seed, counter = (b, particle, step_lo, step_hi),
 * b = 0, 1, 2) and Box-Muller in FP64; then t' = t + R(s) u_t,
 * R' = R(s) R(u_r), read back as roll = atan2(R'21, R'22),
 * pitch = asin(-R'20), yaw = atan2(R'10, R'00) in [-pi, pi).
 * particles (device, P x 6 FP32) are updated in place; delta and sigma are
 * host arrays of 6. EINVAL: P outside [1, 2^31 - 1], a sigma < 0 or not finite. */
mcl_status mcl_motion_update(float* particles, int64_t P, const float delta[6],
                             const float sigma[6], uint64_t seed, uint64_t step,
                             mcl_stream_t stream);

/* ------------------------------------------------------------------ batched update */

/* One session of a batched step: a robot's particle set and its latest scan
 * against its map, with the outputs of mcl_sensor_update and, if
 * resample_idx is not NULL, of mcl_resample (offset set per run with
 * mcl_batch_set_offsets), and if estimate is not NULL, of
 * mcl_sensor_update_estimate. All pointers are device pointers that stay fixed
 * for the life of the batch; the caller writes new particles and scans into
 * the same buffers between runs. */
typedef struct mcl_session_update {
  uint32_t struct_size;    /* sizeof(mcl_session_update) */
  mcl_map_t map;
  const float* particles;  /* P x 6 */
  int64_t P;
  const float* scan;       /* N x 3 */
  int64_t N;
  float sigma_hit;
  int32_t mode;            /* MCL_LOGPROD or MCL_SUM */
  uint32_t flags;          /* MCL_NEGLECT_OUTSIDE or 0 */
  float* logw;             /* P, may be NULL if w is not */
  float* w;                /* P, may be NULL */
  int32_t* resample_idx;   /* P, NULL: no resampling */
  float* particles_out;    /* P x 6, NULL: indices only (must not alias particles) */
  mcl_estimate* estimate;  /* NULL, or the pose estimate of the weighted particles (before
                              resampling), as mcl_sensor_update_estimate; needs w */
  int32_t scan_rings;      /* rings of this session's scan, as mcl_sensor_params.scan_rings
                              (0: staged in the order given); < 0 is EINVAL */
} mcl_session_update;

/* Shape of a batched step. points_per_chunk and lanes_per_particle fix the
 * summation order as in mcl_sensor_params: every session's results equal
 * those of mcl_sensor_update with the same two values (and the session's
 * scan_rings). use_graph = 1
 * captures the whole step into a CUDA graph at the first run and replays it
 * afterwards (the plan owns all scratch, so the graph stays valid). */
typedef struct mcl_batch_params {
  uint32_t struct_size;
  int32_t points_per_chunk, lanes_per_particle, particles_per_item, unroll, pipeline;
  int32_t particle_order;
  int32_t use_graph;
  int32_t item_order;       /* as in mcl_sensor_params, per session */
} mcl_batch_params;

typedef struct mcl_batch_s* mcl_batch_t;

/* Plans a batched step over n sessions (Sec. V-B: every particle evaluated
 * in parallel, here across robots too). Sessions whose maps share kernel
 * kind, storage type, geometry (origin, voxel, dims, truncation) and kind of
 * values, and that share mode, flags and sigma, form a group; each group
 * runs as one persistent kernel over the (session, point chunk, particle
 * block) work items of its sessions, each session reading its own map. The
 * side steps (spatial order, pose matrices and scan packing, log-weights,
 * normalisation with the estimate, resampling) run as one launch each for
 * all sessions, so a step's launches do not grow with n. Allocates the
 * plan's device scratch. EINVAL for any invalid session (as
 * mcl_sensor_update). */
mcl_status mcl_batch_create(const mcl_session_update* sessions, int32_t n,
                            const mcl_batch_params* params, mcl_batch_t* out);

/* Resampling offsets r_s in [0, 1) for the next runs (host array of n, in
 * session order), copied to the device on `stream`. */
mcl_status mcl_batch_set_offsets(mcl_batch_t b, const double* r, mcl_stream_t stream);

/* Enqueues one step for every session on `stream`: spatial order, pose
 * matrices, scan packing, the grouped sensor kernels, log-weights,
 * normalisation (and estimates) and the requested resampling. */
mcl_status mcl_batch_run(mcl_batch_t b, mcl_stream_t stream);

/* Work items and launches of the plan (for reporting): n_groups sensor
 * kernels, kernels_per_run launches in all. */
typedef struct mcl_batch_info {
  uint32_t struct_size;
  int32_t n_sessions, n_groups;
  int64_t n_items, total_evals, workspace_bytes;
  int32_t kernels_per_run, graph_captured;
} mcl_batch_info;

mcl_status mcl_batch_get_info(mcl_batch_t b, mcl_batch_info* out);

/* Waits for the plan's work on every stream, frees its scratch and graph. */
mcl_status mcl_batch_destroy(mcl_batch_t b);

/* ------------------------------------------------------------------ filter */

/* A particle filter for one robot that keeps its particles on the device and
 * runs a whole step of the method per call (Sec. III: motion update, sensor
 * update with weights, pose estimate, resampling). Step k (k = 0, 1, ...)
 * enqueues exactly the work of these calls, with equal results bit for bit:
 *   mcl_motion_update(particles, P, delta, motion_sigma, seed, k)  (skipped
 *     when delta is NULL),
 *   mcl_sensor_update_estimate(map, particles, P, scan, N, &sensor, logw, w,
 *     estimate),
 *   mcl_resample(w, P, r_k, idx, particles, particles') and particles =
 *     particles', with r_k = the SplitMix64 finaliser of
 *     (seed ^ k * 0x9E3779B97F4A7C15) as 53 bits in [0, 1) - the offsets of a
 *     serving session with the same seed.
 * The paper runs the motion update and resampling on the CPU between GPU
 * calls; here with use_graph = 1 the step for each scan size is captured
 * into a CUDA graph at its first use and replayed: the per-step values
 * (increment, counter, offset) are read from device memory when the graph
 * runs, so a step costs one 48-byte copy, one scan copy and a graph launch. */
typedef struct mcl_filter_desc {
  uint32_t struct_size;       /* sizeof(mcl_filter_desc) */
  mcl_map_t map;
  int64_t P;                  /* particles, [1, 2^31 - 1] */
  int64_t max_points;         /* largest scan, [1, 2^31 - 1] */
  mcl_sensor_params sensor;   /* sigma_hit, mode, flags, launch shape */
  float motion_sigma[6];      /* noise sigma of the increment, >= 0 */
  uint64_t seed;              /* motion-noise key and resampling offsets */
  int32_t use_graph;          /* 1: replay each scan size's step from a CUDA graph */
  int32_t max_graphs;         /* graphs kept, least recently used evicted; 0 = 8 */
  int64_t first_step;         /* step counter to start from: 0, or the steps of a
                                 checkpoint (mcl_filter_state) to resume it */
} mcl_filter_desc;

typedef struct mcl_filter_s* mcl_filter_t;

/* Creates a filter on the current device from P particles (device, P x 6
 * FP32, copied before return). The filter owns its device memory, sized at
 * creation for max_points, so steps allocate nothing. EINVAL: bad
 * description; ENOMEM: out of device memory. */
mcl_status mcl_filter_create(const mcl_filter_desc* desc, const float* particles,
                             mcl_filter_t* out);

/* One step: delta (host, 6 FP32, NULL = no motion update), scan (device,
 * N x 3 FP32, 1 <= N <= max_points, copied into the filter on `stream`), out
 * (device mcl_estimate, 8-byte aligned, or NULL) gets the estimate of this
 * step's weighted particles (before resampling). Asynchronous; the caller
 * may reuse delta at once and scan after the stream's work. Steps on one
 * filter must be issued from one host thread at a time. */
mcl_status mcl_filter_step(mcl_filter_t f, const float* delta, const float* scan, int64_t N,
                           mcl_estimate* out, mcl_stream_t stream);

/* Replaces the particles (device, P x 6, copied on `stream`), e.g. for a
 * global relocalisation; the step counter continues. */
mcl_status mcl_filter_reset(mcl_filter_t f, const float* particles, mcl_stream_t stream);

/* The filter's device arrays (valid until mcl_filter_destroy; read them after
 * the stream's work finished) and counters. */
typedef struct mcl_filter_state {
  uint32_t struct_size;
  const float* particles;        /* P x 6, after the last resampling */
  const float* logw;             /* P, of the last sensor update */
  const float* w;                /* P, of the last sensor update */
  const int32_t* idx;            /* P, the last resampling's draw */
  const mcl_estimate* estimate;  /* the last step's estimate */
  int64_t P;
  int64_t steps;                 /* steps enqueued */
  int64_t graph_launches;        /* steps replayed from a graph */
  double last_r;                 /* resampling offset of the last step */
  int64_t device_bytes;          /* device memory the filter holds */
  int32_t graphs;                /* graphs instantiated and kept */
  int32_t reserved;
} mcl_filter_state;

mcl_status mcl_filter_get_state(mcl_filter_t f, mcl_filter_state* out);

/* Waits for the filter's work on the device, then frees it. NULL is a no-op. */
mcl_status mcl_filter_destroy(mcl_filter_t f);

/* ------------------------------------------------------------------ serving */

/* A server keeps robot sessions on the device (particles, weights, scan
 * buffer, scratch) and runs one filter step per submitted scan: optional
 * motion update with the scan's odometry increment, sensor update,
 * normalisation and systematic resampling (Sec. III: motion, sensor,
 * resampling steps). A scheduler thread batches the pending scans of all
 * sessions that are not already on the GPU into one batched step as soon as
 * one of max_in_flight slots (each with its own stream) is free, so scans
 * that arrive while others run are admitted and their work overlaps on the
 * device (continuous batching); the sessions that have waited longest go
 * first, up to max_batch per step. Each session keeps at most one queued
 * scan: a newer scan supersedes a queued, unstarted one (its ticket completes
 * as MCL_RESULT_SUPERSEDED) and its odometry increment is composed with the
 * newer scan's (body frame, FP64), so the motion is not lost. Latency is
 * measured from submission to the host seeing the step complete. */
typedef struct mcl_server_s* mcl_server_t;
typedef struct mcl_session_s* mcl_session_t;
typedef uint64_t mcl_ticket_t;

typedef struct mcl_server_desc {
  uint32_t struct_size;
  int64_t hbm_budget_bytes; /* device bytes all sessions may hold (maps not included) */
  int32_t max_sessions;     /* open sessions at most */
  int32_t max_in_flight;    /* batched steps on the GPU at once, >= 1 (2 recommended) */
  int32_t max_batch;        /* sessions per batched step at most (0 = max_sessions) */
  mcl_batch_params shape;   /* launch shape of every step (use_graph must be 0) */
} mcl_server_desc;

mcl_status mcl_server_create(const mcl_server_desc* desc, mcl_server_t* out);

/* Opens a session of P particles (host array P x 6, copied) on `map`, for
 * scans of at most max_N points. EBUSY: max_sessions reached. ENOMEM: the
 * session's device bytes would exceed the budget (or the device is full). */
typedef struct mcl_session_desc {
  uint32_t struct_size;
  mcl_map_t map;
  int64_t P, max_N;
  const float* particles;   /* host, P x 6 */
  float sigma_hit;
  int32_t mode;
  uint32_t flags;
  float motion_sigma[6];    /* noise of the motion update */
  uint64_t seed;            /* motion noise and resampling offsets */
  int64_t first_step;       /* step counter to start from: 0, or the step of a checkpoint
                               (particles from mcl_session_read, step from
                               mcl_session_get_info) to resume the same sequence */
  int32_t scan_rings;       /* rings of the session's scans, as mcl_sensor_params.scan_rings,
                               applied to each submitted scan by its own N; < 0 is EINVAL */
} mcl_session_desc;

mcl_status mcl_session_open(mcl_server_t s, const mcl_session_desc* desc, mcl_session_t* out);

typedef struct mcl_session_info {
  uint32_t struct_size;
  int64_t P, max_N;
  int64_t step;             /* steps completed (the next step's noise counter) */
  uint64_t seed;
  int64_t device_bytes;     /* counted against the server's budget */
} mcl_session_info;

/* The session's counters after its queued and running steps finished
 * (waits up to timeout_ms; < 0: forever). With mcl_session_read this is a
 * checkpoint: a session opened with those particles, the same parameters and
 * first_step = step continues bit for bit. */
mcl_status mcl_session_get_info(mcl_session_t ss, mcl_session_info* out, int32_t timeout_ms);

/* Queues one scan (host, N x 3, copied before return) with an optional
 * odometry increment (host, 6 values, NULL = none). */
mcl_status mcl_submit_scan(mcl_session_t ss, const float* scan, int64_t N, const float* delta,
                           mcl_ticket_t* out);

enum { MCL_RESULT_DONE = 0, MCL_RESULT_SUPERSEDED = 1, MCL_RESULT_CLOSED = 2 };

typedef struct mcl_result {
  uint32_t struct_size;
  int32_t status;           /* MCL_RESULT_* */
  double latency_ms;        /* submission to completion seen by the host */
  int64_t evals;            /* P x N of the step */
  int64_t step;             /* the session's step counter after this step */
  mcl_estimate estimate;    /* MCL_RESULT_DONE: the pose estimate of the step's weighted
                               particles (before resampling), as mcl_pose_estimate */
} mcl_result;

/* Waits up to timeout_ms (< 0: forever) for a ticket. ETIMEDOUT if it has
 * not completed; EINVAL for an unknown ticket (each completed ticket can be
 * collected once). */
mcl_status mcl_wait(mcl_server_t s, mcl_ticket_t t, int32_t timeout_ms, mcl_result* out);

/* Copies the session's current particles (P x 6) and weights (P) to host
 * arrays (either may be NULL), after its queued and running steps finished. */
mcl_status mcl_session_read(mcl_session_t ss, float* particles, float* w, int32_t timeout_ms);

/* Closes a session after its running step (a queued scan completes as
 * MCL_RESULT_CLOSED) and returns its device bytes to the budget. */
mcl_status mcl_session_close(mcl_session_t ss);

typedef struct mcl_server_stats {
  uint32_t struct_size;
  int64_t completed, superseded, batches, evals;
  double p50_ms, p99_ms, max_ms, mean_batch_sessions;
  double wall_s;            /* since creation or the last reset */
  double evals_per_s;
  int64_t bytes_in_use;
  int32_t sessions, in_flight;
} mcl_server_stats;

mcl_status mcl_server_get_stats(mcl_server_t s, int32_t reset, mcl_server_stats* out);

/* Holds (1) or releases (0) the scheduler: held, no new step starts (for
 * tests of queueing and timeouts). */
mcl_status mcl_server_pause(mcl_server_t s, int32_t pause);

/* Stops the scheduler after the running steps, closes every session. */
mcl_status mcl_server_destroy(mcl_server_t s);

/* ------------------------------------------------------------------ gather roofline */

/* Microbenchmark of the map look-up pattern (Sec. VI-C: random TSDF reads
 * bound the sensor update): blocks x 256 threads each read iters x 8
 * elements of `buf` (device, n_elems elements of elem_bytes = 2 or 4 bytes)
 * at uniform random positions. Gathers issued = blocks * 256 * iters * 8;
 * time the call with events on `stream` to get gathers/s for that footprint.
 * EINVAL: n_elems < 1, elem_bytes not 2 or 4, blocks or iters < 1. */
mcl_status mcl_gather_bench(const void* buf, int64_t n_elems, int32_t elem_bytes, int32_t blocks,
                            int32_t iters, uint64_t seed, mcl_stream_t stream);

/* ------------------------------------------------------------------ runtime */

/* Frees the library workspace kept for (current device, stream), after
 * waiting for the stream. Call before destroying a stream the library used. */
mcl_status mcl_workspace_release(mcl_stream_t stream);

/* Per-phase device timing. Between mcl_profile_begin() and mcl_profile_end()
 * every phase this library enqueues is bracketed by CUDA events recorded on
 * its own stream; mcl_profile_end() waits for them and returns, per phase,
 * the number of kernel launches and the summed elapsed milliseconds. Not for
 * use while a stream is being captured into a graph. Every phase is also an
 * NVTX range named "mcl.<phase>" (pose, pack, sensor, reduce, normalise,
 * resample, motion, other) whether profiling is on or not. */
enum {
  MCL_PHASE_POSE = 0,     /* pose -> [R | t] */
  MCL_PHASE_PACK = 1,     /* scan packing (now done by the pose phase's kernel: no launches) */
  MCL_PHASE_SENSOR = 2,   /* transform, look-up, score, per-chunk sums */
  MCL_PHASE_REDUCE = 3,   /* chunk sums -> log-weights, block statistics */
  MCL_PHASE_NORMALISE = 4,
  MCL_PHASE_RESAMPLE = 5, /* quantise, exact prefix sum, search, gather */
  MCL_PHASE_MOTION = 6,
  MCL_PHASE_OTHER = 7,
  MCL_NUM_PHASES = 8
};

typedef struct mcl_profile {
  uint32_t struct_size;
  int64_t launches[MCL_NUM_PHASES];
  double ms[MCL_NUM_PHASES];
} mcl_profile;

mcl_status mcl_profile_begin(void);
mcl_status mcl_profile_end(mcl_profile* out);

#ifdef __cplusplus
}
#endif

#endif /* MCL_H_ */
