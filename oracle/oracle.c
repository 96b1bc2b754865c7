/*
 * FP64 CPU oracle for the 6D MCL sensor update in TSDF maps
 * (Eisoldt, Mock, Porrmann, Wiemann: "Towards 6D MCL for LiDARs in 3D TSDF
 * Maps on Embedded Systems with GPUs").
 *
 * TEST INFRASTRUCTURE. This file is the slow, plain reference that the CUDA
 * library is checked against. Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it. It shares no code, header,
 * table or constant generator with the CUDA path; it is written from the
 * paper's definitions:
 *
 *   particle  p = (s, w), s = (x, y, z, phi, psi, theta)       Sec. III, Eq. 1-2
 *   sensor model p_hit = exp(-m^2 / (2 sigma^2)) / sqrt(2 pi sigma^2)   Eq. 3
 *   m(x, z) = TSDF value read at the voxel containing the scan point
 *             seen from the particle's pose                    Sec. III
 *             (or interpolated trilinearly between the voxel centres
 *             around it: "pseudo-continuous via interpolation", Sec. III)
 *   cells without stored values are clamped to the truncation value Sec. III
 *   weights summed for normalisation                          Sec. V-A
 *   resampling draws a new set in proportion to the weights   Sec. III
 *
 * Readings where the paper is silent:
 *   - (phi, psi, theta) = (roll, pitch, yaw), R = Rz(yaw) Ry(pitch) Rx(roll).
 *   - per-point scores combine as a product of p_hit (sum of log p_hit, the
 *     normalising constant dropped: mode LOGPROD) or as a plain sum of p_hit
 *     (mode SUM, particle log-weight = log of the sum).
 *   - a point outside the grid or in an unallocated brick reads +tau; with
 *     the neglect flag it is left out of the particle's score instead.
 *   - resampling is systematic with one caller offset r in [0, 1) over
 *     weights quantised to multiples of 2^-52.
 *   - motion: body-frame increment plus per-component Gaussian noise drawn by
 *     Philox4x32-10 (Salmon et al., SC'11) and Box-Muller.
 *
 * Two modes. Parity mode evaluates the scan point's index-rule coordinate in
 * FP32 in a fixed operation order (the pose rows taken into the map's index
 * frame, then one FP32 fma chain per axis; this fixes which voxel a point
 * falls in exactly as an FP32 implementation sees it); from the map value on
 * everything is FP64. Quality mode is FP64 throughout.
 *
 * Compile with -ffp-contract=off: no fused multiply-add is allowed anywhere
 * except the explicit fmaf calls of the parity-mode transform.
 *
 * Parity unpinned: none of the functions below (each has a closed-form,
 * invariant or brute-force pin in the test suite).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

enum { ORA_DENSE = 0, ORA_BRICK = 1, ORA_ANALYTIC = 2 };
enum { ORA_F32 = 0, ORA_F16 = 1, ORA_I16 = 2 };
enum { ORA_LOGPROD = 0, ORA_SUM = 1, ORA_SCORE = 2 };
enum { ORA_PRIM_PLANE = 0, ORA_PRIM_SPHERE = 1, ORA_PRIM_BOX = 2 };

#define BRICK_EDGE 16

typedef struct {
  int kind, dtype;
  float origin_f[3], voxel_f, inv_voxel_f, tau_f;
  double outside; /* value read where nothing is stored: +tau, or the score of +tau for a score map */
  int64_t dims[3];
  const void* values; /* dense: dims[2]*dims[1]*dims[0]; brick: n_bricks * 4096 */
  int64_t n_bricks;
  int64_t nb[3];
  int32_t* coarse; /* brick grid cell -> brick slot, -1 if not allocated */
  int64_t n_prims;
  double* prims; /* analytic: rows of 8 doubles: type, params... */
} ora_map;

/* ------------------------------------------------------------------ map set-up */

/* Dense or brick TSDF. Returns NULL on bad input (dims not multiples of 16 for
 * bricks, brick coordinates out of range or duplicated). */
ora_map* ora_map_create(int kind, int dtype, const float origin[3], float voxel, float inv_voxel,
                        float tau, const int64_t dims[3], const void* values, int64_t n_bricks,
                        const int32_t* brick_coords) {
  if ((kind != ORA_DENSE && kind != ORA_BRICK) || dtype < 0 || dtype > 2) return NULL;
  ora_map* m = (ora_map*)calloc(1, sizeof(ora_map));
  m->kind = kind;
  m->dtype = dtype;
  for (int k = 0; k < 3; ++k) { m->origin_f[k] = origin[k]; m->dims[k] = dims[k]; }
  m->voxel_f = voxel;
  m->inv_voxel_f = inv_voxel;
  m->tau_f = tau;
  m->outside = (double)tau;
  m->values = values;
  if (kind == ORA_BRICK) {
    for (int k = 0; k < 3; ++k) {
      if (dims[k] <= 0 || dims[k] % BRICK_EDGE) { free(m); return NULL; }
      m->nb[k] = dims[k] / BRICK_EDGE;
    }
    int64_t cells = m->nb[0] * m->nb[1] * m->nb[2];
    m->coarse = (int32_t*)malloc((size_t)cells * sizeof(int32_t));
    for (int64_t c = 0; c < cells; ++c) m->coarse[c] = -1;
    m->n_bricks = n_bricks;
    for (int64_t b = 0; b < n_bricks; ++b) {
      int64_t bx = brick_coords[3 * b], by = brick_coords[3 * b + 1], bz = brick_coords[3 * b + 2];
      if (bx < 0 || by < 0 || bz < 0 || bx >= m->nb[0] || by >= m->nb[1] || bz >= m->nb[2]) {
        free(m->coarse); free(m); return NULL;
      }
      int64_t c = (bz * m->nb[1] + by) * m->nb[0] + bx;
      if (m->coarse[c] != -1) { free(m->coarse); free(m); return NULL; }
      m->coarse[c] = (int32_t)b;
    }
  }
  return m;
}

/* Analytic map: union (minimum) of primitives' signed distances, clamped to
 * [-tau, tau], evaluated at the exact point (no grid). Rows of 8 doubles:
 *   plane : 0, nx, ny, nz, d0        sdf = n.x - d0 (n unit)
 *   sphere: 1, cx, cy, cz, R         sdf = |x - c| - R
 *   box   : 2, lox, loy, loz, hix, hiy, hiz
 */
ora_map* ora_map_create_analytic(int64_t n_prims, const double* prims, float tau) {
  ora_map* m = (ora_map*)calloc(1, sizeof(ora_map));
  m->kind = ORA_ANALYTIC;
  m->tau_f = tau;
  m->n_prims = n_prims;
  m->prims = (double*)malloc((size_t)n_prims * 8 * sizeof(double));
  memcpy(m->prims, prims, (size_t)n_prims * 8 * sizeof(double));
  return m;
}

/* Score maps (Sec. III: the exponential of Eq. 3 evaluated once per map
 * entry before the scans): their values are per-voxel scores, and a point
 * where nothing is stored reads the score of +tau, set here. */
void ora_map_set_outside(ora_map* m, double outside) { m->outside = outside; }

void ora_map_destroy(ora_map* m) {
  if (!m) return;
  free(m->coarse);
  free(m->prims);
  free(m);
}

/* ------------------------------------------------------------------ storage decode */

static double half_to_double(uint16_t h) {
  int s = h >> 15, e = (h >> 10) & 31, f = h & 1023;
  double v;
  if (e == 0) v = ldexp((double)f, -24);
  else if (e == 31) v = f ? NAN : INFINITY;
  else v = ldexp((double)(f + 1024), e - 25);
  return s ? -v : v;
}

/* Stored value i of the value array, as the real number it stands for. Scaled
 * int16 stands for q * tau / 32767. */
static double stored_value(const ora_map* m, int64_t i) {
  if (m->dtype == ORA_F32) return (double)((const float*)m->values)[i];
  if (m->dtype == ORA_F16) return half_to_double(((const uint16_t*)m->values)[i]);
  return (double)((const int16_t*)m->values)[i] * ((double)m->tau_f / 32767.0);
}

static double analytic_sdf(const ora_map* m, const double x[3]) {
  double best = INFINITY;
  for (int64_t i = 0; i < m->n_prims; ++i) {
    const double* p = m->prims + 8 * i;
    double d;
    if (p[0] == ORA_PRIM_PLANE) {
      d = p[1] * x[0] + p[2] * x[1] + p[3] * x[2] - p[4];
    } else if (p[0] == ORA_PRIM_SPHERE) {
      double a = x[0] - p[1], b = x[1] - p[2], c = x[2] - p[3];
      d = sqrt(a * a + b * b + c * c) - p[4];
    } else {
      double out2 = 0.0, inside = -INFINITY;
      for (int k = 0; k < 3; ++k) {
        double g = fmax(p[1 + k] - x[k], x[k] - p[4 + k]);
        if (g > 0.0) out2 += g * g;
        inside = fmax(inside, g);
      }
      d = sqrt(out2) + fmin(inside, 0.0);
    }
    if (d < best) best = d;
  }
  return best;
}

/* ------------------------------------------------------------------ pose -> [R | t]  */

/* R = Rz(yaw) Ry(pitch) Rx(roll) from the pose angles, in double, in this
 * fixed operation order (each product and sum rounded on its own):
 *   a = cy*sp, b = sy*sp
 *   R = [ cy*cp   a*sr - sy*cr   a*cr + sy*sr ]
 *       [ sy*cp   b*sr + cy*cr   b*cr - cy*sr ]
 *       [ -sp     cp*sr          cp*cr        ]
 * Parity mode rounds each entry to FP32. Output rows [R_i0 R_i1 R_i2 t_i]. */
static void pose_matrix(const float* s, int parity, double M[12]) {
  double cr = cos((double)s[3]), sr = sin((double)s[3]);
  double cp = cos((double)s[4]), sp = sin((double)s[4]);
  double cy = cos((double)s[5]), sy = sin((double)s[5]);
  double a = cy * sp, b = sy * sp;
  double R[9];
  R[0] = cy * cp; R[1] = a * sr - sy * cr; R[2] = a * cr + sy * sr;
  R[3] = sy * cp; R[4] = b * sr + cy * cr; R[5] = b * cr - cy * sr;
  R[6] = -sp;     R[7] = cp * sr;          R[8] = cp * cr;
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) M[4 * i + j] = parity ? (double)(float)R[3 * i + j] : R[3 * i + j];
    M[4 * i + 3] = (double)s[i];
  }
}

void ora_pose_to_matrix(const float* poses, int64_t P, int parity, double* out) {
  for (int64_t p = 0; p < P; ++p) pose_matrix(poses + 6 * p, parity, out + 12 * p);
}

/* ------------------------------------------------------------------ look-up of one point */

/* Value of voxel (ix, iy, iz): 1 and *d = the stored value if the voxel is
 * inside the grid and (brick maps) in an allocated brick, else 0 and
 * *d = +tau (Sec. III clamping). */
static int voxel_value(const ora_map* m, int64_t ix, int64_t iy, int64_t iz, double* d) {
  *d = m->outside;
  if (ix < 0 || iy < 0 || iz < 0 || ix >= m->dims[0] || iy >= m->dims[1] || iz >= m->dims[2]) return 0;
  if (m->kind == ORA_DENSE) {
    *d = stored_value(m, (iz * m->dims[1] + iy) * m->dims[0] + ix);
    return 1;
  }
  int64_t c = ((iz / BRICK_EDGE) * m->nb[1] + iy / BRICK_EDGE) * m->nb[0] + ix / BRICK_EDGE;
  int32_t slot = m->coarse[c];
  if (slot < 0) return 0;
  int64_t local = ((iz % BRICK_EDGE) * BRICK_EDGE + iy % BRICK_EDGE) * BRICK_EDGE + ix % BRICK_EDGE;
  *d = stored_value(m, (int64_t)slot * BRICK_EDGE * BRICK_EDGE * BRICK_EDGE + local);
  return 1;
}

/* Trilinear read at the point whose coordinates, less 1/2, are f (Sec. III:
 * a pseudo-continuous value by interpolation). Voxel i's value is the SDF at
 * its centre o + (i + 1/2) r, so with f = u - 1/2 per axis (u the index-rule
 * coordinate; parity mode: f in FP32) the eight centres around the point are
 * i0 + c, c in {0, 1}^3, i0 = floor(f), a = f - i0, and
 *   d = sum_c prod_k (c_k ? a_k : 1 - a_k) * value(i0 + c)      (FP64)
 * with +tau for corners outside the grid or in no brick. Returns 1 if any
 * corner holds a stored value. idx3 gets i0 (or -1s if no corner is inside). */
static int trilinear_read(const ora_map* m, const double fc[3], int parity, double* d,
                          int64_t idx3[3]) {
  int64_t i0[3];
  double a[3];
  idx3[0] = idx3[1] = idx3[2] = -1;
  *d = m->outside;
  for (int k = 0; k < 3; ++k) {
    if (parity) {
      float f = (float)fc[k];
      if (!(f >= -1.0f && f < (float)m->dims[k])) return 0;
      float fl = floorf(f);
      i0[k] = (int64_t)fl;
      a[k] = (double)(f - fl);
    } else {
      double f = fc[k];
      if (!(f >= -1.0 && f < (double)m->dims[k])) return 0;
      double fl = floor(f);
      i0[k] = (int64_t)fl;
      a[k] = f - fl;
    }
  }
  double acc = 0.0;
  int any = 0;
  for (int c = 0; c < 8; ++c) {
    int cx = c & 1, cy = (c >> 1) & 1, cz = c >> 2;
    double v;
    any |= voxel_value(m, i0[0] + cx, i0[1] + cy, i0[2] + cz, &v);
    double wgt = (cx ? a[0] : 1.0 - a[0]) * (cy ? a[1] : 1.0 - a[1]) * (cz ? a[2] : 1.0 - a[2]);
    acc += wgt * v;
  }
  *d = acc;
  for (int k = 0; k < 3; ++k) idx3[k] = i0[k];
  return any;
}

/* Scan point z seen from the pose [R | t] (FP64 rows M, Sec. III): the world
 * point x = R z + t (FP64, returned in both modes) and its index-rule
 * coordinates u = (x - o) / r per axis, less `shift` (0: the containing
 * voxel; 1/2: f of the trilinear read).
 * Quality mode: u = (x - o) / r - shift in FP64.
 * Parity mode (the FP32 rule): the rows are first taken into the map's index
 * frame, R'_ij = fl32(R_ij * inv) and t'_i = fl32((t_i - o_i) * inv - shift),
 * each evaluated in FP64 in that order and rounded to FP32 once (inv = the
 * map's FP32 1/r), then u_i = fmaf(R'_i0, z0, fmaf(R'_i1, z1, fmaf(R'_i2, z2,
 * t'_i))) in FP32. */
static void scan_coord(const ora_map* m, const double M[12], const float z[3], int parity,
                       double shift, double u[3], double x[3]) {
  for (int i = 0; i < 3; ++i)
    x[i] = M[4 * i] * (double)z[0] + M[4 * i + 1] * (double)z[1] + M[4 * i + 2] * (double)z[2] +
           M[4 * i + 3];
  if (parity) {
    const double inv = (double)m->inv_voxel_f;
    for (int i = 0; i < 3; ++i) {
      float r0 = (float)(M[4 * i] * inv), r1 = (float)(M[4 * i + 1] * inv),
            r2 = (float)(M[4 * i + 2] * inv);
      float t = (float)((M[4 * i + 3] - (double)m->origin_f[i]) * inv - shift);
      u[i] = (double)fmaf(r0, z[0], fmaf(r1, z[1], fmaf(r2, z[2], t)));
    }
  } else {
    for (int i = 0; i < 3; ++i) u[i] = (x[i] - (double)m->origin_f[i]) / (double)m->voxel_f - shift;
  }
}

/* Value at voxel coordinates u (floor(u) per axis; inside iff 0 <= u < n,
 * NaN fails; parity mode compares the FP32 u), whether it exists, and the
 * voxel index (or -1s). */
static int voxel_at(const ora_map* m, const double u[3], int parity, double* d, int64_t idx3[3]) {
  int64_t ix[3];
  idx3[0] = idx3[1] = idx3[2] = -1;
  for (int k = 0; k < 3; ++k) {
    if (parity) {
      float uf = (float)u[k];
      if (!(uf >= 0.0f && uf < (float)m->dims[k])) { *d = m->outside; return 0; }
      ix[k] = (int64_t)floorf(uf);
    } else {
      double fl = floor(u[k]);
      if (!(fl >= 0.0 && fl < (double)m->dims[k])) { *d = m->outside; return 0; }
      ix[k] = (int64_t)fl;
    }
  }
  for (int k = 0; k < 3; ++k) idx3[k] = ix[k];
  return voxel_value(m, ix[0], ix[1], ix[2], d);
}

/* Scan point z seen from pose M: the voxel containing it (or the trilinear
 * read around it), the value read and whether it is stored. Returns 1 if a
 * stored value was read (d set), 0 if outside the grid or in an unallocated
 * brick (d = +tau). x gets the FP64 world point, idx3 the voxel index (the
 * trilinear read: i0) or -1s. An analytic map is read at x. */
static int lookup_point(const ora_map* m, const double M[12], const float z[3], int parity,
                        int interp, double x[3], double* d, int64_t idx3[3]) {
  double u[3];
  idx3[0] = idx3[1] = idx3[2] = -1;
  scan_coord(m, M, z, parity, interp ? 0.5 : 0.0, u, x);
  if (m->kind == ORA_ANALYTIC) {
    double v = analytic_sdf(m, x);
    double tau = (double)m->tau_f;
    *d = v > tau ? tau : (v < -tau ? -tau : v);
    return 1;
  }
  if (interp) return trilinear_read(m, u, parity, d, idx3);
  return voxel_at(m, u, parity, d, idx3);
}

/* ------------------------------------------------------------------ sensor update */

/* Per-point score of Eq. 3. LOGPROD: log p_hit without the constant,
 * -d^2 / (2 sigma^2). SUM: p_hit itself. SCORE (a score map, mode SUM):
 * the stored value is exp(-d^2 / (2 sigma^2)), so p_hit = value times the
 * constant of Eq. 3. */
static double point_score(double d, double sigma, int mode) {
  if (mode == ORA_SCORE) return d / sqrt(2.0 * M_PI * sigma * sigma); /* d is the stored score */
  double e = -(d * d) / (2.0 * sigma * sigma);
  if (mode == ORA_LOGPROD) return e;
  return exp(e) / sqrt(2.0 * M_PI * sigma * sigma);
}

/* Flags of the sensor update: bit 0 leaves points without a stored value
 * out (neglect), bit 1 reads the TSDF by trilinear interpolation. */
#define ORA_NEGLECT 1
#define ORA_TRILINEAR 2

/* Log-weight of one particle with pose matrix M (Sec. III): LOGPROD sums the
 * per-point log scores, SUM takes the log of the summed p_hit. With the
 * neglect flag points without a stored value are left out. */
static double particle_log_weight(const ora_map* m, const double M[12], const float* scan,
                                  int64_t N, double sigma, int mode, int flags, int parity) {
  double x[3], d, acc = 0.0;
  int64_t idx3[3];
  for (int64_t j = 0; j < N; ++j) {
    int stored = lookup_point(m, M, scan + 3 * j, parity, (flags & ORA_TRILINEAR) != 0, x, &d, idx3);
    if (!stored && (flags & ORA_NEGLECT)) continue;
    acc += point_score(d, sigma, mode);
  }
  return (mode == ORA_LOGPROD) ? acc : log(acc);
}

/* Log-weights L_p of all particles for one scan. Particles are split into
 * contiguous per-thread groups (the CPU design of Sec. V-A) when OpenMP is on. */
void ora_sensor_update(const ora_map* m, const float* poses, int64_t P, const float* scan,
                       int64_t N, double sigma, int mode, int flags, int parity, double* out_L) {
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < P; ++p) {
    double M[12];
    pose_matrix(poses + 6 * p, 0, M); /* FP64 rows; parity mode rounds in scan_coord */
    out_L[p] = particle_log_weight(m, M, scan, N, sigma, mode, flags, parity);
  }
}

/* Same with the poses given as FP64 [R | t] rows (12 per particle), taken as
 * they are (parity mode rounds in the index frame, as for poses). */
void ora_sensor_update_mat(const ora_map* m, const double* mats, int64_t P, const float* scan,
                           int64_t N, double sigma, int mode, int flags, int parity,
                           double* out_L) {
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < P; ++p) {
    double M[12];
    for (int k = 0; k < 12; ++k) M[k] = mats[12 * p + k];
    out_L[p] = particle_log_weight(m, M, scan, N, sigma, mode, flags, parity);
  }
}

/* Per-point detail for one pose: world coordinates, read value d and the
 * voxel index (-1 where outside). Returns the number of stored reads. */
int64_t ora_eval_points(const ora_map* m, const float pose[6], const float* scan, int64_t N,
                        int parity, int interp, double* out_x, double* out_d, int64_t* out_idx) {
  double M[12];
  int64_t n_stored = 0;
  pose_matrix(pose, 0, M);
  for (int64_t j = 0; j < N; ++j) {
    double x[3], d;
    int64_t idx3[3];
    n_stored += lookup_point(m, M, scan + 3 * j, parity, interp, x, &d, idx3);
    if (out_x) memcpy(out_x + 3 * j, x, sizeof(x));
    if (out_d) out_d[j] = d;
    if (out_idx) memcpy(out_idx + 3 * j, idx3, sizeof(idx3));
  }
  return n_stored;
}

/* Map query at FP32 world points: linear voxel index (iz*ny + iy)*nx + ix in
 * the whole grid (-1 outside) and the value read there (+tau outside the grid
 * or in an unallocated brick). The point's coordinates are
 * u = fl32(fl32(x - o) * inv) per axis (two FP32 roundings), then the rule of
 * voxel_at. */
void ora_map_lookup(const ora_map* m, const float* pts, int64_t n, int64_t* out_index,
                    double* out_value) {
  for (int64_t j = 0; j < n; ++j) {
    double u[3], d;
    int64_t idx3[3];
    for (int k = 0; k < 3; ++k) u[k] = (double)((pts[3 * j + k] - m->origin_f[k]) * m->inv_voxel_f);
    voxel_at(m, u, 1, &d, idx3);
    out_index[j] = idx3[0] < 0 ? -1 : (idx3[2] * m->dims[1] + idx3[1]) * m->dims[0] + idx3[0];
    out_value[j] = d;
  }
}

/* ------------------------------------------------------------------ normalisation */

/* w_p = exp(L_p - M) / sum_q exp(L_q - M), M = max L (Sec. V-A). If no L is
 * finite (every particle scored zero in SUM mode) the weights are uniform and
 * the return value is 1 (degenerate), else 0. */
int ora_normalise(const double* L, int64_t P, double* out_w, double* out_max, double* out_sum) {
  double M = -INFINITY, S = 0.0;
  for (int64_t p = 0; p < P; ++p)
    if (L[p] > M) M = L[p];
  if (!isfinite(M)) {
    for (int64_t p = 0; p < P; ++p) out_w[p] = 1.0 / (double)P;
    if (out_max) *out_max = M;
    if (out_sum) *out_sum = 0.0;
    return 1;
  }
  for (int64_t p = 0; p < P; ++p) S += exp(L[p] - M);
  for (int64_t p = 0; p < P; ++p) out_w[p] = exp(L[p] - M) / S;
  if (out_max) *out_max = M;
  if (out_sum) *out_sum = S;
  return 0;
}

/* ------------------------------------------------------------------ systematic resampling */

/* Systematic resampling (Sec. III, drawing in proportion to the weights) with
 * one offset r in [0, 1):
 *   q_p = rint(w_p * 2^52) * 2^-52              (exact in FP64)
 *   C_p = q_0 + ... + q_p                        (exact while the sum < 2)
 *   S   = C_{P-1},  t_j = ((j + r) / P) * S      (IEEE FP64: add, divide, multiply)
 *   idx_j = min { p : C_p > t_j }, else the last p with q_p > 0.
 * If every q_p is zero the draw is the identity. Returns 1 then, else 0. */
int ora_resample(const float* w, int64_t P, double r, int32_t* out_idx) {
  double* C = (double*)malloc((size_t)P * sizeof(double));
  double acc = 0.0;
  int64_t last_pos = -1;
  for (int64_t p = 0; p < P; ++p) {
    double q = rint((double)w[p] * 0x1.0p52) * 0x1.0p-52;
    acc += q;
    C[p] = acc;
    if (q > 0.0) last_pos = p;
  }
  double S = acc;
  if (last_pos < 0) {
    for (int64_t j = 0; j < P; ++j) out_idx[j] = (int32_t)j;
    free(C);
    return 1;
  }
  for (int64_t j = 0; j < P; ++j) {
    double t = (((double)j + r) / (double)P) * S;
    int64_t lo = 0, hi = P; /* first p in [lo, hi) with C_p > t; hi = none */
    while (lo < hi) {
      int64_t mid = lo + (hi - lo) / 2;
      if (C[mid] > t) hi = mid; else lo = mid + 1;
    }
    out_idx[j] = (int32_t)(lo < P ? lo : last_pos);
  }
  free(C);
  return 0;
}

/* ------------------------------------------------------------------ motion update */

/* Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11): each round multiplies two counter
 * words by the round multipliers, swaps and mixes the high halves with the
 * other words and the key; the key is bumped by the Weyl constants between
 * rounds. */
void ora_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    c0 = hi1 ^ c1 ^ k0;
    c1 = lo1;
    c2 = hi0 ^ c3 ^ k1;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Two standard normals from one Philox block by Box-Muller:
 *   u1 = ((hi64(o0,o1) >> 11) + 1/2) 2^-53 in (0,1), u2 = (hi64(o2,o3) >> 11) 2^-53 in [0,1)
 *   n0 = sqrt(-2 ln u1) cos(2 pi u2),  n1 = sqrt(-2 ln u1) sin(2 pi u2). */
static void box_muller(const uint32_t o[4], double n[2]) {
  uint64_t a = (((uint64_t)o[0] << 32) | o[1]) >> 11, b = (((uint64_t)o[2] << 32) | o[3]) >> 11;
  double u1 = ((double)a + 0.5) * 0x1.0p-53, u2 = (double)b * 0x1.0p-53;
  double rho = sqrt(-2.0 * log(u1));
  n[0] = rho * cos(6.283185307179586 * u2);
  n[1] = rho * sin(6.283185307179586 * u2);
}

/* The six noise normals of particle i at `step`: block b in {0,1,2} uses
 * counter (b, i, step_lo, step_hi) and key (seed_lo, seed_hi) and yields
 * components 2b and 2b+1 (x, y | z, roll | pitch, yaw). */
void ora_motion_noise(uint64_t seed, uint64_t step, int64_t i, double n6[6]) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (uint32_t b = 0; b < 3; ++b) {
    uint32_t ctr[4] = {b, (uint32_t)i, (uint32_t)step, (uint32_t)(step >> 32)}, o[4];
    ora_philox4x32_10(ctr, key, o);
    box_muller(o, n6 + 2 * b);
  }
}

/* Motion update (Sec. III: the motion model is applied to each particle):
 * increment u = delta + sigma * n (body frame, n the six normals above);
 *   t' = t + R(s) u_t,   R' = R(s) R(u_r)   (R(.) as in pose_matrix, FP64)
 * and R' is read back as roll = atan2(R'21, R'22), pitch = asin(-R'20),
 * yaw = atan2(R'10, R'00), with yaw = pi mapped to -pi. Everything in FP64,
 * the new pose rounded to FP32 in place. */
void ora_motion_update(float* poses, int64_t P, const float delta[6], const float sigma[6],
                       uint64_t seed, uint64_t step) {
  for (int64_t i = 0; i < P; ++i) {
    float* s = poses + 6 * i;
    double n6[6], u[6], A[12], B[12], Rn[9];
    ora_motion_noise(seed, step, i, n6);
    for (int k = 0; k < 6; ++k) u[k] = (double)delta[k] + (double)sigma[k] * n6[k];
    pose_matrix(s, 0, A);
    double t_new[3];
    for (int r = 0; r < 3; ++r)
      t_new[r] = (double)s[r] + (A[4 * r] * u[0] + A[4 * r + 1] * u[1] + A[4 * r + 2] * u[2]);
    /* rotation of the increment, in double (angles kept unrounded) */
    {
      double cr = cos(u[3]), sr = sin(u[3]), cp = cos(u[4]), sp = sin(u[4]);
      double cy = cos(u[5]), sy = sin(u[5]);
      double a = cy * sp, b = sy * sp;
      B[0] = cy * cp; B[1] = a * sr - sy * cr; B[2] = a * cr + sy * sr;
      B[4] = sy * cp; B[5] = b * sr + cy * cr; B[6] = b * cr - cy * sr;
      B[8] = -sp;     B[9] = cp * sr;          B[10] = cp * cr;
    }
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c)
        Rn[3 * r + c] = A[4 * r] * B[c] + A[4 * r + 1] * B[4 + c] + A[4 * r + 2] * B[8 + c];
    double sp_ = -Rn[6];
    if (sp_ > 1.0) sp_ = 1.0;
    if (sp_ < -1.0) sp_ = -1.0;
    double roll = atan2(Rn[7], Rn[8]), pitch = asin(sp_), yaw = atan2(Rn[3], Rn[0]);
    if (yaw >= M_PI) yaw = -M_PI;
    s[0] = (float)t_new[0]; s[1] = (float)t_new[1]; s[2] = (float)t_new[2];
    s[3] = (float)roll; s[4] = (float)pitch; s[5] = (float)yaw;
  }
}

int ora_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
