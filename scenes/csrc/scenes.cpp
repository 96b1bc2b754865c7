// Seeded synthetic scenes for 6D MCL in TSDF maps: box-set environments,
// TSDF voxelisation (dense grids and 16^3 bricks), raycast LiDAR scans and
// particle clouds.
//
// This is input generation only. It is shared by the FP64 oracle and the
// CUDA path as a source of data, and holds none of the sensor-update
// arithmetic (no scan transform into particle frames, no map look-up, no
// scoring, normalisation or resampling).
//
// Random numbers: SplitMix64 (Steele, Lea, Flood, "Fast splittable
// pseudorandom number generators", OOPSLA 2014) used as a counter-based hash
// of (seed, stream, index), so every output is independent of thread count.
// Normals: Box-Muller (1958).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

inline uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Counter-based 64-bit draw for (seed, stream, index).
inline uint64_t draw(uint64_t seed, uint64_t stream, uint64_t index) {
  return mix64(mix64(seed ^ mix64(stream * 0xD1B54A32D192ED03ull)) + index);
}

// Uniform in [0, 1) with 53 random bits.
inline double unif(uint64_t seed, uint64_t stream, uint64_t index) {
  return (double)(draw(seed, stream, index) >> 11) * 0x1.0p-53;
}

// Standard normal by Box-Muller from two uniforms of the stream.
inline double normal(uint64_t seed, uint64_t stream, uint64_t index) {
  double u1 = ((double)(draw(seed, stream, 2 * index) >> 11) + 0.5) * 0x1.0p-53;
  double u2 = unif(seed, stream, 2 * index + 1);
  return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
}

struct Box {
  double lo[3], hi[3];
};

// Exact Euclidean signed distance to an axis-aligned box (negative inside).
inline double box_sdf(const Box& b, const double p[3]) {
  double d[3], out2 = 0.0, inside = -1e300;
  for (int k = 0; k < 3; ++k) {
    d[k] = std::max(b.lo[k] - p[k], p[k] - b.hi[k]);
    if (d[k] > 0.0) out2 += d[k] * d[k];
    inside = std::max(inside, d[k]);
  }
  return std::sqrt(out2) + std::min(inside, 0.0);
}

// Distance between an axis-aligned box and an axis-aligned cell (0 if they overlap).
inline double box_cell_dist(const Box& b, const double clo[3], const double chi[3]) {
  double s = 0.0;
  for (int k = 0; k < 3; ++k) {
    double g = std::max(b.lo[k] - chi[k], clo[k] - b.hi[k]);
    if (g > 0.0) s += g * g;
  }
  return std::sqrt(s);
}

// Uniform grid of cells over a region, each cell listing the boxes that come
// within `margin` of it (CSR layout). Used for culling only: any box farther
// than `margin` from a cell has signed distance > margin everywhere in it.
struct CellIndex {
  double origin[3];
  double cell;
  int64_t n[3];
  std::vector<int64_t> start;  // n0*n1*n2 + 1
  std::vector<int32_t> items;

  void build(const std::vector<Box>& boxes, const double org[3], double cell_size,
             const int64_t ncell[3], double margin) {
    for (int k = 0; k < 3; ++k) { origin[k] = org[k]; n[k] = ncell[k]; }
    cell = cell_size;
    const int64_t total = n[0] * n[1] * n[2];
    std::vector<int64_t> count(total + 1, 0);
    auto range = [&](const Box& b, int64_t lo[3], int64_t hi[3]) {
      for (int k = 0; k < 3; ++k) {
        lo[k] = (int64_t)std::floor((b.lo[k] - margin - origin[k]) / cell);
        hi[k] = (int64_t)std::floor((b.hi[k] + margin - origin[k]) / cell);
        lo[k] = std::max<int64_t>(lo[k], 0);
        hi[k] = std::min<int64_t>(hi[k], n[k] - 1);
      }
    };
    auto visit = [&](const Box& b, auto&& fn) {
      int64_t lo[3], hi[3];
      range(b, lo, hi);
      for (int64_t z = lo[2]; z <= hi[2]; ++z)
        for (int64_t y = lo[1]; y <= hi[1]; ++y)
          for (int64_t x = lo[0]; x <= hi[0]; ++x) {
            double clo[3] = {origin[0] + x * cell, origin[1] + y * cell, origin[2] + z * cell};
            double chi[3] = {clo[0] + cell, clo[1] + cell, clo[2] + cell};
            if (box_cell_dist(b, clo, chi) <= margin) fn((z * n[1] + y) * n[0] + x);
          }
    };
    for (const Box& b : boxes) visit(b, [&](int64_t c) { count[c + 1]++; });
    for (int64_t c = 0; c < total; ++c) count[c + 1] += count[c];
    start = count;
    items.assign(start[total], 0);
    std::vector<int64_t> fill(start.begin(), start.end() - 1);
    for (size_t i = 0; i < boxes.size(); ++i)
      visit(boxes[i], [&](int64_t c) { items[fill[c]++] = (int32_t)i; });
  }

  // Cell id of a point, or -1 outside the indexed region.
  int64_t cell_of(const double p[3]) const {
    int64_t c[3];
    for (int k = 0; k < 3; ++k) {
      double u = std::floor((p[k] - origin[k]) / cell);
      if (!(u >= 0.0) || u >= (double)n[k]) return -1;
      c[k] = (int64_t)u;
    }
    return (c[2] * n[1] + c[1]) * n[0] + c[0];
  }
};

// Signed distance of the box union (min over boxes), exact wherever it is
// below `margin`; returns +margin-or-more elsewhere.
inline double union_sdf(const std::vector<Box>& boxes, const CellIndex& idx, const double p[3],
                        double margin) {
  int64_t c = idx.cell_of(p);
  double best = 1e300;
  if (c < 0) {
    for (const Box& b : boxes) best = std::min(best, box_sdf(b, p));
    return best;
  }
  for (int64_t i = idx.start[c]; i < idx.start[c + 1]; ++i)
    best = std::min(best, box_sdf(boxes[idx.items[i]], p));
  return best == 1e300 ? 2.0 * margin + 1.0 : best;
}

uint16_t float_to_half_rne(float f) {
  uint32_t x;
  std::memcpy(&x, &f, 4);
  uint32_t sign = (x >> 16) & 0x8000u;
  uint32_t a = x & 0x7fffffffu;
  if (a >= 0x7f800000u) return (uint16_t)(sign | (a > 0x7f800000u ? 0x7e00u : 0x7c00u));
  if (a >= 0x477ff000u) return (uint16_t)(sign | 0x7c00u);
  if (a < 0x38800000u) {  // half subnormal range: units of 2^-24
    float af;
    std::memcpy(&af, &a, 4);
    return (uint16_t)(sign | (uint32_t)std::nearbyint(af * 16777216.0f));
  }
  uint32_t h = (((a >> 23) - 112u) << 10) | ((a & 0x7fffffu) >> 13);
  uint32_t rem = a & 0x1fffu;
  if (rem > 0x1000u || (rem == 0x1000u && (h & 1u))) ++h;
  return (uint16_t)(sign | h);
}

// dtype codes shared with the map descriptors: 0 = f32, 1 = f16, 2 = i16.
inline void store_value(void* out, int dtype, int64_t i, double v, double tau) {
  if (dtype == 0) {
    ((float*)out)[i] = (float)v;
  } else if (dtype == 1) {
    ((uint16_t*)out)[i] = float_to_half_rne((float)v);
  } else {
    double q = std::nearbyint(v / tau * 32767.0);
    q = std::min(32767.0, std::max(-32767.0, q));
    ((int16_t*)out)[i] = (int16_t)q;
  }
}

inline size_t dtype_size(int dtype) { return dtype == 0 ? 4 : 2; }

std::vector<Box> to_boxes(const double* b, int64_t n) {
  std::vector<Box> v((size_t)n);
  for (int64_t i = 0; i < n; ++i)
    for (int k = 0; k < 3; ++k) { v[i].lo[k] = b[6 * i + k]; v[i].hi[k] = b[6 * i + 3 + k]; }
  return v;
}

// Rotation of a sensor pose (x, y, z, roll, pitch, yaw): R = Rz(yaw) Ry(pitch) Rx(roll),
// in double. Used here only to lay out the synthetic rays of the true pose.
void rpy_matrix(const double rpy[3], double R[9]) {
  double cr = std::cos(rpy[0]), sr = std::sin(rpy[0]);
  double cp = std::cos(rpy[1]), sp = std::sin(rpy[1]);
  double cy = std::cos(rpy[2]), sy = std::sin(rpy[2]);
  R[0] = cy * cp; R[1] = cy * sp * sr - sy * cr; R[2] = cy * sp * cr + sy * sr;
  R[3] = sy * cp; R[4] = sy * sp * sr + cy * cr; R[5] = sy * sp * cr - cy * sr;
  R[6] = -sp;     R[7] = cp * sr;                R[8] = cp * cr;
}

}  // namespace

extern "C" {

// ---------------------------------------------------------------- scene layouts
// Every layout writes boxes as rows (lo_x, lo_y, lo_z, hi_x, hi_y, hi_z) in metres.
// With out == NULL the call only returns the number of boxes.

// Single room 6.4 x 6.4 x 3.2 m: four walls, floor, ceiling (0.2 m thick, inside
// the extent) and `n_objects` seeded axis-aligned boxes standing on the floor.
int64_t scn_layout_room(uint64_t seed, int64_t n_objects, double* out) {
  std::vector<Box> v;
  auto add = [&](double a, double b, double c, double d, double e, double f) {
    v.push_back(Box{{a, b, c}, {d, e, f}});
  };
  const double X = 6.4, Y = 6.4, Z = 3.2, t = 0.2;
  add(0, 0, 0, X, Y, t);          // floor
  add(0, 0, Z - t, X, Y, Z);      // ceiling
  add(0, 0, t, t, Y, Z - t);      // wall -x
  add(X - t, 0, t, X, Y, Z - t);  // wall +x
  add(t, 0, t, X - t, t, Z - t);  // wall -y
  add(t, Y - t, t, X - t, Y, Z - t);
  for (int64_t i = 0; i < n_objects; ++i) {
    double sx = 0.3 + 0.9 * unif(seed, 1, 4 * i), sy = 0.3 + 0.9 * unif(seed, 1, 4 * i + 1);
    double sz = 0.3 + 1.2 * unif(seed, 1, 4 * i + 2);
    double cx = t + 0.1 + (X - 2 * t - 0.2 - sx) * unif(seed, 1, 4 * i + 3);
    double cy = t + 0.1 + (Y - 2 * t - 0.2 - sy) * unif(seed, 2, i);
    add(cx, cy, t, cx + sx, cy + sy, t + sz);
  }
  if (out)
    for (size_t i = 0; i < v.size(); ++i)
      for (int k = 0; k < 3; ++k) { out[6 * i + k] = v[i].lo[k]; out[6 * i + 3 + k] = v[i].hi[k]; }
  return (int64_t)v.size();
}

// Multi-room hall 25.6 x 25.6 x 6.4 m: floor, ceiling, outer walls, a 4 x 4 grid
// of rooms separated by 0.15 m walls with seeded door openings, seeded pillars and
// `n_objects` boxes.
int64_t scn_layout_multiroom(uint64_t seed, int64_t n_objects, double* out) {
  std::vector<Box> v;
  auto add = [&](double a, double b, double c, double d, double e, double f) {
    v.push_back(Box{{a, b, c}, {d, e, f}});
  };
  const double X = 25.6, Y = 25.6, Z = 6.4, t = 0.2, w = 0.075;
  add(0, 0, 0, X, Y, t);
  add(0, 0, Z - t, X, Y, Z);
  add(0, 0, t, t, Y, Z - t);
  add(X - t, 0, t, X, Y, Z - t);
  add(t, 0, t, X - t, t, Z - t);
  add(t, Y - t, t, X - t, Y, Z - t);
  const double room = 6.4, door_w = 1.0, door_h = 2.2;
  uint64_t k = 0;
  for (int axis = 0; axis < 2; ++axis) {
    for (int i = 1; i < 4; ++i) {
      double c = i * room;
      for (int s = 0; s < 4; ++s) {
        double a0 = std::max(t, s * room), a1 = std::min(Y - t, (s + 1) * room);
        double d0 = a0 + 0.4 + (a1 - a0 - 0.8 - door_w) * unif(seed, 3, k++);
        double d1 = d0 + door_w;
        // segment [a0, d0) + [d1, a1) full height, lintel over the door
        double segs[3][4] = {{a0, d0, t, Z - t}, {d1, a1, t, Z - t}, {d0, d1, t + door_h, Z - t}};
        for (auto& g : segs) {
          if (axis == 0) add(c - w, g[0], g[2], c + w, g[1], g[3]);
          else add(g[0], c - w, g[2], g[1], c + w, g[3]);
        }
      }
    }
  }
  for (int i = 0; i < 16; ++i) {
    if (unif(seed, 4, 3 * i) < 0.5) continue;
    double rx = (i % 4) * room, ry = (i / 4) * room;
    double px = rx + 1.0 + (room - 2.4) * unif(seed, 4, 3 * i + 1);
    double py = ry + 1.0 + (room - 2.4) * unif(seed, 4, 3 * i + 2);
    add(px, py, t, px + 0.4, py + 0.4, Z - t);
  }
  for (int64_t i = 0; i < n_objects; ++i) {
    double sx = 0.3 + 1.2 * unif(seed, 5, 4 * i), sy = 0.3 + 1.2 * unif(seed, 5, 4 * i + 1);
    double sz = 0.3 + 1.5 * unif(seed, 5, 4 * i + 2);
    double cx = t + 0.2 + (X - 2 * t - 0.4 - sx) * unif(seed, 5, 4 * i + 3);
    double cy = t + 0.2 + (Y - 2 * t - 0.4 - sy) * unif(seed, 6, i);
    add(cx, cy, t, cx + sx, cy + sy, t + sz);
  }
  if (out)
    for (size_t i = 0; i < v.size(); ++i)
      for (int k2 = 0; k2 < 3; ++k2) { out[6 * i + k2] = v[i].lo[k2]; out[6 * i + 3 + k2] = v[i].hi[k2]; }
  return (int64_t)v.size();
}

// Multi-storey building X x Y m with `floors` storeys of 5 m (0.3 m slabs,
// 0.3 m roof), 0.3 m outer walls, interior walls on a 10 m grid (each 10 m
// segment present with probability 0.6, with a door with probability 0.7),
// pillars at grid crossings with probability 0.3 and `n_objects_per_floor`
// boxes per storey. The default workload is 160 x 160 m with four storeys.
int64_t scn_layout_building_sized(uint64_t seed, int64_t n_objects_per_floor, double X, double Y,
                                  int floors, double* out) {
  std::vector<Box> v;
  auto add = [&](double a, double b, double c, double d, double e, double f) {
    v.push_back(Box{{a, b, c}, {d, e, f}});
  };
  const double slab = 0.3, ow = 0.3, w = 0.1;
  const double storey = 5.0, grid = 10.0, door_w = 1.2, door_h = 2.4;
  const double Z = storey * floors;
  const int gx = (int)(X / grid), gy = (int)(Y / grid);
  for (int f = 0; f < floors; ++f) add(0, 0, f * storey, X, Y, f * storey + slab);
  add(0, 0, Z - slab, X, Y, Z);
  add(0, 0, 0, ow, Y, Z);
  add(X - ow, 0, 0, X, Y, Z);
  add(ow, 0, 0, X - ow, ow, Z);
  add(ow, Y - ow, 0, X - ow, Y, Z);
  uint64_t k = 0;
  for (int f = 0; f < floors; ++f) {
    double z0 = f * storey + slab, z1 = (f + 1 < floors) ? (f + 1) * storey : Z - slab;
    for (int axis = 0; axis < 2; ++axis) {
      const int nl = axis == 0 ? gx : gy, ns = axis == 0 ? gy : gx;
      const double span = axis == 0 ? Y : X;
      for (int i = 1; i < nl; ++i) {
        double c = i * grid;
        for (int s = 0; s < ns; ++s) {
          double p_present = unif(seed, 7, k++), p_door = unif(seed, 7, k++);
          double u_door = unif(seed, 7, k++);
          if (p_present >= 0.6) continue;
          double a0 = std::max(ow, s * grid), a1 = std::min(span - ow, (s + 1) * grid);
          if (p_door < 0.7) {
            double d0 = a0 + 0.5 + (a1 - a0 - 1.0 - door_w) * u_door, d1 = d0 + door_w;
            double segs[3][4] = {{a0, d0, z0, z1}, {d1, a1, z0, z1}, {d0, d1, z0 + door_h, z1}};
            for (auto& g : segs) {
              if (axis == 0) add(c - w, g[0], g[2], c + w, g[1], g[3]);
              else add(g[0], c - w, g[2], g[1], c + w, g[3]);
            }
          } else {
            if (axis == 0) add(c - w, a0, z0, c + w, a1, z1);
            else add(a0, c - w, z0, a1, c + w, z1);
          }
        }
      }
    }
    for (int i = 1; i < gx; ++i)
      for (int j = 1; j < gy; ++j) {
        if (unif(seed, 8, (uint64_t)((f * 16 + i) * 16 + j)) >= 0.3) continue;
        double cx = i * grid + 1.5, cy = j * grid + 1.5;
        add(cx - 0.3, cy - 0.3, z0, cx + 0.3, cy + 0.3, z1);
      }
    for (int64_t o = 0; o < n_objects_per_floor; ++o) {
      uint64_t b = (uint64_t)(f * n_objects_per_floor + o) * 5;
      double sx = 0.4 + 1.6 * unif(seed, 9, b), sy = 0.4 + 1.6 * unif(seed, 9, b + 1);
      double sz = 0.4 + 1.6 * unif(seed, 9, b + 2);
      double cx = ow + 0.5 + (X - 2 * ow - 1.0 - sx) * unif(seed, 9, b + 3);
      double cy = ow + 0.5 + (Y - 2 * ow - 1.0 - sy) * unif(seed, 9, b + 4);
      add(cx, cy, z0, cx + sx, cy + sy, z0 + sz);
    }
  }
  if (out)
    for (size_t i = 0; i < v.size(); ++i)
      for (int k2 = 0; k2 < 3; ++k2) { out[6 * i + k2] = v[i].lo[k2]; out[6 * i + 3 + k2] = v[i].hi[k2]; }
  return (int64_t)v.size();
}

int64_t scn_layout_building(uint64_t seed, int64_t n_objects_per_floor, double* out) {
  return scn_layout_building_sized(seed, n_objects_per_floor, 160.0, 160.0, 4, out);
}

// ---------------------------------------------------------------- analytic SDF
// Signed distance of the union of boxes at n points (exact, no truncation).
void scn_sdf(const double* boxes, int64_t nbox, const double* pts, int64_t n, double* out) {
  std::vector<Box> b = to_boxes(boxes, nbox);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double best = 1e300;
    for (const Box& x : b) best = std::min(best, box_sdf(x, pts + 3 * i));
    out[i] = best;
  }
}

// ---------------------------------------------------------------- voxelisation
// Dense TSDF: voxel (ix, iy, iz) covers [o + i*r, o + (i+1)*r) per axis and stores
// the union SDF at its centre o + (i + 1/2) r, clamped to [-tau, tau]. Layout
// x fastest: index (iz*ny + iy)*nx + ix. dtype 0 f32, 1 f16 (round to nearest
// even), 2 i16 (round(v/tau*32767)).
int scn_voxelize_dense(const double* boxes, int64_t nbox, const double origin[3], double voxel,
                       const int64_t dims[3], double tau, int dtype, void* out) {
  if (dtype < 0 || dtype > 2 || voxel <= 0 || tau <= 0) return -1;
  std::vector<Box> b = to_boxes(boxes, nbox);
  const int64_t B = 16;
  int64_t nb[3] = {(dims[0] + B - 1) / B, (dims[1] + B - 1) / B, (dims[2] + B - 1) / B};
  CellIndex idx;
  idx.build(b, origin, B * voxel, nb, tau + 1e-9);
  const int64_t nbrick = nb[0] * nb[1] * nb[2];
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t c = 0; c < nbrick; ++c) {
    int64_t bx = c % nb[0], by = (c / nb[0]) % nb[1], bz = c / (nb[0] * nb[1]);
    for (int64_t lz = 0; lz < B; ++lz)
      for (int64_t ly = 0; ly < B; ++ly)
        for (int64_t lx = 0; lx < B; ++lx) {
          int64_t ix = bx * B + lx, iy = by * B + ly, iz = bz * B + lz;
          if (ix >= dims[0] || iy >= dims[1] || iz >= dims[2]) continue;
          double p[3] = {origin[0] + (ix + 0.5) * voxel, origin[1] + (iy + 0.5) * voxel,
                         origin[2] + (iz + 0.5) * voxel};
          double best = 1e300;
          for (int64_t i = idx.start[c]; i < idx.start[c + 1]; ++i)
            best = std::min(best, box_sdf(b[idx.items[i]], p));
          double v = std::min(tau, std::max(-tau, best));
          store_value(out, dtype, (iz * dims[1] + iy) * dims[0] + ix, v, tau);
        }
  }
  return 0;
}

// Brick-sparse TSDF with 16^3 bricks over a grid of dims voxels (each a multiple
// of 16). A brick is kept iff one of its voxel centres has |sdf| < tau.
// scn_bricks_plan returns an opaque handle listing the kept bricks in
// (bz, by, bx) order; scn_bricks_fill writes their int32 (x, y, z) brick
// coordinates and their values (brick-major, x fastest inside a brick) into
// caller buffers, any of f32 / f16 / i16 (NULL to skip).
struct BrickPlan {
  std::vector<Box> boxes;
  CellIndex idx;
  double origin[3], voxel, tau;
  int64_t nb[3];
  std::vector<int64_t> cells;
};

static double brick_voxel_value(const BrickPlan& pl, int64_t c, int64_t lx, int64_t ly, int64_t lz) {
  const int64_t B = 16;
  int64_t bx = c % pl.nb[0], by = (c / pl.nb[0]) % pl.nb[1], bz = c / (pl.nb[0] * pl.nb[1]);
  double p[3] = {pl.origin[0] + (bx * B + lx + 0.5) * pl.voxel,
                 pl.origin[1] + (by * B + ly + 0.5) * pl.voxel,
                 pl.origin[2] + (bz * B + lz + 0.5) * pl.voxel};
  double best = 1e300;
  for (int64_t i = pl.idx.start[c]; i < pl.idx.start[c + 1]; ++i)
    best = std::min(best, box_sdf(pl.boxes[pl.idx.items[i]], p));
  return std::min(pl.tau, std::max(-pl.tau, best));
}

void* scn_bricks_plan(const double* boxes, int64_t nbox, const double origin[3], double voxel,
                      const int64_t dims[3], double tau, int64_t* n_bricks) {
  if (voxel <= 0 || tau <= 0) return nullptr;
  const int64_t B = 16;
  for (int k = 0; k < 3; ++k)
    if (dims[k] <= 0 || dims[k] % B) return nullptr;
  BrickPlan* pl = new BrickPlan();
  pl->boxes = to_boxes(boxes, nbox);
  for (int k = 0; k < 3; ++k) { pl->origin[k] = origin[k]; pl->nb[k] = dims[k] / B; }
  pl->voxel = voxel;
  pl->tau = tau;
  pl->idx.build(pl->boxes, origin, B * voxel, pl->nb, tau + 1e-9);
  const int64_t ncell = pl->nb[0] * pl->nb[1] * pl->nb[2];
  std::vector<uint8_t> keep((size_t)ncell, 0);
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t c = 0; c < ncell; ++c) {
    if (pl->idx.start[c] == pl->idx.start[c + 1]) continue;
    bool any = false;
    for (int64_t v = 0; v < B * B * B && !any; ++v)
      any = std::fabs(brick_voxel_value(*pl, c, v % B, (v / B) % B, v / (B * B))) < tau;
    keep[(size_t)c] = any ? 1 : 0;
  }
  for (int64_t c = 0; c < ncell; ++c)
    if (keep[(size_t)c]) pl->cells.push_back(c);
  *n_bricks = (int64_t)pl->cells.size();
  return pl;
}

void scn_bricks_fill(void* h, int32_t* coords, float* f32, uint16_t* f16, int16_t* i16) {
  const BrickPlan& pl = *(const BrickPlan*)h;
  const int64_t B = 16, V = B * B * B, n = (int64_t)pl.cells.size();
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < n; ++i) {
    int64_t c = pl.cells[(size_t)i];
    if (coords) {
      coords[3 * i + 0] = (int32_t)(c % pl.nb[0]);
      coords[3 * i + 1] = (int32_t)((c / pl.nb[0]) % pl.nb[1]);
      coords[3 * i + 2] = (int32_t)(c / (pl.nb[0] * pl.nb[1]));
    }
    for (int64_t v = 0; v < V; ++v) {
      double val = brick_voxel_value(pl, c, v % B, (v / B) % B, v / (B * B));
      if (f32) store_value(f32 + i * V, 0, v, val, pl.tau);
      if (f16) store_value(f16 + i * V, 1, v, val, pl.tau);
      if (i16) store_value(i16 + i * V, 2, v, val, pl.tau);
    }
  }
}

void scn_bricks_free(void* h) { delete (BrickPlan*)h; }

// ---------------------------------------------------------------- raycast scan
// LiDAR scan from `pose` (x, y, z, roll, pitch, yaw; R = Rz Ry Rx): `rings`
// elevations evenly spaced over [elev_min, elev_max] (degrees; a single ring sits
// at elev_min), `azimuths` directions evenly spaced over [-pi, pi). Points are
// ring-major (index ring*azimuths + a) in the sensor frame at the first box hit
// plus N(0, sigma^2) range noise. A ray that misses or whose noisy range falls
// outside [rmin, rmax] gets NaN coordinates and hit[i] = 0. Returns hit count.
int64_t scn_raycast(const double* boxes, int64_t nbox, const double pose[6], int64_t rings,
                    int64_t azimuths, double elev_min_deg, double elev_max_deg, double sigma,
                    double rmin, double rmax, uint64_t seed, float* pts, uint8_t* hit) {
  std::vector<Box> b = to_boxes(boxes, nbox);
  double R[9];
  rpy_matrix(pose + 3, R);
  const double deg = 3.141592653589793 / 180.0;
  const int64_t n = rings * azimuths;
  int64_t hits = 0;
#pragma omp parallel for schedule(static) reduction(+ : hits)
  for (int64_t i = 0; i < n; ++i) {
    int64_t r = i / azimuths, a = i % azimuths;
    double el = (rings > 1) ? (elev_min_deg + (elev_max_deg - elev_min_deg) * r / (rings - 1)) * deg
                            : elev_min_deg * deg;
    double az = -3.141592653589793 + 6.283185307179586 * (double)a / (double)azimuths;
    double ds[3] = {std::cos(el) * std::cos(az), std::cos(el) * std::sin(az), std::sin(el)};
    double dw[3];
    for (int k = 0; k < 3; ++k) dw[k] = R[3 * k] * ds[0] + R[3 * k + 1] * ds[1] + R[3 * k + 2] * ds[2];
    double best = 1e300;
    for (const Box& x : b) {
      double tn = -1e300, tf = 1e300;
      for (int k = 0; k < 3; ++k) {
        double inv = 1.0 / dw[k];
        double t0 = (x.lo[k] - pose[k]) * inv, t1 = (x.hi[k] - pose[k]) * inv;
        if (t0 > t1) std::swap(t0, t1);
        tn = std::fmax(tn, t0);
        tf = std::fmin(tf, t1);
      }
      if (tn <= tf && tn > 0.0 && tn < best) best = tn;
    }
    double range = best + sigma * normal(seed, 10, (uint64_t)i);
    bool ok = best < 1e299 && range >= rmin && range <= rmax;
    if (ok) {
      pts[3 * i + 0] = (float)(range * ds[0]);
      pts[3 * i + 1] = (float)(range * ds[1]);
      pts[3 * i + 2] = (float)(range * ds[2]);
      ++hits;
    } else {
      pts[3 * i + 0] = pts[3 * i + 1] = pts[3 * i + 2] = NAN;
    }
    if (hit) hit[i] = ok ? 1 : 0;
  }
  return hits;
}

// ---------------------------------------------------------------- particle clouds
// Gaussian cloud about `mean` (x, y, z, roll, pitch, yaw): per-axis sigma_t (m)
// for translation and sigma_r (rad) for rotation. Rows of 6 float32.
void scn_particles_gaussian(const double mean[6], double sigma_t, double sigma_r, int64_t P,
                            uint64_t seed, float* out) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < P; ++i)
    for (int k = 0; k < 6; ++k)
      out[6 * i + k] = (float)(mean[k] + (k < 3 ? sigma_t : sigma_r) *
                                            normal(seed, 11, (uint64_t)(6 * i + k)));
}

// Uniform cloud over free space: position uniform in [lo, hi] (3-vectors)
// rejected until the union SDF exceeds `clearance`; roll and pitch uniform in
// [-rp_max, rp_max] (rad), yaw uniform in [-pi, pi). Returns 0, or -1 if some
// particle found no free position within 4096 draws.
int scn_particles_free(const double* boxes, int64_t nbox, const double lo[3], const double hi[3],
                       double clearance, double rp_max, int64_t P, uint64_t seed, float* out) {
  std::vector<Box> b = to_boxes(boxes, nbox);
  const double cell = 0.8;
  int64_t nc[3];
  for (int k = 0; k < 3; ++k) nc[k] = std::max<int64_t>(1, (int64_t)std::ceil((hi[k] - lo[k]) / cell));
  CellIndex idx;
  idx.build(b, lo, cell, nc, clearance + 1e-9);
  int failed = 0;
#pragma omp parallel for schedule(static) reduction(| : failed)
  for (int64_t i = 0; i < P; ++i) {
    bool ok = false;
    for (uint64_t t = 0; t < 4096 && !ok; ++t) {
      uint64_t j = ((uint64_t)i << 12) | t;
      double p[3];
      for (int k = 0; k < 3; ++k) p[k] = lo[k] + (hi[k] - lo[k]) * unif(seed, 12 + k, j);
      if (union_sdf(b, idx, p, clearance) > clearance) {
        for (int k = 0; k < 3; ++k) out[6 * i + k] = (float)p[k];
        ok = true;
      }
    }
    if (!ok) failed = 1;
    out[6 * i + 3] = (float)(rp_max * (2.0 * unif(seed, 15, (uint64_t)i) - 1.0));
    out[6 * i + 4] = (float)(rp_max * (2.0 * unif(seed, 16, (uint64_t)i) - 1.0));
    out[6 * i + 5] = (float)(-3.141592653589793 + 6.283185307179586 * unif(seed, 17, (uint64_t)i));
  }
  return failed ? -1 : 0;
}

// Uniform doubles and standard normals of the generator, for tests and for
// drawing the resampling offset r and other scalar inputs.
void scn_uniform(uint64_t seed, uint64_t stream, int64_t n, double* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = unif(seed, stream, (uint64_t)i);
}
void scn_normal(uint64_t seed, uint64_t stream, int64_t n, double* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = normal(seed, stream, (uint64_t)i);
}

}  // extern "C"
