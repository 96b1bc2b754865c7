"""Seeded synthetic inputs for 6D MCL in TSDF maps.

Box-set environments shaped like the paper's workloads (an office-like room
and multi-room hall seen by a VLP-16-shaped scanner, a multi-storey building
seen by an OS0-64-shaped scanner; paper Sec. VI), their TSDF voxelisation
(dense grid or 16^3 bricks kept only within the truncation distance of a
surface, paper Sec. III), raycast scans with Gaussian range noise and particle
clouds (Gaussian about a pose estimate, or uniform over free space; paper
Sec. III, Eq. 1-2).

This module generates inputs only. It holds none of the sensor-update
arithmetic and is shared by the FP64 oracle and the CUDA path alike. The
native part (``csrc/scenes.cpp``) is compiled on first use with g++ and
OpenMP.
"""
from __future__ import annotations

import ctypes
import functools
import math
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csrc", "scenes.cpp")
_LIB = os.path.join(_HERE, "_scenes.so")
_lock = threading.Lock()
_lib = None

F32, F16, I16 = 0, 1, 2
DTYPE_NP = {F32: np.float32, F16: np.float16, I16: np.int16}
BRICK = 16


def build(force: bool = False) -> str:
    """Compile the generator library in place (g++ -O2 -fopenmp)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
               _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _L():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            i64, u64, dbl = ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
            for name in ("scn_layout_room", "scn_layout_multiroom", "scn_layout_building"):
                getattr(lib, name).argtypes = [u64, i64, P]
                getattr(lib, name).restype = i64
            lib.scn_layout_building_sized.argtypes = [u64, i64, dbl, dbl, ctypes.c_int, P]
            lib.scn_layout_building_sized.restype = i64
            lib.scn_sdf.argtypes = [P, i64, P, i64, P]
            lib.scn_voxelize_dense.argtypes = [P, i64, P, dbl, P, dbl, ctypes.c_int, P]
            lib.scn_voxelize_dense.restype = ctypes.c_int
            lib.scn_bricks_plan.argtypes = [P, i64, P, dbl, P, dbl, P]
            lib.scn_bricks_plan.restype = P
            lib.scn_bricks_fill.argtypes = [P, P, P, P, P]
            lib.scn_bricks_free.argtypes = [P]
            lib.scn_raycast.argtypes = [P, i64, P, i64, i64, dbl, dbl, dbl, dbl, dbl, u64, P, P]
            lib.scn_raycast.restype = i64
            lib.scn_particles_gaussian.argtypes = [P, dbl, dbl, i64, u64, P]
            lib.scn_particles_free.argtypes = [P, i64, P, P, dbl, dbl, i64, u64, P]
            lib.scn_particles_free.restype = ctypes.c_int
            lib.scn_uniform.argtypes = [u64, u64, i64, P]
            lib.scn_normal.argtypes = [u64, u64, i64, P]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# ------------------------------------------------------------------ layouts
@dataclass
class Scene:
    name: str
    boxes: np.ndarray  # (n, 6) float64 rows lo_xyz, hi_xyz
    lo: tuple
    hi: tuple
    floors: tuple = (0.0,)  # heights of the walkable floors (top of slab)


def _layout(fn: str, seed: int, n: int) -> np.ndarray:
    lib = _L()
    cnt = getattr(lib, fn)(seed, n, None)
    out = np.zeros((cnt, 6), np.float64)
    getattr(lib, fn)(seed, n, _ptr(out))
    return out


def room(seed: int = 1, n_objects: int = 10) -> Scene:
    return Scene("room", _layout("scn_layout_room", seed, n_objects), (0, 0, 0), (6.4, 6.4, 3.2),
                 (0.2,))


def multiroom(seed: int = 2, n_objects: int = 40) -> Scene:
    return Scene("multiroom", _layout("scn_layout_multiroom", seed, n_objects), (0, 0, 0),
                 (25.6, 25.6, 6.4), (0.2,))


def building(seed: int = 3, n_objects_per_floor: int = 150, size: float = 160.0,
             floors: int = 4) -> Scene:
    """size x size m building with `floors` storeys of 5 m (default 160 x 160 x 20 m)."""
    lib = _L()
    cnt = lib.scn_layout_building_sized(seed, n_objects_per_floor, size, size, floors, None)
    boxes = np.zeros((cnt, 6), np.float64)
    lib.scn_layout_building_sized(seed, n_objects_per_floor, size, size, floors, _ptr(boxes))
    return Scene("building", boxes, (0, 0, 0), (size, size, 5.0 * floors),
                 tuple(5.0 * f + 0.3 for f in range(floors)))


def sdf(scene: Scene, pts) -> np.ndarray:
    pts = np.ascontiguousarray(pts, np.float64).reshape(-1, 3)
    out = np.empty(len(pts), np.float64)
    _L().scn_sdf(_ptr(scene.boxes), len(scene.boxes), _ptr(pts), len(pts), _ptr(out))
    return out


# ------------------------------------------------------------------ maps
@dataclass
class DenseMap:
    """Dense TSDF: values[(iz*ny + iy)*nx + ix] at voxel centres, clamped to +-tau."""
    origin: tuple
    voxel: float
    dims: tuple  # (nx, ny, nz)
    tau: float
    dtype: int
    values: np.ndarray  # shape (nz, ny, nx)
    kind: str = "dense"

    @property
    def inv_voxel(self) -> float:
        """Map-header reciprocal of the voxel edge, as the FP32 value both sides read."""
        return float(np.float32(1.0 / np.float64(np.float32(self.voxel))))


@dataclass
class BrickMap:
    """16^3-brick TSDF: coords (B, 3) int32 brick units; values (B, 16, 16, 16), x fastest."""
    origin: tuple
    voxel: float
    dims: tuple  # grid extent in voxels, multiples of 16
    tau: float
    dtype: int
    coords: np.ndarray
    values: np.ndarray
    kind: str = "brick"

    @property
    def inv_voxel(self) -> float:
        """Map-header reciprocal of the voxel edge, as the FP32 value both sides read."""
        return float(np.float32(1.0 / np.float64(np.float32(self.voxel))))

    @property
    def nbytes(self) -> int:
        return int(self.values.nbytes)


def voxelize_dense(scene: Scene, origin, voxel: float, dims, tau: float, dtype: int = F32) -> DenseMap:
    o = np.asarray(origin, np.float64)
    d = np.asarray(dims, np.int64)
    vals = np.empty((int(d[2]), int(d[1]), int(d[0])), DTYPE_NP[dtype])
    rc = _L().scn_voxelize_dense(_ptr(scene.boxes), len(scene.boxes), _ptr(o), float(voxel),
                                 _ptr(d), float(tau), dtype, _ptr(vals))
    if rc != 0:
        raise ValueError("voxelize_dense: bad arguments")
    return DenseMap(tuple(float(x) for x in origin), float(voxel), tuple(int(x) for x in dims),
                    float(tau), dtype, vals)


def voxelize_bricks_multi(scene: Scene, origin, voxel: float, dims, tau: float,
                          dtypes=(I16,)) -> dict:
    """Brick maps of one scene in several storage types from a single voxelisation pass."""
    lib = _L()
    o = np.asarray(origin, np.float64)
    d = np.asarray(dims, np.int64)
    nb = ctypes.c_int64(0)
    h = lib.scn_bricks_plan(_ptr(scene.boxes), len(scene.boxes), _ptr(o), float(voxel), _ptr(d),
                            float(tau), ctypes.byref(nb))
    if not h:
        raise ValueError("voxelize_bricks: bad arguments (dims must be multiples of 16)")
    try:
        coords = np.empty((nb.value, 3), np.int32)
        vals = {dt: np.empty((nb.value, BRICK, BRICK, BRICK), DTYPE_NP[dt]) for dt in dtypes}
        ptrs = [_ptr(vals[dt]) if dt in vals else None for dt in (F32, F16, I16)]
        lib.scn_bricks_fill(h, _ptr(coords), *ptrs)
    finally:
        lib.scn_bricks_free(h)
    meta = (tuple(float(x) for x in origin), float(voxel), tuple(int(x) for x in dims), float(tau))
    return {dt: BrickMap(*meta, dt, coords, vals[dt]) for dt in dtypes}


def voxelize_bricks(scene: Scene, origin, voxel: float, dims, tau: float, dtype: int = I16) -> BrickMap:
    return voxelize_bricks_multi(scene, origin, voxel, dims, tau, (dtype,))[dtype]


def bricks_to_dense(m: BrickMap) -> DenseMap:
    """Expand a brick map to a dense grid; unallocated voxels hold +tau (for small tests)."""
    nx, ny, nz = m.dims
    if m.dtype == F32:
        fill = np.float32(m.tau)
    elif m.dtype == F16:
        fill = np.float16(m.tau)
    else:
        fill = np.int16(32767)
    out = np.full((nz, ny, nx), fill, DTYPE_NP[m.dtype])
    for (bx, by, bz), v in zip(m.coords, m.values):
        out[bz * 16:(bz + 1) * 16, by * 16:(by + 1) * 16, bx * 16:(bx + 1) * 16] = v
    return DenseMap(m.origin, m.voxel, m.dims, m.tau, m.dtype, out)


# ------------------------------------------------------------------ scans and particles
def raycast(scene: Scene, pose, rings: int, azimuths: int, elev_min_deg: float, elev_max_deg: float,
            sigma: float, rmin: float, rmax: float, seed: int):
    """Ring-major (rings*azimuths, 3) float32 sensor-frame points and a hit mask."""
    p = np.asarray(pose, np.float64)
    n = rings * azimuths
    pts = np.empty((n, 3), np.float32)
    hit = np.empty(n, np.uint8)
    _L().scn_raycast(_ptr(scene.boxes), len(scene.boxes), _ptr(p), rings, azimuths,
                     float(elev_min_deg), float(elev_max_deg), float(sigma), float(rmin),
                     float(rmax), seed, _ptr(pts), _ptr(hit))
    return pts, hit.astype(bool)


def particles_gaussian(mean, P: int, sigma_t: float, sigma_r_deg: float, seed: int) -> np.ndarray:
    m = np.asarray(mean, np.float64)
    out = np.empty((P, 6), np.float32)
    _L().scn_particles_gaussian(_ptr(m), float(sigma_t), math.radians(sigma_r_deg), P, seed,
                                _ptr(out))
    return out


def particles_free(scene: Scene, P: int, clearance: float, rp_max_deg: float, seed: int) -> np.ndarray:
    lo = np.asarray(scene.lo, np.float64)
    hi = np.asarray(scene.hi, np.float64)
    out = np.empty((P, 6), np.float32)
    rc = _L().scn_particles_free(_ptr(scene.boxes), len(scene.boxes), _ptr(lo), _ptr(hi),
                                 float(clearance), math.radians(rp_max_deg), P, seed, _ptr(out))
    if rc != 0:
        raise RuntimeError("particles_free: no free position found for some particle")
    return out


def uniform(seed: int, stream: int, n: int) -> np.ndarray:
    out = np.empty(n, np.float64)
    _L().scn_uniform(seed, stream, n, _ptr(out))
    return out


def normal(seed: int, stream: int, n: int) -> np.ndarray:
    out = np.empty(n, np.float64)
    _L().scn_normal(seed, stream, n, _ptr(out))
    return out


def true_pose(scene: Scene, seed: int, scan_kw: dict, clearance: float = 0.5,
              max_tries: int = 256):
    """A seeded sensor pose in free space from which every ray of the scan hits."""
    u = uniform(seed, 100, 6 * max_tries).reshape(max_tries, 6)
    lo, hi = np.asarray(scene.lo), np.asarray(scene.hi)
    for t in range(max_tries):
        floor = scene.floors[int(u[t, 2] * len(scene.floors)) % len(scene.floors)]
        pos = np.array([lo[0] + 0.5 + (hi[0] - lo[0] - 1.0) * u[t, 0],
                        lo[1] + 0.5 + (hi[1] - lo[1] - 1.0) * u[t, 1],
                        floor + 1.0 + 0.8 * u[t, 3]])
        if sdf(scene, pos)[0] <= clearance:
            continue
        pose = np.array([*pos, math.radians(4.0 * (u[t, 4] - 0.5)),
                         math.radians(4.0 * (u[t, 5] - 0.5)),
                         -math.pi + 2 * math.pi * ((u[t, 0] * 7.31) % 1.0)])
        pts, hit = raycast(scene, pose, seed=seed + 1000 + t, **scan_kw)
        if hit.all():
            return pose, pts
    raise RuntimeError("true_pose: no pose with a full scan")


def _rot(rpy):
    """R = Rz(yaw) Ry(pitch) Rx(roll) (FP64, the pose convention of the inputs)."""
    r, p, y = rpy
    cr, sr, cp, sp, cy, sy = math.cos(r), math.sin(r), math.cos(p), math.sin(p), math.cos(y), math.sin(y)
    return np.array([[cy * cp, cy * sp * sr - sy * cr, cy * sp * cr + sy * sr],
                     [sy * cp, sy * sp * sr + cy * cr, sy * sp * cr - cy * sr],
                     [-sp, cp * sr, cp * cr]])


def trajectory(scene: Scene, start, steps: int, seed: int, step_len: float = 0.1,
               clearance: float = 0.4):
    """A seeded robot path through free space: each step moves step_len
    forward in the body frame and turns by a yaw increment chosen from a
    small set (the first in a seeded order that keeps the new position and
    the midpoint more than `clearance` from every surface; else it turns in
    place by 90 degrees). Returns the true poses (steps + 1, 6) in FP64 and
    the odometry increments (steps, 6) FP32 in the body frame: the simulated
    sensor input of a motion update."""
    u = uniform(seed, 200, steps)
    turns = np.radians([0.0, 5.0, -5.0, 15.0, -15.0, 40.0, -40.0])
    poses = [np.asarray(start, np.float64).copy()]
    deltas = []
    for k in range(steps):
        cur = poses[-1]
        R = _rot(cur[3:])
        order = np.roll(np.arange(len(turns)), int(u[k] * 3)) if u[k] < 0.5 else np.arange(len(turns))
        step = None
        for i in order:
            fwd = R @ np.array([step_len, 0.0, 0.0])
            mid, new = cur[:3] + 0.5 * fwd, cur[:3] + fwd
            if sdf(scene, mid)[0] > clearance and sdf(scene, new)[0] > clearance:
                step = np.array([step_len, 0.0, 0.0, 0.0, 0.0, turns[i]])
                break
        if step is None:
            step = np.array([0.0, 0.0, 0.0, 0.0, 0.0, math.pi / 2])
        R2 = R @ _rot(step[3:])
        t2 = cur[:3] + R @ step[:3]
        rpy = np.array([math.atan2(R2[2, 1], R2[2, 2]), math.asin(max(-1.0, min(1.0, -R2[2, 0]))),
                        math.atan2(R2[1, 0], R2[0, 0])])
        poses.append(np.concatenate([t2, rpy]))
        deltas.append(step.astype(np.float32))
    return np.array(poses), np.array(deltas, np.float32).reshape(steps, 6)


def trajectory_scans(scene: Scene, poses, scan_kw: dict, seed: int):
    """Scans raycast from each true pose; rays without a hit are dropped, so N varies."""
    out = []
    for k, pose in enumerate(poses):
        pts, hit = raycast(scene, pose, seed=seed + 7919 * k, **scan_kw)
        out.append(np.ascontiguousarray(pts[hit]))
    return out


# ------------------------------------------------------------------ workloads
@dataclass
class Workload:
    name: str
    scene: Scene
    map: object
    scan: np.ndarray  # (N, 3) float32, sensor frame
    particles: np.ndarray  # (P, 6) float32
    pose: np.ndarray  # true pose (6,)
    sigma_hit: float
    info: dict = field(default_factory=dict)


VLP16 = dict(rings=16, elev_min_deg=-15.0, elev_max_deg=15.0, sigma=0.02, rmin=0.3)
OS064 = dict(rings=64, elev_min_deg=-45.0, elev_max_deg=45.0, sigma=0.02, rmin=0.3, rmax=100.0)


def room_plain(P: int = 1000, dtype: int = F32, seed: int = 1) -> Workload:
    """Dense 128x128x64 room at 5 cm, tau 0.3, 16x64 VLP-16-shaped scan, Gaussian cloud."""
    sc = room(seed)
    m = voxelize_dense(sc, (0.0, 0.0, 0.0), 0.05, (128, 128, 64), 0.3, dtype)
    kw = dict(VLP16, azimuths=64, rmax=30.0)
    pose, scan = true_pose(sc, seed, kw)
    parts = particles_gaussian(pose, P, 0.2, 2.0, seed + 7)
    return Workload("room_plain_128x128x64_1024pts", sc, m, scan, parts, pose, 0.1)


def vlp16_multiroom(P: int = 50_000, dtype: int = F32, seed: int = 2) -> Workload:
    """Dense 512x512x128 multi-room hall at 5 cm, 16x1800 VLP-16 scan, Gaussian cloud."""
    sc = multiroom(seed)
    m = voxelize_dense(sc, (0.0, 0.0, 0.0), 0.05, (512, 512, 128), 0.3, dtype)
    kw = dict(VLP16, azimuths=1800, rmax=100.0)
    pose, scan = true_pose(sc, seed, kw)
    parts = particles_gaussian(pose, P, 0.2, 2.0, seed + 7)
    return Workload("vlp16_multiroom_512x512x128_28800pts", sc, m, scan, parts, pose, 0.1)


@functools.lru_cache(maxsize=2)
def _building_maps(seed: int, dtypes: tuple, size: float, floors: int):
    sc = building(seed, size=size, floors=floors)
    up16 = lambda v: -(-int(round(v / 0.05)) // 16) * 16  # grid rounded up to whole bricks
    dims = (up16(size), up16(size), up16(5.0 * floors))
    return sc, voxelize_bricks_multi(sc, (0.0, 0.0, 0.0), 0.05, dims, 0.3, dtypes)


def os064_building(P: int = 1_000_000, dtype: int = I16, seed: int = 3, azimuths: int = 1024,
                   size: float = 160.0, floors: int = 4, dtypes: tuple | None = None) -> Workload:
    """Brick-sparse building (default 160x160x20 m) at 5 cm in 16^3 bricks, OS0-64 scan of
    64 rings x `azimuths`, uniform free-space cloud (roll/pitch within 10 deg, yaw uniform).
    `dtypes` voxelises several storage types in one pass (Workload.info['maps'])."""
    dts = tuple(dtypes) if dtypes else (dtype,)
    sc, maps = _building_maps(seed, dts, size, floors)
    m = maps[dtype]
    kw = dict(OS064, azimuths=azimuths)
    pose, scan = true_pose(sc, seed, kw)
    parts = particles_free(sc, P, 0.1, 10.0, seed + 7)
    name = f"os064_building_{int(size)}m_{floors}fl_bricks{len(m.coords)}_{P}x{64 * azimuths}"
    return Workload(name, sc, m, scan, parts, pose, 0.1,
                    {"bricks": int(len(m.coords)), "map_bytes": m.nbytes, "maps": maps})
