"""FP64 CPU oracle for the 6D MCL sensor update (ctypes wrapper of oracle.c).

TEST INFRASTRUCTURE: only the test suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import this package. The
library path never calls it, and it imports nothing from the CUDA package.

Every function follows a definition of the paper (Sec. III, Eq. 1-3; Sec. V-A)
with the readings listed in ``oracle.c``; each is pinned in
``tests/test_oracle_pins.py`` against closed forms, invariants or brute force.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_oracle.so")
_lock = threading.Lock()
_lib = None

LOGPROD, SUM, SCORE = 0, 1, 2
DENSE, BRICK, ANALYTIC = 0, 1, 2
PLANE, SPHERE, BOX = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle in place: plain C, OpenMP, no FP contraction."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-std=gnu11", "-O2", "-fopenmp", "-fPIC", "-shared",
                        "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _L():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P, i64, u64, dbl, flt, cint = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64,
                                           ctypes.c_double, ctypes.c_float, ctypes.c_int)
            lib.ora_map_create.argtypes = [cint, cint, P, flt, flt, flt, P, P, i64, P]
            lib.ora_map_create.restype = P
            lib.ora_map_create_analytic.argtypes = [i64, P, flt]
            lib.ora_map_create_analytic.restype = P
            lib.ora_map_destroy.argtypes = [P]
            lib.ora_map_set_outside.argtypes = [P, dbl]
            lib.ora_pose_to_matrix.argtypes = [P, i64, cint, P]
            lib.ora_sensor_update.argtypes = [P, P, i64, P, i64, dbl, cint, cint, cint, P]
            lib.ora_sensor_update_mat.argtypes = [P, P, i64, P, i64, dbl, cint, cint, cint, P]
            lib.ora_eval_points.argtypes = [P, P, P, i64, cint, cint, P, P, P]
            lib.ora_eval_points.restype = i64
            lib.ora_map_lookup.argtypes = [P, P, i64, P, P]
            lib.ora_normalise.argtypes = [P, i64, P, P, P]
            lib.ora_normalise.restype = cint
            lib.ora_resample.argtypes = [P, i64, dbl, P]
            lib.ora_resample.restype = cint
            lib.ora_philox4x32_10.argtypes = [P, P, P]
            lib.ora_motion_noise.argtypes = [u64, u64, i64, P]
            lib.ora_motion_update.argtypes = [P, i64, P, P, u64, u64]
            lib.ora_num_threads.restype = cint
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f32(a, shape_last=None) -> np.ndarray:
    a = np.ascontiguousarray(a, np.float32)
    return a


class Map:
    """Oracle view of a TSDF (dense, 16^3 bricks) or of an analytic primitive set.

    Holds references to the host arrays it reads; builds its own coarse
    brick-cell index (the fine/coarse split of Sec. III).
    """

    def __init__(self, handle, keep):
        self._h = handle
        self._keep = keep

    @classmethod
    def from_scene_map(cls, m) -> "Map":
        lib = _L()
        origin = np.asarray(m.origin, np.float32)
        dims = np.asarray(m.dims, np.int64)
        vals = np.ascontiguousarray(m.values)
        if m.kind == "dense":
            h = lib.ora_map_create(DENSE, m.dtype, _p(origin), float(np.float32(m.voxel)),
                                   float(m.inv_voxel), float(np.float32(m.tau)), _p(dims), _p(vals),
                                   0, None)
            keep = (origin, dims, vals)
        else:
            coords = np.ascontiguousarray(m.coords, np.int32)
            h = lib.ora_map_create(BRICK, m.dtype, _p(origin), float(np.float32(m.voxel)),
                                   float(m.inv_voxel), float(np.float32(m.tau)), _p(dims), _p(vals),
                                   len(coords), _p(coords))
            keep = (origin, dims, vals, coords)
        if not h:
            raise ValueError("oracle map: bad map description")
        return cls(h, keep)

    def set_outside(self, value: float) -> "Map":
        """Value read where nothing is stored (default +tau)."""
        _L().ora_map_set_outside(self._h, float(value))
        return self

    @classmethod
    def analytic(cls, prims, tau: float) -> "Map":
        pr = np.zeros((len(prims), 8), np.float64)
        for i, row in enumerate(prims):
            pr[i, :len(row)] = row
        h = _L().ora_map_create_analytic(len(pr), _p(pr), float(np.float32(tau)))
        return cls(h, (pr,))

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.ora_map_destroy(self._h)
            self._h = None


def pose_to_matrix(poses, parity: bool = True) -> np.ndarray:
    poses = _f32(poses).reshape(-1, 6)
    out = np.empty((len(poses), 3, 4), np.float64)
    _L().ora_pose_to_matrix(_p(poses), len(poses), int(parity), _p(out))
    return out


def _flags(neglect: bool, trilinear: bool) -> int:
    return int(bool(neglect)) | (2 if trilinear else 0)


def sensor_update(m: Map, poses, scan, sigma: float, mode: int = LOGPROD, neglect: bool = False,
                  parity: bool = True, trilinear: bool = False) -> np.ndarray:
    """Particle log-weights L_p (FP64) for one scan."""
    poses = _f32(poses).reshape(-1, 6)
    scan = _f32(scan).reshape(-1, 3)
    out = np.empty(len(poses), np.float64)
    _L().ora_sensor_update(m._h, _p(poses), len(poses), _p(scan), len(scan),
                           float(np.float32(sigma)), mode, _flags(neglect, trilinear), int(parity),
                           _p(out))
    return out


def sensor_update_mat(m: Map, mats, scan, sigma: float, mode: int = LOGPROD,
                      neglect: bool = False, parity: bool = False,
                      trilinear: bool = False) -> np.ndarray:
    """Particle log-weights for poses given as FP64 [R | t] matrices (P, 3, 4)."""
    mats = np.ascontiguousarray(mats, np.float64).reshape(-1, 12)
    scan = _f32(scan).reshape(-1, 3)
    out = np.empty(len(mats), np.float64)
    _L().ora_sensor_update_mat(m._h, _p(mats), len(mats), _p(scan), len(scan),
                               float(np.float32(sigma)), mode, _flags(neglect, trilinear),
                               int(parity), _p(out))
    return out


def eval_points(m: Map, pose, scan, parity: bool = True, trilinear: bool = False):
    """World points, read values d, voxel indices (-1 outside; the lower corner
    with trilinear) and count of stored reads."""
    pose = _f32(pose).reshape(6)
    scan = _f32(scan).reshape(-1, 3)
    x = np.empty((len(scan), 3), np.float64)
    d = np.empty(len(scan), np.float64)
    idx = np.empty((len(scan), 3), np.int64)
    n = _L().ora_eval_points(m._h, _p(pose), _p(scan), len(scan), int(parity), int(trilinear),
                             _p(x), _p(d), _p(idx))
    return x, d, idx, int(n)


def map_lookup(m: Map, pts):
    pts = _f32(pts).reshape(-1, 3)
    idx = np.empty(len(pts), np.int64)
    val = np.empty(len(pts), np.float64)
    _L().ora_map_lookup(m._h, _p(pts), len(pts), _p(idx), _p(val))
    return idx, val


def normalise(L):
    L = np.ascontiguousarray(L, np.float64)
    w = np.empty(len(L), np.float64)
    M = ctypes.c_double(0)
    S = ctypes.c_double(0)
    deg = _L().ora_normalise(_p(L), len(L), _p(w), ctypes.byref(M), ctypes.byref(S))
    return w, M.value, S.value, bool(deg)


def resample(w, r: float):
    w = _f32(w)
    idx = np.empty(len(w), np.int32)
    deg = _L().ora_resample(_p(w), len(w), float(r), _p(idx))
    return idx, bool(deg)


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    out = np.empty(4, np.uint32)
    _L().ora_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def motion_noise(seed: int, step: int, i: int) -> np.ndarray:
    out = np.empty(6, np.float64)
    _L().ora_motion_noise(seed, step, i, _p(out))
    return out


def motion_update(poses, delta, sigma, seed: int, step: int) -> np.ndarray:
    out = np.array(_f32(poses).reshape(-1, 6), copy=True)
    d = _f32(delta).reshape(6)
    s = _f32(sigma).reshape(6)
    _L().ora_motion_update(_p(out), len(out), _p(d), _p(s), seed, step)
    return out


def num_threads() -> int:
    return int(_L().ora_num_threads())


def _quat_of_pose(poses: np.ndarray) -> np.ndarray:
    """Unit quaternion (w, x, y, z) of R = Rz(yaw) Ry(pitch) Rx(roll) in FP64:
    the product q_z(yaw) * q_y(pitch) * q_x(roll) of the three elementary
    half-angle quaternions (Sec. III pose s = (x, y, z, phi, psi, theta))."""
    h = 0.5 * poses[:, 3:6].astype(np.float64)
    cr, sr = np.cos(h[:, 0]), np.sin(h[:, 0])
    cp, sp = np.cos(h[:, 1]), np.sin(h[:, 1])
    cy, sy = np.cos(h[:, 2]), np.sin(h[:, 2])
    return np.stack([cy * cp * cr + sy * sp * sr,
                     cy * cp * sr - sy * sp * cr,
                     cy * sp * cr + sy * cp * sr,
                     sy * cp * cr - cy * sp * sr], axis=1)


def pose_estimate(poses, w) -> dict:
    """Pose estimate of a weighted particle set (Sec. III: the weighted average
    of the particles, or the particle with the highest weight; Sec. V: the
    weights give the weighted sum of the poses). FP64 on the FP32 inputs:

      W         = sum_p w_p
      mean_pose = sum_p w_p s_p / W, each of the six components as a number
                  (the literal weighted average; its angles are meaningful only
                  while the particles' angles stay away from the +-pi wrap)
      quat      = unit eigenvector of the largest eigenvalue lambda of
                  Q = sum_p w_p q_p q_p^T / W, q_p the quaternion of R(s_p):
                  the rotation that minimises sum_p w_p ||R - R(s_p)||_F^2
                  (||R - R_p||^2 = 8 - 8 (q . q_p)^2); sign: first non-zero
                  component of (w, x, y, z) positive
      rpy       = that rotation as (roll, pitch, yaw), R = Rz Ry Rx
      concentration = lambda, in [1/4, 1]; 1 iff all weighted rotations agree
      n_eff     = W^2 / sum_p w_p^2 (0 if W = 0)
      argmax    = lowest p with the largest w_p (NaN weights ignored; -1 if
                  every weight is NaN), best_pose its row, best_w its weight.
    W = 0 gives NaN means."""
    s = np.ascontiguousarray(poses, np.float32).reshape(-1, 6)
    wf = np.ascontiguousarray(w, np.float32).reshape(-1)
    wd = wf.astype(np.float64)
    W = float(wd.sum())
    W2 = float((wd * wd).sum())
    with np.errstate(invalid="ignore", divide="ignore"):
        mean = (wd[:, None] * s.astype(np.float64)).sum(0) / W
    q = _quat_of_pose(s)
    Q = np.einsum("p,pi,pj->ij", wd, q, q)
    if W != 0.0 and np.all(np.isfinite(Q)):
        Q = Q / W
        lam, vec = np.linalg.eigh(Q)
        v = vec[:, -1].copy()
        nz = np.flatnonzero(v != 0.0)
        if len(nz) and v[nz[0]] < 0:
            v = -v
        qw, qx, qy, qz = v
        r21 = 2.0 * (qy * qz + qw * qx)
        r22 = 1.0 - 2.0 * (qx * qx + qy * qy)
        r20 = 2.0 * (qx * qz - qw * qy)
        r10 = 2.0 * (qx * qy + qw * qz)
        r00 = 1.0 - 2.0 * (qy * qy + qz * qz)
        rpy = np.array([math.atan2(r21, r22), math.asin(min(1.0, max(-1.0, -r20))),
                        math.atan2(r10, r00)])
        conc = float(lam[-1])
    else:
        v = np.full(4, np.nan)
        rpy = np.full(3, np.nan)
        conc = float("nan")
    if np.all(np.isnan(wf)):
        am = -1
    else:
        am = int(np.nanargmax(wf))
    return {
        "weight_sum": W,
        "n_eff": W * W / W2 if W2 > 0 else 0.0,
        "mean_pose": mean,
        "quat": v,
        "rpy": rpy,
        "concentration": conc,
        "argmax": am,
        "best_pose": s[am].copy() if am >= 0 else np.full(6, np.nan, np.float32),
        "best_w": float(wf[am]) if am >= 0 else float("nan"),
    }


def _dequantised(values, dtype: int, tau: float) -> np.ndarray:
    """Stored values as the real numbers they stand for (FP64); scaled int16
    stands for q * tau / 32767 (tau as FP32)."""
    v = np.asarray(values)
    if dtype == 2:
        return v.astype(np.float64) * (float(np.float32(tau)) / 32767.0)
    return v.astype(np.float64)


def score_of(d, sigma: float, dtype: int = 1) -> np.ndarray:
    """Per-voxel score exp(-d^2 / (2 sigma^2)) of Eq. 3 without its constant
    (Sec. III: the exponential evaluated once per map entry before the
    scans), in FP64 and rounded once to the storage type (FP16 or FP32,
    nearest even). sigma is read as FP32."""
    sig = float(np.float32(sigma))
    d = np.asarray(d, np.float64)
    e = np.exp(-(d * d) / (2.0 * sig * sig))
    return e.astype(np.float16 if dtype == 1 else np.float32)


def score_map(scene_map, sigma: float, dtype: int = 1):
    """(values, outside): the score map's stored values (same layout as the
    TSDF's) and the score read where nothing is stored (that of +tau)."""
    vals = score_of(_dequantised(scene_map.values, scene_map.dtype, scene_map.tau), sigma, dtype)
    outside = score_of(float(np.float32(scene_map.tau)), sigma, dtype)
    return vals, float(outside)
