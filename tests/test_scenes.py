"""Input generator checks (CPU): voxelisation against an independent NumPy
box-SDF, brick allocation against the dense grid, raycast points on surfaces,
exact point counts, particle clouds in free space, storage encodings."""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import scenes


def np_box_union_sdf(boxes, pts):
    """Signed distance to a union of axis-aligned boxes, written out in NumPy."""
    pts = np.asarray(pts, np.float64)[:, None, :]
    lo, hi = boxes[None, :, :3], boxes[None, :, 3:]
    g = np.maximum(lo - pts, pts - hi)
    outside = np.sqrt(np.sum(np.maximum(g, 0.0) ** 2, axis=-1))
    inside = np.minimum(np.max(g, axis=-1), 0.0)
    return np.min(outside + inside, axis=1)


def voxel_centres(origin, voxel, dims):
    nx, ny, nz = dims
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    c = np.stack([origin[0] + (ix + 0.5) * voxel, origin[1] + (iy + 0.5) * voxel,
                  origin[2] + (iz + 0.5) * voxel], axis=-1)
    return c.reshape(-1, 3)


def test_dense_voxelisation_matches_numpy_sdf():
    sc = scenes.room(1)
    dims, voxel, tau = (64, 64, 32), 0.1, 0.3
    m = scenes.voxelize_dense(sc, (0, 0, 0), voxel, dims, tau, scenes.F32)
    c = voxel_centres((0, 0, 0), voxel, dims)
    ref = np.clip(np_box_union_sdf(sc.boxes, c), -tau, tau).astype(np.float32)
    assert np.array_equal(m.values.reshape(-1), ref)


def test_plane_tsdf_closed_form():
    """A half-space z <= z0 gives TSDF clamp(c_z - z0, +-tau) at every voxel centre."""
    z0, tau, voxel, dims = 1.03125, 0.3, 0.0625, (32, 32, 32)
    sc = scenes.Scene("plane", np.array([[-100, -100, -100, 100, 100, z0]], np.float64),
                      (0, 0, 0), (2, 2, 2))
    m = scenes.voxelize_dense(sc, (0, 0, 0), voxel, dims, tau, scenes.F32)
    cz = (np.arange(32) + 0.5) * voxel
    ref = np.clip(cz - z0, -tau, tau).astype(np.float32)
    assert np.array_equal(m.values, np.broadcast_to(ref[:, None, None], m.values.shape))


def test_bricks_agree_with_dense_and_are_conservative():
    sc = scenes.room(1)
    dims, tau = (128, 128, 64), 0.3
    dense = scenes.voxelize_dense(sc, (0, 0, 0), 0.05, dims, tau, scenes.F32)
    br = scenes.voxelize_bricks(sc, (0, 0, 0), 0.05, dims, tau, scenes.F32)
    exp = scenes.bricks_to_dense(br).values
    v = dense.values
    near = np.abs(v) < tau
    assert np.array_equal(exp[near], v[near])          # every near-surface voxel is stored
    assert np.all(np.abs(v[exp == np.float32(tau)]) == np.float32(tau))  # the rest is clamped
    # a brick is kept iff it holds a voxel with |d| < tau
    blk = np.abs(v).reshape(4, 16, 8, 16, 8, 16).transpose(0, 2, 4, 1, 3, 5).reshape(4, 8, 8, -1)
    keep = (blk < tau).any(-1)
    got = np.zeros_like(keep)
    got[br.coords[:, 2], br.coords[:, 1], br.coords[:, 0]] = True
    assert np.array_equal(keep, got)
    # coordinates sorted by (bz, by, bx), no duplicates
    key = (br.coords[:, 2] * 8 + br.coords[:, 1]) * 8 + br.coords[:, 0]
    assert np.all(np.diff(key) > 0)


def test_storage_encodings():
    sc = scenes.room(1)
    ms = scenes.voxelize_bricks_multi(sc, (0, 0, 0), 0.05, (128, 128, 64), 0.3,
                                      (scenes.F32, scenes.F16, scenes.I16))
    f32, f16, i16 = ms[scenes.F32].values, ms[scenes.F16].values, ms[scenes.I16].values
    assert np.array_equal(f16, f32.astype(np.float16))  # round to nearest even
    q = np.clip(np.rint(f32.astype(np.float64) / 0.3 * 32767), -32767, 32767)
    assert np.max(np.abs(q - i16)) <= 1  # encoded from the FP64 value, not the FP32 one
    assert np.max(np.abs(i16 * (0.3 / 32767) - f32)) <= 0.3 / 32767


@pytest.mark.parametrize("maker,n", [("room", 1024), ("multiroom", 28800)])
def test_raycast_counts_and_surface(maker, n):
    sc = getattr(scenes, maker)()
    az = 64 if maker == "room" else 1800
    kw = dict(scenes.VLP16, azimuths=az, rmax=30.0 if maker == "room" else 100.0)
    pose, scan = scenes.true_pose(sc, 5, kw)
    assert scan.shape == (n, 3) and np.isfinite(scan).all()
    kw0 = dict(kw, sigma=0.0)
    pts, hit = scenes.raycast(sc, pose, seed=9, **kw0)
    assert hit.all()
    R = Rotation.from_euler("xyz", pose[3:]).as_matrix()
    world = pts.astype(np.float64) @ R.T + pose[:3]
    assert np.max(np.abs(np_box_union_sdf(sc.boxes, world))) < 2e-5


def test_os064_scan_shape_on_building():
    sc = scenes.building()
    pose, scan = scenes.true_pose(sc, 3, dict(scenes.OS064, azimuths=1024))
    assert scan.shape == (65536, 3) and np.isfinite(scan).all()
    r = np.linalg.norm(scan, axis=1)
    assert r.min() >= 0.3 and r.max() <= 100.0
    el = np.degrees(np.arcsin(scan[:, 2] / r)).reshape(64, 1024)
    assert abs(el[0].mean() + 45) < 0.01 and abs(el[-1].mean() - 45) < 0.01


def test_particles():
    sc = scenes.building()
    p = scenes.particles_free(sc, 20000, 0.1, 10.0, 4)
    assert p.shape == (20000, 6) and p.dtype == np.float32
    assert np.all(np_box_union_sdf(sc.boxes[:], p[:2000, :3].astype(np.float64)) > 0.1 - 1e-6)
    assert np.all(np.abs(p[:, 3:5]) <= math.radians(10) + 1e-6)
    assert np.all(np.abs(p[:, 5]) <= math.pi + 1e-6)
    g = scenes.particles_gaussian([1, 2, 3, 0.1, 0.2, 0.3], 200000, 0.2, 2.0, 5)
    assert np.allclose(g.mean(0), [1, 2, 3, 0.1, 0.2, 0.3], atol=3e-3)
    assert np.allclose(g.std(0), [0.2] * 3 + [math.radians(2)] * 3, rtol=1e-2)
    # counter-based: a prefix does not depend on the total count
    assert np.array_equal(scenes.particles_gaussian([0] * 6, 10, 1, 1, 5),
                          scenes.particles_gaussian([0] * 6, 1000, 1, 1, 5)[:10])
