"""The sensor kernels' voxel rule at its edges, against the oracle's FP32 rule.

Both sides form u per axis from the pose rows in the map's index frame
(R inv and (t - o) inv, FP64 then one FP32 rounding) and one FP32 fma chain;
the kernels take floor(u) from the bits of a round-down u + 2^23 and test
0 <= u < n with one unsigned compare per axis (packed FP32x2 for two points
at a time); the oracle compares u with 0 and n in FP32 and truncates (Sec.
III look-up; readings r3 and r19). Here every particle sits at an adversarial
position with identity rotation and the scan is one point at the sensor
origin, so a particle's log-weight is the score of exactly the voxel its
position falls in, or of +tau outside: voxel faces, -0, one ulp below 0,
one ulp below n, n, 2^23 and beyond, 1e30, +-inf, NaN, on maps with negative
and positive origins. Neighbouring voxels hold distinct values, so a wrong
voxel shows as a wrong log-weight. The trilinear read is taken at its own
edges (f = u - 1/2 at and next to -1, 0, n - 1 and n, corners below the first
and past the last brick cell on one axis or on all three at once), with the
cell-grid and the hash index giving the same bits.
"""
import math

import numpy as np
import pytest

import oracle
import scenes

pytestmark = pytest.mark.gpu

TAU = 0.3


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2310_04172_gb300 import _build, mcl
    _build.build()
    mcl.lib()
    torch.cuda.set_device(0)
    return torch, mcl


def values_f64(dims):
    nx, ny, nz = dims
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return TAU * (((7 * ix + 13 * iy + 29 * iz) % 61) / 30.5 - 1.0)


def quantise(v, dtype):
    if dtype == scenes.F32:
        return v.astype(np.float32)
    if dtype == scenes.F16:
        return v.astype(np.float16)
    return np.rint(v / TAU * 32767.0).astype(np.int16)


def dense_map(origin, dims, dtype):
    v = quantise(values_f64(dims), dtype)
    return scenes.DenseMap(tuple(origin), 0.05, tuple(dims), TAU, dtype, v)


def brick_map(origin, dims, dtype):
    """All bricks of the extent but one (which reads +tau)."""
    full = quantise(values_f64(dims), dtype)  # (nz, ny, nx)
    nb = [d // 16 for d in dims]
    coords, vals = [], []
    for bz in range(nb[2]):
        for by in range(nb[1]):
            for bx in range(nb[0]):
                if (bx, by, bz) == (1, 0, 1):
                    continue
                coords.append((bx, by, bz))
                vals.append(full[16 * bz:16 * bz + 16, 16 * by:16 * by + 16, 16 * bx:16 * bx + 16])
    return scenes.BrickMap(tuple(origin), 0.05, tuple(dims), TAU, dtype,
                           np.array(coords, np.int32), np.ascontiguousarray(np.stack(vals)))


def edge_positions(origin, dims, voxel=0.05):
    """Positions whose u = (x - o) / r sits at or next to the rule's edges on
    one axis, the other two coordinates well inside."""
    o = np.asarray(origin, np.float32)
    mid = o + np.float32(voxel) * (np.asarray(dims, np.float32) / 2 + np.float32(0.3))
    pts = []
    for axis in range(3):
        n = dims[axis]
        cand = []
        for u in (0.0, 1.0, 2.0, n - 1.0, float(n), n + 1.0, 0.5, n - 0.5, 2.0 ** 23, 2.0 ** 24):
            x = np.float32(o[axis] + np.float64(u) * voxel)
            cand += [x, np.nextafter(x, np.float32(-np.inf)), np.nextafter(x, np.float32(np.inf)),
                     np.nextafter(np.nextafter(x, np.float32(-np.inf)), np.float32(-np.inf))]
        cand += [o[axis], np.float32(-0.0), np.float32(0.0), np.float32(1e30), np.float32(-1e30),
                 np.float32(np.inf), np.float32(-np.inf), np.float32(np.nan),
                 np.nextafter(o[axis], np.float32(-np.inf))]
        for c in cand:
            p = mid.copy()
            p[axis] = c
            pts.append(p)
    # face crossings in every axis at once
    for k in range(0, 17):
        pts.append(o + np.float32(0.05) * np.float32(k) + np.zeros(3, np.float32))
    return np.array(pts, np.float32)


def run_case(torch, mcl, smap, layout=0, index=0):
    pos = edge_positions(smap.origin, smap.dims)
    parts = np.zeros((len(pos), 6), np.float32)
    parts[:, :3] = pos
    scan = np.zeros((1, 3), np.float32)
    m = mcl.map_from_scene(smap, layout, index) if smap.kind == "brick" else mcl.map_from_scene(smap)
    P = len(parts)
    logw = torch.empty(P, device="cuda")
    results = []
    for shape in (dict(), dict(lanes_per_particle=8), dict(unroll=4), dict(unroll=2)):
        prm = mcl.sensor_params(0.1, **shape)
        mcl.mcl_sensor_update(m, torch.from_numpy(parts).cuda(), torch.from_numpy(scan).cuda(), prm, logw)
        mcl.mcl_sync()
        results.append(logw.cpu().numpy().astype(np.float64))
    m.close()
    Lo = oracle.sensor_update(oracle.Map.from_scene_map(smap), parts, scan, 0.1)
    for Lg in results:
        assert np.array_equal(Lg, results[0])  # the same bits whatever the launch shape
        err = np.abs(Lg - Lo) / np.maximum(1.0, np.abs(Lo))
        bad = np.flatnonzero(~(err <= 1e-5))
        assert len(bad) == 0, f"positions {pos[bad[:5]]}: GPU {Lg[bad[:5]]} oracle {Lo[bad[:5]]}"
    # the outside value is reached for the far positions, so both branches are exercised
    outside = -(TAU * TAU) / (2 * 0.01)
    assert np.any(np.isclose(Lo, outside, rtol=1e-6)) and np.any(~np.isclose(Lo, outside, rtol=1e-6))


@pytest.mark.parametrize("origin", [(0.0, 0.0, 0.0), (-1.6, -0.8, -0.4), (3.15, -2.05, 0.6)])
@pytest.mark.parametrize("dtype", [scenes.F32, scenes.F16, scenes.I16])
@pytest.mark.parametrize("dims", [(48, 32, 32), (45, 30, 21)])
def test_dense_index_edges(env, origin, dtype, dims):
    """Dense grids are stored in 8 x 4 tiles (45 x 30: partial tiles along
    x and y)."""
    torch, mcl = env
    run_case(torch, mcl, dense_map(origin, dims, dtype))


@pytest.mark.parametrize("dims", [(48, 32, 32), (45, 30, 21), (7, 3, 5)])
def test_dense_tiles_trilinear_and_score_map(env, dims):
    """Tiled grids, ragged or not: the trilinear read at its edges, and an
    FP16 score map made from a tiled FP32 grid (which keeps its tiles),
    against the oracle."""
    torch, mcl = env
    origin = (-0.3, 0.25, -0.1)
    smap = dense_map(origin, dims, scenes.F32)
    m = mcl.map_from_scene(smap)
    om = oracle.Map.from_scene_map(smap)
    pos = np.concatenate([tri_positions(origin, dims), edge_positions(origin, dims)])
    parts = np.zeros((len(pos), 6), np.float32)
    parts[:, :3] = pos
    scan = np.zeros((1, 3), np.float32)
    logw = torch.empty(len(parts), device="cuda")
    mcl.mcl_sensor_update(m, torch.from_numpy(parts).cuda(), torch.from_numpy(scan).cuda(),
                          mcl.sensor_params(0.1, flags=mcl.MCL_TRILINEAR), logw)
    mcl.mcl_sync()
    Lg = logw.cpu().numpy().astype(np.float64)
    Lo = oracle.sensor_update(om, parts, scan, 0.1, trilinear=True)
    assert np.all(np.abs(Lg - Lo) <= 1e-5 * np.maximum(1.0, np.abs(Lo)))
    sm = mcl.mcl_map_create_score(m, 0.1, mcl.MCL_F16)
    mcl.mcl_sensor_update(sm, torch.from_numpy(parts).cuda(), torch.from_numpy(scan).cuda(),
                          mcl.sensor_params(0.1, mode=mcl.MCL_SUM), logw)
    mcl.mcl_sync()
    Ls = logw.cpu().numpy().astype(np.float64)
    Lo_sum = oracle.sensor_update(om, parts, scan, 0.1, oracle.SUM)
    # one point per particle: the FP16 score of its voxel against the FP64 p_hit (r16: one FP16 rounding)
    assert np.all(np.abs(np.exp(Ls) - np.exp(Lo_sum)) <= 2.0 ** -10 * np.exp(Lo_sum) + 1e-6)
    sm.close()
    m.close()


@pytest.mark.parametrize("origin", [(0.0, 0.0, 0.0), (-1.6, -0.8, -0.4)])
@pytest.mark.parametrize("layout,index", [(0, 2), (0, 1), (1, 1)])
def test_brick_index_edges(env, origin, layout, index):
    torch, mcl = env
    run_case(torch, mcl, brick_map(origin, (48, 32, 32), scenes.I16), layout, index)


def tri_positions(origin, dims, voxel=0.05):
    """Positions whose f = u - 1/2 sits at or next to the trilinear read's
    edges: corners at -1 or n on one axis, or on all three at once."""
    o = np.asarray(origin, np.float64)
    mid = o + voxel * (np.asarray(dims, np.float64) / 2 + 0.3)
    us = lambda n: (-0.5, -0.49, -0.25, 0.0, 0.25, 0.5, 0.75, 15.6, 16.4, n - 0.75, n - 0.5, n - 0.25,
                    n, n + 0.25, n + 0.49, n + 0.5, n + 0.6)
    pts = []
    for axis in range(3):
        for u in us(dims[axis]):
            p = mid.copy()
            p[axis] = o[axis] + u * voxel
            pts.append(p)
    for u in (-0.5, -0.3, 0.2, 0.5):   # all three axes at the low faces, then the high ones
        pts.append(o + u * voxel)
        pts.append(o + (np.asarray(dims, np.float64) - u) * voxel)
    return np.array(pts, np.float32)


@pytest.mark.parametrize("origin", [(0.0, 0.0, 0.0), (-1.6, -0.8, -0.4)])
@pytest.mark.parametrize("neglect", [False, True])
def test_trilinear_edges_both_indexes(env, origin, neglect):
    torch, mcl = env
    smap = brick_map(origin, (48, 32, 32), scenes.I16)
    pos = tri_positions(smap.origin, smap.dims)
    parts = np.zeros((len(pos), 6), np.float32)
    parts[:, :3] = pos
    scan = np.zeros((1, 3), np.float32)
    flags = mcl.MCL_TRILINEAR | (mcl.MCL_NEGLECT_OUTSIDE if neglect else 0)
    res = []
    for index in (2, 1):
        m = mcl.map_from_scene(smap, 0, index)
        logw = torch.empty(len(parts), device="cuda")
        mcl.mcl_sensor_update(m, torch.from_numpy(parts).cuda(), torch.from_numpy(scan).cuda(),
                              mcl.sensor_params(0.1, flags=flags), logw)
        mcl.mcl_sync()
        res.append(logw.cpu().numpy().astype(np.float64))
        m.close()
    assert np.array_equal(res[0], res[1])
    Lo = oracle.sensor_update(oracle.Map.from_scene_map(smap), parts, scan, 0.1, neglect=neglect,
                              trilinear=True)
    err = np.abs(res[0] - Lo) / np.maximum(1.0, np.abs(Lo))
    bad = np.flatnonzero(~(err <= 1e-5))
    assert len(bad) == 0, f"positions {pos[bad[:5]]}: GPU {res[0][bad[:5]]} oracle {Lo[bad[:5]]}"


@pytest.mark.parametrize("kind", ["dense", "grid", "hash"])
def test_rotated_poses_near_faces(env, kind):
    """Rotated particles placed so that one scan point lands on or within a
    few ulps of voxel faces: each particle's log-weight is the score of the
    voxel the FP32 rule gives, on the GPU as in the oracle."""
    torch, mcl = env
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(17)
    origin, dims = (-1.6, -0.8, -0.4), (48, 32, 32)
    smap = dense_map(origin, dims, scenes.F32) if kind == "dense" else brick_map(origin, dims, scenes.I16)
    m = mcl.map_from_scene(smap) if kind == "dense" else mcl.map_from_scene(smap, 0, 2 if kind == "grid" else 1)
    om = oracle.Map.from_scene_map(smap)
    P = 3000
    for z in ([0.7, -0.3, 0.4], [-0.05, 0.9, -0.6], [0.0, 0.0, 1.3]):
        z = np.asarray(z, np.float32)
        ang = rng.uniform(-math.pi, math.pi, (P, 3))
        R = Rotation.from_euler("ZYX", ang[:, ::-1].astype(np.float32).astype(np.float64)).as_matrix()
        u = rng.integers(0, dims, (P, 3)).astype(np.float64)
        u += rng.choice([0.0, 1e-7, -1e-7, 3e-7, -3e-7, 0.5], (P, 3)) * np.maximum(u, 1.0)
        x = np.asarray(origin, np.float64) + u * np.float64(np.float32(0.05))
        parts = np.concatenate([x - R @ z.astype(np.float64), ang], 1).astype(np.float32)
        logw = torch.empty(P, device="cuda")
        mcl.mcl_sensor_update(m, torch.from_numpy(parts).cuda(), torch.from_numpy(z[None]).cuda(),
                              mcl.sensor_params(0.1), logw)
        mcl.mcl_sync()
        Lg = logw.cpu().numpy().astype(np.float64)
        Lo = oracle.sensor_update(om, parts, z[None], 0.1)
        err = np.abs(Lg - Lo) / np.maximum(1.0, np.abs(Lo))
        bad = np.flatnonzero(~(err <= 1e-5))
        assert len(bad) == 0, f"z {z}: particles {bad[:5]} GPU {Lg[bad[:5]]} oracle {Lo[bad[:5]]}"
    m.close()


def test_dims_beyond_the_index_rule_are_refused(env):
    torch, mcl = env
    empty = np.zeros((0, 16, 16, 16), np.int16)
    with pytest.raises(mcl.MclError) as e:
        mcl.mcl_map_create(mcl.MCL_MAP_BRICK, mcl.MCL_I16, (0.0, 0.0, 0.0), np.float32(0.05),
                           np.float32(TAU), (2 ** 23 + 16, 16, 16), empty, np.zeros((0, 3), np.int32))
    assert e.value.status == mcl.MCL_EINVAL
    m = mcl.mcl_map_create(mcl.MCL_MAP_BRICK, mcl.MCL_I16, (0.0, 0.0, 0.0), np.float32(0.05),
                           np.float32(TAU), (2 ** 23, 16, 16), empty, np.zeros((0, 3), np.int32),
                           index=mcl.MCL_INDEX_HASH)
    m.close()
