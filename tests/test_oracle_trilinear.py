"""Pins of the oracle's trilinear read (Sec. III: "a pseudo-continuous value
via interpolation") against closed forms and a NumPy restatement:
- a linear field (a tilted plane inside the truncation band) is reproduced
  exactly by trilinear interpolation of its samples at the voxel centres;
- at voxel centres the read equals the stored value (weights 1, 0, ...);
- brute force over random dense and brick maps with unallocated bricks,
  points inside, on the edges and outside, in both index modes;
- continuity across voxel faces; the neglect rule (no stored corner)."""
import math

import numpy as np
import pytest

import oracle
import scenes
from test_oracle_pins import (brute_maps, dense_map, fmaf_exact, index_frame_rows, near_face_scan,
                              np_stored_value)


@pytest.fixture
def rng():
    return np.random.default_rng(31)


IDENTITY = np.zeros(6, np.float32)


def tri_points(om, pts, parity):
    x, d, idx, n = oracle.eval_points(om, IDENTITY, np.asarray(pts, np.float32), parity=parity,
                                      trilinear=True)
    return d, idx, n


def tilted_plane(voxel=0.05, tau=0.3, n=24):
    nv = np.array([0.3, -0.5, 0.81])
    nv /= np.linalg.norm(nv)
    c = (np.arange(n) + 0.5) * voxel
    cz, cy, cx = np.meshgrid(c, c, c, indexing="ij")
    d0 = float(nv @ np.full(3, n * voxel / 2))
    field = nv[0] * cx + nv[1] * cy + nv[2] * cz - d0
    vals = np.clip(field, -tau, tau).astype(np.float32)
    return dense_map(vals, (0, 0, 0), voxel, tau), nv, d0


@pytest.mark.parametrize("parity,atol", [(False, 5e-8), (True, 1e-6)])
def test_linear_field_is_reproduced(rng, parity, atol):
    """Inside the band the samples are those of the linear function n.x - d0,
    which trilinear interpolation reproduces; the only errors are the FP32
    storage of the samples (and in parity mode the FP32 index coordinate)."""
    m, nv, d0 = tilted_plane()
    om = oracle.Map.from_scene_map(m)
    pts = rng.uniform(2 * 0.05, 22 * 0.05, (20000, 3)).astype(np.float32)
    x = pts.astype(np.float64)
    # keep points whose eight surrounding centres are all unclamped
    f = x / 0.05 - 0.5
    i0 = np.floor(f)
    ok = np.ones(len(x), bool)
    for c in range(8):
        off = np.array([c & 1, (c >> 1) & 1, c >> 2])
        centre = (i0 + off + 0.5) * 0.05
        ok &= np.abs(centre @ nv - d0) < 0.3 - 1e-6
    assert ok.sum() > 2000
    d, _, n = tri_points(om, pts[ok], parity)
    np.testing.assert_allclose(d, x[ok] @ nv - d0, rtol=0, atol=atol)
    assert n == ok.sum()


def test_centres_read_the_stored_value(rng):
    vals = rng.uniform(-0.3, 0.3, (8, 9, 10)).astype(np.float32)
    m = dense_map(vals, (0, 0, 0), 0.0625, 0.3)        # centres exactly representable
    om = oracle.Map.from_scene_map(m)
    iz, iy, ix = np.meshgrid(np.arange(8), np.arange(9), np.arange(10), indexing="ij")
    pts = (np.stack([ix, iy, iz], -1).reshape(-1, 3) + 0.5) * 0.0625
    for parity in (True, False):
        d, idx, _ = tri_points(om, pts, parity)
        np.testing.assert_array_equal(d, vals.reshape(-1).astype(np.float64))
        np.testing.assert_array_equal(idx, np.stack([ix, iy, iz], -1).reshape(-1, 3))


IDENTITY_ROWS = np.array([[1.0, 0, 0, 0], [0, 1.0, 0, 0], [0, 0, 1.0, 0]])


def np_trilinear(m, x, parity):
    """Plain restatement at scan point x seen from the identity pose: FP64
    (or the FP32 index rule: rows in the index frame with shift 1/2, one
    exactly rounded fma chain per axis), 8 corners with +tau for corners
    without a stored value."""
    tau = float(np.float32(m.tau))
    o32 = np.asarray(m.origin, np.float32)
    if parity:
        Rp, tp = index_frame_rows(m, IDENTITY_ROWS, 0.5)
        z = np.asarray(x, np.float32)
        f = [fmaf_exact(Rp[i, 0], z[0], fmaf_exact(Rp[i, 1], z[1], fmaf_exact(Rp[i, 2], z[2], tp[i])))
             for i in range(3)]
        if not all(-1.0 <= f[k] < m.dims[k] for k in range(3)):
            return tau, False
        i0 = [int(math.floor(f[k])) for k in range(3)]
        a = [float(np.float32(f[k] - np.float32(i0[k]))) for k in range(3)]
    else:
        f = [(float(x[k]) - float(o32[k])) / float(np.float32(m.voxel)) - 0.5 for k in range(3)]
        if not all(-1.0 <= f[k] < m.dims[k] for k in range(3)):
            return tau, False
        i0 = [math.floor(f[k]) for k in range(3)]
        a = [f[k] - i0[k] for k in range(3)]
    acc, any_st = 0.0, False
    for c in range(8):
        cx, cy, cz = c & 1, (c >> 1) & 1, c >> 2
        v = np_stored_value(m, i0[0] + cx, i0[1] + cy, i0[2] + cz)
        any_st |= v is not None
        wgt = (a[0] if cx else 1 - a[0]) * (a[1] if cy else 1 - a[1]) * (a[2] if cz else 1 - a[2])
        acc += wgt * (tau if v is None else v)
    return acc, any_st


@pytest.mark.parametrize("dtype", [scenes.F32, scenes.F16, scenes.I16])
@pytest.mark.parametrize("parity", [True, False])
def test_brute_force_random_maps(rng, dtype, parity):
    dense, brick = brute_maps(rng, dtype)
    lo, hi = np.array([-0.4, -0.3, -0.2]), np.array([-0.4 + 2.4, -0.3 + 2.4, -0.2 + 1.6])
    pts = np.concatenate([rng.uniform(lo - 0.1, hi + 0.1, (1500, 3)),
                          rng.uniform(lo - 0.03, lo + 0.03, (200, 3)),      # lower edges
                          rng.uniform(hi - 0.03, hi + 0.03, (200, 3))]).astype(np.float32)
    for m in (dense, brick):
        om = oracle.Map.from_scene_map(m)
        d, _, n = tri_points(om, pts, parity)
        ref = [np_trilinear(m, p, parity) for p in pts]
        np.testing.assert_allclose(d, [r[0] for r in ref], rtol=0, atol=1e-12)
        assert n == sum(r[1] for r in ref)


def test_parity_corner_rule_per_point(rng):
    """The parity-mode lower corner of every scan point, for rotated poses
    and points on or next to voxel centres (where floor(f) changes):
    floor(f) with f from the rows in the index frame with shift 1/2 and one
    exactly rounded fma chain per axis, or -1s where no corner is inside."""
    dense, _ = brute_maps(rng, scenes.F32)
    om = oracle.Map.from_scene_map(dense)
    poses = np.concatenate([rng.uniform(0.2, 1.6, (6, 3)), rng.uniform(-math.pi, math.pi, (6, 3))],
                           1).astype(np.float32)
    mats = oracle.pose_to_matrix(poses, parity=False)
    for p in range(len(poses)):
        z = near_face_scan(rng, dense, poses[p], 300, shift=0.5)
        _, _, idx, _ = oracle.eval_points(om, poses[p], z, parity=True, trilinear=True)
        Rp, tp = index_frame_rows(dense, mats[p], 0.5)
        for j in range(len(z)):
            f = [fmaf_exact(Rp[i, 0], z[j, 0], fmaf_exact(Rp[i, 1], z[j, 1], fmaf_exact(Rp[i, 2], z[j, 2], tp[i])))
                 for i in range(3)]
            ok = all(-1.0 <= f[k] < dense.dims[k] for k in range(3))
            exp = [int(math.floor(f[k])) for k in range(3)] if ok else [-1, -1, -1]
            assert list(idx[j]) == exp, (p, j)


def test_continuous_across_faces(rng):
    vals = rng.uniform(-0.3, 0.3, (24, 24, 24)).astype(np.float32)
    m = dense_map(vals, (0, 0, 0), 0.05, 0.3)
    om = oracle.Map.from_scene_map(m)
    # points on centre planes (f integer) along x, approached from both sides
    k = rng.integers(2, 20, (300, 3))
    p = (k + 0.5) * 0.05 + rng.uniform(0, 0.05, (300, 3)) * np.array([0, 1, 1])
    eps = 1e-9
    lo = p - np.array([eps, 0, 0])
    hi = p + np.array([eps, 0, 0])
    xo, dlo, *_ = oracle.eval_points(om, IDENTITY, lo, parity=False, trilinear=True)
    xo, dhi, *_ = oracle.eval_points(om, IDENTITY, hi, parity=False, trilinear=True)
    # the FP32 points differ by a few ulps; the slope is at most 2 tau / voxel per axis
    step = np.abs(hi.astype(np.float32).astype(np.float64) - lo.astype(np.float32).astype(np.float64)).max()
    assert np.abs(dhi - dlo).max() <= 3 * (2 * 0.3 / 0.05) * step + 1e-12


def test_neglect_needs_no_stored_corner():
    """One allocated brick: a point half a voxel outside it still has stored
    corners (counted, with +tau at the others); a point a voxel further has
    none (left out with the neglect flag)."""
    tau = 0.3
    vals = np.full((1, 16, 16, 16), 0.1, np.float32)
    m = scenes.BrickMap((0, 0, 0), 0.05, (48, 48, 48), tau, scenes.F32,
                        np.array([[1, 1, 1]], np.int32), vals)
    om = oracle.Map.from_scene_map(m)
    inside = np.array([[1.2, 1.2, 1.2]], np.float32)           # centre of the brick
    edge = np.array([[0.8 - 0.01, 1.2, 1.2]], np.float32)      # 0.2 voxel outside the brick
    far = np.array([[0.8 - 0.1, 1.2, 1.2]], np.float32)        # two voxels outside
    d_in, *_ = tri_points(om, inside, False)
    d_edge, _, n_edge = tri_points(om, edge, False)
    d_far, _, n_far = tri_points(om, far, False)
    assert d_in[0] == pytest.approx(0.1, abs=1e-7)
    f = float(np.float32(0.79)) / 0.05 - 0.5                    # x coordinate in centre units
    a = f - math.floor(f)                                      # weight of the stored corner
    assert d_edge[0] == pytest.approx((1 - a) * tau + a * 0.1, abs=1e-7) and n_edge == 1
    assert d_far[0] == pytest.approx(tau) and n_far == 0
    pose = np.zeros((1, 6), np.float32)
    for mode in (oracle.LOGPROD, oracle.SUM):
        scan = np.concatenate([inside, edge, far])
        L_all = oracle.sensor_update(om, pose, scan, 0.1, mode, parity=False, trilinear=True)
        L_neg = oracle.sensor_update(om, pose, scan, 0.1, mode, neglect=True, parity=False,
                                     trilinear=True)
        sig = float(np.float32(0.1))                            # the oracle reads sigma as FP32
        s = [-(d * d) / (2 * sig ** 2) for d in (d_in[0], d_edge[0], d_far[0])]
        if mode == oracle.LOGPROD:
            assert L_all[0] == pytest.approx(sum(s), rel=1e-12)
            assert L_neg[0] == pytest.approx(s[0] + s[1], rel=1e-12)
        else:
            k = 1 / math.sqrt(2 * math.pi * sig ** 2)
            assert L_neg[0] == pytest.approx(math.log(k * (math.exp(s[0]) + math.exp(s[1]))), rel=1e-12)
