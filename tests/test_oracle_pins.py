"""Pins of the FP64 oracle to things other than itself (CPU only).

- Philox4x32-10 against the published known-answer vectors (tests/golden).
- Pose -> [R | t] against SciPy's extrinsic x-y-z Euler rotation.
- Plane and sphere TSDFs: closed-form values at voxel centres, points placed
  on the surface at the true pose score the maximum (Eq. 3, d = 0).
- Brute force on 8 particles x 16 points against an independent NumPy /
  exact-rational restatement, FP64 quality mode and the FP32 parity mode.
- Invariants: rotating scene and poses together (analytic map), 90-degree grid
  rotation and integer-voxel translation (bit-identical), points outside the
  map (Sec. III clamping rule), log-sum-exp shift invariance.
- Systematic resampling against exact rational arithmetic and its textbook
  properties.
- Motion update: closed-form composition, noise statistics.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy import stats
from scipy.spatial.transform import Rotation

import oracle
import scenes

HERE = os.path.dirname(os.path.abspath(__file__))


# ----------------------------------------------------------------- helpers
def dense_map(values, origin, voxel, tau, dtype=scenes.F32):
    nz, ny, nx = values.shape
    return scenes.DenseMap(tuple(map(float, origin)), float(voxel), (nx, ny, nz), float(tau), dtype,
                           np.ascontiguousarray(values))


def world_from_sensor(pose, z):
    R = Rotation.from_euler("xyz", np.asarray(pose[3:], np.float64)).as_matrix()
    return np.asarray(z, np.float64) @ R.T + np.asarray(pose[:3], np.float64)


def sensor_from_world(pose, x):
    R = Rotation.from_euler("xyz", np.asarray(pose[3:], np.float64)).as_matrix()
    return ((np.asarray(x, np.float64) - np.asarray(pose[:3], np.float64)) @ R).astype(np.float32)


def f32_round(x: Fraction) -> Fraction:
    """Round an exact rational to the nearest FP32 value (ties to even)."""
    if x == 0:
        return Fraction(0)
    s = -1 if x < 0 else 1
    a = abs(x)
    e = math.floor(math.log2(a.numerator) - math.log2(a.denominator))
    while Fraction(2) ** e > a:
        e -= 1
    while Fraction(2) ** (e + 1) <= a:
        e += 1
    e = max(e, -126)
    ulp = Fraction(2) ** (e - 23)
    q = a / ulp
    n = math.floor(q)
    rem = q - n
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and n % 2 == 1):
        n += 1
    return s * n * ulp


def fmaf_exact(a, b, c) -> np.float32:
    r = f32_round(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c)))
    return np.float32(float(r))


# ----------------------------------------------------------------- Philox
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = oracle.philox4x32_10(v[0:4], v[4:6])
        assert list(out) == v[6:10]


# ----------------------------------------------------------------- pose -> matrix
def test_pose_matrix_matches_scipy(rng):
    poses = np.concatenate([rng.normal(0, 10, (500, 3)), rng.uniform(-math.pi, math.pi, (500, 3))],
                           1).astype(np.float32)
    q = oracle.pose_to_matrix(poses, parity=False)
    ref = Rotation.from_euler("xyz", poses[:, 3:].astype(np.float64)).as_matrix()
    assert np.max(np.abs(q[:, :, :3] - ref)) < 2e-15
    assert np.array_equal(q[:, :, 3], poses[:, :3].astype(np.float64))
    par = oracle.pose_to_matrix(poses, parity=True)
    assert np.array_equal(par, q.astype(np.float32).astype(np.float64))


def test_pose_matrix_special_cases():
    h = np.float32(math.pi / 2)
    R = oracle.pose_to_matrix([[0, 0, 0, 0, 0, h]], parity=False)[0, :, :3]
    assert np.allclose(R, [[0, -1, 0], [1, 0, 0], [0, 0, 1]], atol=1e-7)   # yaw
    R = oracle.pose_to_matrix([[0, 0, 0, h, 0, 0]], parity=False)[0, :, :3]
    assert np.allclose(R, [[1, 0, 0], [0, 0, -1], [0, 1, 0]], atol=1e-7)   # roll
    R = oracle.pose_to_matrix([[0, 0, 0, 0, h, 0]], parity=False)[0, :, :3]
    assert np.allclose(R, [[0, 0, 1], [0, 1, 0], [-1, 0, 0]], atol=1e-7)   # pitch


# ----------------------------------------------------------------- plane
def plane_setup(rng, n_pts=400):
    voxel, tau, z0 = 0.0625, 0.3, 1.03125  # z0 = centre height of voxel layer 16
    cz = (np.arange(32) + 0.5) * voxel
    vals = np.broadcast_to(np.clip(cz - z0, -tau, tau).astype(np.float32)[:, None, None],
                           (32, 32, 32)).copy()
    m = dense_map(vals, (0, 0, 0), voxel, tau)
    pose = np.array([1.0, 0.9, 1.6, 0.05, -0.08, 0.7], np.float32)
    xy = rng.uniform(0.3, 1.7, (n_pts, 2))
    world = np.concatenate([xy, np.full((n_pts, 1), z0)], 1)
    scan = sensor_from_world(pose, world)
    return m, pose, scan, z0, tau, voxel


def test_plane_per_point_values_closed_form(rng):
    m, pose, scan, z0, tau, voxel = plane_setup(rng)
    om = oracle.Map.from_scene_map(m)
    for s in [pose, pose + np.float32([0.1, -0.2, 0.17, 0.1, 0.05, -0.3])]:
        x, d, idx, n = oracle.eval_points(om, s, scan, parity=True)
        inside = idx[:, 0] >= 0
        cz = (idx[inside, 2] + 0.5) * voxel
        assert np.array_equal(d[inside], np.clip(cz - z0, -tau, tau).astype(np.float32))
        assert np.all(d[~inside] == np.float32(tau))
        assert n == inside.sum()


def test_plane_points_on_surface_score_maximum(rng):
    m, pose, scan, z0, tau, voxel = plane_setup(rng)
    om = oracle.Map.from_scene_map(m)
    pert = pose + rng.normal(0, [0.1, 0.1, 0.1, 0.05, 0.05, 0.05], (64, 6)).astype(np.float32)
    pert[:32, 2] = pose[2] + np.float32(voxel) * rng.choice([-1.5, 1.5], 32).astype(np.float32)
    for parity in (True, False):
        L = oracle.sensor_update(om, np.vstack([pose, pert]), scan, 0.1, parity=parity)
        assert L[0] == 0.0  # every point reads d = 0 exactly: the maximum of Eq. 3
        assert np.all(L[1:] <= 0.0)  # in-plane motions tie, none scores above
        assert np.all(L[1:33] < 0.0)  # leaving the plane by 1.5 voxels always loses
    # analytic plane n.x - d0 (no grid): d = 0 up to the FP32 scan rounding
    am = oracle.Map.analytic([[oracle.PLANE, 0, 0, 1, z0]], tau)
    L = oracle.sensor_update(am, np.vstack([pose, pert]), scan, 0.1, parity=False)
    assert L[0] > -1e-9 and np.all(L[1:] < L[0])


# ----------------------------------------------------------------- sphere
def sphere_setup(rng, n_pts=500):
    voxel, tau, R0 = 0.05, 0.3, 0.5
    c0 = np.array([0.8, 0.8, 0.8])
    cen = voxel_centres = (np.arange(32) + 0.5) * voxel
    gz, gy, gx = np.meshgrid(cen, cen, cen, indexing="ij")
    vals = np.clip(np.sqrt((gx - c0[0]) ** 2 + (gy - c0[1]) ** 2 + (gz - c0[2]) ** 2) - R0,
                   -tau, tau).astype(np.float32)
    m = dense_map(vals, (0, 0, 0), voxel, tau)
    pose = np.array([0.9, 0.75, 0.88, 0.1, -0.2, 2.0], np.float32)
    u = rng.normal(size=(n_pts, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    scan = sensor_from_world(pose, c0 + R0 * u)
    return m, pose, scan, c0, R0, tau, voxel


def test_sphere_per_point_values_closed_form(rng):
    m, pose, scan, c0, R0, tau, voxel = sphere_setup(rng)
    om = oracle.Map.from_scene_map(m)
    x, d, idx, n = oracle.eval_points(om, pose, scan, parity=False)
    # the transform: x = R z + t with SciPy's rotation
    assert np.max(np.abs(x - world_from_sensor(pose.astype(np.float64), scan))) < 1e-13
    # the containing voxel: floor((x - o) / r) per axis
    exp_idx = np.floor(x / np.float64(np.float32(voxel))).astype(np.int64)
    assert np.array_equal(idx, exp_idx)
    # the value read: clamp(|c_vox - c0| - R) at that voxel's centre
    c = (idx + 0.5) * voxel
    exp_d = np.clip(np.linalg.norm(c - c0, axis=1) - R0, -tau, tau).astype(np.float32)
    assert np.array_equal(d, exp_d.astype(np.float64))


def test_sphere_true_pose_scores_above_perturbed(rng):
    m, pose, scan, c0, R0, tau, voxel = sphere_setup(rng)
    dirs = rng.normal(size=(32, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    pert = np.repeat(pose[None], 32, 0)
    pert[:, :3] += (0.1 * dirs).astype(np.float32)  # two voxels away
    grid = oracle.Map.from_scene_map(m)
    L = oracle.sensor_update(grid, np.vstack([pose, pert]), scan, 0.1, parity=True)
    assert np.all(L[1:] < L[0])
    ana = oracle.Map.analytic([[oracle.SPHERE, *c0, R0]], tau)
    L = oracle.sensor_update(ana, np.vstack([pose, pert]), scan, 0.1, parity=False)
    assert L[0] > -1e-9 and np.all(L[1:] < L[0])


# ----------------------------------------------------------------- brute force
def brute_maps(rng, dtype):
    """A 48 x 40 x 32 dense map and the same field as 16^3 bricks (some absent)."""
    tau = 0.3
    vals64 = rng.uniform(-tau, tau, (32, 48, 48))[:, :40, :]
    vals64 = np.ascontiguousarray(vals64[:, :, :48])
    if dtype == scenes.F32:
        stored = vals64.astype(np.float32)
    elif dtype == scenes.F16:
        stored = vals64.astype(np.float16)
    else:
        stored = np.rint(vals64 / tau * 32767).astype(np.int16)
    dense = dense_map(stored, (-0.4, -0.3, -0.2), 0.05, tau, dtype)
    coords, bricks = [], []
    padded = np.zeros((32, 48, 48), stored.dtype)
    padded[:, :40, :] = stored
    for bz in range(2):
        for by in range(3):
            for bx in range(3):
                if (bx + by + bz) % 3 == 0:
                    continue  # leave some bricks unallocated
                coords.append((bx, by, bz))
                bricks.append(padded[bz * 16:(bz + 1) * 16, by * 16:(by + 1) * 16,
                                     bx * 16:(bx + 1) * 16])
    brick = scenes.BrickMap((-0.4, -0.3, -0.2), 0.05, (48, 48, 32), tau, dtype,
                            np.array(coords, np.int32), np.ascontiguousarray(np.array(bricks)))
    return dense, brick


def np_stored_value(m, ix, iy, iz):
    """None where no value is stored (outside the grid or unallocated brick)."""
    nx, ny, nz = m.dims
    if not (0 <= ix < nx and 0 <= iy < ny and 0 <= iz < nz):
        return None
    if m.kind == "dense":
        raw = m.values[iz, iy, ix]
    else:
        hit = np.where((m.coords == (ix // 16, iy // 16, iz // 16)).all(1))[0]
        if len(hit) == 0:
            return None
        raw = m.values[hit[0], iz % 16, iy % 16, ix % 16]
    if m.dtype == scenes.I16:
        return float(raw) * (float(np.float32(m.tau)) / 32767.0)
    return float(raw)


def index_frame_rows(m, M, shift=0.0):
    """FP32 rows [R' | t'] of the FP64 pose rows M in the map's index frame:
    R' = fl32(R inv), t' = fl32((t - o) inv - shift), each in FP64 first."""
    inv = np.float64(np.float32(m.inv_voxel))
    o64 = np.asarray(m.origin, np.float32).astype(np.float64)
    Rp = (np.asarray(M[:, :3], np.float64) * inv).astype(np.float32)
    tp = (((np.asarray(M[:, 3], np.float64) - o64) * inv) - np.float64(shift)).astype(np.float32)
    return Rp, tp


def np_log_weight(m, M, scan, sigma, mode, neglect, parity):
    """M: FP64 pose rows. Parity: the FP32 index rule (rows in the index
    frame, then one exactly rounded fma chain per axis)."""
    sigma = float(np.float32(sigma))
    tau = float(np.float32(m.tau))
    o32 = np.asarray(m.origin, np.float32)
    r64 = float(np.float32(m.voxel))
    Rp, tp = index_frame_rows(m, M)
    total = 0.0
    for z in scan:
        if parity:
            u = [fmaf_exact(Rp[i, 0], z[0], fmaf_exact(Rp[i, 1], z[1], fmaf_exact(Rp[i, 2], z[2], tp[i])))
                 for i in range(3)]
            ok = all(0 <= u[k] < m.dims[k] for k in range(3))
            idx = [int(math.floor(u[k])) for k in range(3)] if ok else None
        else:
            x = M[:, :3] @ z.astype(np.float64) + M[:, 3]
            u = [math.floor((x[k] - float(o32[k])) / r64) for k in range(3)]
            idx = u if all(0 <= u[k] < m.dims[k] for k in range(3)) else None
        d = np_stored_value(m, *idx) if idx is not None else None
        if d is None:
            if neglect:
                continue
            d = tau
        e = -d * d / (2 * sigma * sigma)
        total += e if mode == oracle.LOGPROD else math.exp(e) / math.sqrt(2 * math.pi * sigma * sigma)
    return total if mode == oracle.LOGPROD else (math.log(total) if total > 0 else -math.inf)


@pytest.mark.parametrize("dtype", [scenes.F32, scenes.F16, scenes.I16])
@pytest.mark.parametrize("parity", [True, False])
def test_brute_force_8_particles_16_points(rng, dtype, parity):
    dense, brick = brute_maps(rng, dtype)
    centre = np.array([0.8, 0.7, 0.6])
    poses = np.concatenate([centre + rng.normal(0, 0.3, (8, 3)),
                            rng.uniform(-math.pi, math.pi, (8, 3))], 1).astype(np.float32)
    dirs = rng.normal(size=(16, 3))
    scan = (dirs / np.linalg.norm(dirs, axis=1, keepdims=True) *
            rng.uniform(0.2, 1.2, (16, 1))).astype(np.float32)
    mats = oracle.pose_to_matrix(poses, parity=False)  # FP64 rows, pinned to SciPy above
    for m in (dense, brick):
        om = oracle.Map.from_scene_map(m)
        for mode in (oracle.LOGPROD, oracle.SUM):
            for neglect in (False, True):
                got = oracle.sensor_update(om, poses, scan, 0.1, mode, neglect, parity)
                ref = [np_log_weight(m, mats[p], scan, 0.1, mode, neglect, parity) for p in range(8)]
                np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def near_face_scan(rng, m, pose, n, shift=0.0):
    """Sensor-frame points whose map coordinates sit on or within a few ulps
    of voxel faces (shift 1/2: of voxel centres) (FP64 solve, then FP32)."""
    R = Rotation.from_euler("ZYX", pose[[5, 4, 3]].astype(np.float64)).as_matrix()
    dims = np.asarray(m.dims)
    u = rng.integers(0, dims, (n, 3)).astype(np.float64) + shift
    u += rng.choice([0.0, 1e-7, -1e-7, 3e-7, -3e-7, 0.5], (n, 3)) * np.maximum(u, 1.0)
    x = np.asarray(m.origin, np.float64) + u * np.float64(np.float32(m.voxel))
    return ((x - pose[:3].astype(np.float64)) @ R).astype(np.float32)


def np_parity_index(m, M, z, shift=0.0, round_rows_first=False):
    if round_rows_first:  # the plausible slip: rows rounded to FP32 before the frame
        M = np.asarray(M, np.float32).astype(np.float64)
    Rp, tp = index_frame_rows(m, M, shift)
    u = [fmaf_exact(Rp[i, 0], z[0], fmaf_exact(Rp[i, 1], z[1], fmaf_exact(Rp[i, 2], z[2], tp[i])))
         for i in range(3)]
    if not all(0 <= u[k] < m.dims[k] for k in range(3)):
        return [-1, -1, -1]
    return [int(math.floor(u[k])) for k in range(3)]


def test_parity_index_rule_per_point(rng):
    """The parity-mode voxel of every scan point, for rotated poses and points
    on or next to voxel faces, is the restated FP32 rule: rows in the map's
    index frame (R inv, (t - o) inv, FP64 then one FP32 rounding), one exactly
    rounded fma chain per axis, floor. Rounding the rows to FP32 before the
    frame moves some of these points to a neighbouring voxel."""
    dense, _ = brute_maps(rng, scenes.F32)
    om = oracle.Map.from_scene_map(dense)
    poses = np.concatenate([rng.uniform(0.2, 1.6, (6, 3)), rng.uniform(-math.pi, math.pi, (6, 3))],
                           1).astype(np.float32)
    mats = oracle.pose_to_matrix(poses, parity=False)
    slipped = 0
    for p in range(len(poses)):
        z = near_face_scan(rng, dense, poses[p], 400)
        _, _, idx, _ = oracle.eval_points(om, poses[p], z, parity=True)
        for j in range(len(z)):
            assert list(idx[j]) == np_parity_index(dense, mats[p], z[j]), (p, j)
            slipped += np_parity_index(dense, mats[p], z[j], round_rows_first=True) != list(idx[j])
    assert slipped > 0


def test_map_lookup_matches_brute_force(rng):
    dense, brick = brute_maps(rng, scenes.I16)
    pts = np.concatenate([rng.uniform(-0.6, 2.8, (3000, 3)),
                          # points exactly on voxel faces go to the upper voxel
                          (np.float32(-0.4) + np.float32(0.05) * rng.integers(0, 40, (200, 3)))],
                         0).astype(np.float32)
    for m in (dense, brick):
        idx, val = oracle.map_lookup(oracle.Map.from_scene_map(m), pts)
        for j in range(len(pts)):
            u = [np.float32(pts[j, k] - np.float32(m.origin[k])) * np.float32(m.inv_voxel)
                 for k in range(3)]
            inside = all(0 <= u[k] < m.dims[k] for k in range(3))
            if not inside:
                assert idx[j] == -1 and val[j] == np.float32(m.tau)
                continue
            ix, iy, iz = (int(math.floor(x)) for x in u)
            assert idx[j] == (iz * m.dims[1] + iy) * m.dims[0] + ix
            v = np_stored_value(m, ix, iy, iz)
            assert val[j] == (np.float32(m.tau) if v is None else v)


# ----------------------------------------------------------------- invariants
def test_rotating_scene_and_poses_leaves_weights_unchanged(rng):
    tau = 0.3
    planes = [[oracle.PLANE, 0, 0, 1, 0.2], [oracle.PLANE, 1, 0, 0, 3.0]]
    spheres = [[oracle.SPHERE, 1.0, 1.2, 0.9, 0.4], [oracle.SPHERE, 2.0, 0.3, 1.1, 0.6]]
    poses = np.concatenate([rng.uniform(0.5, 2.5, (40, 3)), rng.uniform(-3, 3, (40, 3))], 1)
    mats = oracle.pose_to_matrix(poses.astype(np.float32), parity=False)
    scan = rng.normal(0, 1.0, (300, 3)).astype(np.float32)
    base = oracle.Map.analytic(planes + spheres, tau)
    for mode in (oracle.LOGPROD, oracle.SUM):
        L0 = oracle.sensor_update_mat(base, mats, scan, 0.1, mode)
        for seed in range(3):
            Q = Rotation.random(random_state=seed).as_matrix()
            rp = [[oracle.PLANE, *(Q @ np.array(p[1:4])), p[4]] for p in planes]
            rs = [[oracle.SPHERE, *(Q @ np.array(s[1:4])), s[4]] for s in spheres]
            rot = oracle.Map.analytic(rp + rs, tau)
            L1 = oracle.sensor_update_mat(rot, np.einsum("ij,pjk->pik", Q, mats), scan, 0.1, mode)
            np.testing.assert_allclose(L1, L0, rtol=1e-12, atol=1e-12)


def test_grid_rotation_and_translation_bit_identical(rng):
    voxel, tau = 0.125, 0.3
    vals = rng.uniform(-tau, tau, (16, 24, 20)).astype(np.float32)   # nz, ny, nx
    nz, ny, nx = vals.shape
    o = np.array([-1.0, -1.5, -0.5])
    m0 = dense_map(vals, o, voxel, tau)
    poses = np.concatenate([o + rng.uniform(0.5, 2.0, (30, 3)), rng.uniform(-3, 3, (30, 3))], 1)
    mats = oracle.pose_to_matrix(poses.astype(np.float32), parity=False)
    scan = rng.normal(0, 0.8, (200, 3)).astype(np.float32)
    L0 = oracle.sensor_update_mat(oracle.Map.from_scene_map(m0), mats, scan, 0.1)
    # 90 degrees about z: (x, y) -> (-y, x); new grid o' = (-oy - ny r, ox), values permuted
    Q = np.array([[0.0, -1, 0], [1, 0, 0], [0, 0, 1]])
    vr = np.ascontiguousarray(np.transpose(vals[:, ::-1, :], (0, 2, 1)))
    m1 = dense_map(vr, (-o[1] - ny * voxel, o[0], o[2]), voxel, tau)
    L1 = oracle.sensor_update_mat(oracle.Map.from_scene_map(m1),
                                  np.einsum("ij,pjk->pik", Q, mats), scan, 0.1)
    assert np.array_equal(L0, L1)
    # translation by an integer number of voxels
    shift = np.array([3, -2, 5]) * voxel
    m2 = dense_map(vals, o + shift, voxel, tau)
    mats2 = mats.copy()
    mats2[:, :, 3] += shift
    L2 = oracle.sensor_update_mat(oracle.Map.from_scene_map(m2), mats2, scan, 0.1)
    assert np.array_equal(L0, L2)


def test_points_outside_the_map_read_truncation(rng):
    m, pose, scan, z0, tau, voxel = plane_setup(rng, 100)
    om = oracle.Map.from_scene_map(m)
    far = np.array([[1000, -1000, 50, 0.1, 0.2, 0.3]], np.float32)
    sig = np.float64(np.float32(0.1))
    t = np.float64(np.float32(tau))
    assert oracle.sensor_update(om, far, scan, 0.1)[0] == pytest.approx(
        -100 * t * t / (2 * sig * sig), rel=1e-14)
    s = oracle.sensor_update(om, far, scan, 0.1, oracle.SUM)[0]
    assert s == pytest.approx(math.log(100 * math.exp(-t * t / (2 * sig * sig)) /
                                       math.sqrt(2 * math.pi * sig * sig)), rel=1e-14)
    assert oracle.sensor_update(om, far, scan, 0.1, neglect=True)[0] == 0.0
    assert oracle.sensor_update(om, far, scan, 0.1, oracle.SUM, neglect=True)[0] == -math.inf
    # brick maps: an unallocated brick reads +tau exactly like the outside
    br = scenes.voxelize_bricks(scenes.room(1), (0, 0, 0), 0.05, (128, 128, 64), 0.3)
    have = {tuple(c) for c in br.coords.tolist()}
    free = [(x, y, z) for z in range(4) for y in range(8) for x in range(8) if (x, y, z) not in have]
    assert free
    centres = (np.array(free, np.float64) * 16 + 8) * 0.05
    idx, val = oracle.map_lookup(oracle.Map.from_scene_map(br), centres.astype(np.float32))
    assert np.all(idx >= 0) and np.all(val == np.float32(0.3))


def test_normalisation_invariants(rng):
    L = rng.normal(-5000, 20, 1000)
    w, M, S, deg = oracle.normalise(L)
    assert not deg and M == L.max()
    assert abs(w.sum() - 1) < 1e-13
    i, j = rng.integers(0, 1000, (2, 200))
    np.testing.assert_allclose(w[i] / w[j], np.exp(L[i] - L[j]), rtol=1e-10)
    w2, *_ = oracle.normalise(L + 12345.678)
    np.testing.assert_allclose(w2, w, rtol=1e-9, atol=1e-300)
    # a wide spread: far-off particles underflow to 0, the sum stays 1
    Lw = rng.normal(-5000, 3000, 1000)
    ww, *_ = oracle.normalise(Lw)
    assert abs(ww.sum() - 1) < 1e-13 and ww[np.argmax(Lw)] == ww.max()
    wu, _, _, deg = oracle.normalise(np.full(7, -np.inf))
    assert deg and np.allclose(wu, 1 / 7)


# ----------------------------------------------------------------- resampling
def exact_resample(w32, r):
    """min{p : C_p > t_j} with exact rationals for C; t_j from the IEEE FP64 ops."""
    q = [Fraction(int(np.rint(np.float64(x) * 2.0 ** 52))) / 2 ** 52 for x in w32]
    C, acc = [], Fraction(0)
    for v in q:
        acc += v
        C.append(acc)
    S = float(acc)
    assert Fraction(S) == acc  # the FP64 total is exact
    last = max(i for i, v in enumerate(q) if v > 0)
    out = []
    P = len(w32)
    for j in range(P):
        t = Fraction(((float(j) + r) / float(P)) * S)
        out.append(next((p for p, c in enumerate(C) if c > t), last))
    return np.array(out, np.int32), q, acc


def test_resample_exact_rational(rng):
    for P, r in [(1000, 0.37), (777, 0.0), (64, 0.999999)]:
        w = rng.exponential(1.0, P) ** 3
        w[rng.integers(0, P, P // 10)] = 0.0
        w32 = (w / w.sum()).astype(np.float32)
        got, deg = oracle.resample(w32, r)
        exp, q, S = exact_resample(w32, r)
        assert not deg and np.array_equal(got, exp)
        assert np.all(np.diff(got) >= 0)
        assert np.all(np.asarray(q)[got] > 0)  # zero weights are never drawn
        counts = np.bincount(got, minlength=P)
        share = np.array([float(v / S) for v in q]) * P
        assert np.all(counts >= np.floor(share) - 1e-9) and np.all(counts <= np.ceil(share) + 1e-9)


def test_resample_special_cases():
    for P in (8, 1000, 4096):
        for r in (0.0, 0.5, 0.9):
            idx, _ = oracle.resample(np.full(P, 1.0 / P, np.float32), r)
            assert np.array_equal(idx, np.arange(P))
    w = np.zeros(100, np.float32)
    w[42] = 1.0
    assert np.all(oracle.resample(w, 0.3)[0] == 42)
    # dyadic weights with r = 0: counts are exactly P * w
    w = np.array([0.5, 0.25, 0.125, 0.125] + [0.0] * 4, np.float32)
    idx, _ = oracle.resample(w, 0.0)
    assert list(np.bincount(idx, minlength=8)) == [4, 2, 1, 1, 0, 0, 0, 0]
    idx, deg = oracle.resample(np.zeros(5, np.float32), 0.5)
    assert deg and list(idx) == [0, 1, 2, 3, 4]


# ----------------------------------------------------------------- motion
def test_motion_closed_form():
    h = math.pi / 2
    poses = np.array([[1, 2, 3, 0, 0, h]], np.float32)
    out = oracle.motion_update(poses, [1, 0, 0, 0, 0, 0], [0] * 6, 1, 0)
    np.testing.assert_allclose(out[0, :3], [1, 3, 3], atol=1e-6)   # forward is +y at yaw 90
    rng = np.random.default_rng(3)
    for _ in range(20):
        s = np.concatenate([rng.normal(0, 5, 3), rng.uniform(-1.2, 1.2, 3)]).astype(np.float32)
        d = np.concatenate([rng.normal(0, 0.3, 3), rng.uniform(-0.3, 0.3, 3)]).astype(np.float32)
        out = oracle.motion_update(s[None], d, [0] * 6, 1, 0)[0]
        Rs = Rotation.from_euler("xyz", s[3:].astype(np.float64))
        Rd = Rotation.from_euler("xyz", d[3:].astype(np.float64))
        exp_t = s[:3] + Rs.as_matrix() @ d[:3].astype(np.float64)
        np.testing.assert_allclose(out[:3], exp_t, atol=2e-6)
        got = Rotation.from_euler("xyz", out[3:].astype(np.float64)).as_matrix()
        np.testing.assert_allclose(got, (Rs * Rd).as_matrix(), atol=2e-6)


def test_motion_noise_statistics():
    P = 100_000
    sig = np.array([0.1, 0.2, 0.3, 0.01, 0.02, 0.03], np.float32)
    out = oracle.motion_update(np.zeros((P, 6), np.float32), [0] * 6, sig, 77, 5)
    for k in range(3):
        x = out[:, k] / sig[k]
        assert abs(x.mean()) < 4 / math.sqrt(P) and abs(x.std() - 1) < 0.01
        assert stats.kstest(x, "norm").pvalue > 1e-4
    n = np.array([oracle.motion_noise(77, 5, i) for i in range(20000)])
    for k in range(6):
        assert stats.kstest(n[:, k], "norm").pvalue > 1e-4
    assert abs(np.corrcoef(n[:, 0], n[:, 1])[0, 1]) < 0.03
    # counter-based: same (seed, step, i) gives the same draw, another step another
    assert np.array_equal(oracle.motion_noise(77, 5, 3), n[3])
    assert not np.array_equal(oracle.motion_noise(77, 6, 3), n[3])


def test_systematic_properties_hold_for_the_oracle_and_catch_a_planted_error(rng):
    """The property check used on GPU-drawn indices accepts every oracle draw
    and rejects a draw with one index moved."""
    from resample_props import check_systematic
    for P in (1, 7, 1000, 4097):
        w = (rng.exponential(1.0, P) ** 3).astype(np.float32)
        w[rng.random(P) < 0.3] = 0
        for r in (0.0, 0.37, 1 - 2.0 ** -53):
            idx, _ = oracle.resample(w, r)
            check_systematic(idx, w, r)
    # 10 particles: weight 0.25 (2.5 expected draws) at index 3, zero at 5
    w = np.array([0.1, 0.05, 0.1, 0.25, 0.1, 0.0, 0.1, 0.1, 0.1, 0.1], np.float32)
    idx, _ = oracle.resample(w, 0.5)
    check_systematic(idx, w, 0.5)
    planted = []
    bad = idx.copy()
    bad[bad == 4] = 5                      # draws of a zero-weight particle
    planted.append(np.sort(bad))
    bad = idx.copy()
    bad[[0, -1]] = bad[[-1, 0]]            # out of order
    planted.append(bad)
    bad = np.sort(np.concatenate([idx[idx != 7], [3] * int((idx == 7).sum())]))
    planted.append(bad)                    # particle 3 drawn 3 + 1 times
    for b in planted:
        with pytest.raises(AssertionError):
            check_systematic(b, w, 0.5)
    check_systematic(np.arange(5), np.zeros(5, np.float32), 0.2)
