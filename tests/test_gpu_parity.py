"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (float path against FP64):
- voxel indices and resampled indices: bit-exact;
- pose matrices: bit-exact (both sides round the same FP64 expressions);
- log-weights: |L_gpu - L_ora| <= 1e-5 * max(1, |L_ora|);
- normalised weights, LOGPROD: |log w_gpu - log w_ora| <= 1e-5 (max(1, |L_p|) +
  max(1, |M|)) wherever w_ora >= 1e-30, and |sum w - 1| <= 1e-5;
- normalised weights, SUM: |w_gpu - w_ora| <= 1e-5 w_ora (+1e-30);
- motion update: 2e-6 relative on positions, 2e-6 rad on angles (libm ulps).
"""
import ctypes
import math

import numpy as np
import pytest

import oracle
import scenes
from resample_props import check_systematic

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2310_04172_gb300 import _build, mcl
    _build.build()
    mcl.lib()
    torch.cuda.set_device(0)
    return torch


@pytest.fixture(scope="module")
def mcl():
    from paper_2310_04172_gb300 import mcl as m
    return m


@pytest.fixture(scope="module")
def room():
    return scenes.room_plain(P=1000)


def dev(torch, a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def check_logw(Lg, Lo, tol=TOL):
    Lg = np.asarray(Lg, np.float64)
    Lo = np.asarray(Lo, np.float64)
    assert np.all(np.isfinite(Lg) == np.isfinite(Lo))
    fin = np.isfinite(Lo)
    assert np.array_equal(Lg[~fin], Lo[~fin], equal_nan=True)  # the same infinities (SUM, nothing stored: -inf)
    err = np.abs(Lg[fin] - Lo[fin]) / np.maximum(1.0, np.abs(Lo[fin]))
    assert err.max(initial=0) <= tol, f"max rel log-weight error {err.max(initial=0):.3g}"
    return err.max(initial=0)


def check_w(wg, Lo, mode, tol=TOL):
    wo, M, S, deg = oracle.normalise(Lo)
    wg = np.asarray(wg, np.float64)
    assert abs(wg.sum() - 1.0) <= tol
    sel = wo >= 1e-30
    if mode == oracle.LOGPROD:
        bound = tol * (np.maximum(1.0, np.abs(Lo[sel])) + max(1.0, abs(M)))
        assert np.all(np.abs(np.log(wg[sel]) - np.log(wo[sel])) <= bound)
    else:
        assert np.all(np.abs(wg[sel] - wo[sel]) <= tol * wo[sel] + 1e-30)


def run_sensor(torch, mcl, m, parts, scan, sigma, mode=0, flags=0, **shape):
    P = parts.shape[0]
    logw = torch.empty(P, device="cuda")
    w = torch.empty(P, device="cuda")
    prm = mcl.sensor_params(sigma_hit=sigma, mode=mode, flags=flags, **shape)
    mcl.mcl_sensor_update(m, dev(torch, parts), dev(torch, scan), prm, logw, w)
    mcl.mcl_sync()
    return logw.cpu().numpy(), w.cpu().numpy()


# ----------------------------------------------------------------- a2: pose -> [R | t]
def test_pose_matrix_bit_exact(torch_cuda, mcl):
    torch = torch_cuda
    rng = np.random.default_rng(1)
    P = 200_000
    poses = np.concatenate([rng.normal(0, 50, (P, 3)), rng.uniform(-4, 4, (P, 3))], 1).astype(np.float32)
    poses[:8, 3:] = np.float32([[0, 0, 0], [math.pi, -math.pi, math.pi / 2], [-0.0, 0.0, -math.pi / 2],
                                [1e-30, -1e-30, 3e-8], [100, -200, 1e4], [6.2831855, -6.2831855, 3.1415927],
                                [0.5, 0.5, 0.5], [-1.5707964, 1.5707964, 0.0]])
    out = torch.empty((P, 12), device="cuda")
    mcl.mcl_pose_to_matrix(dev(torch, poses), out)
    mcl.mcl_sync()
    got = out.cpu().numpy().reshape(P, 3, 4)
    ref = oracle.pose_to_matrix(poses, parity=True).astype(np.float32)
    bad = np.argwhere(got != ref)
    assert len(bad) == 0, f"{len(bad)} entries differ, first {bad[:3].tolist()}"


# ----------------------------------------------------------------- a4/a5: index and look-up
def lookup_points(rng, m, n=200_000):
    lo = np.asarray(m.origin) - 0.6
    hi = np.asarray(m.origin) + np.asarray(m.dims) * m.voxel + 0.6
    pts = rng.uniform(lo, hi, (n, 3)).astype(np.float32)
    # exactly on voxel faces (FP32 multiples of the voxel): belong to the upper voxel
    k = rng.integers(0, np.asarray(m.dims), (5000, 3))
    pts[:5000] = (np.float32(m.origin) + np.float32(m.voxel) * k.astype(np.float32)).astype(np.float32)
    special = np.float32([np.nan, np.inf, -np.inf, 0.0, -0.0, 1e30, -1e30, 1e-40])
    pts[5000:5000 + 512] = rng.choice(special, (512, 3))
    return pts


# brick: automatic index (the cell grid for these maps); brick_hash: the hash
# index; brick_block4: 4x4x4-block bricks (hash index)
KINDS = ["dense", "brick", "brick_hash", "brick_block4"]


def upload(mcl, sm, kind):
    return mcl.map_from_scene(sm, mcl.MCL_LAYOUT_BLOCK4 if kind == "brick_block4" else 0,
                              mcl.MCL_INDEX_HASH if kind == "brick_hash" else mcl.MCL_INDEX_AUTO)


def room_map(sc, kind, dtype):
    if kind == "dense":
        return scenes.voxelize_dense(sc, (0.0, 0.0, 0.0), 0.05, (128, 128, 64), 0.3, dtype)
    return scenes.voxelize_bricks(sc, (0.0, 0.0, 0.0), 0.05, (128, 128, 64), 0.3, dtype)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("dtype", [scenes.F32, scenes.F16, scenes.I16])
def test_map_lookup_bit_exact(torch_cuda, mcl, kind, dtype):
    torch = torch_cuda
    sm = room_map(scenes.room(1), kind, dtype)
    m = upload(mcl, sm, kind)
    pts = lookup_points(np.random.default_rng(2), sm)
    idx, val = mcl.mcl_map_lookup(m, dev(torch, pts))
    mcl.mcl_sync()
    oi, ov = oracle.map_lookup(oracle.Map.from_scene_map(sm), pts)
    assert np.array_equal(idx.cpu().numpy(), oi)
    v = val.cpu().numpy().astype(np.float64)
    if dtype == scenes.I16:
        assert np.max(np.abs(v - ov)) <= 2 * 0.3 * 2.0 ** -24
    else:
        assert np.array_equal(v, ov)
    m.close()


# ----------------------------------------------------------------- a1-a8: sensor update + normalise
@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("dtype", [scenes.F32, scenes.F16, scenes.I16])
@pytest.mark.parametrize("mode", [oracle.LOGPROD, oracle.SUM])
@pytest.mark.parametrize("neglect", [False, True])
def test_sensor_update_room(torch_cuda, mcl, room, kind, dtype, mode, neglect):
    torch = torch_cuda
    sm = room_map(room.scene, kind, dtype)
    m = upload(mcl, sm, kind)
    parts = room.particles.copy()
    parts[:50, :3] += np.float32(4.0)  # some particles see much of the scan outside the map
    Lg, wg = run_sensor(torch, mcl, m, parts, room.scan, room.sigma_hit, mode,
                        mcl.MCL_NEGLECT_OUTSIDE if neglect else 0)
    Lo = oracle.sensor_update(oracle.Map.from_scene_map(sm), parts, room.scan, room.sigma_hit,
                              mode, neglect, parity=True)
    check_logw(Lg, Lo)
    check_w(wg, Lo, mode)
    m.close()


@pytest.mark.parametrize("chunk,lanes,unroll,ppi", [
    (32, 32, 2, 1), (64, 8, 4, 7), (256, 16, 2, 64), (1024, 32, 4, 500), (2048, 8, 2, 33),
    (8192, 32, 4, 64), (4096, 16, 4, 128), (2048, 32, 8, 64), (512, 16, 8, 9)])
def test_sensor_update_launch_shapes_and_ragged_tails(torch_cuda, mcl, room, chunk, lanes, unroll, ppi):
    torch = torch_cuda
    m = mcl.map_from_scene(room.map)
    parts = np.concatenate([room.particles, room.particles[:1]])  # P = 1001
    scan = room.scan[:1000]  # N = 1000: ragged against every chunk size
    Lg, wg = run_sensor(torch, mcl, m, parts, scan, room.sigma_hit, points_per_chunk=chunk,
                        lanes_per_particle=lanes, unroll=unroll, particles_per_item=ppi)
    Lo = oracle.sensor_update(oracle.Map.from_scene_map(room.map), parts, scan, room.sigma_hit)
    check_logw(Lg, Lo)
    check_w(wg, Lo, oracle.LOGPROD)
    # the launch hints (particles per item, unroll) never change the summation order
    other = dict(points_per_chunk=chunk, lanes_per_particle=lanes,
                 unroll={2: 4, 4: 8, 8: 2}[unroll], particles_per_item=max(1, ppi // 3))
    Lg2, wg2 = run_sensor(torch, mcl, m, parts, scan, room.sigma_hit, **other)
    assert np.array_equal(Lg, Lg2) and np.array_equal(wg, wg2)
    m.close()


def test_sensor_update_edge_cases(torch_cuda, mcl, room):
    torch = torch_cuda
    m = mcl.map_from_scene(room.map)
    om = oracle.Map.from_scene_map(room.map)
    # P = 1, N = 1
    Lg, wg = run_sensor(torch, mcl, m, room.particles[:1], room.scan[:1], 0.1)
    check_logw(Lg, oracle.sensor_update(om, room.particles[:1], room.scan[:1], 0.1))
    assert wg[0] == 1.0
    # every point outside the map, and NaN poses (their points fall outside)
    far = np.tile(np.float32([[500, 500, 500, 0, 0, 0]]), (5, 1))
    far[3, 0] = np.nan
    far[4, 5] = np.inf
    Lg, wg = run_sensor(torch, mcl, m, far, room.scan, 0.1)
    Lo = oracle.sensor_update(om, far, room.scan, 0.1)
    check_logw(Lg, Lo)
    assert np.allclose(wg, 0.2, rtol=1e-6)
    # SUM with neglect and nothing stored: degenerate, uniform weights, S = 0
    Lg, wg = run_sensor(torch, mcl, m, far, room.scan, 0.1, mcl.MCL_SUM, mcl.MCL_NEGLECT_OUTSIDE)
    assert np.all(np.isneginf(Lg)) and np.allclose(wg, 0.2)
    stats = torch.empty(2, device="cuda")
    w = torch.empty(5, device="cuda")
    mcl.mcl_normalise(dev(torch, Lg), w, stats)
    mcl.mcl_sync()
    assert stats[1].item() == 0.0 and np.allclose(w.cpu().numpy(), 0.2)
    m.close()


def test_multiroom_vlp16_parity(torch_cuda, mcl):
    torch = torch_cuda
    for dtype in (scenes.F32, scenes.F16):
        wl = scenes.vlp16_multiroom(P=2000, dtype=dtype)
        m = mcl.map_from_scene(wl.map)
        Lg, wg = run_sensor(torch, mcl, m, wl.particles, wl.scan, wl.sigma_hit)
        Lo = oracle.sensor_update(oracle.Map.from_scene_map(wl.map), wl.particles, wl.scan,
                                  wl.sigma_hit)
        check_logw(Lg, Lo)
        check_w(wg, Lo, oracle.LOGPROD)
        m.close()


@pytest.fixture(scope="module")
def building_i16():
    return scenes.os064_building(P=1_000_000, dtype=scenes.I16)


@pytest.mark.parametrize("layout,index", [(0, 0), (0, 1), (1, 0)])
def test_building_os064_parity_subset(torch_cuda, mcl, building_i16, layout, index):
    torch = torch_cuda
    wl = building_i16
    m = mcl.map_from_scene(wl.map, layout, index)
    assert m.info()["index"] == (2 if (layout, index) == (0, 0) else 1)
    parts = wl.particles[:3000]
    Lg, wg = run_sensor(torch, mcl, m, parts, wl.scan, wl.sigma_hit)
    Lo = oracle.sensor_update(oracle.Map.from_scene_map(wl.map), parts, wl.scan, wl.sigma_hit)
    check_logw(Lg, Lo)
    check_w(wg, Lo, oracle.LOGPROD)
    m.close()


def patch_order(N, R):
    """Points of an R-ring, ring-major scan in 4-ring x 8-point patches: band
    of 4 rings after band, patch after patch along the rings."""
    A = N // R
    return np.arange(N).reshape(R // 4, 4, A // 8, 8).transpose(0, 2, 1, 3).reshape(-1)


def test_scan_rings_staging(torch_cuda, mcl, room, building_i16):
    """scan_rings = R stages the scan in 4 x 8 patches: the same bits as the
    scan permuted that way on the host and staged as given (room: 16 rings of
    64 points in several chunks and lane widths; building: 64 rings of 1,024),
    within the tolerance of the oracle; a ring count that does not fit leaves
    the order as given; a negative one is EINVAL."""
    torch = torch_cuda
    cases = ((room.map, room.particles, room.scan, 16, [dict(points_per_chunk=256), dict(lanes_per_particle=8),
                                                        dict(), dict(flags=mcl.MCL_TRILINEAR)]),
             (building_i16.map, building_i16.particles[:2000], building_i16.scan, 64, [dict()]))
    for sm, parts, scan, R, shapes in cases:
        m = mcl.map_from_scene(sm)
        perm = patch_order(len(scan), R)
        assert np.array_equal(np.sort(perm), np.arange(len(scan)))
        for shape in shapes:
            a = run_sensor(torch, mcl, m, parts, scan, 0.1, scan_rings=R, **shape)
            b = run_sensor(torch, mcl, m, parts, np.ascontiguousarray(scan[perm]), 0.1, **shape)
            assert all(np.array_equal(x, y) for x, y in zip(a, b)), shape
            Lo = oracle.sensor_update(oracle.Map.from_scene_map(sm), parts, scan, 0.1,
                                      trilinear=bool(shape.get("flags", 0)))
            check_logw(a[0], Lo)
        plain = run_sensor(torch, mcl, m, parts, scan, 0.1)
        for bad_r in (3, 12, len(scan) + 4):   # not dividing N, or N / R not a multiple of 8
            if len(scan) % bad_r == 0 and bad_r % 4 == 0 and (len(scan) // bad_r) % 8 == 0:
                continue
            c = run_sensor(torch, mcl, m, parts, scan, 0.1, scan_rings=bad_r)
            assert all(np.array_equal(x, y) for x, y in zip(plain, c))
        with pytest.raises(mcl.MclError):
            run_sensor(torch, mcl, m, parts, scan, 0.1, scan_rings=-4)
        m.close()


def test_particle_order_gives_identical_bits(torch_cuda, mcl, room, building_i16):
    """Spatial processing order moves particles between slots, never changes a result."""
    torch = torch_cuda
    for sm, parts, scan in ((room.map, room.particles, room.scan),
                            (building_i16.map, building_i16.particles[:20000], building_i16.scan)):
        m = mcl.map_from_scene(sm)
        a = run_sensor(torch, mcl, m, parts, scan, 0.1, particle_order=1)
        b = run_sensor(torch, mcl, m, parts, scan, 0.1, particle_order=2)
        c = run_sensor(torch, mcl, m, parts, scan, 0.1, particle_order=2, pipeline=2)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
        assert np.array_equal(a[0], c[0]) and np.array_equal(a[1], c[1])
        m.close()


def test_item_order_gives_identical_bits(torch_cuda, mcl, building_i16):
    """Chunk-major items, static sweeps (each CTA keeping one chunk) and
    dynamic sweeps (items handed out by a device counter) write the same
    partial sums: same bits, with ragged chunk and particle tails. Each run
    follows a run on other particles in another order, so an item that a
    schedule skipped would leave another run's partial sums behind and fail
    the comparison."""
    torch = torch_cuda
    wl = building_i16
    m = mcl.map_from_scene(wl.map)
    parts = wl.particles[:40001]
    other = parts.copy()
    other[:, :3] += np.float32(0.37)
    scan = wl.scan[: len(wl.scan) - 100]
    res = {}
    before = {3: 2, 2: 1, 1: 3, 0: 2}
    for order in (3, 2, 1, 0):
        for kw in (dict(), dict(particles_per_item=64), dict(points_per_chunk=1024),
                   dict(particles_per_item=16)):
            run_sensor(torch, mcl, m, other, scan, wl.sigma_hit, item_order=before[order], **kw)
            res[(order, tuple(kw.items()))] = run_sensor(torch, mcl, m, parts, scan, wl.sigma_hit,
                                                         item_order=order, **kw)
    for (order, kw), r in res.items():
        ref = res[(1, kw)]
        assert np.array_equal(r[0], ref[0]) and np.array_equal(r[1], ref[1]), (order, kw)
    plan = mcl.mcl_sensor_plan_get(m, len(parts), len(scan), mcl.sensor_params(0.1))
    K = -(-len(scan) // plan["points_per_chunk"])
    slots = plan["num_sms"] * plan["blocks_per_sm"]
    assert plan["n_items"] >= 2 * slots                   # auto takes dynamic sweeps here
    assert plan["item_order"] == 3 and plan["blocks_per_sweep"] == slots // K
    assert plan["grid"] == slots
    static = mcl.mcl_sensor_plan_get(m, len(parts), len(scan), mcl.sensor_params(0.1, item_order=2))
    assert static["item_order"] == 2 and static["grid"] == static["blocks_per_sweep"] * K
    small = mcl.mcl_sensor_plan_get(m, 1000, len(scan), mcl.sensor_params(0.1))
    assert small["item_order"] == 1                       # too few items: chunk-major
    tri = mcl.mcl_sensor_plan_get(m, len(parts), len(scan), mcl.sensor_params(0.1, flags=mcl.MCL_TRILINEAR))
    assert tri["item_order"] == 3                         # auto: dynamic sweeps for the trilinear read too
    Lo = oracle.sensor_update(oracle.Map.from_scene_map(wl.map), parts[:200], scan, wl.sigma_hit)
    check_logw(res[(3, ())][0][:200], Lo)
    m.close()


def test_brick_layouts_give_identical_bits(torch_cuda, mcl, room):
    """The device layout and the brick index only move values and change how
    a brick is found: same reads, same sums, same bits."""
    torch = torch_cuda
    for dtype in (scenes.F32, scenes.F16, scenes.I16):
        sm = room_map(room.scene, "brick", dtype)
        res = []
        for layout, index in ((0, 2), (0, 1), (1, 1)):
            m = mcl.map_from_scene(sm, layout, index)
            res.append(run_sensor(torch, mcl, m, room.particles, room.scan, room.sigma_hit))
            for flags in (mcl.MCL_TRILINEAR, mcl.MCL_NEGLECT_OUTSIDE):
                res[-1] += run_sensor(torch, mcl, m, room.particles, room.scan, room.sigma_hit, 0, flags)
            m.close()
        for r in res[1:]:
            assert all(np.array_equal(x, y) for x, y in zip(res[0], r))
    with pytest.raises(mcl.MclError):  # the grid index is built for linear bricks only
        mcl.map_from_scene(sm, 1, 2)


def test_building_full_size_sampled(torch_cuda, mcl, building_i16):
    """1M particles x 65,536 points in the benchmark's launch configuration;
    the oracle recomputes a seeded sample of particles one by one."""
    torch = torch_cuda
    wl = building_i16
    m = mcl.map_from_scene(wl.map)
    Lg, wg = run_sensor(torch, mcl, m, wl.particles, wl.scan, wl.sigma_hit)
    rng = np.random.default_rng(7)
    sample = np.concatenate([rng.choice(len(Lg), 300, replace=False), [int(np.argmax(Lg))]])
    Lo = oracle.sensor_update(oracle.Map.from_scene_map(wl.map), wl.particles[sample], wl.scan,
                              wl.sigma_hit)
    check_logw(Lg[sample], Lo)
    w64 = wg.astype(np.float64)
    assert abs(w64.sum() - 1.0) <= TOL
    # Normalised weights against the oracle: both sides relative to the GPU's
    # most likely particle (the last entry of the sample), under the r9 gate on
    # log-weights; particles the oracle puts below 1e-30 of it must be as
    # unlikely on the GPU (up to the same bound).
    jmax = len(sample) - 1
    assert w64[sample[jmax]] == w64.max()
    Lref = Lo[jmax]
    assert Lo.max() - Lref <= TOL * 2 * max(1.0, abs(Lref)), "oracle's best sampled particle differs"
    lw_o = Lo - Lref
    bound = TOL * (np.maximum(1.0, np.abs(Lo)) + max(1.0, abs(Lref)))
    sel = lw_o >= math.log(1e-30)
    with np.errstate(divide="ignore"):
        lw_g = np.log(w64[sample] / w64.max())
    assert sel.sum() >= 1
    assert np.all(np.abs(lw_g[sel] - lw_o[sel]) <= bound[sel])
    assert np.all(lw_g[~sel] <= lw_o[~sel] + bound[~sel])
    m.close()


# ----------------------------------------------------------------- a9: systematic resampling
@pytest.mark.parametrize("P", [1, 2, 3, 33, 128, 129, 1000, 2049, 4095, 4096, 4097, 65537, 1_000_000])
def test_resample_bit_exact(torch_cuda, mcl, P):
    torch = torch_cuda
    rng = np.random.default_rng(P)
    w = rng.exponential(1.0, P) ** 4
    w[rng.random(P) < 0.2] = 0.0
    if w.sum() == 0:
        w[0] = 1.0
    w32 = (w / w.sum()).astype(np.float32)
    wd = dev(torch, w32)
    parts = rng.normal(0, 1, (P, 6)).astype(np.float32)
    for r in (0.0, 0.5, 1.0 - 2.0 ** -53):
        idx = torch.empty(P, dtype=torch.int32, device="cuda")
        out = torch.empty((P, 6), device="cuda")
        mcl.mcl_resample(wd, r, idx, dev(torch, parts), out)
        mcl.mcl_sync()
        ref, _ = oracle.resample(w32, r)
        got = idx.cpu().numpy()
        assert np.array_equal(got, ref)
        assert np.array_equal(out.cpu().numpy(), parts[ref])


def test_resample_degenerate_and_one_hot(torch_cuda, mcl):
    torch = torch_cuda
    idx = torch.empty(10, dtype=torch.int32, device="cuda")
    mcl.mcl_resample(torch.zeros(10, device="cuda"), 0.3, idx)
    mcl.mcl_sync()
    assert list(idx.cpu().numpy()) == list(range(10))
    w = torch.zeros(10, device="cuda")
    w[7] = 1.0
    mcl.mcl_resample(w, 0.99, idx)
    mcl.mcl_sync()
    assert np.all(idx.cpu().numpy() == 7)


def test_resample_after_sensor_update(torch_cuda, mcl, room):
    torch = torch_cuda
    m = mcl.map_from_scene(room.map)
    _, wg = run_sensor(torch, mcl, m, room.particles, room.scan, room.sigma_hit)
    idx = torch.empty(len(wg), dtype=torch.int32, device="cuda")
    mcl.mcl_resample(dev(torch, wg), 0.25, idx)
    mcl.mcl_sync()
    check_systematic(idx.cpu().numpy(), wg, 0.25)   # GPU weights: properties, not the oracle
    m.close()


# ----------------------------------------------------------------- a13: motion update
def test_motion_update_parity(torch_cuda, mcl):
    torch = torch_cuda
    rng = np.random.default_rng(5)
    P = 50_000
    poses = np.concatenate([rng.normal(0, 30, (P, 3)), rng.uniform(-1.4, 1.4, (P, 3))], 1).astype(np.float32)
    delta = np.float32([0.3, -0.1, 0.05, 0.01, -0.02, 0.2])
    sigma = np.float32([0.1, 0.1, 0.05, 0.01, 0.01, 0.1])
    t = dev(torch, poses)
    mcl.mcl_motion_update(t, delta, sigma, seed=0x1234_5678_9ABC, step=42)
    mcl.mcl_sync()
    got = t.cpu().numpy().astype(np.float64)
    ref = oracle.motion_update(poses, delta, sigma, 0x1234_5678_9ABC, 42).astype(np.float64)
    pos_err = np.abs(got[:, :3] - ref[:, :3]) / np.maximum(1.0, np.abs(ref[:, :3]))
    assert pos_err.max() <= 2e-6
    ang = np.abs(np.angle(np.exp(1j * (got[:, 3:] - ref[:, 3:]))))
    assert ang.max() <= 2e-6
    # Small sets run a kernel that splits each particle's FP64 work over six
    # warps: same bits as the one-thread-per-particle kernel (the noise of
    # particle i depends only on i), for set sizes around the switch.
    for n in (1, 31, 1000, 5120, 5121):
        ts = dev(torch, poses[:n])
        mcl.mcl_motion_update(ts, delta, sigma, seed=0x1234_5678_9ABC, step=42)
        mcl.mcl_sync()
        assert np.array_equal(ts.cpu().numpy(), got[:n].astype(np.float32)), n
    ts = dev(torch, poses[:1000])
    mcl.mcl_motion_update(ts, np.zeros(6, np.float32), sigma, seed=3, step=1)  # noise only
    mcl.mcl_sync()
    ref = oracle.motion_update(poses[:1000], np.zeros(6, np.float32), sigma, 3, 1).astype(np.float64)
    got1 = ts.cpu().numpy().astype(np.float64)
    assert (np.abs(got1[:, :3] - ref[:, :3]) / np.maximum(1.0, np.abs(ref[:, :3]))).max() <= 2e-6
    assert np.abs(np.angle(np.exp(1j * (got1[:, 3:] - ref[:, 3:])))).max() <= 2e-6


# ----------------------------------------------------------------- determinism, errors, profiling
def test_repeat_calls_bit_identical(torch_cuda, mcl, room):
    torch = torch_cuda
    m = mcl.map_from_scene(room.map)
    a = run_sensor(torch, mcl, m, room.particles, room.scan, room.sigma_hit)
    b = run_sensor(torch, mcl, m, room.particles, room.scan, room.sigma_hit)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    m.close()


def test_invalid_arguments_are_refused(torch_cuda, mcl, room):
    torch = torch_cuda
    m = mcl.map_from_scene(room.map)
    parts, scan = dev(torch, room.particles), dev(torch, room.scan)
    logw = torch.empty(len(parts), device="cuda")
    L = mcl.lib()
    for bad in [dict(sigma_hit=0.0), dict(sigma_hit=float("nan")), dict(mode=7), dict(flags=8),
                dict(points_per_chunk=48), dict(lanes_per_particle=12), dict(unroll=3),
                dict(unroll=16), dict(pipeline=3), dict(particle_order=5), dict(item_order=4),
                dict(item_order=-1)]:
        kw = dict(sigma_hit=0.1)
        kw.update(bad)
        with pytest.raises(mcl.MclError) as e:
            mcl.mcl_sensor_update(m, parts, scan, mcl.sensor_params(**kw), logw)
        assert e.value.status == mcl.MCL_EINVAL
    prm = mcl.sensor_params(0.1)
    s = mcl._stream(None)
    assert L.mcl_sensor_update(m.handle, parts.data_ptr(), 0, scan.data_ptr(), 10, ctypes.byref(prm),
                               logw.data_ptr(), None, s) == mcl.MCL_EINVAL
    assert L.mcl_sensor_update(m.handle, parts.data_ptr(), 10, scan.data_ptr(), 0, ctypes.byref(prm),
                               logw.data_ptr(), None, s) == mcl.MCL_EINVAL
    assert L.mcl_sensor_update(m.handle, parts.data_ptr() + 2, 10, scan.data_ptr(), 10,
                               ctypes.byref(prm), logw.data_ptr(), None, s) == mcl.MCL_EINVAL
    assert L.mcl_sensor_update(m.handle, parts.data_ptr(), 10, scan.data_ptr(), 10, ctypes.byref(prm),
                               None, None, s) == mcl.MCL_EINVAL
    idx = torch.empty(10, dtype=torch.int32, device="cuda")
    for r in (-0.1, 1.0, float("nan")):
        with pytest.raises(mcl.MclError):
            mcl.mcl_resample(torch.ones(10, device="cuda"), r, idx)
    with pytest.raises(mcl.MclError):
        mcl.mcl_motion_update(parts, [0] * 6, [0, 0, -1, 0, 0, 0], 1, 1)
    # brick maps: duplicated or out-of-range brick coordinates
    with pytest.raises(mcl.MclError):
        mcl.mcl_map_create(mcl.MCL_MAP_BRICK, mcl.MCL_I16, (0, 0, 0), 0.05, 0.3, (32, 32, 32),
                           np.zeros((2, 16, 16, 16), np.int16), np.int32([[0, 0, 0], [0, 0, 0]]))
    with pytest.raises(mcl.MclError):
        mcl.mcl_map_create(mcl.MCL_MAP_BRICK, mcl.MCL_I16, (0, 0, 0), 0.05, 0.3, (32, 32, 32),
                           np.zeros((1, 16, 16, 16), np.int16), np.int32([[2, 0, 0]]))
    with pytest.raises(mcl.MclError):
        mcl.mcl_map_create(mcl.MCL_MAP_BRICK, mcl.MCL_I16, (0, 0, 0), 0.05, 0.3, (30, 32, 32),
                           np.zeros((1, 16, 16, 16), np.int16), np.int32([[0, 0, 0]]))
    mcl.mcl_sync()  # nothing above reached the device: status stays clean
    m.close()


def test_profile_counts_phases(torch_cuda, mcl, room):
    torch = torch_cuda
    m = mcl.map_from_scene(room.map)
    mcl.mcl_profile_begin()
    run_sensor(torch, mcl, m, room.particles, room.scan, room.sigma_hit)
    prof = mcl.mcl_profile_end()
    assert prof["sensor"]["launches"] == 1 and prof["sensor"]["ms"] > 0
    assert prof["pose"]["launches"] == 1 and prof["normalise"]["launches"] == 1
    assert prof["pack"]["launches"] == 0        # the pose phase's kernel packs the scan
    m.close()


@pytest.mark.parametrize("index", [1, 2])
def test_empty_brick_map_and_non_finite_scan_points(torch_cuda, mcl, room, index):
    """A brick map with no brick reads +tau everywhere (both indexes); scan
    points that are NaN or infinite fall outside the grid."""
    torch = torch_cuda
    empty = scenes.BrickMap((0.0, 0.0, 0.0), 0.05, (128, 128, 64), 0.3, scenes.I16,
                            np.zeros((0, 3), np.int32), np.zeros((0, 16, 16, 16), np.int16))
    m = mcl.map_from_scene(empty, 0, index)
    assert m.info()["n_bricks"] == 0
    scan = room.scan.copy()
    scan[::97] = np.float32([np.nan, 0.0, 1.0])
    scan[5::101] = np.float32([np.inf, -np.inf, 0.0])
    for flags in (0, mcl.MCL_TRILINEAR):
        Lg, wg = run_sensor(torch, mcl, m, room.particles, scan, 0.1, 0, flags)
        Lo = oracle.sensor_update(oracle.Map.from_scene_map(empty), room.particles, scan, 0.1,
                                  trilinear=bool(flags))
        check_logw(Lg, Lo)
        assert np.allclose(wg, 1.0 / len(wg), rtol=1e-6)     # every particle scores the same
    m.close()
    # the room with the same bad points
    m = mcl.map_from_scene(room.map)
    Lg, _ = run_sensor(torch, mcl, m, room.particles, scan, 0.1)
    check_logw(Lg, oracle.sensor_update(oracle.Map.from_scene_map(room.map), room.particles, scan, 0.1))
    m.close()
