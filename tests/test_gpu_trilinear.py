"""GPU parity of the trilinear read (MCL_TRILINEAR; Sec. III: a
pseudo-continuous value by interpolation) against the FP64 oracle, through
the C ABI. The corner indices and weights are FP32 on both sides (parity
mode), the interpolation FP32 on the GPU and FP64 in the oracle, so the
log-weights carry the sensor update's tolerance: |L_gpu - L_ora| <= 1e-5 *
max(1, |L_ora|); weights as in the nearest-voxel parity tests."""
import numpy as np
import pytest

import oracle
import scenes
from test_gpu_parity import KINDS, check_logw, check_w, dev, room_map, upload

pytestmark = pytest.mark.gpu


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


def run_tri(torch, mcl, m, parts, scan, sigma, mode=0, flags=0, **shape):
    P = parts.shape[0]
    logw, w = torch.empty(P, device="cuda"), torch.empty(P, device="cuda")
    prm = mcl.sensor_params(sigma_hit=sigma, mode=mode, flags=flags | mcl.MCL_TRILINEAR, **shape)
    mcl.mcl_sensor_update(m, dev(torch, parts), dev(torch, scan), prm, logw, w)
    mcl.mcl_sync()
    return logw.cpu().numpy(), w.cpu().numpy()


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("dtype", [scenes.F32, scenes.F16, scenes.I16])
@pytest.mark.parametrize("mode", [oracle.LOGPROD, oracle.SUM])
@pytest.mark.parametrize("neglect", [False, True])
def test_trilinear_room(torch_cuda, mcl, room, kind, dtype, mode, neglect):
    torch = torch_cuda
    sm = room_map(room.scene, kind, dtype)
    m = upload(mcl, sm, kind)
    parts = room.particles.copy()
    parts[:50, :3] += np.float32(4.0)   # much of their scan falls outside the grid
    Lg, wg = run_tri(torch, mcl, m, parts, room.scan, room.sigma_hit, mode,
                     mcl.MCL_NEGLECT_OUTSIDE if neglect else 0)
    Lo = oracle.sensor_update(oracle.Map.from_scene_map(sm), parts, room.scan, room.sigma_hit, mode,
                              neglect, parity=True, trilinear=True)
    check_logw(Lg, Lo)
    check_w(wg, Lo, mode)
    # the read is not the nearest-voxel one
    Ln = oracle.sensor_update(oracle.Map.from_scene_map(sm), parts, room.scan, room.sigma_hit, mode,
                              neglect, parity=True)
    fin = np.isfinite(Ln) & np.isfinite(Lo)
    assert np.max(np.abs(Ln[fin] - Lo[fin])) > 1e-3
    m.close()


@pytest.mark.parametrize("chunk,ppi", [(32, 1), (1024, 500), (2048, 33), (8192, 64)])
def test_trilinear_ragged_tails_and_hints(torch_cuda, mcl, room, chunk, ppi):
    torch = torch_cuda
    m = mcl.map_from_scene(room.map)
    parts = np.concatenate([room.particles, room.particles[:1]])   # P = 1001
    scan = room.scan[:1000]                                        # N = 1000
    Lg, wg = run_tri(torch, mcl, m, parts, scan, room.sigma_hit, points_per_chunk=chunk,
                     particles_per_item=ppi)
    Lo = oracle.sensor_update(oracle.Map.from_scene_map(room.map), parts, scan, room.sigma_hit,
                              parity=True, trilinear=True)
    check_logw(Lg, Lo)
    Lh, wh = run_tri(torch, mcl, m, parts, scan, room.sigma_hit, points_per_chunk=chunk,
                     particles_per_item=max(1, ppi // 3), unroll=8, particle_order=2)
    assert np.array_equal(Lg, Lh) and np.array_equal(wg, wh)      # hints change no bit
    m.close()


def test_trilinear_building_full_size_sampled(torch_cuda, mcl):
    """1M particles x 65,536 points in the bench's launch configuration of the
    trilinear variant; the oracle recomputes a seeded sample one by one."""
    torch = torch_cuda
    wl = scenes.os064_building(P=1_000_000, dtype=scenes.I16)
    m = mcl.map_from_scene(wl.map)
    Lg, wg = run_tri(torch, mcl, m, wl.particles, wl.scan, wl.sigma_hit)
    rng = np.random.default_rng(11)
    sample = np.concatenate([rng.choice(len(Lg), 200, replace=False), [int(np.argmax(Lg))]])
    Lo = oracle.sensor_update(oracle.Map.from_scene_map(wl.map), wl.particles[sample], wl.scan,
                              wl.sigma_hit, parity=True, trilinear=True)
    check_logw(Lg[sample], Lo)
    assert abs(wg.astype(np.float64).sum() - 1.0) <= 1e-5
    m.close()


def test_trilinear_building_subset(torch_cuda, mcl):
    torch = torch_cuda
    wl = scenes.os064_building(P=1500, dtype=scenes.I16)
    m = mcl.map_from_scene(wl.map)
    parts = wl.particles[:600]
    Lg, _ = run_tri(torch, mcl, m, parts, wl.scan, wl.sigma_hit)
    Lo = oracle.sensor_update(oracle.Map.from_scene_map(wl.map), parts, wl.scan, wl.sigma_hit,
                              parity=True, trilinear=True)
    check_logw(Lg, Lo)
    m.close()


def test_trilinear_batch_and_filter_match_single_calls(torch_cuda, mcl, room):
    torch = torch_cuda
    m = mcl.map_from_scene(room.map)
    P = 1000
    parts = dev(torch, room.particles)
    scan = dev(torch, room.scan)
    L1, w1 = run_tri(torch, mcl, m, room.particles, room.scan, room.sigma_hit)
    s = {"map": m, "particles": parts, "scan": scan, "sigma_hit": room.sigma_hit,
         "flags": mcl.MCL_TRILINEAR, "logw": torch.empty(P, device="cuda"),
         "w": torch.empty(P, device="cuda")}
    other = dict(s, flags=0, logw=torch.empty(P, device="cuda"), w=torch.empty(P, device="cuda"))
    b = mcl.Batch([s, other], use_graph=True)
    b.run()
    mcl.mcl_sync()
    assert np.array_equal(s["logw"].cpu().numpy(), L1)
    assert b.info()["n_groups"] == 2                    # the read rule splits the group
    b.close()
    prm = mcl.sensor_params(sigma_hit=room.sigma_hit, flags=mcl.MCL_TRILINEAR)
    f = mcl.Filter(m, parts, max_points=len(room.scan), params=prm, seed=3)
    f.step(scan)                                       # no odometry: the weights of the particles
    mcl.mcl_sync()
    assert np.array_equal(f.tensors()["logw"].cpu().numpy(), L1)
    f.close()
    m.close()


def test_trilinear_needs_whole_warp_groups(torch_cuda, mcl, room):
    torch = torch_cuda
    m = mcl.map_from_scene(room.map)
    with pytest.raises(mcl.MclError) as e:
        run_tri(torch, mcl, m, room.particles, room.scan, room.sigma_hit, lanes_per_particle=16)
    assert e.value.status == mcl.MCL_EINVAL
    m.close()
