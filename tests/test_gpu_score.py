"""GPU parity of the score map (mcl_map_create_score; Sec. III: the
exponential of Eq. 3 evaluated once per map entry before the scans) against
the FP64 oracle, through the C ABI:
- the stored scores are bit-exact (both sides evaluate exp in FP64 and round
  once to FP16 / FP32, nearest even);
- the SUM-mode update on a score map matches the oracle's SCORE mode within
  the sensor update's tolerance, and the GPU's own TSDF SUM update within
  the FP16 rounding of the scores;
- batched sessions on a score map equal the single calls bit for bit."""
import math

import numpy as np
import pytest

import oracle
import scenes
from test_gpu_parity import check_logw, check_w, dev, room_map, upload

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


def oracle_score_map(sm, sigma, dtype):
    import dataclasses
    vals, outside = oracle.score_map(sm, sigma, dtype)
    return oracle.Map.from_scene_map(dataclasses.replace(sm, values=vals, dtype=dtype)).set_outside(outside), \
        vals, outside


def voxel_centres(sm, rng, n):
    k = rng.integers(0, np.asarray(sm.dims), (n, 3))
    return ((np.asarray(sm.origin) + (k + 0.5) * sm.voxel).astype(np.float32), k)


@pytest.mark.parametrize("kind", ["dense", "brick"])
@pytest.mark.parametrize("src_dtype", [scenes.F32, scenes.F16, scenes.I16])
@pytest.mark.parametrize("dtype", [scenes.F16, scenes.F32])
def test_score_values_bit_exact(torch_cuda, mcl, room, kind, src_dtype, dtype):
    torch = torch_cuda
    sm = room_map(room.scene, kind, src_dtype)
    m = upload(mcl, sm, kind)
    sc = mcl.mcl_map_create_score(m, 0.1, dtype)
    info = sc.info()
    om, vals, outside = oracle_score_map(sm, 0.1, dtype)
    assert info["score_sigma"] == np.float32(0.1) and info["score_outside"] == np.float32(outside)
    rng = np.random.default_rng(5)
    pts, _ = voxel_centres(sm, rng, 200_000)
    pts = np.concatenate([pts, np.float32([[-1, -1, -1], [100, 0, 0]])])
    out_v = torch.empty(len(pts), device="cuda")
    mcl.mcl_map_lookup(sc, dev(torch, pts), out_value=out_v)
    mcl.mcl_sync()
    _, ov = oracle.map_lookup(om, pts)
    assert np.array_equal(out_v.cpu().numpy().astype(np.float64), ov)
    sc.close()
    m.close()


@pytest.mark.parametrize("kind", ["dense", "brick"])
@pytest.mark.parametrize("neglect", [False, True])
def test_score_map_sensor_update(torch_cuda, mcl, room, kind, neglect):
    torch = torch_cuda
    sm = room_map(room.scene, kind, scenes.I16)
    m = upload(mcl, sm, kind)
    sc = mcl.mcl_map_create_score(m, room.sigma_hit)
    parts = room.particles.copy()
    parts[:50, :3] += np.float32(4.0)
    flags = mcl.MCL_NEGLECT_OUTSIDE if neglect else 0
    P = len(parts)
    out = {}
    for name, mm in (("score", sc), ("tsdf", m)):
        logw, w = torch.empty(P, device="cuda"), torch.empty(P, device="cuda")
        prm = mcl.sensor_params(room.sigma_hit, mode=mcl.MCL_SUM, flags=flags)
        mcl.mcl_sensor_update(mm, dev(torch, parts), dev(torch, room.scan), prm, logw, w)
        mcl.mcl_sync()
        out[name] = (logw.cpu().numpy(), w.cpu().numpy())
    om, _, _ = oracle_score_map(sm, room.sigma_hit, scenes.F16)
    Lo = oracle.sensor_update(om, parts, room.scan, room.sigma_hit, oracle.SCORE, neglect)
    check_logw(out["score"][0], Lo)
    check_w(out["score"][1], Lo, oracle.SUM)
    Ls, Lt = out["score"][0].astype(np.float64), out["tsdf"][0].astype(np.float64)
    fin = np.isfinite(Lt)
    assert np.array_equal(fin, np.isfinite(Ls))
    assert np.all(np.abs(Ls[fin] - Lt[fin]) <= math.log1p(2.0 ** -11) + 2e-5 * np.abs(Lt[fin]))
    sc.close()
    m.close()


def test_score_map_in_batch_and_filter(torch_cuda, mcl, room):
    torch = torch_cuda
    m = mcl.map_from_scene(room.map)
    sc = mcl.mcl_map_create_score(m, room.sigma_hit)
    P = 1000
    parts, scan = dev(torch, room.particles), dev(torch, room.scan)
    prm = mcl.sensor_params(room.sigma_hit, mode=mcl.MCL_SUM)
    L1, w1 = torch.empty(P, device="cuda"), torch.empty(P, device="cuda")
    mcl.mcl_sensor_update(sc, parts, scan, prm, L1, w1)
    s = {"map": sc, "particles": parts, "scan": scan, "sigma_hit": room.sigma_hit, "mode": mcl.MCL_SUM,
         "logw": torch.empty(P, device="cuda"), "w": torch.empty(P, device="cuda")}
    b = mcl.Batch([s], use_graph=True)
    b.run()
    f = mcl.Filter(sc, parts, max_points=len(room.scan), params=prm, seed=1)
    f.step(scan)
    mcl.mcl_sync()
    assert torch.equal(s["logw"], L1) and torch.equal(s["w"], w1)
    assert torch.equal(f.tensors()["logw"], L1)
    f.close()
    b.close()
    sc.close()
    m.close()


def test_score_map_rejects_other_uses(torch_cuda, mcl, room):
    torch = torch_cuda
    m = mcl.map_from_scene(room.map)
    sc = mcl.mcl_map_create_score(m, 0.1)
    parts, scan = dev(torch, room.particles), dev(torch, room.scan)
    logw = torch.empty(1000, device="cuda")
    bad = [mcl.sensor_params(0.1, mode=mcl.MCL_LOGPROD),
           mcl.sensor_params(0.2, mode=mcl.MCL_SUM),
           mcl.sensor_params(0.1, mode=mcl.MCL_SUM, flags=mcl.MCL_TRILINEAR),
           mcl.sensor_params(0.1, mode=mcl.MCL_SUM, pipeline=2)]
    for prm in bad:
        with pytest.raises(mcl.MclError) as e:
            mcl.mcl_sensor_update(sc, parts, scan, prm, logw)
        assert e.value.status == mcl.MCL_EINVAL
    for args in ((sc, 0.1, mcl.MCL_F16), (m, 0.0, mcl.MCL_F16), (m, 0.1, mcl.MCL_I16),
                 (m, float("nan"), mcl.MCL_F32)):
        with pytest.raises(mcl.MclError):
            mcl.mcl_map_create_score(*args)
    sc.close()
    m.close()
