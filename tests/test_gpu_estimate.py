"""GPU parity of the pose estimate (Sec. III: weighted average of the
particles or the particle with the highest weight; Sec. V: weighted sum of the
poses after the weights) against the FP64 oracle, through the C ABI.

Tolerances: the GPU sums in FP64 like the oracle but in another order, and
forms each particle's quaternion in FP32 (a few ulps, ~2e-7 per component):
- weight_sum, n_eff: 1e-12 relative; mean_pose: 1e-12 relative to the
  largest |component| (FP64 sums of the same FP32 products);
- quat: 2e-6 absolute, rpy: 4e-6 rad, concentration: 2e-6 (FP32 quaternion
  terms; clouds are concentrated, so the eigenvector is well conditioned);
- argmax, best_pose, best_w: exact (the maximum is unique or ties resolve to
  the lowest index on both sides).
"""
import math

import numpy as np
import pytest

import oracle
import scenes

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


def _cloud(P, seed, centre, spread_t=0.5, spread_deg=10.0):
    return scenes.particles_gaussian(np.asarray(centre, np.float32), P, spread_t, spread_deg, seed)


def _weights(P, seed):
    z = scenes.normal(seed, 5, P)
    return np.exp(2.0 * z).astype(np.float32)          # unnormalised, positive, seeded


def _gpu_estimate(torch, mcl, parts, w):
    out = mcl.estimate_buffer()
    mcl.mcl_pose_estimate(torch.from_numpy(parts).cuda(), torch.from_numpy(w).cuda(), out)
    mcl.mcl_sync()
    return mcl.estimate_to_dict(out), out


def _compare(g, o):
    assert g["weight_sum"] == pytest.approx(o["weight_sum"], rel=1e-12)
    assert g["n_eff"] == pytest.approx(o["n_eff"], rel=1e-10)
    scale = max(1.0, float(np.abs(o["mean_pose"]).max()))
    np.testing.assert_allclose(g["mean_pose"], o["mean_pose"], rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(g["quat"], o["quat"], rtol=0, atol=2e-6)
    d = (g["rpy"] - o["rpy"] + math.pi) % (2 * math.pi) - math.pi
    assert np.abs(d).max() <= 4e-6
    assert g["concentration"] == pytest.approx(o["concentration"], abs=2e-6)
    assert g["argmax"] == o["argmax"]
    np.testing.assert_array_equal(g["best_pose"], o["best_pose"])
    assert g["best_w"] == o["best_w"]


@pytest.mark.parametrize("P", [1, 7, 1000, 1025, 100_003, 1_048_576, 1_500_001])
def test_estimate_matches_oracle(torch_cuda, mcl, P):
    parts = _cloud(P, 100 + P % 97, [3.0, -2.0, 1.2, 0.1, -0.05, 1.3])
    w = _weights(P, 7 + P % 13)
    g, _ = _gpu_estimate(torch_cuda, mcl, parts, w)
    _compare(g, oracle.pose_estimate(parts, w))


def test_estimate_across_the_yaw_wrap(torch_cuda, mcl):
    parts = _cloud(20_000, 5, [0.0, 0.0, 0.0, 0.0, 0.0, math.pi - 0.02], 0.1, 3.0)
    parts[:, 5] = (parts[:, 5] + np.float32(math.pi)) % np.float32(2 * math.pi) - np.float32(math.pi)
    w = _weights(20_000, 9)
    g, _ = _gpu_estimate(torch_cuda, mcl, parts, w)
    o = oracle.pose_estimate(parts, w)
    _compare(g, o)
    assert abs(abs(g["rpy"][2]) - math.pi) < 0.05     # the rotation mean stays at the wrap


def test_estimate_special_weights(torch_cuda, mcl):
    P = 5000
    parts = _cloud(P, 11, [1.0, 2.0, 3.0, 0.2, 0.1, -2.0])
    one = np.zeros(P, np.float32)
    one[1234] = 0.25
    g, _ = _gpu_estimate(torch_cuda, mcl, parts, one)
    assert g["argmax"] == 1234 and g["n_eff"] == 1.0 and g["weight_sum"] == 0.25
    np.testing.assert_array_equal(g["mean_pose"], parts[1234].astype(np.float64))
    _compare(g, oracle.pose_estimate(parts, one))
    ties = np.full(P, 0.5, np.float32)
    g, _ = _gpu_estimate(torch_cuda, mcl, parts, ties)
    assert g["argmax"] == 0 and g["n_eff"] == pytest.approx(P, rel=1e-12)
    nanw = _weights(P, 3)
    nanw[::3] = np.nan
    g, _ = _gpu_estimate(torch_cuda, mcl, parts, nanw)
    assert g["argmax"] == oracle.pose_estimate(parts, nanw)["argmax"]
    g, _ = _gpu_estimate(torch_cuda, mcl, parts, np.zeros(P, np.float32))
    assert g["argmax"] == 0 and g["n_eff"] == 0.0 and g["weight_sum"] == 0.0
    assert np.all(np.isnan(g["mean_pose"])) and np.all(np.isnan(g["quat"]))


def test_fused_estimate_equals_standalone_and_oracle(torch_cuda, mcl):
    torch = torch_cuda
    wl = scenes.room_plain(P=1000)
    m = mcl.map_from_scene(wl.map)
    parts = torch.from_numpy(wl.particles).cuda()
    scan = torch.from_numpy(wl.scan).cuda()
    prm = mcl.sensor_params(sigma_hit=wl.sigma_hit)
    logw0, w0 = torch.empty(1000, device="cuda"), torch.empty(1000, device="cuda")
    mcl.mcl_sensor_update(m, parts, scan, prm, logw0, w0)
    logw, w, out = torch.empty(1000, device="cuda"), torch.empty(1000, device="cuda"), mcl.estimate_buffer()
    mcl.mcl_sensor_update_estimate(m, parts, scan, prm, logw, w, out)
    ref = mcl.estimate_buffer()
    mcl.mcl_pose_estimate(parts, w, ref)
    mcl.mcl_sync()
    assert torch.equal(logw, logw0) and torch.equal(w, w0)       # the fusion changes no weight
    assert torch.equal(out, ref)                                  # bit for bit
    g = mcl.estimate_to_dict(out)
    # Against the oracle's own weights: the difference is bounded by the
    # weight error times the spread of the poses.
    Lo = oracle.sensor_update(oracle.Map.from_scene_map(wl.map), wl.particles, wl.scan, wl.sigma_hit)
    wo, *_ = oracle.normalise(Lo)
    o = oracle.pose_estimate(wl.particles, wo.astype(np.float32))
    wg = w.cpu().numpy().astype(np.float64)
    dw = np.abs(wg - wo).sum()
    spread = np.abs(wl.particles.astype(np.float64) - o["mean_pose"]).max()
    np.testing.assert_allclose(g["mean_pose"], o["mean_pose"], rtol=0, atol=2 * dw * spread + 1e-9)
    assert np.abs(g["quat"] - o["quat"]).max() <= 2 * dw + 4e-6
    assert g["argmax"] == o["argmax"]
    m.close()


def test_estimate_invalid_arguments(torch_cuda, mcl):
    torch = torch_cuda
    parts = torch.zeros(10, 6, device="cuda")
    w = torch.ones(10, device="cuda")
    lib = mcl.lib()
    out = mcl.estimate_buffer()
    assert lib.mcl_pose_estimate(parts.data_ptr(), w.data_ptr(), 10, None, None) == mcl.MCL_EINVAL
    assert lib.mcl_pose_estimate(parts.data_ptr(), w.data_ptr(), 0, out.data_ptr(), None) == mcl.MCL_EINVAL
    assert lib.mcl_pose_estimate(parts.data_ptr(), w.data_ptr(), 10, out.data_ptr() + 4, None) == mcl.MCL_EINVAL
    assert lib.mcl_pose_estimate(None, w.data_ptr(), 10, out.data_ptr(), None) == mcl.MCL_EINVAL
