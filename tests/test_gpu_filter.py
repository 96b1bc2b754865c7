"""Whole filter steps on the GPU (mcl_filter_*): each step equals the single
C-ABI calls it is made of, bit for bit (plain and replayed from CUDA
graphs, with ragged scan sizes and a step without odometry); the filter
tracks the seeded room path like the oracle's filter; a serving session with
the same seed reaches the same particles."""
import math

import numpy as np
import pytest

import oracle
import scenes
from test_oracle_tracking import MOTION_SIGMA, errors, splitmix_offset, tracking_case

pytestmark = pytest.mark.gpu

SEED = 123


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2310_04172_gb300 import _build, mcl
    _build.build()
    mcl.lib()
    torch.cuda.set_device(0)
    case = tracking_case()
    m = mcl.map_from_scene(case[0].map)
    yield torch, mcl, case, m
    m.close()


def ragged(scans, k):
    return scans[k][: len(scans[k]) - 16 * (k % 3)]


@pytest.mark.parametrize("use_graph", [False, True])
def test_filter_step_equals_single_calls(env, use_graph):
    torch, mcl, (wl, poses, deltas, scans, parts0), m = env
    P = len(parts0)
    prm = mcl.sensor_params(sigma_hit=wl.sigma_hit)
    f = mcl.Filter(m, torch.from_numpy(parts0).cuda(), max_points=1024, params=prm,
                   motion_sigma=MOTION_SIGMA, seed=SEED, use_graph=use_graph)
    ref = torch.from_numpy(parts0).cuda()
    logw, w = torch.empty(P, device="cuda"), torch.empty(P, device="cuda")
    idx, nxt = torch.empty(P, dtype=torch.int32, device="cuda"), torch.empty((P, 6), device="cuda")
    est_f, est_r = mcl.estimate_buffer(), mcl.estimate_buffer()
    views = f.tensors()
    for k in range(8):
        delta = None if k == 0 else deltas[k]
        scan = torch.from_numpy(ragged(scans, k)).cuda()
        f.step(scan, delta, est_f)
        if delta is not None:
            mcl.mcl_motion_update(ref, delta, MOTION_SIGMA, SEED, k)
        mcl.mcl_sensor_update_estimate(m, ref, scan, prm, logw, w, est_r)
        r = splitmix_offset(SEED, k)
        mcl.mcl_resample(w, r, idx, ref, nxt)
        ref.copy_(nxt)
        mcl.mcl_sync()
        st = f.state()
        assert st["last_r"] == r and st["steps"] == k + 1
        assert torch.equal(views["logw"], logw) and torch.equal(views["w"], w)
        assert torch.equal(views["idx"], idx) and torch.equal(views["particles"], ref)
        assert torch.equal(est_f, est_r) and torch.equal(views["estimate"], est_r)
    st = f.state()
    assert st["graph_launches"] == (8 if use_graph else 0)
    assert st["graphs"] == (3 if use_graph else 0)          # three scan sizes
    f.close()


def test_filter_tracks_the_path_like_the_oracle(env):
    torch, mcl, (wl, poses, deltas, scans, parts0), m = env
    f = mcl.Filter(m, torch.from_numpy(parts0).cuda(), max_points=1024,
                   params=mcl.sensor_params(sigma_hit=wl.sigma_hit), motion_sigma=MOTION_SIGMA,
                   seed=SEED, use_graph=True)
    out = mcl.estimate_buffer()
    errs = []
    for k in range(len(deltas)):
        f.step(torch.from_numpy(scans[k]).cuda(), deltas[k], out)
        errs.append(errors(mcl.estimate_to_dict(out), poses[k + 1]))
    errs = np.array(errs)
    assert errs[0, 0] > 0.1
    assert errs[-10:, 0].max() < 0.03
    assert errs[-10:, 1].max() < 0.5
    # The oracle's filter on the same inputs ends at the same place (both on
    # the path; their particles differ once rounding picks other draws).
    om = oracle.Map.from_scene_map(wl.map)
    parts = parts0.copy()
    for k in range(len(deltas)):
        parts = oracle.motion_update(parts, deltas[k], MOTION_SIGMA, SEED, k)
        wo, *_ = oracle.normalise(oracle.sensor_update(om, parts, scans[k], wl.sigma_hit))
        eo = oracle.pose_estimate(parts, wo.astype(np.float32))
        idx, _ = oracle.resample(wo.astype(np.float32), splitmix_offset(SEED, k))
        parts = parts[idx]
    eg = mcl.estimate_to_dict(out)
    assert np.linalg.norm(eg["mean_pose"][:3] - eo["mean_pose"][:3]) < 0.03
    f.close()


def test_filter_matches_a_serving_session(env):
    torch, mcl, (wl, poses, deltas, scans, parts0), m = env
    f = mcl.Filter(m, torch.from_numpy(parts0).cuda(), max_points=1024,
                   params=mcl.sensor_params(sigma_hit=wl.sigma_hit), motion_sigma=MOTION_SIGMA,
                   seed=SEED, use_graph=True)
    srv = mcl.Server(hbm_budget_bytes=1 << 30, max_sessions=2)
    ss = srv.open(m, parts0, max_N=1024, sigma_hit=wl.sigma_hit, motion_sigma=MOTION_SIGMA, seed=SEED)
    for k in range(5):
        f.step(torch.from_numpy(scans[k]).cuda(), deltas[k])
        t = ss.submit(scans[k], deltas[k])
        assert srv.wait(t, 60_000)["status"] == 0
    sp, sw = ss.read(60_000)
    mcl.mcl_sync()
    v = f.tensors()
    np.testing.assert_array_equal(sp, v["particles"].cpu().numpy())
    np.testing.assert_array_equal(sw, v["w"].cpu().numpy())
    ss.close()
    srv.close()
    f.close()


def test_filter_graph_cache_and_errors(env):
    torch, mcl, (wl, poses, deltas, scans, parts0), m = env
    f = mcl.Filter(m, torch.from_numpy(parts0[:500]).cuda(), max_points=1024, seed=1,
                   use_graph=True, max_graphs=2)
    for k, n in enumerate([1000, 900, 800, 1000, 700]):
        f.step(torch.from_numpy(scans[0][:n]).cuda(), deltas[k])
    mcl.mcl_sync()
    st = f.state()
    assert st["graphs"] == 2 and st["graph_launches"] == 5 and st["steps"] == 5
    too_long = torch.zeros((1025, 3), device="cuda")
    with pytest.raises(mcl.MclError) as e:
        f.step(too_long)
    assert e.value.status == mcl.MCL_EINVAL
    with pytest.raises(mcl.MclError):
        f.step(torch.from_numpy(scans[0]).cuda(), [0, 0, float("nan"), 0, 0, 0])
    with pytest.raises(mcl.MclError):
        mcl.Filter(m, torch.from_numpy(parts0).cuda(), max_points=0)
    with pytest.raises(mcl.MclError):
        mcl.Filter(m, torch.from_numpy(parts0).cuda(), max_points=10, motion_sigma=[-1, 0, 0, 0, 0, 0])
    assert f.state()["steps"] == 5                           # failed calls enqueue nothing
    f.close()


def test_filter_and_session_resume_from_a_checkpoint(env):
    """Particles and step counter of step k are a checkpoint: a filter (or a
    serving session) created from them with first_step = k continues the same
    sequence bit for bit."""
    torch, mcl, (wl, poses, deltas, scans, parts0), m = env
    prm = mcl.sensor_params(sigma_hit=wl.sigma_hit)
    kw = dict(max_points=1024, params=prm, motion_sigma=MOTION_SIGMA, seed=SEED)
    a = mcl.Filter(m, torch.from_numpy(parts0).cuda(), **kw)
    for k in range(3):
        a.step(torch.from_numpy(scans[k]).cuda(), deltas[k])
    mcl.mcl_sync()
    ckpt = a.tensors()["particles"].clone()
    steps = a.state()["steps"]
    b = mcl.Filter(m, ckpt, first_step=steps, **kw)
    for k in range(3, 6):
        a.step(torch.from_numpy(scans[k]).cuda(), deltas[k])
        b.step(torch.from_numpy(scans[k]).cuda(), deltas[k])
    mcl.mcl_sync()
    assert torch.equal(a.tensors()["particles"], b.tensors()["particles"])
    a.close()
    b.close()
    srv = mcl.Server(hbm_budget_bytes=1 << 30, max_sessions=2)
    s1 = srv.open(m, parts0, max_N=1024, sigma_hit=wl.sigma_hit, motion_sigma=MOTION_SIGMA, seed=SEED)
    for k in range(2):
        assert srv.wait(s1.submit(scans[k], deltas[k]), 60_000)["status"] == 0
    cp, _ = s1.read(60_000)
    info = s1.info(60_000)
    assert info["step"] == 2 and info["seed"] == SEED
    s2 = srv.open(m, cp, max_N=1024, sigma_hit=wl.sigma_hit, motion_sigma=MOTION_SIGMA, seed=SEED,
                  first_step=info["step"])
    for k in range(2, 4):
        for s in (s1, s2):
            assert srv.wait(s.submit(scans[k], deltas[k]), 60_000)["status"] == 0
    p1, w1 = s1.read(60_000)
    p2, w2 = s2.read(60_000)
    assert np.array_equal(p1, p2) and np.array_equal(w1, w2)
    s1.close()
    s2.close()
    srv.close()
