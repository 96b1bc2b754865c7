"""Serving loop: sessions resident on the device, admission by budget and slot
count, latest-scan-wins queues, continuous batching; a session's result is the
same alone and in the mix, and matches the oracle."""
import threading
import time

import numpy as np
import pytest

import oracle
from resample_props import check_systematic
import scenes

pytestmark = pytest.mark.gpu

MASK = (1 << 64) - 1


def offset_of(seed: int, step: int) -> float:
    """The server's resampling offset for (seed, step): SplitMix64 finaliser."""
    z = (seed ^ ((step * 0x9E3779B97F4A7C15) & MASK)) & MASK
    z = (z + 0x9E3779B97F4A7C15) & MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    z ^= z >> 31
    return (z >> 11) * 2.0 ** -53


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2310_04172_gb300 import _build, mcl
    _build.build()
    mcl.lib()
    torch.cuda.set_device(0)
    room = scenes.room_plain(P=1000)
    hall = scenes.vlp16_multiroom(P=4000, dtype=scenes.F16)
    bld = scenes.os064_building(P=6000, dtype=scenes.I16)
    maps = {"room": mcl.map_from_scene(room.map), "hall": mcl.map_from_scene(hall.map),
            "bld": mcl.map_from_scene(bld.map)}
    yield mcl, room, hall, bld, maps
    for m in maps.values():
        m.close()


def test_same_alone_and_in_the_mix_and_against_the_oracle(env):
    mcl, room, hall, bld, maps = env
    seed = 1234
    alone = mcl.Server(4 << 30, 8)
    s = alone.open(maps["room"], room.particles, 2048, seed=seed)
    t = s.submit(room.scan)
    res = alone.wait(t, 10_000)
    assert res["status"] == mcl.MCL_RESULT_DONE and res["evals"] == 1000 * 1024
    parts_alone, w_alone = s.read()
    alone.close()

    mix = mcl.Server(8 << 30, 8, max_in_flight=2)
    mix.pause(True)
    others = [mix.open(maps["hall"], hall.particles, 28800, seed=5),
              mix.open(maps["bld"], bld.particles, 65536, seed=6),
              mix.open(maps["room"], room.particles[::-1].copy(), 2048, seed=7)]
    s2 = mix.open(maps["room"], room.particles, 2048, seed=seed)
    tickets = [o.submit(sc) for o, sc in zip(others, (hall.scan, bld.scan, room.scan[:900]))]
    t2 = s2.submit(room.scan)
    mix.pause(False)
    for tk in tickets:
        assert mix.wait(tk, 30_000)["status"] == mcl.MCL_RESULT_DONE
    res2 = mix.wait(t2, 30_000)
    assert res2["status"] == mcl.MCL_RESULT_DONE
    parts_mix, w_mix = s2.read()
    # the step's pose estimate: that of its input particles with its weights
    import torch
    ref = mcl.estimate_buffer()
    mcl.mcl_pose_estimate(torch.from_numpy(room.particles).cuda(), torch.from_numpy(w_mix).cuda(), ref)
    mcl.mcl_sync()
    want = mcl.estimate_to_dict(ref)
    for key in ("mean_pose", "quat", "rpy"):
        assert np.array_equal(res2["estimate"][key], want[key])
    assert res2["estimate"]["argmax"] == want["argmax"]
    assert mix.stats()["mean_batch_sessions"] == 4.0  # all four went as one batched step
    assert np.array_equal(parts_alone, parts_mix) and np.array_equal(w_alone, w_mix)
    # against the oracle: weights of the step's input, then systematic resampling
    L = oracle.sensor_update(oracle.Map.from_scene_map(room.map), room.particles, room.scan, 0.1)
    wo, M, _, _ = oracle.normalise(L)
    sel = wo >= 1e-30
    assert abs(w_mix.astype(np.float64).sum() - 1) <= 1e-5
    bound = 1e-5 * (np.maximum(1, np.abs(L[sel])) + max(1, abs(M)))
    assert np.all(np.abs(np.log(w_mix[sel].astype(np.float64)) - np.log(wo[sel])) <= bound)
    # the resampled set: rows of the input drawn systematically by the weights
    rows = {r.tobytes(): i for i, r in enumerate(room.particles)}
    idx = np.array([rows[r.tobytes()] for r in parts_mix])
    order = np.argsort(idx, kind="stable")
    check_systematic(idx[order], w_mix, offset_of(seed, 0))
    mix.close()


def test_continuous_batching_under_load(env):
    mcl, room, hall, bld, maps = env
    srv = mcl.Server(16 << 30, 16, max_in_flight=2)
    rng = np.random.default_rng(0)
    sess = []
    for k in range(12):
        if k % 3 == 0:
            sess.append((srv.open(maps["bld"], bld.particles[: 1000 + 400 * k], 65536, seed=k), bld.scan))
        elif k % 3 == 1:
            sess.append((srv.open(maps["hall"], hall.particles[: 500 + 300 * k], 28800, seed=k), hall.scan))
        else:
            sess.append((srv.open(maps["room"], room.particles, 2048, seed=k), room.scan))
    stop = time.time() + 2.0
    results, lock = [], threading.Lock()

    def client(session, scan, seed):
        r = np.random.default_rng(seed)
        while time.time() < stop:
            t = session.submit(scan, delta=[0.01, 0, 0, 0, 0, 0.001])
            res = srv.wait(t, 20_000)
            with lock:
                results.append(res["status"])
            time.sleep(r.exponential(0.01))

    th = [threading.Thread(target=client, args=(s, sc, i)) for i, (s, sc) in enumerate(sess)]
    for x in th:
        x.start()
    for x in th:
        x.join()
    st = srv.stats()
    assert st["completed"] >= 24 and all(r == mcl.MCL_RESULT_DONE for r in results)
    assert st["mean_batch_sessions"] > 1.0       # scans of several sessions share steps
    assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
    assert st["evals_per_s"] > 0 and st["sessions"] == 12
    srv.close()


def test_admission_supersede_timeout_and_close(env):
    mcl, room, hall, bld, maps = env
    srv = mcl.Server(1 << 30, 2, max_in_flight=2)
    a = srv.open(maps["room"], room.particles, 2048, seed=1)
    b = srv.open(maps["room"], room.particles, 2048, seed=2)
    with pytest.raises(mcl.MclError) as e:               # no slot left
        srv.open(maps["room"], room.particles, 2048)
    assert e.value.status == mcl.MCL_EBUSY
    b.close()
    with pytest.raises(mcl.MclError) as e:               # over the device-memory budget
        srv.open(maps["bld"], np.tile(bld.particles, (1000, 1)), 65536)
    assert e.value.status == mcl.MCL_ENOMEM
    srv.pause(True)
    t1 = a.submit(room.scan)
    t2 = a.submit(room.scan[:512])                       # supersedes t1 (not started)
    assert srv.wait(t1, 1000)["status"] == mcl.MCL_RESULT_SUPERSEDED
    with pytest.raises(mcl.MclError) as e:               # held scheduler: the wait runs out
        srv.wait(t2, 50)
    assert e.value.status == mcl.MCL_ETIMEDOUT
    srv.pause(False)
    r = srv.wait(t2, 10_000)
    assert r["status"] == mcl.MCL_RESULT_DONE and r["evals"] == 1000 * 512
    srv.pause(True)
    t3 = a.submit(room.scan)
    a.close()                                            # queued scan completes as closed
    assert srv.wait(t3, 1000)["status"] == mcl.MCL_RESULT_CLOSED
    with pytest.raises(mcl.MclError):
        srv.wait(12345678, 0)                            # unknown ticket
    srv.close()


def _compose(a, b):
    """Body-frame increment a then b, FP64 (t = t_a + R_a t_b, R = R_a R_b)."""
    def rot(r, p, y):
        cr, sr, cp, sp, cy, sy = np.cos(r), np.sin(r), np.cos(p), np.sin(p), np.cos(y), np.sin(y)
        return np.array([[cy * cp, cy * sp * sr - sy * cr, cy * sp * cr + sy * sr],
                         [sy * cp, sy * sp * sr + cy * cr, sy * sp * cr - cy * sr],
                         [-sp, cp * sr, cp * cr]])
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    A, B = rot(*a[3:]), rot(*b[3:])
    C = A @ B
    t = a[:3] + A @ b[:3]
    ang = [np.arctan2(C[2, 1], C[2, 2]), np.arcsin(np.clip(-C[2, 0], -1, 1)), np.arctan2(C[1, 0], C[0, 0])]
    return np.concatenate([t, ang]).astype(np.float32)


def test_superseded_odometry_is_composed(env):
    """A superseded scan's odometry increment is not lost: the step that runs
    moves the particles by both increments, composed."""
    import torch
    mcl, room, hall, bld, maps = env
    sig = [0.01, 0.01, 0.005, 0.002, 0.002, 0.005]
    d1 = np.float32([0.1, 0.0, 0.0, 0.0, 0.0, 0.3])
    d2 = np.float32([0.05, 0.02, 0.0, 0.0, 0.0, 0.1])
    srv = mcl.Server(1 << 30, 2, max_in_flight=2)
    ss = srv.open(maps["room"], room.particles, 2048, sigma_hit=room.sigma_hit, motion_sigma=sig, seed=9)
    srv.pause(True)
    t1 = ss.submit(room.scan, d1)
    t2 = ss.submit(room.scan, d2)                        # supersedes t1
    srv.pause(False)
    assert srv.wait(t1, 10_000)["status"] == mcl.MCL_RESULT_SUPERSEDED
    r = srv.wait(t2, 10_000)
    assert r["status"] == mcl.MCL_RESULT_DONE
    scan = torch.from_numpy(room.scan).cuda()
    prm = mcl.sensor_params(room.sigma_hit)
    got = r["estimate"]["mean_pose"]
    for delta, same in ((_compose(d1, d2), True), (d2, False)):
        f = mcl.Filter(maps["room"], torch.from_numpy(room.particles).cuda(), max_points=2048, params=prm,
                       motion_sigma=sig, seed=9, use_graph=False)
        est = mcl.estimate_buffer()
        f.step(scan, delta, est)
        mcl.mcl_sync()
        ref = mcl.estimate_to_dict(est)["mean_pose"]
        if same:
            np.testing.assert_allclose(got, ref, rtol=0, atol=1e-5)
        else:
            assert np.abs(np.asarray(got[:3]) - np.asarray(ref[:3])).max() > 0.05
        f.close()
    ss.close()
    srv.close()


def test_score_map_and_trilinear_sessions_match_single_calls(env):
    """Sessions on a score map (SUM) and with the trilinear read, served in one
    batch beside a plain session: each session's weights equal the single
    call's bit for bit."""
    import torch
    mcl, room, hall, bld, maps = env
    sc = mcl.mcl_map_create_score(maps["room"], 0.1)
    parts = torch.from_numpy(room.particles).cuda()
    scan = torch.from_numpy(room.scan).cuda()
    singles = []
    for m, mode, flags in ((sc, mcl.MCL_SUM, 0), (maps["room"], mcl.MCL_LOGPROD, mcl.MCL_TRILINEAR),
                           (maps["room"], mcl.MCL_LOGPROD, 0)):
        w = torch.empty(1000, device="cuda")
        mcl.mcl_sensor_update(m, parts, scan, mcl.sensor_params(0.1, mode=mode, flags=flags), None, w)
        singles.append(w.cpu().numpy())
    srv = mcl.Server(8 << 30, 4)
    srv.pause(True)
    sessions = [srv.open(sc, room.particles, 2048, mode=mcl.MCL_SUM, seed=1),
                srv.open(maps["room"], room.particles, 2048, flags=mcl.MCL_TRILINEAR, seed=2),
                srv.open(maps["room"], room.particles, 2048, seed=3)]
    tickets = [s.submit(room.scan) for s in sessions]
    srv.pause(False)
    for t in tickets:
        assert srv.wait(t, 30_000)["status"] == mcl.MCL_RESULT_DONE
    assert srv.stats()["mean_batch_sessions"] == 3.0
    for s, ref in zip(sessions, singles):
        _, w = s.read()
        assert np.array_equal(w, ref)
        s.close()
    srv.close()
    sc.close()


def test_scan_rings_by_each_scans_own_size(env):
    """A session opened with the scan's ring count stages each submitted scan
    in 4 x 8 patches by that scan's own size (1,024 points of 16 rings, 512 of
    16 rings of 32, and 900, which does not fit and is staged as given): each
    step's weights equal the single call's with the same ring count, bit for
    bit, and the 1,024-point step differs from the points-as-given session."""
    import torch
    mcl, room, hall, bld, maps = env
    parts = torch.from_numpy(room.particles).cuda()
    cases = (room.scan, np.ascontiguousarray(room.scan[:512]), np.ascontiguousarray(room.scan[:900]))
    singles = []
    for scan in cases:
        w = torch.empty(1000, device="cuda")
        mcl.mcl_sensor_update(maps["room"], parts, torch.from_numpy(scan).cuda(),
                              mcl.sensor_params(0.1, scan_rings=16), None, w)
        singles.append(w.cpu().numpy())
    srv = mcl.Server(8 << 30, 8)
    srv.pause(True)
    sessions = [srv.open(maps["room"], room.particles, 2048, seed=10 + k, scan_rings=16) for k in range(3)]
    given = srv.open(maps["room"], room.particles, 2048, seed=20)
    tickets = [s.submit(sc) for s, sc in zip(sessions, cases)] + [given.submit(room.scan)]
    srv.pause(False)
    for t in tickets:
        assert srv.wait(t, 30_000)["status"] == mcl.MCL_RESULT_DONE
    for s, ref in zip(sessions, singles):
        _, w = s.read()
        assert np.array_equal(w, ref)
    _, w_given = given.read()
    assert not np.array_equal(w_given, singles[0])
    for s in sessions + [given]:
        s.close()
    with pytest.raises(mcl.MclError):
        srv.open(maps["room"], room.particles, 2048, scan_rings=-16)
    srv.close()
