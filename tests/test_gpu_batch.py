"""Batched step (one persistent sensor kernel per group of sessions whose maps
share geometry, over (session, chunk, particle block) items of uneven size;
one launch per side step for all sessions): every session's log-weights,
weights and resampled indices (and pose estimates) are identical, bit for bit,
to the single-session calls with the same chunk and lane split and the same
ring count of the scan (staged in 4 x 8 patches, or as given) — alone or in
the mix, plain or replayed from a CUDA graph — and the launches of a step do
not grow with the number of sessions."""
import numpy as np
import pytest

import oracle
import scenes
from resample_props import check_systematic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2310_04172_gb300 import _build, mcl
    _build.build()
    mcl.lib()
    torch.cuda.set_device(0)
    room = scenes.room_plain(P=1000)
    hall = scenes.vlp16_multiroom(P=3000, dtype=scenes.F16)
    bld = scenes.os064_building(P=5000, dtype=scenes.I16)
    room_i16 = scenes.voxelize_bricks(room.scene, (0, 0, 0), 0.05, (128, 128, 64), 0.3, scenes.I16)
    maps = {"room": mcl.map_from_scene(room.map), "room_i16": mcl.map_from_scene(room_i16),
            "hall": mcl.map_from_scene(hall.map), "bld": mcl.map_from_scene(bld.map)}
    yield torch, mcl, room, hall, bld, maps
    for m in maps.values():
        m.close()


def make_sessions(torch, room, hall, bld, maps, rng):
    def t(a):
        return torch.from_numpy(np.ascontiguousarray(a)).cuda()

    # scan rings: 16 for the VLP-16 scans, 64 for OS0-64, 0 for points as
    # given; 777 points of 16 rings do not fit the patches (staged as given)
    specs = [
        ("room", room.particles, room.scan, 0, True, 16),
        ("room_i16", room.particles[:700], room.scan, 0, False, 0),
        ("hall", hall.particles, hall.scan, 0, True, 16),
        ("bld", bld.particles, bld.scan, 0, True, 64),
        ("room", room.particles[::-1].copy(), room.scan[:777], 0, False, 16),   # same map, ragged N
        ("room", room.particles[:333], room.scan, 1, True, 0),                  # SUM mode: own group
    ]
    sessions = []
    for name, parts, scan, mode, res, rings in specs:
        P = len(parts)
        s = {"map": maps[name], "particles": t(parts), "scan": t(scan), "sigma_hit": 0.1,
             "mode": mode, "logw": torch.empty(P, device="cuda"), "w": torch.empty(P, device="cuda"),
             "scan_rings": rings}
        if res:
            s["resample_idx"] = torch.empty(P, dtype=torch.int32, device="cuda")
            s["particles_out"] = torch.empty((P, 6), device="cuda")
        sessions.append(s)
    return sessions


def single(torch, mcl, s, r, chunk, lanes):
    P = s["particles"].shape[0]
    logw, w = torch.empty(P, device="cuda"), torch.empty(P, device="cuda")
    prm = mcl.sensor_params(s["sigma_hit"], mode=s["mode"], points_per_chunk=chunk,
                            lanes_per_particle=lanes, scan_rings=s.get("scan_rings", 0))
    if "estimate" in s:
        est = mcl.estimate_buffer()
        mcl.mcl_sensor_update_estimate(s["map"], s["particles"], s["scan"], prm, logw, w, est)
    else:
        mcl.mcl_sensor_update(s["map"], s["particles"], s["scan"], prm, logw, w)
    out = [logw.cpu().numpy(), w.cpu().numpy()]
    if "resample_idx" in s:
        idx = torch.empty(P, dtype=torch.int32, device="cuda")
        po = torch.empty((P, 6), device="cuda")
        mcl.mcl_resample(w, r, idx, s["particles"], po)
        out += [idx.cpu().numpy(), po.cpu().numpy()]
    if "estimate" in s:
        out.append(est.cpu().numpy())
    mcl.mcl_sync()
    return out


def batch_outputs(s):
    out = [s["logw"].cpu().numpy(), s["w"].cpu().numpy()]
    if "resample_idx" in s:
        out += [s["resample_idx"].cpu().numpy(), s["particles_out"].cpu().numpy()]
    if "estimate" in s:
        out.append(s["estimate"].cpu().numpy())
    return out


@pytest.mark.parametrize("use_graph", [False, True])
@pytest.mark.parametrize("chunk,lanes,item_order", [(2048, 32, 0), (1024, 16, 0), (2048, 32, 1),
                                                     (2048, 32, 3)])
def test_batch_matches_single_sessions(env, use_graph, chunk, lanes, item_order):
    torch, mcl, room, hall, bld, maps = env
    rng = np.random.default_rng(11)
    sessions = make_sessions(torch, room, hall, bld, maps, rng)
    for k in (0, 3, 4):  # pose estimates fused into the batched normalisation
        sessions[k]["estimate"] = mcl.estimate_buffer()
    b = mcl.Batch(sessions, points_per_chunk=chunk, lanes_per_particle=lanes, use_graph=use_graph,
                  item_order=item_order)
    info = b.info()
    assert info["n_sessions"] == 6 and info["n_groups"] == 5  # two sessions share the room group
    for run in range(2):
        r = rng.uniform(0, 1, len(sessions))
        if run == 1:  # new particles in the same buffers, as a filter step would write them
            for s in sessions:
                s["particles"][:, :3] += 0.05 * torch.randn_like(s["particles"][:, :3])
        b.set_offsets(r)
        b.run()
        mcl.mcl_sync()
        for k, s in enumerate(sessions):
            got = batch_outputs(s)
            ref = single(torch, mcl, s, float(r[k]), chunk, lanes)
            for g, e in zip(got, ref):
                assert np.array_equal(g, e), f"session {k} run {run}"
    assert b.info()["graph_captured"] == int(use_graph)
    b.close()


def test_batch_shares_launches_across_maps(env):
    """Sessions on two different building maps of one geometry (different
    seeds) form one group: one sensor launch reads each session's own map.
    The step's launches are the same for 1, 2, 4 and 8 sessions, and every
    session equals its single call bit for bit, whether its scan is staged in
    4 x 8 patches or as given (both in one group)."""
    torch, mcl, room, hall, bld, maps = env
    b1 = scenes.os064_building(P=3000, dtype=scenes.I16, seed=21, size=80.0, floors=2)
    b2 = scenes.os064_building(P=3000, dtype=scenes.I16, seed=22, size=80.0, floors=2)
    m1, m2 = mcl.map_from_scene(b1.map), mcl.map_from_scene(b2.map)
    rng = np.random.default_rng(5)
    counts = []
    for S in (1, 2, 4, 8):
        sessions = []
        for k in range(S):
            m, wl = (m1, b1) if k % 2 == 0 else (m2, b2)
            P = 500 + 300 * k
            parts = torch.from_numpy(np.ascontiguousarray(wl.particles[:P])).cuda()
            s = {"map": m, "particles": parts, "scan": torch.from_numpy(wl.scan).cuda(),
                 "sigma_hit": 0.1, "mode": 0, "logw": torch.empty(P, device="cuda"),
                 "w": torch.empty(P, device="cuda"),
                 "resample_idx": torch.empty(P, dtype=torch.int32, device="cuda"),
                 "particles_out": torch.empty((P, 6), device="cuda"),
                 "scan_rings": 64 if k % 4 < 2 else 0}
            if k % 3 == 0:
                s["estimate"] = mcl.estimate_buffer()
            sessions.append(s)
        b = mcl.Batch(sessions, use_graph=(S % 4 == 0))
        info = b.info()
        assert info["n_groups"] == 1
        counts.append(info["kernels_per_run"])
        r = rng.uniform(0, 1, S)
        b.set_offsets(r)
        b.run()
        mcl.mcl_sync()
        for k, s in enumerate(sessions):
            ref = single(torch, mcl, s, float(r[k]), 0, 0)
            for g, e in zip(batch_outputs(s), ref):
                assert np.array_equal(g, e), f"S={S} session {k}"
        b.close()
    assert len(set(counts)) == 1, counts
    m1.close()
    m2.close()


def test_batch_against_oracle(env):
    torch, mcl, room, hall, bld, maps = env
    sessions = make_sessions(torch, room, hall, bld, maps, np.random.default_rng(3))
    b = mcl.Batch(sessions)
    b.set_offsets(np.full(len(sessions), 0.5))
    b.run()
    mcl.mcl_sync()
    for s, wl in ((sessions[0], room), (sessions[2], hall)):
        L = oracle.sensor_update(oracle.Map.from_scene_map(wl.map), wl.particles, wl.scan, 0.1)
        Lg = s["logw"].cpu().numpy().astype(np.float64)
        assert np.max(np.abs(Lg - L) / np.maximum(1, np.abs(L))) <= 1e-5
        check_systematic(s["resample_idx"].cpu().numpy(), s["w"].cpu().numpy(), 0.5)
    b.close()


def test_batch_rejects_bad_sessions(env):
    torch, mcl, room, hall, bld, maps = env
    parts = torch.from_numpy(room.particles).cuda()
    scan = torch.from_numpy(room.scan).cuda()
    ok = {"map": maps["room"], "particles": parts, "scan": scan, "logw": torch.empty(1000, device="cuda")}
    with pytest.raises(mcl.MclError):   # resampling needs the normalised weights
        mcl.Batch([dict(ok, resample_idx=torch.empty(1000, dtype=torch.int32, device="cuda"))])
    with pytest.raises(mcl.MclError):   # no output at all
        mcl.Batch([{"map": maps["room"], "particles": parts, "scan": scan}])
    with pytest.raises(mcl.MclError):
        mcl.Batch([dict(ok, sigma_hit=-1.0)])
    with pytest.raises(mcl.MclError):
        mcl.Batch([dict(ok, scan_rings=-4)])
    b = mcl.Batch([ok])
    with pytest.raises(mcl.MclError):
        b.set_offsets([1.0])
    b.close()
