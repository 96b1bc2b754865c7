"""Autotuner: times launch shapes on the caller's data, caches the winner per
(GPU, map, storage type, mode, flags, scan staging, size buckets), and its
shapes keep parity."""
import numpy as np
import pytest

import oracle
import scenes

pytestmark = pytest.mark.gpu


def test_autotune_picks_a_valid_faster_shape_and_caches_it(tmp_path):
    import torch
    from paper_2310_04172_gb300 import _build, mcl
    _build.build()
    torch.cuda.set_device(0)
    wl = scenes.os064_building(P=20000, dtype=scenes.I16)
    m = mcl.map_from_scene(wl.map)
    parts = torch.from_numpy(wl.particles).cuda()
    scan = torch.from_numpy(wl.scan).cuda()
    cache = str(tmp_path / "tune.jsonl")
    base = mcl.sensor_params(0.1)
    best, info = mcl.mcl_autotune(m, parts, scan, base, max_particles=8192, cache_path=cache,
                                  tune_summation=True)
    assert not info["from_cache"] and info["candidates"] >= 8
    assert info["best_ms"] <= info["default_ms"]
    assert open(cache).read().count('"key"') == 1
    best2, info2 = mcl.mcl_autotune(m, parts, scan, base, max_particles=8192, cache_path=cache,
                                    tune_summation=True)
    assert info2["from_cache"] and info2["shape"] == info["shape"]
    # another read (trilinear) or another scan staging is another key: timed, not served
    # (the trilinear read keeps 32 lanes while the summation is tuned)
    for other in (mcl.sensor_params(0.1, flags=mcl.MCL_TRILINEAR), mcl.sensor_params(0.1, scan_rings=64)):
        b3, info3 = mcl.mcl_autotune(m, parts, scan, other, max_particles=4096, cache_path=cache,
                                     tune_summation=True)
        assert not info3["from_cache"] and info3["candidates"] >= 1
        assert b3.flags == other.flags and b3.scan_rings == other.scan_rings
        if other.flags:
            assert b3.lanes_per_particle in (0, 32)
    assert open(cache).read().count('"key"') == 3
    # the tuned shape is a valid shape with parity against the oracle
    P = 2000
    logw = torch.empty(P, device="cuda")
    mcl.mcl_sensor_update(m, parts[:P].contiguous(), scan, best, logw)
    mcl.mcl_sync()
    Lo = oracle.sensor_update(oracle.Map.from_scene_map(wl.map), wl.particles[:P], wl.scan, 0.1)
    err = np.abs(logw.cpu().numpy().astype(np.float64) - Lo) / np.maximum(1, np.abs(Lo))
    assert err.max() <= 1e-5
    m.close()
