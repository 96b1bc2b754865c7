"""Failure detection on the GPU without a fault: a CTA waits, with the
sensor kernel's bounded wait, on a barrier phase that nothing completes. The
wait must give up after about a second, the timeout must reach the host
through the device status word, and the context must stay usable (a sensor
update afterwards still matches the oracle)."""
import numpy as np
import pytest

import oracle
import scenes

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2310_04172_gb300 import _build, mcl
    _build.build()
    torch.cuda.set_device(0)
    waited = mcl.mcl_selftest_wait()
    assert 0.5 <= waited <= 5.0, f"waited {waited:.3f} s"
    mcl.mcl_sync()                          # the status word was cleared
    wl = scenes.room_plain(P=200)
    m = mcl.map_from_scene(wl.map)
    logw = torch.empty(200, device="cuda")
    mcl.mcl_sensor_update(m, torch.from_numpy(wl.particles).cuda(), torch.from_numpy(wl.scan).cuda(),
                          mcl.sensor_params(wl.sigma_hit), logw)
    mcl.mcl_sync()
    Lo = oracle.sensor_update(oracle.Map.from_scene_map(wl.map), wl.particles, wl.scan, wl.sigma_hit)
    Lg = logw.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(Lg - Lo) / np.maximum(1.0, np.abs(Lo))) <= 1e-5
    m.close()
