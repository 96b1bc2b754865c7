"""The C ABI used from plain C (tests/c/mcl_example.c, compiled with gcc
against include/mcl.h, libmcl.so and the CUDA runtime): the sensor update
with the fused estimate and the resampling give the oracle's results."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
import scenes
from resample_props import check_systematic

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def cuda_home():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))


def test_plain_c_program(tmp_path):
    from paper_2310_04172_gb300 import _build, mcl
    lib = _build.build()
    cuda = cuda_home()
    exe = tmp_path / "mcl_example"
    subprocess.run(["gcc", "-O2", "-std=c11", "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(cuda, "include"), os.path.join(ROOT, "tests", "c", "mcl_example.c"),
                    "-o", str(exe), "-L", os.path.dirname(lib), "-lmcl",
                    "-L", os.path.join(cuda, "lib64"), "-lcudart",
                    "-Wl,-rpath," + os.path.dirname(lib) + ":" + os.path.join(cuda, "lib64")],
                   check=True)
    wl = scenes.room_plain(P=700)
    m = wl.map
    with open(tmp_path / "map.bin", "wb") as f:
        f.write(np.array(m.dims, np.int64).tobytes())
        f.write(np.array([*m.origin, m.voxel, m.tau], np.float32).tobytes())
        f.write(np.ascontiguousarray(m.values, np.float32).tobytes())
    with open(tmp_path / "particles.bin", "wb") as f:
        f.write(np.int64(len(wl.particles)).tobytes() + wl.particles.astype(np.float32).tobytes())
    with open(tmp_path / "scan.bin", "wb") as f:
        f.write(np.int64(len(wl.scan)).tobytes() + wl.scan.astype(np.float32).tobytes())
    r = subprocess.run([str(exe), str(tmp_path)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    raw = (tmp_path / "out.bin").read_bytes()
    P = len(wl.particles)
    logw = np.frombuffer(raw, np.float32, P, 0).astype(np.float64)
    w = np.frombuffer(raw, np.float32, P, 4 * P)
    idx = np.frombuffer(raw, np.int32, P, 8 * P)
    est = mcl.estimate_to_dict(np.frombuffer(raw, np.uint8, mcl.ESTIMATE_BYTES, 12 * P))
    Lo = oracle.sensor_update(oracle.Map.from_scene_map(m), wl.particles, wl.scan, 0.1)
    assert np.max(np.abs(logw - Lo) / np.maximum(1.0, np.abs(Lo))) <= 1e-5
    check_systematic(idx, w, 0.5)          # GPU weights: properties, not the oracle
    # the estimate against the oracle's estimate of its own weights: bounded by
    # the weight difference times the spread of the poses
    wo, *_ = oracle.normalise(Lo)
    eo = oracle.pose_estimate(wl.particles, wo.astype(np.float32))
    dw = np.abs(w.astype(np.float64) - wo).sum()
    spread = np.abs(wl.particles.astype(np.float64) - eo["mean_pose"]).max()
    np.testing.assert_allclose(est["mean_pose"], eo["mean_pose"], rtol=0, atol=2 * dw * spread + 1e-9)
    assert est["argmax"] == eo["argmax"]
