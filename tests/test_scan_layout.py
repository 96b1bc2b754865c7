"""The scan staging order and pair layout (host code, no GPU): 4-ring x
8-point patches of a ring-major scan as a bijection, the rule that decides
when a ring count applies, and the pair layout's sizes
(tests/c/scan_layout_check.cpp, compiled against the library's headers)."""
import os
import shutil
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_scan_layout(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = tmp_path / "scan_layout_check"
    csrc = os.path.join(ROOT, "paper_2310_04172_gb300", "csrc")
    subprocess.run([nvcc, "-std=c++17", "-I", os.path.join(ROOT, "include"), "-I", csrc,
                    os.path.join(ROOT, "tests", "c", "scan_layout_check.cpp"), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout + r.stderr


def test_host_patch_order_matches_the_definition():
    """The host permutation the GPU parity test stages its reference scan
    with (a reshape and transpose) is the patch order written as nested loops
    (band of 4 rings, patch of 8 points along them, ring, point), so that test
    compares the kernel's staging with the definition."""
    import numpy as np
    from test_gpu_parity import patch_order
    for R, A in ((4, 8), (8, 16), (12, 24), (16, 64), (64, 1024)):
        want = [(band * 4 + ring) * A + col * 8 + a
                for band in range(R // 4) for col in range(A // 8) for ring in range(4) for a in range(8)]
        assert np.array_equal(patch_order(R * A, R), np.array(want))
