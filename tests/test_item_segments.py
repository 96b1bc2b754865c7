"""The batched sensor launch's item order (host code, no GPU): sessions that
read one map are interleaved sweep by sweep, every item exactly once
(tests/c/item_segments_check.cpp, linked against the library)."""
import os
import shutil
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_item_segments(tmp_path):
    from paper_2310_04172_gb300 import _build
    lib = _build.build()
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = tmp_path / "item_segments_check"
    csrc = os.path.join(ROOT, "paper_2310_04172_gb300", "csrc")
    subprocess.run([nvcc, "-std=c++17", "-I", os.path.join(ROOT, "include"), "-I", csrc,
                    os.path.join(ROOT, "tests", "c", "item_segments_check.cpp"), "-o", str(exe),
                    "-L", os.path.dirname(lib), "-lmcl", "-Xlinker", f"-rpath={os.path.dirname(lib)}"],
                   check=True, capture_output=True, text=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout + r.stderr
