"""The C-ABI library builds, loads and exports every entry point that
include/*.h declares; the Python binding's structures match the C layout.
No compute call runs here (no GPU needed)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2310_04172_gb300 import _build
    return _build.build()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(mcl_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mcl_map_create", "mcl_map_destroy", "mcl_sensor_update", "mcl_resample",
                     "mcl_motion_update", "mcl_normalise", "mcl_map_lookup", "mcl_sync"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (mcl_[a-z0-9_]+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    L = ctypes.CDLL(lib_path)
    for n in declared_functions():
        assert getattr(L, n) is not None


def test_binding_covers_every_symbol_and_loads(lib_path):
    from paper_2310_04172_gb300 import mcl
    assert set(declared_functions()) == set(mcl.SIGNATURES)
    assert mcl.lib() is not None and mcl.mcl_version() == 200


def test_struct_layouts_match_c(tmp_path):
    from paper_2310_04172_gb300 import mcl
    src = tmp_path / "sz.c"
    structs = sorted(n for n, v in vars(mcl).items()
                     if n.startswith("mcl_") and isinstance(v, type) and issubclass(v, ctypes.Structure))
    assert len(structs) >= 10
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "mcl.h"', "int main(void){"]
    for s in structs:
        lines.append(f'printf("{s} %zu\\n", sizeof({s}));')
        for f, _ in getattr(mcl, s)._fields_:
            lines.append(f'printf("{s}.{f} %zu\\n", offsetof({s}, {f}));')
    lines.append("return 0;}")
    src.write_text("\n".join(lines))
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                 check=True).stdout.splitlines())
    for s in structs:
        cls = getattr(mcl, s)
        assert int(got[s]) == ctypes.sizeof(cls), s
        for f, _ in cls._fields_:
            assert int(got[f"{s}.{f}"]) == getattr(cls, f).offset, f"{s}.{f}"


def test_library_refuses_to_run_without_build(monkeypatch, tmp_path):
    from paper_2310_04172_gb300 import mcl
    monkeypatch.setattr(mcl, "_lib", None)
    monkeypatch.setattr(mcl, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="no fallback"):
        mcl.lib()


def test_product_path_does_not_reach_the_oracle():
    for f in glob.glob(os.path.join(ROOT, "paper_2310_04172_gb300", "**", "*.*"), recursive=True):
        if f.endswith((".py", ".cu", ".cpp", ".h", ".cuh")):
            text = open(f).read()
            assert "import oracle" not in text and "from oracle" not in text, f
            assert "_oracle.so" not in text and "oracle.c" not in text, f


def test_debug_bounds_build_compiles(tmp_path):
    """The debug variant (slot bounds checks that set the status word instead
    of reading) builds for sm_103a."""
    import shutil
    import subprocess
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = os.path.join(ROOT, "paper_2310_04172_gb300", "csrc", "k_sensor_i16_grid.cu")
    r = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                        "-DMCL_DEBUG_BOUNDS=1", "-I", os.path.join(ROOT, "include"),
                        "-I", os.path.dirname(src), "-c", src, "-o", str(tmp_path / "k.o")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
