"""mcl_resample_noalloc: systematic resampling that allocates no device memory.

Some callers may not allocate: a real-time robot control loop that forbids
allocation after start-up (cudaMalloc and cudaFree can block, and cudaFree
synchronises the device), or a plug-in whose host application owns every
device allocation. For them the library keeps the resampling scratch in a
static device array (at most 2^20 particles). This test calls the entry point
through the C ABI and checks it against mcl_resample, bit for bit, on calls
in a row, the last at the array's limit of 2^20 particles (every tile entry
of the scratch in use); it runs last so that a failure here leaves every
other test already run.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _inputs(rng, P):
    import torch
    w = rng.exponential(1.0, P) ** 3
    w[rng.random(P) < 0.1] = 0.0
    w[0] = max(w[0], 1e-3)
    w32 = (w / w.sum()).astype(np.float32)
    parts = rng.normal(size=(P, 6)).astype(np.float32)
    return torch.from_numpy(w32).cuda(), torch.from_numpy(parts).cuda()


def test_resample_noalloc_matches_resample_twice():
    import torch
    from paper_2310_04172_gb300 import _build, mcl
    _build.build()
    L = mcl.lib()
    torch.cuda.set_device(0)
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rng = np.random.default_rng(2024)
    for call, (P, r) in enumerate([(1_000_000, 0.37), (4097, 0.81), (1 << 20, 0.52)]):
        w, parts = _inputs(rng, P)
        idx_ref = torch.empty(P, dtype=torch.int32, device="cuda")
        out_ref = torch.empty_like(parts)
        idx_new = torch.full((P,), -1, dtype=torch.int32, device="cuda")
        out_new = torch.zeros_like(parts)
        assert L.mcl_resample(w.data_ptr(), P, r, idx_ref.data_ptr(), parts.data_ptr(),
                              out_ref.data_ptr(), s) == mcl.MCL_OK
        assert L.mcl_sync(s) == mcl.MCL_OK
        free_before = torch.cuda.mem_get_info()[0]
        assert L.mcl_resample_noalloc(w.data_ptr(), P, r, idx_new.data_ptr(), parts.data_ptr(),
                                      out_new.data_ptr(), s) == mcl.MCL_OK, \
            L.mcl_last_error().decode()
        assert L.mcl_sync(s) == mcl.MCL_OK
        assert torch.equal(idx_new, idx_ref), f"call {call}: indices differ"
        assert torch.equal(out_new, out_ref), f"call {call}: gathered particles differ"
        if call > 0:  # after the per-device set-up of the first call, nothing is allocated
            assert torch.cuda.mem_get_info()[0] == free_before


def test_resample_noalloc_refuses_sizes_beyond_its_array():
    import torch
    from paper_2310_04172_gb300 import _build, mcl
    _build.build()
    L = mcl.lib()
    torch.cuda.set_device(0)
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    P = (1 << 20) + 1
    w = torch.full((P,), 1.0 / P, device="cuda")
    idx = torch.empty(P, dtype=torch.int32, device="cuda")
    assert L.mcl_resample_noalloc(w.data_ptr(), P, 0.5, idx.data_ptr(), None, None, s) == mcl.MCL_EINVAL
    assert b"static scratch limit" in L.mcl_last_error()
    assert L.mcl_sync(s) == mcl.MCL_OK
