"""The cell-grid index addresses at most 2^20 bricks (its kernels form value
indices slot * 4096 + offset in 32 bits). At exactly 2^20 bricks the grid is
used and the last brick's values read correctly; one brick more and the
automatic choice is the hash index, while an explicit grid request is EINVAL.

Expected values come from the definition (LOGPROD log-weight of one particle
at the identity pose whose points sit at voxel centres of the last brick:
L = -1/(2 sigma^2) * sum d^2 with d = q * tau / 32767), not from the GPU."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TAU, VOXEL, SIGMA = 0.3, 0.05, 0.1


def _make(mcl, n_bricks, index):
    nbx, nby, nbz = 128, 128, 65                      # 1,064,960 brick cells
    cells = np.arange(n_bricks, dtype=np.int64)
    coords = np.stack([cells % nbx, (cells // nbx) % nby, cells // (nbx * nby)], 1).astype(np.int32)
    values = np.zeros(n_bricks * 4096, np.int16)      # zero pages until written
    last = values[(n_bricks - 1) * 4096:]
    q = (np.arange(4096, dtype=np.int64) * 7919 % 60001 - 30000).astype(np.int16)
    last[:] = q
    m = mcl.mcl_map_create(mcl.MCL_MAP_BRICK, mcl.MCL_I16, (0.0, 0.0, 0.0), np.float32(VOXEL),
                           np.float32(TAU), (16 * nbx, 16 * nby, 16 * nbz), values, coords,
                           index=index)
    return m, coords[-1], q


def _last_brick_logw(torch, mcl, m, bc, q):
    # 256 voxel centres of the last brick (every 16th voxel), one particle at the identity pose
    local = np.arange(0, 4096, 16)
    lx, ly, lz = local % 16, (local // 16) % 16, local // 256
    ix, iy, iz = 16 * bc[0] + lx, 16 * bc[1] + ly, 16 * bc[2] + lz
    pts = ((np.stack([ix, iy, iz], 1) + 0.5) * VOXEL).astype(np.float32)
    parts = np.zeros((1, 6), np.float32)
    logw = torch.empty(1, device="cuda")
    mcl.mcl_sensor_update(m, torch.from_numpy(parts).cuda(), torch.from_numpy(pts).cuda(),
                          mcl.sensor_params(SIGMA), logw)
    mcl.mcl_sync()
    d = q[local].astype(np.float64) * (TAU / 32767.0)
    expect = -0.5 / SIGMA ** 2 * np.sum(d * d)
    return float(logw.cpu().numpy()[0]), expect


def test_grid_index_brick_limit():
    import torch
    from paper_2310_04172_gb300 import _build, mcl
    _build.build()
    torch.cuda.set_device(0)
    m, bc, q = _make(mcl, 1 << 20, mcl.MCL_INDEX_AUTO)
    assert m.info()["index"] == mcl.MCL_INDEX_GRID
    got, expect = _last_brick_logw(torch, mcl, m, bc, q)
    assert abs(got - expect) <= 1e-5 * max(1.0, abs(expect))
    m.close()
    m, bc, q = _make(mcl, (1 << 20) + 1, mcl.MCL_INDEX_AUTO)
    assert m.info()["index"] == mcl.MCL_INDEX_HASH
    got, expect = _last_brick_logw(torch, mcl, m, bc, q)
    assert abs(got - expect) <= 1e-5 * max(1.0, abs(expect))
    m.close()
    with pytest.raises(mcl.MclError) as e:
        _make(mcl, (1 << 20) + 1, mcl.MCL_INDEX_GRID)
    assert e.value.status == mcl.MCL_EINVAL
