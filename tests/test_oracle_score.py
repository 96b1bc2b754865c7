"""Pins of the oracle's score map (Sec. III: the exponential of Eq. 3 is
evaluated once per map entry before the scans, so the sensor update only
sums the stored scores): closed values of the stored score, and the SUM-mode
sensor update on the score map equals the one on the TSDF it came from up to
the FP16 rounding of each score (the latter is pinned by brute force)."""
import math

import numpy as np
import pytest

import oracle
import scenes
from test_oracle_pins import brute_maps


@pytest.fixture
def rng():
    return np.random.default_rng(47)


def test_score_closed_values():
    sig = 0.1
    s32 = float(np.float32(sig))
    d_half = s32 * math.sqrt(2.0 * math.log(2.0))          # exp(-d^2 / 2 sigma^2) = 1/2
    got = oracle.score_of([0.0, -0.0, d_half, -d_half, 1e3], sig)
    assert got.dtype == np.float16
    assert list(got[:4]) == [1.0, 1.0, 0.5, 0.5] and got[4] == 0.0
    d = np.linspace(-0.3, 0.3, 20001)
    sc = oracle.score_of(d, sig).astype(np.float64)
    assert np.all(sc == sc[::-1])                            # even in d
    half = sc[10000:]
    assert np.all(np.diff(half) <= 0)                        # non-increasing in |d|


def scored(m, sigma):
    vals, outside = oracle.score_map(m, sigma)
    import dataclasses
    sm = dataclasses.replace(m, values=vals, dtype=scenes.F16)
    return oracle.Map.from_scene_map(sm).set_outside(outside)


@pytest.mark.parametrize("dtype", [scenes.F32, scenes.F16, scenes.I16])
@pytest.mark.parametrize("neglect", [False, True])
def test_score_map_sum_equals_tsdf_sum(rng, dtype, neglect):
    dense, brick = brute_maps(rng, dtype)
    centre = np.array([0.8, 0.7, 0.6])
    poses = np.concatenate([centre + rng.normal(0, 0.6, (40, 3)),
                            rng.uniform(-math.pi, math.pi, (40, 3))], 1).astype(np.float32)
    dirs = rng.normal(size=(300, 3))
    scan = (dirs / np.linalg.norm(dirs, axis=1, keepdims=True) *
            rng.uniform(0.2, 1.5, (300, 1))).astype(np.float32)
    for m in (dense, brick):
        for sigma in (0.1, 0.05):
            L_tsdf = oracle.sensor_update(oracle.Map.from_scene_map(m), poses, scan, sigma, oracle.SUM,
                                          neglect)
            L_score = oracle.sensor_update(scored(m, sigma), poses, scan, sigma, oracle.SCORE, neglect)
            fin = np.isfinite(L_tsdf)
            assert np.array_equal(fin, np.isfinite(L_score))
            # every term carries at most a relative FP16 rounding of 2^-11
            # (plus the FP16 subnormal step for tiny scores at sigma = 0.05)
            tol = math.log1p(2.0 ** -11) + 1e-12
            err = np.abs(L_score[fin] - L_tsdf[fin])
            if sigma == 0.1:
                assert err.max() <= tol
            else:
                k = 1 / math.sqrt(2 * math.pi * float(np.float32(sigma)) ** 2)
                bound = np.log1p(2.0 ** -11 + len(scan) * 2.0 ** -25 * k / np.exp(L_tsdf[fin]))
                assert np.all(err <= bound + 1e-12)
