"""The oracle's whole filter (Sec. III: motion update, sensor update,
normalisation, pose estimate, resampling, step after step) tracks a seeded
robot path through the synthetic room: starting 0.33 m and 8 degrees off, the
weighted estimate reaches the true pose. This pins the composition of the
oracle's steps (a wrong sign in the motion composition, a transposed rotation
or a resampling that ignores the weights would leave the estimate off the
path)."""
import math

import numpy as np
import pytest

import oracle
import scenes

MOTION_SIGMA = np.array([0.02, 0.02, 0.01, 0.005, 0.005, 0.01], np.float32)


def splitmix_offset(seed: int, step: int) -> float:
    """Resampling offset of a filter step: the SplitMix64 finaliser (Steele,
    Lea, Flood, OOPSLA 2014) of seed ^ step * golden-ratio increment, 53 bits."""
    m = (1 << 64) - 1
    z = (seed ^ (step * 0x9E3779B97F4A7C15)) & m
    z = (z + 0x9E3779B97F4A7C15) & m
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
    z ^= z >> 31
    return (z >> 11) * 2.0 ** -53


def tracking_case(steps=40, P=2000):
    wl = scenes.room_plain(P=1000)
    poses, deltas = scenes.trajectory(wl.scene, wl.pose, steps, seed=5)
    kw = dict(scenes.VLP16, azimuths=64, rmax=30.0)
    scans = scenes.trajectory_scans(wl.scene, poses[1:], kw, seed=9)
    start = poses[0] + np.array([0.25, -0.2, 0.05, 0.0, 0.0, math.radians(8.0)])
    parts = scenes.particles_gaussian(start, P, 0.3, 6.0, 77)
    return wl, poses, deltas, scans, parts


def errors(est, truth):
    dt = float(np.linalg.norm(est["mean_pose"][:3] - truth[:3]))
    dyaw = (est["rpy"][2] - truth[5] + math.pi) % (2 * math.pi) - math.pi
    return dt, abs(math.degrees(dyaw))


def test_oracle_filter_tracks_the_path():
    wl, poses, deltas, scans, parts = tracking_case()
    om = oracle.Map.from_scene_map(wl.map)
    errs = []
    for k in range(len(deltas)):
        parts = oracle.motion_update(parts, deltas[k], MOTION_SIGMA, 123, k)
        L = oracle.sensor_update(om, parts, scans[k], wl.sigma_hit)
        w, *_ = oracle.normalise(L)
        w32 = w.astype(np.float32)
        errs.append(errors(oracle.pose_estimate(parts, w32), poses[k + 1]))
        idx, _ = oracle.resample(w32, splitmix_offset(123, k))
        parts = parts[idx]
    errs = np.array(errs)
    assert errs[0, 0] > 0.1                       # it starts off the path
    assert errs[-10:, 0].max() < 0.03             # metres
    assert errs[-10:, 1].max() < 0.5             # degrees of yaw


def test_splitmix_offset_reference_values():
    # SplitMix64 of state 0: the first output of the published generator
    # (seed 0, one increment) is 0xE220A8397B1DCDAF.
    m = (1 << 64) - 1
    z = 0x9E3779B97F4A7C15
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
    z ^= z >> 31
    assert z == 0xE220A8397B1DCDAF
    assert splitmix_offset(0, 0) == (0xE220A8397B1DCDAF >> 11) * 2.0 ** -53
    assert all(0.0 <= splitmix_offset(s, k) < 1.0 for s in (0, 1, 2 ** 63) for k in range(50))
