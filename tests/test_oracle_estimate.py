"""Pins of the oracle's pose estimate (Sec. III: weighted average or the
particle with the highest weight; Sec. V: weighted sum of the poses) against
closed forms, SciPy's independent rotation code and invariants."""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle


@pytest.fixture
def rng():
    return np.random.default_rng(20231004)


def _sign_fix(q):
    q = np.asarray(q, np.float64)
    nz = np.flatnonzero(q != 0)
    return -q if q[nz[0]] < 0 else q


def _scipy_quat(rpy):
    """SciPy extrinsic x-y-z Euler angles = Rz(yaw) Ry(pitch) Rx(roll);
    SciPy's quaternion is (x, y, z, w)."""
    x, y, z, w = Rotation.from_euler("xyz", rpy).as_quat()
    return _sign_fix([w, x, y, z])


def _poses(rpy, t=None):
    rpy = np.atleast_2d(np.asarray(rpy, np.float32))
    out = np.zeros((len(rpy), 6), np.float32)
    out[:, 3:] = rpy
    if t is not None:
        out[:, :3] = t
    return out


def test_translation_and_component_means_closed_form():
    s = np.array([[1, 2, 3, 0.1, 0.2, 0.3],
                  [5, -2, 7, 0.5, -0.2, 1.0]], np.float32)
    e = oracle.pose_estimate(s, [1.0, 3.0])              # unnormalised weights
    s64 = s.astype(np.float64)
    assert e["weight_sum"] == 4.0
    np.testing.assert_allclose(e["mean_pose"], (s64[0] + 3 * s64[1]) / 4, rtol=0, atol=1e-15)
    assert e["n_eff"] == pytest.approx(16.0 / 10.0, abs=1e-15)


def test_identical_rotations_give_that_rotation(rng):
    for _ in range(20):
        rpy = rng.uniform([-math.pi, -1.5, -math.pi], [math.pi, 1.5, math.pi]).astype(np.float32)
        s = _poses(np.repeat(rpy[None], 7, 0))
        e = oracle.pose_estimate(s, rng.uniform(0.1, 2.0, 7))
        np.testing.assert_allclose(e["quat"], _scipy_quat(rpy.astype(np.float64)), atol=1e-12)
        assert e["concentration"] == pytest.approx(1.0, abs=1e-12)
        rot = Rotation.from_quat([e["quat"][1], e["quat"][2], e["quat"][3], e["quat"][0]])
        np.testing.assert_allclose(e["rpy"], rot.as_euler("xyz"), atol=1e-12)


def test_rotations_about_one_axis_give_the_circular_mean(rng):
    """For rotations about one axis n by angles a_i, ||R(phi) - R(a_i)||^2 =
    4 (1 - cos(phi - a_i)), so the chordal mean is the circular mean
    atan2(sum w sin a, sum w cos a) of the full angles."""
    for _ in range(10):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        a = rng.uniform(-1.0, 1.0, 9) + rng.uniform(-math.pi, math.pi)
        w = rng.uniform(0.1, 1.0, 9).astype(np.float32).astype(np.float64)
        rots = Rotation.from_rotvec(a[:, None] * n[None])
        rpy = rots.as_euler("xyz").astype(np.float32)
        # The estimate sees the FP32-rounded angles: take the angles about n
        # of exactly those rotations.
        r32 = Rotation.from_euler("xyz", rpy.astype(np.float64))
        a32 = np.array([np.dot(rv, n) for rv in r32.as_rotvec()])
        phi = math.atan2(float(np.sum(w * np.sin(a32))), float(np.sum(w * np.cos(a32))))
        want = Rotation.from_rotvec(phi * n)
        e = oracle.pose_estimate(_poses(rpy), w)
        x, y, z, qw = want.as_quat()
        np.testing.assert_allclose(e["quat"], _sign_fix([qw, x, y, z]), atol=2e-7)


def test_yaw_wrap_literal_mean_fails_rotation_mean_holds():
    s = _poses([[0, 0, 3.1], [0, 0, -3.1]])
    e = oracle.pose_estimate(s, [1.0, 1.0])
    assert e["mean_pose"][5] == 0.0                       # the literal average
    assert abs(abs(e["rpy"][2]) - math.pi) < 1e-12        # the rotation mean


def test_left_invariance(rng):
    rpy = (rng.normal(scale=0.2, size=(50, 3)) + [0.1, -0.2, 2.5]).astype(np.float32)
    w = rng.uniform(0, 1, 50)
    r0 = Rotation.from_euler("xyz", [0.4, -0.3, 1.1])
    moved = (r0 * Rotation.from_euler("xyz", rpy.astype(np.float64))).as_euler("xyz").astype(np.float32)
    e1 = oracle.pose_estimate(_poses(rpy), w)
    e2 = oracle.pose_estimate(_poses(moved), w)
    q1 = Rotation.from_quat([*e1["quat"][1:], e1["quat"][0]])
    q2 = Rotation.from_quat([*e2["quat"][1:], e2["quat"][0]])
    assert (r0 * q1).inv().__mul__(q2).magnitude() < 1e-6   # FP32 rounding of moved angles


def test_chordal_mean_is_optimal(rng):
    rpy = (rng.normal(scale=0.5, size=(40, 3))).astype(np.float32)
    w = rng.uniform(0, 1, 40).astype(np.float32).astype(np.float64)   # the oracle reads FP32 weights
    e = oracle.pose_estimate(_poses(rpy), w)
    mats = Rotation.from_euler("xyz", rpy.astype(np.float64)).as_matrix()

    def cost(R):
        return float(np.sum(w * np.sum((R[None] - mats) ** 2, axis=(1, 2))))

    best = Rotation.from_quat([*e["quat"][1:], e["quat"][0]]).as_matrix()
    c0 = cost(best)
    # cost = W (8 - 8 lambda)
    assert c0 == pytest.approx(np.sum(w) * (8 - 8 * e["concentration"]), rel=1e-12)
    for _ in range(300):
        d = Rotation.from_rotvec(rng.normal(scale=0.05, size=3)).as_matrix()
        assert cost(d @ best) >= c0 - 1e-12


def test_matches_scipy_weighted_mean(rng):
    rpy = (rng.normal(scale=0.3, size=(100, 3)) + [0.0, 0.1, -2.0]).astype(np.float32)
    w = rng.uniform(0, 1, 100).astype(np.float32).astype(np.float64)
    e = oracle.pose_estimate(_poses(rpy), w)
    m = Rotation.from_euler("xyz", rpy.astype(np.float64)).mean(weights=w)
    x, y, z, qw = m.as_quat()
    np.testing.assert_allclose(e["quat"], _sign_fix([qw, x, y, z]), atol=1e-10)


def test_argmax_and_effective_size():
    s = np.arange(30, dtype=np.float32).reshape(5, 6)
    e = oracle.pose_estimate(s, [0.1, 0.4, 0.1, 0.4, 0.0])     # tie: lowest index
    assert e["argmax"] == 1 and e["best_w"] == np.float32(0.4)
    np.testing.assert_array_equal(e["best_pose"], s[1])
    assert oracle.pose_estimate(s, np.full(5, 0.2))["n_eff"] == pytest.approx(5.0, abs=1e-12)
    assert oracle.pose_estimate(s, [0, 0, 1, 0, 0])["n_eff"] == 1.0
    e = oracle.pose_estimate(s, [np.nan, 0.3, np.nan, 0.5, 0.2])
    assert e["argmax"] == 3
    e = oracle.pose_estimate(s, np.zeros(5))
    assert e["argmax"] == 0 and e["n_eff"] == 0.0 and np.all(np.isnan(e["mean_pose"]))
