"""Pins for the oracle's SO(3) maps: closed forms, an independent library, round trips."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import so3


def _rz(t):
    c, s = np.cos(t), np.sin(t)
    return np.array([[c, -s, 0], [s, c, 0], [0, 0, 1.0]])


def _rx(t):
    c, s = np.cos(t), np.sin(t)
    return np.array([[1.0, 0, 0], [0, c, -s], [0, s, c]])


def test_exp_axis_rotations_closed_form():
    for t in (0.3, -1.2, 2.9):
        assert np.allclose(so3.exp(np.array([0, 0, t]))[0], _rz(t), atol=1e-15)
        assert np.allclose(so3.exp(np.array([t, 0, 0]))[0], _rx(t), atol=1e-15)


def test_hat_is_cross_product():
    rng = np.random.default_rng(0)
    w, v = rng.normal(size=(2, 50, 3))
    assert np.allclose(np.einsum("nij,nj->ni", so3.hat(w), v), np.cross(w, v), atol=1e-14)


def test_exp_log_match_scipy_rotation():
    rng = np.random.default_rng(1)
    ax = rng.normal(size=(300, 3))
    ax /= np.linalg.norm(ax, axis=1, keepdims=True)
    ang = np.concatenate([rng.uniform(0, np.pi - 1e-6, 280), [1e-12, 1e-9, 1e-6, 1e-4,
                          1.0001e-4, 9.999e-5, 1e-3, 0.5, np.pi - 1e-3, np.pi - 1.0001e-3,
                          np.pi - 1e-5, np.pi - 1e-8, 2.0, 3.0, 1.5, 0.1, 0.2, 0.01, 2.5, 3.1]])
    w = ax * ang[:, None]
    R = so3.exp(w)
    Rs = Rotation.from_rotvec(w).as_matrix()
    assert np.max(np.abs(R - Rs)) < 1e-14
    assert np.max(np.abs(R @ np.transpose(R, (0, 2, 1)) - np.eye(3))) < 1e-14
    assert np.allclose(np.linalg.det(R), 1.0, atol=1e-14)
    w2 = so3.log(Rs)
    ws = Rotation.from_matrix(Rs).as_rotvec()
    assert np.max(np.abs(w2 - ws)) < 1e-7  # near-pi axis conditioning limits both
    far = ang < np.pi - 1e-3
    assert np.max(np.abs(w2[far] - w[far])) < 1e-13


def test_small_angle_series_is_continuous():
    ax = np.array([0.3, -0.5, 0.81])
    ax /= np.linalg.norm(ax)
    lo = so3.exp(ax * (1e-4 * (1 - 1e-9)))[0]
    hi = so3.exp(ax * (1e-4 * (1 + 1e-9)))[0]
    assert np.max(np.abs(lo - hi)) < 1e-12


@pytest.mark.parametrize("seed", [0, 1])
def test_left_update_composes(seed):
    rng = np.random.default_rng(seed)
    w = rng.normal(size=(20, 3))
    dw = 0.1 * rng.normal(size=(20, 3))
    w2 = so3.left_update(dw, w)
    ref = (Rotation.from_rotvec(dw) * Rotation.from_rotvec(w)).as_matrix()
    assert np.max(np.abs(so3.exp(w2) - ref)) < 1e-14
