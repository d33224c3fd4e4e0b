"""Pins for the oracle's BAL reprojection edge: hand-computed values, the synthetic
renderer at noise-free ground truth, central finite differences on the update chart,
gauge invariance, whitening."""
import numpy as np
import pytest

from oracle import ba, lm, so3
from paper_2509_26581_gb300 import synth


def test_projection_hand_computed():
    # w = 0, t = 0, X = (1, 2, -4): P = X, p = -(1, 2)/(-4) = (0.25, 0.5), |p|^2 = 0.3125
    cam = np.array([0, 0, 0, 0, 0, 0, 100.0, 0.0, 0.0])
    X = np.array([1.0, 2.0, -4.0])
    assert np.array_equal(ba.project(cam, X)[0], [25.0, 50.0])
    # with k1 = 0.1, k2 = 0.01: d = 1 + 0.03125 + 0.0009765625 = 1.0322265625
    cam[7:9] = [0.1, 0.01]
    assert np.allclose(ba.project(cam, X)[0], [25.8056640625, 51.611328125], rtol=0, atol=1e-12)
    # translation enters before the division: t = (1, 0, -4) -> P = (2, 2, -8), p = (0.25, 0.25)
    cam = np.array([0, 0, 0, 1.0, 0, -4.0, 100.0, 0.0, 0.0])
    assert np.allclose(ba.project(cam, X)[0], [25.0, 25.0], atol=1e-12)
    # rotation by pi/2 about z: R X = (-2, 1, -4) -> p = (-0.5, 0.25)
    cam = np.array([0, 0, np.pi / 2, 0, 0, 0, 100.0, 0.0, 0.0])
    assert np.allclose(ba.project(cam, X)[0], [-50.0, 25.0], atol=1e-12)


@pytest.mark.parametrize("gen", ["ring", "path"])
def test_zero_residual_at_noise_free_ground_truth(gen):
    if gen == "ring":
        p = synth.ba_ring(3, 10, 200, 6, pixel_sigma=0.0)
    else:
        p = synth.ba_path(3, 80, 2000, "geom", pixel_sigma=0.0, outlier_frac=0.0)
    r = ba.residual(p.cams_gt[p.cam_idx], p.pts_gt[p.pt_idx], p.obs)
    assert np.max(np.abs(r)) < 1e-9
    prob = lm.ba_problem(p.cams_gt, p.pts_gt, p.cam_idx, p.pt_idx, p.obs)
    assert lm.total_cost(prob) < 1e-15


def _fd_check(cams, X, eps=1e-6):
    Jc, Jp = ba.jacobians(cams, X)
    n = cams.shape[0]
    for k in range(9):
        d = np.zeros((n, 9))
        d[:, k] = eps
        rp = ba.project(ba.retract_cams(cams, d), X)
        rm = ba.project(ba.retract_cams(cams, -d), X)
        fd = (rp - rm) / (2 * eps)
        scale = np.maximum(np.abs(Jc).max(axis=(1, 2)), 1.0)
        assert np.max(np.abs(fd - Jc[:, :, k]) / scale[:, None]) < 1e-6, k
    for k in range(3):
        d = np.zeros((n, 3))
        d[:, k] = eps
        fd = (ba.project(cams, X + d) - ba.project(cams, X - d)) / (2 * eps)
        scale = np.maximum(np.abs(Jp).max(axis=(1, 2)), 1.0)
        assert np.max(np.abs(fd - Jp[:, :, k]) / scale[:, None]) < 1e-6, k


def test_jacobians_central_differences():
    p = synth.ba_ring(5, 10, 100, 6)
    cams = p.cams0[p.cam_idx]
    X = p.pts0[p.pt_idx]
    # exaggerate distortion so that the k-terms are exercised
    cams[:, 7] = 0.05
    cams[:, 8] = -0.02
    _fd_check(cams, X)


def test_jacobians_small_rotation():
    rng = np.random.default_rng(2)
    cams = np.zeros((20, 9))
    cams[:, 0:3] = 1e-7 * rng.normal(size=(20, 3))
    cams[:, 3:6] = [0.1, -0.2, -8.0]
    cams[:, 6] = 480.0
    cams[:, 7:9] = [0.01, 0.001]
    X = rng.uniform(-2, 2, size=(20, 3))
    _fd_check(cams, X)


def _similarity(cams, X, s, wg, tg):
    """Apply X' = s Rg X + tg; cameras R' = R Rg^T, t' = s t - R' tg (P' = s P)."""
    Rg = so3.exp(wg)[0]
    X2 = s * X @ Rg.T + tg
    R = so3.exp(cams[:, 0:3])
    R2 = R @ Rg.T
    c2 = cams.copy()
    c2[:, 0:3] = so3.log(R2)
    c2[:, 3:6] = s * cams[:, 3:6] - np.einsum("nij,j->ni", R2, tg)
    return c2, X2


def test_gauge_invariance_of_cost():
    p = synth.ba_ring(6, 10, 300, 6)
    prob = lm.ba_problem(p.cams0, p.pts0, p.cam_idx, p.pt_idx, p.obs, huber_delta=2.0)
    F = lm.total_cost(prob)
    c2, X2 = _similarity(p.cams0, p.pts0, 1.7, np.array([0.3, -0.2, 0.5]), np.array([1.0, -2.0, 0.5]))
    prob2 = lm.ba_problem(c2, X2, p.cam_idx, p.pt_idx, p.obs, huber_delta=2.0)
    assert abs(lm.total_cost(prob2) - F) < 1e-12 * F


def test_whitening_scales_cost():
    p = synth.ba_ring(7, 10, 100, 6)
    E = p.n_edges
    base = lm.total_cost(lm.ba_problem(p.cams0, p.pts0, p.cam_idx, p.pt_idx, p.obs))
    U = np.broadcast_to(2.0 * np.eye(2), (E, 2, 2)).copy()   # Omega = 4 I
    w = lm.total_cost(lm.ba_problem(p.cams0, p.pts0, p.cam_idx, p.pt_idx, p.obs, sqrt_info=U))
    assert abs(w - 4.0 * base) < 1e-10 * w
