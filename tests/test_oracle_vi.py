"""Pins for the oracle's visual-inertial terms: preintegration closed forms, the
first-order bias correction, covariance closed forms, zero residuals at noise-free
ground truth, central differences for every Jacobian, and the Schur step against a
brute-force dense solve with 15-dim navigation blocks."""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.spatial.transform import Rotation

from oracle import lm, so3, vi
from paper_2509_26581_gb300 import synth


def test_preintegration_constant_acceleration_closed_form():
    N, dt = 50, 0.005
    a = np.array([0.3, -0.2, 9.81])
    pim = vi.preintegrate(np.zeros((N, 3)), np.tile(a, (N, 1)), dt, np.zeros(3), np.zeros(3), 1e-3, 1e-2)
    T = N * dt
    assert np.allclose(pim["dR"], np.eye(3), atol=1e-15)
    assert np.allclose(pim["dv"], a * T, rtol=0, atol=1e-13)
    assert np.allclose(pim["dp"], 0.5 * a * T * T, rtol=0, atol=1e-13)


def test_preintegration_constant_rate_closed_form():
    N, dt = 40, 0.005
    w = np.array([0.4, -0.1, 0.7])
    pim = vi.preintegrate(np.tile(w, (N, 1)), np.zeros((N, 3)), dt, np.zeros(3), np.zeros(3), 1e-3, 1e-2)
    assert np.allclose(pim["dR"], Rotation.from_rotvec(w * N * dt).as_matrix(), atol=1e-13)
    assert np.allclose(pim["dv"], 0, atol=1e-15) and np.allclose(pim["dp"], 0, atol=1e-15)


def test_preintegration_covariance_closed_form_at_rest():
    N, dt, sg, sa = 50, 0.005, 2e-3, 3e-2
    pim = vi.preintegrate(np.zeros((N, 3)), np.zeros((N, 3)), dt, np.zeros(3), np.zeros(3), sg, sa)
    T = N * dt
    C = pim["cov"]
    assert np.allclose(C[0:3, 0:3], sg * sg * T * np.eye(3), rtol=1e-12)
    assert np.allclose(C[3:6, 3:6], sa * sa * T * np.eye(3), rtol=1e-12)
    pp = sa * sa * dt ** 3 * (N ** 3 / 3.0 - N / 12.0)
    assert np.allclose(C[6:9, 6:9], pp * np.eye(3), rtol=1e-12)
    assert np.allclose(C, C.T) and np.all(np.linalg.eigvalsh(C) > 0)


def test_bias_correction_is_first_order():
    rng = np.random.default_rng(0)
    N, dt = 50, 0.005
    w = 0.5 * rng.normal(size=(N, 3))
    a = np.array([0.0, 0.0, 9.81]) + rng.normal(size=(N, 3))
    pim = vi.preintegrate(w, a, dt, np.zeros(3), np.zeros(3), 1e-3, 1e-2)
    errs = []
    for h in (1e-2, 5e-3):
        dbg, dba = h * np.array([1.0, -0.5, 0.3]), h * np.array([-0.4, 1.0, 0.2])
        ref = vi.preintegrate(w, a, dt, dbg, dba, 1e-3, 1e-2)
        dR = pim["dR"] @ so3.exp(pim["JRg"] @ dbg)[0]
        dv = pim["dv"] + pim["Jvg"] @ dbg + pim["Jva"] @ dba
        dp = pim["dp"] + pim["Jpg"] @ dbg + pim["Jpa"] @ dba
        errs.append(max(np.abs(so3.log(dR.T @ ref["dR"])).max(), np.abs(dv - ref["dv"]).max(),
                        np.abs(dp - ref["dp"]).max()))
    assert errs[1] < errs[0] / 3.0          # quadratic: halving the deviation quarters the error
    assert errs[0] < 1e-5


@pytest.fixture(scope="module")
def small():
    return synth.vi_problem(1, 12, 400)


def test_zero_residual_at_noise_free_ground_truth():
    p = synth.vi_problem(2, 10, 300, imu_noise=False, pixel_sigma=0.0)
    cam = vi.camera_of(p.camera)
    r, _ = cam.evaluate([p.nav_gt[p.kf_idx], p.pts_gt[p.pt_idx]], p.obs)
    assert np.abs(r).max() < 1e-9
    pims = vi.preintegrate_all(p, bg0=p.nav_gt[0, 10:13], ba0=p.nav_gt[0, 13:16])
    for k, pm in enumerate(pims):
        res = vi.imu_residual_one(pm, p.nav_gt[k:k + 1], p.nav_gt[k + 1:k + 2])
        assert np.abs(res).max() < 1e-10


def _fd_nav(f, x, eps=1e-6):
    cols = []
    for k in range(15):
        d = np.zeros((1, 15))
        d[0, k] = eps
        cols.append((f(vi.retract_nav(x, d)) - f(vi.retract_nav(x, -d))) / (2 * eps))
    return np.stack(cols, axis=-1)


FISHEYE = (-0.013, 0.021, -0.006, 0.0009)   # Kannala-Brandt k1..k4 of a wide-angle lens


def test_fisheye_projection_closed_form():
    """With k = 0 the Kannala-Brandt model is the equidistant one: a point at angle
    theta off the axis lands fx theta from the principal point; with k it lands at
    fx theta (1 + k1 theta^2 + ... + k4 theta^8)."""
    th = np.linspace(0.05, 1.4, 12)
    x, y, z = np.sin(th) * 3.0, np.zeros_like(th), np.cos(th) * 3.0
    u, v, _ = vi.kb_project(x, y, z, 400.0, 410.0, 320.0, 240.0, (0.0, 0.0, 0.0, 0.0))
    assert np.allclose(u, 400.0 * th + 320.0, rtol=0, atol=1e-10) and np.allclose(v, 240.0, atol=1e-12)
    k1, k2, k3, k4 = FISHEYE
    u, _, _ = vi.kb_project(x, y, z, 400.0, 410.0, 320.0, 240.0, FISHEYE)
    t2 = th * th
    assert np.allclose(u, 400.0 * th * (1 + k1 * t2 + k2 * t2 ** 2 + k3 * t2 ** 3 + k4 * t2 ** 4) + 320.0,
                       rtol=0, atol=1e-10)


@pytest.mark.parametrize("fisheye", [False, True])
def test_stereo_jacobians_central_differences(small, fisheye):
    p = small
    cam = vi.camera_of(dict(p.camera, fisheye=FISHEYE) if fisheye else p.camera)
    for e in range(0, p.n_edges, max(1, p.n_edges // 25)):
        x = p.nav0[p.kf_idx[e]][None]
        X = p.pts0[p.pt_idx[e]][None]
        r, (Jn, Jp) = cam.evaluate([x, X], p.obs[e][None])
        fd = _fd_nav(lambda xx: cam.project(xx, X)[0], x)
        assert np.abs(fd - Jn[0]).max() < 1e-5 * max(1.0, np.abs(Jn).max())
        fdp = np.stack([(cam.project(x, X + h)[0] - cam.project(x, X - h)[0]) / 2e-6
                        for h in 1e-6 * np.eye(3)], axis=-1)
        assert np.abs(fdp - Jp[0]).max() < 1e-5 * max(1.0, np.abs(Jp).max())


def test_imu_jacobians_central_differences(small):
    p = small
    pims = vi.preintegrate_all(p)
    rng = np.random.default_rng(1)
    for k in (0, 4, 10):
        xi = p.nav0[k:k + 1].copy()
        xj = p.nav0[k + 1:k + 2].copy()
        xi[0, 10:16] += 1e-3 * rng.normal(size=6)           # bias deviation exercises J_R^g etc.
        Ji, Jj = vi.imu_jacobians_one(pims[k], xi, xj)
        fi = _fd_nav(lambda xx: vi.imu_residual_one(pims[k], xx, xj), xi)
        fj = _fd_nav(lambda xx: vi.imu_residual_one(pims[k], xi, xx), xj)
        assert np.abs(fi - Ji).max() < 1e-6 * max(1.0, np.abs(Ji).max())
        assert np.abs(fj - Jj).max() < 1e-6 * max(1.0, np.abs(Jj).max())


def test_bias_edges_central_differences(small):
    p = small
    xi, xj = p.nav0[0:1], p.nav0[1:2]
    _, (Ji, Jj) = vi.bias_rw_evaluate([xi, xj], None)
    fi = _fd_nav(lambda xx: vi.bias_rw_evaluate([xx, xj], None)[0][0], xi)
    assert np.abs(fi - Ji[0]).max() < 1e-8
    _, (J,) = vi.bias_prior_evaluate([xi], np.zeros((1, 6)))
    f = _fd_nav(lambda xx: vi.bias_prior_evaluate([xx], np.zeros((1, 6)))[0][0], xi)
    assert np.abs(f - J[0]).max() < 1e-8


def test_vi_schur_step_equals_dense_solve(small):
    p = small
    prob = vi.problem(p, p.nav0, p.pts0, vi.preintegrate_all(p))
    layout = lm.make_layout(prob)
    lin = lm.linearize(prob, layout)
    H, b = lm.normal_equations(lin)
    Hl = H + sp.diags(1e-3 * lm.damping_diagonal(H, lm.LMParams()))
    dx, _, _ = lm.schur_solve(Hl, b, layout)
    ref = lm.dense_solve(Hl, b)
    assert np.abs(dx - ref).max() <= 1e-8 * np.abs(ref).max()


def test_vi_lm_decreases_cost(small):
    p = small
    prob = vi.problem(p, p.nav0, p.pts0, vi.preintegrate_all(p))
    _, rep = lm.levenberg_marquardt(prob, 8)
    assert rep.final_cost < 0.2 * rep.initial_cost


def test_huber_inertial_edges_reduce_to_the_plain_and_the_huber_forms(small):
    """Huber on the inertial edges: a threshold above every whitened residual leaves the
    objective unchanged; a finite one replaces each large edge's s by 2 delta sqrt(s) -
    delta^2 (Eq. 7) and leaves the other edge sets as they were."""
    p = small
    pims = vi.preintegrate_all(p)
    plain = vi.problem(p, p.nav0, p.pts0, pims)
    c0 = lm.edge_costs(plain)
    s = 2.0 * c0[1]                                   # whitened squared norms of the inertial edges
    big = vi.problem(p, p.nav0, p.pts0, pims, imu_huber=10.0 * np.sqrt(s.max()))
    assert np.array_equal(lm.edge_costs(big)[1], c0[1])
    delta = float(np.median(np.sqrt(s)))
    hub = lm.edge_costs(vi.problem(p, p.nav0, p.pts0, pims, imu_huber=delta))
    want = np.where(s > delta ** 2, 2.0 * delta * np.sqrt(s) - delta ** 2, s) / 2.0
    assert np.allclose(hub[1], want, rtol=1e-15, atol=0.0)
    assert (s > delta ** 2).any() and (s <= delta ** 2).any()
    for k in (0, 2, 3):
        assert np.array_equal(hub[k], c0[k])


def test_monocular_edges_are_the_left_camera_rows(small):
    """The monocular edge is the stereo residual's first two rows (left camera), with the
    matching Jacobian rows (central differences pin the stereo ones); a problem with
    every observation monocular sums their squared norms."""
    p = small
    cam = vi.camera_of(p.camera)
    states = (p.nav0[p.kf_idx], p.pts0[p.pt_idx])
    r3, (Jn3, Jp3) = cam.evaluate(states, np.asarray(p.obs, float))
    r2, (Jn2, Jp2) = vi.mono_evaluate(cam)(states, np.asarray(p.obs, float)[:, :2])
    assert np.array_equal(r2, r3[:, :2])
    assert np.array_equal(Jn2, Jn3[:, :2]) and np.array_equal(Jp2, Jp3[:, :2])
    pims = vi.preintegrate_all(p)
    allmono = vi.problem(p, p.nav0, p.pts0, pims, huber=False, mono=np.ones(len(p.kf_idx), bool))
    assert [e.name for e in allmono.edges] == ["mono", "imu", "bias_rw", "bias_prior"]
    costs = lm.edge_costs(allmono)
    assert np.allclose(costs[0], 0.5 * np.sum(r2 * r2, axis=1), rtol=1e-15, atol=0)
