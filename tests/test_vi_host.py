"""Host-side IMU preintegration of the library (gpo_imu_preintegrate, a C-ABI call that
needs no GPU) against the oracle's preintegration.

Tolerance: 1e-13 relative to each block's largest entry.  Both sides run the same
recurrences over 50 samples in FP64 and differ only in operation order, so each block
agrees to a few ulps times the number of steps; the information matrix is the inverse
of a covariance of condition number ~2e2, which adds that factor."""
import numpy as np
import pytest

from oracle import vi as ovi
from paper_2509_26581_gb300 import synth

BLOCKS = {"dR": (0, 9), "dv": (9, 12), "dp": (12, 15), "JRg": (15, 24), "Jvg": (24, 33),
          "Jva": (33, 42), "Jpg": (42, 51), "Jpa": (51, 60), "T": (60, 61), "bg0": (61, 64),
          "ba0": (64, 67)}


@pytest.fixture(scope="module")
def gpo():
    from paper_2509_26581_gb300 import gpo as m
    return m


@pytest.fixture(scope="module")
def problem():
    return synth.vi_problem(5, n_kf=8, n_pts=200)


def _rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("bias", ["zero", "nonzero"])
def test_preintegration_matches_oracle(gpo, problem, bias):
    p = problem
    rng = np.random.default_rng(1)
    for k in range(p.imu_gyro.shape[0]):
        bg0 = np.zeros(3) if bias == "zero" else rng.normal(scale=1e-3, size=3)
        ba0 = np.zeros(3) if bias == "zero" else rng.normal(scale=5e-2, size=3)
        meas, cov, info = gpo.imu_preintegrate(p.imu_gyro[k], p.imu_acc[k], p.dt, bg0, ba0,
                                               p.noise["sigma_g"], p.noise["sigma_a"])
        pm = ovi.preintegrate(p.imu_gyro[k], p.imu_acc[k], p.dt, bg0, ba0, p.noise["sigma_g"],
                              p.noise["sigma_a"])
        for name, (a, b) in BLOCKS.items():
            ref = np.atleast_1d(pm[name]).ravel()
            assert _rel(meas[a:b], ref) <= 1e-13, name
        assert _rel(cov, pm["cov"]) <= 1e-13
        assert _rel(info, np.linalg.inv(pm["cov"])) <= 1e-13 * np.linalg.cond(pm["cov"])
        assert np.allclose(info @ cov, np.eye(9), atol=1e-10)


def test_preintegration_rejects_bad_arguments(gpo, problem):
    p = problem
    import ctypes as C
    out = np.zeros(gpo.GPO_IMU_MEAS_LEN)
    w = np.ascontiguousarray(p.imu_gyro[0])
    a = np.ascontiguousarray(p.imu_acc[0])
    z = np.zeros(3)
    ptr = lambda x: x.ctypes.data_as(C.c_void_p)
    assert gpo.lib.gpo_imu_preintegrate(ptr(w), ptr(a), 0, p.dt, ptr(z), ptr(z), 1e-3, 1e-3, ptr(out),
                                        None, None) == gpo.GPO_ERR_ARG
    assert gpo.lib.gpo_imu_preintegrate(ptr(w), ptr(a), 10, -1.0, ptr(z), ptr(z), 1e-3, 1e-3, ptr(out),
                                        None, None) == gpo.GPO_ERR_ARG
    assert gpo.lib.gpo_imu_preintegrate(None, ptr(a), 10, p.dt, ptr(z), ptr(z), 1e-3, 1e-3, ptr(out),
                                        None, None) == gpo.GPO_ERR_ARG
    assert gpo.lib.gpo_imu_preintegrate(ptr(w), ptr(a), 10, p.dt, ptr(z), ptr(z), 0.0, 1e-3, ptr(out),
                                        None, None) == gpo.GPO_ERR_ARG


def test_single_sample_closed_form(gpo):
    """One sample: dR = Exp(w dt), dv = a dt, dp = a dt^2 / 2, JRg = -Jr(w dt) dt."""
    w = np.array([[0.3, -0.2, 0.5]])
    a = np.array([[0.1, 9.7, -0.4]])
    dt = 0.005
    meas, cov, _ = gpo.imu_preintegrate(w, a, dt, np.zeros(3), np.zeros(3), 1e-3, 1e-2, with_info=False)
    from oracle import so3
    assert np.allclose(meas[0:9].reshape(3, 3), so3.exp(w * dt)[0], rtol=0, atol=1e-15)
    assert np.allclose(meas[9:12], a[0] * dt, rtol=1e-15, atol=0)
    assert np.allclose(meas[12:15], 0.5 * a[0] * dt * dt, rtol=1e-15, atol=0)
    assert np.allclose(meas[15:24].reshape(3, 3), -ovi.right_jacobian(w * dt)[0] * dt, rtol=0, atol=1e-17)
    # first-step covariance: rotation block (sigma_g^2/dt) Jr Jr^T dt^2, velocity (sigma_a^2/dt) dt^2 I
    Jr = ovi.right_jacobian(w * dt)[0]
    assert np.allclose(cov[0:3, 0:3], 1e-6 / dt * Jr @ Jr.T * dt * dt, rtol=0, atol=1e-13 * 1e-6 * dt)
    assert np.allclose(cov[3:6, 3:6], 1e-4 / dt * dt * dt * np.eye(3), rtol=1e-13, atol=1e-30)
    assert meas[60] == dt
