"""Planted mistakes in the oracle (on the CPU): each must make one of its pins fail.

This shows that the pins in test_oracle_*.py constrain the oracle, and are not
satisfied by a plausible wrong implementation (a wrong sign, a transposed operand,
a dropped term)."""
import numpy as np
import pytest

import oracle.ba as ba
import oracle.lm as lm
import oracle.so3 as so3
from tests import test_oracle_ba as pins_ba
from tests import test_oracle_lm as pins_lm


def test_wrong_rotation_jacobian_sign_fails_fd(monkeypatch):
    orig = ba.jacobians

    def bad(cams, X):
        Jc, Jp = orig(cams, X)
        Jc = Jc.copy()
        Jc[:, :, 0:3] *= -1.0
        return Jc, Jp

    monkeypatch.setattr(ba, "jacobians", bad)
    with pytest.raises(AssertionError):
        pins_ba.test_jacobians_central_differences()


def test_right_instead_of_left_perturbation_fails_fd(monkeypatch):
    monkeypatch.setattr(so3, "left_update", lambda dw, w: so3.log(so3.exp(w) @ so3.exp(dw)))
    with pytest.raises(AssertionError):
        pins_ba.test_jacobians_central_differences()


def test_transposed_rotation_fails_ground_truth(monkeypatch):
    orig = so3.exp
    monkeypatch.setattr(so3, "exp", lambda w: np.transpose(orig(w), (0, 2, 1)))
    with pytest.raises(AssertionError):
        pins_ba.test_zero_residual_at_noise_free_ground_truth("ring")


def test_dropped_distortion_term_fails_hand_values(monkeypatch):
    def bad(cams, X):
        cams = np.atleast_2d(cams).copy()
        cams[:, 8] = 0.0
        R = so3.exp(cams[:, 0:3])
        P = np.einsum("nij,nj->ni", R, np.atleast_2d(X)) + cams[:, 3:6]
        p = -P[:, 0:2] / P[:, 2:3]
        r2 = np.sum(p * p, axis=1)
        return (cams[:, 6] * (1.0 + cams[:, 7] * r2))[:, None] * p

    monkeypatch.setattr(ba, "project", bad)
    with pytest.raises(AssertionError):
        pins_ba.test_projection_hand_computed()


def test_missing_schur_term_fails_brute_force(monkeypatch):
    orig = lm.schur_solve

    def bad(Hl, b, layout):
        nr = layout.n_reduced
        dx, S, g = orig(Hl, b, layout)
        Hrr = Hl.tocsr()[:nr, :nr].toarray()
        import scipy.linalg
        dxr = scipy.linalg.solve(Hrr, g)
        dx = dx.copy()
        dx[:nr] = dxr
        return dx, Hrr, g

    monkeypatch.setattr(lm, "schur_solve", bad)
    with pytest.raises(AssertionError):
        pins_lm.test_schur_step_equals_dense_full_solve(0, 1e-4, None)


def test_wrong_model_decrease_sign_fails_identity(monkeypatch):
    def bad(lin, b, dx):
        Jdx = lin.J @ dx
        return float(-b @ dx + 0.5 * Jdx @ Jdx)

    monkeypatch.setattr(lm, "model_decrease", bad)
    with pytest.raises(AssertionError):
        pins_lm.test_model_decrease_identity(1e-2)


def test_unclamped_damping_diagonal_fails_values(monkeypatch):
    monkeypatch.setattr(lm, "damping_diagonal", lambda H, params: H.diagonal())
    with pytest.raises(AssertionError):
        pins_lm.test_damping_diagonal_clamp_values()


def test_clamping_lambda_times_diagonal_fails_closed_form(monkeypatch):
    # plausible mistake: clamp lambda diag(H) instead of diag(H) before scaling by lambda
    def bad(problem, lam, params=None):
        params = params or lm.LMParams()
        layout = lm.make_layout(problem)
        lin = lm.linearize(problem, layout)
        H, b = lm.normal_equations(lin)
        D = np.clip(lam * H.diagonal(), params.diag_min, params.diag_max) / lam
        dx, _, _ = lm.schur_solve(H + lm.sp.diags(lam * D), b, layout)
        return dx, layout, H, b, D, lin

    monkeypatch.setattr(lm, "step", bad)
    with pytest.raises(AssertionError):
        pins_lm.test_damped_step_closed_form_with_clamped_diagonal(1e-4)


def test_missing_lambda_clamp_fails_bounds(monkeypatch):
    monkeypatch.setattr(lm, "clamp_lambda", lambda lam, params: lam)
    with pytest.raises(AssertionError):
        pins_lm.test_lambda_rises_to_upper_bound_at_exact_optimum()
    with pytest.raises(AssertionError):
        pins_lm.test_lambda_falls_to_lower_bound_on_linear_problem()


def test_rejected_step_keeping_lambda_fails_bounds(monkeypatch):
    orig = lm.nielsen_update
    monkeypatch.setattr(lm, "nielsen_update",
                        lambda lam, nu, rho, acc: orig(lam, nu, rho, acc) if acc else (lam * 2.0, 2.0))
    with pytest.raises(AssertionError):
        pins_lm.test_lambda_rises_to_upper_bound_at_exact_optimum()
