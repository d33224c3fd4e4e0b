"""BAL camera reprojection edge (FP64 oracle, test infrastructure).

Sec. V evaluates on Bundle Adjustment in the Large problems; the paper does not
print the camera model, so this is the BAL convention as a stated reading:
a camera is c = [w(3), t(3), f, k1, k2],
    P = R(w) X + t,  p = -P_xy / P_z,  u = f (1 + k1 |p|^2 + k2 |p|^4) p,
and the residual of an observation z is r = u - z (Eq. 1 with Sigma = I unless an
information matrix is given).

Analytic Jacobians (Sec. IV-B) are taken on the chart
    w <- Log(Exp(dw) Exp(w))  (left perturbation), t, f, k1, k2 and X additive.
With y = R X:
    dP/ddw = -[y]_x,  dP/dt = I,  dP/dX = R
    dp/dP  = [[-1/Pz, 0, Px/Pz^2], [0, -1/Pz, Py/Pz^2]]
    du/dp  = f (d I + (2 k1 + 4 k2 |p|^2) p p^T),  d = 1 + k1 |p|^2 + k2 |p|^4
    du/df  = d p,  du/dk1 = f |p|^2 p,  du/dk2 = f |p|^4 p
"""
import numpy as np

from . import so3


def project(cams: np.ndarray, X: np.ndarray) -> np.ndarray:
    cams = np.atleast_2d(cams)
    X = np.atleast_2d(X)
    R = so3.exp(cams[:, 0:3])
    P = np.einsum("nij,nj->ni", R, X) + cams[:, 3:6]
    p = -P[:, 0:2] / P[:, 2:3]
    r2 = np.sum(p * p, axis=1)
    d = 1.0 + cams[:, 7] * r2 + cams[:, 8] * r2 * r2
    return (cams[:, 6] * d)[:, None] * p


def residual(cams: np.ndarray, X: np.ndarray, obs: np.ndarray) -> np.ndarray:
    return project(cams, X) - obs


def jacobians(cams: np.ndarray, X: np.ndarray):
    """(J_cam (n,2,9), J_point (n,2,3)) of the residual at (cams, X)."""
    cams = np.atleast_2d(cams)
    X = np.atleast_2d(X)
    n = cams.shape[0]
    R = so3.exp(cams[:, 0:3])
    y = np.einsum("nij,nj->ni", R, X)
    P = y + cams[:, 3:6]
    Px, Py, Pz = P[:, 0], P[:, 1], P[:, 2]
    p = -P[:, 0:2] / P[:, 2:3]
    r2 = np.sum(p * p, axis=1)
    f, k1, k2 = cams[:, 6], cams[:, 7], cams[:, 8]
    d = 1.0 + k1 * r2 + k2 * r2 * r2
    dp_dP = np.zeros((n, 2, 3))
    dp_dP[:, 0, 0] = -1.0 / Pz
    dp_dP[:, 0, 2] = Px / (Pz * Pz)
    dp_dP[:, 1, 1] = -1.0 / Pz
    dp_dP[:, 1, 2] = Py / (Pz * Pz)
    du_dp = f[:, None, None] * (d[:, None, None] * np.eye(2)[None]
                                + (2.0 * k1 + 4.0 * k2 * r2)[:, None, None]
                                * np.einsum("ni,nj->nij", p, p))
    du_dP = du_dp @ dp_dP
    Jc = np.zeros((n, 2, 9))
    Jc[:, :, 0:3] = du_dP @ (-so3.hat(y))
    Jc[:, :, 3:6] = du_dP
    Jc[:, :, 6] = d[:, None] * p
    Jc[:, :, 7] = (f * r2)[:, None] * p
    Jc[:, :, 8] = (f * r2 * r2)[:, None] * p
    Jp = du_dP @ R
    return Jc, Jp


def retract_cams(cams: np.ndarray, delta: np.ndarray) -> np.ndarray:
    """cams [+] delta on the chart above."""
    out = np.array(cams, dtype=np.float64, copy=True)
    out[:, 0:3] = so3.left_update(delta[:, 0:3], cams[:, 0:3])
    out[:, 3:9] = cams[:, 3:9] + delta[:, 3:9]
    return out


def retract_points(X: np.ndarray, delta: np.ndarray) -> np.ndarray:
    return X + delta


def evaluate(states, data):
    """Edge evaluator for the generic LM: states = [cams (n,9), points (n,3)], data = obs."""
    cams, X = states
    return residual(cams, X, data), list(jacobians(cams, X))
