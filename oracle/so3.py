"""SO(3) exponential and logarithm on angle-axis vectors (FP64), vectorised over rows.

Used by the BA camera chart: a rotation update is applied on the left,
R <- Exp(dw) R, and stored back as the angle-axis vector Log(Exp(dw) Exp(w)).
Sec. V evaluates on BAL problems whose cameras store angle-axis rotations; the
paper gives no formula for the chart, so this one is a stated reading.
"""
import numpy as np


def hat(w: np.ndarray) -> np.ndarray:
    """Skew matrices [w]_x with [w]_x v = w x v, for w of shape (n, 3)."""
    w = np.asarray(w, dtype=np.float64)
    K = np.zeros(w.shape[:-1] + (3, 3))
    K[..., 0, 1] = -w[..., 2]
    K[..., 0, 2] = w[..., 1]
    K[..., 1, 0] = w[..., 2]
    K[..., 1, 2] = -w[..., 0]
    K[..., 2, 0] = -w[..., 1]
    K[..., 2, 1] = w[..., 0]
    return K


def exp(w: np.ndarray) -> np.ndarray:
    """Rodrigues' formula R = I + a [w]_x + b [w]_x^2, a = sin(t)/t, b = (1 - cos t)/t^2.

    Below t = 1e-4 the two coefficients use their Taylor series (terms to t^4)."""
    w = np.atleast_2d(np.asarray(w, dtype=np.float64))
    th2 = np.sum(w * w, axis=-1)
    th = np.sqrt(th2)
    small = th < 1e-4
    ths = np.where(small, 1.0, th)
    a = np.where(small, 1.0 - th2 / 6.0 + th2 * th2 / 120.0, np.sin(ths) / ths)
    b = np.where(small, 0.5 - th2 / 24.0 + th2 * th2 / 720.0, (1.0 - np.cos(ths)) / (ths * ths))
    K = hat(w)
    I = np.broadcast_to(np.eye(3), K.shape)
    return I + a[..., None, None] * K + b[..., None, None] * (K @ K)


def log(R: np.ndarray) -> np.ndarray:
    """Angle-axis w with Exp(w) = R, |w| in [0, pi].

    t = atan2(|v|, (tr R - 1)/2) with v = vee(R - R^T)/2 = sin(t) * axis.  Away from
    t = pi, w = t / sin(t) * v (series for small t).  Near t = pi the axis is read from
    the symmetric part (R + R^T)/2 - cos(t) I = (1 - cos t) a a^T, its sign from v."""
    R = np.asarray(R, dtype=np.float64)
    if R.ndim == 2:
        R = R[None]
    v = 0.5 * np.stack([R[:, 2, 1] - R[:, 1, 2], R[:, 0, 2] - R[:, 2, 0],
                        R[:, 1, 0] - R[:, 0, 1]], axis=1)
    s = np.linalg.norm(v, axis=1)
    c = 0.5 * (R[:, 0, 0] + R[:, 1, 1] + R[:, 2, 2] - 1.0)
    th = np.arctan2(s, c)
    out = np.empty_like(v)
    near_pi = th > np.pi - 1e-3
    regular = ~near_pi
    small = regular & (th < 1e-4)
    mid = regular & ~small
    out[small] = v[small] * (1.0 + th[small] ** 2 / 6.0)[:, None]
    out[mid] = v[mid] * (th[mid] / s[mid])[:, None]
    for i in np.nonzero(near_pi)[0]:
        Sym = 0.5 * (R[i] + R[i].T) - c[i] * np.eye(3)
        d = np.diag(Sym) / (1.0 - c[i])
        k = int(np.argmax(d))
        a = Sym[k] / (np.sqrt(d[k]) * (1.0 - c[i]))
        a = a / np.linalg.norm(a)
        if np.dot(a, v[i]) < 0:
            a = -a
        out[i] = th[i] * a
    return out


def left_update(dw: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Angle-axis of Exp(dw) Exp(w)."""
    return log(exp(dw) @ exp(w))
