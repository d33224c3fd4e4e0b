"""Huber robust kernel (Eq. 7) in the reading used throughout (test infrastructure).

For a whitened squared error s = r^T Omega r and threshold delta:
    rho(s)  = s                          if s <= delta^2
            = 2 delta sqrt(s) - delta^2  otherwise
    rho'(s) = min(1, delta / sqrt(s))
The cost of an edge is rho(s)/2, matching the 1/2 of Eq. 1.  The normal equations
use first-order (IRLS) weighting: the whitened residual and Jacobian rows are
scaled by sqrt(rho'(s)), so H gains rho' J^T Omega J and b gains rho' J^T Omega r.
"""
import numpy as np


def huber_rho(s: np.ndarray, delta: float) -> np.ndarray:
    s = np.asarray(s, dtype=np.float64)
    d2 = delta * delta
    return np.where(s <= d2, s, 2.0 * delta * np.sqrt(np.maximum(s, d2)) - d2)


def huber_weight(s: np.ndarray, delta: float) -> np.ndarray:
    s = np.asarray(s, dtype=np.float64)
    return np.where(s <= delta * delta, 1.0, delta / np.sqrt(np.maximum(s, delta * delta)))


def rho(s: np.ndarray, loss) -> np.ndarray:
    """loss is None (plain squares) or ('huber', delta)."""
    if loss is None:
        return np.asarray(s, dtype=np.float64)
    kind, delta = loss
    assert kind == "huber"
    return huber_rho(s, delta)


def weight(s: np.ndarray, loss) -> np.ndarray:
    if loss is None:
        return np.ones_like(np.asarray(s, dtype=np.float64))
    kind, delta = loss
    assert kind == "huber"
    return huber_weight(s, delta)
