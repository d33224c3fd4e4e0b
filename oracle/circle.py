"""The paper's worked example (Sec. IV, Listings 1-5): 2-D points pulled onto a circle.

Vertex: a 2-D point, additive update.  Constraint (one per point, residual size 1):
    r = x^2 + y^2 - radius^2,   J = [2x, 2y].
The example fixes the last point and disables the constraint of the third point.
"""
import numpy as np


def evaluate(states, data):
    (pts,) = states
    radius = data
    r = (pts[:, 0] ** 2 + pts[:, 1] ** 2 - radius ** 2)[:, None]
    J = (2.0 * pts)[:, None, :]
    return r, [J]


def retract(pts: np.ndarray, delta: np.ndarray) -> np.ndarray:
    return pts + delta
