"""Oracle for the library's generic edge kinds (test infrastructure only: the library
never imports this).  The paper's running example (Sec. III, Listings 1-5): 2-D points
pulled onto a circle by the constraint x^2 + y^2 - R^2 = 0, optionally tied to each
other by squared-distance constraints |x_i - x_j|^2 - d^2 = 0.  Residuals and analytic
Jacobians in FP64, solved by the generic LM of oracle.lm (exact steps)."""
import numpy as np

from . import lm


def circle_evaluate(states, R):
    """r = x^2 + y^2 - R^2; J = [2x, 2y]."""
    (X,) = states
    r = (X[:, 0] ** 2 + X[:, 1] ** 2 - np.asarray(R, float) ** 2)[:, None]
    J = (2.0 * X)[:, None, :]
    return r, [J]


def distance_evaluate(states, d):
    """r = |x_i - x_j|^2 - d^2; J_i = 2 (x_i - x_j), J_j = -J_i."""
    Xi, Xj = states
    dl = Xi - Xj
    r = (np.sum(dl * dl, axis=1) - np.asarray(d, float) ** 2)[:, None]
    return r, [(2.0 * dl)[:, None, :], (-2.0 * dl)[:, None, :]]


def problem(x0, circle_ids, radius, distance_pairs=None, distances=None, fixed=None, circle_active=None,
            loss=None):
    """Generic-LM problem: one vertex set of 2-D points (not eliminated), circle edges on
    circle_ids (radius per edge), squared-distance edges on distance_pairs."""
    vs = {"pt": lm.VertexSet("pt", 2, x0, lambda s, d: s + d, False,
                             None if fixed is None else np.asarray(fixed, bool))}
    edges = [lm.EdgeSet("circle", ["pt"], np.asarray(circle_ids, np.int64)[:, None], circle_evaluate,
                        np.asarray(radius, float), None, loss,
                        None if circle_active is None else np.asarray(circle_active, bool))]
    if distance_pairs is not None and len(distance_pairs):
        edges.append(lm.EdgeSet("distance", ["pt", "pt"], np.asarray(distance_pairs, np.int64), distance_evaluate,
                                np.asarray(distances, float), None, loss))
    return lm.Problem(vs, edges)
