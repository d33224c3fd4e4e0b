"""Pins of the generic-edge oracle (the paper's circle example): its Jacobians against
central differences, and its LM run against the closed form — with identity damping
every step of a point lies along its constraint's gradient (the radius), so every free
point with an active circle constraint ends on its radial projection onto the circle,
with zero cost; a fixed point and a point whose only constraint is disabled do not
move."""
import numpy as np

from oracle import generic as og
from oracle import lm


def _points(seed, n):
    rng = np.random.default_rng(seed)
    ang = rng.uniform(0, 2 * np.pi, n)
    rad = rng.uniform(0.5, 3.0, n)
    return np.stack([rad * np.cos(ang), rad * np.sin(ang)], axis=1)


def test_jacobians_central_differences():
    rng = np.random.default_rng(0)
    X = rng.normal(size=(20, 2))
    Y = rng.normal(size=(20, 2))
    R = rng.uniform(0.5, 2, 20)
    d = rng.uniform(0.5, 2, 20)
    eps = 1e-6
    _, (J,) = og.circle_evaluate([X], R)
    _, (Ji, Jj) = og.distance_evaluate([X, Y], d)
    for k in range(2):
        e = np.zeros(2)
        e[k] = eps
        fd = (og.circle_evaluate([X + e], R)[0] - og.circle_evaluate([X - e], R)[0]) / (2 * eps)
        assert np.abs(fd[:, 0] - J[:, 0, k]).max() < 1e-8
        fdi = (og.distance_evaluate([X + e, Y], d)[0] - og.distance_evaluate([X - e, Y], d)[0]) / (2 * eps)
        fdj = (og.distance_evaluate([X, Y + e], d)[0] - og.distance_evaluate([X, Y - e], d)[0]) / (2 * eps)
        assert np.abs(fdi[:, 0] - Ji[:, 0, k]).max() < 1e-8
        assert np.abs(fdj[:, 0] - Jj[:, 0, k]).max() < 1e-8


def test_circle_example_closed_form():
    x0 = _points(1, 50)
    R = 1.5
    fixed = np.zeros(50, bool)
    fixed[3] = True
    active = np.ones(50, bool)
    active[7] = False
    prob = og.problem(x0, np.arange(50), np.full(50, R), fixed=fixed, circle_active=active)
    out, rep = lm.levenberg_marquardt(prob, 30, lm.LMParams(damping="identity"))
    x = out.vertices["pt"].state
    free = ~fixed & active
    proj = x0 * (R / np.linalg.norm(x0, axis=1))[:, None]
    assert np.abs(x[free] - proj[free]).max() < 1e-9
    assert np.array_equal(x[3], x0[3]) and np.array_equal(x[7], x0[7])
    # the fixed point keeps its (nonzero) share of the cost; everything else is zero
    s3 = (x0[3] @ x0[3] - R * R) ** 2 / 2
    assert abs(rep.final_cost - s3) <= 1e-12 * max(s3, 1.0)
