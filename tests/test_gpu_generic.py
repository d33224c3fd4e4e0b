"""Generic edge kinds (gpo_generic_*: residuals differentiated in forward mode on the
GPU) against the generic-edge oracle, through the C ABI.

Tolerances (written here, derived from the arithmetic): FP64 on both sides with exact
(oracle) and 1e-14-relative PCG (library) steps, so LM runs agree to 1e-9 relative in
cost and 1e-7 in the states; the circle example's closed form (radial projection) to
1e-9.
"""
import numpy as np
import pytest

from oracle import generic as og
from oracle import lm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpo():
    from paper_2509_26581_gb300 import gpo as m
    return m


def _points(seed, n):
    rng = np.random.default_rng(seed)
    ang = rng.uniform(0, 2 * np.pi, n)
    rad = rng.uniform(0.5, 3.0, n)
    return np.stack([rad * np.cos(ang), rad * np.sin(ang)], axis=1)


def _params(gpo, **kw):
    return gpo.default_params(pcg_max_iters=200, pcg_tol=1e-14, pcg_rejection_ratio=0.0, **kw)


def test_circle_example(gpo):
    """The paper's running example: 2-D points pulled onto a circle (identity damping),
    one fixed point, one disabled constraint."""
    x0 = _points(1, 50)
    R = 1.5
    g = gpo.Generic(x0)
    g.add_edges(gpo.GPO_GE_CIRCLE, np.arange(50)[:, None], np.full((50, 1), R))
    g.set_fixed(3)
    g.set_edge_active(7, False)
    rep = g.optimize(30, _params(gpo, damping_mode=1))
    x = g.state()
    free = np.ones(50, bool)
    free[[3, 7]] = False
    proj = x0 * (R / np.linalg.norm(x0, axis=1))[:, None]
    assert np.abs(x[free] - proj[free]).max() < 1e-9
    assert np.array_equal(x[3], x0[3]) and np.array_equal(x[7], x0[7])
    fixed = np.zeros(50, bool)
    fixed[3] = True
    active = np.ones(50, bool)
    active[7] = False
    _, orep = lm.levenberg_marquardt(og.problem(x0, np.arange(50), np.full(50, R), fixed=fixed,
                                                circle_active=active), 30, lm.LMParams(damping="identity"))
    assert abs(rep.initial_cost - orep.initial_cost) <= 1e-12 * orep.initial_cost
    assert abs(rep.final_cost - orep.final_cost) <= 1e-9 * max(orep.final_cost, 1e-12)


@pytest.mark.parametrize("huber", [None, 0.5])
def test_circle_and_distance_edges_match_the_oracle(gpo, huber):
    """Binary squared-distance edges between neighbours beside the circle edges (an
    n-ary coupling the full-system PCG has to solve), Marquardt damping, with and
    without the Huber loss."""
    n = 40
    x0 = _points(2, n)
    R = 2.0
    pairs = np.stack([np.arange(n), (np.arange(n) + 1) % n], axis=1)
    d = np.full(n, 2 * R * np.sin(np.pi / n))
    loss = None if huber is None else ("huber", huber)
    g = gpo.Generic(x0)
    kw = {} if huber is None else dict(loss_kind=gpo.GPO_LOSS_HUBER, loss_delta=huber)
    g.add_edges(gpo.GPO_GE_CIRCLE, np.arange(n)[:, None], np.full((n, 1), R), **kw)
    g.add_edges(gpo.GPO_GE_DISTANCE, pairs, d[:, None], **kw)
    rep = g.optimize(15, _params(gpo))
    prob = og.problem(x0, np.arange(n), np.full(n, R), pairs, d, loss=loss)
    out, orep = lm.levenberg_marquardt(prob, 15)
    assert abs(rep.initial_cost - orep.initial_cost) <= 1e-12 * orep.initial_cost
    assert abs(rep.final_cost - orep.final_cost) <= 1e-9 * orep.final_cost
    assert rep.accepted == orep.accepted
    assert np.abs(g.state() - out.vertices["pt"].state).max() < 1e-7
