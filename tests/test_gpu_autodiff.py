"""Forward-mode automatic differentiation of the edges (gpo_debug_autodiff_edges) against
the analytic Jacobians of the linearisation kernels and against the oracle, through
the C ABI.

Tolerances (written here, derived from the arithmetic): dual numbers and the analytic
formulas evaluate the same FP64 expressions in a different order, so per-edge rows
agree to 1e-12 relative to the edge's largest entry (1e-11 for the stereo rows, whose
projection goes through two rotations), residuals near the optimum to 1e-10 absolute
(the rounding of projections of a few hundred pixels); against the rows a BF16 graph
stores, the storage rounding (2^-8) bounds the difference.
"""
import numpy as np
import pytest

from oracle import ba as oba
from oracle import robust
from paper_2509_26581_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpo():
    from paper_2509_26581_gb300 import gpo as m
    return m


def _edge_rel(a, b, floor):
    a = a.reshape(a.shape[0], -1)
    b = b.reshape(b.shape[0], -1)
    scale = np.maximum(np.abs(b).max(axis=1), floor)
    return (np.abs(a - b).max(axis=1) / scale).max()


@pytest.mark.parametrize("case", ["tiny", "huber_outliers", "info", "fixed_inactive"])
def test_autodiff_rows_match_the_analytic_rows_fp64(gpo, case):
    if case == "tiny":
        p = synth.ba_tiny(0)
    else:
        p = synth.ba_ring(11, 12, 400, 5, outlier_frac=0.05, huber_delta=2.0)
    info = active = cam_fixed = pt_fixed = None
    if case == "info":
        rng = np.random.default_rng(0)
        A = rng.normal(size=(p.n_edges, 2, 2))
        info = A @ np.transpose(A, (0, 2, 1)) + 0.5 * np.eye(2)
    if case == "fixed_inactive":
        cam_fixed = np.zeros(p.n_cams, bool)
        cam_fixed[[0, 3]] = True
        pt_fixed = np.zeros(p.n_pts, bool)
        pt_fixed[::17] = True
        active = np.ones(p.n_edges, bool)
        active[::7] = False
    g, _, _ = gpo.ba_graph(p.cams0, p.pts0, p.cam_idx, p.pt_idx, p.obs, p.huber_delta, "fp64",
                           cam_fixed=cam_fixed, pt_fixed=pt_fixed, active=active, info=info)
    ids = np.arange(p.n_edges)
    r, J = g.debug_linearize_edges(ids)
    ra, Ja = g.debug_autodiff_edges(ids)
    assert _edge_rel(ra, r, 1e-9) < 1e-12
    assert _edge_rel(Ja, J, 1e-9) < 1e-12
    if active is not None:
        assert np.all(ra[~active] == 0) and np.all(Ja[~active] == 0)


def test_autodiff_rows_match_the_oracle_after_steps(gpo):
    """Away from the start (after three LM iterations), against the oracle's analytic
    Jacobians at the graph's current state."""
    p = synth.ba_ring(3, 10, 300, 5, outlier_frac=0.05, huber_delta=2.0)
    g, c0, p0 = gpo.ba_graph(p.cams0, p.pts0, p.cam_idx, p.pt_idx, p.obs, p.huber_delta, "fp64")
    g.optimize(3)
    cams, pts = g.get_state(c0, p.n_cams, 9), g.get_state(p0, p.n_pts, 3)
    ra, Ja = g.debug_autodiff_edges(np.arange(p.n_edges))
    c, X = cams[p.cam_idx], pts[p.pt_idx]
    ro = oba.residual(c, X, p.obs)
    Jc, Jp = oba.jacobians(c, X)
    w = np.sqrt(robust.weight(np.sum(ro * ro, axis=1), ("huber", p.huber_delta)))
    Jo = np.concatenate([Jc, Jp], axis=2) * w[:, None, None]
    # near the optimum a residual is the small difference u - z of projections of a few
    # hundred pixels: rounding of u (~1e-16 x 1e2) sets its floor, not the row's size
    assert np.abs(ra - ro * w[:, None]).max() < 1e-10
    assert _edge_rel(Ja, Jo, 1e-9) < 1e-12


def test_autodiff_bounds_the_bf16_rows(gpo):
    p = synth.ba_ring(5, 12, 400, 5, outlier_frac=0.02, huber_delta=2.0)
    g, _, _ = gpo.ba_graph(p.cams0, p.pts0, p.cam_idx, p.pt_idx, p.obs, p.huber_delta, "bf16")
    ids = np.arange(p.n_edges)
    _, J = g.debug_linearize_edges(ids)
    _, Ja = g.debug_autodiff_edges(ids)
    assert _edge_rel(J, Ja, 1e-9) < 2.0 ** -7


def test_autodiff_stereo_rows_match_the_analytic_rows(gpo):
    p = synth.vi_problem(5, n_kf=8, n_pts=200)
    g, _, _, rg = gpo.vi_graph(p, precision="fp64", imu=None)
    a, b = rg["stereo"]
    ids = np.arange(a, b)
    r, J = g.debug_linearize_edges(ids, nav=True)
    ra, Ja = g.debug_autodiff_edges(ids, nav=True)
    assert _edge_rel(ra[:, :3], r[:, :3], 1e-9) < 1e-11
    assert _edge_rel(Ja[:, :3], J[:, :3], 1e-9) < 1e-11
    # camera-side edges have no observation rows to differentiate here
    n_ids = rg["bias_prior"][1]
    rest = np.arange(b, n_ids)
    rz, Jz = g.debug_autodiff_edges(rest, nav=True)
    assert np.all(rz == 0) and np.all(Jz == 0)
