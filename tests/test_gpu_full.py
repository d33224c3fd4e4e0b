"""GPU parity of the full-system PCG (GPO_SOLVER_FULL: block-Jacobi PCG on cameras and
points together, the paper's form of the solve) against the FP64 oracle, through the
C ABI.

The oracle solves the damped normal equations exactly (Schur elimination and dense
Cholesky); an exact solve of the full system gives the same step, which a direct
sparse solve of the full damped system also pins here.  Tolerances (written here,
derived from the arithmetic):
  * one LM step by full-system PCG to 1e-14 relative residual vs the exact step:
    1e-8 relative (stopping error times the condition number of the full system);
  * final cost after 20 LM iterations on the 10-camera problem, FP64: 1e-9 relative;
  * mixed precision (FP32, BF16 storage) vs FP64 on a converged problem: 1e-6;
  * the Schur and full forms in FP64 on a 12-keyframe visual-inertial problem: final
    cost 1e-9 relative.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import lm as olm
from paper_2509_26581_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpo():
    from paper_2509_26581_gb300 import gpo as m
    return m


def _oracle_problem(p):
    return olm.ba_problem(p.cams0, p.pts0, p.cam_idx, p.pt_idx, p.obs, huber_delta=p.huber_delta)


def _full_params(gpo, **kw):
    base = dict(pcg_max_iters=3000, pcg_tol=1e-14, pcg_tol_relative=1, pcg_rejection_ratio=0.0,
                solver=gpo.GPO_SOLVER_FULL)
    base.update(kw)
    return gpo.default_params(**base)


@pytest.mark.parametrize("lam", [1e-4, 1e-1])
def test_full_system_step_matches_the_exact_step(gpo, lam):
    p = synth.ba_tiny(0)
    prob = _oracle_problem(p)
    layout = olm.make_layout(prob)
    H, b = olm.normal_equations(olm.linearize(prob, layout))
    D = olm.damping_diagonal(H, olm.LMParams())
    Hl = (H + sp.diags(lam * D)).tocsc()
    dxo, _, _ = olm.schur_solve(Hl, b, layout)
    dxd = spla.spsolve(Hl, -b)                    # the full system, solved directly
    assert np.abs(dxd - dxo).max() <= 1e-9 * np.abs(dxo).max()
    g, _, _ = gpo.ba_graph(p.cams0, p.pts0, p.cam_idx, p.pt_idx, p.obs, None, "fp64")
    dx, iters = g.debug_step(lam, 9 * p.n_cams + 3 * p.n_pts, _full_params(gpo))
    assert np.abs(dx - dxo).max() <= 1e-8 * np.abs(dxo).max()
    assert 0 < iters <= 3000


def test_full_system_lm_matches_the_oracle(gpo):
    p = synth.ba_tiny(0)
    g, _, _ = gpo.ba_graph(p.cams0, p.pts0, p.cam_idx, p.pt_idx, p.obs, None, "fp64")
    rep = g.optimize(20, _full_params(gpo))
    _, orep = olm.levenberg_marquardt(_oracle_problem(p), 20)
    assert abs(rep.initial_cost - orep.initial_cost) <= 1e-12 * orep.initial_cost
    assert abs(rep.final_cost - orep.final_cost) <= 1e-9 * orep.final_cost


def test_full_system_restarts_match_the_oracle(gpo):
    """True-residual restarts (r = g - H x over cameras and points every 25
    iterations): the LM run still matches the oracle, one extra product per restart."""
    p = synth.ba_ring(0, 10, 500, 6)
    g, _, _ = gpo.ba_graph(p.cams0, p.pts0, p.cam_idx, p.pt_idx, p.obs, None, "fp64")
    rep = g.optimize(10, _full_params(gpo, pcg_restart_every=25))
    _, orep = olm.levenberg_marquardt(_oracle_problem(p), 10)
    assert abs(rep.final_cost - orep.final_cost) <= 1e-9 * orep.final_cost
    hist = g.history()
    assert any(h["pcg_iters"] > 25 for h in hist)
    for h in hist:
        restarts = h["pcg_products"] - h["pcg_iters"]
        assert restarts == (h["pcg_iters"] - 1) // 25 or restarts == h["pcg_iters"] // 25


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_full_system_mixed_precision_close_to_fp64(gpo, prec):
    p = synth.ba_ring(7, 20, 4000, 6, outlier_frac=0.01, huber_delta=2.0)
    g, _, _ = gpo.ba_graph(p.cams0, p.pts0, p.cam_idx, p.pt_idx, p.obs, p.huber_delta, "fp64")
    ref = g.optimize(30).final_cost
    h, _, _ = gpo.ba_graph(p.cams0, p.pts0, p.cam_idx, p.pt_idx, p.obs, p.huber_delta, prec)
    params = gpo.default_params(pcg_max_iters=400, pcg_tol=1e-6, solver=gpo.GPO_SOLVER_FULL)
    cost = h.optimize(30, params).final_cost
    assert abs(cost - ref) <= 1e-6 * ref


def test_full_system_captured_groups_bitwise(gpo):
    """Captured PCG groups (production) and direct launches (profiling) give the same
    full-system solve bit for bit; the graph's footprint counts the point vectors."""
    p = synth.ba_path(4, 40, 6000, "pareto")
    out = []
    for prof in (False, True):
        g, c0, p0 = gpo.ba_graph(p.cams0, p.pts0, p.cam_idx, p.pt_idx, p.obs, p.huber_delta, "fp32")
        before = g.footprint()
        g.set_profiling(prof)
        rep = g.optimize(4, gpo.default_params(pcg_max_iters=60, pcg_tol=1e-12, solver=gpo.GPO_SOLVER_FULL))
        assert g.footprint() >= before + 7 * 3 * 4 * p.n_pts
        out.append((rep.final_cost, rep.pcg_iters_total, g.get_state(c0, p.n_cams, 9), g.get_state(p0, p.n_pts, 3)))
        assert rep.pcg_iters_total > 16
    assert out[0][0] == out[1][0] and out[0][1] == out[1][1]
    assert np.array_equal(out[0][2], out[1][2]) and np.array_equal(out[0][3], out[1][3])


def test_full_and_schur_forms_agree_on_visual_inertial(gpo):
    """Navigation states with inertial, bias and stereo edges (the camera-side coupling
    blocks enter the full system's camera rows): both forms, FP64, same final cost."""
    p = synth.vi_problem(6, n_kf=12, n_pts=400)
    costs = []
    for solver in (gpo.GPO_SOLVER_SCHUR, gpo.GPO_SOLVER_FULL):
        g, _, _, _ = gpo.vi_graph(p, precision="fp64")
        params = gpo.default_params(pcg_max_iters=3000, pcg_tol=1e-12, pcg_rejection_ratio=0.0, solver=solver)
        costs.append(g.optimize(15, params).final_cost)
    assert abs(costs[1] - costs[0]) <= 1e-9 * costs[0]


def test_full_system_fixed_and_disabled_vertices(gpo):
    """A fixed camera, a fixed point and a point that loses every observation stay where
    they are, and the run matches the oracle (whose exact steps eliminate them)."""
    p = synth.ba_ring(4, 8, 200, 5)
    cam_fixed = np.zeros(p.n_cams, bool)
    cam_fixed[0] = True
    pt_fixed = np.zeros(p.n_pts, bool)
    pt_fixed[5] = True
    active = np.ones(p.n_edges, bool)
    active[p.pt_idx == 9] = False
    g, c0, p0 = gpo.ba_graph(p.cams0, p.pts0, p.cam_idx, p.pt_idx, p.obs, None, "fp64",
                             cam_fixed=cam_fixed, pt_fixed=pt_fixed, active=active)
    rep = g.optimize(10, _full_params(gpo))
    cams, pts = g.get_state(c0, p.n_cams, 9), g.get_state(p0, p.n_pts, 3)
    assert np.array_equal(cams[0], p.cams0[0])
    assert np.array_equal(pts[5], p.pts0[5]) and np.array_equal(pts[9], p.pts0[9])
    prob = olm.ba_problem(p.cams0, p.pts0, p.cam_idx, p.pt_idx, p.obs, cam_fixed=cam_fixed,
                          pt_fixed=pt_fixed, active=active)
    _, orep = olm.levenberg_marquardt(prob, 10)
    assert abs(rep.final_cost - orep.final_cost) <= 1e-9 * orep.final_cost


def test_batched_solves_use_the_schur_form(gpo):
    """Graphs solved together share launches in the Schur form: asking for the full
    system there gives the Schur results bit for bit."""
    from paper_2509_26581_gb300 import serving
    wins = synth.window_pool(5, 3, kf=(5, 8), pts=(200, 600))
    out = []
    for solver in (gpo.GPO_SOLVER_SCHUR, gpo.GPO_SOLVER_FULL):
        built = [serving.window_graph(w, "fp32") for w in wins]
        reps = gpo.optimize_batch([b[0] for b in built], 4, gpo.default_params(solver=solver))
        out.append([(r.final_cost, r.pcg_iters_total) for r in reps])
    assert out[0] == out[1]
