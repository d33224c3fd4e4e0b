"""Pins for the oracle's LM: brute-force dense solve vs Schur, the model-decrease
identity, monotone accepted costs, the noise-floor cost at convergence, the Huber
kernel, Nielsen's damping rule and the paper's circle example."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import generic, lm, robust
from paper_2509_26581_gb300 import synth


def _tiny(seed, C=5, P=30, views=4, **kw):
    p = synth.ba_ring(seed, C, P, views, **kw)
    return p


@pytest.mark.parametrize("seed,lam,huber", [(0, 1e-4, None), (1, 1e-1, 2.0), (2, 10.0, 2.0)])
def test_schur_step_equals_dense_full_solve(seed, lam, huber):
    p = _tiny(seed, outlier_frac=0.1 if huber else 0.0)
    prob = lm.ba_problem(p.cams0, p.pts0, p.cam_idx, p.pt_idx, p.obs, huber_delta=huber)
    layout = lm.make_layout(prob)
    lin = lm.linearize(prob, layout)
    H, b = lm.normal_equations(lin)
    D = lm.damping_diagonal(H, lm.LMParams())
    Hl = H + sp.diags(lam * D)
    dx, S, g = lm.schur_solve(Hl, b, layout)
    ref = lm.dense_solve(Hl, b)
    assert np.max(np.abs(dx - ref)) <= 1e-10 * np.max(np.abs(ref))
    # the dense matrix really is J^T J: compare with an explicit dense Jacobian product
    Jd = lin.J.toarray()
    assert np.allclose(H.toarray(), Jd.T @ Jd, rtol=0, atol=1e-9 * np.abs(H).max())


def test_schur_with_fixed_vertices_and_inactive_edges():
    p = _tiny(3)
    cam_fixed = np.zeros(p.n_cams, bool)
    cam_fixed[0] = True
    pt_fixed = np.zeros(p.n_pts, bool)
    pt_fixed[[1, 7]] = True
    active = np.ones(p.n_edges, bool)
    active[::9] = False
    prob = lm.ba_problem(p.cams0, p.pts0, p.cam_idx, p.pt_idx, p.obs, cam_fixed=cam_fixed,
                         pt_fixed=pt_fixed, active=active)
    layout = lm.make_layout(prob)
    assert layout.n_total == 9 * 4 + 3 * 28
    lin = lm.linearize(prob, layout)
    assert lin.J.shape[0] == 2 * int(active.sum())
    H, b = lm.normal_equations(lin)
    Hl = H + sp.diags(1e-3 * lm.damping_diagonal(H, lm.LMParams()))
    dx, _, _ = lm.schur_solve(Hl, b, layout)
    assert np.max(np.abs(dx - lm.dense_solve(Hl, b))) < 1e-10 * np.max(np.abs(dx))
    new = lm.apply_step(prob, layout, dx)
    assert np.array_equal(new["cam"][0], p.cams0[0])
    assert np.array_equal(new["pt"][[1, 7]], p.pts0[[1, 7]])


@pytest.mark.parametrize("lam", [1e-6, 1e-2, 3.0])
def test_model_decrease_identity(lam):
    p = _tiny(4)
    prob = lm.ba_problem(p.cams0, p.pts0, p.cam_idx, p.pt_idx, p.obs, huber_delta=2.0)
    dx, layout, H, b, D, lin = lm.step(prob, lam)
    L = lm.model_decrease(lin, b, dx)
    assert L > 0
    assert abs(L - 0.5 * dx @ (lam * D * dx - b)) < 1e-9 * abs(L)


def test_lm_tiny_monotone_and_noise_floor():
    p = synth.ba_tiny(0)
    prob = lm.ba_problem(p.cams0, p.pts0, p.cam_idx, p.pt_idx, p.obs)
    _, rep = lm.levenberg_marquardt(prob, 20)
    costs = [h["cost"] for h in rep.history] + [rep.final_cost]
    assert all(b <= a for a, b in zip(costs, costs[1:]))
    for h in rep.history:
        if h["accepted"]:
            assert h["cand_cost"] < h["cost"]
    # At the optimum of a Gaussian-noise least-squares problem, 2F ~ chi^2 with
    # 2E - (free parameters - 7 gauge) degrees of freedom (sigma = 1).
    dof = 2 * p.n_edges - (9 * p.n_cams + 3 * p.n_pts - 7)
    assert abs(2 * rep.final_cost - dof) < 5 * np.sqrt(2 * dof)
    assert rep.initial_cost > 10 * rep.final_cost


def test_huber_kernel():
    d = 2.0
    s = np.array([0.0, 1.0, 3.99999999, 4.0, 4.00000001, 9.0, 100.0])
    rho = robust.huber_rho(s, d)
    assert np.allclose(rho[:4], s[:4])
    assert np.allclose(rho[5:], 2 * d * np.sqrt(s[5:]) - d * d)
    # continuity of value and derivative at s = delta^2
    assert abs(rho[2] - rho[4]) < 1e-7
    w = robust.huber_weight(s, d)
    assert np.allclose(w[:4], 1.0) and np.allclose(w[5:], d / np.sqrt(s[5:]))
    # rho'(s) is the derivative of rho: central differences
    for si in (5.0, 30.0, 1.0):
        h = 1e-6
        assert abs((robust.huber_rho(si + h, d) - robust.huber_rho(si - h, d)) / (2 * h)
                   - robust.huber_weight(si, d)) < 1e-8


def test_nielsen_rule():
    assert lm.nielsen_update(1.0, 8.0, 0.5, True) == (1.0, 2.0)          # 1 - 0^3 = 1
    assert lm.nielsen_update(1.0, 8.0, 1.0, True) == (1.0 / 3.0, 2.0)    # max(1/3, 0)
    lam, nu = lm.nielsen_update(1.0, 8.0, 0.25, True)
    assert abs(lam - 1.125) < 1e-15 and nu == 2.0                        # 1 - (-0.5)^3
    assert lm.nielsen_update(3.0, 4.0, -1.0, False) == (12.0, 8.0)


def _circle_problem(n=12, radius=2.0, seed=0):
    rng = np.random.default_rng(seed)
    ang = rng.uniform(0, 2 * np.pi, n)
    rad = radius * rng.uniform(0.5, 1.6, n)
    pts = np.stack([rad * np.cos(ang), rad * np.sin(ang)], axis=1)
    fixed = np.zeros(n, bool)
    fixed[n - 1] = True          # Listing 5: fix the last point
    active = np.ones(n, bool)
    active[2] = False            # Listing 5: disable the constraint of the third point
    vs = {"p": lm.VertexSet("p", 2, pts, lambda s, d: s + d, False, fixed)}
    es = lm.EdgeSet("circle", ["p"], np.arange(n)[:, None], generic.circle_evaluate, radius,
                    None, None, active)
    return lm.Problem(vs, [es]), pts


def test_circle_example_identity_damping_radial_projection():
    prob, pts0 = _circle_problem()
    out, rep = lm.levenberg_marquardt(prob, 10, lm.LMParams(initial_damping=1e-6,
                                                            damping="identity"))
    pts = out.vertices["p"].state
    free = np.ones(len(pts0), bool)
    free[[2, 11]] = False
    proj = 2.0 * pts0[free] / np.linalg.norm(pts0[free], axis=1, keepdims=True)
    # on the circle to rounding; tangential drift only from rounding amplified by 1/lambda
    assert np.max(np.abs(np.linalg.norm(pts[free], axis=1) - 2.0)) < 1e-12
    assert np.max(np.abs(pts[free] - proj)) < 1e-7
    assert np.array_equal(pts[11], pts0[11]) and np.array_equal(pts[2], pts0[2])
    # only the fixed point's constraint keeps a residual
    fixed_term = 0.5 * (pts0[11] @ pts0[11] - 4.0) ** 2
    assert abs(rep.final_cost - fixed_term) < 1e-12 * fixed_term


def test_circle_example_marquardt_damping():
    prob, pts0 = _circle_problem(seed=1)
    out, rep = lm.levenberg_marquardt(prob, 10, lm.LMParams(initial_damping=1e-6))
    pts = out.vertices["p"].state
    free = np.ones(len(pts0), bool)
    free[[2, 11]] = False
    assert np.max(np.abs(np.linalg.norm(pts[free], axis=1) - 2.0)) < 1e-9
    assert np.array_equal(pts[11], pts0[11]) and np.array_equal(pts[2], pts0[2])


# ---------------------------------------------------------------- damping clamps
# Sec. IV-E clamps the Hessian diagonal that scales the damping; the bounds
# (1e-6, 1e32) and the damping bounds (1e-16, 1e32) are this library's readings.

def _scalar_problem(a, y, x0, active=None):
    """Independent scalar unknowns x_i with linear residuals r_i = a_i x_i - y_i:
    H = diag(a^2), b = a r, so every quantity of a damped step has a closed form."""
    a, y = np.asarray(a, float), np.asarray(y, float)
    n = len(a)

    def evaluate(states, data):
        (x,) = states
        return (data[:, 0] * x[:, 0] - data[:, 1])[:, None], [data[:, 0][:, None, None]]

    vs = {"x": lm.VertexSet("x", 1, np.asarray(x0, float).reshape(n, 1), lambda s, d: s + d)}
    es = lm.EdgeSet("lin", ["x"], np.arange(n)[:, None], evaluate, np.stack([a, y], axis=1),
                    None, None, active)
    return lm.Problem(vs, [es])


def test_damping_diagonal_clamp_values():
    d = np.array([1e-9, 0.0, -3.0, 1e-6, 5.0, 1e32, 1e40, 2.5e31])
    H = sp.diags(d) + sp.csr_matrix(np.triu(np.ones((8, 8)), 1))   # off-diagonal entries are ignored
    D = lm.damping_diagonal(H, lm.LMParams())
    assert np.array_equal(D, [1e-6, 1e-6, 1e-6, 1e-6, 5.0, 1e32, 1e32, 2.5e31])
    D = lm.damping_diagonal(H, lm.LMParams(diag_min=0.5, diag_max=10.0))
    assert np.array_equal(D, [0.5, 0.5, 0.5, 0.5, 5.0, 10.0, 10.0, 10.0])
    assert np.array_equal(lm.damping_diagonal(H, lm.LMParams(damping="identity")), np.ones(8))


@pytest.mark.parametrize("lam", [1e-4, 1.0, 1e3])
def test_damped_step_closed_form_with_clamped_diagonal(lam):
    # H_ii = a_i^2 below, inside and above the clamp range: the step of Eq. 5 with the
    # Marquardt scaling is dx_i = -a_i r_i / (a_i^2 + lam clamp(a_i^2, 1e-6, 1e32))
    a = np.array([1e-4, 3.0, 1e20])
    y = np.array([2.0, -1.0, 5.0])
    x0 = np.array([0.7, 0.2, 3e-20])
    dx, _, H, b, D, _ = lm.step(_scalar_problem(a, y, x0), lam)
    r = a * x0 - y
    expect = -a * r / (a * a + lam * np.array([1e-6, 9.0, 1e32]))
    assert np.allclose(dx, expect, rtol=1e-14, atol=0)


def test_lambda_rises_to_upper_bound_at_exact_optimum():
    # r = 0 at x0: b = 0, dx = 0, model decrease 0, so every step is rejected and
    # Nielsen's rule multiplies lambda by nu = 2, 4, 8, ...: lambda_k = lambda_0 2^(k(k+1)/2)
    # until the clamp at lambda_max holds it there.
    a = np.array([2.0, -0.5])
    x0 = np.array([1.5, 4.0])
    prob = _scalar_problem(a, a * x0, x0)
    prm = lm.LMParams(initial_damping=1e-4, lambda_max=1.0)
    _, rep = lm.levenberg_marquardt(prob, 8, prm)
    lams = [h["lam"] for h in rep.history]
    expect = [min(1e-4 * 2.0 ** (k * (k + 1) // 2), 1.0) for k in range(8)]
    assert np.allclose(lams, expect, rtol=1e-15, atol=0)
    assert lams[-1] == 1.0 and rep.final_lambda == 1.0 and rep.accepted == 0
    assert rep.final_cost == 0.0


def test_lambda_falls_to_lower_bound_on_linear_problem():
    # A linear residual has an exact quadratic model, so rho = 1 on every step and
    # lambda shrinks by max(1/3, 1 - (2 rho - 1)^3) = 1/3 until lambda_min holds it.
    a = np.array([1.0, 2.0, 0.5])
    y = np.array([3.0, -1.0, 2.0])
    prob = _scalar_problem(a, y, np.zeros(3))
    prm = lm.LMParams(initial_damping=1e3, lambda_min=10.0)
    _, rep = lm.levenberg_marquardt(prob, 8, prm)
    assert rep.accepted == 8
    for h in rep.history:
        assert abs(h["rho"] - 1.0) < 1e-9
    lams = [h["lam"] for h in rep.history]
    expect = [max(1e3 / 3.0 ** k, 10.0) for k in range(8)]
    assert np.allclose(lams, expect, rtol=1e-14, atol=0)
    assert rep.final_lambda == 10.0
    # each accepted step scales the residual by lambda D / (H + lambda D) = lambda / (1 + lambda)
    r = -y.copy()
    for lam in lams:
        r = r * lam / (1.0 + lam)
    assert abs(rep.final_cost - 0.5 * r @ r) <= 1e-12 * rep.final_cost
