"""GPU parity of the visual-inertial path (stereo reprojection on navigation states,
inertial, bias random-walk and bias-prior edges) against the FP64 oracle, through the
C ABI.

The graphs here take the oracle's preintegrated measurements and information
matrices, so both sides evaluate the same edges (the library's own preintegration is
pinned against the oracle's in test_vi_host.py).  Tolerances (derived from the
arithmetic):
  * per-edge residual and Jacobian, FP64: 1e-12 relative to the edge's largest entry
    (stereo); inertial edges 1e-11: their whitening U has entries up to ~1e5 and the
    residual's rotation part comes from a logarithm of a product of four rotations,
    each side rounding differently;
  * cost: 1e-12 relative;
  * Schur blocks and reduced right-hand side, FP64: 1e-10 relative to the largest entry
    of the block (the inertial terms make the 15x15 blocks span ~10 orders of magnitude,
    so small entries are compared against the block scale);
  * one LM step, PCG to 1e-14 relative residual vs dense Cholesky: 1e-7 relative (the
    reduced system's condition number is ~1e6 higher than in bundle adjustment);
  * final cost after 15 LM iterations: 1e-9 relative;
  * mixed precision (FP32, BF16 storage) vs FP64 on the GPU: 1e-6 relative, once both
    have converged (PCG run to 1e-10 relative, 30 LM iterations).
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import lm as olm
from oracle import robust
from oracle import vi as ovi
from paper_2509_26581_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpo():
    from paper_2509_26581_gb300 import gpo as m
    return m


@pytest.fixture(scope="module")
def small():
    p = synth.vi_problem(5, n_kf=8, n_pts=200)
    return p, ovi.preintegrate_all(p)


def _records(pims):
    meas = np.stack([np.r_[pm["dR"].ravel(), pm["dv"], pm["dp"], pm["JRg"].ravel(), pm["Jvg"].ravel(),
                           pm["Jva"].ravel(), pm["Jpg"].ravel(), pm["Jpa"].ravel(), pm["T"], pm["bg0"],
                           pm["ba0"]] for pm in pims])
    info = np.stack([np.linalg.inv(pm["cov"]) for pm in pims])
    return meas, info


def _graph(gpo, p, pims, precision="fp64", **kw):
    return gpo.vi_graph(p, precision=precision, imu=_records(pims), **kw)


def _rel_rows(a, b, floor=1e-300):
    a = a.reshape(a.shape[0], -1)
    b = b.reshape(b.shape[0], -1)
    scale = np.maximum(np.abs(b).max(axis=1), floor)
    return (np.abs(a - b).max(axis=1) / scale).max()


def _oracle_rows(p, pims, nav, pts, prior_sigma=(1e-2, 1e-1)):
    """Whitened, Huber-weighted rows of every edge, in the graph's edge order."""
    cam = ovi.camera_of(p.camera)
    r, (Jn, Jp) = cam.evaluate((nav[p.kf_idx], pts[p.pt_idx]), p.obs)
    w = np.sqrt(robust.weight(np.sum(r * r, axis=1), ("huber", p.huber_delta)))
    st_r = r * w[:, None]
    st_J = np.concatenate([Jn, Jp], axis=2) * w[:, None, None]
    K = nav.shape[0]
    imu_r, imu_J = [], []
    for k, pm in enumerate(pims):
        U = np.linalg.cholesky(np.linalg.inv(pm["cov"])).T
        rr = ovi.imu_residual_one(pm, nav[k:k + 1], nav[k + 1:k + 2])
        Ji, Jj = ovi.imu_jacobians_one(pm, nav[k:k + 1], nav[k + 1:k + 2])
        imu_r.append(U @ rr)
        imu_J.append(np.concatenate([U @ Ji, U @ Jj], axis=1))
    T = np.array([pm["T"] for pm in pims])
    rw_r, rw_J = [], []
    for k in range(K - 1):
        u = np.r_[np.full(3, 1 / np.sqrt(p.noise["sigma_bg"] ** 2 * T[k])),
                  np.full(3, 1 / np.sqrt(p.noise["sigma_ba"] ** 2 * T[k]))]
        rr, (Ji, Jj) = ovi.bias_rw_evaluate((nav[k:k + 1], nav[k + 1:k + 2]), None)
        rw_r.append(u * rr[0])
        rw_J.append(np.concatenate([u[:, None] * Ji[0], u[:, None] * Jj[0]], axis=1))
    u = np.r_[np.full(3, 1 / prior_sigma[0]), np.full(3, 1 / prior_sigma[1])]
    pr, (Jpr,) = ovi.bias_prior_evaluate((nav[0:1],), np.zeros((1, 6)))
    return (st_r, st_J), (np.array(imu_r), np.array(imu_J)), (np.array(rw_r), np.array(rw_J)), \
        (u * pr, u[None, :, None] * Jpr)


def test_edge_rows_fp64(gpo, small):
    p, pims = small
    g, n0, p0, rg = _graph(gpo, p, pims)
    n_ids = rg["bias_prior"][1]
    r, J = g.debug_linearize(n_ids, nav=True)
    (sr, sJ), (ir, iJ), (wr, wJ), (pr, pJ) = _oracle_rows(p, pims, p.nav0, p.pts0)
    a, b = rg["stereo"]
    assert _rel_rows(r[a:b, :3], sr) < 1e-12
    assert np.all(r[a:b, 3:] == 0)
    Jg = np.concatenate([J[a:b, :3, :15], J[a:b, :3, 15:18]], axis=2)
    assert _rel_rows(Jg, sJ) < 1e-12
    assert np.all(J[a:b, :3, 6:15] == 0) and np.all(J[a:b, :3, 18:] == 0)
    a, b = rg["imu"]
    assert _rel_rows(r[a:b], ir) < 1e-11
    assert _rel_rows(J[a:b], iJ) < 1e-11
    a, b = rg["bias_rw"]
    assert _rel_rows(r[a:b, :6], wr) < 1e-12 and _rel_rows(J[a:b, :6], wJ) < 1e-12
    a, b = rg["bias_prior"]
    assert _rel_rows(r[a:b, :6], pr, 1e-30) < 1e-12 or np.abs(r[a:b, :6] - pr).max() < 1e-15
    assert _rel_rows(J[a:b, :6, :15], pJ) < 1e-12
    F = olm.total_cost(ovi.problem(p, p.nav0, p.pts0, pims))
    assert abs(g.cost() - F) <= 1e-12 * F


def test_edge_rows_away_from_the_start(gpo, small):
    """Rows at a perturbed state with nonzero biases (the bias-correction terms of the
    inertial residual are exercised)."""
    p, pims = small
    rng = np.random.default_rng(3)
    nav = p.nav0.copy()
    nav[:, 10:13] += rng.normal(scale=2e-3, size=(nav.shape[0], 3))
    nav[:, 13:16] += rng.normal(scale=5e-2, size=(nav.shape[0], 3))
    nav[:, 7:10] += rng.normal(scale=1e-2, size=(nav.shape[0], 3))
    g, n0, p0, rg = _graph(gpo, p, pims, nav=nav)
    r, J = g.debug_linearize(rg["bias_prior"][1], nav=True)
    _, (ir, iJ), (wr, wJ), _ = _oracle_rows(p, pims, nav, p.pts0)
    a, b = rg["imu"]
    assert _rel_rows(r[a:b], ir) < 1e-11
    assert _rel_rows(J[a:b], iJ) < 1e-11
    a, b = rg["bias_rw"]
    assert _rel_rows(r[a:b, :6], wr) < 1e-12


def _oracle_schur(p, pims, lam):
    prob = ovi.problem(p, p.nav0, p.pts0, pims)
    layout = olm.make_layout(prob)
    lin = olm.linearize(prob, layout)
    H, b = olm.normal_equations(lin)
    D = olm.damping_diagonal(H, olm.LMParams())
    Hl = H + sp.diags(lam * D)
    return olm.schur_solve(Hl, b, layout)


@pytest.mark.parametrize("lam", [1e-4, 1.0])
def test_schur_blocks_and_rhs_fp64(gpo, small, lam):
    p, pims = small
    g, _, _, _ = _graph(gpo, p, pims)
    K = p.n_kf
    S, gv = g.debug_schur(lam, K, db=15)
    _, So, go = _oracle_schur(p, pims, lam)
    for c in range(K):
        blk = So[15 * c:15 * c + 15, 15 * c:15 * c + 15]
        assert np.abs(S[c] - blk).max() <= 1e-10 * np.abs(blk).max()
        gb = go[15 * c:15 * c + 15]
        assert np.abs(gv[c] - gb).max() <= 1e-10 * np.abs(go).max()


def _parity_params(gpo, **kw):
    return gpo.default_params(pcg_max_iters=2000, pcg_tol=1e-14, pcg_tol_relative=1,
                              pcg_rejection_ratio=0.0, **kw)


@pytest.mark.parametrize("lam", [1e-4, 1e-1])
def test_one_step_matches_dense_cholesky(gpo, small, lam):
    p, pims = small
    g, _, _, _ = _graph(gpo, p, pims)
    n = 15 * p.n_kf + 3 * p.n_pts
    dx, iters = g.debug_step(lam, n, _parity_params(gpo))
    dxo, _, _ = _oracle_schur(p, pims, lam)
    assert np.abs(dx - dxo).max() <= 1e-7 * np.abs(dxo).max()
    assert 0 < iters <= 2000


def test_lm_final_cost_matches_oracle(gpo, small):
    p, pims = small
    g, n0, p0, _ = _graph(gpo, p, pims)
    rep = g.optimize(15, _parity_params(gpo))
    _, orep = olm.levenberg_marquardt(ovi.problem(p, p.nav0, p.pts0, pims), 15)
    assert abs(rep.initial_cost - orep.initial_cost) <= 1e-12 * orep.initial_cost
    assert abs(rep.final_cost - orep.final_cost) <= 1e-9 * orep.final_cost
    for h, o in zip(g.history(), orep.history):
        if abs(o["cost"] - o["cand_cost"]) > 1e-8 * o["cost"]:
            assert h["accepted"] == o["accepted"]
        assert abs(h["cost"] - o["cost"]) <= 1e-9 * o["cost"]
    nav = g.get_state(n0, p.n_kf, 16)
    assert np.allclose(np.linalg.norm(nav[:, :4], axis=1), 1.0, atol=1e-14)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_mixed_precision_close_to_fp64(gpo, prec):
    # The inertial chain couples neighbouring keyframes strongly, which block-Jacobi
    # leaves to the PCG iterations: their residual norm rises by orders of magnitude
    # before it falls, so the rejection-ratio guard is off (ratio inf) and the PCG runs
    # to 1e-10; then every precision converges to the optimum within 30 LM iterations.
    p = synth.vi_problem(6, n_kf=12, n_pts=400)
    prm = gpo.default_params(pcg_max_iters=500, pcg_tol=1e-10, pcg_rejection_ratio=0.0)
    costs = {}
    for pr in ("fp64", prec):
        g, _, _, _ = gpo.vi_graph(p, precision=pr)
        costs[pr] = g.optimize(30, prm).final_cost
    assert abs(costs[prec] - costs["fp64"]) <= 1e-6 * costs["fp64"]
    _, orep = olm.levenberg_marquardt(ovi.problem(p, p.nav0, p.pts0, ovi.preintegrate_all(p)), 30)
    assert abs(costs["fp64"] - orep.final_cost) <= 1e-9 * orep.final_cost


def test_library_preintegration_graph_matches_oracle(gpo, small):
    """The graph built with the library's own preintegration reaches the oracle's cost."""
    p, pims = small
    g, _, _, _ = gpo.vi_graph(p, precision="fp64")
    rep = g.optimize(15, _parity_params(gpo))
    _, orep = olm.levenberg_marquardt(ovi.problem(p, p.nav0, p.pts0, pims), 15)
    assert abs(rep.final_cost - orep.final_cost) <= 1e-9 * orep.final_cost


def test_huber_inertial_edges_match_the_oracle(gpo, small):
    """Huber loss on the inertial edges (threshold: the median whitened residual at the
    start, so about half the edges are beyond it): the initial cost to 1e-12 and the
    LM run to the oracle's final cost to 1e-9, FP64."""
    p, pims = small
    c0 = olm.edge_costs(ovi.problem(p, p.nav0, p.pts0, pims))
    delta = float(np.median(np.sqrt(2.0 * c0[1])))
    g, _, _, _ = gpo.vi_graph(p, precision="fp64", imu=_records(pims), imu_huber=delta)
    rep = g.optimize(15, _parity_params(gpo))
    _, orep = olm.levenberg_marquardt(ovi.problem(p, p.nav0, p.pts0, pims, imu_huber=delta), 15)
    assert abs(rep.initial_cost - orep.initial_cost) <= 1e-12 * orep.initial_cost
    assert abs(rep.final_cost - orep.final_cost) <= 1e-9 * orep.final_cost
    plain, _, _, _ = gpo.vi_graph(p, precision="fp64", imu=_records(pims))
    assert plain.cost() > rep.initial_cost   # rho(s) < s beyond the threshold


def test_monocular_edges_match_the_oracle(gpo, small):
    """A third of the observations as monocular (left camera) edges beside stereo ones:
    their rows against the oracle's (the first two stereo rows; the stored third row is
    whitened to zero), the initial cost to 1e-12 and the LM run's final cost to 1e-9."""
    p, pims = small
    mono = np.zeros(len(p.kf_idx), bool)
    mono[::3] = True
    g, _, _, rg = gpo.vi_graph(p, precision="fp64", imu=_records(pims), mono=mono)
    a, b = rg["mono"]
    r, J = g.debug_linearize_edges(np.arange(a, b), nav=True)
    cam = ovi.camera_of(p.camera)
    ro, (Jn, Jp) = ovi.mono_evaluate(cam)((p.nav0[p.kf_idx[mono]], p.pts0[p.pt_idx[mono]]), p.obs[mono, :2])
    w = np.sqrt(robust.weight(np.sum(ro * ro, axis=1), ("huber", p.huber_delta)))
    assert _rel_rows(r[:, :2], ro * w[:, None]) < 1e-12 and np.all(r[:, 2:] == 0)
    Jg = np.concatenate([J[:, :2, :15], J[:, :2, 15:18]], axis=2)
    assert _rel_rows(Jg, np.concatenate([Jn, Jp], axis=2) * w[:, None, None]) < 1e-12
    assert np.all(J[:, 2:] == 0)
    rep = g.optimize(15, _parity_params(gpo))
    _, orep = olm.levenberg_marquardt(ovi.problem(p, p.nav0, p.pts0, pims, mono=mono), 15)
    assert abs(rep.initial_cost - orep.initial_cost) <= 1e-12 * orep.initial_cost
    assert abs(rep.final_cost - orep.final_cost) <= 1e-9 * orep.final_cost


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_monocular_edges_mixed_precision_close_to_fp64(gpo, prec):
    """Stereo and monocular edges together in the mixed forms: within 1e-6 of FP64 after
    the run converges (the setting of the stereo-only mixed test)."""
    p = synth.vi_problem(6, n_kf=12, n_pts=400)
    mono = np.zeros(len(p.kf_idx), bool)
    mono[1::3] = True
    prm = gpo.default_params(pcg_max_iters=500, pcg_tol=1e-10, pcg_rejection_ratio=0.0)
    costs = {}
    for pr in ("fp64", prec):
        g, _, _, _ = gpo.vi_graph(p, precision=pr, mono=mono)
        costs[pr] = g.optimize(30, prm).final_cost
    assert abs(costs[prec] - costs["fp64"]) <= 1e-6 * costs["fp64"]


FISHEYE = (-0.013, 0.021, -0.006, 0.0009)   # Kannala-Brandt k1..k4 of a wide-angle lens


def _fisheye_problem(p):
    """The same trajectory and landmarks seen through a Kannala-Brandt fisheye rig: the
    observations are the oracle's fisheye projections of the ground truth plus the
    problem's pixel noise (seeded)."""
    import dataclasses
    cam = dict(p.camera, fisheye=FISHEYE)
    oc = ovi.camera_of(cam)
    rng = np.random.default_rng(p.seed + 100)
    obs = oc.project(p.nav_gt[p.kf_idx], p.pts_gt[p.pt_idx]) + rng.normal(size=p.obs.shape)
    return dataclasses.replace(p, camera=cam, obs=obs)


def test_fisheye_rows_and_lm_match_the_oracle(gpo, small):
    """Stereo edges of a fisheye rig: rows against the oracle's (analytic, pinned by
    central differences), the autodiff rows against both, and the LM run to the
    oracle's final cost."""
    p0, pims = small
    p = _fisheye_problem(p0)
    g, _, _, rg = gpo.vi_graph(p, precision="fp64", imu=_records(pims))
    a, b = rg["stereo"]
    ids = np.arange(a, b)
    r, J = g.debug_linearize_edges(ids, nav=True)
    ra, Ja = g.debug_autodiff_edges(ids, nav=True)
    cam = ovi.camera_of(p.camera)
    ro, (Jn, Jp) = cam.evaluate((p.nav0[p.kf_idx], p.pts0[p.pt_idx]), p.obs)
    w = np.sqrt(robust.weight(np.sum(ro * ro, axis=1), ("huber", p.huber_delta)))
    assert _rel_rows(r[:, :3], ro * w[:, None]) < 1e-12
    Jg = np.concatenate([J[:, :3, :15], J[:, :3, 15:18]], axis=2)
    assert _rel_rows(Jg, np.concatenate([Jn, Jp], axis=2) * w[:, None, None]) < 1e-11
    assert _rel_rows(Ja[:, :3], J[:, :3]) < 1e-11 and _rel_rows(ra[:, :3], r[:, :3]) < 1e-12
    rep = g.optimize(15, _parity_params(gpo))
    _, orep = olm.levenberg_marquardt(ovi.problem(p, p.nav0, p.pts0, pims), 15)
    assert abs(rep.initial_cost - orep.initial_cost) <= 1e-12 * orep.initial_cost
    assert abs(rep.final_cost - orep.final_cost) <= 1e-9 * orep.final_cost


def test_fixed_keyframe_and_disabled_edges(gpo, small):
    p, pims = small
    g, n0, p0, rg = _graph(gpo, p, pims)
    g.set_fixed(n0)
    g.set_edge_active(rg["imu"][0] + 2, False)
    rep = g.optimize(8, _parity_params(gpo))
    nav = g.get_state(n0, p.n_kf, 16)
    assert np.array_equal(nav[0], p.nav0[0])
    assert rep.final_cost < rep.initial_cost
    prob = ovi.problem(p, p.nav0, p.pts0, pims)
    prob.vertices["nav"].fixed[0] = True
    prob.edges[1].active = np.ones(p.n_kf - 1, bool)
    prob.edges[1].active[2] = False
    _, orep = olm.levenberg_marquardt(prob, 8)
    assert abs(rep.final_cost - orep.final_cost) <= 1e-9 * orep.final_cost


def test_kind_errors(gpo):
    g = gpo.Graph("fp64")
    g.add_vertices(gpo.GPO_V_BA_CAMERA9, 9, 1)
    with pytest.raises(gpo.GpoError):
        g.add_vertices(gpo.GPO_V_NAV15, 15, 1)     # one camera kind per graph
    h = gpo.Graph("fp64")
    a = h.add_vertices(gpo.GPO_V_NAV15, 15, 2)
    q = h.add_vertices(gpo.GPO_V_POINT3, 3, 1)
    with pytest.raises(gpo.GpoError):
        h.add_edges(gpo.GPO_E_BA_REPROJ, np.array([[a, q]]), np.zeros((1, 2)))
    with pytest.raises(gpo.GpoError):
        h.add_edges(gpo.GPO_E_BIAS_RW, np.array([[a, a]]), None)   # distinct keyframes
    with pytest.raises(gpo.GpoError):
        h.add_edges(gpo.GPO_E_IMU, np.array([[a, a + 1]]), np.zeros((1, gpo.GPO_IMU_MEAS_LEN)))  # T = 0
    h.add_edges(gpo.GPO_E_STEREO, np.array([[a, q]]), np.array([[320.0, 240.0, 300.0]]))
    with pytest.raises(gpo.GpoError):
        h.optimize(1)                               # stereo edges need the rig


def test_schur_product_variants_bitwise_vi(gpo, small):
    p, pims = small
    out = []
    for variant in (1, 2, 3):
        g, n0, p0, _ = _graph(gpo, p, pims, precision="fp32", spmv_variant=variant)
        rep = g.optimize(4)
        out.append((rep.final_cost, g.get_state(n0, p.n_kf, 16), g.get_state(p0, p.n_pts, 3)))
    for o in out[1:]:
        assert out[0][0] == o[0]
        assert np.array_equal(out[0][1], o[1]) and np.array_equal(out[0][2], o[2])


def test_sampled_edges_at_full_size(gpo):
    """The full global workload (3,000 keyframes, 200,000 landmarks, ~1.9M stereo edges)
    as the benchmark runs it (library preintegration): a random sample of stereo edges
    and every inertial and bias edge are checked against the oracle one edge at a time.
    The oracle evaluates the inertial edges with the library's own records (whose
    agreement with the oracle's preintegration test_vi_host.py pins), so this checks the
    GPU evaluation only.  Tolerances: stereo 1e-12 relative to the edge's largest entry
    plus the cancellation in X - p (positions reach hundreds of metres): 64 eps |p| /
    depth; inertial 1e-11 as in the small test, plus the same cancellation in
    p_j - p_i - v_i T scaled by the whitening."""
    p = synth.vi_global()
    g, n0, p0, rg = gpo.vi_graph(p, precision="fp64")
    rng = np.random.default_rng(0)
    a, b = rg["stereo"]
    sid = np.sort(rng.choice(b - a, 3000, replace=False)) + a
    r, J = g.debug_linearize_edges(sid, nav=True)
    cam = ovi.camera_of(p.camera)
    k = sid - a
    nav, X = p.nav0[p.kf_idx[k]], p.pts0[p.pt_idx[k]]
    ro, (Jn, Jp) = cam.evaluate((nav, X), p.obs[k])
    w = np.sqrt(robust.weight(np.sum(ro * ro, axis=1), ("huber", p.huber_delta)))
    ro = ro * w[:, None]
    Jo = np.concatenate([Jn, Jp], axis=2) * w[:, None, None]
    _, Xc = cam.point_in_camera(nav, X)
    eps = np.finfo(np.float64).eps
    kappa = 64 * eps * (np.linalg.norm(nav[:, 4:7], axis=1) + np.linalg.norm(X, axis=1)) / np.abs(Xc[:, 2])
    scale_r = np.maximum(np.abs(ro).max(axis=1), 1.0)
    assert np.all(np.abs(r[:, :3] - ro).max(axis=1) <= (1e-12 + kappa * 450.0) * scale_r)
    Jg = np.concatenate([J[:, :3, :15], J[:, :3, 15:18]], axis=2)
    assert np.all(np.abs(Jg - Jo).reshape(len(sid), -1).max(axis=1)
                  <= (1e-12 + kappa) * np.abs(Jo).reshape(len(sid), -1).max(axis=1) + 1e-300)
    # every inertial edge, with the library's records
    ia, ib = rg["imu"]
    ids = np.arange(ia, ib)
    ri, Ji = g.debug_linearize_edges(ids, nav=True)
    meas = np.zeros((p.n_kf - 1, gpo.GPO_IMU_MEAS_LEN))
    info = np.zeros((p.n_kf - 1, 9, 9))
    worst_r = worst_J = 0.0
    for q in range(p.n_kf - 1):
        m, _, inf = gpo.imu_preintegrate(p.imu_gyro[q], p.imu_acc[q], p.dt, p.nav0[q, 10:13], p.nav0[q, 13:16],
                                         p.noise["sigma_g"], p.noise["sigma_a"])
        pm = dict(dR=m[0:9].reshape(3, 3), dv=m[9:12], dp=m[12:15], JRg=m[15:24].reshape(3, 3),
                  Jvg=m[24:33].reshape(3, 3), Jva=m[33:42].reshape(3, 3), Jpg=m[42:51].reshape(3, 3),
                  Jpa=m[51:60].reshape(3, 3), T=m[60], bg0=m[61:64], ba0=m[64:67])
        U = np.linalg.cholesky(inf).T
        rr = U @ ovi.imu_residual_one(pm, p.nav0[q:q + 1], p.nav0[q + 1:q + 2])
        Jq = np.concatenate([U @ x for x in ovi.imu_jacobians_one(pm, p.nav0[q:q + 1], p.nav0[q + 1:q + 2])], axis=1)
        # cancellation in p_j - p_i - v_i T at |p| of hundreds of metres, through U
        cancel = 64 * eps * np.linalg.norm(p.nav0[q, 4:7]) * np.abs(U).max()
        worst_r = max(worst_r, np.abs(ri[q] - rr).max() / (1e-11 * max(np.abs(rr).max(), 1.0) + cancel))
        worst_J = max(worst_J, np.abs(Ji[q] - Jq).max() / (1e-11 * np.abs(Jq).max()))
    assert worst_r <= 1.0 and worst_J <= 1.0
