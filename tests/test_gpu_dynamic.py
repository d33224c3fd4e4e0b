"""Dynamic Jacobians (spmv_variant 4: no rows are stored; every kernel that needs an
edge's rows -- the Schur preparation, each Schur product, the back-substitution --
evaluates them from the state) against the FP64 oracle and against stored rows,
through the C ABI.

Tolerances (written here, derived from the arithmetic):
  * FP64: the rows are the stored rows (same evaluation, same accumulation order), so
    the LM run matches the stored-row run to 1e-12 relative in cost and 1e-10 in the
    states (rounding and FMA contraction of the same expressions in another kernel),
    and the oracle's exact-step LM run to 1e-9 in cost, as the stored-row tests do;
  * FP32 accumulation (BF16 or FP32 storage, one mode here since nothing is stored):
    FP32 rows everywhere, so the run converges to the FP64 optimum within 1e-6, the
    mixed-precision bar.
"""
import numpy as np
import pytest

from oracle import lm as olm
from paper_2509_26581_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpo():
    from paper_2509_26581_gb300 import gpo as m
    return m


def _exact(gpo):
    return gpo.default_params(pcg_max_iters=500, pcg_tol=1e-14, pcg_rejection_ratio=0.0)


def test_dynamic_fp64_matches_stored_rows_and_the_oracle(gpo):
    """A fixed camera and a fixed point (zeroed columns) included."""
    p = synth.ba_ring(0, 10, 500, 6)
    cf = np.zeros(p.n_cams, bool)
    cf[0] = True
    pf = np.zeros(p.n_pts, bool)
    pf[5] = True
    runs = []
    for variant in (4, 2):
        g, c0, p0 = gpo.ba_graph(p.cams0, p.pts0, p.cam_idx, p.pt_idx, p.obs, None, "fp64", cam_fixed=cf,
                                 pt_fixed=pf, spmv_variant=variant, chunk_edges=256)
        rep = g.optimize(10, _exact(gpo))
        info = g.info()
        assert info["spmv_kernel"] == variant and (info["j_bytes"] == 0) == (variant == 4)
        runs.append((rep, g.get_state(c0, p.n_cams, 9), g.get_state(p0, p.n_pts, 3)))
    (rd, cd, pd), (rs, cs, ps) = runs
    assert abs(rd.final_cost - rs.final_cost) <= 1e-12 * rs.final_cost
    assert np.abs(cd - cs).max() <= 1e-10 * max(np.abs(cs).max(), 1.0)
    assert np.abs(pd - ps).max() <= 1e-10 * max(np.abs(ps).max(), 1.0)
    _, orep = olm.levenberg_marquardt(olm.ba_problem(p.cams0, p.pts0, p.cam_idx, p.pt_idx, p.obs,
                                                     cam_fixed=cf, pt_fixed=pf), 10)
    assert abs(rd.final_cost - orep.final_cost) <= 1e-9 * orep.final_cost
    assert np.array_equal(cd[0], p.cams0[0]) and np.array_equal(pd[5], p.pts0[5])


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_dynamic_mixed_precision_reaches_the_fp64_optimum(gpo, prec):
    """Huber loss with outliers (IRLS weights evaluated inside the product)."""
    p = synth.ba_ring(7, 20, 4000, 6, outlier_frac=0.01, huber_delta=2.0)
    g, _, _ = gpo.ba_graph(p.cams0, p.pts0, p.cam_idx, p.pt_idx, p.obs, p.huber_delta, "fp64")
    ref = g.optimize(30).final_cost
    h, _, _ = gpo.ba_graph(p.cams0, p.pts0, p.cam_idx, p.pt_idx, p.obs, p.huber_delta, prec,
                           spmv_variant=4, chunk_edges=512)
    cost = h.optimize(30).final_cost
    assert h.info()["spmv_kernel"] == 4 and h.info()["j_bytes"] == 0
    assert abs(cost - ref) <= 1e-6 * ref


def test_dynamic_vi_fp64_matches_stored_rows(gpo):
    """Stereo edges of navigation states beside the camera-side inertial edges."""
    p = synth.vi_problem(5, n_kf=8, n_pts=200)
    runs = []
    for variant in (4, 2):
        g, n0, p0, _ = gpo.vi_graph(p, precision="fp64", spmv_variant=variant, chunk_edges=256)
        rep = g.optimize(6, _exact(gpo))
        assert g.info()["spmv_kernel"] == variant
        runs.append((rep.final_cost, g.get_state(n0, p.n_kf, 16), g.get_state(p0, p.n_pts, 3)))
    (fd, nd, qd), (fs, ns, qs) = runs
    assert abs(fd - fs) <= 1e-12 * fs
    assert np.abs(nd - ns).max() <= 1e-10 * max(np.abs(ns).max(), 1.0)
    assert np.abs(qd - qs).max() <= 1e-10 * max(np.abs(qs).max(), 1.0)


def test_dynamic_rows_are_not_stored(gpo):
    """The device footprint drops by the row array; BF16 and FP32 requests are one mode
    (FP32 rows evaluated where used) and give the same run bit for bit; what needs stored
    rows is refused with GPO_ERR_UNSUPPORTED.  (The optimum reached is checked against
    FP64 above; five unconverged iterations of stored BF16 rows and of FP32 rows follow
    different trajectories.)"""
    p = synth.ba_path(3, 40, 6000, "pareto")
    out = {}
    for prec, variant in (("bf16", 2), ("bf16", 4), ("fp32", 4)):
        g, _, _ = gpo.ba_graph(p.cams0, p.pts0, p.cam_idx, p.pt_idx, p.obs, p.huber_delta, prec,
                               spmv_variant=variant, chunk_edges=512)
        rep = g.optimize(5)
        out[(prec, variant)] = (rep.final_cost, g.footprint(), g.info())
        if variant == 4:
            with pytest.raises(gpo.GpoError) as ei:
                g.debug_linearize(p.n_edges)
            assert ei.value.status == gpo.GPO_ERR_UNSUPPORTED
            with pytest.raises(gpo.GpoError) as ei:
                g.optimize(1, gpo.default_params(solver=gpo.GPO_SOLVER_FULL))
            assert ei.value.status == gpo.GPO_ERR_UNSUPPORTED
        g.close()
    stored, dyn16, dyn32 = out[("bf16", 2)], out[("bf16", 4)], out[("fp32", 4)]
    assert stored[2]["j_bytes"] >= 24 * 2 * p.n_edges and dyn16[2]["j_bytes"] == 0
    assert stored[1] - dyn16[1] >= stored[2]["j_bytes"] - 4096
    assert dyn16[0] == dyn32[0]


def test_dynamic_graphs_are_solved_alone(gpo):
    p = synth.ba_ring(0, 10, 500, 6)
    gs = [gpo.ba_graph(p.cams0, p.pts0, p.cam_idx, p.pt_idx, p.obs, None, "fp32", spmv_variant=4)[0]
          for _ in range(2)]
    with pytest.raises(gpo.GpoError) as ei:
        gpo.optimize_batch(gs, 2)
    assert ei.value.status == gpo.GPO_ERR_UNSUPPORTED
