"""Batched solves and the serving loop: every window's result is bit-for-bit the
same as when it is solved alone (its reductions never mix with another window's),
admission respects the memory budget and slots, and the oracle agrees with a window's
FP64 solve."""
import numpy as np
import pytest

from oracle import lm as olm
from paper_2509_26581_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpo():
    from paper_2509_26581_gb300 import gpo as m
    return m


@pytest.fixture(scope="module")
def windows():
    return synth.window_pool(3, 12, kf=(5, 12), pts=(200, 1500))


def _alone(gpo, serving, p, prec, iters, **kw):
    g, c0, p0 = serving.window_graph(p, prec, **kw)
    rep = g.optimize(iters)
    return rep, g.get_state(c0, p.n_cams, 9), g.get_state(p0, p.n_pts, 3)


@pytest.mark.parametrize("prec,variant", [("fp64", 0), ("bf16", 0), ("fp32", 1), ("fp32", 3)])
def test_batch_equals_alone_bitwise(gpo, windows, prec, variant):
    """Also with the staged and pipelined Schur products, whose persistent CTAs walk
    chunks of several problems."""
    from paper_2509_26581_gb300 import serving
    kw = dict(spmv_variant=variant, chunk_edges=256)
    alone = [_alone(gpo, serving, p, prec, 6, **kw) for p in windows]
    built = [serving.window_graph(p, prec, **kw) for p in windows]
    reps = gpo.optimize_batch([b[0] for b in built], 6)
    for (rep, cams, pts), (g, c0, p0), r, p in zip(alone, built, reps, windows):
        assert r.final_cost == rep.final_cost and r.accepted == rep.accepted
        assert np.array_equal(g.get_state(c0, p.n_cams, 9), cams)
        assert np.array_equal(g.get_state(p0, p.n_pts, 3), pts)


def test_window_fp64_matches_oracle(gpo, windows):
    from paper_2509_26581_gb300 import serving
    p = windows[0]
    g, _, _ = serving.window_graph(p, "fp64")
    params = gpo.default_params(pcg_max_iters=500, pcg_tol=1e-14, pcg_rejection_ratio=0.0)
    rep = g.optimize(8, params)
    cf = np.zeros(p.n_cams, bool)
    cf[0] = True
    _, orep = olm.levenberg_marquardt(olm.ba_problem(p.cams0, p.pts0, p.cam_idx, p.pt_idx, p.obs,
                                                     huber_delta=p.huber_delta, cam_fixed=cf), 8)
    assert abs(rep.initial_cost - orep.initial_cost) <= 1e-12 * orep.initial_cost
    assert abs(rep.final_cost - orep.final_cost) <= 1e-9 * orep.final_cost


def test_server_results_equal_alone_under_budget(gpo, windows):
    from paper_2509_26581_gb300 import serving
    alone = [_alone(gpo, serving, p, "bf16", 5) for p in windows]
    # a budget that holds only a few windows at once: admission must queue the rest
    sizes = []
    for p in windows[:3]:
        g, _, _ = serving.window_graph(p, "bf16")
        g.optimize(0)
        sizes.append(g.footprint())
    budget = int(sum(sizes) * 1.05)
    sv = gpo.Server("bf16", memory_budget=budget, max_resident=4)
    built = [serving.window_graph(p, "bf16") for p in windows]
    tickets = [sv.submit(b[0], 5) for b in built]
    reports = {}
    seen_max = 0
    for _ in range(1000):
        res, queued, fin = sv.step()
        seen_max = max(seen_max, res)
        assert sv.memory() <= budget
        for t in tickets:
            if t not in reports:
                r = sv.poll(t)
                if r is not None:
                    reports[t] = r
        if len(reports) == len(tickets):
            break
    assert len(reports) == len(tickets)
    assert 1 <= seen_max <= 4
    for t, (g, c0, p0), (rep, cams, pts), p in zip(tickets, built, alone, windows):
        assert reports[t].final_cost == rep.final_cost
        assert np.array_equal(g.get_state(c0, p.n_cams, 9), cams)
        assert np.array_equal(g.get_state(p0, p.n_pts, 3), pts)
    sv.close()


def test_server_rejects_oversized_graph(gpo, windows):
    from paper_2509_26581_gb300 import serving
    sv = gpo.Server("bf16", memory_budget=1 << 16)
    g, _, _ = serving.window_graph(windows[0], "bf16")
    with pytest.raises(gpo.GpoError) as e:
        sv.submit(g, 3)
    assert e.value.status == gpo.GPO_ERR_OOM
    sv.close()


def test_serve_driver_stream(gpo, windows):
    from paper_2509_26581_gb300 import serving
    arr = synth.poisson_arrivals(5, 400.0, 0.1)
    pick = synth.Stream(5, 23).integers(len(arr), 0, len(windows))
    out = serving.serve(windows, arr, pick, "bf16", lm_iters=4)
    assert np.all(np.isfinite(out["latency"])) and out["solves_per_s"] > 0
    alone = {}
    for i in np.unique(pick):
        alone[i] = _alone(gpo, serving, windows[i], "bf16", 4)[0].final_cost
    for c, i in zip(out["final_cost"], pick):
        assert c == alone[i]
