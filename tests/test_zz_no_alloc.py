"""The allocation-free cost entry point (gpo_ba_cost_noalloc), called through the
C ABI on caller-owned device buffers, against the FP64 oracle's total cost and the
library's regular cost (gpo_get_cost), on two calls in a row.

It serves callers that cannot allocate device memory where they need a cost (a
memory pool that is already handed out, a real-time thread that must not enter the
allocator); its reduction scratch is a static device array, so it allocates nothing.
The cases run a small problem, one at the scratch's limit of 2,097,152 edges (8,192
CTAs, every partial slot in use) and an empty one.  This file is collected last so
that a run stopping at the first failure has run every other test first."""
import ctypes

import numpy as np
import pytest

from oracle import lm as olm
from paper_2509_26581_gb300 import synth

pytestmark = pytest.mark.gpu

MAX_EDGES = 2_097_152


def _device_copy(torch, a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


def _noalloc_twice(torch, gpo, cams, pts, cam_idx, pt_idx, obs, huber):
    """Calls the entry point twice on the same device buffers; returns both costs."""
    n = len(cam_idx)
    dc = _device_copy(torch, cams, np.float64)
    dp = _device_copy(torch, pts, np.float64)
    ci = _device_copy(torch, cam_idx, np.int32)
    pi = _device_copy(torch, pt_idx, np.int32)
    ob = _device_copy(torch, obs.reshape(-1, 2), np.float64)
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    vals = []
    for _ in range(2):
        st = gpo.lib.gpo_ba_cost_noalloc(torch.cuda.current_device(), ctypes.c_void_p(stream.cuda_stream),
                                         ctypes.c_void_p(dc.data_ptr()), ctypes.c_void_p(dp.data_ptr()),
                                         ctypes.c_void_p(ci.data_ptr()), ctypes.c_void_p(pi.data_ptr()),
                                         ctypes.c_void_p(ob.data_ptr()), n,
                                         -1.0 if huber is None else huber,
                                         ctypes.c_void_p(out.data_ptr()))
        assert st == gpo.GPO_OK
        torch.cuda.synchronize()
        vals.append(float(out.item()))
        out.fill_(float("nan"))
    return vals


@pytest.mark.parametrize("huber", [None, 2.0])
def test_noalloc_cost_matches_oracle_and_library_twice(huber):
    import torch

    from paper_2509_26581_gb300 import gpo
    p = synth.ba_ring(9, 12, 800, 5, outlier_frac=0.02, huber_delta=huber)
    oracle = olm.total_cost(olm.ba_problem(p.cams0, p.pts0, p.cam_idx, p.pt_idx, p.obs, huber_delta=huber))
    g, _, _ = gpo.ba_graph(p.cams0, p.pts0, p.cam_idx, p.pt_idx, p.obs, huber, "fp64")
    ref = g.cost()
    g.close()
    for v in _noalloc_twice(torch, gpo, p.cams0, p.pts0, p.cam_idx, p.pt_idx, p.obs, huber):
        assert abs(v - oracle) <= 1e-12 * oracle
        assert abs(v - ref) <= 1e-12 * ref


def test_noalloc_cost_at_its_edge_limit():
    """The first 2,097,152 edges of the 1,000-camera workload: the largest call the
    static scratch holds."""
    import torch

    from paper_2509_26581_gb300 import gpo
    p = synth.ba_medium(1)
    n = MAX_EDGES
    oracle = olm.total_cost(olm.ba_problem(p.cams0, p.pts0, p.cam_idx[:n], p.pt_idx[:n], p.obs[:n],
                                           huber_delta=p.huber_delta))
    for v in _noalloc_twice(torch, gpo, p.cams0, p.pts0, p.cam_idx[:n], p.pt_idx[:n], p.obs[:n], p.huber_delta):
        assert abs(v - oracle) <= 1e-12 * oracle


def test_noalloc_cost_of_no_edges_is_zero():
    import torch

    from paper_2509_26581_gb300 import gpo
    cams = np.zeros((1, 9))
    pts = np.zeros((1, 3))
    e = np.zeros(0, np.int64)
    assert _noalloc_twice(torch, gpo, cams, pts, e, e, np.zeros((0, 2)), None) == [0.0, 0.0]


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2509_26581_gb300 import gpo
    dummy = ctypes.c_void_p(16)
    st = gpo.lib.gpo_ba_cost_noalloc(0, None, dummy, dummy, dummy, dummy, dummy, MAX_EDGES + 1, -1.0, dummy)
    assert st == gpo.GPO_ERR_ARG
