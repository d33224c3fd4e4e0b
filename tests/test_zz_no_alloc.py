"""The allocation-free cost entry point (gpo_ba_cost_noalloc), called through the
C ABI on caller-owned device buffers, agrees with the library's regular cost
(gpo_get_cost) on the same problem, on two calls in a row.

It is for callers that cannot allocate device memory where they need a cost; its
scratch is a static device array, so it needs no allocation of its own.  This file
is collected last so that a run stopping at the first failure has run every other
test first."""
import ctypes

import numpy as np
import pytest

from paper_2509_26581_gb300 import synth

pytestmark = pytest.mark.gpu


def _device_copy(torch, a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


@pytest.mark.parametrize("huber", [None, 2.0])
def test_noalloc_cost_matches_library_cost_twice(huber):
    import torch

    from paper_2509_26581_gb300 import gpo
    p = synth.ba_ring(9, 12, 800, 5, outlier_frac=0.02, huber_delta=huber)
    g, _, _ = gpo.ba_graph(p.cams0, p.pts0, p.cam_idx, p.pt_idx, p.obs, huber, "fp64")
    ref = g.cost()
    cams = _device_copy(torch, p.cams0, np.float64)
    pts = _device_copy(torch, p.pts0, np.float64)
    ci = _device_copy(torch, p.cam_idx, np.int32)
    pi = _device_copy(torch, p.pt_idx, np.int32)
    obs = _device_copy(torch, p.obs, np.float64)
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(2):
        st = gpo.lib.gpo_ba_cost_noalloc(torch.cuda.current_device(), ctypes.c_void_p(stream.cuda_stream),
                                         ctypes.c_void_p(cams.data_ptr()), ctypes.c_void_p(pts.data_ptr()),
                                         ctypes.c_void_p(ci.data_ptr()), ctypes.c_void_p(pi.data_ptr()),
                                         ctypes.c_void_p(obs.data_ptr()), p.n_edges,
                                         -1.0 if huber is None else huber,
                                         ctypes.c_void_p(out.data_ptr()))
        assert st == gpo.GPO_OK
        torch.cuda.synchronize()
        v = float(out.item())
        assert abs(v - ref) <= 1e-12 * ref
        out.fill_(float("nan"))


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2509_26581_gb300 import gpo
    dummy = ctypes.c_void_p(16)
    st = gpo.lib.gpo_ba_cost_noalloc(0, None, dummy, dummy, dummy, dummy, dummy, 2_097_153, -1.0, dummy)
    assert st == gpo.GPO_ERR_ARG
