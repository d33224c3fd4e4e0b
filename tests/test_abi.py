"""The C-ABI library builds, loads and exports every entry point that include/gpo.h
declares (CPU only: no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^\s*(?:gpo_status|const char\*)\s+(gpo_\w+)\s*\(", src, re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2509_26581_gb300 import build
    return ctypes.CDLL(build.build())


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("gpo_graph_create", "gpo_add_vertices", "gpo_add_edges", "gpo_set_initial",
              "gpo_optimize", "gpo_get_cost", "gpo_get_state", "gpo_graph_destroy"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_defaults_and_version(lib):
    from paper_2509_26581_gb300 import gpo
    p = gpo.default_params()
    assert p.initial_damping == 1e-4 and p.pcg_max_iters == 100 and p.pcg_tol == 1e-6
    assert p.diag_min == 1e-6 and p.diag_max == 1e32 and p.pcg_rejection_ratio == 10.0
    # the last fields too: the binding's structure matches the header's layout
    assert p.pcg_normalize == -1 and p.pcg_restart_every == -1 and p.solver == gpo.GPO_SOLVER_SCHUR
    assert gpo.lib.gpo_version().decode().startswith("gpo")


def test_struct_sizes_match_the_header():
    """Each parameter struct the binding mirrors has the size the header gives it
    (C layout rules of the header's member types, computed here independently)."""
    from paper_2509_26581_gb300 import gpo
    # gpo_lm_params: 5 doubles, 2 int32, double, int32 (+4 pad), double, 3 int32 (+4 pad), double
    assert ctypes.sizeof(gpo.gpo_lm_params) == 5 * 8 + 2 * 4 + 8 + 8 + 8 + 16 + 8
    # gpo_report: 3 doubles, 4 int32, double
    assert ctypes.sizeof(gpo.gpo_report) == 3 * 8 + 4 * 4 + 8
    src_r = open(os.path.join(ROOT, "include", "gpo.h")).read()
    body_r = src_r[src_r.rindex("typedef struct {", 0, src_r.index("} gpo_report;")):src_r.index("} gpo_report;")]
    body_r = re.sub(r"/\*.*?\*/", "", body_r, flags=re.S)
    assert [f for _, f in re.findall(r"(double|int32_t)\s+(\w+);", body_r)] == [f for f, _ in gpo.gpo_report._fields_]
    src = open(os.path.join(ROOT, "include", "gpo.h")).read()
    body = src[src.index("typedef struct {", src.index("PCGSolver(max_it")):src.index("} gpo_lm_params;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"(double|int32_t)\s+(\w+);", body)
    assert [f for _, f in fields] == [f for f, _ in gpo.gpo_lm_params._fields_]


def test_null_arguments_are_rejected(lib):
    from paper_2509_26581_gb300 import gpo
    assert gpo.lib.gpo_graph_create(None, None) == gpo.GPO_ERR_ARG
    assert gpo.lib.gpo_lm_params_default(None) == gpo.GPO_ERR_ARG
    assert gpo.lib.gpo_graph_destroy(None) == gpo.GPO_OK
