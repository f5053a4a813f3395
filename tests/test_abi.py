"""The C-ABI library loads and exports every symbol include/hsein.h declares;
host-side argument checks work without a GPU (no compute calls here)."""
import ctypes
import os
import re

import pytest

import paper_2101_05063_gb300 as hs
from paper_2101_05063_gb300 import build as hsbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hsein.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hsein_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    return hs.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["hsein_plan", "hsein_solve", "hsein_backtransform", "hsein_plan_destroy",
                     "hsein_status_string", "hsein_plan_sync_status", "hsein_default_options",
                     "hsein_plan_info"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_python_binding_mirrors_every_symbol():
    for name in declared_functions():
        assert hasattr(hs, name), name


def test_library_is_built_for_sm_103a():
    assert "compute_103a,code=sm_103a" in hsbuild.GENCODE
    assert os.path.exists(hsbuild.LIB)


def test_status_strings(lib):
    assert hs.hsein_status_string(0) == "ok"
    assert "reduced" in hs.hsein_status_string(-3)
    assert hs.hsein_status_string(12345) == "unknown status"


def test_default_options(lib):
    o = hs.hsein_default_options()
    assert o.br == 64 and o.robust == 1 and o.omega_log2 == 1000 and o.precision == 0
    assert o.wait_limit_cycles == 1 << 32
    assert hs.hsein_status_string(-6) != "unknown status"


@pytest.mark.parametrize("args", [(0, 1, 0), (4, -1, 0), (4, 0, -2), (4, 0, 0)])
def test_plan_rejects_bad_sizes(lib, args):
    with pytest.raises(hs.HseinError) as e:
        hs.hsein_plan(*args)
    assert e.value.code == -1


def test_plan_rejects_bad_options(lib):
    for field, value in [("br", 4), ("br", 129), ("omega_log2", 8), ("robust", 2), ("precision", 3),
                         ("wait_limit_cycles", -1), ("wait_limit_cycles", 1 << 61)]:
        o = hs.hsein_default_options()
        setattr(o, field, value)
        with pytest.raises(hs.HseinError) as e:
            hs.hsein_plan(16, 2, 1, o)
        assert e.value.code == -1, field


def test_solve_rejects_null_plan_and_pointers(lib):
    assert lib.hsein_solve(None, None, 0, None, None, None, 0, None, 0, None, None, 0, None) == -1
    assert lib.hsein_backtransform(None, None, 0, None, 0, None, 0, None, 0, None) == -1
    assert lib.hsein_plan_destroy(None) == 0


def test_graph_entry_points_reject_null_arguments(lib):
    import ctypes
    g = ctypes.c_void_p(1)
    assert lib.hsein_graph_create(None, None, 0, None, None, None, 0, None, 0, None, None, 0,
                                  None, 0, None, 0, ctypes.byref(g)) == -1
    assert not g.value  # no handle on failure
    assert lib.hsein_graph_create(None, None, 0, None, None, None, 0, None, 0, None, None, 0,
                                  None, 0, None, 0, None) == -1
    assert lib.hsein_graph_launch(None, None) == -1
    assert lib.hsein_graph_destroy(None) == 0
