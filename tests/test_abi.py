"""The C-ABI library builds for sm_103a, loads, and exports every entry point
include/pc.h declares (no GPU needed; no compute call is made)."""
import ctypes as C
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "pc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pc_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("pc_plan_create", "pc_propagate", "pc_plan_destroy", "pc_status_string"):
        assert required in names


def test_library_builds_loads_and_exports_every_symbol():
    from paper_2301_03989_gb300 import build, pcprop
    path = build.build()
    assert os.path.exists(path)
    L = C.CDLL(path)
    for name in declared_symbols():
        assert hasattr(L, name), name
    assert set(pcprop.EXPORTS) <= set(declared_symbols())


def test_host_only_entry_points():
    from paper_2301_03989_gb300 import pcprop
    o = pcprop.options_default()
    assert o.tol == 1e-13 and o.max_iters == 60 and o.relative == 1 and o.trunc_tol == 1e-13
    assert o.precision == pcprop.PC_PREC_FP64 and o.switch_tol == 0.0 and o.refine32 == 1
    assert pcprop.status_string(pcprop.PC_EINVAL) == "invalid argument"
    assert pcprop.lib().pc_options_default(None) == pcprop.PC_EINVAL
