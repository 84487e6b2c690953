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


def test_argument_errors_without_a_gpu():
    """Every entry point refuses a missing plan or bad arguments with PC_EINVAL
    before touching the device (so this runs without a GPU)."""
    import ctypes as C
    from paper_2301_03989_gb300 import pcprop as pc
    L = pc.lib()
    E = pc.PC_EINVAL
    null = None
    out = C.c_void_p()
    fm = pc.ForceModel(0, 1.0, None, 1)
    assert L.pc_plan_create(1, 4, C.byref(fm), None, None, C.byref(out)) == E          # N < 2
    assert L.pc_plan_create(64, 0, C.byref(fm), None, None, C.byref(out)) == E         # no segments
    assert L.pc_plan_create(64, 4, None, None, None, C.byref(out)) == E                # no force model
    assert L.pc_plan_create(64, 4, C.byref(fm), None, None, None) == E                 # no output
    bad = pc.ForceModel(2, 1.0, None, 1)                                                # bodies without GMs
    assert L.pc_plan_create(64, 4, C.byref(bad), None, None, C.byref(out)) == E
    bad = pc.ForceModel(0, 1.0, None, 1, -1.0)                                          # negative speed of light
    assert L.pc_plan_create(64, 4, C.byref(bad), None, None, C.byref(out)) == E
    o = pc.options_default(precision=pc.PC_PREC_MIXED)
    assert L.pc_plan_create(300, 4, C.byref(fm), None, C.byref(o), C.byref(out)) == E  # mixed needs N <= 287
    o = pc.options_default(refine32=2)
    assert L.pc_plan_create(64, 4, C.byref(fm), None, C.byref(o), C.byref(out)) == E
    for bad_opts, N in ((dict(order=3), 64), (dict(order=2, contraction=pc.PC_CONTRACT_DMMA), 64),
                        (dict(order=2), 300), (dict(contraction=2), 64), (dict(fp32_mma=2), 64)):
        o = pc.options_default(**bad_opts)                                              # second order: split, N <= 255
        assert L.pc_plan_create(N, 4, C.byref(fm), None, C.byref(o), C.byref(out)) == E, bad_opts
    assert L.pc_propagate(null, 4, null, 0.0, 1.0, 0.0, null, null, null, null) == E
    assert L.pc_propagate_ex(null, 4, null, 0.0, 1.0, 0.0, null, null, null, null, 0, null, null, null) == E
    assert L.pc_propagate_tape(null, 4, null, null, null, null, 0.0, null, null, null, 1, null, null) == E
    assert L.pc_adjoint_tape(null, 4, null, 1, null, null, 0.0, null, null, null, null) == E
    assert L.pc_propagate_adjoint(null, 4, null, 0.0, 1.0, 0.0, null, null, null) == E
    assert L.pc_bplane(null, 0, 1.0, 4, null, null, null, null, null, null, null) == E
    assert L.pc_plan_get_tuning(null, null) == E
    assert L.pc_plan_set_tuning(null, null) == E
    assert L.pc_plan_autotune(null, 4, null, 0.0, 1.0, 64, null, null) == E
    assert L.pc_plan_set_profiling(null, 1) == E
    assert L.pc_apply_operator(null, 4, null, null, null, null) == E
    assert L.pc_apply_operator_static(null, 4, null, null, null, null) == E
    hp = (C.c_void_p * 1)(None)
    hc = (C.c_longlong * 1)(4)
    assert L.pc_propagate_groups(hp, 1, hc, null, null, null, null, 0.0, null, null, null, null, null, null) == E
    assert L.pc_propagate_groups(None, 0, None, null, null, null, null, 0.0, null, null, null, null, null, null) == E
    L.pc_plan_destroy(None)                                                             # NULL is allowed
