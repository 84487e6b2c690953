"""Mixed-precision path (FP32 sweeps on the deviation from the warm start,
then FP64 sweeps to tol) against the FP64 oracle.  After the FP64 refinement
the result must meet the same bound as the plain FP64 path: 1e-10 relative in
position and velocity (segment by segment across flybys)."""
import numpy as np
import pytest

from paper_2301_03989_gb300 import workloads as W
from test_gpu_parity import TOL, _segment_local, rel_err, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pc():
    import torch
    from paper_2301_03989_gb300 import build, pcprop
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return pcprop


@pytest.mark.parametrize("switch_tol", [1e-6, 0.0])
def test_mixed_config1_vs_oracle(pc, ora, switch_tol):
    w = W.config1()
    g = run_gpu(pc, w, w.x0, precision=pc.PC_PREC_MIXED, switch_tol=switch_tol)
    o = run_oracle(ora, w, w.x0)
    assert g["code"] == pc.PC_OK
    er, ev = rel_err(g["xf"], o["xf"])
    assert er.max() < TOL and ev.max() < TOL, (er.max(), ev.max())
    np.testing.assert_array_equal(g["nseg"], o["nseg"])


def test_mixed_config3_subset_vs_oracle(pc, ora):
    """Config 3 system and ICs, 2-year arcs in 25 segments, N = 128."""
    w = W.config3(M=64)
    g = run_gpu(pc, w, w.x0, precision=pc.PC_PREC_MIXED)
    o = run_oracle(ora, w, w.x0)
    er, ev = rel_err(g["xf"], o["xf"])
    assert er.max() < TOL and ev.max() < TOL, (er.max(), ev.max())


def test_precision_study_error_report(pc, ora):
    """Config 3 at full size (65,536 trajectories, 2-year arcs, N = 128), FP32
    sweeps until the change is below 1e-6 then FP64 to 1e-13, and the plain FP64
    path: per-trajectory error against the oracle on a seeded subset of 4096
    trajectories."""
    import os
    w = W.config3()
    idx = np.sort(np.random.default_rng(0).choice(w.n_ic, size=4096, replace=False))
    o = run_oracle(ora, w, w.x0[idx], threads=os.cpu_count() or 8)
    for name, prec, sw in (("mixed", pc.PC_PREC_MIXED, 1e-6), ("fp64", pc.PC_PREC_FP64, 0.0)):
        g = run_gpu(pc, w, w.x0, precision=prec, switch_tol=sw)
        assert g["code"] == pc.PC_OK, name
        er, ev = rel_err(g["xf"][idx], o["xf"])
        print(f"config 3 {name}: error vs oracle on {idx.size} trajectories: position max {er.max():.2e} "
              f"median {np.median(er):.2e}, velocity max {ev.max():.2e} median {np.median(ev):.2e}")
        assert er.max() < TOL and ev.max() < TOL, (name, er.max(), ev.max())


def test_mixed_config2_short_and_segment_local(pc, ora):
    w = W.config2(M=32)
    tf = 20 * W.DAY
    g = run_gpu(pc, w, w.x0, tf=tf, precision=pc.PC_PREC_MIXED)
    o = run_oracle(ora, w, w.x0, tf=tf)
    er, ev = rel_err(g["xf"], o["xf"])
    assert er.max() < TOL and ev.max() < TOL, (er.max(), ev.max())
    g = run_gpu(pc, w, w.x0[:8], max_ckpt=600, precision=pc.PC_PREC_MIXED)
    assert g["code"] == pc.PC_OK
    assert _segment_local(ora, w, g, range(8)) < TOL


def test_mixed_does_fewer_fp64_sweeps(pc):
    """The FP32 phase must carry sweeps: FP64 trajectory-sweeps drop well below
    the plain path's on the same inputs (half a year from the flybys, where the
    deviation from the warm start is large and the FP32 floor high)."""
    import torch
    w = W.config2(M=256)
    tf = 0.5 * W.YEAR
    counts = {}
    for prec in (pc.PC_PREC_FP64, pc.PC_PREC_MIXED):
        plan = pc.plan_from_workload(w, precision=prec)
        x0 = torch.as_tensor(W.to_planar(w.x0), device="cuda")
        xf = torch.zeros_like(x0)
        pc.kernel_times(plan)
        pc.propagate(plan, x0, w.t0, tf, xf)
        kt = pc.kernel_times(plan)
        counts[prec] = (kt["sweeps64"], kt["sweeps32"], kt["kernel_launches"])
        plan.close()
    s64_plain, s32_plain, _ = counts[pc.PC_PREC_FP64]
    s64_mixed, s32_mixed, launches = counts[pc.PC_PREC_MIXED]
    assert s32_plain == 0 and s32_mixed > 0 and launches > 0
    assert s64_mixed < 0.7 * s64_plain, (s64_mixed, s64_plain)


def test_mixed_repack_and_edge_cases(pc, ora):
    w = W.config2(M=64)
    tf = 30 * W.DAY
    x = w.x0.copy()
    x[::2, 1] = np.nan
    g = run_gpu(pc, w, x, tf=tf, precision=pc.PC_PREC_MIXED)
    ref = run_gpu(pc, w, w.x0[1::2], tf=tf, precision=pc.PC_PREC_MIXED)
    assert (g["status"][::2] == pc.PC_IC_NONFINITE).all()
    np.testing.assert_array_equal(g["xf"][1::2], ref["xf"])
    np.testing.assert_array_equal(g["iters"][1::2], ref["iters"])
