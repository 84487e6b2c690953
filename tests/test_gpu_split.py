"""End-to-end parity of the split-digit FP64 contraction (PC_CONTRACT_SPLIT:
exact 8-bit digit products on the bf16 tensor cores) against the CPU oracle,
plain FP64 and mixed precision, and its agreement with the FP64 tensor-core
contraction (PC_CONTRACT_DMMA) on the same inputs.  Same bound as every other
path: 1e-10 relative in position and velocity."""
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


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_split_config1_vs_oracle(pc, ora, precision):
    w = W.config1()
    prec = pc.PC_PREC_MIXED if precision == "mixed" else pc.PC_PREC_FP64
    g = run_gpu(pc, w, w.x0, precision=prec, contraction=pc.PC_CONTRACT_SPLIT)
    o = run_oracle(ora, w, w.x0)
    assert g["code"] == pc.PC_OK
    er, ev = rel_err(g["xf"], o["xf"])
    assert er.max() < TOL and ev.max() < TOL, (er.max(), ev.max())
    np.testing.assert_array_equal(g["status"], o["status"])
    np.testing.assert_array_equal(g["nseg"], o["nseg"])
    if precision == "fp64":  # (mixed precision counts its FP32 sweeps too)
        assert np.abs(g["iters"] - o["iters"]).max() <= 2


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_split_config3_subset_vs_oracle(pc, ora, precision):
    w = W.config3(M=256)
    prec = pc.PC_PREC_MIXED if precision == "mixed" else pc.PC_PREC_FP64
    g = run_gpu(pc, w, w.x0, precision=prec, switch_tol=1e-6 if precision == "mixed" else 0.0,
                contraction=pc.PC_CONTRACT_SPLIT)
    o = run_oracle(ora, w, w.x0)
    assert g["code"] == pc.PC_OK
    er, ev = rel_err(g["xf"], o["xf"])
    print(f"config 3 split {precision}: error vs oracle on {w.n_ic} trajectories: position max {er.max():.2e}, "
          f"velocity max {ev.max():.2e}")
    assert er.max() < TOL and ev.max() < TOL, (er.max(), ev.max())


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_split_config2_short_arc_and_segment_local(pc, ora, precision):
    """Close Venus flybys (Sun + 8 planets + Moon): 20 days end to end, and a
    full 4-year arc segment by segment."""
    w = W.config2(M=48)
    prec = pc.PC_PREC_MIXED if precision == "mixed" else pc.PC_PREC_FP64
    tf = 20 * W.DAY
    g = run_gpu(pc, w, w.x0, tf=tf, precision=prec, contraction=pc.PC_CONTRACT_SPLIT)
    o = run_oracle(ora, w, w.x0, tf=tf)
    er, ev = rel_err(g["xf"], o["xf"])
    assert er.max() < TOL and ev.max() < TOL, (er.max(), ev.max())
    assert (g["nseg"] != o["nseg"]).mean() <= 1 / 16
    g = run_gpu(pc, w, w.x0[:12], max_ckpt=600, precision=prec, contraction=pc.PC_CONTRACT_SPLIT)
    assert g["code"] == pc.PC_OK
    assert _segment_local(ora, w, g, range(12)) < TOL


def test_split_matches_dmma(pc):
    """Config 3, 1024 trajectories, plain FP64: the two contractions give the
    same trajectories to well within the tolerance, and the same segment
    counts."""
    w = W.config3(M=1024)
    a = run_gpu(pc, w, w.x0, contraction=pc.PC_CONTRACT_DMMA)
    b = run_gpu(pc, w, w.x0, contraction=pc.PC_CONTRACT_SPLIT)
    er, ev = rel_err(b["xf"], a["xf"])
    print(f"split vs DMMA, config 3 (1024): position max {er.max():.2e}, velocity max {ev.max():.2e}; "
          f"sweeps {int(a['iters'].sum())} vs {int(b['iters'].sum())}")
    assert er.max() < 1e-11 and ev.max() < 1e-11
    np.testing.assert_array_equal(a["nseg"], b["nseg"])
    assert abs(int(a["iters"].sum()) - int(b["iters"].sum())) <= 0.01 * int(a["iters"].sum())
