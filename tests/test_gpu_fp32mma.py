"""FP32 sweeps with the operator contraction on the tensor cores
(pc_options.fp32_mma = 1: three TF32 products per term, FP32 accumulation)
against the FP64 oracle: after the FP64 sweeps the result meets the same
1e-10 bound as every other path; the sweep counts stay within a few per cent
of those of the FP32 multiply-add contraction; and the launch shape (slots per CTA, the
ignored fp32_rows) does not change a bit."""
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


@pytest.mark.parametrize("order", [1, 2])
def test_fp32_mma_config1_vs_oracle(pc, ora, order):
    w = W.config1()
    g = run_gpu(pc, w, w.x0, precision=pc.PC_PREC_MIXED, switch_tol=1e-6, order=order, fp32_mma=1)
    o = run_oracle(ora, w, w.x0, order=order)
    assert g["code"] == pc.PC_OK
    er, ev = rel_err(g["xf"], o["xf"])
    assert er.max() < TOL and ev.max() < TOL, (er.max(), ev.max())
    np.testing.assert_array_equal(g["nseg"], o["nseg"])


@pytest.mark.parametrize("order", [1, 2])
def test_fp32_mma_config3_subset_vs_oracle_and_sweeps(pc, ora, order):
    """Config 3, 256 trajectories, 2-year arcs: error against the oracle, and
    the FP64 sweeps the mixed path needs within 2 % of those of the
    multiply-add contraction (FP32 sweeps within 10 %)."""
    import torch
    w = W.config3(M=256)
    g = run_gpu(pc, w, w.x0, precision=pc.PC_PREC_MIXED, switch_tol=1e-6, order=order, fp32_mma=1)
    o = run_oracle(ora, w, w.x0, order=order)
    assert g["code"] == pc.PC_OK
    er, ev = rel_err(g["xf"], o["xf"])
    print(f"config 3 fp32_mma order {order}: error vs oracle position {er.max():.2e} velocity {ev.max():.2e}")
    assert er.max() < TOL and ev.max() < TOL, (er.max(), ev.max())
    counts = {}
    for mma in (0, 1):
        plan = pc.plan_from_workload(w, precision=pc.PC_PREC_MIXED, switch_tol=1e-6, order=order, fp32_mma=mma)
        x0d = torch.as_tensor(W.to_planar(w.x0), device="cuda")
        xf = torch.zeros_like(x0d)
        pc.kernel_times(plan)  # clears the sweep counters
        pc.propagate(plan, x0d, w.t0, w.tf, xf)
        torch.cuda.synchronize()
        kt = pc.kernel_times(plan)
        counts[mma] = (kt["sweeps64"], kt["sweeps32"])
        plan.close()
    print("sweeps (FP64, FP32) multiply-add / tensor cores:", counts[0], counts[1])
    # the two contractions round differently (tensor-core FP32 accumulation),
    # so an FP32 phase can end a sweep apart; the work stays the same
    assert abs(counts[1][0] - counts[0][0]) <= 0.02 * counts[0][0]
    assert abs(counts[1][1] - counts[0][1]) <= 0.1 * counts[0][1]


def test_fp32_mma_config2_many_bodies(pc, ora):
    """Config 2 (Sun, 8 planets, Moon; Venus flybys), 32 trajectories: 20-day
    arcs end to end, and the full arcs segment by segment."""
    w = W.config2(M=32)
    tf = 20 * W.DAY
    g = run_gpu(pc, w, w.x0, tf=tf, precision=pc.PC_PREC_MIXED, fp32_mma=1)
    o = run_oracle(ora, w, w.x0, tf=tf)
    assert g["code"] == pc.PC_OK
    er, ev = rel_err(g["xf"], o["xf"])
    assert er.max() < TOL and ev.max() < TOL, (er.max(), ev.max())
    g = run_gpu(pc, w, w.x0[:8], max_ckpt=600, precision=pc.PC_PREC_MIXED, fp32_mma=1)
    assert g["code"] == pc.PC_OK
    assert _segment_local(ora, w, g, range(8)) < TOL


def test_fp32_mma_launch_shapes_bitwise_neutral(pc):
    """Slots per CTA (8, 16, 32: fewer when shared memory is short), FP32 CTAs
    per SM, graphs, and fp32_rows (ignored by this path) give bitwise the
    same results, order 1 and 2."""
    import torch
    w = W.config3(M=600)
    x0d = torch.as_tensor(W.to_planar(w.x0), device="cuda")
    for order in (1, 2):
        plan = pc.plan_from_workload(w, precision=pc.PC_PREC_MIXED, switch_tol=1e-6, order=order, fp32_mma=1)
        res = []
        for kw in (dict(), dict(fp32_slots=8), dict(fp32_slots=32, fp32_ctas_per_sm=2), dict(fp32_rows=0),
                   dict(fp32_rows=8, graphs=0)):
            pc.set_tuning(plan, **kw)
            xf = torch.zeros_like(x0d)
            it = torch.zeros(w.n_ic, dtype=torch.int32, device="cuda")
            pc.propagate(plan, x0d, w.t0, 0.3 * W.YEAR, xf, iters=it)
            torch.cuda.synchronize()
            res.append((xf.clone(), it.clone()))
            pc.set_tuning(plan, fp32_slots=16, fp32_ctas_per_sm=1, fp32_rows=4, graphs=1)
        for a, b in res[1:]:
            assert torch.equal(a, res[0][0]) and torch.equal(b, res[0][1]), order
        plan.close()
