"""The second-order sweep on the GPU (pc_options.order = 2: V' = v0 + omega2 K
A(R), then R' = r0 + omega2 K V', in the FP64 split-digit contraction as two
passes and in both FP32 kernels) against the oracle's second-order
propagation on the same inputs, within 1e-10 relative; and against the
first-order GPU path: the same answer in fewer sweeps."""
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
def test_order2_config1_vs_oracle(pc, ora, precision):
    w = W.config1()
    prec = pc.PC_PREC_MIXED if precision == "mixed" else pc.PC_PREC_FP64
    g = run_gpu(pc, w, w.x0, precision=prec, order=2)
    o = run_oracle(ora, w, w.x0, order=2)
    assert g["code"] == pc.PC_OK
    er, ev = rel_err(g["xf"], o["xf"])
    assert er.max() < TOL and ev.max() < TOL, (er.max(), ev.max())
    np.testing.assert_array_equal(g["status"], o["status"])
    np.testing.assert_array_equal(g["nseg"], o["nseg"])
    if precision == "fp64":
        assert np.abs(g["iters"] - o["iters"]).max() <= 2


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_order2_config3_subset_vs_oracle(pc, ora, precision):
    w = W.config3(M=256)
    prec = pc.PC_PREC_MIXED if precision == "mixed" else pc.PC_PREC_FP64
    g = run_gpu(pc, w, w.x0, precision=prec, switch_tol=1e-6 if precision == "mixed" else 0.0, order=2)
    o = run_oracle(ora, w, w.x0, order=2)
    assert g["code"] == pc.PC_OK
    er, ev = rel_err(g["xf"], o["xf"])
    print(f"config 3 order 2 {precision}: error vs oracle (order 2) on {w.n_ic}: position max {er.max():.2e}, "
          f"velocity max {ev.max():.2e}")
    assert er.max() < TOL and ev.max() < TOL, (er.max(), ev.max())


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_order2_config2_short_arc_and_segment_local(pc, ora, precision):
    w = W.config2(M=32)
    prec = pc.PC_PREC_MIXED if precision == "mixed" else pc.PC_PREC_FP64
    tf = 20 * W.DAY
    g = run_gpu(pc, w, w.x0, tf=tf, precision=prec, order=2)
    o = run_oracle(ora, w, w.x0, tf=tf, order=2)
    er, ev = rel_err(g["xf"], o["xf"])
    assert er.max() < TOL and ev.max() < TOL, (er.max(), ev.max())
    g = run_gpu(pc, w, w.x0[:8], max_ckpt=600, precision=prec, order=2)
    assert g["code"] == pc.PC_OK
    assert _segment_local(ora, w, g, range(8), order=2) < TOL


def test_order2_fewer_sweeps_same_answer(pc):
    """Config 3, 1024 trajectories: the second-order sweep reaches the
    first-order answer (within 1e-11) in far fewer FP64 sweeps (plain FP64) and
    FP32 sweeps (mixed)."""
    import torch
    w = W.config3(M=1024)
    x0 = torch.as_tensor(W.to_planar(w.x0), device="cuda")
    out = {}
    for prec in (pc.PC_PREC_FP64, pc.PC_PREC_MIXED):
        for order in (1, 2):
            plan = pc.plan_from_workload(w, precision=prec, switch_tol=1e-6 if prec else 0.0, order=order)
            xf = torch.zeros_like(x0)
            pc.kernel_times(plan)
            code, _ = pc.propagate(plan, x0, w.t0, w.tf, xf)
            kt = pc.kernel_times(plan)
            torch.cuda.synchronize()
            assert code == pc.PC_OK
            out[(prec, order)] = (W.from_planar(xf.cpu().numpy()), kt["sweeps64"], kt["sweeps32"])
            plan.close()
    for prec in (pc.PC_PREC_FP64, pc.PC_PREC_MIXED):
        (x1, s64a, s32a), (x2, s64b, s32b) = out[(prec, 1)], out[(prec, 2)]
        er, ev = rel_err(x2, x1)
        print(f"precision {prec}: order 1 -> 2 sweeps FP64 {s64a} -> {s64b}, FP32 {s32a} -> {s32b}; "
              f"difference position {er.max():.2e} velocity {ev.max():.2e}")
        assert er.max() < 1e-11 and ev.max() < 1e-11
    assert out[(pc.PC_PREC_FP64, 2)][1] < 0.75 * out[(pc.PC_PREC_FP64, 1)][1]
    assert out[(pc.PC_PREC_MIXED, 2)][2] < 0.8 * out[(pc.PC_PREC_MIXED, 1)][2]


def test_order2_fp32_variants_bitwise_neutral_and_validation(pc):
    import torch
    w = W.config3(M=600)
    # FP32 multiply-adds in every variant (the tensor-core contraction has its own test)
    plan = pc.plan_from_workload(w, precision=pc.PC_PREC_MIXED, switch_tol=1e-6, order=2, fp32_mma=0)
    x0d = torch.as_tensor(W.to_planar(w.x0), device="cuda")
    res = []
    for kw in (dict(fp32_rows=0, fp32_ctas_per_sm=4), dict(fp32_rows=4, fp32_slots=8, fp32_ctas_per_sm=1),
               dict(fp32_rows=8, fp32_slots=8, fp32_ctas_per_sm=1)):
        pc.set_tuning(plan, **kw)
        xf = torch.zeros_like(x0d)
        it = torch.zeros(w.n_ic, dtype=torch.int32, device="cuda")
        pc.propagate(plan, x0d, w.t0, 0.3 * W.YEAR, xf, iters=it)
        torch.cuda.synchronize()
        res.append((xf.clone(), it.clone()))
    for a, b in res[1:]:
        assert torch.equal(a, res[0][0]) and torch.equal(b, res[0][1])
    plan.close()
    with pytest.raises(pc.PCError):
        pc.plan_from_workload(w, order=2, contraction=pc.PC_CONTRACT_DMMA)
    with pytest.raises(pc.PCError):
        pc.plan_from_workload(w, order=3)
    w1 = W.config1(M=4)
    with pytest.raises(pc.PCError):
        pc.plan_create(256, 4, w1.mu_central, w1.mu, w1.t_begin, w1.granule, w1.coef,
                       options=pc.options_default(order=2))
