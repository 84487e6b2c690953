"""Launch tuning, CUDA-graph replay and the autotuner: none of them may change
a single bit of the results (they move work between CTAs, batch the host's
round loop, or replay the same launches from a graph)."""
import numpy as np
import pytest

from paper_2301_03989_gb300 import workloads as W

pytestmark = pytest.mark.gpu

DEFAULT_TUNING = dict(setup_ctas_per_sm=4, fp32_ctas_per_sm=1, contract_ctas_per_sm=4, rounds_per_batch=8,
                      repack_div=8, graphs=1, side_priority=1, fp32_rows=4, fp32_slots=16, grid_cache=1)


@pytest.fixture(scope="module")
def pc():
    import torch
    from paper_2301_03989_gb300 import build, pcprop
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return pcprop


def _run(pc, plan, w, x0d, tf, stream=None):
    import torch
    M = x0d.shape[1]
    xf = torch.zeros_like(x0d)
    st = torch.zeros(M, dtype=torch.int32, device="cuda")
    it = torch.zeros(M, dtype=torch.int32, device="cuda")
    ns = torch.zeros(M, dtype=torch.int32, device="cuda")
    code, rounds = pc.propagate(plan, x0d, w.t0, tf, xf, status=st, iters=it, nseg=ns, stream=stream)
    torch.cuda.synchronize()
    return code, rounds, xf.clone(), st.clone(), it.clone(), ns.clone()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_tunings_and_graphs_are_bitwise_neutral(pc, precision):
    import torch
    w = W.config2(M=384)
    prec = pc.PC_PREC_MIXED if precision == "mixed" else pc.PC_PREC_FP64
    plan = pc.plan_from_workload(w, precision=prec)
    x0d = torch.as_tensor(W.to_planar(w.x0), device="cuda")
    tf = 0.25 * W.YEAR
    base = _run(pc, plan, w, x0d, tf)
    assert base[0] in (pc.PC_OK, pc.PC_ENOTCONV)
    settings = [dict(graphs=0), dict(graphs=1, rounds_per_batch=2), dict(contract_ctas_per_sm=1, setup_ctas_per_sm=1),
                dict(contract_ctas_per_sm=8, fp32_ctas_per_sm=16, setup_ctas_per_sm=16),
                dict(repack_div=2, rounds_per_batch=16), dict(repack_div=64, rounds_per_batch=5, graphs=1),
                dict(side_priority=0, contract_ctas_per_sm=16), dict(grid_cache=0),
                # FP32 kernels: one trajectory per CTA, and tiles of 4 / 8 rows per thread with 8..64 slots
                dict(fp32_rows=0, fp32_ctas_per_sm=4), dict(fp32_rows=4, fp32_slots=8, fp32_ctas_per_sm=2),
                dict(fp32_rows=8, fp32_slots=32), dict(fp32_rows=4, fp32_slots=64, fp32_ctas_per_sm=3)]
    for kw in settings:
        pc.set_tuning(plan, **kw)
        r = _run(pc, plan, w, x0d, tf)
        for a, b in zip(base[2:], r[2:]):
            assert torch.equal(a, b), kw
        pc.set_tuning(plan, **DEFAULT_TUNING)
    # the caller's own (non-default) stream: no fork, graph captured on it directly
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        r = _run(pc, plan, w, x0d, tf, stream=s)
    for a, b in zip(base[2:], r[2:]):
        assert torch.equal(a, b)
    plan.close()


def test_fp32_variants_are_bitwise_neutral_on_few_bodies(pc):
    """Config 3 (Sun + Venus + Earth): the tiled FP32 kernel keeps its
    trajectories' node records in shared memory (with many bodies they do not
    fit and the one-trajectory-per-CTA kernel runs instead); every tile shape
    and the one-trajectory-per-CTA kernel give bitwise the same results."""
    import torch
    w = W.config3(M=600)
    # FP32 multiply-adds (fp32_mma = 0): every tiled shape against the one-trajectory kernel
    plan = pc.plan_from_workload(w, precision=pc.PC_PREC_MIXED, switch_tol=1e-6, fp32_mma=0)
    x0d = torch.as_tensor(W.to_planar(w.x0), device="cuda")
    tf = 0.3 * W.YEAR
    pc.set_tuning(plan, fp32_rows=0, fp32_ctas_per_sm=4)
    base = _run(pc, plan, w, x0d, tf)
    assert base[0] == pc.PC_OK
    # 8 slots stage their node records in shared memory; 16 and more read them
    # from global memory (4 rows per thread: 512 threads per CTA)
    for kw in (dict(fp32_rows=4, fp32_slots=8, fp32_ctas_per_sm=1), dict(fp32_rows=8, fp32_slots=8),
               dict(fp32_rows=4, fp32_slots=16), dict(fp32_rows=4, fp32_slots=64, fp32_ctas_per_sm=2),
               dict(fp32_rows=8, fp32_slots=16, graphs=0)):
        pc.set_tuning(plan, **kw)
        r = _run(pc, plan, w, x0d, tf)
        for a, b in zip(base[2:], r[2:]):
            assert torch.equal(a, b), kw
        pc.set_tuning(plan, **DEFAULT_TUNING)
    plan.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_grid_cache_is_bitwise_neutral_on_shared_grids(pc, precision):
    """Config 3 (uniform segments over a common arc): most segments of a round
    share their node times, so the set-up kernel copies body positions from the
    per-grid ephemeris cache; with the cache off every segment evaluates its
    own.  Both give bitwise the same results, order 1 and 2, and so does a
    batch whose trajectories start at two different epochs."""
    import torch
    w = W.config3(M=1000)
    prec = pc.PC_PREC_MIXED if precision == "mixed" else pc.PC_PREC_FP64
    x0d = torch.as_tensor(W.to_planar(w.x0), device="cuda")
    for order in (1, 2):
        plan = pc.plan_from_workload(w, precision=prec, switch_tol=1e-6 if precision == "mixed" else 0.0,
                                     order=order)
        tf = 0.4 * W.YEAR
        base = _run(pc, plan, w, x0d, tf)
        assert base[0] == pc.PC_OK
        pc.set_tuning(plan, grid_cache=0)
        r = _run(pc, plan, w, x0d, tf)
        for a, b in zip(base[2:], r[2:]):
            assert torch.equal(a, b), order
        plan.close()
    # per-trajectory arcs from two epochs: two families of grids in one round
    plan = pc.plan_from_workload(w, precision=prec, switch_tol=1e-6 if precision == "mixed" else 0.0)
    M = 1000
    t0 = torch.full((M,), w.t0, dtype=torch.float64, device="cuda")
    t0[1::2] += 3.0 * W.DAY
    tf = t0 + 0.3 * W.YEAR
    outs = []
    for gc in (1, 0):
        pc.set_tuning(plan, grid_cache=gc)
        xf = torch.zeros_like(x0d)
        st = torch.zeros(M, dtype=torch.int32, device="cuda")
        code, _ = pc.propagate_groups([plan], [M], x0d, t0, tf, xf, status=st)
        torch.cuda.synchronize()
        assert code == pc.PC_OK
        outs.append(xf.clone())
    assert torch.equal(outs[0], outs[1])
    plan.close()


def test_grid_cache_over_capacity_is_bitwise_neutral(pc):
    """40,000 flyby trajectories whose segments follow their own osculating
    periods: every segment of the first round has its own node-time grid, more
    than the cache's 32,768, so the grids past the capacity are evaluated per
    segment; with the cache off all are.  Bitwise the same results."""
    import torch
    w = W.config2(M=40000)
    x0d = torch.as_tensor(W.to_planar(w.x0), device="cuda")
    tf = w.t0 + 2.0 * W.DAY
    plan = pc.plan_from_workload(w)
    base = _run(pc, plan, w, x0d, tf)
    assert base[0] in (pc.PC_OK, pc.PC_ENOTCONV)
    pc.set_tuning(plan, grid_cache=0)
    r = _run(pc, plan, w, x0d, tf)
    for a, b in zip(base[2:], r[2:]):
        assert torch.equal(a, b)
    plan.close()


def test_tuning_validation(pc):
    w = W.config1(M=8)
    plan = pc.plan_from_workload(w)
    for bad in (dict(setup_ctas_per_sm=0), dict(contract_ctas_per_sm=17), dict(rounds_per_batch=0),
                dict(repack_div=1), dict(graphs=2), dict(fp32_ctas_per_sm=17), dict(side_priority=2),
                dict(fp32_rows=2), dict(fp32_slots=12), dict(fp32_slots=0), dict(fp32_slots=72),
                dict(grid_cache=2), dict(grid_cache=-1)):
        with pytest.raises(pc.PCError):
            pc.set_tuning(plan, **bad)
    assert pc.get_tuning(plan) == DEFAULT_TUNING
    plan.close()


def test_autotune_picks_a_neutral_setting(pc):
    import torch
    w = W.config2(M=512)
    plan = pc.plan_from_workload(w, precision=pc.PC_PREC_MIXED)
    x0d = torch.as_tensor(W.to_planar(w.x0), device="cuda")
    tf = 0.25 * W.YEAR
    pc.set_tuning(plan, graphs=0)
    base = _run(pc, plan, w, x0d, tf)
    best = pc.autotune(plan, x0d, w.t0, tf, max_rounds=64)
    assert pc.get_tuning(plan) == best
    r = _run(pc, plan, w, x0d, tf)
    for a, b in zip(base[2:], r[2:]):
        assert torch.equal(a, b)
    print("autotuned:", best)
    plan.close()
