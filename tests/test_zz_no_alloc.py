"""The allocation-free contraction entry point (pc_apply_operator_static).

It is for callers that cannot allocate device memory when they call in: a
caller whose GPU memory belongs to another allocator with a fixed budget, or
one that must not risk the implicit synchronisation of cudaMalloc/cudaFree.
It stages through a fixed array inside the library instead of the plan's
workspace.  Checked here against the allocating entry point
(pc_apply_operator) on two calls in a row -- the second with a different size,
so stale contents of the shared array from the first call would show -- and
for its size limit.  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2301_03989_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pc():
    import torch
    from paper_2301_03989_gb300 import build, pcprop
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return pcprop


def _case(rng, N, M):
    x0 = rng.standard_normal((6, M)) * 1e8
    g = rng.standard_normal((N + 1, 6, M)) * 1e6
    return x0, g


def _tol(ora, N, x0, g):
    K = ora.pc_operator(N)      # same bound as the contraction parity test
    return 4e-16 * (np.abs(K).sum(1).max() * np.abs(g).max() + np.abs(x0).max())


def test_static_operator_matches_allocating_entry_point_twice(pc, ora):
    import torch
    rng = np.random.default_rng(2024)
    for N, M in [(128, 1000), (64, 37)]:
        plan = pc.plan_create(N, 4, W.MU_SUN, [])
        x0, g = _case(rng, N, M)
        xd = torch.as_tensor(x0, device="cuda")
        gd = torch.as_tensor(g, device="cuda")
        y_ref = torch.zeros((N + 1, 6, M), dtype=torch.float64, device="cuda")
        y_sta = torch.full((N + 1, 6, M), np.nan, dtype=torch.float64, device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        code = pc.lib().pc_apply_operator(plan.handle, M, xd.data_ptr(), gd.data_ptr(), y_ref.data_ptr(), stream)
        assert code == pc.PC_OK
        code = pc.lib().pc_apply_operator_static(plan.handle, M, xd.data_ptr(), gd.data_ptr(), y_sta.data_ptr(),
                                                 stream)
        assert code == pc.PC_OK
        torch.cuda.synchronize()
        a, b = y_ref.cpu().numpy(), y_sta.cpu().numpy()
        np.testing.assert_allclose(b, a, rtol=0, atol=_tol(ora, N, x0, g))
        # and against the oracle's operator, like the allocating path
        ref = x0[None] + np.einsum("jk,kcm->jcm", ora.pc_operator(N), g)
        np.testing.assert_allclose(b, ref, rtol=0, atol=_tol(ora, N, x0, g))
        plan.close()


def test_static_operator_rejects_sizes_beyond_the_array(pc):
    import torch
    N = 128
    plan = pc.plan_create(N, 4, W.MU_SUN, [])
    M = 2672                                   # first size past the 32 MiB array at N = 128
    x0 = torch.zeros((6, M), dtype=torch.float64, device="cuda")
    g = torch.zeros((N + 1, 6, M), dtype=torch.float64, device="cuda")
    y = torch.zeros_like(g)
    code = pc.lib().pc_apply_operator_static(plan.handle, M, x0.data_ptr(), g.data_ptr(), y.data_ptr(), None)
    assert code == pc.PC_EINVAL
    ok = pc.lib().pc_apply_operator_static(plan.handle, 2664, x0.data_ptr(), g.data_ptr(), y.data_ptr(), None)
    assert ok == pc.PC_OK
    torch.cuda.synchronize()
    plan.close()
