"""Kernel-level parity: each device kernel of the sweep, run through the C ABI,
against the CPU oracle's routine on the same seeded inputs."""
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


@pytest.fixture(scope="module")
def cfg2():
    return W.config2(M=64)


def _dev(a, dtype=None):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype or torch.float64, device="cuda")


@pytest.mark.parametrize("N", [16, 64, 128, 256])
@pytest.mark.parametrize("truncated", [0, 1])
def test_operator_matches_oracle(pc, ora, N, truncated):
    plan = pc.plan_create(N, 4, W.MU_SUN, [], options=pc.options_default(truncated=truncated))
    K, tau = pc.plan_operator(plan)
    np.testing.assert_array_equal(tau, ora.cgl_nodes(N))
    np.testing.assert_allclose(K, ora.pc_operator(N, bool(truncated)), rtol=0, atol=2e-16 * max(1, N // 32))
    plan.close()


@pytest.mark.parametrize("contraction", ["dmma", "split"])
@pytest.mark.parametrize("N", [16, 64, 128, 255, 256])
@pytest.mark.parametrize("M", [1, 3, 33, 1000])
def test_contraction_vs_oracle_operator(pc, ora, N, M, contraction):
    """The contraction y = x0 + K g (FP64 tensor cores, or exact digit products
    on the bf16 tensor cores; N = 256 has no digit operator and takes the FP64
    path) against the oracle's K applied in FP64 (numpy matmul): several node
    tiles, column tiles and a ragged tail."""
    import torch
    rng = np.random.default_rng(N * 1000 + M)
    mode = pc.PC_CONTRACT_SPLIT if contraction == "split" else pc.PC_CONTRACT_DMMA
    plan = pc.plan_create(N, 4, W.MU_SUN, [], options=pc.options_default(contraction=mode))
    x0 = rng.standard_normal((6, M)) * 1e8
    g = rng.standard_normal((N + 1, 6, M)) * 1e6
    y = torch.zeros((N + 1, 6, M), dtype=torch.float64, device="cuda")
    pc.apply_operator(plan, _dev(x0), _dev(g), y)
    torch.cuda.synchronize()
    K = ora.pc_operator(N)
    ref = x0[None] + np.einsum("jk,kcm->jcm", K, g)
    # a few ulps of the magnitudes that are summed (the order of the sum differs)
    scale = np.abs(K).sum(1).max() * np.abs(g).max() + np.abs(x0).max()
    np.testing.assert_allclose(y.cpu().numpy(), ref, rtol=0, atol=4e-16 * scale)
    np.testing.assert_array_equal(y.cpu().numpy()[0], x0)
    plan.close()


def test_split_contraction_edge_cases(pc, ora):
    """Digit contraction: columns of very different scale in one tile (each is
    cut against its own exponent), an all-zero column, subnormal and tiny
    entries next to large ones, and a NaN or an inf in one trajectory's
    columns, which must reach every node of that trajectory and no other."""
    import torch
    N, M = 128, 21
    rng = np.random.default_rng(3)
    plan = pc.plan_create(N, 4, W.MU_SUN, [], options=pc.options_default(contraction=pc.PC_CONTRACT_SPLIT))
    x0 = rng.standard_normal((6, M)) * 1e8
    g = rng.standard_normal((N + 1, 6, M)) * (10.0 ** rng.integers(-30, 30, size=(1, 6, M)))
    g[:, 2, 4] = 0.0
    g[5, 1, 6] = 5e-320
    g[7, 0, 6] = 1e-300
    g[11, 3, 9] = np.nan
    g[13, 5, 17] = np.inf
    y = torch.zeros((N + 1, 6, M), dtype=torch.float64, device="cuda")
    pc.apply_operator(plan, _dev(x0), _dev(g), y)
    torch.cuda.synchronize()
    got = y.cpu().numpy()
    K = ora.pc_operator(N)
    ok = np.ones(M, dtype=bool)
    ok[[9, 17]] = False
    assert np.isnan(got[1:, :, ~ok]).all()
    np.testing.assert_array_equal(got[0], x0)
    ld = np.longdouble
    ref = (x0[None, :, ok].astype(ld) + np.einsum("jk,kcm->jcm", K.astype(ld), g[:, :, ok].astype(ld))).astype(float)
    # per column: a few ulps of sum |K| times the column's own largest |g|
    scale = np.abs(K).sum(1).max() * np.abs(g[:, :, ok]).max(0)[None] + np.abs(x0[None, :, ok])
    assert (np.abs(got[:, :, ok] - ref) <= 4e-16 * scale).all()
    plan.close()


def test_ephemeris_vs_oracle(pc, ora, cfg2):
    import torch
    plan = pc.plan_from_workload(cfg2)
    m = ora.Model.from_workload(cfg2)
    rng = np.random.default_rng(5)
    t = np.concatenate([rng.uniform(cfg2.t0, cfg2.tf, 997),
                        cfg2.t_begin + cfg2.granule * np.arange(3, 9)])       # boundary ties
    B = len(cfg2.mu)
    rb = torch.zeros((B, 3, t.size), dtype=torch.float64, device="cuda")
    pc.eval_ephemeris(plan, _dev(t), rb)
    got = rb.cpu().numpy()
    ref = np.stack([ora.ephem_eval(m, ti) for ti in t], axis=-1)          # [B][3][n]
    # The oracle sums the series by Clenshaw's recurrence, the library by a
    # power sum over recurrence-built T_k: the same series in two rounding
    # orders.  Bound per value: 4 (deg+1) ulps of sum_k |c_k| of its granule,
    # which a wrong granule, sigma map or axis stride exceeds by many orders.
    deg = cfg2.coef.shape[3] - 1
    g = np.clip(np.floor((t - cfg2.t_begin) / cfg2.granule).astype(int), 0, cfg2.coef.shape[1] - 1)
    scale = np.abs(cfg2.coef[:, g, :, :]).sum(-1).transpose(0, 2, 1)      # [B][3][n]
    err = np.abs(got - ref)
    assert (err <= 4 * (deg + 1) * 2.2e-16 * scale).all(), (err / scale).max()
    plan.close()


def test_dynamics_vs_oracle(pc, ora, cfg2):
    """Force at states near and far from the bodies (including 1e4 km from Venus)."""
    import torch
    plan = pc.plan_from_workload(cfg2)
    m = ora.Model.from_workload(cfg2)
    o = ora.Opts()
    rng = np.random.default_rng(6)
    n = 515
    t = rng.uniform(cfg2.t0, cfg2.tf, n)
    y = np.zeros((6, n))
    for i in range(n):
        rb = ora.ephem_eval(m, t[i])
        if i % 5 == 0:
            d = rng.standard_normal(3)
            y[:3, i] = rb[1] + d / np.linalg.norm(d) * rng.uniform(1e4, 1e6)
        else:
            y[:3, i] = rng.standard_normal(3) * 1.5e8
        y[3:, i] = rng.standard_normal(3) * 30.0
    f = torch.zeros((6, n), dtype=torch.float64, device="cuda")
    pc.eval_dynamics(plan, _dev(t), _dev(y), f)
    got = f.cpu().numpy()
    deg = cfg2.coef.shape[3] - 1
    for i in range(n):
        ref = ora.dynamics(m, o, t[i], y[:, i])
        np.testing.assert_array_equal(got[:3, i], ref[:3])
        # rounding bound: a few ulps of each term's magnitude (direct and
        # indirect), plus the body-position difference of the two ephemeris
        # summation orders (bounded as in test_ephemeris_vs_oracle) times the
        # tidal factor 3 mu_b / |r - r_b|^3 of each body
        rb = ora.ephem_eval(m, t[i])
        r = y[:3, i]
        g = int(np.clip(np.floor((t[i] - cfg2.t_begin) / cfg2.granule), 0, cfg2.coef.shape[1] - 1))
        eps_b = 4 * (deg + 1) * 2.2e-16 * np.abs(cfg2.coef[:, g]).sum(-1).max(-1)
        mag = W.MU_SUN / (r @ r) + sum(mu / ((r - p) @ (r - p)) + mu / (p @ p) for mu, p in zip(cfg2.mu, rb))
        eph = sum(3 * mu * e / np.linalg.norm(r - p) ** 3 + 3 * mu * e / np.linalg.norm(p) ** 3
                  for mu, p, e in zip(cfg2.mu, rb, eps_b))
        np.testing.assert_allclose(got[3:, i], ref[3:], rtol=0, atol=2e-15 * mag + eph)
    plan.close()


def test_warm_start_vs_oracle_kepler(pc, ora):
    import torch
    plan = pc.plan_create(16, 4, W.MU_SUN, [])
    rng = np.random.default_rng(7)
    n = 300
    x0 = np.zeros((6, n))
    dt = rng.uniform(-3e7, 3e7, n)
    for i in range(n):
        x0[:, i] = W.elements_to_state(rng.uniform(0.3, 5) * W.AU, rng.uniform(0, 0.9), rng.uniform(0, 3),
                                       rng.uniform(0, 6), rng.uniform(0, 6), rng.uniform(0, 6), W.MU_SUN)
    x0[:, -1] = [1e8, 0, 0, 0, 60.0, 0]       # hyperbolic: copied unchanged (cold start)
    x = torch.zeros((6, n), dtype=torch.float64, device="cuda")
    pc.eval_warm_start(plan, _dev(x0), _dev(dt), x)
    got = x.cpu().numpy()
    for i in range(n - 1):
        ref, rc = ora.kepler(W.MU_SUN, x0[:, i], dt[i])
        assert rc == 0
        np.testing.assert_allclose(got[:3, i], ref[:3], rtol=0, atol=1e-11 * np.linalg.norm(ref[:3]))
        np.testing.assert_allclose(got[3:, i], ref[3:], rtol=0, atol=1e-11 * np.linalg.norm(ref[3:]))
    np.testing.assert_array_equal(got[:, -1], x0[:, -1])
    plan.close()
