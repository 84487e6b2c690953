"""Reverse mode (pc_propagate_tape / pc_adjoint_tape / pc_propagate_adjoint),
the b-plane (pc_bplane) and the autograd wrappers, on the differentiation
workload (config-1 system, one close Venus flyby per arc, N = 128).

References:
  * the oracle's PC run of the variational equations (6 + 36 states) over the
    GPU's own segment schedule -- the derivative of the same discrete map;
  * central finite differences of the GPU forward pass, 1e-3 km / 1e-6 km/s
    steps (and their Richardson extrapolation), on trajectories whose segment and sweep counts are the same at both
    steps (a halving decided differently, or one sweep more, is a different
    discrete map; the segment times themselves move smoothly with x0 when the
    base length follows the osculating period, at no first-order cost);
  * the oracle's b-plane and central differences of it.
Jacobians are compared with column j scaled by its step h_j (km vs km/s)."""
import numpy as np
import pytest

from paper_2301_03989_gb300 import workloads as W
from test_gpu_parity import TOL, rel_err

pytestmark = pytest.mark.gpu
H6 = np.array([1e-3, 1e-3, 1e-3, 1e-6, 1e-6, 1e-6])


@pytest.fixture(scope="module")
def pc():
    import torch
    from paper_2301_03989_gb300 import build, pcprop
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return pcprop


def _dev(a, dtype=None):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype or torch.float64, device="cuda")


def _scaled_rel(J, Jref, h):
    d = np.abs((J - Jref) * h[None, :])
    return d.max() / np.abs(Jref * h[None, :]).max()


def _tape_run(pc, plan, x0, t0, tf, cap=256):
    import torch
    M = x0.shape[0]
    rec = pc.tape_record(plan)
    tape = torch.zeros(M * cap * rec, dtype=torch.float64, device="cuda")
    xf = torch.zeros((6, M), dtype=torch.float64, device="cuda")
    ns = torch.zeros(M, dtype=torch.int32, device="cuda")
    st = torch.zeros(M, dtype=torch.int32, device="cuda")
    code = pc.propagate_tape(plan, _dev(W.to_planar(x0)), _dev(np.broadcast_to(t0, (M,))),
                             _dev(np.broadcast_to(tf, (M,))), xf, ns, tape, cap, status=st)
    torch.cuda.synchronize()
    assert int(ns.max()) <= cap
    return code, xf, ns, st, tape, cap


def _jacobians(pc, plan, ns, cap, tape, M):
    """Phi [M][6][6] from six reverse sweeps with unit cotangents."""
    import torch
    Phi = np.zeros((M, 6, 6))
    for i in range(6):
        xb = torch.zeros((6, M), dtype=torch.float64, device="cuda")
        xb[i] = 1.0
        x0b = torch.zeros_like(xb)
        ast = torch.zeros(M, dtype=torch.int32, device="cuda")
        code = pc.adjoint_tape(plan, ns, cap, tape, xb, x0b, status=ast)
        assert code == pc.PC_OK and int(ast.max()) & ~pc.PC_IC_STALLED == 0
        Phi[:, i, :] = x0b.cpu().numpy().T
    return Phi


def test_adjoint_matches_oracle_variational(pc, ora):
    """x0_bar = Phi^T xf_bar with Phi from the oracle's variational PC run over
    the GPU's segment schedule, through the flyby (first 20 days of the arc)."""
    w = W.config4(M=6)
    plan = pc.plan_from_workload(w)
    tf = 20 * W.DAY
    code, xf, ns, st, tape, cap = _tape_run(pc, plan, w.x0, w.t0, tf)
    assert code == pc.PC_OK
    Phi = _jacobians(pc, plan, ns, cap, tape, w.n_ic)
    rec = pc.tape_record(plan)
    tp = tape.cpu().numpy().reshape(w.n_ic, cap, rec)
    m = ora.Model.from_workload(w)
    o = ora.Opts(N=w.N, tol=w.tol, max_iters=w.max_iters)
    xg = W.from_planar(xf.cpu().numpy())
    worst = 0.0
    for i in range(w.n_ic):
        k = int(ns.cpu()[i])
        bounds = np.r_[tp[i, :k, 0], tp[i, k - 1, 1]]
        assert bounds[-1] == tf and k >= 2
        x_ora, P_ora, capped, _ = ora.stm_propagate(m, o, w.x0[i], bounds)
        assert capped == 0
        er, ev = rel_err(xg[i:i + 1], x_ora[None])
        assert er.max() < TOL and ev.max() < TOL
        worst = max(worst, _scaled_rel(Phi[i], P_ora, H6))
    print(f"adjoint vs oracle variational: worst scaled rel {worst:.3e}; segments {ns.cpu().numpy().tolist()}")
    assert worst < 1e-8
    plan.close()


def _fd_jacobian(pc, plan, w, h, base_ns):
    """Central differences of the GPU forward pass with steps h [6], and a mask
    of the trajectories whose segment and sweep counts match at both steps."""
    import torch
    M = w.n_ic
    xs = np.concatenate([w.x0 + s * h[q] * np.eye(6)[q] for q in range(6) for s in (1.0, -1.0)])
    n = xs.shape[0]
    xd = _dev(W.to_planar(xs))
    xo = torch.zeros_like(xd)
    it = torch.zeros(n, dtype=torch.int32, device="cuda")
    nn = torch.zeros(n, dtype=torch.int32, device="cuda")
    pc.propagate(plan, xd, w.t0, w.tf, xo, iters=it, nseg=nn)
    torch.cuda.synchronize()
    xo = W.from_planar(xo.cpu().numpy()).reshape(6, 2, M, 6)
    it = it.cpu().numpy().reshape(6, 2, M)
    nn = nn.cpu().numpy().reshape(6, 2, M)
    same = np.ones(M, dtype=bool)
    fd = np.zeros((M, 6, 6))
    for q in range(6):
        same &= (nn[q, 0] == base_ns) & (nn[q, 0] == nn[q, 1]) & (it[q, 0] == it[q, 1])
        fd[:, :, q] = (xo[q, 0] - xo[q, 1]) / (2 * h[q])
    return fd, same


def test_adjoint_matches_finite_differences(pc):
    """Adjoint Jacobian of xf over a full config-4 arc (flyby included) against
    central differences of the GPU forward pass at the 1e-3 km / 1e-6 km/s
    steps, and against their Richardson extrapolation with the half steps
    ((4 D(h/2) - D(h)) / 3 removes the h^2 term, which dominates on the most
    strongly bent flybys)."""
    w = W.config4(M=256)
    plan = pc.plan_from_workload(w)
    M = w.n_ic
    code, xf, ns, st, tape, cap = _tape_run(pc, plan, w.x0, w.t0, w.tf)
    Phi = _jacobians(pc, plan, ns, cap, tape, M)
    base_ns = ns.cpu().numpy()
    fd1, same1 = _fd_jacobian(pc, plan, w, H6, base_ns)
    fd2, same2 = _fd_jacobian(pc, plan, w, 0.5 * H6, base_ns)
    same = same1 & same2
    fdr = (4.0 * fd2 - fd1) / 3.0
    e1 = np.array([_scaled_rel(Phi[i], fd1[i], H6) for i in range(M)])[same]
    er = np.array([_scaled_rel(Phi[i], fdr[i], H6) for i in range(M)])[same]
    print(f"adjoint vs FD: {same.sum()} of {M} with equal counts; central median {np.median(e1):.2e} "
          f"max {e1.max():.2e}; Richardson median {np.median(er):.2e} max {er.max():.2e}")
    assert same.mean() > 0.6
    assert np.median(e1) < 1e-7 and np.quantile(e1, 0.95) < 1e-6
    assert er.max() < 1e-6
    plan.close()


def test_propagate_adjoint_entry_point(pc):
    """pc_propagate_adjoint (plan-held tape, scalar arc) equals the tape path."""
    import torch
    w = W.config4(M=16)
    plan = pc.plan_from_workload(w)
    M = w.n_ic
    code, xf, ns, st, tape, cap = _tape_run(pc, plan, w.x0, w.t0, w.tf)
    rng = np.random.default_rng(7)
    xb = _dev(rng.standard_normal((6, M)))
    a = torch.zeros_like(xb)
    pc.adjoint_tape(plan, ns, cap, tape, xb, a)
    b = torch.zeros_like(xb)
    code = pc.propagate_adjoint(plan, _dev(W.to_planar(w.x0)), w.t0, w.tf, xb, b)
    torch.cuda.synchronize()
    assert code == pc.PC_OK
    assert torch.equal(a, b)
    plan.close()


def _venus_rel(ora, w, t, x):
    m = ora.Model.from_workload(w)
    b = w.meta["body"]
    return x - np.r_[ora.ephem_eval(m, t)[b], ora.ephem_vel(m, t)[b]]


def test_bplane_matches_oracle(pc, ora):
    """pc_bplane against the oracle's b-plane of the same Venus-relative state
    (body velocity from the table derivative), and its Jacobian against central
    differences of the oracle's b-plane."""
    import torch
    w = W.config4(M=64)
    plan = pc.plan_from_workload(w)
    m = ora.Model.from_workload(w)
    b, mu = w.meta["body"], w.meta["mu_body"]
    t = np.full(w.n_ic, w.t0)          # the ICs themselves: 2-5 days before periapsis
    out = torch.zeros((2, w.n_ic), dtype=torch.float64, device="cuda")
    jac = torch.zeros((12, w.n_ic), dtype=torch.float64, device="cuda")
    code = pc.bplane(plan, b, mu, _dev(t), _dev(W.to_planar(w.x0)), out=out, jac=jac)
    assert code == pc.PC_OK
    out = out.cpu().numpy().T
    jac = jac.cpu().numpy().T.reshape(w.n_ic, 2, 6)
    hs = np.array([1e-2, 1e-2, 1e-2, 1e-5, 1e-5, 1e-5])
    for i in range(w.n_ic):
        rel = _venus_rel(ora, w, t[i], w.x0[i])
        ref, rc = ora.bplane(mu, rel)
        assert rc == 0
        np.testing.assert_allclose(out[i], ref, rtol=0, atol=1e-11 * np.abs(ref).max())
        fd = np.zeros((2, 6))
        for q in range(6):
            e = np.zeros(6)
            e[q] = hs[q]
            fd[:, q] = (ora.bplane(mu, rel + e)[0] - ora.bplane(mu, rel - e)[0]) / (2 * hs[q])
        assert _scaled_rel(jac[i], fd, hs) < 1e-7
    # bound (not hyperbolic) relative states give NaN and PC_ENONFINITE
    xv = np.r_[ora.ephem_eval(m, 0.0)[b] + [1e5, 0, 0], ora.ephem_vel(m, 0.0)[b] + [0, 0.1, 0]]
    o1 = torch.zeros((2, 1), dtype=torch.float64, device="cuda")
    code = pc.bplane(plan, b, mu, _dev([0.0]), _dev(xv.reshape(6, 1)), out=o1)
    assert code == pc.PC_ENONFINITE and torch.isnan(o1).all()
    plan.close()


def test_autograd_final_state_and_bplane(pc):
    """Gradients of xf and of (B.T, B.R) at the nominal flyby epoch with respect
    to x0 and an impulsive dv at t0, through torch.autograd: the arc is split at
    the flyby epoch and the b-plane taken there.  Checked against directional
    central differences of the same composed forward pass, and d/d(dv) against
    d/d(v0) (identical by construction of the impulse)."""
    import torch
    from paper_2301_03989_gb300 import autodiff as AD
    w = W.config4(M=128)
    plan = pc.plan_from_workload(w)
    M = w.n_ic
    b, mu = w.meta["body"], w.meta["mu_body"]
    t0 = _dev(np.full(M, w.t0))
    tca = _dev(w.meta["t_ca"])
    tf = _dev(np.full(M, w.tf))
    rng = np.random.default_rng(11)
    wf = _dev(rng.standard_normal((6, M)) * np.array([1e-6] * 3 + [1.0] * 3)[:, None])
    wb = _dev(rng.standard_normal((2, M)) * 1e-3)

    def per_ic(x0p, dv):
        x = torch.cat([x0p[:3], x0p[3:] + dv])
        xca, s1, _ = AD.propagate(x, plan, t0, tca)
        bp = AD.bplane(xca, plan, b, mu, tca)
        xf, s2, _ = AD.propagate(xca, plan, tca, tf)
        return (wf * xf).sum(0) + (wb * bp).sum(0), s1, s2

    x0 = _dev(W.to_planar(w.x0)).requires_grad_(True)
    dv = torch.zeros((3, M), dtype=torch.float64, device="cuda", requires_grad=True)
    L, s1, s2 = per_ic(x0, dv)
    ok = ~pc.PC_IC_STALLED
    assert int((s1 & ok).max()) == 0 and int((s2 & ok).max()) == 0
    L.sum().backward()
    g = x0.grad.detach()
    assert torch.equal(dv.grad, g[3:])
    d = _dev(rng.standard_normal((6, M)) * 10.0 * H6[:, None])
    with torch.no_grad():
        Lp, _, _ = per_ic(x0.detach() + d, torch.zeros_like(dv))
        Lm, _, _ = per_ic(x0.detach() - d, torch.zeros_like(dv))
    fd = ((Lp - Lm) / 2).cpu().numpy()
    ad = (g * d).sum(0).cpu().numpy()
    rel = np.abs(fd - ad) / np.maximum(np.abs(ad), 1e-300)
    print(f"autograd vs directional FD: median {np.median(rel):.2e}, 90% {np.quantile(rel, 0.9):.2e}, "
          f"max {rel.max():.2e}")
    assert np.median(rel) < 1e-7 and np.quantile(rel, 0.9) < 1e-6
    plan.close()
