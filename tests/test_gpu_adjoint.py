"""Reverse mode (pc_propagate_tape / pc_adjoint_tape / pc_propagate_adjoint),
the b-plane (pc_bplane) and the autograd wrappers, on the differentiation
workload (config-1 system, one close Venus flyby per arc, N = 128).

References:
  * the oracle's PC run of the variational equations (6 + 36 states) over the
    GPU's own segment schedule -- the derivative of the same discrete map;
  * central finite differences of the GPU forward map, 1e-3 km / 1e-6 km/s
    steps (and their Richardson extrapolation), run over the base point's own
    segment schedule (so no halving can be decided differently), on the
    trajectories whose sweep counts are the same at +h and -h in every segment
    (one sweep more is a different discrete map); every exclusion is printed;
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


@pytest.mark.parametrize("arc", ["20 days", "full"])
def test_adjoint_matches_oracle_variational(pc, ora, arc):
    """x0_bar = Phi^T xf_bar with Phi from the oracle's variational PC run over
    the GPU's segment schedule, through the flyby: the first 20 days of the arc
    (6 trajectories) and the whole one-revolution arc (4 trajectories)."""
    w = W.config4(M=6 if arc == "20 days" else 4)
    plan = pc.plan_from_workload(w)
    tf = 20 * W.DAY if arc == "20 days" else w.tf
    code, xf, ns, st, tape, cap = _tape_run(pc, plan, w.x0, w.t0, tf)
    assert code == pc.PC_OK
    Phi = _jacobians(pc, plan, ns, cap, tape, w.n_ic)
    rec = pc.tape_record(plan)
    tp = tape.cpu().numpy().reshape(w.n_ic, cap, rec)
    m = ora.Model.from_workload(w)
    o = ora.Opts(N=w.N, tol=w.tol, max_iters=w.max_iters)
    xg = W.from_planar(xf.cpu().numpy())
    from test_gpu_parity import pmap

    def one(i):
        k = int(ns.cpu()[i])
        bounds = np.r_[tp[i, :k, 0], tp[i, k - 1, 1]]
        assert bounds[-1] == tf and k >= 2
        return ora.stm_propagate(m, o, w.x0[i], bounds)
    worst = 0.0
    for i, (x_ora, P_ora, capped, _) in enumerate(pmap(one, range(w.n_ic))):
        assert capped == 0
        er, ev = rel_err(xg[i:i + 1], x_ora[None])
        # same schedule, so the states differ only by tolerance-level
        # differences grown by the flyby: 1e-10, or 1e-13 times the
        # state-transition norm in relative units if that is larger
        s0 = np.r_[[np.linalg.norm(w.x0[i, :3])] * 3, [np.linalg.norm(w.x0[i, 3:])] * 3]
        sf = np.r_[[np.linalg.norm(x_ora[:3])] * 3, [np.linalg.norm(x_ora[3:])] * 3]
        bound = max(TOL, 1e-13 * np.linalg.norm(P_ora * s0[None, :] / sf[:, None], 2))
        assert er.max() < bound and ev.max() < bound, (i, er.max(), ev.max(), bound)
        worst = max(worst, _scaled_rel(Phi[i], P_ora, H6))
    print(f"adjoint vs oracle variational ({arc}): worst scaled rel {worst:.3e}; segments "
          f"{ns.cpu().numpy().tolist()}")
    assert worst < 1e-8
    plan.close()


def _propagate_fixed(pc, plan1, x, bounds, nseg):
    """Forward map over a given segment schedule: trajectory i (column of the
    planar device array x) is propagated over [bounds[i][k], bounds[i][k+1]]
    for k < nseg[i], one segment per call (plan1: one segment per arc, no
    halving, no resolution test).  Returns the end states (planar, device) and
    the sweeps of every segment [n][max nseg]."""
    import torch
    n = x.shape[1]
    seg1 = torch.ones(n, dtype=torch.int32, device="cuda")
    it = torch.zeros(n, dtype=torch.int32, device="cuda")
    sweeps = np.zeros((n, int(nseg.max())), dtype=np.int64)
    for k in range(int(nseg.max())):
        has = nseg > k
        last = bounds[np.arange(n), nseg]
        ta = np.where(has, bounds[:, min(k, bounds.shape[1] - 1)], last)
        tb = np.where(has, bounds[:, min(k + 1, bounds.shape[1] - 1)], last)
        xo = torch.zeros_like(x)
        code, _ = pc.propagate_groups([plan1], [n], x, _dev(ta), _dev(tb), xo, segments=seg1, iters=it)
        torch.cuda.synchronize()
        assert code == pc.PC_OK
        sweeps[:, k] = np.where(has, it.cpu().numpy(), 0)
        x = xo
    return x, sweeps


def _fd_fixed_schedule(pc, plan1, x0, h, bounds, nseg):
    """Central differences of the forward map over the base run's own segment
    schedule, steps h [6].  Returns fd [M][6][6] (d xf / d x0) and, per
    trajectory, the first segment whose sweep count differs between +h_q and
    -h_q for some q (-1: none), where the discrete maps differ."""
    M = x0.shape[0]
    xs = np.concatenate([x0 + sg * h[q] * np.eye(6)[q] for q in range(6) for sg in (1.0, -1.0)])
    xo, sw = _propagate_fixed(pc, plan1, _dev(W.to_planar(xs)), np.tile(bounds, (12, 1)), np.tile(nseg, 12))
    xo = W.from_planar(xo.cpu().numpy()).reshape(6, 2, M, 6)
    sw = sw.reshape(6, 2, M, -1)
    fd = np.zeros((M, 6, 6))
    flip = np.full(M, -1)
    for q in range(6):
        fd[:, :, q] = (xo[q, 0] - xo[q, 1]) / (2 * h[q])
        for i in np.flatnonzero((sw[q, 0] != sw[q, 1]).any(axis=1)):
            k = int(np.flatnonzero(sw[q, 0, i] != sw[q, 1, i])[0])
            flip[i] = k if flip[i] < 0 else min(flip[i], k)
    return fd, flip


def _schedule(pc, plan, tape, ns, cap, M):
    """Segment bounds [M][max nseg + 1] of a taped run (padded with the end)."""
    rec = pc.tape_record(plan)
    tp = tape.cpu().numpy().reshape(M, cap, rec)
    ns = ns.cpu().numpy()
    b = np.zeros((M, int(ns.max()) + 1))
    for i in range(M):
        k = int(ns[i])
        b[i, :k] = tp[i, :k, 0]
        b[i, k:] = tp[i, k - 1, 1]
    return b, ns


def test_adjoint_matches_finite_differences(pc):
    """Adjoint Jacobian of xf over a full config-4 arc (flyby included) against
    central differences of the forward map at the 1e-3 km / 1e-6 km/s steps,
    and against their Richardson extrapolation with the half steps ((4 D(h/2) -
    D(h)) / 3 removes the h^2 term, which dominates on the most strongly bent
    flybys).  The perturbed runs follow the base run's own segment schedule, so
    no halving decision can differ; a trajectory is compared unless some
    segment took a different number of sweeps at +h and -h (a different
    discrete map) -- each such exclusion is printed with its segment."""
    w = W.config4(M=256)
    plan = pc.plan_from_workload(w)
    plan1 = pc.plan_from_workload(w, seg_mode=0, max_depth=0, trunc_tol=0.0)
    M = w.n_ic
    code, xf, ns, st, tape, cap = _tape_run(pc, plan, w.x0, w.t0, w.tf)
    Phi = _jacobians(pc, plan, ns, cap, tape, M)
    bounds, nsv = _schedule(pc, plan, tape, ns, cap, M)
    fd1, flip1 = _fd_fixed_schedule(pc, plan1, w.x0, H6, bounds, nsv)
    fd2, flip2 = _fd_fixed_schedule(pc, plan1, w.x0, 0.5 * H6, bounds, nsv)
    same = (flip1 < 0) & (flip2 < 0)
    for i in np.flatnonzero(~same):
        k = flip1[i] if flip1[i] >= 0 else flip2[i]
        print(f"  excluded trajectory {i}: sweep count differs at +-h in segment {k} of {nsv[i]} "
              f"({'h' if flip1[i] >= 0 else 'h/2'} steps)")
    fdr = (4.0 * fd2 - fd1) / 3.0
    e1 = np.array([_scaled_rel(Phi[i], fd1[i], H6) for i in range(M)])[same]
    er = np.array([_scaled_rel(Phi[i], fdr[i], H6) for i in range(M)])[same]
    print(f"adjoint vs FD on the fixed schedule: {same.sum()} of {M} comparable; central median {np.median(e1):.2e} "
          f"max {e1.max():.2e}; Richardson median {np.median(er):.2e} max {er.max():.2e}")
    assert same.mean() >= 0.9
    assert np.median(e1) < 1e-7
    assert er.max() < 1e-6
    plan.close()
    plan1.close()


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
    # directional central differences of the same composition over each leg's
    # own segment schedule (recorded by a tape run of the base point), with
    # Richardson extrapolation; a trajectory whose +d / -d runs took different
    # sweep counts in some segment is excluded and printed
    plan1 = pc.plan_from_workload(w, seg_mode=0, max_depth=0, trunc_tol=0.0)
    x0n = W.to_planar(w.x0)
    _, xca0, ns1, _, tape1, cap1 = _tape_run(pc, plan, w.x0, w.t0, w.meta["t_ca"])
    b1, n1 = _schedule(pc, plan, tape1, ns1, cap1, M)
    _, _, ns2, _, tape2, cap2 = _tape_run(pc, plan, W.from_planar(xca0.cpu().numpy()), w.meta["t_ca"], w.tf)
    b2, n2 = _schedule(pc, plan, tape2, ns2, cap2, M)

    def fixed(x0p):
        xca, sw1 = _propagate_fixed(pc, plan1, x0p, b1, n1)
        bp = torch.zeros((2, M), dtype=torch.float64, device="cuda")
        pc.bplane(plan, b, mu, tca, xca, out=bp)
        xf, sw2 = _propagate_fixed(pc, plan1, xca, b2, n2)
        return ((wf * xf).sum(0) + (wb * bp).sum(0)).cpu().numpy(), np.concatenate([sw1, sw2], axis=1)

    d = rng.standard_normal((6, M)) * 10.0 * H6[:, None]
    fds, flip = [], np.zeros(M, dtype=bool)
    for sc in (1.0, 0.5):
        Lp, swp = fixed(_dev(x0n + sc * d))
        Lm, swm = fixed(_dev(x0n - sc * d))
        fds.append((Lp - Lm) / (2 * sc))
        flip |= (swp != swm).any(axis=1)
    fd = (4.0 * fds[1] - fds[0]) / 3.0
    ad = (g.cpu().numpy() * d).sum(0)
    rel = np.abs(fd - ad) / np.maximum(np.abs(ad), 1e-300)
    for i in np.flatnonzero(flip):
        print(f"  excluded trajectory {i}: sweep count differs between the +d and -d runs")
    r = rel[~flip]
    print(f"autograd vs directional FD (Richardson, fixed schedule): {r.size} of {M} comparable; median "
          f"{np.median(r):.2e}, max {r.max():.2e}")
    assert r.size >= 0.9 * M
    assert r.max() < 1e-6
    plan.close()
    plan1.close()
