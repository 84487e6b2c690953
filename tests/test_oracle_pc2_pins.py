"""Pins of the oracle's second-order sweep (ora_pc2_segment: velocities from the
integrated accelerations, then positions from the integrated new velocities):
exactness on constant acceleration, the harmonic oscillator's closed form, the
same fixed point as the first-order sweep, and fewer sweeps to reach it."""
import numpy as np
import pytest

from paper_2301_03989_gb300 import workloads as W


def test_pc2_constant_acceleration_exact(ora):
    m = ora.Model(mu_central=1.0, mu=np.zeros(0))
    a_c = (1e-3, -2e-3, 5e-4)
    o = ora.Opts(N=16, tol=1e-15, relative=False, warm_start=False, dyn=ora.DYN_CONST_ACCEL, dyn_param=a_c,
                 trunc_tol=0)
    x0 = np.array([10.0, -3.0, 2.0, 0.1, 0.2, -0.3])
    Y, it, err, out = ora.pc2_segment(m, o, 100.0, 300.0, x0)
    assert out == ora.SEG_OK and it <= 3
    dt = (100.0 * (ora.cgl_nodes(16) + 1.0))[:, None]
    ref = np.hstack([x0[:3] + x0[3:] * dt + 0.5 * np.array(a_c) * dt**2, x0[3:] + np.array(a_c) * dt])
    np.testing.assert_allclose(Y, ref, rtol=1e-14, atol=1e-12)


def test_pc2_harmonic_oscillator(ora):
    m = ora.Model(mu_central=1.0, mu=np.zeros(0))
    w = 0.01
    o = ora.Opts(N=32, tol=1e-15, relative=False, warm_start=False, dyn=ora.DYN_HARMONIC, dyn_param=(w * w, 0, 0),
                 max_iters=200, trunc_tol=0)
    x0 = np.array([1.0, 0.5, -0.2, 0.0, 0.01, 0.003])
    Y, it, err, out = ora.pc2_segment(m, o, 0.0, 400.0, x0)
    assert out in (ora.SEG_OK, ora.SEG_STALLED)
    t = 200.0 * (ora.cgl_nodes(32) + 1.0)
    ref_r = x0[:3] * np.cos(w * t)[:, None] + x0[3:] / w * np.sin(w * t)[:, None]
    ref_v = -x0[:3] * w * np.sin(w * t)[:, None] + x0[3:] * np.cos(w * t)[:, None]
    assert max(np.abs(Y[:, :3] - ref_r).max(), np.abs(Y[:, 3:] - ref_v).max() / w) < 1e-13


def test_pc2_same_fixed_point_fewer_sweeps(ora):
    """Both sweeps solve R = r0 + omega2 K V, V = v0 + omega2 K A(R): on a config-1
    segment they agree to the tolerance, the second-order one in fewer sweeps
    (a cold start makes the difference in contraction rate visible)."""
    w = W.config1(M=1)
    m = ora.Model.from_workload(w)
    x0 = w.x0[0]
    ta, tb = w.t0, w.t0 + w.tf / 8
    for warm in (True, False):
        o = ora.Opts(N=64, tol=1e-13, warm_start=warm, max_iters=200, trunc_tol=0)
        Y1, it1, _, out1 = ora.pc_segment(m, o, ta, tb, x0)
        Y2, it2, _, out2 = ora.pc2_segment(m, o, ta, tb, x0)
        assert out1 in (ora.SEG_OK, ora.SEG_STALLED) and out2 in (ora.SEG_OK, ora.SEG_STALLED)
        er = np.linalg.norm(Y2[:, :3] - Y1[:, :3], axis=1) / np.linalg.norm(Y1[:, :3], axis=1)
        ev = np.linalg.norm(Y2[:, 3:] - Y1[:, 3:], axis=1) / np.linalg.norm(Y1[:, 3:], axis=1)
        assert er.max() < 1e-12 and ev.max() < 1e-12
        assert it2 < it1, (warm, it1, it2)


def test_order2_core_is_bitwise_the_pinned_second_order_segment(ora):
    """The segment core with order 2 (used by the whole-arc propagator) does
    the arithmetic of ora_pc2_segment: bitwise the same iterate, sweep count
    and change on a config-1 segment (resolution test off, as
    ora_pc2_segment has none) and on the harmonic oscillator."""
    w = W.config1(M=2)
    m = ora.Model.from_workload(w)
    for x0, (ta, tb) in ((w.x0[0], (w.t0, w.t0 + w.tf / 8)), (w.x0[1], (w.tf / 3, w.tf / 3 + w.tf / 6))):
        o = ora.Opts(N=64, tol=1e-13, max_iters=100, trunc_tol=0, order=2)
        Y2, it2, e2, out2 = ora.pc2_segment(m, o, ta, tb, x0)
        Yc, itc, ec, outc = ora.pc_segment(m, o, ta, tb, x0)
        np.testing.assert_array_equal(Yc, Y2)
        assert (itc, ec, outc) == (it2, e2, out2)
    mh = ora.Model(mu_central=1.0, mu=np.zeros(0))
    o = ora.Opts(N=32, tol=1e-15, relative=False, warm_start=False, dyn=ora.DYN_HARMONIC, dyn_param=(1e-4, 0, 0),
                 max_iters=200, trunc_tol=0, order=2)
    x0 = np.array([1.0, 0.5, -0.2, 0.0, 0.01, 0.003])
    np.testing.assert_array_equal(ora.pc_segment(mh, o, 0.0, 400.0, x0)[0], ora.pc2_segment(mh, o, 0.0, 400.0, x0)[0])


def test_order2_propagation_same_answer_fewer_sweeps(ora):
    """Whole config-1 arcs (8 trajectories, one revolution, resolution test on):
    the second-order sweep lands on the first-order answer to 1e-12 with the
    same statuses, in at least a third fewer sweeps; both agree with a
    step-converged Gauss-Legendre run to 1e-12."""
    w = W.config1(M=8)
    m = ora.Model.from_workload(w)
    o1 = ora.Opts(N=w.N, segments=w.segments, tol=w.tol)
    o2 = ora.Opts(N=w.N, segments=w.segments, tol=w.tol, order=2)
    r1 = ora.propagate(m, o1, w.x0, w.t0, w.tf, threads=4)
    r2 = ora.propagate(m, o2, w.x0, w.t0, w.tf, threads=4)
    np.testing.assert_array_equal(r1["status"], r2["status"])
    er = np.linalg.norm(r2["xf"][:, :3] - r1["xf"][:, :3], axis=1) / np.linalg.norm(r1["xf"][:, :3], axis=1)
    ev = np.linalg.norm(r2["xf"][:, 3:] - r1["xf"][:, 3:], axis=1) / np.linalg.norm(r1["xf"][:, 3:], axis=1)
    assert er.max() < 1e-12 and ev.max() < 1e-12, (er.max(), ev.max())
    assert r2["iters"].sum() < (2 / 3) * r1["iters"].sum(), (r1["iters"].sum(), r2["iters"].sum())
    g, _ = ora.gl_propagate(m, o1, w.x0[0], w.t0, w.tf, 2400)
    rel = np.linalg.norm(r2["xf"][0] - g) / np.linalg.norm(g)
    assert rel < 1e-12, rel


def test_order2_planted_mistake_fails(ora):
    """A second-order sweep that integrated the old velocities (the first-order
    position update) would not be bitwise ora_pc2_segment: the pinned segment
    differs from the first-order core on the same inputs."""
    w = W.config1(M=1)
    m = ora.Model.from_workload(w)
    ta, tb = w.t0, w.t0 + w.tf / 8
    o1 = ora.Opts(N=64, tol=1e-13, max_iters=100, trunc_tol=0, order=1)
    o2 = ora.Opts(N=64, tol=1e-13, max_iters=100, trunc_tol=0, order=2)
    Y1, it1, _, _ = ora.pc_segment(m, o1, ta, tb, w.x0[0])
    Y2, it2, _, _ = ora.pc2_segment(m, o2, ta, tb, w.x0[0])
    assert it2 < it1 and not np.array_equal(Y1, Y2)
