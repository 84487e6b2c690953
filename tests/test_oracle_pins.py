"""Pins of the CPU oracle against facts that do not come from the oracle itself:
closed forms, textbook values (tests/golden/), library routines used as
independent constructions (numpy.polynomial, scipy), conservation laws,
an independent Gauss-Legendre collocation integrator and brute force.

Each test names the oracle function it pins and the plausible mistake that
would make it fail.  No GPU is needed.
"""
import os
from fractions import Fraction

import numpy as np
import numpy.polynomial.chebyshev as npc
import pytest

from paper_2301_03989_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
MU = W.MU_SUN


# ---------------------------------------------------------------- nodes (Eq. chnodes1/2)
@pytest.mark.parametrize("N", [1, 2, 7, 64, 128, 256])
def test_cgl_nodes(ora, N):
    tau = ora.cgl_nodes(N)
    assert tau[0] == -1.0 and tau[-1] == 1.0              # tau_0 = -1 is the segment start
    assert np.all(np.diff(tau) > 0)                         # ordered (a reversed order fails)
    np.testing.assert_allclose(tau + tau[::-1], 0.0, atol=2e-16)   # symmetry
    np.testing.assert_allclose(tau, npc.chebpts2(N + 1), rtol=0, atol=4e-16)  # library: 2nd-kind points


# ---------------------------------------------------------------- operator K
def _poly_exact(tau, p):
    return (tau ** (p + 1) - (-1.0) ** (p + 1)) / (p + 1)


@pytest.mark.parametrize("N", [4, 16, 64, 128])
def test_operator_exact_on_polynomials(ora, N):
    """K integrates every polynomial of degree <= N exactly from tau = -1 (a
    transposed K, a wrong node sign or a dropped beta term fails)."""
    K = ora.pc_operator(N)
    tau = ora.cgl_nodes(N)
    for p in range(N + 1):
        err = np.abs(K @ tau**p - _poly_exact(tau, p)).max()
        assert err < 2e-15 * max(1, N / 16), (p, err)


@pytest.mark.parametrize("N", [8, 32, 128])
def test_operator_truncated_variant(ora, N):
    """The paper's B has N+1 rows, which drops beta_{N+1}: exact up to degree
    N-1; for tau^N the difference is the dropped term beta_{N+1} T_{N+1} with
    beta_{N+1} = a_N/(2(N+1)) and a_N = 2^(1-N) (leading Chebyshev coefficient)."""
    Kt = ora.pc_operator(N, truncated=True)
    K = ora.pc_operator(N)
    tau = ora.cgl_nodes(N)
    for p in range(N):
        assert np.abs(Kt @ tau**p - _poly_exact(tau, p)).max() < 2e-15 * max(1, N / 16)
    beta = 2.0 ** (1 - N) / (2 * (N + 1))
    TN1 = npc.chebval(tau, [0] * (N + 1) + [1])          # T_{N+1}(tau_j)
    expected = beta * (TN1 - (-1.0) ** (N + 1))
    np.testing.assert_allclose(K @ tau**N - Kt @ tau**N, expected, rtol=1e-6, atol=2e-17 * N)
    assert np.abs(expected).max() > 1e3 * 2e-17 * N or N > 16   # the term is visible above round-off


@pytest.mark.parametrize("N", [5, 16, 64])
def test_operator_vs_numpy_construction(ora, N):
    """Independent construction of K through numpy's Chebyshev module:
    interpolate a unit vector at the CGL nodes, integrate from -1, evaluate."""
    tau = ora.cgl_nodes(N)
    Kn = np.zeros((N + 1, N + 1))
    for k in range(N + 1):
        e = np.zeros(N + 1)
        e[k] = 1.0
        c = npc.chebfit(tau, e, N)
        Kn[:, k] = npc.chebval(tau, npc.chebint(c, lbnd=-1))
    np.testing.assert_allclose(ora.pc_operator(N), Kn, atol=5e-14)


@pytest.mark.parametrize("N", [3, 16, 64, 128])
def test_operator_structure(ora, N):
    K = ora.pc_operator(N)
    tau = ora.cgl_nodes(N)
    assert np.abs(K[0]).max() < 1e-18                         # y_0 = x0
    np.testing.assert_allclose(K @ np.ones(N + 1), tau + 1.0, atol=4e-16 * N)
    w = K[-1]                                                  # Clenshaw-Curtis weights
    assert np.all(w > 0)
    assert abs(w.sum() - 2.0) < 1e-14
    # the weights integrate T_k exactly: int_{-1}^{1} T_k = (1 + (-1)^k)/(1 - k^2)
    V = npc.chebvander(tau, N)
    mom = np.array([(1 + (-1) ** k) / (1 - k * k) if k != 1 else 0.0 for k in range(N + 1)])
    np.testing.assert_allclose(w @ V, mom, atol=1e-14)


def test_operator_golden_cc_weights(ora):
    """Textbook Clenshaw-Curtis weights (tests/golden/clenshaw_curtis_weights.txt)."""
    for line in open(os.path.join(GOLDEN, "clenshaw_curtis_weights.txt")):
        if line.startswith("#") or not line.strip():
            continue
        n_s, ws = line.split(":")
        N = int(n_s)
        w = np.array([float(Fraction(x)) for x in ws.split()])
        np.testing.assert_allclose(ora.pc_operator(N)[-1], w, rtol=0, atol=4e-16)


# ---------------------------------------------------------------- ephemeris
@pytest.fixture(scope="module")
def cfg1():
    return W.config1(M=8)


@pytest.fixture(scope="module")
def cfg2():
    return W.config2(M=8)


def test_ephem_vs_chebval(ora, cfg2):
    """The oracle's Clenshaw evaluation equals numpy's chebval of the same
    granule to rounding (a wrong granule index, sigma map or axis stride fails)."""
    m = ora.Model.from_workload(cfg2)
    rng = np.random.default_rng(0)
    L, tb = cfg2.granule, cfg2.t_begin
    for t in rng.uniform(cfg2.t0, cfg2.tf, 25):
        g = int(np.floor((t - tb) / L))
        sig = 2.0 * (t - (tb + g * L)) / L - 1.0
        ref = np.array([[npc.chebval(sig, cfg2.coef[b, g, ax]) for ax in range(3)] for b in range(len(cfg2.mu))])
        np.testing.assert_allclose(ora.ephem_eval(m, t), ref, rtol=2e-15, atol=1e-6)


def test_ephem_interpolates_fit_samples(ora, cfg2):
    """At the generator's fitting points the table reproduces the sampled orbit."""
    m = ora.Model.from_workload(cfg2)
    names, bodies = W._full_system(np.random.Generator(np.random.PCG64(2)))
    deg = cfg2.coef.shape[3] - 1
    sig = np.cos(np.pi * np.arange(deg + 1) / deg)
    g = 5
    ts = cfg2.t_begin + g * cfg2.granule + (sig + 1) * 0.5 * cfg2.granule
    for t in ts[1:-1]:                     # interior points: no granule-boundary tie
        got = ora.ephem_eval(m, t)
        ref = np.array([b.position(np.array([t]))[0] for b in bodies])
        np.testing.assert_allclose(got, ref, rtol=1e-13, atol=2e-6)


def test_ephem_boundary_uses_later_granule(ora, cfg2):
    m = ora.Model.from_workload(cfg2)
    g = 7
    t = cfg2.t_begin + g * cfg2.granule
    got = ora.ephem_eval(m, t)
    ref = np.array([[npc.chebval(-1.0, cfg2.coef[b, g, ax]) for ax in range(3)] for b in range(len(cfg2.mu))])
    np.testing.assert_allclose(got, ref, rtol=1e-15)


# ---------------------------------------------------------------- force
def _potential(mu_c, mus, rb, r, indirect=True):
    """Heliocentric disturbing potential, U = -mu_S/|r| - sum mu_b (1/|r-r_b| - r.r_b/|r_b|^3)."""
    r = np.asarray(r, dtype=np.longdouble)
    U = -mu_c / np.sqrt((r * r).sum())
    for mu_b, p in zip(mus, rb):
        p = np.asarray(p, dtype=np.longdouble)
        d = r - p
        U -= mu_b / np.sqrt((d * d).sum())
        if indirect:
            U += mu_b * (r * p).sum() / np.sqrt((p * p).sum()) ** 3
    return U


@pytest.mark.parametrize("indirect", [True, False])
def test_accel_is_minus_gradient_of_potential(ora, cfg2, indirect):
    """a = -grad U by 4th-order central differences in long double (a wrong sign,
    a dropped or doubled indirect term, or a body-index error fails)."""
    m = ora.Model.from_workload(cfg2)
    m.indirect = indirect
    rng = np.random.default_rng(1)
    for _ in range(6):
        t = rng.uniform(cfg2.t0, cfg2.tf)
        rb = ora.ephem_eval(m, t)
        # a point 3e6 km from Venus, so that the planet term matters
        r = rb[1] + rng.standard_normal(3) * 3e6
        a = ora.accel(m, rb, r)
        h = 50.0
        g = np.zeros(3)
        for ax in range(3):
            e = np.zeros(3)
            e[ax] = h
            U = [_potential(m.mu_central, m.mu, rb, r + k * e, indirect) for k in (-2, -1, 1, 2)]
            g[ax] = float((U[0] - 8 * U[1] + 8 * U[2] - U[3]) / (12 * h))
        np.testing.assert_allclose(a, -g, rtol=1e-7, atol=1e-7 * np.abs(a).max())


def test_accel_collinear_closed_form(ora):
    """mu_S = 0, one body at r_b, particle at 2 r_b: direct term -mu r_b/|r_b|^3
    and indirect term -mu r_b/|r_b|^3."""
    rb = np.array([[3.0e7, -4.0e7, 1.2e7]])
    mu_b = 1.0e8
    m = ora.Model(mu_central=0.0, mu=np.array([mu_b]))
    a = ora.accel(m, rb, 2 * rb[0])
    n3 = np.linalg.norm(rb[0]) ** 3
    np.testing.assert_allclose(a, -2 * mu_b * rb[0] / n3, rtol=1e-15)
    m.indirect = False
    np.testing.assert_allclose(ora.accel(m, rb, 2 * rb[0]), -mu_b * rb[0] / n3, rtol=1e-15)


# ---------------------------------------------------------------- Kepler warm start
def _invariants(x, mu):
    r, v = x[:3], x[3:]
    h = np.cross(r, v)
    E = v @ v / 2 - mu / np.linalg.norm(r)
    evec = np.cross(v, h) / mu - r / np.linalg.norm(r)
    return E, h, evec


@pytest.mark.parametrize("e", [0.0, 0.3, 0.9])
def test_kepler_invariants_and_period(ora, e):
    a = 0.75 * W.AU
    x0 = W.elements_to_state(a, e, np.deg2rad(2.0), 0.3, 1.1, 0.7, MU)
    T = 2 * np.pi * np.sqrt(a**3 / MU)
    E0, h0, e0 = _invariants(x0, MU)
    for dt in [0.0, 0.01 * T, 0.37 * T, -0.61 * T, 2.3 * T]:
        x, rc = ora.kepler(MU, x0, dt)
        assert rc == 0
        E, h, ev = _invariants(x, MU)
        assert abs(E - E0) < 1e-13 * abs(E0)
        np.testing.assert_allclose(h, h0, rtol=0, atol=1e-13 * np.linalg.norm(h0))
        np.testing.assert_allclose(ev, e0, rtol=0, atol=1e-12)
    x, _ = ora.kepler(MU, x0, T)
    np.testing.assert_allclose(x[:3], x0[:3], rtol=0, atol=1e-11 * np.linalg.norm(x0[:3]))


def test_kepler_vs_scipy_dop853(ora):
    from scipy.integrate import solve_ivp
    x0 = W.elements_to_state(0.75 * W.AU, 0.3, np.deg2rad(2), 0, 0, 0, MU)
    T = 2 * np.pi * np.sqrt((0.75 * W.AU) ** 3 / MU)

    def f(t, y):
        r = y[:3]
        return np.concatenate([y[3:], -MU * r / np.linalg.norm(r) ** 3])

    sol = solve_ivp(f, (0, 0.3 * T), x0, method="DOP853", rtol=1e-13, atol=1e-9)
    x, rc = ora.kepler(MU, x0, 0.3 * T)
    np.testing.assert_allclose(x, sol.y[:, -1], rtol=2e-10)


def test_kepler_rejects_hyperbolic(ora):
    x0 = np.array([1.0e8, 0, 0, 0, 60.0, 0])       # above escape speed at 1e8 km
    assert ora.kepler(MU, x0, 1e5)[1] == 1


# ---------------------------------------------------------------- PC segment on analytic problems
def test_pc_constant_acceleration_exact(ora):
    """f = (v, a_c): the solution is quadratic, so the PC iteration reaches it
    exactly after three sweeps (cold start, absolute mode)."""
    a_c = (1e-3, -2e-3, 5e-4)
    m = ora.Model(mu_central=1.0, mu=np.zeros(0))
    o = ora.Opts(N=16, tol=1e-15, relative=False, warm_start=False, dyn=ora.DYN_CONST_ACCEL, dyn_param=a_c,
                 trunc_tol=0)
    x0 = np.array([10.0, -3.0, 2.0, 0.1, 0.2, -0.3])
    Y, it, err, out = ora.pc_segment(m, o, 100.0, 300.0, x0)
    assert out == ora.SEG_OK and it <= 4
    t = 100.0 + 100.0 * (ora.cgl_nodes(16) + 1.0)
    dt = (t - 100.0)[:, None]
    ref = np.hstack([x0[:3] + x0[3:] * dt + 0.5 * np.array(a_c) * dt**2, x0[3:] + np.array(a_c) * dt])
    np.testing.assert_allclose(Y, ref, rtol=1e-14, atol=1e-12)


@pytest.mark.parametrize("N,tol_err", [(8, 1e-3), (16, 1e-8), (32, 1e-13)])
def test_pc_harmonic_oscillator_spectral(ora, N, tol_err):
    """x'' = -w^2 x over w*dt = 4 rad: closed form cos/sin; error falls
    spectrally with N."""
    w2 = 0.01 ** 2
    m = ora.Model(mu_central=1.0, mu=np.zeros(0))
    o = ora.Opts(N=N, tol=1e-15, relative=False, warm_start=False, dyn=ora.DYN_HARMONIC, dyn_param=(w2, 0, 0),
                 max_iters=200, trunc_tol=0, stall_factor=1e3)
    x0 = np.array([1.0, 0.5, -0.2, 0.0, 0.01, 0.003])
    Y, it, err, out = ora.pc_segment(m, o, 0.0, 400.0, x0)
    assert out in (ora.SEG_OK, ora.SEG_STALLED)
    t = 200.0 * (ora.cgl_nodes(N) + 1.0)
    w = 0.01
    ref_r = x0[:3] * np.cos(w * t)[:, None] + x0[3:] / w * np.sin(w * t)[:, None]
    ref_v = -x0[:3] * w * np.sin(w * t)[:, None] + x0[3:] * np.cos(w * t)[:, None]
    e = max(np.abs(Y[:, :3] - ref_r).max(), np.abs(Y[:, 3:] - ref_v).max() / w)
    assert e < tol_err, e


def test_pc_two_body_vs_kepler_and_conservation(ora):
    """Two-body problem (no planets), cold start over one revolution in 8
    segments: the PC end state equals Kepler's; energy and angular momentum
    are conserved at every node of every segment."""
    a, e = 0.75 * W.AU, 0.3
    x0 = W.elements_to_state(a, e, np.deg2rad(2), 0, 0, 0, MU)
    T = 2 * np.pi * np.sqrt(a**3 / MU)
    m = ora.Model(mu_central=MU, mu=np.zeros(0))
    o = ora.Opts(N=64, tol=1e-13, warm_start=False, segments=8, max_iters=120)
    r = ora.propagate(m, o, x0[None], 0.0, T, max_ckpt=16)
    assert r["status"][0] == 0
    xk, _ = ora.kepler(MU, x0, T)
    np.testing.assert_allclose(r["xf"][0][:3], xk[:3], rtol=0, atol=1e-12 * np.linalg.norm(xk[:3]))
    np.testing.assert_allclose(r["xf"][0][3:], xk[3:], rtol=0, atol=1e-12 * np.linalg.norm(xk[3:]))
    E0, h0, _ = _invariants(x0, MU)
    ck = r["ckpt"][0]
    for s in range(int(r["nseg"][0])):
        ta = ck[s, 0]
        tb = ck[s + 1, 0] if s + 1 < r["nseg"][0] else T
        Y, _, _, out = ora.pc_segment(m, o, ta, tb, ck[s, 1:])
        for y in Y:
            E, h, _ = _invariants(y, MU)
            assert abs(E / E0 - 1) < 5e-14
            assert np.linalg.norm(h - h0) < 5e-14 * np.linalg.norm(h0)


# ---------------------------------------------------------------- Gauss-Legendre independent integrator
def test_gl_coeffs_golden_two_stage(ora):
    c, A, b = ora.gl_coeffs(2)
    s3 = np.sqrt(3.0)
    np.testing.assert_allclose(c, [0.5 - s3 / 6, 0.5 + s3 / 6], rtol=1e-15)
    np.testing.assert_allclose(A, [[0.25, 0.25 - s3 / 6], [0.25 + s3 / 6, 0.25]], rtol=1e-14, atol=1e-16)
    np.testing.assert_allclose(b, [0.5, 0.5], rtol=1e-15)
    assert os.path.exists(os.path.join(GOLDEN, "gauss_legendre_2stage.txt"))


@pytest.mark.parametrize("s", [3, 6])
def test_gl_coeffs_order_conditions(ora, s):
    c, A, b = ora.gl_coeffs(s)
    xg, wg = np.polynomial.legendre.leggauss(s)                  # library nodes
    np.testing.assert_allclose(np.sort(c), (xg + 1) / 2, atol=1e-15)
    np.testing.assert_allclose(np.sort(b), np.sort(wg / 2), atol=1e-15)
    for k in range(2 * s):                                       # B(2s)
        assert abs(b @ c**k - 1.0 / (k + 1)) < 1e-15
    for k in range(s):                                           # C(s)
        np.testing.assert_allclose(A @ c**k, c ** (k + 1) / (k + 1), atol=1e-15)


def _rel(a, b):
    return max(np.linalg.norm(a[:3] - b[:3]) / np.linalg.norm(b[:3]), np.linalg.norm(a[3:] - b[3:]) / np.linalg.norm(b[3:]))


def test_pc_vs_gauss_legendre_config1(ora, cfg1):
    """Config-1 dynamics over one revolution: PC (N = 64, 8 segments) and a
    6-stage Gauss-Legendre integrator (step-converged) agree to 1e-12."""
    m = ora.Model.from_workload(cfg1)
    o = ora.Opts(N=cfg1.N, segments=cfg1.segments, tol=cfg1.tol)
    r = ora.propagate(m, o, cfg1.x0[:2], cfg1.t0, cfg1.tf)
    for i in range(2):
        g1, _ = ora.gl_propagate(m, o, cfg1.x0[i], cfg1.t0, cfg1.tf, 1200)
        g2, _ = ora.gl_propagate(m, o, cfg1.x0[i], cfg1.t0, cfg1.tf, 2400)
        assert _rel(g1, g2) < 1e-13
        assert _rel(r["xf"][i], g2) < 1e-12, _rel(r["xf"][i], g2)


def test_pc_vs_gauss_legendre_flyby(ora, cfg2):
    """Through a close Venus flyby the resolution test must halve the segment;
    PC then agrees with a step-converged Gauss-Legendre run to 1e-11 after 5
    days (without the test the converged PC answer is off by ~1e-2)."""
    m = ora.Model.from_workload(cfg2)
    o = ora.Opts(N=cfg2.N, segments=cfg2.segments, seg_mode=cfg2.seg_mode, tol=cfg2.tol,
                 max_depth=cfg2.max_depth)
    tf = 5 * W.DAY
    r = ora.propagate(m, o, cfg2.x0[:1], 0.0, tf)
    g1, _ = ora.gl_propagate(m, o, cfg2.x0[0], 0.0, tf, 6000)
    g2, _ = ora.gl_propagate(m, o, cfg2.x0[0], 0.0, tf, 12000)
    assert _rel(g1, g2) < 1e-12
    assert _rel(r["xf"][0], g2) < 1e-11, _rel(r["xf"][0], g2)
    o.trunc_tol = 0.0
    r_bad = ora.propagate(m, o, cfg2.x0[:1], 0.0, tf)
    assert _rel(r_bad["xf"][0], g2) > 1e-6


def test_tail_estimate_tracks_chebyshev_coefficients(ora):
    """For g = exp(tau) the interpolant's top coefficients are close to the
    series coefficients 2 I_k(1) (scipy Bessel); the estimate is
    2|w2|(|a_{N-1}| + |a_N|) and must fall with N."""
    from scipy.special import iv
    vals = []
    for N in (6, 8, 10):
        tau = ora.cgl_nodes(N)
        G = np.repeat(np.exp(tau)[:, None], 6, axis=1)
        o = ora.Opts(N=N, relative=False)
        est = ora.tail_estimate(o, G, np.ones((N + 1, 6)), 1.0)
        ref = 2.0 * (2 * iv(N - 1, 1.0) + iv(N, 1.0))   # a_N carries the 1/2 of the interpolant
        assert 0.5 * ref < est < 2.0 * ref, (N, est, ref)
        vals.append(est)
    assert vals[0] > vals[1] > vals[2]


# ---------------------------------------------------------------- invariants of the propagation
def test_batch_invariance_and_threads(ora, cfg1):
    """Augmentation leaves each trajectory's arithmetic unchanged: batch,
    single-IC and multi-threaded runs are bitwise identical."""
    m = ora.Model.from_workload(cfg1)
    o = ora.Opts(N=cfg1.N, segments=cfg1.segments, tol=cfg1.tol)
    rb = ora.propagate(m, o, cfg1.x0[:4], cfg1.t0, cfg1.tf, threads=1)
    rt = ora.propagate(m, o, cfg1.x0[:4], cfg1.t0, cfg1.tf, threads=3)
    assert np.array_equal(rb["xf"], rt["xf"])
    for i in range(4):
        r1 = ora.propagate(m, o, cfg1.x0[i:i + 1], cfg1.t0, cfg1.tf)
        assert np.array_equal(r1["xf"][0], rb["xf"][i])


def test_forward_backward(ora, cfg1):
    m = ora.Model.from_workload(cfg1)
    o = ora.Opts(N=cfg1.N, segments=cfg1.segments, tol=cfg1.tol)
    f = ora.propagate(m, o, cfg1.x0[:2], cfg1.t0, cfg1.tf)
    b = ora.propagate(m, o, f["xf"], cfg1.tf, cfg1.t0)
    for i in range(2):
        assert _rel(b["xf"][i], cfg1.x0[i]) < 1e-12


def test_cold_and_warm_start_same_fixed_point(ora, cfg1):
    m = ora.Model.from_workload(cfg1)
    ow = ora.Opts(N=cfg1.N, segments=cfg1.segments, tol=cfg1.tol)
    oc = ora.Opts(N=cfg1.N, segments=cfg1.segments, tol=cfg1.tol, warm_start=False, max_iters=150)
    rw = ora.propagate(m, ow, cfg1.x0[:2], cfg1.t0, cfg1.tf)
    rc = ora.propagate(m, oc, cfg1.x0[:2], cfg1.t0, cfg1.tf)
    assert (rc["iters"] > rw["iters"]).all()
    for i in range(2):
        assert _rel(rw["xf"][i], rc["xf"][i]) < 1e-12


def test_status_codes(ora, cfg1):
    m = ora.Model.from_workload(cfg1)
    o = ora.Opts(N=cfg1.N, segments=cfg1.segments, tol=0.0, max_iters=8, max_depth=1)
    r = ora.propagate(m, o, cfg1.x0[:1], cfg1.t0, cfg1.tf)
    assert r["status"][0] == ora.IC_NOT_CONVERGED and r["nseg"][0] == 0
    x = cfg1.x0[:2].copy()
    x[1, 2] = np.nan
    o = ora.Opts(N=cfg1.N, segments=cfg1.segments, tol=cfg1.tol)
    r = ora.propagate(m, o, x, cfg1.t0, cfg1.tf)
    assert r["status"][0] == ora.IC_OK and r["status"][1] == ora.IC_NONFINITE
    r = ora.propagate(m, o, cfg1.x0[:1], 5.0, 5.0)                    # empty arc
    assert r["nseg"][0] == 0 and np.array_equal(r["xf"][0], cfg1.x0[0])
