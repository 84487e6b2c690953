"""Pins of the oracle's differentiation routines (table velocities, gravity
gradient, PC on the variational equations, Gauss-Legendre variational
integration, b-plane) against facts that do not come from those routines:
library Chebyshev differentiation, finite differences of independent code
(analytic Kepler, the 6-state oracle), symplecticity of Hamiltonian flows,
the straight-line limit and a hyperbola built from its asymptote.

No GPU is needed."""
import numpy as np
import numpy.polynomial.chebyshev as npc
import pytest

from paper_2301_03989_gb300 import workloads as W


def _model(ora, w):
    return ora.Model.from_workload(w)


def _opts(ora, w, **kw):
    o = ora.Opts(N=w.N, segments=w.segments, seg_mode=w.seg_mode, tol=w.tol, max_iters=w.max_iters,
                 max_depth=w.max_depth)
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _scaled_rel(J, Jref, h):
    """Largest entry difference of two Jacobians with column j scaled by step h_j,
    relative to the largest scaled entry of the reference."""
    d = np.abs((J - Jref) * h[None, :])
    return d.max() / np.abs(Jref * h[None, :]).max()


H6 = np.array([1.0, 1.0, 1.0, 1e-6, 1e-6, 1e-6])   # 1 km, 1 mm/s


# ------------------------------------------------------------- table velocities
def test_ephem_vel_matches_library_derivative(ora):
    """ora_ephem_vel against numpy's Chebyshev derivative of the same table
    (a wrong U index, a missing factor k or 2/L fails)."""
    w = W.config2(M=1)
    m = _model(ora, w)
    rng = np.random.default_rng(0)
    for t in rng.uniform(w.t0, w.tf, 25):
        g = int(np.floor((t - w.t_begin) / w.granule))
        sig = 2.0 * (t - (w.t_begin + g * w.granule)) / w.granule - 1.0
        ref = np.array([[npc.chebval(sig, npc.chebder(w.coef[b, g, ax])) * 2.0 / w.granule for ax in range(3)]
                        for b in range(len(w.mu))])
        got = ora.ephem_vel(m, t)
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_ephem_vel_circular_speed(ora):
    """On the circular config-1 planets the table's velocity has the circular
    speed sqrt(mu/a) and is perpendicular to the position (fit error level)."""
    w = W.config1(M=1)
    m = _model(ora, w)
    for t in np.linspace(w.t0, w.tf, 11):
        r = ora.ephem_eval(m, t)
        v = ora.ephem_vel(m, t)
        for b, nm in enumerate(w.body_names):
            vc = np.sqrt(W.MU_SUN / (W.A_AU[nm] * W.AU))
            assert abs(np.linalg.norm(v[b]) / vc - 1.0) < 1e-9
            assert abs(r[b].dot(v[b])) / (np.linalg.norm(r[b]) * np.linalg.norm(v[b])) < 1e-9


# ------------------------------------------------------------- gravity gradient
def test_tidal_matches_finite_differences(ora):
    """ora_tidal against central differences of ora_accel, near the Sun, near
    each body and far away (a wrong sign or factor 3 fails)."""
    w = W.config1(M=1)
    m = _model(ora, w)
    t = 0.3 * w.tf
    rb = ora.ephem_eval(m, t)
    rng = np.random.default_rng(1)
    pts = [np.array([0.75 * W.AU, 0.1 * W.AU, 0.01 * W.AU])]
    for b in range(len(w.mu)):
        for dist in (2e4, 3e5):
            u = rng.standard_normal(3)
            pts.append(rb[b] + dist * u / np.linalg.norm(u))
    for r in pts:
        A = ora.tidal(m, rb, r)
        hstep = 1e-5 * min([np.linalg.norm(r)] + [np.linalg.norm(r - p) for p in rb])
        fd = np.zeros((3, 3))
        for q in range(3):
            e = np.zeros(3)
            e[q] = hstep
            fd[:, q] = (ora.accel(m, rb, r + e) - ora.accel(m, rb, r - e)) / (2 * hstep)
        np.testing.assert_allclose(A, fd, rtol=0, atol=1e-7 * np.abs(fd).max())


def test_tidal_symmetric_traceless(ora):
    """Outside the masses the potential is harmonic: da/dr is symmetric with
    zero trace (a coefficient other than 3 in the r r^T term fails)."""
    w = W.config2(M=1)
    m = _model(ora, w)
    rb = ora.ephem_eval(m, 1e7)
    for r in (np.array([1.1e8, -2e7, 3e6]), rb[1] + np.array([2e4, 1e4, -3e3])):
        A = ora.tidal(m, rb, r)
        s = np.abs(A).max()
        assert np.abs(A - A.T).max() <= 1e-15 * s
        assert abs(np.trace(A)) <= 1e-12 * s


# ------------------------------------------------------------- b-plane
def _tr(S):
    T = np.cross(S, [0.0, 0.0, 1.0])
    T /= np.linalg.norm(T)
    return T, np.cross(S, T)


def test_bplane_straight_line_limit(ora):
    """mu -> 0: B is the perpendicular offset of the straight line r + v t
    from the planet, T and R built on the direction of v."""
    rng = np.random.default_rng(2)
    for _ in range(20):
        r = rng.standard_normal(3) * 1e5
        v = rng.standard_normal(3) * 5.0
        out, rc = ora.bplane(1e-12, np.r_[r, v])
        assert rc == 0
        s = v / np.linalg.norm(v)
        bvec = r - r.dot(s) * s
        T, R = _tr(s)
        ref = np.array([bvec.dot(T), bvec.dot(R)])
        np.testing.assert_allclose(out, ref, rtol=0, atol=1e-9 * np.linalg.norm(bvec))


def test_bplane_hyperbola_from_asymptote(ora):
    """A periapsis state built from a chosen incoming asymptote S, aim point B
    (perpendicular to S), v_inf and mu: e = sqrt(1 + b^2 v_inf^4/mu^2),
    r_p = (mu/v_inf^2)(e - 1), periapsis along S/e + sqrt(e^2-1)/e B_hat, velocity
    along -B_hat/e + sqrt(e^2-1)/e S.  The b-plane of that state must give back
    B.T, B.R (taking the outgoing asymptote, or a sign slip in S, fails)."""
    mu = W.GM["venus"]
    rng = np.random.default_rng(3)
    for _ in range(20):
        S = rng.standard_normal(3)
        S /= np.linalg.norm(S)
        bh = rng.standard_normal(3)
        bh -= bh.dot(S) * S
        bh /= np.linalg.norm(bh)
        b = rng.uniform(1e4, 1e5)
        vinf = rng.uniform(3.0, 6.0)
        e = np.sqrt(1.0 + b * b * vinf**4 / mu**2)
        rp = mu / vinf**2 * (e - 1.0)
        s1 = np.sqrt(e * e - 1.0) / e
        P = S / e + s1 * bh
        Q = -bh / e + s1 * S
        vp = np.sqrt(vinf**2 + 2.0 * mu / rp)
        out, rc = ora.bplane(mu, np.r_[rp * P, vp * Q])
        assert rc == 0
        T, R = _tr(S)
        ref = b * np.array([bh.dot(T), bh.dot(R)])
        np.testing.assert_allclose(out, ref, rtol=0, atol=1e-10 * b)
    out, rc = ora.bplane(mu, np.r_[1e5, 0, 0, 0, 0.1, 0])     # bound orbit
    assert rc == 1


# ------------------------------------------------------------- variational PC
def _schedule(ora, w, x0):
    """Accepted segment bounds of the 6-state oracle run of one IC."""
    r = ora.propagate(_model(ora, w), _opts(ora, w), x0[None, :], w.t0, w.tf, max_ckpt=4096)
    k = int(r["nseg"][0])
    return np.r_[r["ckpt"][0, :k, 0], w.tf], r["xf"][0]


def test_stm_two_body_matches_kepler_fd(ora):
    """Sun only: the PC STM over one revolution (8 segments) against central
    differences of analytic Kepler propagation (ora_kepler), which shares no
    code with the variational sweep."""
    w = W.config1(M=1)
    m = ora.Model(mu_central=W.MU_SUN, mu=np.zeros(0))
    o = _opts(ora, w)
    x0 = w.x0[0]
    bounds = np.linspace(w.t0, w.tf, 9)
    xf, Phi, capped, _ = ora.stm_propagate(m, o, x0, bounds)
    assert capped == 0
    fd = np.zeros((6, 6))
    for q in range(6):
        e = np.zeros(6)
        e[q] = H6[q]
        xp, rc1 = ora.kepler(W.MU_SUN, x0 + e, w.tf - w.t0)
        xm, rc2 = ora.kepler(W.MU_SUN, x0 - e, w.tf - w.t0)
        assert rc1 == rc2 == 0
        fd[:, q] = (xp - xm) / (2 * H6[q])
    assert _scaled_rel(Phi, fd, H6) < 1e-7


def _omega():
    O = np.zeros((6, 6))
    O[:3, 3:] = np.eye(3)
    O[3:, :3] = -np.eye(3)
    return O


def test_stm_symplectic(ora):
    """The N-body flow is Hamiltonian, so Phi^T Omega Phi = Omega (a non-symmetric
    gravity gradient or a wrong block of F fails)."""
    w = W.config1(M=2)
    m, o = _model(ora, w), _opts(ora, w)
    for x0 in w.x0:
        bounds, _ = _schedule(ora, w, x0)
        _, Phi, capped, _ = ora.stm_propagate(m, o, x0, bounds)
        assert capped == 0
        O = _omega()
        assert np.abs(Phi.T @ O @ Phi - O).max() < 1e-10 * np.abs(Phi).max() ** 2


def test_stm_state_part_matches_propagate(ora):
    """The y part of the variational sweep is the state sweep: same final state
    as ora_propagate on the same schedule (to the convergence tolerance)."""
    w = W.config1(M=2)
    m, o = _model(ora, w), _opts(ora, w)
    for x0 in w.x0:
        bounds, xf6 = _schedule(ora, w, x0)
        xf, _, _, _ = ora.stm_propagate(m, o, x0, bounds)
        assert np.linalg.norm(xf[:3] - xf6[:3]) < 1e-11 * np.linalg.norm(xf6[:3])
        assert np.linalg.norm(xf[3:] - xf6[3:]) < 1e-11 * np.linalg.norm(xf6[3:])


def test_stm_matches_gauss_legendre(ora):
    """PC variational sweep against Gauss-Legendre collocation (order 12) on the
    same variational equations, one config-1 revolution."""
    w = W.config1(M=1)
    m, o = _model(ora, w), _opts(ora, w)
    x0 = w.x0[0]
    bounds, _ = _schedule(ora, w, x0)
    _, Phi, _, _ = ora.stm_propagate(m, o, x0, bounds)
    _, Pg, capped = ora.gl_stm_propagate(m, x0, w.t0, w.tf, 1200)
    assert capped == 0
    _, Pg2, _ = ora.gl_stm_propagate(m, x0, w.t0, w.tf, 2400)
    assert _scaled_rel(Pg, Pg2, H6) < 1e-11          # GL itself converged
    assert _scaled_rel(Phi, Pg2, H6) < 1e-9


def test_stm_matches_propagate_fd(ora):
    """PC variational sweep against central differences of the 6-state oracle
    (ora_propagate, uniform schedule of config 1: no halving), 10 km / 1e-5 km/s
    steps."""
    w = W.config1(M=2)
    m, o = _model(ora, w), _opts(ora, w)
    h = 10.0 * H6
    for x0 in w.x0:
        bounds, _ = _schedule(ora, w, x0)
        assert len(bounds) == w.segments + 1
        _, Phi, _, _ = ora.stm_propagate(m, o, x0, bounds)
        xs = np.array([x0 + s * h[q] * np.eye(6)[q] for q in range(6) for s in (1.0, -1.0)])
        r = ora.propagate(m, o, xs, w.t0, w.tf)
        assert np.all(r["nseg"] == w.segments)
        fd = ((r["xf"][0::2] - r["xf"][1::2]) / (2 * h[:, None])).T
        assert _scaled_rel(Phi, fd, h) < 3e-8


def test_stm_composition(ora):
    """Phi(t2, t0) = Phi(t2, t1) Phi(t1, t0) with t1 an interior segment bound."""
    w = W.config1(M=1)
    m, o = _model(ora, w), _opts(ora, w)
    x0 = w.x0[0]
    bounds, _ = _schedule(ora, w, x0)
    k = len(bounds) // 2
    _, P_all, _, _ = ora.stm_propagate(m, o, x0, bounds)
    x1, P1, _, _ = ora.stm_propagate(m, o, x0, bounds[: k + 1])
    _, P2, _, _ = ora.stm_propagate(m, o, x1, bounds[k:])
    assert _scaled_rel(P2 @ P1, P_all, H6) < 1e-11


def test_gl_stm_matches_gl_finite_differences(ora):
    """Gauss-Legendre variational integration against central differences of
    the 6-state Gauss-Legendre integrator (same steps; 10 km / 1e-5 km/s)."""
    w = W.config1(M=1)
    m, o = _model(ora, w), _opts(ora, w)
    x0 = w.x0[0]
    steps = 600
    _, P, capped = ora.gl_stm_propagate(m, x0, w.t0, w.tf, steps)
    assert capped == 0
    h = 10.0 * H6
    fd = np.zeros((6, 6))
    for q in range(6):
        e = np.zeros(6)
        e[q] = h[q]
        xp, c1 = ora.gl_propagate(m, o, x0 + e, w.t0, w.tf, steps)
        xm, c2 = ora.gl_propagate(m, o, x0 - e, w.t0, w.tf, steps)
        assert c1 == c2 == 0
        fd[:, q] = (xp - xm) / (2 * h[q])
    assert _scaled_rel(P, fd, h) < 3e-8
