"""Pins of the oracle's Einstein-Infeld-Hoffmann (1PN) force terms
(ora_eih_terms, and the model wrapper that builds the bodies from the
ephemeris tables): the Newtonian limit, the Schwarzschild field of one body
at rest, the field of a uniformly moving body seen by a comoving particle (the
rest-frame field carried through a Lorentz transformation), and the
perihelion advance of a Mercury-like orbit against 6 pi mu / (c^2 a (1 - e^2)), and
every term (including those of the bodies' accelerations and potentials)
against the geodesic of the harmonic-gauge 1PN metric of the bodies."""
import numpy as np
import pytest

from paper_2301_03989_gb300 import workloads as W

C_LIGHT = 299792.458  # km/s
MU = W.MU_SUN


def test_newtonian_limit(ora):
    """With c -> infinity the EIH dynamics are the Newtonian ones, bit for bit."""
    w = W.config2(M=8)
    o = ora.Opts(N=w.N)
    newt = ora.Model.from_workload(w)
    huge = ora.Model.from_workload(w, c_light=1e40)
    for i in range(8):
        t = 86400.0 * (3 + 40 * i)
        np.testing.assert_array_equal(ora.dynamics(huge, o, t, w.x0[i]), ora.dynamics(newt, o, t, w.x0[i]))


def test_schwarzschild_field(ora):
    """One body at rest: the 1/c^2 terms are mu/(c^2 r^2) [(4 mu/r - v^2) n + 4 (n.v) v]."""
    rng = np.random.default_rng(1)
    for _ in range(20):
        X = rng.standard_normal(3) * 10.0 ** rng.uniform(6, 9)
        Wv = rng.standard_normal(3) * 40.0
        got = ora.eih_terms([MU], np.zeros(3), np.zeros(3), np.zeros(3), [0.0], X, Wv, C_LIGHT)
        r = np.linalg.norm(X)
        n = X / r
        ref = MU / (C_LIGHT**2 * r**2) * ((4 * MU / r - Wv @ Wv) * n + 4 * (n @ Wv) * Wv)
        np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())


def test_comoving_particle_in_the_field_of_a_moving_body(ora):
    """A body moving uniformly with velocity u and a particle momentarily at
    rest relative to it (same velocity).  In the body's rest frame the particle
    is at X' (the lab separation stretched by gamma along u) and feels the
    Schwarzschild acceleration of a particle at rest, -mu X'/|X'|^3 (1 - 4 mu /
    (|X'| c^2)); carried back to the lab frame (components along u divided by
    gamma^3, across by gamma^2) and stripped of the lab-frame Newtonian term it
    must equal the EIH 1/c^2 terms up to O(1/c^4)."""
    rng = np.random.default_rng(2)
    c = C_LIGHT
    for _ in range(20):
        u = rng.standard_normal(3)
        u *= 300.0 / np.linalg.norm(u)
        X = rng.standard_normal(3)
        X *= 1.0e6 / np.linalg.norm(X)
        gam = 1.0 / np.sqrt(1.0 - (u @ u) / c**2)
        uh = u / np.linalg.norm(u)
        Xpar, Xperp = (X @ uh) * uh, X - (X @ uh) * uh
        Xr = gam * Xpar + Xperp
        rr = np.linalg.norm(Xr)
        ar = -MU * Xr / rr**3 * (1.0 - 4.0 * MU / (rr * c**2))
        apar, aperp = (ar @ uh) * uh, ar - (ar @ uh) * uh
        a_lab = apar / gam**3 + aperp / gam**2
        ref = a_lab - (-MU * X / np.linalg.norm(X) ** 3)
        got = ora.eih_terms([MU], np.zeros(3), u, np.zeros(3), [0.0], X, u, c)
        # the 1PN part is ~1e-6 of the Newtonian one; O(1/c^4) leaves ~1e-6 of it
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-5 * np.abs(ref).max())


def _perihelion_angle(ora, model, x0, T, N=64, segments=16):
    """Propagates x0 (at perihelion on the x axis, orbit in the xy plane) to the
    next perihelion, found by Newton's method on r.v, and returns its angle."""
    o = ora.Opts(N=N, segments=segments, tol=1e-13)
    t = T
    for _ in range(6):
        y = ora.propagate(model, o, x0[None], 0.0, t)["xf"][0]
        r, v = y[:3], y[3:]
        f = r @ v
        df = v @ v - MU / np.linalg.norm(r)
        t -= f / df
    y = ora.propagate(model, o, x0[None], 0.0, t)["xf"][0]
    return np.arctan2(y[1], y[0])


def test_perihelion_advance(ora):
    """Sun alone, a = 0.387 AU, e = 0.2056: the angle between successive
    perihelia is 6 pi mu / (c^2 a (1 - e^2)) (5.0e-7 rad) to 1e-4, and zero
    without the EIH terms."""
    a, e = 0.387 * W.AU, 0.2056
    rp = a * (1 - e)
    vp = np.sqrt(MU * (1 + e) / rp)
    x0 = np.array([rp, 0.0, 0.0, 0.0, vp, 0.0])
    T = 2 * np.pi * np.sqrt(a**3 / MU)
    rel = ora.Model(mu_central=MU, mu=np.zeros(0), c_light=C_LIGHT)
    newt = ora.Model(mu_central=MU, mu=np.zeros(0))
    expected = 6 * np.pi * MU / (C_LIGHT**2 * a * (1 - e * e))
    d_rel = _perihelion_angle(ora, rel, x0, T)
    d_newt = _perihelion_angle(ora, newt, x0, T)
    assert abs(d_newt) < 1e-11, d_newt
    assert abs(d_rel / expected - 1.0) < 1e-4, (d_rel, expected)


def test_model_wrapper_builds_barycentric_bodies(ora):
    """The wrapper's bodies: the Sun at the heliocentric origin and the table's
    bodies, velocities shifted by -sum mu_b v_b / sum mu, Newtonian
    accelerations and potentials of each body from the others."""
    w = W.config2(M=4)
    m = ora.Model.from_workload(w, c_light=C_LIGHT)
    t = 123456.0
    rb = ora.ephem_eval(m, t).reshape(-1, 3)
    vb = ora.ephem_vel(m, t).reshape(-1, 3)
    mu = np.r_[w.mu_central, w.mu]
    vs = -(w.mu[:, None] * vb).sum(0) / mu.sum()
    P = np.vstack([np.zeros(3), rb])
    V = np.vstack([vs, vb + vs])
    A = np.zeros_like(P)
    Phi = np.zeros(len(mu))
    for j in range(len(mu)):
        for k in range(len(mu)):
            if k != j:
                d = P[k] - P[j]
                A[j] += mu[k] * d / np.linalg.norm(d) ** 3
                Phi[j] += mu[k] / np.linalg.norm(d)
    for i in range(4):
        y = w.x0[i]
        ref = ora.eih_terms(mu, P, V, A, Phi, y[:3], y[3:] + vs, C_LIGHT)
        np.testing.assert_allclose(ora.eih_at(m, t, y), ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def _geodesic_1pn_terms(mp, mu, P, V, A, Phi, X, W, c):
    """1/c^2 part of the coordinate acceleration of a test particle at X with
    velocity W (t = 0) on a geodesic of the harmonic-gauge 1PN metric of point
    masses mu_A moving as x_A(t) = P_A + V_A t + A_A t^2 / 2:
      g00 = -1 + 2U/c^2 + 2(psi - U^2)/c^4,  g0j = -4 U_j/c^3,  gjk = (1 + 2U/c^2) delta_jk,
      U = sum mu_A/r_A,  U_j = sum mu_A v_A^j / r_A,
      psi = sum mu_A (3/2 v_A^2 - Phi_A)/r_A + 1/2 d^2/dt^2 sum mu_A r_A
    (Phi_A the potential of the other bodies at body A).  The Christoffel
    symbols come from 50-digit numerical derivatives of the metric; the
    acceleration is d^2x^i/dt^2 = -Gamma^i_ab xd^a xd^b + (v^i/c) Gamma^0_ab
    xd^a xd^b with xd = (c, v), minus the Newtonian grad U."""
    mp.mp.dps = 50
    c = mp.mpf(c)
    M = lambda a: [mp.mpf(float(v)) for v in np.ravel(a)]
    mu, Phi = M(mu), M(Phi)
    nb = len(mu)
    P, V, A = [[M(q)[3 * b:3 * b + 3] for b in range(nb)] for q in (P, V, A)]

    def metric(x0, x1, x2, x3):
        t, xp = x0 / c, (x1, x2, x3)
        U, Uj, psi = mp.mpf(0), [mp.mpf(0)] * 3, mp.mpf(0)
        for a in range(nb):
            va = [V[a][k] + A[a][k] * t for k in range(3)]
            s = [xp[k] - (P[a][k] + V[a][k] * t + A[a][k] * t * t / 2) for k in range(3)]
            r = mp.sqrt(sum(q * q for q in s))
            v2 = sum(q * q for q in va)
            sv = sum(s[k] * va[k] for k in range(3))
            sa = sum(s[k] * A[a][k] for k in range(3))
            U += mu[a] / r
            Uj = [Uj[k] + mu[a] * va[k] / r for k in range(3)]
            d2r = (v2 - sa) / r - sv * sv / r**3  # d^2/dt^2 |x - x_A(t)|
            psi += mu[a] * (mp.mpf(3) / 2 * v2 - Phi[a]) / r + mu[a] * d2r / 2
        g = mp.zeros(4, 4)
        g[0, 0] = -1 + 2 * U / c**2 + 2 * (psi - U * U) / c**4
        for k in range(3):
            g[0, k + 1] = g[k + 1, 0] = -4 * Uj[k] / c**3
            g[k + 1, k + 1] = 1 + 2 * U / c**2
        return g

    pt = [mp.mpf(0)] + M(X)
    gi = metric(*pt) ** -1
    dg = []
    for m in range(4):
        d = mp.zeros(4, 4)
        for i in range(4):
            for j in range(i, 4):
                def comp(u, i=i, j=j, m=m):
                    q = list(pt)
                    q[m] = u
                    return metric(*q)[i, j]
                d[i, j] = d[j, i] = mp.diff(comp, pt[m])
        dg.append(d)
    gam = lambda l, a, b: sum(gi[l, s] * (dg[a][s, b] + dg[b][s, a] - dg[s][a, b]) for s in range(4)) / 2
    xd = [c] + M(W)
    quad = lambda l: sum(gam(l, a, b) * xd[a] * xd[b] for a in range(4) for b in range(4))
    g0 = quad(0)
    out = []
    for i in range(1, 4):
        newton = mp.mpf(0)
        for a in range(nb):
            s = [pt[k + 1] - P[a][k] for k in range(3)]
            newton -= mu[a] * s[i - 1] / mp.sqrt(sum(q * q for q in s)) ** 3
        out.append(float(-quad(i) + xd[i] / c * g0 - newton))
    return np.array(out)


def test_geodesic_of_the_1pn_metric(ora):
    """Bodies with arbitrary positions, velocities, accelerations and
    potentials (the Sun and two planets' GMs, the Sun near the origin): the EIH
    1/c^2 terms equal the geodesic's 1/c^2 part to 1e-6 of their size (the
    difference is O(1/c^4), about 1e-8).  The terms of the bodies' accelerations
    carry up to about the whole 1PN correction here and those of their
    potentials a few per cent: dropping either fails by far."""
    mp = pytest.importorskip("mpmath")
    rng = np.random.default_rng(5)
    mu = np.array([MU, W.GM["venus"], W.GM["earth"]])
    for _ in range(6):
        P = np.vstack([rng.standard_normal(3) * 1e6, rng.standard_normal(3) * 1e8, rng.standard_normal(3) * 1.5e8])
        V = rng.standard_normal((3, 3)) * 30.0
        A = rng.standard_normal((3, 3)) * 1e-5
        Phi = rng.uniform(1e2, 1e3, 3)
        X = rng.standard_normal(3) * 1.2e8
        Wv = rng.standard_normal(3) * 35.0
        ref = _geodesic_1pn_terms(mp, mu, P, V, A, Phi, X, Wv, C_LIGHT)
        got = ora.eih_terms(mu, P, V, A, Phi, X, Wv, C_LIGHT)
        n = np.abs(ref).max()
        assert np.abs(got - ref).max() < 1e-6 * n, (got, ref)
        # the planted omissions are far outside the bound
        no_acc = ora.eih_terms(mu, P, V, np.zeros_like(A), Phi, X, Wv, C_LIGHT)
        no_phi = ora.eih_terms(mu, P, V, A, np.zeros(3), X, Wv, C_LIGHT)
        assert np.abs(no_acc - ref).max() > 1e-3 * n and np.abs(no_phi - ref).max() > 1e-3 * n
