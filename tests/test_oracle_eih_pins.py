"""Pins of the oracle's Einstein-Infeld-Hoffmann (1PN) force terms
(ora_eih_terms, and the model wrapper that builds the bodies from the
ephemeris tables): the Newtonian limit, the Schwarzschild field of one body
at rest, the field of a uniformly moving body seen by a comoving particle (the
rest-frame field carried through a Lorentz transformation), and the
perihelion advance of a Mercury-like orbit against 6 pi mu / (c^2 a (1 - e^2)).
The terms in the bodies' own accelerations are not pinned."""
import numpy as np

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
