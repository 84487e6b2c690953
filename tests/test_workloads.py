"""The seeded input generators: structure of the uneven and differentiation
workloads, layout round trips, and the Venus-relative flyby hyperbola checked
against an independent integration of the two-body problem (scipy DOP853)."""
import numpy as np
import pytest

from paper_2301_03989_gb300 import workloads as W


def test_uneven_workload_structure():
    uw = W.config5(M=4096, seed=5)
    years = (uw.tf - uw.t0) / W.YEAR
    assert years.min() >= 0.5 and years.max() <= 10.0
    assert set(np.unique(uw.N)) == {32, 64, 128, 256}
    assert uw.S.min() >= 4 and uw.S.max() <= 80
    # S = clamp(ceil(D / L(N)), 4, 80) with L(N) = revolution / SEGMENTS_PER_REV[N]
    T = 2.0 * np.pi * np.sqrt((0.75 * W.AU) ** 3 / W.MU_SUN)
    L = np.array([T / W.SEGMENTS_PER_REV[int(n)] for n in uw.N])
    np.testing.assert_array_equal(uw.S, np.clip(np.ceil((uw.tf - uw.t0) / L), 4, 80).astype(np.int32))
    perm, degs, counts = uw.groups()
    assert sorted(perm.tolist()) == list(range(uw.n_ic))
    assert list(degs) == sorted(degs) and sum(counts) == uw.n_ic
    off = 0
    for d, c in zip(degs, counts):
        assert np.all(uw.N[perm[off:off + c]] == d)
        off += c


def test_planar_round_trip():
    x = np.random.default_rng(0).standard_normal((7, 6))
    p = W.to_planar(x)
    assert p.shape == (6, 7) and p.flags.c_contiguous
    np.testing.assert_array_equal(W.from_planar(p), x)


def test_differentiation_workload_epochs():
    w = W.config4(M=64)
    t_ca = w.meta["t_ca"]
    assert np.all((t_ca - w.t0 >= 2 * W.DAY) & (t_ca - w.t0 <= 5 * W.DAY))
    assert w.tf - w.t0 == pytest.approx(w.meta["revolution_s"])
    assert w.body_names[w.meta["body"]] == "venus"


def test_flyby_hyperbola_reaches_its_periapsis():
    """The generator's Venus-relative state dt before periapsis, integrated
    forward by dt under Venus alone, arrives at distance r_p with velocity
    perpendicular to the radius (independent integrator)."""
    from scipy.integrate import solve_ivp
    mu = W.GM["venus"]
    rng = np.random.Generator(np.random.PCG64(11))
    for rp, vinf, dt in [(1.2e4, 3.5, 0.7 * W.DAY), (4.5e4, 5.8, 1.4 * W.DAY), (2.0e4, 4.0, 4.0 * W.DAY)]:
        r, v = W._hyperbola_state(rng, mu, rp, vinf, dt)
        # energy fixes v_inf: v^2/2 - mu/r = vinf^2/2
        assert 0.5 * v.dot(v) - mu / np.linalg.norm(r) == pytest.approx(0.5 * vinf**2, rel=1e-12)

        def f(t, y):
            rr = y[:3]
            return np.r_[y[3:], -mu * rr / np.linalg.norm(rr) ** 3]
        sol = solve_ivp(f, (0.0, dt), np.r_[r, v], method="DOP853", rtol=1e-12, atol=1e-9)
        rf, vf = sol.y[:3, -1], sol.y[3:, -1]
        assert np.linalg.norm(rf) == pytest.approx(rp, rel=1e-7)
        assert abs(rf.dot(vf)) / (np.linalg.norm(rf) * np.linalg.norm(vf)) < 1e-6
