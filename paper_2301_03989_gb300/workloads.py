"""Seeded synthetic workloads for the batched Picard-Chebyshev propagator.

The paper's own data set (13,509 initial conditions from a Solar Orbiter-like
Venus resonant-phase optimisation, Section "Test case") is not available, so
these generators build stand-ins with the same structure: many heliocentric
trajectories, Sun plus planets as point masses whose positions come from
Chebyshev ephemeris tables, arcs of a fraction of an orbit to several years.

This module is shared by the oracle tests, the GPU tests and the benchmark.
It holds none of the PC method's arithmetic (no nodes, operators, force
evaluation, warm start or iteration): it only draws initial conditions and
fits ephemeris tables to synthetic Keplerian planet orbits.  Its own orbit
arithmetic (planet positions, the Venus-relative hyperbola of the flyby
workload) is written independently of both the oracle and the CUDA library.

Units: km, s, km^3/s^2.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

AU = 149597870.7            # km, IAU 2012 (exact)
DAY = 86400.0
YEAR = 365.25 * DAY
MU_SUN = 1.32712440018e11   # km^3/s^2

# DE440-class GMs (km^3/s^2); the workloads are synthetic, these only set scales.
GM = {
    "mercury": 22031.868551, "venus": 324858.592, "earth": 398600.435507, "moon": 4902.800118,
    "mars": 42828.375816, "jupiter": 126712764.1, "saturn": 37940584.8418, "uranus": 5794556.4,
    "neptune": 6836527.10058,
}
A_AU = {"mercury": 0.387, "venus": 0.723, "earth": 1.000, "mars": 1.524, "jupiter": 5.203,
        "saturn": 9.537, "uranus": 19.19, "neptune": 30.07}

GRANULE = 32.0 * DAY        # ephemeris granule length
TABLE_DEGREE = 13           # Chebyshev degree per granule and axis


@dataclass
class Workload:
    """A complete synthetic problem: force model, ephemeris table, ICs, arc."""
    name: str
    mu_central: float
    body_names: list
    mu: np.ndarray            # [B]
    t_begin: float            # table start epoch
    granule: float
    coef: np.ndarray          # [B][G][3][deg+1]
    x0: np.ndarray            # [M][6] initial states (heliocentric)
    t0: float
    tf: float
    N: int                    # Chebyshev degree of the PC segments
    segments: int             # segments per arc (seg_mode 0) or per osculating period (1)
    seg_mode: int = 0
    tol: float = 1e-13
    max_iters: int = 60
    max_depth: int = 8
    indirect: bool = True
    meta: dict = field(default_factory=dict)

    @property
    def n_ic(self) -> int:
        return int(self.x0.shape[0])

    def subset(self, idx) -> "Workload":
        idx = np.asarray(idx)
        w = Workload(**{**self.__dict__})
        w.x0 = np.ascontiguousarray(self.x0[idx])
        w.meta = dict(self.meta, subset=idx.tolist() if idx.size <= 64 else f"{idx.size} of {self.n_ic}")
        return w


# --------------------------------------------------------------------------
# Synthetic planet orbits (two-body ellipses, generator-only arithmetic)
# --------------------------------------------------------------------------
def _rot(i, raan, argp):
    """Perifocal -> inertial rotation R3(-raan) R1(-i) R3(-argp)."""
    cO, sO, ci, si, cw, sw = np.cos(raan), np.sin(raan), np.cos(i), np.sin(i), np.cos(argp), np.sin(argp)
    return np.array([
        [cO * cw - sO * sw * ci, -cO * sw - sO * cw * ci, sO * si],
        [sO * cw + cO * sw * ci, -sO * sw + cO * cw * ci, -cO * si],
        [sw * si, cw * si, ci],
    ])


def ellipse_state(el: dict, mu: float, t):
    """Position and velocity on a fixed ellipse at times t (array).  The
    eccentric anomaly comes from the fixed-point iteration E <- M + e sin E,
    which converges for the small eccentricities (<= 0.3) used here."""
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    a, e = el["a"], el["e"]
    n = np.sqrt(mu / a**3)
    M = el["M0"] + n * t
    E = M.copy()
    for _ in range(200):
        E = M + e * np.sin(E)
    cE, sE = np.cos(E), np.sin(E)
    b = a * np.sqrt(1.0 - e * e)
    Edot = n / (1.0 - e * cE)
    pf_r = np.stack([a * (cE - e), b * sE, np.zeros_like(E)], axis=-1)
    pf_v = np.stack([-a * sE * Edot, b * cE * Edot, np.zeros_like(E)], axis=-1)
    R = _rot(el["i"], el["raan"], el["argp"])
    return pf_r @ R.T, pf_v @ R.T


def elements_to_state(a, e, i, raan, argp, M0, mu):
    r, v = ellipse_state(dict(a=a, e=e, i=i, raan=raan, argp=argp, M0=M0), mu, 0.0)
    return np.concatenate([r[0], v[0]])


class _Body:
    def __init__(self, name, el, mu_orbit, parent=None):
        self.name, self.el, self.mu_orbit, self.parent = name, el, mu_orbit, parent

    def position(self, t):
        r, _ = ellipse_state(self.el, self.mu_orbit, t)
        if self.parent is not None:
            r = r + self.parent.position(t)
        return r

    def state(self, t):
        r, v = ellipse_state(self.el, self.mu_orbit, t)
        if self.parent is not None:
            pr, pv = self.parent.state(t)
            r, v = r + pr, v + pv
        return r, v


def fit_tables(bodies, t_begin: float, n_granules: int, granule: float = GRANULE, degree: int = TABLE_DEGREE):
    """Chebyshev tables [B][G][3][deg+1]: per granule, interpolation at the
    deg+1 Chebyshev-Gauss-Lobatto points sigma_i = cos(i pi/deg) of the local
    variable sigma = 2 (t - t_g)/L - 1 (numpy's chebfit with as many points as
    coefficients is exact interpolation)."""
    sig = np.cos(np.pi * np.arange(degree + 1) / degree)
    coef = np.zeros((len(bodies), n_granules, 3, degree + 1))
    for g in range(n_granules):
        tg = t_begin + g * granule
        ts = tg + (sig + 1.0) * 0.5 * granule
        for b, body in enumerate(bodies):
            r = body.position(ts)                                  # [deg+1][3]
            coef[b, g] = np.polynomial.chebyshev.chebfit(sig, r, degree).T
    return coef


def _table_span(t_lo: float, t_hi: float, granule: float = GRANULE):
    """One granule of margin on each side of [t_lo, t_hi]."""
    t_begin = t_lo - granule
    n_gr = int(np.ceil((t_hi - t_lo) / granule)) + 2
    return t_begin, n_gr


# --------------------------------------------------------------------------
# Config 1: Sun + Venus + Earth (circular, coplanar), 64 ICs, 1 revolution
# --------------------------------------------------------------------------
def _circular_system():
    names = ["venus", "earth"]
    phases = {"venus": 0.0, "earth": 0.5 * np.pi}
    bodies = [_Body(nm, dict(a=A_AU[nm] * AU, e=0.0, i=0.0, raan=0.0, argp=0.0, M0=phases[nm]), MU_SUN)
              for nm in names]
    return names, bodies


def _jittered_ics(rng, M, a, e, inc, sig_r=1.0, sig_v=1e-6):
    x = elements_to_state(a, e, inc, 0.0, 0.0, 0.0, MU_SUN)
    jit = rng.standard_normal((M, 6)) * np.array([sig_r] * 3 + [sig_v] * 3)
    return x[None, :] + jit


def config1(M: int = 64, seed: int = 1) -> Workload:
    """Plain FP64 PC, Sun + Venus + Earth point masses on circular coplanar
    orbits (0.723, 1.0 AU); ICs a = 0.75 AU, e = 0.3, i = 2 deg at perihelion,
    Gaussian jitter 1 km / 1 mm/s per component; one revolution in 8 uniform
    segments, degree N = 64, tol 1e-13."""
    rng = np.random.Generator(np.random.PCG64(seed))
    names, bodies = _circular_system()
    a = 0.75 * AU
    T = 2.0 * np.pi * np.sqrt(a**3 / MU_SUN)
    t0, tf = 0.0, T
    tb, ng = _table_span(t0, tf)
    coef = fit_tables(bodies, tb, ng)
    x0 = _jittered_ics(rng, M, a, 0.3, np.deg2rad(2.0))
    return Workload("cfg1_sun_venus_earth_64ic_1rev_N64", MU_SUN, names, np.array([GM[n] for n in names]),
                    tb, GRANULE, coef, x0, t0, tf, N=64, segments=8, seg_mode=0, tol=1e-13,
                    meta=dict(seed=seed, revolution_s=T))


# --------------------------------------------------------------------------
# Config 2: Sun + 8 planets + Moon, 4096 ICs with close Venus flybys, 4 years
# --------------------------------------------------------------------------
def _full_system(rng):
    planets = ["mercury", "venus", "earth", "mars", "jupiter", "saturn", "uranus", "neptune"]
    bodies = []
    by = {}
    for nm in planets:
        el = dict(a=A_AU[nm] * AU, e=rng.uniform(0.0, 0.1), i=np.deg2rad(rng.uniform(0.0, 7.0)),
                  raan=rng.uniform(0, 2 * np.pi), argp=rng.uniform(0, 2 * np.pi), M0=rng.uniform(0, 2 * np.pi))
        b = _Body(nm, el, MU_SUN)
        by[nm] = b
        bodies.append(b)
    mel = dict(a=384400.0, e=rng.uniform(0.0, 0.1), i=np.deg2rad(rng.uniform(0.0, 7.0)),
               raan=rng.uniform(0, 2 * np.pi), argp=rng.uniform(0, 2 * np.pi), M0=rng.uniform(0, 2 * np.pi))
    bodies.append(_Body("moon", mel, GM["earth"] + GM["moon"], parent=by["earth"]))
    return planets + ["moon"], bodies


def _hyperbola_state(rng, mu, rp, vinf, dt_before):
    """Venus-relative state dt_before seconds before periapsis on a hyperbola
    with periapsis radius rp and hyperbolic excess speed vinf, with a random
    incoming-asymptote direction and a random orbit plane containing it."""
    e = 1.0 + rp * vinf**2 / mu
    a = mu / vinf**2                       # |a|
    s = rng.standard_normal(3)
    s /= np.linalg.norm(s)                 # incoming asymptote direction
    q = rng.standard_normal(3)
    q -= q.dot(s) * s
    nrm = q / np.linalg.norm(q)            # orbit normal, perpendicular to s
    w = np.cross(nrm, s)
    al, be = 1.0 / e, np.sqrt(1.0 - 1.0 / e**2)
    p_hat = al * s - be * w                # periapsis direction
    q_hat = np.cross(nrm, p_hat)
    n = np.sqrt(mu / a**3)
    Mh = -n * dt_before                    # hyperbolic mean anomaly (before periapsis)
    H = np.arcsinh(Mh / e)
    for _ in range(100):                   # Newton on e sinh H - H = Mh
        f = e * np.sinh(H) - H - Mh
        H -= f / (e * np.cosh(H) - 1.0)
    Hd = n / (e * np.cosh(H) - 1.0)
    x_pf = a * (e - np.cosh(H))
    y_pf = a * np.sqrt(e * e - 1.0) * np.sinh(H)
    vx_pf = -a * np.sinh(H) * Hd
    vy_pf = a * np.sqrt(e * e - 1.0) * np.cosh(H) * Hd
    return x_pf * p_hat + y_pf * q_hat, vx_pf * p_hat + vy_pf * q_hat


def config2(M: int = 4096, seed: int = 2, years: float = 4.0) -> Workload:
    """Plain FP64 PC, Sun + Mercury..Neptune + Moon (B = 9) on seeded
    Keplerian orbits (real-scale a, e <= 0.1, i <= 7 deg) fitted to Chebyshev
    tables (32-day granules, degree 13); every IC starts 0.5-1.5 days before a
    close Venus flyby (periapsis 1e4-5e4 km, v_inf 3-6 km/s, random geometry)
    and is propagated for `years` years; degree N = 128, 16 base segments per
    osculating period with segment halving."""
    rng = np.random.Generator(np.random.PCG64(seed))
    names, bodies = _full_system(rng)
    t0, tf = 0.0, years * YEAR
    tb, ng = _table_span(min(t0, tf), max(t0, tf))
    coef = fit_tables(bodies, tb, ng)
    venus = bodies[names.index("venus")]
    vr, vv = venus.state(np.array([t0]))
    x0 = np.zeros((M, 6))
    rp = rng.uniform(1e4, 5e4, M)
    vinf = rng.uniform(3.0, 6.0, M)
    dtp = rng.uniform(0.5, 1.5, M) * DAY
    for m in range(M):
        r, v = _hyperbola_state(rng, GM["venus"], rp[m], vinf[m], dtp[m])
        x0[m, :3] = vr[0] + r
        x0[m, 3:] = vv[0] + v
    return Workload(f"cfg2_sun_8planets_moon_{M}ic_venus_flyby_{years:g}yr_N128", MU_SUN, names,
                    np.array([GM[n] for n in names]), tb, GRANULE, coef, x0, t0, tf, N=128, segments=16,
                    seg_mode=1, tol=1e-13, max_iters=60, max_depth=12,
                    meta=dict(seed=seed, rp_km=rp, vinf_kms=vinf, t_periapsis_s=dtp))


# --------------------------------------------------------------------------
# Config 3: config-1 system, 65,536 ICs, 2-year arcs, N = 128
# --------------------------------------------------------------------------
def config3(M: int = 65536, seed: int = 3) -> Workload:
    """Config-1 system and IC distribution; 2-year arcs (63,115,200 s) in 25
    uniform segments, N = 128, tol 1e-13 (the precision study workload)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    names, bodies = _circular_system()
    t0, tf = 0.0, 2.0 * YEAR
    tb, ng = _table_span(t0, tf)
    coef = fit_tables(bodies, tb, ng)
    x0 = _jittered_ics(rng, M, 0.75 * AU, 0.3, np.deg2rad(2.0))
    return Workload(f"cfg3_sun_venus_earth_{M}ic_2yr_N128", MU_SUN, names, np.array([GM[n] for n in names]),
                    tb, GRANULE, coef, x0, t0, tf, N=128, segments=25, seg_mode=0, tol=1e-13,
                    meta=dict(seed=seed))


# --------------------------------------------------------------------------
# Config 4: differentiation -- config-1 system, one Venus flyby per arc
# --------------------------------------------------------------------------
def config4(M: int = 1024, seed: int = 4) -> Workload:
    """Config-1 system (Sun + Venus + Earth, circular coplanar).  Every IC
    starts 2-5 days before periapsis of a close Venus flyby (periapsis
    1e4-5e4 km, v_inf 3-6 km/s, random geometry, taken on the Venus-relative
    hyperbola) and is propagated for one config-1 revolution; N = 128, 16 base
    segments per osculating period with halving.  meta["t_ca"] holds each
    IC's nominal periapsis epoch (where its b-plane is taken), meta["body"]
    the flyby body's index and meta["mu_body"] its GM."""
    rng = np.random.Generator(np.random.PCG64(seed))
    names, bodies = _circular_system()
    a = 0.75 * AU
    T = 2.0 * np.pi * np.sqrt(a**3 / MU_SUN)
    t0, tf = 0.0, T
    tb, ng = _table_span(t0, tf)
    coef = fit_tables(bodies, tb, ng)
    venus = bodies[names.index("venus")]
    rp = rng.uniform(1e4, 5e4, M)
    vinf = rng.uniform(3.0, 6.0, M)
    dtp = rng.uniform(2.0, 5.0, M) * DAY
    x0 = np.zeros((M, 6))
    vr, vv = venus.state(np.zeros(1) + t0)
    for m in range(M):
        r, v = _hyperbola_state(rng, GM["venus"], rp[m], vinf[m], dtp[m])
        x0[m, :3] = vr[0] + r
        x0[m, 3:] = vv[0] + v
    return Workload(f"cfg4_sun_venus_earth_{M}ic_venus_flyby_1rev_N128", MU_SUN, names,
                    np.array([GM[n] for n in names]), tb, GRANULE, coef, x0, t0, tf, N=128, segments=16,
                    seg_mode=1, tol=1e-13, max_iters=60, max_depth=12,
                    meta=dict(seed=seed, rp_km=rp, vinf_kms=vinf, t_ca=t0 + dtp, body=names.index("venus"),
                              mu_body=GM["venus"], revolution_s=T))


# --------------------------------------------------------------------------
# Config 5: uneven batching -- per-trajectory durations, degrees and segments
# --------------------------------------------------------------------------
# Segments per revolution of the config-1 orbit at which the oracle converges to
# 1e-13 within 40 sweeps without halving, by degree (oracle/calibrate_segment_lengths.py).
SEGMENTS_PER_REV = {32: 4, 64: 2, 128: 1, 256: 1}


@dataclass
class UnevenWorkload:
    """Per-trajectory arcs [t0, tf], degrees N and base segment counts S."""
    name: str
    base: Workload            # force model, tables, options (N, segments unused)
    x0: np.ndarray            # [M][6]
    t0: np.ndarray            # [M]
    tf: np.ndarray            # [M]
    N: np.ndarray             # [M] Chebyshev degree per trajectory
    S: np.ndarray             # [M] base segments per trajectory (per arc)
    meta: dict = field(default_factory=dict)

    @property
    def n_ic(self) -> int:
        return int(self.x0.shape[0])

    def groups(self):
        """Stable order by degree: (perm, degrees, counts) -- perm lists the
        trajectories group by group."""
        degs = sorted(set(int(n) for n in self.N))
        perm = np.concatenate([np.flatnonzero(self.N == d) for d in degs])
        counts = [int((self.N == d).sum()) for d in degs]
        return perm, degs, counts


def config5(M: int = 1048576, seed: int = 5, years_max: float = 10.0) -> UnevenWorkload:
    """Config-1 system and IC distribution; durations D ~ U(0.5, years_max) yr,
    degree N ~ U{32, 64, 128, 256}, S = clamp(ceil(D / L(N)), 4, 80) with
    L(N) = revolution / SEGMENTS_PER_REV[N]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    names, bodies = _circular_system()
    a = 0.75 * AU
    T = 2.0 * np.pi * np.sqrt(a**3 / MU_SUN)
    tb, ng = _table_span(0.0, years_max * YEAR)
    coef = fit_tables(bodies, tb, ng)
    x0 = _jittered_ics(rng, M, a, 0.3, np.deg2rad(2.0))
    D = rng.uniform(0.5, years_max, M) * YEAR
    N = rng.choice(np.array([32, 64, 128, 256]), M)
    L = np.array([T / SEGMENTS_PER_REV[int(n)] for n in N])
    S = np.clip(np.ceil(D / L), 4, 80).astype(np.int32)
    base = Workload(f"cfg5_sun_venus_earth_{M}ic_uneven", MU_SUN, names, np.array([GM[n] for n in names]),
                    tb, GRANULE, coef, x0, 0.0, years_max * YEAR, N=128, segments=4, seg_mode=0, tol=1e-13,
                    meta=dict(seed=seed))
    return UnevenWorkload(base.name, base, x0, np.zeros(M), D, N.astype(np.int32), S, meta=dict(seed=seed))


def to_planar(x: np.ndarray) -> np.ndarray:
    """[M][6] -> component-planar [6][M] (the paper's component-stacked layout)."""
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(-1, 6).T)


def from_planar(x: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x).reshape(6, -1).T)
