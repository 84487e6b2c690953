"""ctypes wrapper of the plain FP64 CPU oracle (oracle/pc_oracle.c).

TEST INFRASTRUCTURE ONLY: the oracle is what the CUDA library is checked
against.  Only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It never imports the CUDA library and the
library never imports it.

Every function follows a passage of Masat, Colombo & Boutonnet (arXiv
2301.03989); the citations are in pc_oracle.c next to each routine.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pc_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

# Outcomes / statuses (mirror the enums in pc_oracle.c)
SEG_OK, SEG_STALLED, SEG_FAIL_CAP, SEG_FAIL_DIV, SEG_FAIL_TRUNC = 0, 1, 2, 3, 4
IC_OK, IC_STALLED, IC_UNRESOLVED, IC_NOT_CONVERGED, IC_NONFINITE = 0, 1, 2, 4, 8   # bit flags
DYN_NBODY, DYN_CONST_ACCEL, DYN_HARMONIC = 0, 1, 2


def build(force: bool = False) -> str:
    """Compiles the oracle with gcc (FP64, no fast-math, no FP contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fno-fast-math", "-ffp-contract=off",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm", "-lpthread"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Model(C.Structure):
    _fields_ = [("n_bodies", C.c_int), ("mu_central", C.c_double), ("mu", C.POINTER(C.c_double)),
                ("indirect", C.c_int), ("t_begin", C.c_double), ("granule", C.c_double),
                ("degree", C.c_int), ("n_granules", C.c_int), ("coef", C.POINTER(C.c_double)),
                ("c_light", C.c_double)]


class _Opts(C.Structure):
    _fields_ = [("N", C.c_int), ("truncated", C.c_int), ("tol", C.c_double), ("relative", C.c_int),
                ("max_iters", C.c_int), ("max_depth", C.c_int), ("warm_start", C.c_int),
                ("seg_mode", C.c_int), ("segments", C.c_int), ("stall_sweeps", C.c_int),
                ("stall_factor", C.c_double), ("div_limit", C.c_double), ("trunc_tol", C.c_double),
                ("dyn", C.c_int),
                ("dyn_param", C.c_double * 3), ("order", C.c_int)]


class _StopState(C.Structure):
    _fields_ = [("e_best", C.c_double), ("nstall", C.c_int)]


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P = C.POINTER
            L.ora_cgl_nodes.argtypes = [C.c_int, P(C.c_double)]
            L.ora_pc_operator.argtypes = [C.c_int, C.c_int, P(C.c_double)]
            L.ora_ephem_eval.argtypes = [P(_Model), C.c_double, P(C.c_double)]
            L.ora_accel.argtypes = [P(_Model), P(C.c_double), P(C.c_double), P(C.c_double)]
            L.ora_dynamics.argtypes = [P(_Model), P(_Opts), C.c_double, P(C.c_double), P(C.c_double)]
            L.ora_eih_terms.argtypes = [C.c_int, P(C.c_double), P(C.c_double), P(C.c_double), P(C.c_double),
                                        P(C.c_double), P(C.c_double), P(C.c_double), C.c_double, P(C.c_double)]
            L.ora_eih_at.argtypes = [P(_Model), C.c_double, P(C.c_double), P(C.c_double)]
            L.ora_kepler.argtypes = [C.c_double, P(C.c_double), C.c_double, P(C.c_double)]
            L.ora_kepler.restype = C.c_int
            L.ora_pc_segment.argtypes = [P(_Model), P(_Opts), C.c_double, C.c_double, P(C.c_double),
                                         P(C.c_double), P(C.c_int), P(C.c_double)]
            L.ora_pc_segment.restype = C.c_int
            L.ora_propagate.argtypes = [P(_Model), P(_Opts), C.c_long, P(C.c_double), C.c_double, C.c_double,
                                        P(C.c_double), P(C.c_int), P(C.c_int), P(C.c_int), C.c_int,
                                        P(C.c_double), C.c_int]
            L.ora_tail_estimate.argtypes = [P(_Opts), P(C.c_double), P(C.c_double), C.c_double]
            L.ora_tail_estimate.restype = C.c_double
            L.ora_gl_coeffs.argtypes = [C.c_int, P(C.c_double), P(C.c_double), P(C.c_double)]
            L.ora_gl_propagate.argtypes = [P(_Model), P(_Opts), C.c_int, P(C.c_double), C.c_double, C.c_double,
                                           C.c_long, P(C.c_double)]
            L.ora_gl_propagate.restype = C.c_int
            L.ora_ephem_vel.argtypes = [P(_Model), C.c_double, P(C.c_double)]
            L.ora_tidal.argtypes = [P(_Model), P(C.c_double), P(C.c_double), P(C.c_double)]
            L.ora_stm_propagate.argtypes = [P(_Model), P(_Opts), P(C.c_double), C.c_int, P(C.c_double),
                                            P(C.c_double), P(C.c_double), P(C.c_int)]
            L.ora_stm_propagate.restype = C.c_int
            L.ora_gl_stm_propagate.argtypes = [P(_Model), C.c_int, P(C.c_double), C.c_double, C.c_double,
                                               C.c_long, P(C.c_double), P(C.c_double)]
            L.ora_gl_stm_propagate.restype = C.c_int
            L.ora_bplane.argtypes = [C.c_double, P(C.c_double), P(C.c_double)]
            L.ora_bplane.restype = C.c_int
            L.ora_pc2_segment.argtypes = [P(_Model), P(_Opts), C.c_double, C.c_double, P(C.c_double),
                                          P(C.c_double), P(C.c_int), P(C.c_double)]
            L.ora_pc2_segment.restype = C.c_int
            L.ora_stop_rule.argtypes = [P(_Opts), P(_StopState), C.c_double, C.c_int]
            L.ora_stop_rule.restype = C.c_int
            L.ora_propagate_log.argtypes = [P(_Model), P(_Opts), P(C.c_double), C.c_double, C.c_double,
                                            P(C.c_double), P(C.c_int), P(C.c_int), P(C.c_int), C.c_int,
                                            P(C.c_double), P(C.c_int)]
            _lib = L
    return _lib


@dataclass
class Model:
    """Force model + ephemeris table (arrays kept alive here)."""
    mu_central: float
    mu: np.ndarray                      # [B]
    t_begin: float = 0.0
    granule: float = 1.0
    coef: np.ndarray | None = None      # [B][G][3][deg+1]
    indirect: bool = True
    c_light: float = 0.0                # km/s; > 0 adds the EIH (1PN) terms
    _s: _Model = field(default=None, repr=False)

    def struct(self) -> _Model:
        self.mu = np.ascontiguousarray(self.mu, dtype=np.float64).reshape(-1)
        B = int(self.mu.size)
        if self.coef is None:
            self.coef = np.zeros((max(B, 1), 1, 3, 1))
        self.coef = np.ascontiguousarray(self.coef, dtype=np.float64)
        s = _Model()
        s.n_bodies = B
        s.mu_central = float(self.mu_central)
        s.mu = _dp(self.mu) if B else C.cast(0, C.POINTER(C.c_double))
        s.indirect = int(bool(self.indirect))
        s.t_begin = float(self.t_begin)
        s.granule = float(self.granule)
        s.degree = int(self.coef.shape[3] - 1)
        s.n_granules = int(self.coef.shape[1])
        s.coef = _dp(self.coef)
        s.c_light = float(self.c_light)
        self._s = s
        return s

    @staticmethod
    def from_workload(w, c_light: float = 0.0) -> "Model":
        return Model(mu_central=w.mu_central, mu=np.asarray(w.mu, dtype=np.float64), t_begin=w.t_begin,
                     granule=w.granule, coef=np.asarray(w.coef, dtype=np.float64), indirect=w.indirect,
                     c_light=c_light)


@dataclass
class Opts:
    N: int = 64
    truncated: bool = False
    tol: float = 1e-13
    relative: bool = True
    max_iters: int = 60
    max_depth: int = 8
    warm_start: bool = True
    seg_mode: int = 0
    segments: int = 8
    stall_sweeps: int = 5
    stall_factor: float = 1e3
    div_limit: float = 1e3
    trunc_tol: float = 1e-13
    dyn: int = DYN_NBODY
    dyn_param: tuple = (0.0, 0.0, 0.0)
    order: int = 1

    def struct(self) -> _Opts:
        s = _Opts()
        s.N, s.truncated, s.tol, s.relative = int(self.N), int(bool(self.truncated)), float(self.tol), int(bool(self.relative))
        s.max_iters, s.max_depth, s.warm_start = int(self.max_iters), int(self.max_depth), int(bool(self.warm_start))
        s.seg_mode, s.segments, s.stall_sweeps = int(self.seg_mode), int(self.segments), int(self.stall_sweeps)
        s.stall_factor, s.div_limit, s.dyn = float(self.stall_factor), float(self.div_limit), int(self.dyn)
        s.trunc_tol = float(self.trunc_tol)
        s.order = int(self.order)
        for i in range(3):
            s.dyn_param[i] = float(self.dyn_param[i])
        return s


def cgl_nodes(N: int) -> np.ndarray:
    tau = np.zeros(N + 1)
    lib().ora_cgl_nodes(N, _dp(tau))
    return tau


def pc_operator(N: int, truncated: bool = False) -> np.ndarray:
    K = np.zeros((N + 1, N + 1))
    lib().ora_pc_operator(N, int(truncated), _dp(K))
    return K


def ephem_eval(model: Model, t: float) -> np.ndarray:
    s = model.struct()
    out = np.zeros((max(s.n_bodies, 1), 3))
    lib().ora_ephem_eval(C.byref(s), float(t), _dp(out))
    return out[: s.n_bodies]


def accel(model: Model, rb: np.ndarray, r) -> np.ndarray:
    s = model.struct()
    rb = np.ascontiguousarray(rb, dtype=np.float64).reshape(-1)
    if rb.size == 0:
        rb = np.zeros(3)
    r = np.ascontiguousarray(r, dtype=np.float64)
    a = np.zeros(3)
    lib().ora_accel(C.byref(s), _dp(rb), _dp(r), _dp(a))
    return a


def dynamics(model: Model, opts: Opts, t: float, y) -> np.ndarray:
    s, o = model.struct(), opts.struct()
    y = np.ascontiguousarray(y, dtype=np.float64)
    f = np.zeros(6)
    lib().ora_dynamics(C.byref(s), C.byref(o), float(t), _dp(y), _dp(f))
    return f


def eih_terms(mu, P, V, A, Phi, X, W, c: float) -> np.ndarray:
    """The 1/c^2 EIH terms of a massless particle at X, W among explicit
    bodies (mu [nb], P, V, A [nb][3], Phi [nb])."""
    f = lambda a: np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
    mu, P, V, A, Phi, X, W = map(f, (mu, P, V, A, Phi, X, W))
    out = np.zeros(3)
    lib().ora_eih_terms(int(mu.size), _dp(mu), _dp(P), _dp(V), _dp(A), _dp(Phi), _dp(X), _dp(W), float(c), _dp(out))
    return out


def eih_at(model: Model, t: float, y) -> np.ndarray:
    """The model's EIH terms at t for the heliocentric state y."""
    s = model.struct()
    y = np.ascontiguousarray(y, dtype=np.float64)
    out = np.zeros(3)
    lib().ora_eih_at(C.byref(s), float(t), _dp(y), _dp(out))
    return out


def kepler(mu: float, x0, dt: float):
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    x = np.zeros(6)
    rc = lib().ora_kepler(float(mu), _dp(x0), float(dt), _dp(x))
    return x, rc


def pc_segment(model: Model, opts: Opts, ta: float, tb: float, x0):
    s, o = model.struct(), opts.struct()
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    Y = np.zeros((opts.N + 1, 6))
    it = C.c_int(0)
    err = C.c_double(0.0)
    outcome = lib().ora_pc_segment(C.byref(s), C.byref(o), float(ta), float(tb), _dp(x0), _dp(Y), C.byref(it),
                                   C.byref(err))
    return Y, int(it.value), float(err.value), int(outcome)


def propagate(model: Model, opts: Opts, x0, t0: float, tf: float, threads: int = 1, max_ckpt: int = 0) -> dict:
    """x0: [M][6].  Returns xf [M][6], status, iters (total sweeps), nseg and,
    if max_ckpt > 0, ckpt [M][max_ckpt][7] = (t_a, x_a) of each accepted segment."""
    s, o = model.struct(), opts.struct()
    x0 = np.ascontiguousarray(np.asarray(x0, dtype=np.float64).reshape(-1, 6))
    M = x0.shape[0]
    xf = np.zeros_like(x0)
    status = np.zeros(M, dtype=np.int32)
    iters = np.zeros(M, dtype=np.int32)
    nseg = np.zeros(M, dtype=np.int32)
    ck = np.zeros((M, max(max_ckpt, 1), 7)) if max_ckpt > 0 else None
    lib().ora_propagate(C.byref(s), C.byref(o), M, _dp(x0), float(t0), float(tf), _dp(xf), _ip(status), _ip(iters),
                        _ip(nseg), int(max_ckpt), _dp(ck) if ck is not None else C.cast(0, C.POINTER(C.c_double)),
                        int(threads))
    out = dict(xf=xf, status=status, iters=iters, nseg=nseg)
    if ck is not None:
        out["ckpt"] = ck
    return out


def stop_rule(opts: Opts, changes) -> tuple[int, int]:
    """Feeds the sweep changes one by one to the oracle's stop rule; returns
    (outcome, sweep) at the first sweep that ends the attempt, or (-1, len)
    if none does."""
    o = opts.struct()
    st = _StopState(float("inf"), 0)
    for i, e in enumerate(changes, start=1):
        out = lib().ora_stop_rule(C.byref(o), C.byref(st), float(e), i)
        if out >= 0:
            return int(out), i
    return -1, len(changes)


def propagate_log(model: Model, opts: Opts, x0, t0: float, tf: float, max_log: int = 256) -> dict:
    """One trajectory with its segment-attempt log: log [k] = (t_a, t_b,
    outcome, sweeps, depth) of each attempt in order."""
    s, o = model.struct(), opts.struct()
    x0 = np.ascontiguousarray(np.asarray(x0, dtype=np.float64).reshape(6))
    xf = np.zeros(6)
    status, iters, nseg, nlog = C.c_int(0), C.c_int(0), C.c_int(0), C.c_int(0)
    log = np.zeros((max_log, 5))
    lib().ora_propagate_log(C.byref(s), C.byref(o), _dp(x0), float(t0), float(tf), _dp(xf), C.byref(status),
                            C.byref(iters), C.byref(nseg), int(max_log), _dp(log), C.byref(nlog))
    k = min(int(nlog.value), max_log)
    return dict(xf=xf, status=int(status.value), iters=int(iters.value), nseg=int(nseg.value),
                n_attempts=int(nlog.value), log=log[:k])


def tail_estimate(opts: Opts, G, Y, w2: float) -> float:
    o = opts.struct()
    G = np.ascontiguousarray(G, dtype=np.float64)
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    return float(lib().ora_tail_estimate(C.byref(o), _dp(G), _dp(Y), float(w2)))


def gl_coeffs(s: int):
    c = np.zeros(s)
    A = np.zeros((s, s))
    b = np.zeros(s)
    lib().ora_gl_coeffs(s, _dp(c), _dp(A), _dp(b))
    return c, A, b


def gl_propagate(model: Model, opts: Opts, x0, t0: float, tf: float, nsteps: int, stages: int = 6):
    s, o = model.struct(), opts.struct()
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    xf = np.zeros(6)
    capped = lib().ora_gl_propagate(C.byref(s), C.byref(o), int(stages), _dp(x0), float(t0), float(tf),
                                    int(nsteps), _dp(xf))
    return xf, int(capped)


# ---- differentiation checks ------------------------------------------------

def ephem_vel(model: Model, t: float) -> np.ndarray:
    """Body velocities [B][3] from the table (time derivative of the series)."""
    s = model.struct()
    out = np.zeros((max(s.n_bodies, 1), 3))
    lib().ora_ephem_vel(C.byref(s), float(t), _dp(out))
    return out[: s.n_bodies]


def tidal(model: Model, rb: np.ndarray, r) -> np.ndarray:
    """Gravity gradient da/dr [3][3] at r with body positions rb [B][3]."""
    s = model.struct()
    rb = np.ascontiguousarray(rb, dtype=np.float64).reshape(-1)
    if rb.size == 0:
        rb = np.zeros(3)
    r = np.ascontiguousarray(r, dtype=np.float64)
    A = np.zeros((3, 3))
    lib().ora_tidal(C.byref(s), _dp(rb), _dp(r), _dp(A))
    return A


def stm_propagate(model: Model, opts: Opts, x0, bounds) -> tuple[np.ndarray, np.ndarray, int, int]:
    """PC on the variational equations over the segment bounds [nseg+1].
    Returns (xf [6], Phi [6][6] = d xf / d x0, segments that hit the cap, sweeps)."""
    s, o = model.struct(), opts.struct()
    x0 = np.ascontiguousarray(x0, dtype=np.float64).reshape(6)
    tb = np.ascontiguousarray(bounds, dtype=np.float64).reshape(-1)
    xf = np.zeros(6)
    Phi = np.zeros((6, 6))
    sw = C.c_int(0)
    capped = lib().ora_stm_propagate(C.byref(s), C.byref(o), _dp(x0), int(tb.size - 1), _dp(tb), _dp(xf), _dp(Phi),
                                     C.byref(sw))
    return xf, Phi, int(capped), int(sw.value)


def gl_stm_propagate(model: Model, x0, t0: float, tf: float, nsteps: int, stages: int = 6):
    """Gauss-Legendre collocation on the variational equations: (xf, Phi, capped steps)."""
    s = model.struct()
    x0 = np.ascontiguousarray(x0, dtype=np.float64).reshape(6)
    xf = np.zeros(6)
    Phi = np.zeros((6, 6))
    capped = lib().ora_gl_stm_propagate(C.byref(s), int(stages), _dp(x0), float(t0), float(tf), int(nsteps),
                                        _dp(xf), _dp(Phi))
    return xf, Phi, int(capped)


def bplane(mu: float, rel) -> tuple[np.ndarray, int]:
    """(B.T, B.R) of the planet-relative state rel = (r, v); rc 1 if not hyperbolic."""
    rel = np.ascontiguousarray(rel, dtype=np.float64).reshape(6)
    out = np.zeros(2)
    rc = lib().ora_bplane(float(mu), _dp(rel), _dp(out))
    return out, int(rc)


def pc2_segment(model: Model, opts: Opts, ta: float, tb: float, x0):
    """Second-order form of the sweep (velocities from the accelerations, then
    positions from the new velocities): (Y [n][6], sweeps, last change, outcome)."""
    s, o = model.struct(), opts.struct()
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    Y = np.zeros((opts.N + 1, 6))
    it = C.c_int(0)
    err = C.c_double(0.0)
    outcome = lib().ora_pc2_segment(C.byref(s), C.byref(o), float(ta), float(tb), _dp(x0), _dp(Y), C.byref(it),
                                    C.byref(err))
    return Y, int(it.value), float(err.value), int(outcome)
