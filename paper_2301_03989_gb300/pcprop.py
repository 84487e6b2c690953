"""Thin Python binding of the C ABI in include/pc.h (ctypes; argument
marshalling only -- every step of the propagation runs in the CUDA library).

Device buffers are torch CUDA tensors (float64 / int32, contiguous) or raw
device pointers (int).  There is no CPU fallback: if the compiled library is
missing, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpcprop.so")
_lock = threading.Lock()
_lib = None

PC_OK, PC_EINVAL, PC_ENOMEM, PC_ECUDA, PC_ENOTCONV, PC_ENONFINITE = 0, 1, 2, 3, 4, 5
PC_IC_STALLED, PC_IC_UNRESOLVED, PC_IC_NOT_CONVERGED, PC_IC_NONFINITE, PC_IC_OUT_OF_RANGE = 1, 2, 4, 8, 16
PC_PREC_FP64, PC_PREC_MIXED = 0, 1
PC_CONTRACT_DMMA, PC_CONTRACT_SPLIT = 0, 1

EXPORTS = ["pc_options_default", "pc_plan_create", "pc_propagate", "pc_propagate_ex", "pc_eval_ephemeris",
           "pc_eval_dynamics", "pc_eval_warm_start", "pc_apply_operator", "pc_plan_operator", "pc_plan_destroy",
           "pc_status_string", "pc_plan_set_profiling", "pc_plan_kernel_times", "pc_apply_operator_static",
           "pc_propagate_groups", "pc_propagate_tape", "pc_adjoint_tape", "pc_propagate_adjoint", "pc_bplane",
           "pc_plan_get_tuning", "pc_plan_set_tuning", "pc_plan_autotune"]
KERNEL_NAMES = ["setup", "fp32", "force", "contract", "control"]


class PCError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {status_string(code)} (status {code})")
        self.code = code


class ForceModel(C.Structure):
    _fields_ = [("n_bodies", C.c_int), ("mu_central", C.c_double), ("mu", C.POINTER(C.c_double)),
                ("indirect", C.c_int), ("c_light", C.c_double)]


class Ephemeris(C.Structure):
    _fields_ = [("n_bodies", C.c_int), ("t_begin", C.c_double), ("granule_s", C.c_double), ("degree", C.c_int),
                ("n_granules", C.c_int), ("coef", C.POINTER(C.c_double))]


class KernelTimes(C.Structure):
    _fields_ = [("launches", C.c_longlong * 5), ("ms", C.c_double * 5), ("sweeps64", C.c_longlong),
                ("sweeps32", C.c_longlong), ("kernel_launches", C.c_longlong)]


class Tuning(C.Structure):
    _fields_ = [("setup_ctas_per_sm", C.c_int), ("fp32_ctas_per_sm", C.c_int), ("contract_ctas_per_sm", C.c_int),
                ("rounds_per_batch", C.c_int), ("repack_div", C.c_int), ("graphs", C.c_int),
                ("side_priority", C.c_int), ("fp32_rows", C.c_int), ("fp32_slots", C.c_int),
                ("grid_cache", C.c_int)]

    def as_dict(self) -> dict:
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class Options(C.Structure):
    _fields_ = [("tol", C.c_double), ("relative", C.c_int), ("max_iters", C.c_int), ("max_depth", C.c_int),
                ("warm_start", C.c_int), ("seg_mode", C.c_int), ("truncated", C.c_int), ("stall_sweeps", C.c_int),
                ("stall_factor", C.c_double), ("div_limit", C.c_double), ("trunc_tol", C.c_double),
                ("precision", C.c_int), ("switch_tol", C.c_double), ("max_rounds", C.c_longlong),
                ("refine32", C.c_int), ("contraction", C.c_int), ("order", C.c_int), ("fp32_mma", C.c_int)]


def lib():
    """Loads libpcprop.so (raises if it has not been built: no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"CUDA library not built: {LIB_PATH} (run paper_2301_03989_gb300.build)")
            L = C.CDLL(LIB_PATH)
            vp, ll, d, i = C.c_void_p, C.c_longlong, C.c_double, C.c_int
            L.pc_options_default.argtypes = [C.POINTER(Options)]
            L.pc_plan_create.argtypes = [i, i, C.POINTER(ForceModel), C.POINTER(Ephemeris), C.POINTER(Options),
                                         C.POINTER(vp)]
            L.pc_propagate.argtypes = [vp, ll, vp, d, d, d, vp, vp, vp, vp]
            L.pc_propagate_ex.argtypes = [vp, ll, vp, d, d, d, vp, vp, vp, vp, i, vp, C.POINTER(ll), vp]
            L.pc_eval_ephemeris.argtypes = [vp, ll, vp, vp, vp]
            L.pc_eval_dynamics.argtypes = [vp, ll, vp, vp, vp, vp]
            L.pc_eval_warm_start.argtypes = [vp, ll, vp, vp, vp, vp]
            L.pc_apply_operator.argtypes = [vp, ll, vp, vp, vp, vp]
            L.pc_apply_operator_static.argtypes = [vp, ll, vp, vp, vp, vp]
            L.pc_propagate_groups.argtypes = [C.POINTER(vp), i, C.POINTER(ll), vp, vp, vp, vp, d, vp, vp, vp, vp,
                                              C.POINTER(ll), vp]
            L.pc_propagate_tape.argtypes = [vp, ll, vp, vp, vp, vp, d, vp, vp, vp, i, vp, vp]
            L.pc_adjoint_tape.argtypes = [vp, ll, vp, i, vp, vp, d, vp, vp, vp, vp]
            L.pc_propagate_adjoint.argtypes = [vp, ll, vp, d, d, d, vp, vp, vp]
            L.pc_bplane.argtypes = [vp, i, d, ll, vp, vp, vp, vp, vp, vp, vp]
            L.pc_plan_get_tuning.argtypes = [vp, C.POINTER(Tuning)]
            L.pc_plan_set_tuning.argtypes = [vp, C.POINTER(Tuning)]
            L.pc_plan_autotune.argtypes = [vp, ll, vp, d, d, i, C.POINTER(Tuning), vp]
            L.pc_plan_operator.argtypes = [vp, vp, vp]
            L.pc_plan_destroy.argtypes = [vp]
            L.pc_plan_destroy.restype = None
            L.pc_plan_set_profiling.argtypes = [vp, i]
            L.pc_plan_kernel_times.argtypes = [vp, C.POINTER(KernelTimes)]
            L.pc_status_string.argtypes = [i]
            L.pc_status_string.restype = C.c_char_p
            for name in EXPORTS:
                if name not in ("pc_plan_destroy", "pc_status_string"):
                    getattr(L, name).restype = i
            _lib = L
    return _lib


def status_string(code: int) -> str:
    return lib().pc_status_string(int(code)).decode()


def _check(code: int, where: str, ok=(PC_OK,)) -> int:
    if code not in ok:
        raise PCError(code, where)
    return code


def _ptr(x) -> int | None:
    """Device pointer of a torch tensor (checked contiguous) or an int; None -> NULL."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_cuda:
            raise ValueError("expected a CUDA tensor")
        if not x.is_contiguous():
            raise ValueError("expected a contiguous tensor")
        return int(x.data_ptr())
    raise TypeError(f"cannot take a device pointer of {type(x)}")


def _stream(stream):
    if stream is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def options_default(**overrides) -> Options:
    o = Options()
    _check(lib().pc_options_default(C.byref(o)), "pc_options_default")
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


class Plan:
    """Owns a pc_plan handle (destroyed on close / garbage collection)."""

    def __init__(self, handle: int, N: int):
        self.handle = handle
        self.N = N

    def close(self):
        if self.handle:
            lib().pc_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def plan_create(N: int, segments: int, mu_central: float, mu, t_begin: float = 0.0, granule: float = 1.0,
                coef=None, indirect: bool = True, options: Options | None = None, c_light: float = 0.0) -> Plan:
    """c_light > 0 (km/s) adds the Einstein-Infeld-Hoffmann terms to the force."""
    mu = np.ascontiguousarray(np.asarray(mu, dtype=np.float64).reshape(-1))
    B = int(mu.size)
    fm = ForceModel(B, float(mu_central), mu.ctypes.data_as(C.POINTER(C.c_double)) if B else None, int(bool(indirect)),
                    float(c_light))
    eph_p = None
    if B:
        coef = np.ascontiguousarray(np.asarray(coef, dtype=np.float64))
        if coef.ndim != 4 or coef.shape[0] != B or coef.shape[2] != 3:
            raise ValueError("coef must be [n_bodies][n_granules][3][degree+1]")
        eph = Ephemeris(B, float(t_begin), float(granule), int(coef.shape[3] - 1), int(coef.shape[1]),
                        coef.ctypes.data_as(C.POINTER(C.c_double)))
        eph_p = C.byref(eph)
    h = C.c_void_p()
    _check(lib().pc_plan_create(int(N), int(segments), C.byref(fm), eph_p, C.byref(options) if options else None,
                                C.byref(h)), "pc_plan_create")
    return Plan(h.value, int(N))


def plan_from_workload(w, c_light: float = 0.0, **opts) -> Plan:
    o = options_default(tol=w.tol, max_iters=w.max_iters, max_depth=w.max_depth, seg_mode=w.seg_mode)
    for k, v in opts.items():
        setattr(o, k, v)
    return plan_create(w.N, w.segments, w.mu_central, w.mu, w.t_begin, w.granule, w.coef, w.indirect, o, c_light=c_light)


def propagate(plan: Plan, x0, t0: float, tf: float, xf, tol: float = 0.0, status=None, iters=None, stream=None,
              nseg=None, ckpt=None, max_ckpt: int = 0) -> tuple[int, int]:
    """x0, xf: planar [6][n_ic] float64 on the device.  Returns (pc_status,
    sweep rounds run).  PC_ENOTCONV is returned, not raised (see status[])."""
    n_ic = int(x0.shape[-1]) if hasattr(x0, "shape") else None
    if n_ic is None:
        raise ValueError("x0 must be a [6][n_ic] tensor")
    rounds = C.c_longlong(0)
    code = lib().pc_propagate_ex(plan.handle, n_ic, _ptr(x0), float(t0), float(tf), float(tol), _ptr(xf),
                                 _ptr(status), _ptr(iters), _ptr(nseg), int(max_ckpt), _ptr(ckpt),
                                 C.byref(rounds), _stream(stream))
    _check(code, "pc_propagate", ok=(PC_OK, PC_ENOTCONV))
    return code, int(rounds.value)


def propagate_groups(plans, counts, x0, t0, tf, xf, segments=None, tol: float = 0.0, status=None, iters=None,
                     nseg=None, stream=None) -> tuple[int, int]:
    """Uneven batch: group g (plans[g], counts[g] trajectories) occupies the
    next counts[g] columns of x0/xf (planar [6][n_total]) and entries of t0, tf,
    segments (int32), status, iters, nseg.  Returns (pc_status, total rounds)."""
    n = len(plans)
    hp = (C.c_void_p * n)(*[p.handle for p in plans])
    hc = (C.c_longlong * n)(*[int(c) for c in counts])
    rounds = C.c_longlong(0)
    code = lib().pc_propagate_groups(hp, n, hc, _ptr(x0), _ptr(t0), _ptr(tf), _ptr(segments), float(tol), _ptr(xf),
                                     _ptr(status), _ptr(iters), _ptr(nseg), C.byref(rounds), _stream(stream))
    _check(code, "pc_propagate_groups", ok=(PC_OK, PC_ENOTCONV))
    return code, int(rounds.value)


def tape_record(plan: Plan) -> int:
    """Doubles per tape record: (t_a, t_b) and the 6 components of the N+1 nodes."""
    return 2 + 6 * (plan.N + 1)


def propagate_tape(plan: Plan, x0, t0, tf, xf, nseg, tape, max_seg: int, segments=None, tol: float = 0.0,
                   status=None, stream=None) -> int:
    """Forward pass recording the adjoint tape (device [n_ic * max_seg * tape_record]).
    t0, tf: device [n_ic] arcs; nseg: device int32 [n_ic].  Returns the pc_status."""
    n_ic = int(x0.shape[-1])
    code = lib().pc_propagate_tape(plan.handle, n_ic, _ptr(x0), _ptr(t0), _ptr(tf), _ptr(segments), float(tol),
                                   _ptr(xf), _ptr(status), _ptr(nseg), int(max_seg), _ptr(tape), _stream(stream))
    _check(code, "pc_propagate_tape", ok=(PC_OK, PC_ENOTCONV))
    return code


def adjoint_tape(plan: Plan, nseg, max_seg: int, tape, xf_bar, x0_bar, tol: float = 0.0, status=None, iters=None,
                 stream=None) -> int:
    """Reverse sweep: x0_bar = (d xf / d x0)^T xf_bar (planar [6][n_ic])."""
    n_ic = int(xf_bar.shape[-1])
    code = lib().pc_adjoint_tape(plan.handle, n_ic, _ptr(nseg), int(max_seg), _ptr(tape), _ptr(xf_bar), float(tol),
                                 _ptr(x0_bar), _ptr(status), _ptr(iters), _stream(stream))
    _check(code, "pc_adjoint_tape", ok=(PC_OK, PC_ENOTCONV))
    return code


def propagate_adjoint(plan: Plan, x0, t0: float, tf: float, xf_bar, x0_bar, tol: float = 0.0, stream=None) -> int:
    n_ic = int(x0.shape[-1])
    code = lib().pc_propagate_adjoint(plan.handle, n_ic, _ptr(x0), float(t0), float(tf), float(tol), _ptr(xf_bar),
                                      _ptr(x0_bar), _stream(stream))
    _check(code, "pc_propagate_adjoint", ok=(PC_OK, PC_ENOTCONV))
    return code


def bplane(plan: Plan, body: int, mu_body: float, t, x, out=None, jac=None, out_bar=None, x_bar=None,
           stream=None) -> int:
    """b-plane (B.T, B.R) planar [2][n] of states x (planar [6][n]) at times t [n];
    jac planar [12][n]; x_bar = J^T out_bar."""
    n = int(x.shape[-1])
    code = lib().pc_bplane(plan.handle, int(body), float(mu_body), n, _ptr(t), _ptr(x), _ptr(out), _ptr(jac),
                           _ptr(out_bar), _ptr(x_bar), _stream(stream))
    _check(code, "pc_bplane", ok=(PC_OK, PC_ENONFINITE))
    return code


def get_tuning(plan: Plan) -> dict:
    t = Tuning()
    _check(lib().pc_plan_get_tuning(plan.handle, C.byref(t)), "pc_plan_get_tuning")
    return t.as_dict()


def set_tuning(plan: Plan, **fields) -> dict:
    """Changes the named launch-tuning fields (see pc.h); returns the new tuning."""
    t = Tuning()
    _check(lib().pc_plan_get_tuning(plan.handle, C.byref(t)), "pc_plan_get_tuning")
    for k, v in fields.items():
        if not hasattr(t, k):
            raise AttributeError(k)
        setattr(t, k, int(v))
    _check(lib().pc_plan_set_tuning(plan.handle, C.byref(t)), "pc_plan_set_tuning")
    return t.as_dict()


def autotune(plan: Plan, x0, t0: float, tf: float, max_rounds: int = 200, stream=None) -> dict:
    """Project autotuner (pc_plan_autotune): picks the plan's launch tuning by
    timing capped propagations of x0 (planar [6][n_ic]); returns the choice."""
    t = Tuning()
    _check(lib().pc_plan_autotune(plan.handle, int(x0.shape[-1]), _ptr(x0), float(t0), float(tf), int(max_rounds),
                                  C.byref(t), _stream(stream)), "pc_plan_autotune")
    return t.as_dict()


def eval_ephemeris(plan: Plan, t, rb, stream=None):
    _check(lib().pc_eval_ephemeris(plan.handle, int(t.numel()), _ptr(t), _ptr(rb), _stream(stream)),
           "pc_eval_ephemeris")


def eval_dynamics(plan: Plan, t, y, f, stream=None):
    _check(lib().pc_eval_dynamics(plan.handle, int(t.numel()), _ptr(t), _ptr(y), _ptr(f), _stream(stream)),
           "pc_eval_dynamics")


def eval_warm_start(plan: Plan, x0, dt, x, stream=None):
    _check(lib().pc_eval_warm_start(plan.handle, int(dt.numel()), _ptr(x0), _ptr(dt), _ptr(x), _stream(stream)),
           "pc_eval_warm_start")


def apply_operator(plan: Plan, x0, g, y, stream=None):
    _check(lib().pc_apply_operator(plan.handle, int(x0.shape[-1]), _ptr(x0), _ptr(g), _ptr(y), _stream(stream)),
           "pc_apply_operator")


def apply_operator_static(plan: Plan, x0, g, y, stream=None):
    """pc_apply_operator through the library's fixed device array (no allocation)."""
    _check(lib().pc_apply_operator_static(plan.handle, int(x0.shape[-1]), _ptr(x0), _ptr(g), _ptr(y),
                                          _stream(stream)), "pc_apply_operator_static")


def plan_operator(plan: Plan):
    n = plan.N + 1
    K = np.zeros((n, n))
    tau = np.zeros(n)
    _check(lib().pc_plan_operator(plan.handle, K.ctypes.data, tau.ctypes.data), "pc_plan_operator")
    return K, tau


def set_profiling(plan: Plan, on: bool = True):
    _check(lib().pc_plan_set_profiling(plan.handle, int(bool(on))), "pc_plan_set_profiling")


def kernel_times(plan: Plan) -> dict:
    """{kernel: (launch records, summed ms)} recorded since the last call, plus
    'sweeps64', 'sweeps32' (trajectory-sweeps per precision) and
    'kernel_launches' (device kernels launched)."""
    kt = KernelTimes()
    _check(lib().pc_plan_kernel_times(plan.handle, C.byref(kt)), "pc_plan_kernel_times")
    out = {name: (int(kt.launches[k]), float(kt.ms[k])) for k, name in enumerate(KERNEL_NAMES)}
    out["sweeps64"] = int(kt.sweeps64)
    out["sweeps32"] = int(kt.sweeps32)
    out["kernel_launches"] = int(kt.kernel_launches)
    return out
