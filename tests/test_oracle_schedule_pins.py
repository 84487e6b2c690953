"""Pins of the oracle's control rules: the stop rule of a segment attempt and
the segment schedule (halve on failure, grow back one level after success,
clip at tf, forward and backward arcs).

The paper stops a segment on the sweep-to-sweep change (Section "Matrix
form", stopping criterion) and integrates piecewise, segment after segment,
forward or backward; the cap, the stall acceptance and the halving schedule
are this restatement's readings.  Every expected outcome below is written out
by hand from those readings -- none is produced by running the oracle -- so a
wrong comparison, a counter that is not reset, a schedule that never grows
back or a last segment clipped at the wrong place fails here even though the
end state of a propagation would still be right.  No GPU is needed.
"""
import numpy as np
import pytest

SEG_OK, SEG_STALLED, SEG_FAIL_CAP, SEG_FAIL_DIV, SEG_FAIL_TRUNC = 0, 1, 2, 3, 4


# ---------------------------------------------------------------- stop rule
def _opts(ora, **kw):
    base = dict(tol=1e-13, stall_sweeps=5, stall_factor=1e3, div_limit=1e3, max_iters=60)
    base.update(kw)
    return ora.Opts(**base)


def test_stop_rule_tolerance_is_strict(ora):
    o = _opts(ora)
    assert ora.stop_rule(o, [1e-3, 1e-8, 9.99e-14]) == (SEG_OK, 3)
    # a change equal to tol is not below it: the attempt goes on
    assert ora.stop_rule(o, [1e-3, 1e-13]) == (-1, 2)
    assert ora.stop_rule(o, [1e-3, 1e-13, 5e-14]) == (SEG_OK, 3)


def test_stop_rule_stalls_at_the_fifth_non_improving_sweep(ora):
    """Best change 4e-11 at sweep 5 (below stall_factor * tol = 1e-10); sweeps
    6..10 do not go below it, so the fifth of them (sweep 10) stalls."""
    o = _opts(ora)
    seq = [1e-3, 1e-6, 1e-9, 5e-11, 4e-11, 6e-11, 5e-11, 4.5e-11, 7e-11, 4.2e-11, 1e-14]
    assert ora.stop_rule(o, seq) == (SEG_STALLED, 10)
    # one more improving sweep in between resets the count: sweep 7 improves
    # (3e-11 < 4e-11), so the five non-improving sweeps are 8..12
    seq2 = [1e-3, 1e-6, 1e-9, 5e-11, 4e-11, 6e-11, 3e-11, 4e-11, 5e-11, 3.5e-11, 3.1e-11, 3e-11, 1e-14]
    assert ora.stop_rule(o, seq2) == (SEG_STALLED, 12)


def test_stop_rule_equal_change_counts_as_no_improvement(ora):
    o = _opts(ora)
    seq = [1e-3, 2e-11, 2e-11, 2e-11, 2e-11, 2e-11, 2e-11]
    assert ora.stop_rule(o, seq) == (SEG_STALLED, 7)


def test_stop_rule_no_stall_above_stall_factor_times_tol(ora):
    """A best change of 2e-10 is above 1e3 * 1e-13: no stall however long the
    plateau; the attempt runs to the cap."""
    o = _opts(ora, max_iters=12)
    seq = [1e-3, 1e-6, 2e-10] + [3e-10] * 20
    assert ora.stop_rule(o, seq) == (SEG_FAIL_CAP, 12)
    # with a larger factor the same plateau stalls after five sweeps (sweep 8)
    assert ora.stop_rule(_opts(ora, max_iters=12, stall_factor=1e4), seq) == (SEG_STALLED, 8)


def test_stop_rule_stall_count_follows_the_option(ora):
    seq = [1e-3, 2e-11] + [3e-11] * 10
    assert ora.stop_rule(_opts(ora, stall_sweeps=3), seq) == (SEG_STALLED, 5)
    assert ora.stop_rule(_opts(ora, stall_sweeps=8), seq) == (SEG_STALLED, 10)


def test_stop_rule_blow_up_and_nan(ora):
    o = _opts(ora)
    assert ora.stop_rule(o, [1e-3, 5e2, 1.5e3]) == (SEG_FAIL_DIV, 3)
    assert ora.stop_rule(o, [1e-3, float("nan")]) == (SEG_FAIL_DIV, 2)
    assert ora.stop_rule(o, [float("inf")]) == (SEG_FAIL_DIV, 1)
    # exactly div_limit is still finite enough to go on
    assert ora.stop_rule(o, [1e3]) == (-1, 1)


def test_stop_rule_cap_counts_sweeps(ora):
    o = _opts(ora, max_iters=4)
    assert ora.stop_rule(o, [1e-1, 1e-2, 1e-3, 1e-4, 1e-5]) == (SEG_FAIL_CAP, 4)
    # a converging last sweep wins over the cap
    assert ora.stop_rule(o, [1e-1, 1e-2, 1e-3, 1e-14]) == (SEG_OK, 4)


def test_stop_rule_is_what_a_segment_uses(ora):
    """The segment iteration ends where the rule says: at the cap for a
    cold start that needs more sweeps, on a blow-up for a segment far too long
    for Picard iteration, and with the change below tol otherwise."""
    m = ora.Model(mu_central=1.0, mu=np.zeros(0))
    om = 1e-3
    x0 = np.array([1.0, 0.3, -0.2, 0.0, 2e-4, 1e-4])
    base = dict(N=24, dyn=ora.DYN_HARMONIC, dyn_param=(om * om, 0, 0), trunc_tol=0.0)
    _, it, err, out = ora.pc_segment(m, ora.Opts(max_iters=60, **base), 0.0, 1000.0, x0)
    assert out == SEG_OK and err < 1e-13 and 3 < it < 60
    _, itc, _, outc = ora.pc_segment(m, ora.Opts(max_iters=it - 1, **base), 0.0, 1000.0, x0)
    assert (outc, itc) == (SEG_FAIL_CAP, it - 1)
    # z = w w2 = 40: the Picard iterates grow like z^k/k! before they shrink;
    # in absolute mode the change passes div_limit = 1e3 within a few sweeps
    _, itd, errd, outd = ora.pc_segment(m, ora.Opts(N=64, dyn=ora.DYN_HARMONIC, dyn_param=(om * om, 0, 0),
                                                    trunc_tol=0.0, relative=False), 0.0, 80000.0, x0)
    assert outd == SEG_FAIL_DIV and not (errd <= 1e3)


# ---------------------------------------------------------------- segment schedule
# A harmonic oscillator x'' = -w^2 x at degree N = 16 under the resolution
# test (trunc_tol 1e-13): the tail estimate of a segment of half-length w2 is
# about 4 z J_15(z), z = w w2 (Bessel coefficients of cos).  With w T = 8:
# z = 4 (whole arc) and z = 2 (half arc, 4 * 2 * 7.6e-13 ~ 6e-12) fail it,
# z = 1 (quarter, ~1e-16) passes with a margin of three orders.  With w T = 16
# the quarter fails too and the eighth passes.
OM = 1e-3
X0 = np.array([1.0, 0.3, -0.2, 0.0, 2e-4, 1e-4])


def _ho_log(ora, wT, t0_frac, tf_frac, depth=4):
    T = wT / OM
    m = ora.Model(mu_central=1.0, mu=np.zeros(0))
    o = ora.Opts(N=16, segments=1, dyn=ora.DYN_HARMONIC, dyn_param=(OM * OM, 0, 0), max_depth=depth,
                 tol=1e-13, trunc_tol=1e-13)
    r = ora.propagate_log(m, o, X0, t0_frac * T, tf_frac * T)
    return r, T


def _check(r, T, expected):
    """expected: (t_a/T, t_b/T, accepted, depth) per attempt, in order;
    `accepted` is True/False (a failure is the resolution test's) or an
    explicit outcome code."""
    log = r["log"]
    assert r["n_attempts"] == len(expected), [tuple(np.round(x[:2] / T, 6)) for x in log]
    for k, (a, b, acc, d) in enumerate(expected):
        ta, tb, out, _, dep = log[k]
        assert abs(ta / T - a) < 1e-14 and abs(tb / T - b) < 1e-14, (k, ta / T, tb / T, a, b)
        want = acc if not isinstance(acc, bool) else (SEG_OK if acc else SEG_FAIL_TRUNC)
        assert int(out) == want, (k, int(out), want)
        assert int(dep) == d, (k, int(dep), d)


def test_schedule_halve_accept_grow_clip_forward(ora):
    r, T = _ho_log(ora, 8.0, 0.0, 1.0)
    _check(r, T, [
        (0.00, 1.00, False, 0),
        (0.00, 0.50, False, 1),
        (0.00, 0.25, True, 2),
        (0.25, 0.75, False, 1),   # grown back one level after the success
        (0.25, 0.50, True, 2),
        (0.50, 1.00, False, 1),
        (0.50, 0.75, True, 2),
        (0.75, 1.00, True, 1),    # a depth-1 segment [0.75, 1.25] clipped at tf
    ])
    assert r["nseg"] == 4 and r["status"] == 0


def test_schedule_backward_arc(ora):
    r, T = _ho_log(ora, 8.0, 1.0, 0.0)
    _check(r, T, [
        (1.00, 0.00, False, 0),
        (1.00, 0.50, False, 1),
        (1.00, 0.75, True, 2),
        (0.75, 0.25, False, 1),
        (0.75, 0.50, True, 2),
        (0.50, 0.00, False, 1),
        (0.50, 0.25, True, 2),
        (0.25, 0.00, True, 1),
    ])
    assert r["nseg"] == 4


def test_schedule_grows_one_level_at_a_time(ora):
    """Threshold between T/8 and T/4: after a success at depth 3 the next
    attempt is at depth 2 (not 0), fails, and the depth-3 half is accepted."""
    r, T = _ho_log(ora, 16.0, 0.0, 1.0)
    # the whole arc (z = 8) does not even converge within the 60-sweep cap
    exp = [(0.0, 1.0, SEG_FAIL_CAP, 0), (0.0, 0.5, False, 1), (0.0, 0.25, False, 2), (0.0, 0.125, True, 3)]
    for k in range(1, 7):
        a = 0.125 * k
        exp += [(a, min(a + 0.25, 1.0), False, 2), (a, a + 0.125, True, 3)]
    exp += [(0.875, 1.0, True, 2)]          # [0.875, 1.125] clipped at tf
    _check(r, T, exp)
    assert r["nseg"] == 8


def test_schedule_depth_limit_accepts_unresolved(ora):
    """With max_depth 1 the half-arc segments still fail the resolution test:
    at the deepest level they are accepted and flagged unresolved (status 2)."""
    r, T = _ho_log(ora, 8.0, 0.0, 1.0, depth=1)
    log = r["log"]
    assert [(round(x[0] / T, 6), round(x[1] / T, 6), int(x[4])) for x in log] == [
        (0.0, 1.0, 0), (0.0, 0.5, 1), (0.5, 1.0, 0), (0.5, 1.0, 1)]
    assert [int(x[2]) for x in log] == [SEG_FAIL_TRUNC] * 4
    assert r["nseg"] == 2 and r["status"] == 2


def test_schedule_uniform_and_per_period_with_clip(ora):
    """No failure: `segments` equal pieces at depth 0.  Per osculating period
    (seg_mode 1): base = P/8 of the starting two-body orbit, an arc of 1.3 P
    gives ten full segments and an eleventh [1.25 P, 1.3 P] clipped at tf."""
    mu = 1.0
    m = ora.Model(mu_central=mu, mu=np.zeros(0))
    x0 = np.array([1.0, 0.0, 0.0, 0.0, 1.05, 0.0])       # e = 0.1025, a = 1/(2 - 1.1025)
    a = 1.0 / (2.0 - 1.05 ** 2)
    P = 2 * np.pi * np.sqrt(a ** 3 / mu)
    o = ora.Opts(N=32, segments=5, seg_mode=0, tol=1e-13)
    r = ora.propagate_log(m, o, x0, 0.0, 0.5 * P)
    assert r["n_attempts"] == 5 and r["nseg"] == 5
    for k, row in enumerate(r["log"]):
        assert abs(row[0] - 0.1 * P * k) < 1e-12 * P and abs(row[1] - 0.1 * P * (k + 1)) < 1e-12 * P
        assert int(row[4]) == 0 and int(row[2]) == SEG_OK
    o1 = ora.Opts(N=32, segments=8, seg_mode=1, tol=1e-13)
    r = ora.propagate_log(m, o1, x0, 0.0, 1.3 * P)
    assert r["n_attempts"] == 11 and r["nseg"] == 11
    for k, row in enumerate(r["log"]):
        assert abs(row[0] - P / 8 * k) < 1e-12 * P
        end = min(P / 8 * (k + 1), 1.3 * P)
        assert abs(row[1] - end) < 1e-12 * P, (k, row[1] / P)
    assert r["log"][-1][1] == 1.3 * P                         # the last segment ends exactly at tf
