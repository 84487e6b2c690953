"""Uneven batching (pc_propagate_groups): per-trajectory arcs, segment counts
and Chebyshev degrees in one call, grouped by degree, against the oracle run
trajectory by trajectory with the same arc, degree and segment count."""
import numpy as np
import pytest

from paper_2301_03989_gb300 import workloads as W
from test_gpu_parity import TOL, pmap, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pc():
    import torch
    from paper_2301_03989_gb300 import build, pcprop
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return pcprop


def _plans(pc, w, degs, **opts):
    b = w.base
    out = []
    for d in degs:
        o = pc.options_default(tol=b.tol, max_iters=b.max_iters, max_depth=b.max_depth, seg_mode=0)
        for k, v in opts.items():
            setattr(o, k, v)
        out.append(pc.plan_create(d, 4, b.mu_central, b.mu, b.t_begin, b.granule, b.coef, b.indirect, o))
    return out


def run_groups(pc, w, tf=None, **opts):
    import torch
    perm, degs, counts = w.groups()
    plans = _plans(pc, w, degs, **opts)
    tfv = (w.tf if tf is None else tf)[perm]
    dev = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    x0 = dev(W.to_planar(w.x0[perm]))
    xf = torch.zeros_like(x0)
    st = torch.zeros(w.n_ic, dtype=torch.int32, device="cuda")
    it = torch.zeros_like(st)
    ns = torch.zeros_like(st)
    code, rounds = pc.propagate_groups(plans, counts, x0, dev(w.t0[perm]), dev(tfv), xf,
                                       segments=dev(w.S[perm], torch.int32), status=st, iters=it, nseg=ns)
    torch.cuda.synchronize()
    for p in plans:
        p.close()
    inv = np.argsort(perm)
    return dict(code=code, xf=W.from_planar(xf.cpu().numpy())[inv], status=st.cpu().numpy()[inv],
                iters=it.cpu().numpy()[inv], nseg=ns.cpu().numpy()[inv])


def run_oracle_each(ora, w, tf=None):
    """The oracle per trajectory (its own arc, degree and segment count), over
    the host's cores."""
    m = ora.Model.from_workload(w.base)
    b = w.base
    tfv = w.tf if tf is None else tf

    def one(i):
        o = ora.Opts(N=int(w.N[i]), segments=int(w.S[i]), seg_mode=0, tol=b.tol, max_iters=b.max_iters,
                     max_depth=b.max_depth)
        r = ora.propagate(m, o, w.x0[i:i + 1], float(w.t0[i]), float(tfv[i]))
        return r["xf"][0], r["status"][0], r["nseg"][0]
    res = pmap(one, range(w.n_ic))
    return dict(xf=np.array([r[0] for r in res]), status=np.array([r[1] for r in res], dtype=np.int32),
                nseg=np.array([r[2] for r in res], dtype=np.int32))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_uneven_groups_vs_oracle(pc, ora, precision):
    """256 trajectories of the uneven workload: arcs of 0.5-10 years, all four
    degrees (32, 64, 128, 256), 4-80 base segments each."""
    w = W.config5(M=256)
    assert set(int(n) for n in w.N) == {32, 64, 128, 256}
    assert w.tf.max() - w.t0.min() > 9 * W.YEAR and (w.tf - w.t0).min() < W.YEAR
    prec = pc.PC_PREC_MIXED if precision == "mixed" else pc.PC_PREC_FP64
    g = run_groups(pc, w, precision=prec)
    o = run_oracle_each(ora, w)
    assert g["code"] == pc.PC_OK
    np.testing.assert_array_equal(g["status"], o["status"])
    er, ev = rel_err(g["xf"], o["xf"])
    for d in (32, 64, 128, 256):
        k = w.N == d
        print(f"config 5 {precision}, N = {d}: {int(k.sum())} trajectories, error vs oracle position max "
              f"{er[k].max():.2e}, velocity max {ev[k].max():.2e}")
    assert er.max() < TOL and ev.max() < TOL, (er.max(), ev.max())
    assert (g["nseg"] != o["nseg"]).mean() <= 1 / 16


def test_uneven_out_of_table_and_backward(pc, ora):
    w = W.config5(M=40, years_max=2.0)
    tf = w.tf.copy()
    tf[3] = 50 * W.YEAR                     # beyond the ephemeris table
    g = run_groups(pc, w, tf=tf)
    assert g["code"] == pc.PC_ENOTCONV
    assert g["status"][3] == pc.PC_IC_OUT_OF_RANGE
    np.testing.assert_array_equal(g["xf"][3], w.x0[3])
    ok = np.arange(w.n_ic) != 3
    o = run_oracle_each(ora, w)
    er, ev = rel_err(g["xf"][ok], o["xf"][ok])
    assert er.max() < TOL and ev.max() < TOL
    # backward arcs: start at the forward end states and return
    wb = W.config5(M=16, years_max=1.0)
    fwd = run_oracle_each(ora, wb)
    back = W.UnevenWorkload(wb.name, wb.base, fwd["xf"], wb.tf.copy(), wb.t0.copy(), wb.N, wb.S)
    g = run_groups(pc, back)
    er, ev = rel_err(g["xf"], wb.x0)
    assert er.max() < 1e-11 and ev.max() < 1e-11
