"""Uneven batching (pc_propagate_groups): per-trajectory arcs, segment counts
and Chebyshev degrees in one call, grouped by degree, against the oracle run
trajectory by trajectory with the same arc, degree and segment count."""
import numpy as np
import pytest

from paper_2301_03989_gb300 import workloads as W
from test_gpu_parity import TOL, rel_err

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
    m = ora.Model.from_workload(w.base)
    b = w.base
    tfv = w.tf if tf is None else tf
    xf = np.zeros_like(w.x0)
    st = np.zeros(w.n_ic, dtype=np.int32)
    ns = np.zeros(w.n_ic, dtype=np.int32)
    for i in range(w.n_ic):
        o = ora.Opts(N=int(w.N[i]), segments=int(w.S[i]), seg_mode=0, tol=b.tol, max_iters=b.max_iters,
                     max_depth=b.max_depth)
        r = ora.propagate(m, o, w.x0[i:i + 1], float(w.t0[i]), float(tfv[i]))
        xf[i], st[i], ns[i] = r["xf"][0], r["status"][0], r["nseg"][0]
    return dict(xf=xf, status=st, nseg=ns)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_uneven_groups_vs_oracle(pc, ora, precision):
    w = W.config5(M=48, years_max=3.0)
    prec = pc.PC_PREC_MIXED if precision == "mixed" else pc.PC_PREC_FP64
    g = run_groups(pc, w, precision=prec)
    o = run_oracle_each(ora, w)
    assert g["code"] == pc.PC_OK
    np.testing.assert_array_equal(g["status"], o["status"])
    er, ev = rel_err(g["xf"], o["xf"])
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
