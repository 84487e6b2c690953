"""Einstein-Infeld-Hoffmann (1PN) force on the GPU (pc_force_model.c_light > 0)
against the oracle's EIH model: kernel-level dynamics (the relativistic part
to 1e-9 of itself), and whole propagations within 1e-10 relative (FP64 and mixed
precision, whose FP32 sweeps keep the Newtonian terms while the FP64 sweeps
and their residual carry the relativistic ones)."""
import numpy as np
import pytest

from paper_2301_03989_gb300 import workloads as W
from test_gpu_parity import TOL, rel_err, run_oracle

pytestmark = pytest.mark.gpu
C_LIGHT = 299792.458


@pytest.fixture(scope="module")
def pc():
    import torch
    from paper_2301_03989_gb300 import build, pcprop
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return pcprop


def _dev(a, dtype=None):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype or torch.float64, device="cuda")


def run_gpu_eih(pc, w, x0, t0=None, tf=None, max_ckpt=0, **opts):
    import torch
    plan = pc.plan_from_workload(w, c_light=C_LIGHT, **opts)
    M = x0.shape[0]
    xd = _dev(W.to_planar(x0))
    xf = torch.zeros_like(xd)
    st = torch.zeros(M, dtype=torch.int32, device="cuda")
    it = torch.zeros(M, dtype=torch.int32, device="cuda")
    ns = torch.zeros(M, dtype=torch.int32, device="cuda")
    ck = torch.zeros((M, max(max_ckpt, 1), 7), dtype=torch.float64, device="cuda") if max_ckpt else None
    code, _ = pc.propagate(plan, xd, w.t0 if t0 is None else t0, w.tf if tf is None else tf, xf, status=st,
                           iters=it, nseg=ns, ckpt=ck, max_ckpt=max_ckpt)
    torch.cuda.synchronize()
    out = dict(code=code, xf=W.from_planar(xf.cpu().numpy()), status=st.cpu().numpy(), iters=it.cpu().numpy(),
               nseg=ns.cpu().numpy())
    if ck is not None:
        out["ckpt"] = ck.cpu().numpy()
    plan.close()
    return out


def run_oracle_eih(ora, w, x0, tf=None, threads=8, **opts):
    m = ora.Model.from_workload(w, c_light=C_LIGHT)
    kw = dict(N=w.N, segments=w.segments, seg_mode=w.seg_mode, tol=w.tol, max_iters=w.max_iters,
              max_depth=w.max_depth)
    kw.update(opts)
    return ora.propagate(m, ora.Opts(**kw), x0, w.t0, w.tf if tf is None else tf, threads=threads)


def test_eih_dynamics_vs_oracle(pc, ora):
    """States near and far from the bodies at random times: the GPU's EIH
    acceleration minus its Newtonian one equals the oracle's relativistic
    terms to 1e-9 of their size (plus the Newtonian parts' rounding)."""
    import torch
    w = W.config2(M=8)
    rng = np.random.default_rng(9)
    n = 301
    mN, mE = ora.Model.from_workload(w), ora.Model.from_workload(w, c_light=C_LIGHT)
    t = rng.uniform(w.t0, w.tf, n)
    y = np.zeros((6, n))
    for i in range(n):
        rb = ora.ephem_eval(mN, t[i])
        d = rng.standard_normal(3)
        y[:3, i] = rb[1] + d / np.linalg.norm(d) * rng.uniform(1e4, 1e6) if i % 4 == 0 else rng.standard_normal(3) * 1.5e8
        y[3:, i] = rng.standard_normal(3) * 30.0
    out = {}
    for name, cl in (("newton", 0.0), ("eih", C_LIGHT)):
        plan = pc.plan_from_workload(w, c_light=cl)
        f = torch.zeros((6, n), dtype=torch.float64, device="cuda")
        pc.eval_dynamics(plan, _dev(t), _dev(y), f)
        torch.cuda.synchronize()
        out[name] = f.cpu().numpy()
        plan.close()
    o = ora.Opts()
    for i in range(n):
        rel_ora = ora.eih_at(mE, t[i], y[:, i])
        rel_gpu = out["eih"][3:, i] - out["newton"][3:, i]
        nrm = np.abs(rel_ora).max()
        a = np.abs(ora.dynamics(mN, o, t[i], y[:, i])[3:]).max()
        # (the Newtonian parts of both accelerations are checked against the
        # oracle, to their rounding bound, by the kernel-level dynamics test)
        assert np.abs(rel_gpu - rel_ora).max() <= 1e-9 * nrm + 4e-16 * a, (i, rel_gpu, rel_ora)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_eih_config1_vs_oracle(pc, ora, precision):
    w = W.config1()
    prec = pc.PC_PREC_MIXED if precision == "mixed" else pc.PC_PREC_FP64
    g = run_gpu_eih(pc, w, w.x0, precision=prec)
    o = run_oracle_eih(ora, w, w.x0)
    assert g["code"] == pc.PC_OK
    er, ev = rel_err(g["xf"], o["xf"])
    assert er.max() < TOL and ev.max() < TOL, (er.max(), ev.max())
    np.testing.assert_array_equal(g["nseg"], o["nseg"])
    # the relativistic terms move the end state far beyond the tolerance
    newt = run_oracle(ora, w, w.x0)
    er2, _ = rel_err(o["xf"], newt["xf"])
    assert er2.min() > 100 * TOL, er2.min()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_eih_config2_short_arc_and_config3(pc, ora, precision):
    prec = pc.PC_PREC_MIXED if precision == "mixed" else pc.PC_PREC_FP64
    w = W.config2(M=32)
    tf = 20 * W.DAY
    g = run_gpu_eih(pc, w, w.x0, tf=tf, precision=prec)
    o = run_oracle_eih(ora, w, w.x0, tf=tf)
    er, ev = rel_err(g["xf"], o["xf"])
    assert er.max() < TOL and ev.max() < TOL, (er.max(), ev.max())
    w3 = W.config3(M=128)
    g = run_gpu_eih(pc, w3, w3.x0, precision=prec, switch_tol=1e-6 if precision == "mixed" else 0.0, order=2)
    o = run_oracle_eih(ora, w3, w3.x0, order=2)
    assert g["code"] == pc.PC_OK
    er, ev = rel_err(g["xf"], o["xf"])
    print(f"config 3 EIH {precision} order 2: error vs oracle position {er.max():.2e} velocity {ev.max():.2e}")
    assert er.max() < TOL and ev.max() < TOL, (er.max(), ev.max())


def test_eih_refused_by_reverse_mode(pc):
    import torch
    w = W.config4(M=4)
    plan = pc.plan_from_workload(w, c_light=C_LIGHT)
    M = w.n_ic
    tape = torch.zeros(M * 8 * pc.tape_record(plan), dtype=torch.float64, device="cuda")
    xf = torch.zeros((6, M), dtype=torch.float64, device="cuda")
    ns = torch.zeros(M, dtype=torch.int32, device="cuda")
    with pytest.raises(pc.PCError) as e:
        pc.propagate_tape(plan, _dev(W.to_planar(w.x0)), _dev(np.full(M, w.t0)), _dev(np.full(M, w.tf)), xf, ns,
                          tape, 8)
    assert e.value.code == pc.PC_EINVAL
    plan.close()
