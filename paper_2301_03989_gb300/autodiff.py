"""torch.autograd wrappers of the propagator and the b-plane.

Both directions run in the library's kernels: the forward pass is
pc_propagate_tape (which keeps every accepted segment's converged nodes), the
backward pass pc_adjoint_tape (the reverse sweep through those segments); the
b-plane's value and vector-Jacobian product come from pc_bplane.  The tensors
here only carry device memory between the two calls.
"""
from __future__ import annotations

import torch

from . import pcprop


class _Propagate(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x0, plan, t0, tf, segments, tol, max_seg):
        x0 = x0.detach().contiguous()
        M = int(x0.shape[1])
        rec = pcprop.tape_record(plan)
        cap = max(1, int(max_seg))
        for _ in range(2):
            tape = torch.empty(M * cap * rec, dtype=torch.float64, device=x0.device)
            xf = torch.empty_like(x0)
            nseg = torch.zeros(M, dtype=torch.int32, device=x0.device)
            status = torch.zeros(M, dtype=torch.int32, device=x0.device)
            pcprop.propagate_tape(plan, x0, t0, tf, xf, nseg, tape, cap, segments=segments, tol=tol, status=status)
            top = int(nseg.max().item()) if M else 0
            if top <= cap:
                break
            cap = top                      # room for every segment, then once more
        ctx.save_for_backward(nseg, tape)
        ctx.plan, ctx.cap, ctx.tol = plan, cap, tol
        ctx.mark_non_differentiable(status, nseg)
        return xf, status, nseg

    @staticmethod
    def backward(ctx, xf_bar, _s, _n):
        nseg, tape = ctx.saved_tensors
        xf_bar = xf_bar.contiguous()
        x0_bar = torch.empty_like(xf_bar)
        pcprop.adjoint_tape(ctx.plan, nseg, ctx.cap, tape, xf_bar, x0_bar, tol=ctx.tol)
        return x0_bar, None, None, None, None, None, None


def propagate(x0: torch.Tensor, plan: pcprop.Plan, t0: torch.Tensor, tf: torch.Tensor, segments=None,
              tol: float = 0.0, max_seg: int = 64):
    """Differentiable propagation.  x0: planar [6][M] float64 CUDA tensor;
    t0, tf: [M] float64 arcs; segments: [M] int32 or None.  Returns
    (xf [6][M], status [M], nseg [M]); gradients flow to x0 through the
    converged segments (schedule held fixed)."""
    return _Propagate.apply(x0, plan, t0, tf, segments, tol, max_seg)


class _BPlane(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, plan, body, mu_body, t):
        x = x.detach().contiguous()
        out = torch.empty((2, x.shape[1]), dtype=torch.float64, device=x.device)
        pcprop.bplane(plan, body, mu_body, t, x, out=out)
        ctx.save_for_backward(x, t)
        ctx.plan, ctx.body, ctx.mu = plan, body, mu_body
        return out

    @staticmethod
    def backward(ctx, out_bar):
        x, t = ctx.saved_tensors
        x_bar = torch.empty_like(x)
        pcprop.bplane(ctx.plan, ctx.body, ctx.mu, t, x, out_bar=out_bar.contiguous(), x_bar=x_bar)
        return x_bar, None, None, None, None


def bplane(x: torch.Tensor, plan: pcprop.Plan, body: int, mu_body: float, t: torch.Tensor) -> torch.Tensor:
    """Differentiable b-plane (B.T, B.R), planar [2][M], of heliocentric states
    x (planar [6][M]) relative to body `body` of the plan's ephemeris at t [M]."""
    return _BPlane.apply(x, plan, body, mu_body, t)
