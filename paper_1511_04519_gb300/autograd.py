"""torch.autograd.Function over the C ABI: node voltages at the output rows as
a function of the node capacitances and the source amplitude scales.

Forward: matex_set_caps / matex_set_sources, then matex_run (the batched
R-MATEX transient).  Backward: matex_grad, the hand-written discrete adjoint
of that run (same factors, Krylov dimensions as the forward chose).  Every
numeric step runs in the CUDA library; this module only moves arguments.
"""
from __future__ import annotations

import numpy as np
import torch

from . import matex as M


class IRDrop(torch.autograd.Function):
    """X = IRDrop.apply(c, amp, sim): voltages [N+1][n_rows] of ``sim`` (a
    ``matex.Sim`` built with ``tape=True``) for capacitances c [n] and
    per-source amplitude scales amp [n_src] (both float64; the currents of
    source s are amp_s times those given at setup)."""

    @staticmethod
    def forward(ctx, c, amp, sim):
        cn = c.detach().cpu().numpy().astype(np.float64)
        if getattr(sim, "_caps", None) is None or not np.array_equal(sim._caps, cn):
            sim.set_caps(cn)
            sim._caps = cn
        an = amp.detach().cpu().numpy().astype(np.float64)
        sim.set_sources(sim.base_pwl_v * an[sim.pwl_source])
        X = sim.run()
        ctx.sim = sim
        ctx.devices = (c.device, amp.device)
        return X

    @staticmethod
    def backward(ctx, xbar):
        dc, da = ctx.sim.grad(xbar)
        return dc.to(ctx.devices[0]), da.to(ctx.devices[1]), None


def hinge_ir_drop_loss(X, vdd, theta, dt):
    """sum over rows of the trapezoid integral of max(0, Vdd - v - theta)^2."""
    w = torch.full((X.shape[0],), dt, dtype=X.dtype, device=X.device)
    w[0] = w[-1] = dt / 2
    a = torch.clamp(vdd - X - theta, min=0.0)
    return (w[:, None] * a * a).sum()


def make_sim(p, rows, tape=True, **kw):
    """A Sim that keeps what ``IRDrop``'s backward needs (tape: True or
    "full" for the full tape, "checkpoint" for checkpoints recomputed per
    window), with the problem's base currents."""
    sim = M.Sim(p, rows=rows, tape=tape, **kw)
    sim.base_pwl_v = np.asarray(p.pwl_v, dtype=np.float64).copy()
    sim.pwl_source = np.repeat(np.arange(p.n_src), np.diff(np.asarray(p.pwl_off)))
    sim._caps = np.asarray(p.c, dtype=np.float64).copy()
    return sim
