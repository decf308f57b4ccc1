"""torch.autograd.Function over many leap-format steps.

Forward: `nsteps` calls of the C-ABI step (no intermediate storage).
Backward: the hand-written step adjoint (agcm_step_adjoint) in a binomial
checkpointing schedule (checkpoint.py) with a fixed number of stored states,
so multi-step gradients of a scalar diagnostic with respect to the initial
state cost O(snapshots) state copies of memory.
"""
from __future__ import annotations

import torch

from . import agcm
from .checkpoint import reverse_sweep

FIELDS = agcm.FIELDS


class AgcmSteps(torch.autograd.Function):
    """x_N = step^N(x_0) on a given grid/precision; differentiable in x_0."""

    @staticmethod
    def forward(ctx, state, nsteps, dt, snaps, U, V, Phi, pi):
        x0 = {"U": U.detach().contiguous(), "V": V.detach().contiguous(), "Phi": Phi.detach().contiguous(),
              "pi": pi.detach().contiguous()}
        state.load(x0)
        state.step(nsteps, dt)
        out = state.store()
        ctx.state, ctx.nsteps, ctx.dt, ctx.snaps = state, int(nsteps), float(dt), int(snaps)
        ctx.x0 = x0
        return out["U"], out["V"], out["Phi"], out["pi"]

    @staticmethod
    def backward(ctx, gU, gV, gPhi, gpi):
        s, dt = ctx.state, ctx.dt

        def zeros_like_or(g, ref):
            return torch.zeros_like(ref) if g is None else g.contiguous()

        lam = {"U": zeros_like_or(gU, ctx.x0["U"]), "V": zeros_like_or(gV, ctx.x0["V"]),
               "Phi": zeros_like_or(gPhi, ctx.x0["Phi"]), "pi": zeros_like_or(gpi, ctx.x0["pi"])}

        def advance(x, n):
            s.load(x)
            s.step(n, dt)
            return s.store()

        def adjoint(x, g):
            s.load(x)
            return s.step_adjoint(g, dt)

        def copy(x):
            return {f: v.clone() for f, v in x.items()}

        grad, stats = reverse_sweep(ctx.x0, ctx.nsteps, ctx.snaps, advance, adjoint, lam, copy)
        ctx.stats = stats
        AgcmSteps.last_stats = stats
        return None, None, None, None, grad["U"], grad["V"], grad["Phi"], grad["pi"]


def run(state, x0, nsteps, dt, snaps=8):
    """Differentiable nsteps-step map: returns the dict of final fields."""
    out = AgcmSteps.apply(state, nsteps, dt, snaps, x0["U"], x0["V"], x0["Phi"], x0["pi"])
    return dict(zip(FIELDS, out))


def box_mask(nlon, nlat, lat0=35.0, lat1=55.0, lon0=170.0, lon1=190.0, device="cuda", dtype=torch.float64):
    """Scalar points with latitude in [lat0, lat1] and longitude in [lon0, lon1] (degrees)."""
    import math

    th = (torch.arange(nlat, dtype=torch.float64) + 0.5) * (math.pi / nlat)
    lat = 90.0 - torch.rad2deg(th)
    lon = torch.arange(nlon, dtype=torch.float64) * (360.0 / nlon)
    m = ((lat >= lat0) & (lat <= lat1))[:, None] & ((lon >= lon0) & (lon <= lon1))[None, :]
    return m.to(device=device, dtype=dtype)


def box_objective(pi, mask):
    """J = mean of pi^2 over the box (the surface-pressure anomaly p'_sa/p0)."""
    return (pi.to(mask.dtype) ** 2 * mask).sum() / mask.sum()
