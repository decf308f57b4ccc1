"""Binomial checkpointing for the reverse sweep over time steps.

Reversing t steps with s free snapshot slots (the start state is always held)
costs F(t, s) forward steps, with
    F(1, s) = 0,  F(t, 0) = t (t - 1) / 2,
    F(t, s) = min over 1 <= m < t of  m + F(t - m, s - 1) + F(m, s):
advance m steps and store a snapshot there, reverse the last t - m steps with
one slot fewer, then reverse the first m steps with the slot freed again.
Its minimum equals the binomial (revolve) optimum; the split that attains it is
tabulated once per (t, s) and replayed by `reverse_sweep`.
"""
from __future__ import annotations

from functools import lru_cache


@lru_cache(maxsize=None)
def _table(t: int, s: int):
    """(cost, split) for reversing t steps with s snapshot slots."""
    if t <= 1:
        return 0, 0
    if s == 0:
        return t * (t - 1) // 2, 0
    best, arg = None, 1
    for m in range(1, t):
        c = m + _table(t - m, s - 1)[0] + _table(m, s)[0]
        if best is None or c < best:
            best, arg = c, m
    return best, arg


def forward_cost(t: int, s: int) -> int:
    """Forward steps the reverse sweep recomputes (on top of the first forward run)."""
    return _table(t, s)[0]


def reverse_sweep(x0, nsteps: int, snaps: int, advance, adjoint, lam, copy):
    """Gradient with respect to x0 of a scalar whose gradient with respect to
    x_nsteps is `lam`.

    advance(x, n) -> state after n steps from x (must not modify x);
    adjoint(x, lam) -> (d x_{k+1} / d x_k)^T lam at x = x_k;
    copy(x) -> an independent copy (a snapshot).
    At most `snaps` snapshots are alive besides x0.
    Returns (gradient, stats) with stats = {"forward_steps", "max_snapshots"}.
    """
    stats = {"forward_steps": 0, "max_snapshots": 0, "live": 0}

    def adv(x, n):
        stats["forward_steps"] += n
        return advance(x, n) if n else x

    def rev(x, t, s, g):
        # x: state at the start of this segment (held by the caller)
        if t == 0:
            return g
        if t == 1:
            return adjoint(x, g)
        if s == 0:
            for q in range(t - 1, -1, -1):
                g = adjoint(adv(x, q) if q else x, g)
            return g
        m = _table(t, s)[1]
        xm = copy(adv(x, m))
        stats["live"] += 1
        stats["max_snapshots"] = max(stats["max_snapshots"], stats["live"])
        g = rev(xm, t - m, s - 1, g)
        del xm
        stats["live"] -= 1
        return rev(x, m, s, g)

    g = rev(x0, nsteps, snaps, lam)
    stats.pop("live")
    return g, stats
