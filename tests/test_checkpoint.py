"""Host logic of the binomial checkpointing schedule (no GPU)."""
import math

import numpy as np
import pytest

from paper_2103_10114_gb300.checkpoint import forward_cost, reverse_sweep


def binomial_cost(t, s):
    """Closed form of the optimal recomputation count (Griewank's binomial
    bound), with c = s + 1 checkpoints counting the held start state: r is the
    least integer with C(c + r, c) >= t and the count is r t - C(c + r, c + 1)."""
    if t <= 1:
        return 0
    c = s + 1
    r = 0
    while math.comb(c + r, c) < t:
        r += 1
    return r * t - math.comb(c + r, c + 1)


@pytest.mark.parametrize("s", [1, 2, 3, 8])
def test_cost_matches_binomial_bound(s):
    for t in range(1, 60):
        assert forward_cost(t, s) == binomial_cost(t, s), (t, s)


@pytest.mark.parametrize("t,s", [(1, 8), (7, 0), (13, 2), (50, 8), (50, 3)])
def test_gradient_equals_storing_all_states(t, s):
    rng = np.random.default_rng(t * 10 + s)
    n = 6
    mats = [0.95 * np.linalg.qr(rng.normal(size=(n, n)))[0] for _ in range(t)]
    # nonlinear step so the state really matters: x' = A_k x + 0.05 sin(x), k = step index
    def step(x, k):
        return mats[k] @ x + 0.05 * np.sin(x)

    def jac_t(x, k, g):
        return mats[k].T @ g + 0.05 * np.cos(x) * g

    x0 = rng.normal(size=n)
    lam = rng.normal(size=n)
    # direct: store every state
    xs = [x0]
    for k in range(t):
        xs.append(step(xs[-1], k))
    g = lam.copy()
    for k in range(t - 1, -1, -1):
        g = jac_t(xs[k], k, g)
    # checkpointed: states carry their step index
    def advance(x, m):
        y, k = x
        for q in range(m):
            y = step(y, k + q)
        return (y, k + m)

    def adjoint(x, gg):
        return jac_t(x[0], x[1], gg)

    got, stats = reverse_sweep((x0, 0), t, s, advance, adjoint, lam, lambda x: (x[0].copy(), x[1]))
    assert np.allclose(got, g, rtol=1e-12, atol=1e-12)
    assert stats["max_snapshots"] <= s
    assert stats["forward_steps"] == forward_cost(t, s)
