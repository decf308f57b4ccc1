"""Multi-step gradients: torch.autograd.Function + binomial checkpointing over
the hand-written step adjoint."""
import numpy as np
import pytest

import oracle
from paper_2103_10114_gb300 import agcm, autograd, inputs

pytestmark = pytest.mark.gpu
FIELDS = agcm.FIELDS


@pytest.fixture(scope="module", autouse=True)
def _built(cuda_ok):
    agcm.build()
    agcm.lib()


def as_dev(st, dtype, grad=False):
    import torch

    return {f: torch.as_tensor(np.ascontiguousarray(st[f]), dtype=dtype, device="cuda").requires_grad_(grad)
            for f in FIELDS}


def grad_of_box(state, x0_np, nsteps, dt, snaps, dtype):
    import torch

    x0 = as_dev(x0_np, dtype, grad=True)
    out = autograd.run(state, x0, nsteps, dt, snaps)
    mask = autograd.box_mask(state.grid.nlon, state.grid.nlat)
    J = autograd.box_objective(out["pi"], mask)
    J.backward()
    return float(J.detach()), {f: x0[f].grad.double().cpu().numpy() for f in FIELDS}


def test_gradient_matches_oracle_tangent_linear_fp64():
    """<dJ/dx0, v> == <dJ/dx_N, J_N v> with J_N v from the oracle's dual numbers."""
    import math

    I, J, K, n = 32, 16, 5, 6
    st = inputs.baroclinic_jet(I, J, K, seed=9, noise=1e-2, terrain_seed=2)
    g = agcm.Grid(I, J, K, phis=st["phis"])
    dt = g.dt(100.0)
    s = agcm.State(g, agcm.AGCM_FP64)
    x0 = {f: st[f] for f in FIELDS}
    _, grad = grad_of_box(s, x0, n, dt, 2, s.dtype)
    o = oracle.Oracle(I, J, K, phis=st["phis"])
    mask = autograd.box_mask(I, J, device="cpu").numpy()
    assert mask.sum() > 0
    for seed in (1, 2, 3):
        v = inputs.random_direction(I, J, K, seed=seed)
        xN, jv = o.step_jvp(x0, v, dt, n)
        want = float(np.sum(2.0 * xN["pi"] * mask * jv["pi"]) / mask.sum())
        got = sum(float(np.sum(grad[f] * v[f])) for f in FIELDS)
        assert abs(got - want) <= 1e-11 * abs(want) + 1e-30, (got, want)
    assert math.isfinite(got)


def test_checkpointing_equals_storing_every_state():
    I, J, K, n = 48, 24, 6, 13
    st = inputs.baroclinic_jet(I, J, K, seed=10, noise=1e-2, terrain_seed=2)
    g = agcm.Grid(I, J, K, phis=st["phis"])
    dt = g.dt(100.0)
    s = agcm.State(g, agcm.AGCM_FP64)
    x0 = {f: st[f] for f in FIELDS}
    _, g2 = grad_of_box(s, x0, n, dt, 2, s.dtype)
    stats2 = dict(autograd.AgcmSteps.last_stats)
    _, gall = grad_of_box(s, x0, n, dt, n, s.dtype)
    assert stats2["max_snapshots"] <= 2
    for f in FIELDS:
        assert np.abs(g2[f] - gall[f]).max() <= 1e-12 * np.abs(gall[f]).max()


def _J64(state, x, nsteps, dt, mask):
    import torch

    state.load(as_dev(x, torch.float64))
    state.step(nsteps, dt)
    pi = state.store()["pi"]
    return float(autograd.box_objective(pi, mask))


def test_config3_gradient_fd_and_dot():
    """720 x 360 x 30, FP32, 50 steps, 8 stored states: the gradient of
    J = mean pi^2 over [35N, 55N] x [170E, 190E] against central finite
    differences of the FP64 forward along 10 seeded directions; and the same
    with the FP64 adjoint."""
    I, J, K, n = 720, 360, 30, 50
    st = inputs.baroclinic_jet(I, J, K, seed=3, noise=1e-2, terrain_seed=2)
    g = agcm.Grid(I, J, K, phis=st["phis"])
    dt = g.dt(100.0)
    x0 = {f: st[f] for f in FIELDS}
    s32 = agcm.State(g, agcm.AGCM_FP32)
    _, grad32 = grad_of_box(s32, x0, n, dt, 8, s32.dtype)
    stats = dict(autograd.AgcmSteps.last_stats)
    assert stats["max_snapshots"] <= 8
    s32.close()
    s64 = agcm.State(g, agcm.AGCM_FP64)
    _, grad64 = grad_of_box(s64, x0, n, dt, 8, s64.dtype)
    mask = autograd.box_mask(I, J)
    errs32, errs64 = [], []
    for q in range(10):
        v = inputs.random_direction(I, J, K, seed=4000 + q)
        h = 2e-3
        jp = _J64(s64, {f: x0[f] + h * v[f] for f in FIELDS}, n, dt, mask)
        jm = _J64(s64, {f: x0[f] - h * v[f] for f in FIELDS}, n, dt, mask)
        fd = (jp - jm) / (2 * h)
        d32 = sum(float(np.sum(grad32[f] * v[f])) for f in FIELDS)
        d64 = sum(float(np.sum(grad64[f] * v[f])) for f in FIELDS)
        errs32.append(abs(d32 - fd) / abs(fd))
        errs64.append(abs(d64 - fd) / abs(fd))
    assert max(errs64) <= 1e-6, (errs64, errs32)
    assert max(errs32) <= 1e-3, (errs64, errs32)
