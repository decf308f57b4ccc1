"""GPU adjoint of one step (agcm_step_adjoint) against the oracle.

The oracle's step JVP (forward-mode dual numbers through the FP64 oracle) is
the exact tangent-linear of the scheme; the GPU adjoint must be its transpose:
  dot test   <lam, J v> (oracle) == <J^T lam, v> (GPU), FP64, 1e-12 relative;
  full check on a tiny grid: every column J e_q from the oracle, compared
             element by element with the GPU's J^T lam.
"""
import numpy as np
import pytest

import oracle
from paper_2103_10114_gb300 import agcm, inputs

pytestmark = pytest.mark.gpu
FIELDS = agcm.FIELDS


@pytest.fixture(scope="module", autouse=True)
def _built(cuda_ok):
    agcm.build()
    agcm.lib()


def to_np(d):
    return {f: v.double().cpu().numpy() for f, v in d.items()}


def dot(a, b):
    return sum(float(np.sum(a[f] * b[f])) for f in FIELDS)


def absdot(a, b):
    return sum(float(np.sum(np.abs(a[f] * b[f]))) for f in FIELDS)


def setup(I, J, K, seed, kind="random", ones=False, strides=None):
    if kind == "random":
        st = inputs.random_state(I, J, K, seed=seed)
    elif kind == "rh4":
        st = inputs.rossby_haurwitz4(I, J, K, seed=1)
    else:
        st = inputs.baroclinic_jet(I, J, K, seed=3, noise=1e-2, terrain_seed=2)
    mu = mv = None
    if ones:
        mu, mv = np.ones(J, np.int32), np.ones(J - 1, np.int32)
    if strides is not None:
        mu, mv = (np.asarray(a, np.int32) for a in strides)
    g = agcm.Grid(I, J, K, leap_u=mu, leap_v=mv, phis=st["phis"])
    o = oracle.Oracle(I, J, K, leap_u=mu, leap_v=mv, phis=st["phis"])
    x = {f: st[f] for f in FIELDS}
    return g, o, x


CASES = [(16, 10, 4, "random", False), (20, 9, 3, "random", False), (5, 3, 1, "random", True),
         (12, 6, 70, "random", False),
         (37, 23, 7, "random", False), (128, 64, 8, "rh4", False), (64, 32, 10, "jet", False)]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}x{c[2]}-{c[3]}")
def test_dot_product_fp64(case):
    I, J, K, kind, ones = case
    g, o, x = setup(I, J, K, 21, kind, ones)
    dt = g.dt(100.0)
    s = agcm.State(g, agcm.AGCM_FP64)
    s.load(x)
    for seed in (1, 2):
        v = inputs.random_direction(I, J, K, seed=100 + seed)
        lam = inputs.random_direction(I, J, K, seed=200 + seed)
        _, jv = o.step_jvp(x, v, dt, 1)
        jtl = to_np(s.step_adjoint(lam, dt))
        lhs, rhs = dot(lam, jv), dot(jtl, v)
        scale = max(absdot(lam, jv), absdot(jtl, v))
        assert abs(lhs - rhs) <= 1e-12 * scale, (lhs, rhs, scale)
    # the state is unchanged by the adjoint
    after = to_np(s.store())
    for f in FIELDS:
        assert np.array_equal(after[f], x[f])


def test_dot_product_fp64_wide_strides():
    """Rows whose strides reach past the row-segment halo (here 49, 51 and a
    V-row stride of 53 on 128 longitudes) take the general gather kernel, the
    other rows (among them the row whose northern V row has stride 53) the
    row-segment kernel, in one product."""
    I, J, K = 128, 8, 3
    mu = [51, 1, 3, 1, 5, 3, 1, 49]
    mv = [3, 1, 1, 53, 1, 3, 1]
    g, o, x = setup(I, J, K, 71, strides=(mu, mv))
    dt = g.dt(100.0) * 0.5
    for prec, tol in ((agcm.AGCM_FP64, 1e-12), (agcm.AGCM_FP32, 1e-5)):
        s = agcm.State(g, prec)
        s.load(x)
        v = inputs.random_direction(I, J, K, seed=171)
        lam = inputs.random_direction(I, J, K, seed=271)
        _, jv = o.step_jvp(x, v, dt, 1)
        jtl = to_np(s.step_adjoint(lam, dt))
        lhs, rhs = dot(lam, jv), dot(jtl, v)
        scale = max(absdot(lam, jv), absdot(jtl, v))
        assert abs(lhs - rhs) <= tol * scale, (prec, lhs, rhs, scale)
        s.close()


def test_full_transpose_tiny_fp64():
    I, J, K = 8, 6, 2
    g, o, x = setup(I, J, K, 31)
    dt = g.dt(100.0)
    s = agcm.State(g, agcm.AGCM_FP64)
    s.load(x)
    shapes = o.shapes()
    sizes = [int(np.prod(shapes[f])) for f in FIELDS]
    cols = []
    for fi, f in enumerate(FIELDS):
        for q in range(sizes[fi]):
            d = o.zeros()
            d[f].reshape(-1)[q] = 1.0
            _, jv = o.step_jvp(x, d, dt, 1)
            cols.append(np.concatenate([jv[h].reshape(-1) for h in FIELDS]))
    Jm = np.stack(cols, axis=1)
    for seed in (5, 6, 7):
        lam = inputs.random_direction(I, J, K, seed=seed)
        lam_vec = np.concatenate([lam[h].reshape(-1) for h in FIELDS])
        want = Jm.T @ lam_vec
        got = to_np(s.step_adjoint(lam, dt))
        got_vec = np.concatenate([got[h].reshape(-1) for h in FIELDS])
        assert np.abs(got_vec - want).max() <= 1e-12 * np.abs(want).max()


def test_fp32_adjoint_close_to_fp64_oracle():
    I, J, K = 64, 32, 10
    g, o, x = setup(I, J, K, 41, "jet")
    dt = g.dt(100.0)
    s = agcm.State(g, agcm.AGCM_FP32)
    s.load(x)
    v = inputs.random_direction(I, J, K, seed=301)
    lam = inputs.random_direction(I, J, K, seed=302)
    _, jv = o.step_jvp(x, v, dt, 1)
    jtl = to_np(s.step_adjoint(lam, dt))
    lhs, rhs = dot(lam, jv), dot(jtl, v)
    assert abs(lhs - rhs) <= 1e-5 * max(absdot(lam, jv), absdot(jtl, v))
    # per field against the FP64 GPU adjoint
    s64 = agcm.State(g, agcm.AGCM_FP64)
    s64.load(x)
    ref = to_np(s64.step_adjoint(lam, dt))
    for f in FIELDS:
        err = np.abs(jtl[f] - ref[f]).max() / np.abs(ref[f]).max()
        assert err <= 1e-4, (f, err)


def test_dot_product_fp64_config3_size():
    """The dot test at the differentiation configuration's full size
    (720 x 360 x 30, jet over terrain; its polar rows take the L1 gather form,
    the others the row-segment form): <lam, J v> from the oracle's exact
    tangent-linear step against <J^T lam, v> from the GPU adjoint.  At the
    same size the FP32 adjoint is within 1e-4 of the FP64 one per field and
    passes the dot test at 1e-5, and a second FP32 call is bit-identical."""
    import torch

    I, J, K = 720, 360, 30
    g, o, x = setup(I, J, K, 21, kind="jet")
    dt = g.dt(100.0)
    s = agcm.State(g, agcm.AGCM_FP64)
    s.load(x)
    v = inputs.random_direction(I, J, K, seed=131)
    lam = inputs.random_direction(I, J, K, seed=231)
    _, jv = o.step_jvp(x, v, dt, 1)
    jtl = to_np(s.step_adjoint(lam, dt))
    lhs, rhs = dot(lam, jv), dot(jtl, v)
    scale = max(absdot(lam, jv), absdot(jtl, v))
    assert abs(lhs - rhs) <= 1e-12 * scale, (lhs, rhs, scale)
    s.close()
    s32 = agcm.State(g, agcm.AGCM_FP32)
    s32.load(x)
    a = s32.step_adjoint(lam, dt)
    b = s32.step_adjoint(lam, dt)
    for f in FIELDS:
        assert torch.equal(a[f], b[f]), f
    j32 = to_np(a)
    for f in FIELDS:
        err = np.abs(j32[f] - jtl[f]).max() / np.abs(jtl[f]).max()
        assert err <= 1e-4, (f, err)
    assert abs(lhs - dot(j32, v)) <= 1e-5 * scale
    s32.close()


@pytest.mark.parametrize("prec", [agcm.AGCM_FP32, agcm.AGCM_FP64], ids=["fp32", "fp64"])
def test_adjoint_is_deterministic(prec):
    """Every element of the adjoint is formed by one thread (no atomics), so
    two calls on the same inputs agree bit for bit; the grid spans many tiles
    and rows of every stride class."""
    import torch

    I, J, K = 256, 128, 30
    g, _, x = setup(I, J, K, 51, "jet")
    s = agcm.State(g, prec)
    s.load(x)
    lam = inputs.random_direction(I, J, K, seed=401)
    dt = g.dt(100.0)
    a = s.step_adjoint(lam, dt)
    b = s.step_adjoint(lam, dt)
    for f in FIELDS:
        assert torch.equal(a[f], b[f]), f
    s.close()


def test_adjoint_refuses_aliased_buffers():
    import ctypes

    I, J, K = 16, 10, 4
    g, _, x = setup(I, J, K, 61)
    s = agcm.State(g, agcm.AGCM_FP64)
    s.load(x)
    lam = s.empty()
    ptrs = (ctypes.c_void_p * 4)(*[lam[f].data_ptr() for f in FIELDS])
    rc = agcm.lib().agcm_step_adjoint(s._h, ptrs, ptrs, 1.0, None)
    assert rc == agcm.AGCM_EINVAL
    s.close()
