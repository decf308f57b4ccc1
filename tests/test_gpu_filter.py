"""GPU parity of the low-latitude filters (Table "Conventional Filtering
scheme") against the FP64 oracle, element by element.

Tolerances: FP64 1e-13 relative to each field's largest value (the two-grid
amplitude is summed in a different order); FP32 2e-7 against the oracle run on
the FP32-rounded state (one rounding of the FP64 projection, or three
single-precision operations of the 3-point operator).
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


def rel_err(a, b):
    den = np.abs(b).max()
    return np.abs(a - b).max() / (den if den > 0 else 1.0)


def rounded32(st):
    return {f: np.asarray(st[f], np.float32).astype(np.float64) for f in FIELDS}


@pytest.mark.parametrize("shape", [(16, 10, 4), (37, 23, 3), (3, 2, 1), (4, 6, 2), (18, 9, 2), (300, 150, 5),
                                   (1440, 720, 2)],
                         ids=lambda c: "x".join(map(str, c)))
@pytest.mark.parametrize("r", [0.25, 0.1])
def test_filter_matches_oracle(shape, r):
    I, J, K = shape
    st = inputs.random_state(I, J, K, seed=I + J)
    kw = {}
    if I <= 5:  # Eq. 7 strides do not fit such a short row
        kw = dict(leap_u=np.ones(J, np.int32), leap_v=np.ones(J - 1, np.int32))
    g = agcm.Grid(I, J, K, phis=st["phis"], **kw)
    o = oracle.Oracle(I, J, K, phis=st["phis"], **kw)
    for prec, tol in ((agcm.AGCM_FP64, 1e-13), (agcm.AGCM_FP32, 2e-7)):
        src = st if prec == agcm.AGCM_FP64 else rounded32(st)
        ref = o.filter(src, r)
        s = agcm.State(g, prec)
        s.load(st)
        s.filter(r)
        out = to_np(s.store())
        for f in FIELDS:
            assert rel_err(out[f], ref[f]) <= tol, (prec, f, rel_err(out[f], ref[f]))
        s.close()


def test_filter_then_step_uses_fresh_vertical_means():
    """A step after the filter sees the filtered state, vertical means included."""
    I, J, K = 64, 32, 6
    st = inputs.rossby_haurwitz4(I, J, K, seed=1)
    g = agcm.Grid(I, J, K, phis=st["phis"])
    o = oracle.Oracle(I, J, K, phis=st["phis"])
    dt = g.dt(100.0)
    ref = o.step(o.filter(o.step(st, dt, 1)), dt, 1)
    for prec, tol in ((agcm.AGCM_FP64, 1e-12), (agcm.AGCM_FP32, 1e-5)):
        s = agcm.State(g, prec)
        s.load(st)
        s.step(1, dt)
        s.filter()
        s.step(1, dt)
        out = to_np(s.store())
        for f in FIELDS:
            assert rel_err(out[f], ref[f]) <= tol, (prec, f)
        s.close()


def test_filter_rejects_bad_weight():
    g = agcm.Grid(16, 8, 2)
    s = agcm.State(g, agcm.AGCM_FP32)
    for r in (0.0, -0.1, 0.3, float("nan")):
        with pytest.raises(agcm.AgcmError) as e:
            s.filter(r)
        assert e.value.code == agcm.AGCM_EINVAL
    s.close()
