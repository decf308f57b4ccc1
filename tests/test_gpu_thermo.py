"""GPU parity of Eq. 1's thermodynamics (agcm_grid_set_thermo) against the
FP64 oracle: a lapse-rate standard atmosphere with per-level b, the
delta_c / delta_p factors, and the nonlinear delta kappa Phi/P term.

Tolerances as in the other parity tests (normwise per field, max|gpu - orc| /
max|orc|): FP64 1e-12 for one tendency or step, FP32 with FP64 column sums
1e-5 after one step.
"""
import numpy as np
import pytest

import oracle
from paper_2103_10114_gb300 import agcm, inputs
from paper_2103_10114_gb300.ensemble import Ensemble

pytestmark = pytest.mark.gpu
FIELDS = agcm.FIELDS
LAPSE = dict(profile=1, Ts0=288.15, lapse=6.5e-3, Ttrop=216.65)
LINEAR = dict(LAPSE, delta_c=0.3, delta_p=0.2)
FULL = dict(LINEAR, delta=1.0)
ISO300 = dict(profile=0, T0=300.0, delta=1.0)


@pytest.fixture(scope="module", autouse=True)
def _built(cuda_ok):
    agcm.build()
    agcm.lib()


def rel_err(a, b):
    den = np.abs(b).max()
    return np.abs(a - b).max() / (den if den > 0 else 1.0)


def to_np(d):
    return {f: v.double().cpu().numpy() for f, v in d.items()}


def make(I, J, K, thermo, kind="random", seed=11):
    if kind == "random":
        st = inputs.random_state(I, J, K, seed=seed)
    else:
        st = inputs.baroclinic_jet(I, J, K, seed=3, noise=1e-2, terrain_seed=2)
    g = agcm.Grid(I, J, K, phis=st["phis"], thermo=thermo)
    o = oracle.Oracle(I, J, K, phis=st["phis"], thermo=thermo)
    return g, o, {f: st[f] for f in FIELDS}


CASES = [(37, 23, 7, "random"), (128, 64, 8, "random"), (256, 128, 30, "jet")]
THERMOS = {"lapse": LAPSE, "linear": LINEAR, "full": FULL, "iso300": ISO300}


@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c[:3])))
@pytest.mark.parametrize("tname", list(THERMOS))
def test_tendency_and_step(case, tname, stage_kernel):
    I, J, K, kind = case
    g, o, x = make(I, J, K, THERMOS[tname], kind)
    dt = g.dt(100.0)
    t_ref = o.tendency(x)
    s_ref = o.step(x, dt, 1)
    s = agcm.State(g, agcm.AGCM_FP64)
    s.load(x)
    t = to_np(s.tendency())
    for f in FIELDS:
        assert rel_err(t[f], t_ref[f]) <= 1e-12, ("tendency", f, rel_err(t[f], t_ref[f]))
    s.step(1, dt)
    out = to_np(s.store())
    for f in FIELDS:
        assert rel_err(out[f], s_ref[f]) <= 1e-12, ("fp64 step", f)
    s.close()
    s = agcm.State(g, agcm.AGCM_FP32)
    s.load(x)
    s.step(1, dt)
    out = to_np(s.store())
    for f in FIELDS:
        assert rel_err(out[f], s_ref[f]) <= 1e-5, ("fp32 step", f, rel_err(out[f], s_ref[f]))
    s.close()


def test_twenty_steps_and_energy_diagnostics():
    I, J, K = 128, 64, 8
    g, o, x = make(I, J, K, FULL, "jet")
    dt = g.dt(100.0)
    ref = o.step(x, dt, 20)
    s = agcm.State(g, agcm.AGCM_FP64)
    s.load(x)
    d0 = s.diagnostics()
    o0 = o.diagnostics(x)
    for k in ("mass", "e_kin", "e_pot", "e_ps", "energy"):
        assert abs(d0[k] - o0[k]) <= 1e-12 * abs(o0[k]), k
    s.step(20, dt)
    out = to_np(s.store())
    for f in FIELDS:
        assert rel_err(out[f], ref[f]) <= 1e-10, f
    s.close()


def test_split_step_with_the_nonlinear_term():
    I, J, K = 128, 64, 8
    g, o, x = make(I, J, K, FULL, "jet")
    dt, msub = g.dt_split(100.0)
    ada = oracle.TERM_COR | oracle.TERM_PGF_PI | oracle.TERM_PGF_PHI
    ref = x
    for _ in range(2):
        ref = o.step(ref, dt / msub, msub, terms=ada)
        ref = o.step(ref, dt, 1, terms=oracle.TERM_ADV)
    for prec, tol in ((agcm.AGCM_FP64, 1e-11), (agcm.AGCM_FP32, 1e-5)):
        s = agcm.State(g, prec)
        s.load(x)
        s.step_split(2, dt, msub)
        out = to_np(s.store())
        for f in FIELDS:
            assert rel_err(out[f], ref[f]) <= tol, (prec, f, rel_err(out[f], ref[f]))
        s.close()


def test_adjoint_with_per_level_b():
    """The adjoint covers the linear thermodynamics (per-level b, delta_c,
    delta_p): dot test against the oracle's tangent-linear step."""
    I, J, K = 37, 23, 7
    g, o, x = make(I, J, K, LINEAR)
    dt = g.dt(100.0)
    s = agcm.State(g, agcm.AGCM_FP64)
    s.load(x)
    v = inputs.random_direction(I, J, K, seed=101)
    lam = inputs.random_direction(I, J, K, seed=201)
    _, jv = o.step_jvp(x, v, dt, 1)
    jtl = to_np(s.step_adjoint(lam, dt))
    lhs = sum(float(np.sum(lam[f] * jv[f])) for f in FIELDS)
    rhs = sum(float(np.sum(jtl[f] * v[f])) for f in FIELDS)
    scale = sum(float(np.sum(np.abs(lam[f] * jv[f]))) for f in FIELDS)
    assert abs(lhs - rhs) <= 1e-12 * scale
    s.close()


@pytest.mark.parametrize("case", [(37, 23, 7, "full"), (64, 32, 10, "full"), (48, 24, 6, "iso300")],
                         ids=lambda c: f"{c[0]}x{c[1]}x{c[2]}-{c[3]}")
def test_adjoint_with_the_nonlinear_term(case):
    """The adjoint covers Eq. 1's delta kappa Phi/P term: dot test of one step
    against the oracle's tangent-linear step (dual numbers through the same
    scheme), FP64 to 1e-12, and FP32 within 1e-4 of the FP64 adjoint."""
    I, J, K, tname = case
    g, o, x = make(I, J, K, THERMOS[tname])
    dt = g.dt(100.0)
    v = inputs.random_direction(I, J, K, seed=102)
    lam = inputs.random_direction(I, J, K, seed=202)
    _, jv = o.step_jvp(x, v, dt, 1)
    out = {}
    for prec in (agcm.AGCM_FP64, agcm.AGCM_FP32):
        s = agcm.State(g, prec)
        s.load(x)
        out[prec] = to_np(s.step_adjoint(lam, dt))
        s.close()
    jtl = out[agcm.AGCM_FP64]
    lhs = sum(float(np.sum(lam[f] * jv[f])) for f in FIELDS)
    rhs = sum(float(np.sum(jtl[f] * v[f])) for f in FIELDS)
    scale = sum(float(np.sum(np.abs(lam[f] * jv[f]))) for f in FIELDS)
    assert abs(lhs - rhs) <= 1e-12 * scale, (lhs, rhs)
    for f in FIELDS:
        assert rel_err(out[agcm.AGCM_FP32][f], jtl[f]) <= 1e-4, f


def test_nonlinear_term_is_refused_where_not_covered():
    I, J, K = 16, 10, 4
    g, _, x = make(I, J, K, FULL)
    s = agcm.State(g, agcm.AGCM_FP64)
    s.load(x)
    with pytest.raises(agcm.AgcmError) as e:
        Ensemble([s])
    assert e.value.code == agcm.AGCM_EINVAL
    # and the grid's tables are fixed once a state exists
    with pytest.raises(agcm.AgcmError) as e:
        g.set_thermo(**LAPSE)
    assert e.value.code == agcm.AGCM_EINVAL
    s.close()


def test_ensemble_member_with_lapse_profile():
    I, J, K = 64, 32, 10
    g, o, x = make(I, J, K, LINEAR, "jet")
    dt = g.dt(100.0)
    s = agcm.State(g, agcm.AGCM_FP64)
    s.load(x)
    ens = Ensemble([s])
    ens.step(2, [dt])
    ens.status()
    ref = o.step(x, dt, 2)
    out = to_np(s.store())
    for f in FIELDS:
        assert rel_err(out[f], ref[f]) <= 1e-12, f
    ens.close()
    s.close()


def test_terrain_above_the_tropopause():
    """Terrain scaled to 15 km puts some columns' standard surface above the
    11 km tropopause (the isothermal branch of the standard atmosphere): the
    library's surface tables still match the oracle's, through one step."""
    I, J, K = 64, 32, 8
    st = inputs.baroclinic_jet(I, J, K, seed=3, noise=1e-2, terrain_seed=2)
    phis = st["phis"] * 5.0
    assert phis.max() / 9.80665 > 11000.0
    g = agcm.Grid(I, J, K, phis=phis, thermo=FULL)
    o = oracle.Oracle(I, J, K, phis=phis, thermo=FULL)
    x = {f: st[f] for f in FIELDS}
    dt = g.dt(100.0)
    ref = o.step(x, dt, 1)
    d_ref = o.diagnostics(x)
    s = agcm.State(g, agcm.AGCM_FP64)
    s.load(x)
    d = s.diagnostics()
    assert abs(d["e_ps"] - d_ref["e_ps"]) <= 1e-12 * abs(d_ref["e_ps"])
    s.step(1, dt)
    out = to_np(s.store())
    for f in FIELDS:
        assert rel_err(out[f], ref[f]) <= 1e-12, f
    s.close()


@pytest.mark.parametrize("prec,tol", [(agcm.AGCM_FP64, 1e-11), (agcm.AGCM_FP32, 1e-5)])
def test_every_option_on_a_ragged_grid(prec, tol, stage_kernel):
    """Non-uniform sigma, terrain, the full
    thermodynamics, split stepping and the low-latitude filter on a ragged
    38 x 23 x 7 grid (nlon even, so the two-grid removal runs; 38 is not a
    multiple of 4, so the FP32 filter takes its scalar path): two split steps,
    each followed by the filter, against the oracle's same composition."""
    I, J, K = 38, 23, 7
    sig = [0.0, 0.03, 0.1, 0.22, 0.4, 0.6, 0.82, 1.0]
    mu = mv = None  # Eq. 7: the split dt assumes the 45-degree spacing it keeps
    # the jet (a random state is not stable at the advective dt of split stepping)
    st = inputs.baroclinic_jet(I, J, K, seed=21, noise=1e-2, terrain_seed=2)
    g = agcm.Grid(I, J, K, sigma_half=sig, leap_u=mu, leap_v=mv, phis=st["phis"], thermo=FULL)
    o = oracle.Oracle(I, J, K, sigma_half=sig, leap_u=mu, leap_v=mv, phis=st["phis"], thermo=FULL)
    x = {f: st[f] for f in FIELDS}
    dt, msub = g.dt_split(100.0)
    ada = oracle.TERM_COR | oracle.TERM_PGF_PI | oracle.TERM_PGF_PHI
    ref = x
    for _ in range(2):
        ref = o.step(ref, dt / msub, msub, terms=ada)
        ref = o.step(ref, dt, 1, terms=oracle.TERM_ADV)
        ref = o.filter(ref, 0.25)
    s = agcm.State(g, prec)
    s.load(x)
    for _ in range(2):
        s.step_split(1, dt, msub)
        s.filter(0.25)
    out = to_np(s.store())
    for f in FIELDS:
        assert np.isfinite(ref[f]).all()
        assert rel_err(out[f], ref[f]) <= tol, (prec, f, rel_err(out[f], ref[f]))
    s.close()
