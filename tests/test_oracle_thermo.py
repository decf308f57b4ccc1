"""Pins of the oracle's thermodynamic extension (Eq. 1's standard
stratification and its delta switches; readings T1..T4).

* The default and an explicit isothermal 250 K with the switches off give the
  same tendency bit for bit (the pinned scheme is the special case).
* The standard atmosphere: the oracle's closed-form surface pressure satisfies
  hydrostatic balance, checked by numerical quadrature of R T~(p) dp/p; its
  values at 1 km and at the tropopause match the standard-atmosphere table.
* Energy neutrality of the whole spatial operator for the lapse-rate profile
  with every switch on (weights written here from their closed form).
* delta_p = 1 removes exactly the Phi part of the pressure gradient and the
  Omega~ conversion; delta_c scales exactly that part by (1 + delta_c).
* The delta kappa Phi/P term makes the operator nonlinear in Phi; the forward
  derivative still matches central differences.
"""
import math

import numpy as np
import pytest
from scipy import integrate, optimize

import oracle
from oracle import TERM_ALL, TERM_PGF_PHI
from paper_2103_10114_gb300 import inputs

R, G0 = 287.04, 9.80665
A_E = 6.371e6
FIELDS = ("U", "V", "Phi", "pi")
LAPSE = dict(profile=1, Ts0=288.15, lapse=6.5e-3, Ttrop=216.65)
FULL = dict(LAPSE, delta=1.0, delta_c=0.3, delta_p=0.2)


def _surface_ref(phis, Ts0=288.15, lapse=6.5e-3, Ttrop=216.65):
    """Standard-atmosphere surface pressure / p0 and temperature, written from
    the textbook lapse-rate and isothermal-layer formulas."""
    z = phis / G0
    ztr = (Ts0 - Ttrop) / lapse
    n = G0 / (R * lapse)
    if z <= ztr:
        T = Ts0 - lapse * z
        return (T / Ts0) ** n, T
    return (Ttrop / Ts0) ** n * math.exp(-G0 * (z - ztr) / (R * Ttrop)), Ttrop


def _weights(I, J, K, phis, thermo=None):
    dl, dth = 2 * math.pi / I, math.pi / J
    s = np.sin((np.arange(J) + 0.5) * dth)
    sv = np.sin((np.arange(J - 1) + 1.0) * dth)
    A = A_E**2 * s * dth * dl
    Av = A_E**2 * sv * dth * dl
    ds = np.full(K, 1.0 / K)
    if thermo is None:
        wpi = R * 250.0 / np.exp(-np.asarray(phis) / (R * 250.0))
    else:
        ref = np.vectorize(lambda p: _surface_ref(p))
        pit, Ts = ref(np.asarray(phis))
        wpi = R * Ts / pit
    return {
        "U": ds[:, None, None] * A[None, :, None] * np.ones((K, J, I)),
        "V": ds[:, None, None] * Av[None, :, None] * np.ones((K, J - 1, I)),
        "Phi": ds[:, None, None] * A[None, :, None] * np.ones((K, J, I)),
        "pi": A[:, None] * wpi,
    }


def _inner(w, x, y):
    return sum(float(np.sum(w[f] * x[f] * y[f])) for f in FIELDS)


def _absinner(w, x, y):
    return sum(float(np.sum(w[f] * np.abs(x[f] * y[f]))) for f in FIELDS)


def _case(I=16, J=10, K=5, seed=3, thermo=None):
    st = inputs.random_state(I, J, K, seed=seed)
    o = oracle.Oracle(I, J, K, phis=st["phis"], thermo=thermo)
    return o, {f: st[f] for f in FIELDS}, st["phis"]


def test_explicit_default_is_bit_identical():
    o0, st, phis = _case()
    o1 = oracle.Oracle(16, 10, 5, phis=phis, thermo=dict(oracle.THERMO_DEFAULT))
    t0, t1 = o0.tendency(st), o1.tendency(st)
    assert all(np.array_equal(t0[f], t1[f]) for f in FIELDS)
    assert o0.diagnostics(st) == o1.diagnostics(st)


@pytest.mark.parametrize("phis", [0.0, 4.9e3, 2.9e4, 1.2e5, 1.6e5])
def test_standard_surface_is_hydrostatic(phis):
    """phi_s = integral from pi~ to 1 of R T~(p) dp / p, by quadrature of the
    oracle's own T~; and T~_s = T~(pi~)."""
    pit, Ts = oracle.std_surface(phis, **LAPSE)
    if phis == 0.0:
        assert pit == 1.0 and Ts == 288.15
        return
    ptr = (216.65 / 288.15) ** (G0 / (R * 6.5e-3))
    pts = [ptr] if pit < ptr < 1 else None
    val, err = integrate.quad(lambda p: R * oracle.std_temp(p, **LAPSE) / p, pit, 1.0, points=pts,
                              epsabs=1e-10, epsrel=1e-12)
    assert abs(val - phis) <= 1e-8 * phis
    assert abs(Ts - oracle.std_temp(pit, **LAPSE)) <= 1e-9 * Ts


def test_standard_atmosphere_table_values():
    """Standard-atmosphere table: p(1 km)/p(0) = 0.88700 and p(11 km)/p(0) =
    0.22336 (226.32 / 1013.25 hPa), T = 281.65 K and 216.65 K; this gas
    constant differs from the table's by 5e-5, hence the tolerances."""
    p1, T1 = oracle.std_surface(G0 * 1000.0, **LAPSE)
    p11, T11 = oracle.std_surface(G0 * 11000.0, **LAPSE)
    assert abs(p1 / 0.88700 - 1) < 3e-5 and abs(T1 - 281.65) < 1e-9
    assert abs(p11 / (226.32 / 1013.25) - 1) < 4e-4 and abs(T11 - 216.65) < 1e-6
    # and the oracle agrees with the textbook formulas written in this file
    for ph in (0.0, 7e3, 9e4, 1.3e5):
        a, b = oracle.std_surface(ph, **LAPSE), _surface_ref(ph)
        assert abs(a[0] - b[0]) <= 1e-13 * b[0] and abs(a[1] - b[1]) <= 1e-12 * b[1]
    assert oracle.std_temp(0.1, **LAPSE) == 216.65  # stratosphere
    assert abs(oracle.std_temp(0.5, **LAPSE) - 288.15 * 0.5 ** (R * 6.5e-3 / G0)) < 1e-12


@pytest.mark.parametrize("thermo", [LAPSE, FULL, dict(FULL, delta_p=0.0, delta_c=-0.4)])
def test_energy_neutral_with_thermodynamics(thermo):
    I, J, K = 16, 10, 5
    o, st, phis = _case(I, J, K, seed=7, thermo=thermo)
    w = _weights(I, J, K, phis, thermo)
    t = o.tendency(st)
    assert abs(_inner(w, st, t)) <= 1e-13 * _absinner(w, st, t)
    # the diagnostics use the same surface weight
    d = o.diagnostics(st)
    eps = 0.5 * float(np.sum(w["pi"] * st["pi"] ** 2))
    assert abs(d["e_ps"] - eps) <= 1e-12 * eps


def test_energy_pin_sees_a_mismatched_coefficient():
    """Were the Omega~ conversion to use b while psi uses c, energy would not be
    neutral: the split tendency with delta_c on only one side breaks the pin."""
    I, J, K = 16, 10, 5
    o1, st, phis = _case(I, J, K, seed=7, thermo=dict(LAPSE, delta_c=0.3))
    o0 = oracle.Oracle(I, J, K, phis=phis, thermo=LAPSE)
    w = _weights(I, J, K, phis, LAPSE)
    t1, t0 = o1.tendency(st), o0.tendency(st)
    mixed = dict(t1)
    mixed["Phi"] = t0["Phi"]  # Omega~ from c without delta_c, psi with it
    assert abs(_inner(w, st, mixed)) > 1e-6 * _absinner(w, st, mixed)


def test_delta_p_one_removes_the_phi_coupling():
    o0, st, phis = _case(seed=9)
    o1 = oracle.Oracle(16, 10, 5, phis=phis, thermo=dict(delta_p=1.0, delta=1.0))
    t1 = o1.tendency(st)
    t0 = o0.tendency(st, TERM_ALL & ~TERM_PGF_PHI)
    assert all(np.array_equal(t0[f], t1[f]) for f in FIELDS)


def test_delta_c_scales_the_phi_coupling():
    o0, st, phis = _case(seed=11, thermo=LAPSE)
    o1 = oracle.Oracle(16, 10, 5, phis=phis, thermo=dict(LAPSE, delta_c=0.3))
    base = o0.tendency(st, TERM_ALL & ~TERM_PGF_PHI)
    part = o0.tendency(st, TERM_PGF_PHI)
    t1 = o1.tendency(st)
    for f in FIELDS:
        want = base[f] + 1.3 * part[f]
        assert np.abs(t1[f] - want).max() <= 1e-12 * np.abs(want).max(), f


def test_nonlinear_term_derivative_matches_differences():
    I, J, K = 16, 10, 5
    o, st, _ = _case(I, J, K, seed=13, thermo=FULL)
    d = {f: v for f, v in inputs.random_direction(I, J, K, seed=14).items() if f in FIELDS}
    jv = o.tendency_jvp(st, d)
    h = 1e-5
    tp = o.tendency({f: st[f] + h * d[f] for f in FIELDS})
    tm = o.tendency({f: st[f] - h * d[f] for f in FIELDS})
    for f in FIELDS:
        fd = (tp[f] - tm[f]) / (2 * h)
        assert np.abs(fd - jv[f]).max() <= 1e-6 * np.abs(jv[f]).max(), f
    # and the delta term matters: the tendency differs from delta = 0
    o_lin = oracle.Oracle(I, J, K, phis=_case(I, J, K, seed=13)[2], thermo=dict(FULL, delta=0.0))
    t_lin, t_nl = o_lin.tendency(st), o.tendency(st)
    assert np.abs(t_lin["Phi"] - t_nl["Phi"]).max() > 1e-6 * np.abs(t_nl["Phi"]).max()


def test_rejects_bad_thermo():
    for bad in (dict(profile=2), dict(T0=-1.0), dict(delta_p=1.5), dict(delta_c=-1.0), dict(Ttrop=300.0),
                dict(lapse=-1e-3)):
        with pytest.raises(ValueError):
            oracle.Oracle(8, 4, 2, thermo=bad)
