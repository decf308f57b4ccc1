"""Closed-form pins of the oracle's Coriolis parameter and hydrostatic matrix.

Energy neutrality cannot see these two: it holds for any f* and for any H
(the Omega~ term uses H^T).  So each is pinned here against a value the
mathematics fixes, written in this file from Eq. 1 and the grid definition
(reading R1), not from the oracle:

* Coriolis (Eq. 1, the gamma* f* V and gamma* f* U terms, with
  f* = 2 Omega cos(theta) + u cot(theta) / a, theta colatitude).  A single
  nonzero U (or V) value makes the Coriolis-only tendency a handful of
  closed-form numbers at the corner-adjacent V (or U) points and zero
  elsewhere; rows in both hemispheres catch a cos/sin or sign slip, and
  P != 1 catches u = U/P^u dropped to U.
* Hydrostatic geopotential (Eq. 1's P_lambda, P_theta terms; reading R7).
  For Phi_k / P uniform in k the discrete integral must equal the continuous
  one, phi'_k = b (Phi/P) ln(1/sigma_k) at the layer midpoints sigma_k, and the
  pressure gradient is then the closed-form leap difference of that phi'.

The last tests plant the slips the pins are for in a copy of the oracle's
source (compiled on the CPU, never imported by anything else) and check that
each pin fails on it.
"""
import ctypes
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from oracle import TERM_COR, TERM_PGF_PHI

A_E = 6.371e6
OMEGA = 7.292e-5
R_D, CP = 287.04, 1004.64
B_ISO = math.sqrt(R_D / CP * R_D * 250.0)  # b = sqrt(kappa R T0), reading R2


def _geometry(I, J):
    dl, dth = 2 * math.pi / I, math.pi / J
    th = (np.arange(J) + 0.5) * dth          # scalar / U rows
    thv = (np.arange(J - 1) + 1.0) * dth     # V rows
    return dl, dth, th, thv


def _rel(got, want):
    scale = max(np.abs(want).max(), 1e-300)
    return float(np.abs(got - want).max() / scale)


# ------------------------------------------------------------------ Coriolis
def coriolis_errors(O=None):
    """Max relative error of the Coriolis-only tendency against the closed
    forms, over four single-point states (U or V, northern or southern row)."""
    O = O or oracle.Oracle
    I, J, K = 12, 10, 2
    dl, dth, th, thv = _geometry(I, J)
    pi0 = 0.3                     # uniform pi: P = P^u = P^v = sqrt(1 + pi0) (flat terrain)
    P = math.sqrt(1.0 + pi0)
    o = O(I, J, K)
    errs = []
    c = 37.0
    # U at one point (k0, j0, u0): dV/dt at V rows j0-1 and j0, columns u0 and u0+1
    for j0, u0, k0 in ((2, 5, 1), (7, 11, 0)):   # north, south (u0 = I-1 wraps)
        st = o.zeros()
        st["pi"][:] = pi0
        st["U"][k0, j0, u0] = c
        t = o.tendency(st, TERM_COR)
        fstar = 2 * OMEGA * math.cos(th[j0]) + (c / P) * (math.cos(th[j0]) / math.sin(th[j0])) / A_E
        A = A_E**2 * math.sin(th[j0]) * dth * dl
        want = {f: np.zeros_like(v) for f, v in st.items()}
        for jv in (j0 - 1, j0):
            Av = A_E**2 * math.sin(thv[jv]) * dth * dl
            for i in (u0, (u0 + 1) % I):
                want["V"][k0, jv, i] = 0.25 * A * fstar * c / Av
        errs.append(max(_rel(t[f], want[f]) for f in ("U", "V")) if np.abs(want["V"]).max() else 1.0)
        errs.append(max(float(np.abs(t[f]).max()) for f in ("Phi", "pi")))
    # V at one point (k0, j0, i0): dU/dt at U rows j0 and j0+1, columns i0-1 and i0
    for j0, i0, k0 in ((1, 0, 0), (6, 4, 1)):    # north (i0 = 0 wraps), south
        st = o.zeros()
        st["pi"][:] = pi0
        st["V"][k0, j0, i0] = c
        t = o.tendency(st, TERM_COR)
        want = {f: np.zeros_like(v) for f, v in st.items()}
        for ju in (j0, j0 + 1):
            f0 = 2 * OMEGA * math.cos(th[ju])  # U = 0 there: f* = 2 Omega cos(theta)
            for u in ((i0 - 1) % I, i0):
                want["U"][k0, ju, u] = -0.25 * f0 * c
        errs.append(max(_rel(t[f], want[f]) for f in ("U", "V")))
        errs.append(max(float(np.abs(t[f]).max()) for f in ("Phi", "pi")))
    return max(errs)


def test_coriolis_matches_closed_form():
    assert coriolis_errors() <= 1e-13


# ------------------------------------------------------------- hydrostatics
SIG = [0.0, 0.05, 0.13, 0.3, 0.52, 0.77, 1.0]  # non-uniform half levels


def hydrostatic_errors(O=None):
    """Max relative error of the hydrostatic pressure gradient against the
    continuous integral, for Phi_k / P = g(j, i) uniform in k."""
    O = O or oracle.Oracle
    I, J, K = 24, 12, len(SIG) - 1
    dl, dth, th, thv = _geometry(I, J)
    o = O(I, J, K, sigma_half=SIG)
    mu, mv = o.leap_u, o.leap_v
    assert mu.max() > 1, "the grid must have leap rows"
    pi0 = -0.2
    P = math.sqrt(1.0 + pi0)
    lam = np.arange(I) * dl
    g = (40.0 + 25.0 * np.cos(lam)[None, :] * np.sin(th)[:, None] + 9.0 * np.sin(3 * lam)[None, :]
         + 6.0 * np.cos(2 * th)[:, None])                      # Phi / P, J x I
    st = o.zeros()
    st["pi"][:] = pi0
    st["Phi"][:] = P * g[None, :, :]
    t = o.tendency(st, TERM_PGF_PHI)
    sh = np.asarray(SIG)
    sig = 0.5 * (sh[:-1] + sh[1:])
    phi = B_ISO * np.log(1.0 / sig)[:, None, None] * g[None, :, :]   # continuous integral, K x J x I
    want = {f: np.zeros_like(v) for f, v in st.items()}
    for j in range(J):
        M = int(mu[j])
        for u in range(I):
            e, w = (u + (M + 1) // 2) % I, (u - (M - 1) // 2) % I
            want["U"][:, j, u] = -P * (phi[:, j, e] - phi[:, j, w]) / (A_E * math.sin(th[j]) * M * dl)
    for j in range(J - 1):
        want["V"][:, j, :] = -P * (phi[:, j + 1, :] - phi[:, j, :]) / (A_E * dth)
    errs = [_rel(t[f], want[f]) for f in ("U", "V")]
    errs += [float(np.abs(t[f]).max()) for f in ("Phi", "pi")]  # D = 0: no Omega~, no dpi/dt
    return max(errs)


def test_hydrostatic_matches_continuous_integral():
    assert hydrostatic_errors() <= 1e-12


# ------------------------------------------------------------ planted slips
SRC = os.path.join(os.path.dirname(oracle.__file__), "orc_agcm.cpp")
MUTANTS = {
    # f* with sin instead of cos
    "coriolis_sin": ("2.0 * kOmega * g.c[j] +", "2.0 * kOmega * g.s[j] +", coriolis_errors),
    # f* with the metric term's sign flipped
    "coriolis_metric_sign": ("2.0 * kOmega * g.c[j] + (U", "2.0 * kOmega * g.c[j] - (U", coriolis_errors),
    # f* with U instead of u = U / P^u
    "coriolis_no_P": ("(U[x.s3(k, j, u)] / Pu[x.s2(j, u)]) * g.cot[j]", "U[x.s3(k, j, u)] * g.cot[j]",
                      coriolis_errors),
    # diagonal of H from the half levels instead of the layer midpoint
    "H_diagonal": ("g->H[(size_t)k * K + k] = std::log(g->sh[k + 1] / sig);",
                   "g->H[(size_t)k * K + k] = std::log(g->sh[k + 1] / std::max(g->sh[k], 0.5 * sig));",
                   hydrostatic_errors),
    # off-diagonal of H over the layer midpoint instead of the half levels
    "H_offdiagonal": ("std::log(g->sh[kk + 1] / g->sh[kk]);",
                      "std::log(g->sh[kk + 1] / (0.5 * (g->sh[kk] + g->sh[kk + 1])));", hydrostatic_errors),
}


@pytest.fixture(scope="module")
def mutant_dir(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    return tmp_path_factory.mktemp("oracle_mutants")


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pin_fails_on_planted_slip(name, mutant_dir, monkeypatch):
    old, new, check = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    path = os.path.join(str(mutant_dir), f"orc_{name}.cpp")
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    so = path[:-4] + ".so"
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-o", so, path])
    mutant = oracle.bind(ctypes.CDLL(so))
    monkeypatch.setattr(oracle, "_lib", mutant)
    err = check()
    assert err > 1e-6, (name, err)
