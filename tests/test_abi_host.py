"""CPU-side checks of the C ABI: the library loads, exports every symbol the
header declares, and its host-only calls (grid validation, Eq. 7 tables, the
CFL time step) behave as specified.  No kernel runs here."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import oracle
from paper_2103_10114_gb300 import agcm

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "agcm.h")


@pytest.fixture(scope="module")
def L():
    agcm.build()
    return agcm.lib()


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(agcm_[a-z0-9_]+)\s*\(", text))
    return sorted(n for n in names if not n.endswith("_fn"))


def test_every_declared_symbol_is_exported(L):
    names = declared_symbols()
    assert "agcm_step" in names and "agcm_step_adjoint" in names and "agcm_grid_create" in names
    for n in names:
        assert hasattr(L, n), n
        assert n in agcm.SIGNATURES, f"binding lacks {n}"


def test_binding_names_match_header():
    assert set(agcm.SIGNATURES) == set(declared_symbols())


@pytest.mark.parametrize("nlon,nlat", [(128, 64), (256, 128), (720, 360), (1440, 720), (37, 23)])
def test_leap_tables_match_oracle(L, nlon, nlat):
    g = agcm.Grid(nlon, nlat, 3)
    lu, lv = g.leap()
    ou, ov = oracle.leap_table(nlon, nlat)
    assert np.array_equal(lu, ou) and np.array_equal(lv, ov)


def test_grid_validation(L):
    bad = [
        dict(nlon=2, nlat=4, nlev=2),
        dict(nlon=16, nlat=1, nlev=2),
        dict(nlon=16, nlat=8, nlev=0),
        dict(nlon=16, nlat=8, nlev=2, leap_u=np.full(8, 2)),
        dict(nlon=16, nlat=8, nlev=2, leap_u=np.full(8, 9)),
        dict(nlon=16, nlat=8, nlev=2, leap_v=np.full(7, -1)),
        dict(nlon=16, nlat=8, nlev=2, sigma_half=[0.0, 0.7, 0.6]),
        dict(nlon=16, nlat=8, nlev=2, sigma_half=[0.1, 0.5, 1.0]),
        dict(nlon=16, nlat=8, nlev=2, phis=np.full(128, np.nan)),
        dict(nlon=65536, nlat=32768, nlev=1),  # more columns than 32-bit column indices allow
        dict(nlon=16, nlat=70000, nlev=1),     # more rows than one launch row per latitude allows
        dict(nlon=4000, nlat=2000, nlev=600),  # more than 4e9 points
    ]
    for kw in bad:
        with pytest.raises(agcm.AgcmError) as e:
            agcm.Grid(**kw)
        assert e.value.code == agcm.AGCM_EINVAL
        assert L.agcm_last_error().decode()


def test_null_arguments_are_errors(L):
    assert L.agcm_grid_create(16, 8, 2, None, None, None, None, None) == agcm.AGCM_EINVAL
    assert L.agcm_step(None, 1, 1.0, None) == agcm.AGCM_EINVAL
    assert L.agcm_diagnostics(None, None, None) == agcm.AGCM_EINVAL
    assert L.agcm_state_create(None, 0, 1, None) == agcm.AGCM_EINVAL


def test_cfl_dt_matches_column_eigenproblem(L):
    """R10: dt = 1.6 / ((c_max + umax) * sqrt(...)), c_max^2 = the largest
    eigenvalue of the column operator, here from numpy on a matrix written out."""
    for K, sig in ((8, None), (30, None), (5, [0.0, 0.05, 0.2, 0.5, 0.8, 1.0])):
        I, J = 128, 64
        g = agcm.Grid(I, J, K, sigma_half=sig)
        sh = np.arange(K + 1) / K if sig is None else np.asarray(sig)
        ds = np.diff(sh)
        mid = 0.5 * (sh[:-1] + sh[1:])
        H = np.zeros((K, K))
        for k in range(K):
            H[k, k] = math.log(sh[k + 1] / mid[k])
            for kk in range(k + 1, K):
                H[k, kk] = math.log(sh[kk + 1] / sh[kk])
        R, cp, T0 = 287.04, 1004.64, 250.0
        b2 = (R / cp) * R * T0
        N = b2 * H @ np.diag(1 / ds) @ H.T @ np.diag(ds) + R * T0 * np.outer(np.ones(K), ds)
        cmax = math.sqrt(max(np.linalg.eigvals(N).real))
        a = 6.371e6
        dl, dth = 2 * math.pi / I, math.pi / J
        want = 1.6 / ((cmax + 100.0) * math.hypot(2 / (a * math.cos(math.pi / 4) * dl), 2 / (a * dth)))
        assert abs(g.dt(100.0) / want - 1) < 1e-10


def test_split_dt_rule(L):
    """Advective dt from the flow speed alone, and enough adaptation sub-steps
    for each to respect the gravity-wave dt."""
    g = agcm.Grid(256, 128, 30)
    dt, m = g.dt_split(100.0)
    a = 6.371e6
    dl, dth = 2 * math.pi / 256, math.pi / 128
    want = 1.6 / (100.0 * math.hypot(2 / (a * math.cos(math.pi / 4) * dl), 2 / (a * dth)))
    assert abs(dt / want - 1) < 1e-12
    assert dt / m <= g.dt(0.0) * (1 + 1e-12) and dt / (m - 1) > g.dt(0.0)


def test_thermo_dt_and_validation(L):
    """With a lapse-rate standard atmosphere and Eq. 1's delta_c, delta_p the
    dt rule weights each level's hydrostatic coupling by
    (1 - delta_p)(1 + delta_c) sqrt(kappa R T~(sigma_k)) and uses the largest
    R T~_s; the numpy eigenproblem below is written from that statement."""
    I, J, K = 128, 64, 30
    rng = np.random.default_rng(2)
    phis = np.abs(rng.normal(0, 5e3, (J, I)))
    th = dict(profile=1, Ts0=288.15, lapse=6.5e-3, Ttrop=216.65, delta_c=0.3, delta_p=0.2)
    g = agcm.Grid(I, J, K, phis=phis, thermo=th)
    R, cp, G0 = 287.04, 1004.64, 9.80665
    sh = np.arange(K + 1) / K
    ds, mid = np.diff(sh), 0.5 * (sh[:-1] + sh[1:])
    T = np.maximum(288.15 * mid ** (R * 6.5e-3 / G0), 216.65)
    beta = 0.8 * 1.3 * np.sqrt((R / cp) * R * T)
    H = np.zeros((K, K))
    for k in range(K):
        H[k, k] = math.log(sh[k + 1] / mid[k])
        for kk in range(k + 1, K):
            H[k, kk] = math.log(sh[kk + 1] / sh[kk])
    Ts = 288.15 - 6.5e-3 * phis / G0
    N = H @ np.diag(beta**2 / ds) @ H.T @ np.diag(ds) + R * Ts.max() * np.outer(np.ones(K), ds)
    cmax = math.sqrt(max(np.linalg.eigvals(N).real))
    a = 6.371e6
    dl, dth = 2 * math.pi / I, math.pi / J
    want = 1.6 / ((cmax + 100.0) * math.hypot(2 / (a * math.cos(math.pi / 4) * dl), 2 / (a * dth)))
    assert abs(g.dt(100.0) / want - 1) < 1e-10
    # defaults restored by an explicit default
    g2 = agcm.Grid(I, J, K, phis=phis)
    g.set_thermo()
    assert abs(g.dt(100.0) / g2.dt(100.0) - 1) < 1e-14
    for bad in (dict(profile=3), dict(T0=0.0), dict(delta_p=-0.1), dict(delta_c=-1.0), dict(Ttrop=400.0),
                dict(lapse=float("nan")), dict(delta=float("inf"))):
        with pytest.raises(agcm.AgcmError) as e:
            g.set_thermo(**bad)
        assert e.value.code == agcm.AGCM_EINVAL


def test_header_is_c99_and_links_from_c(L, tmp_path):
    """The boundary is a C ABI: a C99 program includes the header with every
    warning as an error, links against the library and calls its host-only
    entry points (grid geometry, Eq. 7 tables, the dt rule, errors)."""
    import shutil
    import subprocess

    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "abi.c"
    src.write_text(r'''
#include <stdio.h>
#include "agcm.h"
int main(void) {
  agcm_grid_t* g = NULL;
  int32_t lu[64], lv[63];
  double dt = 0.0;
  int msub = 0;
  agcm_thermo_t th = {1, 250.0, 288.15, 6.5e-3, 216.65, 0.0, 0.0, 0.0};
  if (agcm_version() <= 0) return 1;
  if (agcm_grid_create(128, 64, 8, NULL, NULL, NULL, NULL, &g) != AGCM_OK) return 2;
  if (agcm_grid_leap(g, lu, lv) != AGCM_OK || lu[0] < lu[32]) return 3;
  if (agcm_grid_set_thermo(g, &th) != AGCM_OK) return 4;
  if (agcm_grid_dt(g, 100.0, &dt) != AGCM_OK || !(dt > 0.0)) return 5;
  if (agcm_grid_dt_split(g, 100.0, &dt, &msub) != AGCM_OK || msub < 1) return 6;
  if (agcm_grid_destroy(g) != AGCM_OK) return 9;
  if (agcm_grid_create(2, 64, 8, NULL, NULL, NULL, NULL, &g) != AGCM_EINVAL || g != NULL) return 7;
  if (agcm_last_error()[0] == '\0') return 8;
  printf("%d %g %d\n", lu[0], dt, msub);
  return 0;
}
''')
    inc = os.path.join(os.path.dirname(HEADER))
    libdir = os.path.dirname(agcm.LIB_PATH)
    exe = tmp_path / "abi"
    cmd = [gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", inc, str(src), "-o", str(exe),
           "-L", libdir, "-l:" + os.path.basename(agcm.LIB_PATH), "-Wl,-rpath," + libdir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    first, dt, msub = r.stdout.split()
    assert int(first) > 1 and float(dt) > 0 and int(msub) >= 1
