"""Pins of the oracle's geometry against what the paper prints (Eq. 7, the
printed N_leap values, and the zonal grid-size table)."""
import math
import os

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    out = []
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                out.append(line.split())
    return out


def test_eq7_printed_values():
    # Eq. 7 with ceil() reproduces "41 or 82" (0.5 deg) and "87 or 173" (0.25 deg)
    rows = _rows("eq7_printed_values.txt")
    assert len(rows) == 4
    for dl, dt, n, want in rows:
        dlam, dth = math.radians(float(dl)), math.radians(float(dt))
        r = oracle.leap_ratio(int(n) * dth, dlam)
        assert math.ceil(r) == int(want), (dl, dt, n, r)


def test_eq7_reference_latitude_is_one():
    # at 45 degrees the spacing is the reference itself (Eq. 7 ratio = 1)
    for res in (0.25, 1.0, 2.8125):
        assert abs(oracle.leap_ratio(math.radians(45.0), math.radians(res)) - 1.0) < 1e-12


def _unit(s):
    return 10.0 ** (-(len(s.split(".")[1]) if "." in s else 0))


def test_tab2_zonal_grid_size():
    rows = _rows("tab2_zonal_grid_size.txt")
    assert len(rows) == 5
    for res, eq, pu, pv in rows:
        d = math.radians(float(res))
        got = [oracle.zonal_dx(math.pi / 2, d), oracle.zonal_dx(d, d), oracle.zonal_dx(d / 2, d)]
        for g, s in zip(got, (eq, pu, pv)):
            assert abs(g / 1000.0 - float(s)) <= _unit(s) + 1e-9, (res, g / 1000.0, s)


@pytest.mark.parametrize("nlon,nlat", [(128, 64), (256, 128), (360, 180), (720, 360), (1440, 720)])
def test_leap_table_properties(nlon, nlat):
    mu, mv = oracle.leap_table(nlon, nlat)
    for M in (mu, mv):
        assert np.all(M >= 1) and np.all(M % 2 == 1) and np.all(2 * M < nlon)
        assert np.array_equal(M, M[::-1])  # north-south symmetric
    dlam, dth = 2 * math.pi / nlon, math.pi / nlat
    th = (np.arange(nlat) + 0.5) * dth
    lat = 90 - np.degrees(th)
    # stride 1 equatorward of 45 degrees, > 1 poleward
    assert np.all(mu[np.abs(lat) < 45.0] == 1)
    assert np.all(mu[np.abs(lat) > 45.0 + 1e-9] > 1)
    # the leap stride keeps every zonal spacing at least the 45-degree spacing
    assert np.all(mu * np.sin(th) >= math.cos(math.pi / 4) * (1 - 1e-6))
    # and never more than needed: one odd step less would fall below it
    big = mu > 1
    assert np.all((mu[big] - 2) * np.sin(th[big]) < math.cos(math.pi / 4))


def test_leap_table_high_resolution_max():
    mu, _ = oracle.leap_table(1440, 720)
    assert mu.max() == 325 and mu[0] == 325


def test_reference_latitude_row_is_stride_one():
    # 64 rows: the V row at colatitude 16*dth is exactly 45 degrees
    mu, mv = oracle.leap_table(128, 64)
    assert mv[15] == 1 and mv[14] > 1
