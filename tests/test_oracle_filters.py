"""Pins of the oracle's low-latitude filters (Table "Conventional Filtering
scheme"): band boundaries, exact closed-form responses on zonal waves, row
sums (mass) preserved."""
import math

import numpy as np
import pytest

import oracle
from paper_2103_10114_gb300 import inputs


def test_bands():
    band = lambda lat: oracle.filter_band(math.radians(90.0 - lat))
    assert band(0.0) == 1 and band(37.9) == 1 and band(-37.9) == 1
    assert band(38.001) == 2 and band(55.0) == 2 and band(-69.999) == 2
    assert band(70.1) == 0 and band(-89.0) == 0


def _one_row_grid(I, lat):
    """A 1-level grid whose row j sits at latitude `lat` (nearest row)."""
    J = 90
    o = oracle.Oracle(I, J, 1, leap_u=np.ones(J), leap_v=np.ones(J - 1))
    dth = math.pi / J
    j = int(round((math.radians(90.0 - lat)) / dth - 0.5))
    return o, j


@pytest.mark.parametrize("n", [1, 5, 17, 31])
def test_two_grid_wave_removal_leaves_other_waves(n):
    I = 64
    o, j = _one_row_grid(I, 10.0)
    x = np.arange(I)
    st = o.zeros()
    smooth = np.cos(2 * math.pi * n * x / I + 0.3)
    st["Phi"][0, j] = smooth + 2.5 * (-1.0) ** x
    out = o.filter(st)
    assert np.allclose(out["Phi"][0, j], smooth, atol=1e-13)  # the (-1)^x mode is gone, the rest untouched
    again = o.filter(out)
    assert np.allclose(again["Phi"][0, j], out["Phi"][0, j], atol=1e-14)  # idempotent


@pytest.mark.parametrize("n", [1, 8, 16, 32])
@pytest.mark.parametrize("r", [0.25, 0.1])
def test_three_point_response(n, r):
    I = 64
    o, j = _one_row_grid(I, 55.0)
    x = np.arange(I)
    st = o.zeros()
    st["U"][0, j] = np.cos(2 * math.pi * n * x / I)
    out = o.filter(st, r)
    want = (1 - 4 * r * math.sin(math.pi * n / I) ** 2) * st["U"][0, j]
    assert np.allclose(out["U"][0, j], want, atol=1e-13)


def test_polar_rows_untouched_and_mass_kept():
    I, J, K = 32, 24, 3
    st = inputs.random_state(I, J, K, seed=70)
    o = oracle.Oracle(I, J, K, phis=st["phis"])
    out = o.filter(st)
    lat = 90 - np.degrees((np.arange(J) + 0.5) * math.pi / J)
    polar = np.abs(lat) > 70
    assert polar.any()
    assert np.array_equal(out["U"][:, polar], st["U"][:, polar])
    assert not np.allclose(out["U"][:, ~polar], st["U"][:, ~polar])
    # every row sum is kept, so the mass sum A_j (pi~ + pi) is kept
    assert np.allclose(out["pi"].sum(axis=1), st["pi"].sum(axis=1), rtol=0, atol=1e-15)
    assert abs(o.diagnostics(out)["mass"] / o.diagnostics(st)["mass"] - 1) < 1e-15
