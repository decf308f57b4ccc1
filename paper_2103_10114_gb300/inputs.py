"""Seeded synthetic inputs shared by the tests, the smoke check and the bench.

This module holds no arithmetic of the dynamical core.  It only lays closed-form
or random fields on the grid points of the pole-free offset grid (the paper's
720 x 361 counts imply pole rows; this grid has none):

* scalar / Phi / pi points at longitude ``i*dlam`` and colatitude ``(j+1/2)*dth``;
* U points at longitude ``(i+1/2)*dlam`` on the scalar rows;
* V points at longitude ``i*dlam`` and colatitude ``(j+1)*dth``, ``j < nlat-1``;

with ``dlam = 2 pi / nlon`` and ``dth = pi / nlat``.  V is the component
along increasing colatitude (southward), so a northward wind enters as ``-v``.
Fields are returned in the prognostic variables directly (U, V, Phi in the
IAP units of m/s, pi = p'_sa/p0), float64, storage ``[k][j][i]``.

The paper names its workloads (the Rossby-Haurwitz wave test and F_2000 runs,
Sec. "Validation of AGCM-3DLF") but prints no constants for them; the
amplitudes below are this project's choices; each is stated where it is set.
"""
from __future__ import annotations

import numpy as np

G_ACC = 9.80616  # m/s^2, converts terrain height to surface geopotential
PHI_SCALE = 500.0  # ~ R*T0/b at T0 = 250 K: Phi noise of PHI_SCALE*eps ~ relative T noise eps


def coords(nlon: int, nlat: int):
    dlam = 2.0 * np.pi / nlon
    dth = np.pi / nlat
    lam_s = np.arange(nlon) * dlam
    lam_u = (np.arange(nlon) + 0.5) * dlam
    th_s = (np.arange(nlat) + 0.5) * dth
    th_v = (np.arange(nlat - 1) + 1.0) * dth
    return lam_s, lam_u, th_s, th_v


def _legendre_normalized(lmax: int, x: np.ndarray) -> np.ndarray:
    """Fully normalised associated Legendre functions Pbar[l, m, :] for cos(theta) = x,
    by the standard column recurrences (geodesy normalisation, unit mean square)."""
    s = np.sqrt(np.maximum(0.0, 1.0 - x * x))
    P = np.zeros((lmax + 1, lmax + 1, x.size))
    P[0, 0] = 1.0
    if lmax >= 1:
        P[1, 1] = np.sqrt(3.0) * s
    for m in range(2, lmax + 1):
        P[m, m] = np.sqrt((2.0 * m + 1.0) / (2.0 * m)) * s * P[m - 1, m - 1]
    for m in range(0, lmax + 1):
        for l in range(m + 1, lmax + 1):
            a = np.sqrt((2.0 * l + 1.0) * (2.0 * l - 1.0) / ((l - m) * (l + m)))
            if l - 2 >= m:
                b = np.sqrt((2.0 * l + 1.0) * (l + m - 1.0) * (l - m - 1.0) / ((l - m) * (l + m) * (2.0 * l - 3.0)))
                P[l, m] = a * x * P[l - 1, m] - b * P[l - 2, m]
            else:
                P[l, m] = a * x * P[l - 1, m]
    return P


def terrain_phis(nlon: int, nlat: int, seed: int = 2, lmax: int = 42, hmax: float = 3000.0,
                 slope: float = 1.5) -> np.ndarray:
    """Surface geopotential [m^2/s^2] from a seeded spherical-harmonic series of
    degree <= lmax with coefficient std ~ l^-slope, scaled to a maximum height of
    hmax metres and clipped at sea level (no negative heights)."""
    rng = np.random.default_rng(seed)
    lam_s, _, th_s, _ = coords(nlon, nlat)
    P = _legendre_normalized(lmax, np.cos(th_s))
    h = np.zeros((nlat, nlon))
    for l in range(1, lmax + 1):
        amp = l ** (-slope)
        for m in range(0, l + 1):
            ca, sa = rng.normal(0.0, amp, 2)
            h += P[l, m][:, None] * (ca * np.cos(m * lam_s)[None, :] + (sa * np.sin(m * lam_s)[None, :] if m else 0.0))
    h *= hmax / np.max(np.abs(h))
    h = np.clip(h, 0.0, None)
    return G_ACC * h


def rossby_haurwitz4(nlon: int, nlat: int, nlev: int, seed: int = 1, noise: float = 1e-3,
                     umax: float = 50.0):
    """Wave-number-4 Rossby-Haurwitz flow from the stream function
    psi = -a^2 w sin(phi) + a^2 K cos^4(phi) sin(phi) cos(4 lam), with w = K and
    the pair scaled so that max|u| = umax.  Vertically uniform wind, isothermal
    (Phi = 0), uniform surface pressure (pi = 0), flat terrain, then seeded
    N(0, noise) relative perturbations on U, V, Phi (temperature) and pi."""
    R = 4
    _, lam_u, th_s, th_v = coords(nlon, nlat)
    phi_u = np.pi / 2 - th_s
    phi_v = np.pi / 2 - th_v
    # u = -(1/a) dpsi/dphi and v = (1/(a cos phi)) dpsi/dlam, with a*w = a*K = 1
    cu = np.cos(phi_u)[:, None]
    su = np.sin(phi_u)[:, None]
    u = cu + cu ** (R - 1) * (R * su ** 2 - cu ** 2) * np.cos(R * lam_u)[None, :]
    cv = np.cos(phi_v)[:, None]
    sv = np.sin(phi_v)[:, None]
    lam_s = coords(nlon, nlat)[0]
    v_north = -R * cv ** (R - 1) * sv * np.sin(R * lam_s)[None, :]
    scale = umax / np.max(np.abs(u))
    u = u * scale
    v_north = v_north * scale
    rng = np.random.default_rng(seed)
    U = np.broadcast_to(u, (nlev, nlat, nlon)).copy()
    V = np.broadcast_to(-v_north, (nlev, nlat - 1, nlon)).copy()
    U += rng.normal(0.0, noise * umax, U.shape)
    V += rng.normal(0.0, noise * umax, V.shape)
    Phi = rng.normal(0.0, noise * PHI_SCALE, (nlev, nlat, nlon))
    pi = rng.normal(0.0, noise, (nlat, nlon))
    return {"U": U, "V": V, "Phi": Phi, "pi": pi, "phis": np.zeros((nlat, nlon))}


def sigma_mid(nlev: int):
    return (np.arange(nlev) + 0.5) / nlev


def baroclinic_jet(nlon: int, nlat: int, nlev: int, seed: int = 3, noise: float = 1e-3,
                   terrain_seed: int | None = 2, ujet: float = 35.0):
    """Zonal jet u = ujet exp(-((|lat| - 45deg)/10deg)^2) f(sigma), with the
    vertical profile f = exp(-((sigma - 0.25)/0.3)^2) on uniform mid-levels,
    plus seeded N(0, noise) relative perturbations on U, V, Phi and pi, over
    the seeded terrain of ``terrain_phis`` (flat when terrain_seed is None)."""
    _, _, th_s, _ = coords(nlon, nlat)
    lat = np.degrees(np.pi / 2 - th_s)
    prof = np.exp(-(((np.abs(lat) - 45.0) / 10.0) ** 2))
    f = np.exp(-(((sigma_mid(nlev) - 0.25) / 0.3) ** 2))
    rng = np.random.default_rng(seed)
    U = ujet * f[:, None, None] * prof[None, :, None] * np.ones((1, 1, nlon))
    U = U + rng.normal(0.0, noise * ujet, U.shape)
    V = rng.normal(0.0, noise * ujet, (nlev, nlat - 1, nlon))
    Phi = rng.normal(0.0, noise * PHI_SCALE, (nlev, nlat, nlon))
    pi = rng.normal(0.0, noise, (nlat, nlon))
    phis = terrain_phis(nlon, nlat, seed=terrain_seed) if terrain_seed is not None else np.zeros((nlat, nlon))
    return {"U": U, "V": V, "Phi": Phi, "pi": pi, "phis": phis}


def random_state(nlon: int, nlat: int, nlev: int, seed: int = 0, uamp: float = 20.0,
                 phiamp: float = 50.0, piamp: float = 0.02, terrain: bool = True):
    """White-noise state for algebraic tests (any values are admissible as long
    as pi~ + pi stays positive); optional random terrain up to 3 km."""
    rng = np.random.default_rng(seed)
    st = {
        "U": rng.normal(0.0, uamp, (nlev, nlat, nlon)),
        "V": rng.normal(0.0, uamp, (nlev, nlat - 1, nlon)),
        "Phi": rng.normal(0.0, phiamp, (nlev, nlat, nlon)),
        "pi": rng.normal(0.0, piamp, (nlat, nlon)),
        "phis": (rng.uniform(0.0, 3000.0, (nlat, nlon)) * G_ACC) if terrain else np.zeros((nlat, nlon)),
    }
    return st


def random_direction(nlon: int, nlat: int, nlev: int, seed: int = 4):
    """Unit-scale random perturbation direction (finite-difference and dot tests)."""
    rng = np.random.default_rng(seed)
    return {
        "U": rng.normal(0.0, 1.0, (nlev, nlat, nlon)),
        "V": rng.normal(0.0, 1.0, (nlev, nlat - 1, nlon)),
        "Phi": rng.normal(0.0, 1.0, (nlev, nlat, nlon)),
        "pi": rng.normal(0.0, 1e-3, (nlat, nlon)),
    }


def ensemble_members(seed0: int = 100, noise: float = 1e-2):
    """The 64-member mix: 32 at 256x128x30, 24 at 360x180x30, 8 at 720x360x30,
    member n seeded seed0 + n."""
    shapes = [(256, 128, 30)] * 32 + [(360, 180, 30)] * 24 + [(720, 360, 30)] * 8
    return [(s, seed0 + n, noise) for n, s in enumerate(shapes)]
