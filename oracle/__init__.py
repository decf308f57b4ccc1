"""Oracle for the leap-format IAP dynamical-core step (arXiv 2103.10114).

TEST INFRASTRUCTURE ONLY.  A ctypes wrapper around ``orc_agcm.cpp``, the plain
FP64 CPU statement of the scheme.  Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
this package.  The product library never depends on it, and it shares no code
with the product library.

Arrays follow the same storage order as the product: ``U, Phi: [K][J][I]``,
``V: [K][J-1][I]``, ``pi: [J][I]``, longitude fastest, float64.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "orc_agcm.cpp")
_LIB = os.path.join(_HERE, "_build", "liborc_agcm.so")

TERM_ADV = 1
TERM_COR = 2
TERM_PGF_PI = 4
TERM_PGF_PHI = 8
TERM_ALL = 15


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (no fast-math, portable flags)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def bind(cdll):
    """Declare the oracle's C signatures on a loaded library and return it."""
    d, i32, vp = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p
    cdll.orc_leap_ratio.restype = ctypes.c_double
    cdll.orc_leap_ratio.argtypes = [ctypes.c_double, ctypes.c_double]
    cdll.orc_zonal_dx.restype = ctypes.c_double
    cdll.orc_zonal_dx.argtypes = [ctypes.c_double, ctypes.c_double]
    cdll.orc_leap_table.argtypes = [ctypes.c_int, ctypes.c_int, i32, i32]
    cdll.orc_create.restype = vp
    cdll.orc_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, d, i32, i32, d]
    cdll.orc_destroy.argtypes = [vp]
    cdll.orc_get_leap.argtypes = [vp, i32, i32]
    cdll.orc_tendency.argtypes = [vp] + [d] * 8 + [ctypes.c_uint]
    cdll.orc_step.argtypes = [vp] + [d] * 4 + [ctypes.c_double, ctypes.c_int, ctypes.c_uint]
    cdll.orc_tendency_jvp.argtypes = [vp] + [d] * 12 + [ctypes.c_uint]
    cdll.orc_step_jvp.argtypes = [vp] + [d] * 8 + [ctypes.c_double, ctypes.c_int, ctypes.c_uint]
    cdll.orc_diagnostics.argtypes = [vp] + [d] * 5
    cdll.orc_filter_band.restype = ctypes.c_int
    cdll.orc_filter_band.argtypes = [ctypes.c_double]
    cdll.orc_filter.argtypes = [vp] + [d] * 4 + [ctypes.c_double]
    cdll.orc_set_thermo.restype = ctypes.c_int
    cdll.orc_set_thermo.argtypes = [vp, d]
    cdll.orc_std_temp.restype = ctypes.c_double
    cdll.orc_std_temp.argtypes = [d, ctypes.c_double]
    cdll.orc_std_surface.argtypes = [d, ctypes.c_double, d]
    cdll.orc_tendency_opcount.argtypes = [vp] + [d] * 8 + [ctypes.c_uint, ctypes.POINTER(ctypes.c_ulonglong)]
    return cdll


def lib():
    global _lib
    if _lib is None:
        _lib = bind(ctypes.CDLL(build()))
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def leap_ratio(theta: float, dlam: float) -> float:
    """Eq. 7 before rounding: spacing at 45 degrees over spacing at colatitude theta."""
    return lib().orc_leap_ratio(theta, dlam)


def zonal_dx(theta: float, dlam: float) -> float:
    """Zonal grid size a sin(theta) dlam in metres."""
    return lib().orc_zonal_dx(theta, dlam)


def filter_band(colat: float) -> int:
    """0: none, 1: two-grid-wave removal (|lat| < 38), 2: 3-point (38..70)."""
    return lib().orc_filter_band(colat)


def leap_table(nlon: int, nlat: int):
    mu = np.zeros(nlat, np.int32)
    mv = np.zeros(max(nlat - 1, 1), np.int32)
    lib().orc_leap_table(nlon, nlat, _ip(mu), _ip(mv))
    return mu, mv[: nlat - 1]


FIELDS = ("U", "V", "Phi", "pi")

# Standard stratification and Eq. 1's switches (readings T1..T4); the default
# is the isothermal 250 K atmosphere with every switch off.
THERMO_DEFAULT = dict(profile=0, T0=250.0, Ts0=288.15, lapse=6.5e-3, Ttrop=216.65, delta=0.0, delta_c=0.0,
                      delta_p=0.0)
_THERMO_KEYS = ("profile", "T0", "Ts0", "lapse", "Ttrop", "delta", "delta_c", "delta_p")


def _thermo_vec(thermo):
    t = dict(THERMO_DEFAULT)
    t.update(thermo or {})
    unknown = set(t) - set(_THERMO_KEYS)
    if unknown:
        raise ValueError(f"unknown thermo keys {sorted(unknown)}")
    return np.array([float(t[k]) for k in _THERMO_KEYS])


def std_temp(p_over_p0, **thermo):
    """T~ at p / p0 of the standard stratification (reading T1)."""
    v = _thermo_vec(thermo)
    return lib().orc_std_temp(_dp(v), float(p_over_p0))


def std_surface(phis, **thermo):
    """(pi~, T~_s): standard surface pressure / p0 and temperature under phis (T3)."""
    v = _thermo_vec(thermo)
    out = np.zeros(2)
    lib().orc_std_surface(_dp(v), float(phis), _dp(out))
    return float(out[0]), float(out[1])


class Oracle:
    """One grid of the oracle.  ``state`` arguments are dicts with keys U, V, Phi, pi."""

    def __init__(self, nlon, nlat, nlev, sigma_half=None, leap_u=None, leap_v=None, phis=None, thermo=None):
        self.I, self.J, self.K = int(nlon), int(nlat), int(nlev)
        keep = []

        def opt(a, dtype, n):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=dtype).reshape(-1)
            assert a.size == n
            keep.append(a)
            return a

        sh = opt(sigma_half, np.float64, self.K + 1)
        mu = opt(leap_u, np.int32, self.J)
        mv = opt(leap_v, np.int32, self.J - 1)
        ph = opt(phis, np.float64, self.J * self.I)
        self._L = L = lib()
        self._h = L.orc_create(
            self.I, self.J, self.K,
            _dp(sh) if sh is not None else None,
            _ip(mu) if mu is not None else None,
            _ip(mv) if mv is not None else None,
            _dp(ph) if ph is not None else None,
        )
        if not self._h:
            raise ValueError("oracle rejected the grid arguments")
        if thermo is not None:
            v = _thermo_vec(thermo)
            if L.orc_set_thermo(self._h, _dp(v)) != 0:
                raise ValueError("oracle rejected the thermo arguments")
        self.leap_u = np.zeros(self.J, np.int32)
        self.leap_v = np.zeros(max(self.J - 1, 1), np.int32)
        L.orc_get_leap(self._h, _ip(self.leap_u), _ip(self.leap_v))
        self.leap_v = self.leap_v[: self.J - 1]

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._L.orc_destroy(h)
            self._h = None

    # -- shapes ----------------------------------------------------------
    def shapes(self):
        K, J, I = self.K, self.J, self.I
        return {"U": (K, J, I), "V": (K, J - 1, I), "Phi": (K, J, I), "pi": (J, I)}

    def _in(self, st):
        sh = self.shapes()
        return [np.ascontiguousarray(st[f], dtype=np.float64).reshape(sh[f]) for f in FIELDS]

    def zeros(self):
        return {f: np.zeros(s) for f, s in self.shapes().items()}

    # -- calls -----------------------------------------------------------
    def tendency(self, st, terms=TERM_ALL):
        x = self._in(st)
        t = self.zeros()
        self._L.orc_tendency(self._h, *[_dp(a) for a in x], *[_dp(t[f]) for f in FIELDS], terms)
        return t

    def tendency_opcount(self, st, terms=TERM_ALL):
        """The tendency evaluated through the counting type: (tendency, counts)
        with counts of adds (incl. subtracts), multiplies, divides and square
        roots on state values."""
        x = self._in(st)
        t = self.zeros()
        ops = (ctypes.c_ulonglong * 4)()
        self._L.orc_tendency_opcount(self._h, *[_dp(a) for a in x], *[_dp(t[f]) for f in FIELDS], terms, ops)
        return t, dict(zip(("add", "mul", "div", "sqrt"), [int(v) for v in ops]))

    def step(self, st, dt, nsteps=1, terms=TERM_ALL):
        x = [a.copy() for a in self._in(st)]
        self._L.orc_step(self._h, *[_dp(a) for a in x], float(dt), int(nsteps), terms)
        return dict(zip(FIELDS, x))

    def tendency_jvp(self, st, dst, terms=TERM_ALL):
        x, dx = self._in(st), self._in(dst)
        j = self.zeros()
        self._L.orc_tendency_jvp(self._h, *[_dp(a) for a in x], *[_dp(a) for a in dx],
                               *[_dp(j[f]) for f in FIELDS], terms)
        return j

    def step_jvp(self, st, dst, dt, nsteps=1, terms=TERM_ALL):
        """Returns (state after nsteps, Jacobian of the nsteps map applied to dst)."""
        x = [a.copy() for a in self._in(st)]
        dx = [a.copy() for a in self._in(dst)]
        self._L.orc_step_jvp(self._h, *[_dp(a) for a in x], *[_dp(a) for a in dx], float(dt),
                           int(nsteps), terms)
        return dict(zip(FIELDS, x)), dict(zip(FIELDS, dx))

    def filter(self, st, r=0.25):
        """Low-latitude filters (Table "Conventional Filtering scheme"), a new state."""
        x = [a.copy() for a in self._in(st)]
        self._L.orc_filter(self._h, *[_dp(a) for a in x], float(r))
        return dict(zip(FIELDS, x))

    def diagnostics(self, st):
        x = self._in(st)
        out = np.zeros(8)
        self._L.orc_diagnostics(self._h, *[_dp(a) for a in x], _dp(out))
        keys = ("mass", "e_kin", "e_pot", "e_ps", "energy", "max_u", "max_v", "finite")
        return dict(zip(keys, out.tolist()))
