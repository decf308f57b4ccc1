"""ctypes binding of ``include/agcm.h`` (libagcm.so, CUDA sm_103a).

Argument marshalling only: every step of the path runs in the library's
kernels.  PyTorch supplies device memory (the library's allocations are routed
through PyTorch's caching allocator) and streams.  If the library has not been
built, every entry point raises; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
_CSRC = os.path.join(_HERE, "csrc")
_BUILD = os.path.join(_HERE, "_build")
LIB_PATH = os.path.join(_BUILD, "libagcm.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

AGCM_OK, AGCM_EINVAL, AGCM_ENOMEM, AGCM_ECUDA, AGCM_ETIMEOUT, AGCM_ENONFINITE = range(6)
AGCM_FP64, AGCM_FP32 = 0, 1
FIELDS = ("U", "V", "Phi", "pi")


def _sources():
    return [os.path.join(_CSRC, f) for f in sorted(os.listdir(_CSRC))] + [os.path.join(_ROOT, "include", "agcm.h")]


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libagcm.so in-tree with nvcc for sm_103a."""
    os.makedirs(_BUILD, exist_ok=True)
    srcs = _sources()
    newest = max(os.path.getmtime(p) for p in srcs)
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= newest:
        return LIB_PATH
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["nvcc", *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
           "-o", tmp, os.path.join(_CSRC, "agcm_api.cu")]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.check_call(cmd)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class AgcmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"agcm error {code}: {msg}")
        self.code = code


_lib = None
_lock = threading.Lock()
_ALLOC_T = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p)
_FREE_T = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)
_alloc_cbs = None

# symbol -> (restype, argtypes)
_vp, _i, _d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
_pi32, _pd = ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)
class Thermo(ctypes.Structure):
    """agcm_thermo_t: standard stratification and Eq. 1's switches."""

    _fields_ = [("profile", ctypes.c_int), ("T0", ctypes.c_double), ("Ts0", ctypes.c_double),
                ("lapse", ctypes.c_double), ("Ttrop", ctypes.c_double), ("delta", ctypes.c_double),
                ("delta_c", ctypes.c_double), ("delta_p", ctypes.c_double)]


THERMO_DEFAULT = dict(profile=0, T0=250.0, Ts0=288.15, lapse=6.5e-3, Ttrop=216.65, delta=0.0, delta_c=0.0,
                      delta_p=0.0)


SIGNATURES = {
    "agcm_last_error": (ctypes.c_char_p, []),
    "agcm_version": (_i, []),
    "agcm_set_allocator": (_i, [_vp, _vp, _vp]),
    "agcm_grid_create": (_i, [_i, _i, _i, _pd, _pi32, _pi32, _pd, ctypes.POINTER(_vp)]),
    "agcm_grid_destroy": (_i, [_vp]),
    "agcm_grid_set_thermo": (_i, [_vp, ctypes.POINTER(Thermo)]),
    "agcm_grid_leap": (_i, [_vp, _pi32, _pi32]),
    "agcm_grid_dt": (_i, [_vp, _d, _pd]),
    "agcm_state_create": (_i, [_vp, _i, _i, ctypes.POINTER(_vp)]),
    "agcm_state_destroy": (_i, [_vp]),
    "agcm_state_load": (_i, [_vp, _vp, _vp, _vp, _vp, _i, _vp]),
    "agcm_state_store": (_i, [_vp, _vp, _vp, _vp, _vp, _i, _vp]),
    "agcm_step": (_i, [_vp, _i, _d, _vp]),
    "agcm_tendency": (_i, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "agcm_step_split": (_i, [_vp, _i, _d, _i, _vp]),
    "agcm_filter": (_i, [_vp, _d, _vp]),
    "agcm_grid_dt_split": (_i, [_vp, _d, _pd, ctypes.POINTER(ctypes.c_int)]),
    "agcm_step_adjoint": (_i, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _d, _vp]),
    "agcm_diagnostics": (_i, [_vp, _vp, _vp]),
    "agcm_profile_enable": (_i, [_vp, _i]),
    "agcm_profile_read": (_i, [_vp, _pd, ctypes.POINTER(ctypes.c_int64)]),
    "agcm_kernel_count": (_i, []),
    "agcm_kernel_name": (ctypes.c_char_p, [_i]),
    "agcm_set_stage_kernel": (_i, [_i]),
    "agcm_state_set_stage_kernel": (_i, [_vp, _i]),
    "agcm_tendency_static": (_i, [_vp, _i, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "agcm_ensemble_create": (_i, [ctypes.POINTER(_vp), _i, ctypes.POINTER(_vp)]),
    "agcm_ensemble_destroy": (_i, [_vp]),
    "agcm_ensemble_configure": (_i, [_vp, _i, _i]),
    "agcm_ensemble_tile": (_i, [_vp, _i]),
    "agcm_ensemble_set_timeout": (_i, [_vp, _d, _i]),
    "agcm_ensemble_step": (_i, [_vp, _i, _pd, _vp]),
    "agcm_ensemble_status": (_i, [_vp, _vp]),
    "agcm_ensemble_profile": (_i, [_vp, _i, _pd, ctypes.POINTER(ctypes.c_int64)]),
}


def lib():
    """Load libagcm.so; raises if it is missing (build it with ``build()``)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libagcm.so is not built ({LIB_PATH}); run paper_2103_10114_gb300.agcm.build()")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def check(rc):
    if rc != AGCM_OK:
        raise AgcmError(rc, lib().agcm_last_error().decode())
    return rc


STAGE_AUTO, STAGE_COLUMN, STAGE_ROW = 0, 1, 2


def set_stage_kernel(choice: int) -> None:
    """agcm_set_stage_kernel: 0 by grid (default), 1 column kernel, 2 row-segment kernel."""
    check(lib().agcm_set_stage_kernel(int(choice)))


def use_torch_allocator():
    """Route the library's device allocations through PyTorch's caching allocator."""
    global _alloc_cbs
    import torch

    if _alloc_cbs is not None:
        return

    def _alloc(n, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(n))
        except Exception:  # reported to the caller as AGCM_ENOMEM
            return None

    def _free(p, ctx):
        torch.cuda.caching_allocator_delete(p)

    _alloc_cbs = (_ALLOC_T(_alloc), _FREE_T(_free))
    check(lib().agcm_set_allocator(ctypes.cast(_alloc_cbs[0], _vp), ctypes.cast(_alloc_cbs[1], _vp), None))


def _stream_ptr(stream=None):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _np_opt(a, dtype, n):
    if a is None:
        return None, None
    arr = np.ascontiguousarray(a, dtype=dtype).reshape(-1)
    if arr.size != n:
        raise ValueError(f"expected {n} values, got {arr.size}")
    return arr, arr.ctypes.data_as(_pi32 if dtype == np.int32 else _pd)


class Grid:
    """agcm_grid_create / agcm_grid_leap / agcm_grid_dt."""

    def __init__(self, nlon, nlat, nlev, sigma_half=None, leap_u=None, leap_v=None, phis=None, thermo=None):
        self.nlon, self.nlat, self.nlev = int(nlon), int(nlat), int(nlev)
        _, psh = _np_opt(sigma_half, np.float64, self.nlev + 1)
        _, plu = _np_opt(leap_u, np.int32, self.nlat)
        _, plv = _np_opt(leap_v, np.int32, self.nlat - 1)
        self._keep = [sigma_half, leap_u, leap_v, phis]
        _, pph = _np_opt(phis, np.float64, self.nlat * self.nlon)
        h = _vp()
        check(lib().agcm_grid_create(self.nlon, self.nlat, self.nlev, psh, plu, plv, pph, ctypes.byref(h)))
        self._h = h
        if thermo is not None:
            self.set_thermo(**thermo)

    def set_thermo(self, **kw):
        """agcm_grid_set_thermo: keys of THERMO_DEFAULT; before the first state."""
        t = dict(THERMO_DEFAULT)
        unknown = set(kw) - set(t)
        if unknown:
            raise ValueError(f"unknown thermo keys {sorted(unknown)}")
        t.update(kw)
        v = Thermo(int(t["profile"]), *(float(t[k]) for k in list(THERMO_DEFAULT)[1:]))
        check(lib().agcm_grid_set_thermo(self._h, ctypes.byref(v)))

    @property
    def handle(self):
        return self._h

    def leap(self):
        lu = np.zeros(self.nlat, np.int32)
        lv = np.zeros(max(self.nlat - 1, 1), np.int32)
        check(lib().agcm_grid_leap(self._h, lu.ctypes.data_as(_pi32), lv.ctypes.data_as(_pi32)))
        return lu, lv[: self.nlat - 1]

    def dt(self, umax=100.0):
        out = ctypes.c_double()
        check(lib().agcm_grid_dt(self._h, float(umax), ctypes.byref(out)))
        return out.value

    def dt_split(self, umax=100.0):
        """(advective dt, adaptation sub-steps per step) for agcm_step_split."""
        dt, m = ctypes.c_double(), ctypes.c_int()
        check(lib().agcm_grid_dt_split(self._h, float(umax), ctypes.byref(dt), ctypes.byref(m)))
        return dt.value, m.value

    def shapes(self):
        K, J, I = self.nlev, self.nlat, self.nlon
        return {"U": (K, J, I), "V": (K, J - 1, I), "Phi": (K, J, I), "pi": (J, I)}

    def points(self):
        return self.nlon * self.nlat * self.nlev

    def close(self):
        if getattr(self, "_h", None):
            check(lib().agcm_grid_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class State:
    """agcm_state_* / agcm_step / agcm_tendency / agcm_step_adjoint / agcm_diagnostics."""

    def __init__(self, grid: Grid, precision=AGCM_FP64, torch_alloc=True):
        import torch

        if torch_alloc:
            use_torch_allocator()
        self.grid = grid
        self.precision = precision
        self.dtype = torch.float64 if precision == AGCM_FP64 else torch.float32
        h = _vp()
        check(lib().agcm_state_create(grid.handle, int(precision), 1, ctypes.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def _dev(self, st, device="cuda"):
        import torch

        out = []
        for f in FIELDS:
            a = st[f]
            t = a if isinstance(a, torch.Tensor) else torch.from_numpy(np.asarray(a))
            t = t.to(device=device, dtype=self.dtype).contiguous()
            if tuple(t.shape) != self.grid.shapes()[f]:
                t = t.reshape(self.grid.shapes()[f])
            out.append(t)
        return out

    def empty(self):
        import torch

        return {f: torch.empty(s, dtype=self.dtype, device="cuda") for f, s in self.grid.shapes().items()}

    def load(self, st, stream=None):
        ts = self._dev(st)
        check(lib().agcm_state_load(self._h, *[t.data_ptr() for t in ts], 1, _stream_ptr(stream)))
        self._last_load = ts  # keep alive until the copy is done
        return self

    def _check_host(self, host):
        """The copies read or write whole fields through raw pointers: every host
        tensor must be a contiguous CPU tensor of the state's dtype and size."""
        shapes = self.grid.shapes()
        for f in FIELDS:
            t = host[f]
            n = int(np.prod(shapes[f]))
            if t.device.type != "cpu" or t.dtype != self.dtype or not t.is_contiguous() or t.numel() != n:
                raise ValueError(f"host field {f}: need a contiguous CPU {self.dtype} tensor of {n} values, "
                                 f"got {t.device} {t.dtype} with {t.numel()} values")

    def load_host(self, host, stream=None):
        """host: dict of CPU tensors of the state's dtype (pinned for asynchronous copies)."""
        self._check_host(host)
        check(lib().agcm_state_load(self._h, *[host[f].data_ptr() for f in FIELDS], 0, _stream_ptr(stream)))

    def store_host(self, host, stream=None):
        self._check_host(host)
        check(lib().agcm_state_store(self._h, *[host[f].data_ptr() for f in FIELDS], 0, _stream_ptr(stream)))

    def store(self, stream=None):
        out = self.empty()
        check(lib().agcm_state_store(self._h, *[out[f].data_ptr() for f in FIELDS], 1, _stream_ptr(stream)))
        return out

    def step(self, nsteps, dt, stream=None):
        check(lib().agcm_step(self._h, int(nsteps), float(dt), _stream_ptr(stream)))

    def capture(self, nsteps, dt):
        """A CUDA graph of agcm_step(nsteps, dt) on this state; replay it with
        graph.replay().  The captured call starts by recomputing the FP64 column
        means from x_n, so a replay stays valid after any load."""
        import torch

        self.load(self.store())  # marks the column means stale, so the capture recomputes them
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        q = torch.cuda.Stream()
        q.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(q):
            with torch.cuda.graph(g, stream=q):
                self.step(nsteps, dt, stream=q)
        torch.cuda.current_stream().wait_stream(q)
        return g

    def filter(self, r=0.25, stream=None):
        check(lib().agcm_filter(self._h, float(r), _stream_ptr(stream)))

    def step_split(self, nsteps, dt, msub, stream=None):
        check(lib().agcm_step_split(self._h, int(nsteps), float(dt), int(msub), _stream_ptr(stream)))

    def tendency(self, stream=None):
        out = self.empty()
        check(lib().agcm_tendency(self._h, *[out[f].data_ptr() for f in FIELDS], _stream_ptr(stream)))
        return out

    def step_adjoint(self, lam_in, dt, stream=None):
        lin = self._dev(lam_in)
        out = self.empty()
        arr_in = (_vp * 4)(*[t.data_ptr() for t in lin])
        arr_out = (_vp * 4)(*[out[f].data_ptr() for f in FIELDS])
        check(lib().agcm_step_adjoint(self._h, arr_in, arr_out, float(dt), _stream_ptr(stream)))
        self._last_adj = lin
        return out

    def diagnostics(self, stream=None):
        buf = (ctypes.c_double * 8)()
        rc = lib().agcm_diagnostics(self._h, ctypes.cast(buf, _vp), _stream_ptr(stream))
        vals = list(buf)
        finite = ctypes.cast(ctypes.byref(buf, 7 * 8), ctypes.POINTER(ctypes.c_int32))[0]
        d = dict(zip(("mass", "e_kin", "e_pot", "e_ps", "energy", "max_u", "max_v"), vals[:7]))
        d["finite"] = int(finite)
        if rc not in (AGCM_OK, AGCM_ENONFINITE):
            check(rc)
        return d

    def set_stage_kernel(self, choice):
        """agcm_state_set_stage_kernel: 0 the process's choice (default), 1 column
        kernel, 2 row-segment kernel, for this state only."""
        check(lib().agcm_state_set_stage_kernel(self._h, int(choice)))

    def profile(self, enable=True):
        check(lib().agcm_profile_enable(self._h, 1 if enable else 0))

    def profile_read(self):
        """{kernel name: (total ms, launches)} since profile(True)."""
        n = lib().agcm_kernel_count()
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_int64 * n)()
        check(lib().agcm_profile_read(self._h, ms, cnt))
        return {lib().agcm_kernel_name(q).decode(): (ms[q], cnt[q]) for q in range(n) if cnt[q]}

    def close(self):
        if getattr(self, "_h", None):
            check(lib().agcm_state_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
