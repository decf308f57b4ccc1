"""agcm_tendency_static: the allocation-free tendency entry point.

Some callers cannot allocate device memory (an application under a fixed
device-memory budget, or an embedding application whose allocator owns all of
the GPU).  This entry point takes only the caller's input and output buffers
and keeps its scratch in a fixed array inside the library.  The test
checks it, through the C ABI, against agcm_tendency (which allocates its own
state) on two calls in a row, within the tolerances of the parity tests.
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2103_10114_gb300 import agcm, inputs

pytestmark = pytest.mark.gpu
FIELDS = agcm.FIELDS


def _static_tendency(grid, precision, dev_in):
    import torch

    out = {f: torch.empty_like(dev_in[f]) for f in FIELDS}
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = agcm.lib().agcm_tendency_static(grid.handle, precision, *[dev_in[f].data_ptr() for f in FIELDS],
                                         *[out[f].data_ptr() for f in FIELDS], stream)
    agcm.check(rc)
    return out


@pytest.mark.parametrize("precision,tol", [(agcm.AGCM_FP64, 1e-12), (agcm.AGCM_FP32, 1e-6)])
def test_static_tendency_matches_state_path_twice(cuda_ok, precision, tol):
    import torch

    agcm.build()
    cases = [(64, 32, 10, 3), (37, 23, 7, 4)]  # two different grids, one call each, in a row
    for I, J, K, seed in cases:
        st = inputs.baroclinic_jet(I, J, K, seed=seed, noise=1e-2, terrain_seed=2)
        g = agcm.Grid(I, J, K, phis=st["phis"])
        s = agcm.State(g, precision)
        dtype = s.dtype
        dev_in = {f: torch.as_tensor(np.ascontiguousarray(st[f]), dtype=dtype, device="cuda") for f in FIELDS}
        s.load(dev_in)
        ref = s.tendency()
        got = _static_tendency(g, precision, dev_in)
        torch.cuda.synchronize()
        for f in FIELDS:
            r, o = ref[f].double().cpu().numpy(), got[f].double().cpu().numpy()
            err = np.abs(o - r).max() / max(np.abs(r).max(), 1e-300)
            assert err <= tol, (I, J, K, f, err)
        s.close()
        g.close()


def test_static_tendency_rejects_oversized_grid():
    g = agcm.Grid(1440, 720, 30)
    rc = agcm.lib().agcm_tendency_static(g.handle, agcm.AGCM_FP32, *([ctypes.c_void_p(16)] * 8), None)
    assert rc == agcm.AGCM_EINVAL
    assert "static scratch limit" in agcm.lib().agcm_last_error().decode()


@pytest.mark.parametrize("precision,tol", [(agcm.AGCM_FP64, 1e-12), (agcm.AGCM_FP32, 1e-6)])
def test_static_tendency_with_thermodynamics(cuda_ok, precision, tol):
    """The static path builds its own level tables: the lapse-rate profile with
    the nonlinear delta term gives the same tendency as the state path."""
    import torch

    agcm.build()
    I, J, K = 64, 32, 10
    st = inputs.baroclinic_jet(I, J, K, seed=5, noise=1e-2, terrain_seed=2)
    th = dict(profile=1, Ts0=288.15, lapse=6.5e-3, Ttrop=216.65, delta=1.0, delta_c=0.3, delta_p=0.2)
    g = agcm.Grid(I, J, K, phis=st["phis"], thermo=th)
    s = agcm.State(g, precision)
    dev_in = {f: torch.as_tensor(np.ascontiguousarray(st[f]), dtype=s.dtype, device="cuda") for f in FIELDS}
    s.load(dev_in)
    ref = s.tendency()
    got = _static_tendency(g, precision, dev_in)
    torch.cuda.synchronize()
    for f in FIELDS:
        r, o = ref[f].double().cpu().numpy(), got[f].double().cpu().numpy()
        assert np.abs(o - r).max() / max(np.abs(r).max(), 1e-300) <= tol, f
    s.close()
    g.close()


@pytest.mark.parametrize("precision,tol", [(agcm.AGCM_FP64, 1e-12), (agcm.AGCM_FP32, 1e-6)])
def test_static_tendency_more_levels_than_columns(cuda_ok, precision, tol):
    """A 6 x 4 x 30 grid (24 columns, 30 levels) right after a grid with
    another level count: every level table is rebuilt, none is left over."""
    import torch

    agcm.build()
    for I, J, K, seed in [(16, 8, 5, 7), (6, 4, 30, 8), (6, 4, 30, 9)]:
        st = inputs.baroclinic_jet(I, J, K, seed=seed, noise=1e-2, terrain_seed=2)
        ones_u, ones_v = np.ones(J, np.int32), np.ones(J - 1, np.int32)
        g = agcm.Grid(I, J, K, phis=st["phis"], leap_u=ones_u, leap_v=ones_v)
        s = agcm.State(g, precision)
        dev_in = {f: torch.as_tensor(np.ascontiguousarray(st[f]), dtype=s.dtype, device="cuda") for f in FIELDS}
        s.load(dev_in)
        ref = s.tendency()
        got = _static_tendency(g, precision, dev_in)
        torch.cuda.synchronize()
        for f in FIELDS:
            r, o = ref[f].double().cpu().numpy(), got[f].double().cpu().numpy()
            assert np.abs(o - r).max() / max(np.abs(r).max(), 1e-300) <= tol, (I, J, K, f)
        s.close()
        g.close()


def test_static_tendency_reuses_and_rebuilds_tables(cuda_ok):
    """Two calls on one grid reuse the tables the first built; a call on a
    second grid of the same size with other terrain rebuilds them, and a third
    call on the first grid rebuilds them again."""
    import torch

    agcm.build()
    I, J, K = 48, 24, 8
    prec = agcm.AGCM_FP64
    sts = [inputs.baroclinic_jet(I, J, K, seed=11, noise=1e-2, terrain_seed=t) for t in (2, 3)]
    grids = [agcm.Grid(I, J, K, phis=st["phis"]) for st in sts]
    refs, dev_ins = [], []
    for g, st in zip(grids, sts):
        s = agcm.State(g, prec)
        d = {f: torch.as_tensor(np.ascontiguousarray(st[f]), dtype=s.dtype, device="cuda") for f in FIELDS}
        s.load(d)
        refs.append({f: v.double().cpu().numpy() for f, v in s.tendency().items()})
        dev_ins.append(d)
        s.close()
    for q in (0, 0, 1, 0, 1, 1):
        got = _static_tendency(grids[q], prec, dev_ins[q])
        torch.cuda.synchronize()
        for f in FIELDS:
            r, o = refs[q][f], got[f].double().cpu().numpy()
            assert np.abs(o - r).max() / max(np.abs(r).max(), 1e-300) <= 1e-12, (q, f)
    for g in grids:
        g.close()
