"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (reading R11, normwise per field, max|gpu - orc| / max|orc|):
  FP64: 1e-12 for one tendency or one step (rounding-order differences only;
        the column sums run as scans on the GPU and as plain sums in the oracle);
        1e-10 after 20 steps (round-off growth of a nonlinear flow).
  FP32 with FP64 column sums: 1e-5 after one step (the stated precision target).
"""
import numpy as np
import pytest

import oracle
from paper_2103_10114_gb300 import agcm, inputs

pytestmark = pytest.mark.gpu
FIELDS = agcm.FIELDS


@pytest.fixture(scope="module", autouse=True)
def _built(cuda_ok):
    agcm.build()
    agcm.lib()


def rel_err(a, b):
    den = np.abs(b).max()
    return np.abs(a - b).max() / (den if den > 0 else 1.0)


def to_np(d):
    return {f: v.double().cpu().numpy() for f, v in d.items()}


CASES = [
    # (nlon, nlat, nlev, kind, extra)
    (16, 10, 4, "random", {}),
    (12, 8, 3, "random", {"sigma_half": [0.0, 0.1, 0.45, 1.0]}),
    (20, 9, 5, "random", {"rand_leap": True}),
    (37, 23, 7, "random", {}),  # ragged sizes, odd nlat
    (3, 2, 1, "random", {"ones": True}),  # smallest grid: one V row
    (5, 3, 1, "random", {"ones": True}),  # Eq. 7 would ask for 2M >= nlon here
    (128, 64, 8, "rh4", {}),
    (256, 128, 30, "jet", {}),
    # the stride-1 row band (interior rows whose Mu_j, Mv_j, Mu_{j+1} are 1)
    # runs a specialised column body beside the general one
    (24, 10, 4, "random", {"ones": True}),  # band = rows 1..J-3, general body for 0, J-2, J-1
    (24, 4, 3, "random", {"ones": True}),  # a one-row band
    (30, 14, 5, "random", {"two_runs": True}),  # the shorter stride-1 run takes the general body
]


def make_case(nlon, nlat, nlev, kind, extra, seed=11):
    if kind == "random":
        st = inputs.random_state(nlon, nlat, nlev, seed=seed)
    elif kind == "rh4":
        st = inputs.rossby_haurwitz4(nlon, nlat, nlev, seed=1)
    else:
        st = inputs.baroclinic_jet(nlon, nlat, nlev, seed=3, terrain_seed=2)
    mu = mv = None
    if extra.get("rand_leap"):
        rng = np.random.default_rng(seed + 100)
        mu = 2 * rng.integers(0, (nlon - 1) // 4 + 1, nlat) + 1
        mv = 2 * rng.integers(0, (nlon - 1) // 4 + 1, nlat - 1) + 1
    if extra.get("ones"):
        mu, mv = np.ones(nlat, np.int32), np.ones(nlat - 1, np.int32)
    if extra.get("two_runs"):  # stride-1 runs at rows 1-2 and 6-10
        mu = np.array([3, 1, 1, 1, 3, 3, 1, 1, 1, 1, 1, 1, 3, 3], np.int32)
        mv = np.ones(nlat - 1, np.int32)
        mv[4] = 3
    sig = extra.get("sigma_half")
    g = agcm.Grid(nlon, nlat, nlev, sigma_half=sig, leap_u=mu, leap_v=mv, phis=st["phis"])
    o = oracle.Oracle(nlon, nlat, nlev, sigma_half=sig, leap_u=mu, leap_v=mv, phis=st["phis"])
    return g, o, st


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}x{c[2]}-{c[3]}")
def test_tendency_fp64(case, stage_kernel):
    g, o, st = make_case(*case)
    s = agcm.State(g, agcm.AGCM_FP64)
    s.load(st)
    t = to_np(s.tendency())
    ref = o.tendency(st)
    for f in FIELDS:
        assert rel_err(t[f], ref[f]) <= 1e-12, (f, rel_err(t[f], ref[f]))


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}x{c[2]}-{c[3]}")
def test_one_step_fp64_and_fp32(case, stage_kernel):
    g, o, st = make_case(*case)
    dt = g.dt(100.0)
    ref = o.step(st, dt, 1)
    for prec, tol in ((agcm.AGCM_FP64, 1e-12), (agcm.AGCM_FP32, 1e-5)):
        s = agcm.State(g, prec)
        s.load(st)
        s.step(1, dt)
        out = to_np(s.store())
        for f in FIELDS:
            assert rel_err(out[f], ref[f]) <= tol, (prec, f, rel_err(out[f], ref[f]))


def test_config1_twenty_steps(stage_kernel):
    """128 x 64 x 8 R-H wave, 20 steps at the CFL dt: FP64 parity, and the
    energy / mass drift of the GPU run equal the oracle's."""
    g, o, st = make_case(128, 64, 8, "rh4", {})
    dt = g.dt(100.0)
    ref = o.step(st, dt, 20)
    s = agcm.State(g, agcm.AGCM_FP64)
    s.load(st)
    d0 = s.diagnostics()
    s.step(20, dt)
    out = to_np(s.store())
    for f in FIELDS:
        assert rel_err(out[f], ref[f]) <= 1e-10, (f, rel_err(out[f], ref[f]))
    d1 = s.diagnostics()
    r0, r1 = o.diagnostics(st), o.diagnostics(ref)
    assert abs(d1["mass"] / d0["mass"] - 1) < 1e-13
    drift_gpu = d1["energy"] / d0["energy"] - 1
    drift_orc = r1["energy"] / r0["energy"] - 1
    assert abs(drift_gpu - drift_orc) <= 1e-8 * abs(drift_orc) + 1e-15


@pytest.mark.parametrize("prec", [agcm.AGCM_FP64, agcm.AGCM_FP32])
def test_diagnostics_match_oracle(prec):
    g, o, st = make_case(37, 23, 7, "random", {})
    s = agcm.State(g, prec)
    s.load(st)
    d = s.diagnostics()
    ref = o.diagnostics(to_np(s.store()))  # same (rounded) state on both sides
    for k in ("mass", "e_kin", "e_pot", "e_ps", "energy", "max_u", "max_v"):
        assert abs(d[k] - ref[k]) <= 1e-12 * abs(ref[k]), (k, d[k], ref[k])
    assert d["finite"] == 1


def test_diagnostics_flag_nonfinite():
    g, o, st = make_case(16, 10, 4, "random", {})
    st = dict(st)
    st["Phi"] = st["Phi"].copy()
    st["Phi"][1, 2, 3] = np.nan
    s = agcm.State(g, agcm.AGCM_FP64)
    s.load(st)
    d = s.diagnostics()
    assert d["finite"] == 0


def test_energy_neutral_on_gpu_full_size():
    """<x, T(x)>_W = 0 holds at any size: check it on the 1440 x 720 x 30 grid
    (the bench workload) in FP64 with weights written from the closed form."""
    import math

    I, J, K = 1440, 720, 30
    st = inputs.baroclinic_jet(I, J, K, seed=5, noise=1e-2, terrain_seed=2)
    g = agcm.Grid(I, J, K, phis=st["phis"])
    s = agcm.State(g, agcm.AGCM_FP64)
    s.load(st)
    t = to_np(s.tendency())
    a = 6.371e6
    dl, dth = 2 * math.pi / I, math.pi / J
    A = a * a * np.sin((np.arange(J) + 0.5) * dth) * dth * dl
    Av = a * a * np.sin((np.arange(J - 1) + 1.0) * dth) * dth * dl
    ds = 1.0 / K
    pit = np.exp(-st["phis"] / (287.04 * 250.0))
    terms = [
        ds * A[None, :, None] * st["U"] * t["U"],
        ds * Av[None, :, None] * st["V"] * t["V"],
        ds * A[None, :, None] * st["Phi"] * t["Phi"],
        A[:, None] * (287.04 * 250.0 / pit) * st["pi"] * t["pi"],
    ]
    tot = sum(float(np.sum(x)) for x in terms)
    mag = sum(float(np.sum(np.abs(x))) for x in terms)
    assert abs(tot) <= 1e-12 * mag, tot / mag
    # and the mass tendency integrates to zero
    assert abs(np.sum(A[:, None] * t["pi"])) <= 1e-13 * np.sum(A[:, None] * np.abs(t["pi"]))


@pytest.mark.parametrize("prec", [agcm.AGCM_FP64, agcm.AGCM_FP32], ids=["fp64", "fp32"])
def test_stage_kernels_are_deterministic(prec, stage_kernel):
    """Every output element of a stage has one writer and every read is
    ordered by the kernel's barriers, so the tendency and a step are the same
    bit for bit on fresh states; 720 x 360 x 30 spans every stride class and
    the polar rows, with several waves of CTAs."""
    import torch

    I, J, K = 720, 360, 30
    st = inputs.baroclinic_jet(I, J, K, seed=5, noise=1e-2, terrain_seed=2)
    g = agcm.Grid(I, J, K, phis=st["phis"])
    dt = g.dt(100.0)
    ref = None
    for _ in range(3):
        s = agcm.State(g, prec)
        s.load(st)
        t = {f: v.clone() for f, v in s.tendency().items()}
        s.step(2, dt)
        x = s.store()
        torch.cuda.synchronize()
        if ref is None:
            ref = (t, x)
        else:
            for f in FIELDS:
                assert torch.equal(t[f], ref[0][f]), ("tendency", f)
                assert torch.equal(x[f], ref[1][f]), ("step", f)
        s.close()


def test_full_size_one_step_fp32():
    """The bench workload itself (1440 x 720 x 30, FP32 with FP64 column sums,
    the same launch path as bench.py): one step against the FP64 oracle."""
    I, J, K = 1440, 720, 30
    st = inputs.baroclinic_jet(I, J, K, seed=5, noise=1e-2, terrain_seed=2)
    g = agcm.Grid(I, J, K, phis=st["phis"])
    dt = g.dt(100.0)
    s = agcm.State(g, agcm.AGCM_FP32)
    s.load(st)
    s.step(1, dt)
    out = to_np(s.store())
    s.close()
    ref = oracle.Oracle(I, J, K, phis=st["phis"]).step(st, dt, 1)
    for f in FIELDS:
        assert rel_err(out[f], ref[f]) <= 1e-5, (f, rel_err(out[f], ref[f]))


def test_allocation_failure_is_reported_and_leaks_nothing():
    """An allocator that refuses after a few allocations: agcm_state_create
    returns AGCM_ENOMEM and frees what it had; the default allocator then works."""
    import ctypes

    L = agcm.lib()
    calls = {"n": 0, "live": set()}

    def alloc(n, ctx):
        calls["n"] += 1
        if calls["n"] > 5:
            return None
        import torch

        p = torch.cuda.caching_allocator_alloc(int(n))
        calls["live"].add(p)
        return p

    def free(p, ctx):
        import torch

        calls["live"].discard(p)
        torch.cuda.caching_allocator_delete(p)

    A = agcm._ALLOC_T(alloc)
    F = agcm._FREE_T(free)
    agcm.check(L.agcm_set_allocator(ctypes.cast(A, ctypes.c_void_p), ctypes.cast(F, ctypes.c_void_p), None))
    try:
        g = agcm.Grid(24, 12, 3)
        h = ctypes.c_void_p()
        rc = L.agcm_state_create(g.handle, agcm.AGCM_FP64, 1, ctypes.byref(h))
        assert rc == agcm.AGCM_ENOMEM
        assert "allocation" in L.agcm_last_error().decode()
        live_after = len(calls["live"])
        assert live_after <= 1  # only the grid's tables stay (owned by the grid)
    finally:
        agcm._alloc_cbs = None
        agcm.use_torch_allocator()
    s = agcm.State(g, agcm.AGCM_FP64)
    s.close()


def _oracle_split(o, st, dt, msub, nsteps):
    """The split step from the oracle's term groups: msub three-stage steps of
    the adaptation terms with dt/msub, then one of the advection terms with dt."""
    ada = oracle.TERM_COR | oracle.TERM_PGF_PI | oracle.TERM_PGF_PHI
    x = {f: st[f] for f in FIELDS}
    for _ in range(nsteps):
        x = o.step(x, dt / msub, msub, terms=ada)
        x = o.step(x, dt, 1, terms=oracle.TERM_ADV)
    return x


@pytest.mark.parametrize("case", [(37, 23, 7, "random", {}), (128, 64, 8, "rh4", {}), (256, 128, 30, "jet", {})],
                         ids=lambda c: f"{c[0]}x{c[1]}x{c[2]}")
def test_split_step_matches_oracle(case, stage_kernel):
    g, o, st = make_case(*case)
    dt, msub = g.dt_split(100.0)
    assert msub >= 2
    ref = _oracle_split(o, st, dt, msub, 2)
    for prec, tol in ((agcm.AGCM_FP64, 1e-11), (agcm.AGCM_FP32, 1e-5)):
        s = agcm.State(g, prec)
        s.load(st)
        s.step_split(2, dt, msub)
        out = to_np(s.store())
        for f in FIELDS:
            assert rel_err(out[f], ref[f]) <= tol, (prec, f, rel_err(out[f], ref[f]))
        s.close()


@pytest.mark.parametrize("prec", [agcm.AGCM_FP64, agcm.AGCM_FP32])
def test_zonal_translation_invariance_on_gpu(prec, stage_kernel):
    """Shifting every field (and the terrain) by s longitudes shifts the GPU
    tendency and step by s, bit for bit: no column is treated differently,
    whether its leap partners wrap across the seam or it sits in a ragged
    last warp (nlon = 100)."""
    I, J, K, shift = 100, 48, 8, 37
    st = inputs.baroclinic_jet(I, J, K, seed=3, noise=1e-2, terrain_seed=2)
    phis = np.asarray(st["phis"]).reshape(J, I)
    g = agcm.Grid(I, J, K, phis=phis)
    gs = agcm.Grid(I, J, K, phis=np.roll(phis, shift, axis=-1))
    x = {f: st[f] for f in FIELDS}
    xs = {f: np.roll(np.asarray(v), shift, axis=-1) for f, v in x.items()}
    dt = g.dt(100.0)
    a, b = agcm.State(g, prec), agcm.State(gs, prec)
    a.load(x)
    b.load(xs)
    ta, tb = to_np(a.tendency()), to_np(b.tendency())
    for f in FIELDS:
        assert np.array_equal(np.roll(ta[f], shift, axis=-1), tb[f]), ("tendency", f)
    a.step(2, dt)
    b.step(2, dt)
    ya, yb = to_np(a.store()), to_np(b.store())
    for f in FIELDS:
        assert np.array_equal(np.roll(ya[f], shift, axis=-1), yb[f]), ("step", f)
    a.close()
    b.close()
