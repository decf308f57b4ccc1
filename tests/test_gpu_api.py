"""The C ABI's contract on the GPU: states on different streams do not
interfere (the library keeps no hidden mutable state between them), argument
errors are refused with AGCM_EINVAL and leave the state usable, and the
per-kernel profiler counts what ran."""
import ctypes

import numpy as np
import pytest

from paper_2103_10114_gb300 import agcm, inputs

pytestmark = pytest.mark.gpu
FIELDS = agcm.FIELDS


@pytest.fixture(scope="module", autouse=True)
def _built(cuda_ok):
    agcm.build()
    agcm.lib()


def to_np(d):
    return {f: v.double().cpu().numpy() for f, v in d.items()}


@pytest.mark.parametrize("prec", [agcm.AGCM_FP32, agcm.AGCM_FP64])
def test_concurrent_states_on_streams_match_sequential(prec):
    import torch

    cases = [(128, 64, 8, 3), (96, 48, 6, 4), (128, 64, 8, 5)]  # two share a grid shape
    grids, states, ref = [], [], []
    for I, J, K, seed in cases:
        st = inputs.baroclinic_jet(I, J, K, seed=seed, noise=1e-2, terrain_seed=2)
        g = agcm.Grid(I, J, K, phis=st["phis"])
        dt = g.dt(100.0)
        s = agcm.State(g, prec)
        s.load(st)
        for _ in range(4):  # one call per step, as below (FP32 refreshes its column means per call)
            s.step(1, dt)
        ref.append(to_np(s.store()))
        s.load(st)  # back to the initial state
        grids.append((g, dt))
        states.append(s)
    torch.cuda.synchronize()
    streams = [torch.cuda.Stream() for _ in states]
    for _ in range(4):  # interleave single steps on three streams
        for (g, dt), s, q in zip(grids, states, streams):
            s.step(1, dt, stream=q)
    torch.cuda.synchronize()
    for s, r in zip(states, ref):
        out = to_np(s.store())
        for f in FIELDS:
            assert np.array_equal(out[f], r[f]), f
        s.close()


def test_argument_errors_leave_the_state_usable():
    I, J, K = 64, 32, 6
    st = inputs.rossby_haurwitz4(I, J, K, seed=1)
    g = agcm.Grid(I, J, K, phis=st["phis"])
    s = agcm.State(g, agcm.AGCM_FP32)
    s.load(st)
    L = agcm.lib()
    stream = ctypes.c_void_p(0)
    assert L.agcm_step(s.handle, -1, 10.0, stream) == agcm.AGCM_EINVAL
    assert L.agcm_step(s.handle, 1, float("nan"), stream) == agcm.AGCM_EINVAL
    assert L.agcm_step(s.handle, 1, float("inf"), stream) == agcm.AGCM_EINVAL
    assert L.agcm_step_split(s.handle, 1, 10.0, 0, stream) == agcm.AGCM_EINVAL
    assert L.agcm_filter(s.handle, 0.5, stream) == agcm.AGCM_EINVAL
    assert L.agcm_step(s.handle, 0, 10.0, stream) == agcm.AGCM_OK  # nothing to do
    # the grid cannot go while a state uses it
    assert L.agcm_grid_destroy(g.handle) == agcm.AGCM_EINVAL
    before = to_np(s.store())
    s.step(1, g.dt(100.0))
    after = to_np(s.store())
    assert all(np.isfinite(after[f]).all() for f in FIELDS)
    assert any(not np.array_equal(after[f], before[f]) for f in FIELDS)
    s.close()


def test_profiler_counts_launches():
    I, J, K = 64, 32, 6
    st = inputs.rossby_haurwitz4(I, J, K, seed=1)
    g = agcm.Grid(I, J, K, phis=st["phis"])
    s = agcm.State(g, agcm.AGCM_FP32)
    s.load(st)
    s.profile(True)
    s.step(5, g.dt(100.0))
    s.filter()
    prof = s.profile_read()
    s.profile(False)
    # three stages per step; a stage is two launches when the grid has both a
    # band of interior rows whose strides Mu_j, Mv_j, Mu_{j+1} are all 1 and
    # other rows
    lu, lv = g.leap()
    band = [j for j in range(1, J - 2) if lu[j] == 1 and lv[j] == 1 and lu[j + 1] == 1]
    assert 0 < len(band) < J
    assert prof["k_fused_stage"][1] == 30
    assert prof["k_vsum"][1] == 1  # exact vertical means once per step call after a load
    assert prof["k_filter"][1] == 1
    assert all(ms > 0 for ms, n in prof.values())
    s.close()


def _row_kernel_launches(lu, lv, I):
    """Launches of one stage of a step on the row-segment path: one per
    stride class present (rows whose strides Mu_j, Mv_j, Mu_{j+1} are all 1,
    all 3, all 5, all 7, other rows with a halo of at most 64 columns) and
    one for the rows left to the column kernel."""
    J = len(lu)
    classes, col = set(), False
    for j in range(J):
        hv = j < J - 1
        Mu, Mv, M1 = lu[j], (lv[j] if hv else lu[j]), (lu[j + 1] if hv else lu[j])
        H = (max(Mu, Mv if hv else 1, M1 if hv else 1) + 4) & ~3
        if I % 4 or ((256 - 2 * H) & ~3) < 128:
            col = True
        elif hv and Mu == Mv == M1 and Mu in (1, 3, 5, 7):
            classes.add(Mu)
        else:
            classes.add(0)
    return len(classes) + (1 if col else 0)


@pytest.mark.parametrize("grid", [(64, 32, 6), (24, 10, 3), (48, 40, 4)])
def test_row_kernel_launches_one_per_stride_class(grid, stage_kernel):
    """With the row-segment kernel a stage is one launch per stride class
    present plus one for the rows it leaves to the column kernel; with the
    column kernel, one or two (the stride-1 band)."""
    I, J, K = grid
    g = agcm.Grid(I, J, K)
    lu, lv = g.leap()
    s = agcm.State(g, agcm.AGCM_FP32)
    s.load(inputs.random_state(I, J, K, seed=2))
    s.profile(True)
    s.step(2, g.dt(100.0))
    n = s.profile_read()["k_fused_stage"][1]
    s.profile(False)
    if stage_kernel == "row":
        assert n == 6 * _row_kernel_launches(lu, lv, I), (grid, n)
    else:
        band = [j for j in range(1, J - 2) if lu[j] == 1 and lv[j] == 1 and lu[j + 1] == 1]
        assert n == 6 * (2 if 0 < len(band) < J else 1), (grid, n)
    s.close()


def test_state_stage_kernel_choice_overrides_the_process_one():
    """agcm_state_set_stage_kernel: a state set to 2 runs the row-segment
    kernel on a grid too small for the process's default to pick it, a state
    left at 0 keeps the default, and both agree with each other to rounding."""
    I, J, K = 64, 32, 6
    g = agcm.Grid(I, J, K)
    lu, lv = g.leap()
    x = inputs.random_state(I, J, K, seed=4)
    dt = g.dt(100.0)
    out, launches = {}, {}
    for choice in (0, 2):
        s = agcm.State(g, agcm.AGCM_FP32)
        s.set_stage_kernel(choice)
        s.load(x)
        s.profile(True)
        s.step(2, dt)
        launches[choice] = s.profile_read()["k_fused_stage"][1]
        s.profile(False)
        out[choice] = {f: v.double().cpu().numpy() for f, v in s.store().items()}
        s.close()
    assert launches[2] == 6 * _row_kernel_launches(lu, lv, I)
    band = [j for j in range(1, J - 2) if lu[j] == 1 and lv[j] == 1 and lu[j + 1] == 1]
    assert launches[0] == 6 * (2 if 0 < len(band) < J else 1)
    for f in FIELDS:
        err = np.abs(out[2][f] - out[0][f]).max() / np.abs(out[0][f]).max()
        assert err <= 1e-5, (f, err)
    with pytest.raises(agcm.AgcmError):
        agcm.State(g, agcm.AGCM_FP32).set_stage_kernel(3)


@pytest.mark.parametrize("leap", ["ones", "eq7", "none"])
def test_stage_launch_count_follows_the_stride1_band(leap):
    """A stage is two launches when the grid has a run of interior rows
    whose strides Mu_j, Mv_j, Mu_{j+1} are all 1 and rows outside it, else
    one; the tendency matches the oracle either way (parity tests)."""
    I, J, K = (24, 10, 3) if leap != "none" else (5, 3, 2)
    mu = mv = None
    if leap != "eq7":
        mu, mv = np.ones(J, np.int32), np.ones(J - 1, np.int32)
    g = agcm.Grid(I, J, K, leap_u=mu, leap_v=mv)
    lu, lv = g.leap()
    band = [j for j in range(1, J - 2) if lu[j] == 1 and lv[j] == 1 and lu[j + 1] == 1]
    s = agcm.State(g, agcm.AGCM_FP64)
    s.load(inputs.random_state(I, J, K, seed=2))
    s.profile(True)
    s.step(2, g.dt(100.0))
    n = s.profile_read()["k_fused_stage"][1]
    s.profile(False)
    assert n == 6 * (2 if band else 1), (leap, band, n)
    assert (leap == "none") == (not band)
    s.close()


def test_states_created_from_many_threads_share_one_grid():
    """ctypes releases the interpreter lock in foreign calls, so these threads
    create states on one fresh grid (whose device tables are built by the
    first) truly at once; every state then steps to the same result."""
    import threading

    import torch

    I, J, K = 64, 32, 6
    st = inputs.rossby_haurwitz4(I, J, K, seed=1)
    g = agcm.Grid(I, J, K, phis=st["phis"])
    dt = g.dt(100.0)
    states, errors = [None] * 8, []
    barrier = threading.Barrier(8)

    def work(q):
        try:
            torch.cuda.set_device(0)
            barrier.wait()
            states[q] = agcm.State(g, agcm.AGCM_FP32 if q % 2 else agcm.AGCM_FP64)
        except Exception as e:  # collected and asserted below
            errors.append(e)

    threads = [threading.Thread(target=work, args=(q,)) for q in range(8)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    outs = {}
    for q, s in enumerate(states):
        s.load(st)
        s.step(2, dt)
        outs.setdefault(q % 2, []).append(to_np(s.store()))
    for group in outs.values():
        for o in group[1:]:
            for f in FIELDS:
                assert np.array_equal(o[f], group[0][f]), f
    for s in states:
        s.close()
    g.close()  # no state holds the grid any more


@pytest.mark.parametrize("prec", [agcm.AGCM_FP32, agcm.AGCM_FP64])
def test_step_graph_replay_equals_eager_calls(prec):
    I, J, K = 96, 48, 8
    st = inputs.baroclinic_jet(I, J, K, seed=4, noise=1e-2, terrain_seed=2)
    g = agcm.Grid(I, J, K, phis=st["phis"])
    dt = g.dt(100.0)
    a = agcm.State(g, prec)
    a.load(st)
    for _ in range(3):
        a.step(2, dt)
    want = to_np(a.store())
    b = agcm.State(g, prec)
    b.load(st)
    graph = b.capture(2, dt)
    for _ in range(3):
        graph.replay()
    import torch

    torch.cuda.synchronize()
    got = to_np(b.store())
    # FP32 recomputes its column means at every call, eager or replayed: the
    # same launches, bit for bit; FP64 replays recompute them where the eager
    # calls carry them, which differs by rounding only
    tol = 0.0 if prec == agcm.AGCM_FP32 else 1e-13
    for f in FIELDS:
        assert np.abs(got[f] - want[f]).max() <= tol * np.abs(want[f]).max(), f
    a.close()
    b.close()


@pytest.mark.timeout(120, method="thread")
def test_garbage_collection_inside_the_allocator_hook():
    """The allocator hook may run arbitrary code of the embedding runtime, and
    a garbage collector there may destroy other states and grids through this
    library.  The library must not hold its grid lock across the hook: here a
    state kept alive only by a reference cycle is collected from inside the
    allocations that build a new grid's device tables."""
    import gc

    import torch

    L = agcm.lib()
    g0 = agcm.Grid(32, 16, 3)
    s0 = agcm.State(g0, agcm.AGCM_FP32)
    s0.cycle = s0  # only the cyclic collector can free it
    del s0, g0
    collected = {"n": 0}

    def alloc(n, ctx):
        collected["n"] += gc.collect()
        return torch.cuda.caching_allocator_alloc(int(n))

    def free(p, ctx):
        gc.collect()
        torch.cuda.caching_allocator_delete(p)

    A, F = agcm._ALLOC_T(alloc), agcm._FREE_T(free)
    agcm.check(L.agcm_set_allocator(ctypes.cast(A, ctypes.c_void_p), ctypes.cast(F, ctypes.c_void_p), None))
    try:
        g1 = agcm.Grid(40, 20, 3)
        s1 = agcm.State(g1, agcm.AGCM_FP32)  # the grid upload allocates first
        s1.close()
        g1.close()
        assert collected["n"] > 0
    finally:
        agcm.check(L.agcm_set_allocator(None, None, None))
        agcm._alloc_cbs = None
        agcm.use_torch_allocator()


def test_host_copies_reject_wrong_buffers():
    import torch

    I, J, K = 32, 16, 3
    g = agcm.Grid(I, J, K)
    s = agcm.State(g, agcm.AGCM_FP32)
    good = {f: torch.zeros(sh, dtype=torch.float32) for f, sh in g.shapes().items()}
    s.load_host(good)
    s.store_host(good)
    bad_size = dict(good, U=torch.zeros(K * J * I - 1, dtype=torch.float32))
    bad_type = dict(good, Phi=torch.zeros(g.shapes()["Phi"], dtype=torch.float64))
    bad_dev = dict(good, pi=torch.zeros(g.shapes()["pi"], dtype=torch.float32, device="cuda"))
    for bad in (bad_size, bad_type, bad_dev):
        with pytest.raises(ValueError):
            s.load_host(bad)
        with pytest.raises(ValueError):
            s.store_host(bad)
    s.close()
