"""Ensemble persistent kernel: member k equals its own single-state run, graph
replay equals eager launches, the bounded barrier reports a timeout without
hanging, and the autotuner picks a valid shape."""
import numpy as np
import pytest

from paper_2103_10114_gb300 import agcm, inputs
from paper_2103_10114_gb300.ensemble import Ensemble

pytestmark = pytest.mark.gpu
FIELDS = agcm.FIELDS
MIX = [(64, 32, 6), (48, 24, 5), (37, 23, 4), (96, 48, 8)]


@pytest.fixture(scope="module", autouse=True)
def _built(cuda_ok):
    agcm.build()
    agcm.lib()


def members(prec, mix=MIX, seed0=100):
    out = []
    for n, (I, J, K) in enumerate(mix):
        st = inputs.baroclinic_jet(I, J, K, seed=seed0 + n, noise=1e-2, terrain_seed=2)
        g = agcm.Grid(I, J, K, phis=st["phis"])
        s = agcm.State(g, prec)
        s.load(st)
        out.append((g, s, st, g.dt(100.0)))
    return out


def np_state(s):
    return {f: v.double().cpu().numpy() for f, v in s.store().items()}


@pytest.mark.parametrize("prec,shape", [(agcm.AGCM_FP32, (1, 0, 1)), (agcm.AGCM_FP64, (1, 0, 1)),
                                        (agcm.AGCM_FP32, (1, 0, 2)), (agcm.AGCM_FP64, (1, 0, 4)),
                                        (agcm.AGCM_FP32, (8, 0, 1)), (agcm.AGCM_FP64, (8, 0, 1)),
                                        (agcm.AGCM_FP32, (8, 1, 1))])
def test_member_equals_single_run(prec, shape):
    """Every member after three ensemble steps equals its own run; row tiles
    of 2 and 4 rows leave ragged last tiles on the member grids (nlat 23);
    the 256-thread launch runs the row-segment body (the 37-column member,
    whose rows are not 16-byte aligned, on the column body)."""
    mem = members(prec)
    ens = Ensemble([m[1] for m in mem])
    ens.configure(*shape)
    dts = [m[3] for m in mem]
    ens.step(3, dts)
    ens.status()
    for g, s, st, dt in mem:
        got = np_state(s)
        alone = agcm.State(g, prec)
        alone.load(st)
        alone.step(3, dt)
        want = np_state(alone)
        # the same column body in two kernels: the compiler may fuse
        # multiply-adds differently, so agreement is to about one rounding
        tol = 1e-6 if prec == agcm.AGCM_FP32 else 1e-13
        for f in FIELDS:
            err = np.abs(got[f] - want[f]).max() / np.abs(want[f]).max()
            assert err <= tol, (g.nlon, f, err)
    ens.close()


@pytest.mark.parametrize("shape", [(1, 0, 1), (8, 0, 1)])
def test_graph_replay_equals_eager(shape):
    import torch

    mem = members(agcm.AGCM_FP32)
    ens = Ensemble([m[1] for m in mem])
    ens.configure(*shape)
    dts = [m[3] for m in mem]
    x0 = [m[1].store() for m in mem]
    graph = ens.capture(2, dts)
    graph.replay()
    graph.replay()
    torch.cuda.synchronize()
    ens.status()
    replayed = [np_state(m[1]) for m in mem]
    for (g, s, st, dt), x in zip(mem, x0):
        s.load(x)
    ens.step(2, dts)  # the same call sequence as the two replays (each call
    ens.step(2, dts)  # starts from freshly summed FP64 vertical means)
    ens.status()
    for m, r in zip(mem, replayed):
        e = np_state(m[1])
        for f in FIELDS:
            assert np.array_equal(e[f], r[f])
    ens.close()


@pytest.mark.parametrize("shape", [(1, 0, 1), (8, 0, 1)])
def test_barrier_timeout_is_reported_and_context_survives(shape):
    mem = members(agcm.AGCM_FP32, mix=[(64, 32, 6), (48, 24, 5)])
    ens = Ensemble([m[1] for m in mem])
    ens.configure(*shape)
    dts = [m[3] for m in mem]
    x0 = [m[1].store() for m in mem]
    ens.set_timeout(0.2, test_missing_blocks=1)  # every barrier waits for a block that never comes
    ens.step(1, dts)
    with pytest.raises(agcm.AgcmError) as e:
        ens.status()
    assert e.value.code == agcm.AGCM_ETIMEOUT
    # the context is still usable: a normal run afterwards is correct
    ens.set_timeout(1.0, 0)
    for m, x in zip(mem, x0):
        m[1].load(x)
    ens.step(2, dts)
    ens.status()
    for g, s, st, dt in mem:
        alone = agcm.State(g, agcm.AGCM_FP32)
        alone.load(st)
        alone.step(2, dt)
        a, b = np_state(s), np_state(alone)
        for f in FIELDS:
            assert np.abs(a[f] - b[f]).max() <= 1e-6 * np.abs(b[f]).max()
    ens.close()


@pytest.mark.parametrize("graph", [False, True], ids=["eager", "graph"])
def test_autotune_picks_a_shape_and_keeps_state(graph):
    mem = members(agcm.AGCM_FP32)
    ens = Ensemble([m[1] for m in mem])
    dts = [m[3] for m in mem]
    before = [np_state(m[1]) for m in mem]
    shape, times = ens.autotune(dts, steps=1, graph=graph)
    assert shape in times and all(t > 0 for t in times.values())
    after = [np_state(m[1]) for m in mem]
    for a, b in zip(before, after):
        for f in FIELDS:
            assert np.array_equal(a[f], b[f])
    ens.close()


def test_config4_full_mix_sampled_members():
    """Config 4 as the bench runs it (64 members: 32 at 256x128x30, 24 at
    360x180x30, 8 at 720x360x30, FP32; autotuned shape, CUDA-graph replay):
    after two steps, one member of each size equals its own single-state run,
    and the first member matches the FP64 oracle within the FP32 tolerance."""
    import torch

    import oracle

    mix = [(256, 128, 30)] * 32 + [(360, 180, 30)] * 24 + [(720, 360, 30)] * 8
    mem = members(agcm.AGCM_FP32, mix=mix, seed0=100)
    ens = Ensemble([m[1] for m in mem])
    dts = [m[3] for m in mem]
    ens.autotune(dts, steps=1, graph=True)
    graph = ens.capture(2, dts)
    graph.replay()
    torch.cuda.synchronize()
    ens.status()
    for q in (0, 40, 63):
        g, s, st, dt = mem[q]
        got = np_state(s)
        alone = agcm.State(g, agcm.AGCM_FP32)
        alone.set_stage_kernel(2 if ens.shape[0] == "streams-row" else 0)  # the member's stage kernel
        alone.load(st)
        alone.step(2, dt)
        want = np_state(alone)
        for f in FIELDS:
            err = np.abs(got[f] - want[f]).max() / np.abs(want[f]).max()
            assert err <= 1e-6, (q, f, err)
        alone.close()
    g, s, st, dt = mem[0]
    o = oracle.Oracle(g.nlon, g.nlat, g.nlev, phis=st["phis"])
    ref = o.step(st, dt, 2)
    got = np_state(s)
    for f in FIELDS:
        err = np.abs(got[f] - ref[f]).max() / np.abs(ref[f]).max()
        assert err <= 1e-5, (f, err)
    ens.close()


@pytest.mark.parametrize("mode", ["streams", "streams-row"])
@pytest.mark.parametrize("prec", [agcm.AGCM_FP32, agcm.AGCM_FP64])
def test_streams_mode_equals_single_runs_and_replays(prec, mode):
    """The streams modes step every member with the single-state kernel (in
    "streams-row" the row-segment kernel), so each member equals its own run
    on the same kernel bit for bit, eagerly and from a graph."""
    import torch

    mem = members(prec)
    ens = Ensemble([m[1] for m in mem])
    ens.configure(mode, 3)
    dts = [m[3] for m in mem]
    ens.step(2, dts)
    graph = ens.capture(2, dts)
    graph.replay()
    torch.cuda.synchronize()
    for g, s, st, dt in mem:
        got = np_state(s)
        alone = agcm.State(g, prec)
        alone.set_stage_kernel(2 if mode == "streams-row" else 0)
        alone.load(st)
        alone.step(2, dt)
        alone.step(2, dt)
        want = np_state(alone)
        for f in FIELDS:
            assert np.array_equal(got[f], want[f]), (g.nlon, f)
        alone.close()
    ens.close()
