"""Long-run precision and conservation reports (printed; run with -s to see them).

* 256 x 128 x 30 (about 1.4 deg) with terrain, jet + perturbation, 200 steps:
  plain FP64 and FP32-with-FP64-column-sums against the FP64 oracle, per-field
  normwise error (reading R11) and the mass / energy drift of each run.
* 1440 x 720 x 30 (0.25 deg), FP32, 1000 steps: drift, and the state stays finite.
"""
import json

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


def to_np(d):
    return {f: v.double().cpu().numpy() for f, v in d.items()}


def test_config2_200_steps_fp64_and_fp32():
    I, J, K, n = 256, 128, 30, 200
    st = inputs.baroclinic_jet(I, J, K, seed=3, noise=1e-3, terrain_seed=2)
    g = agcm.Grid(I, J, K, phis=st["phis"])
    dt = g.dt(100.0)
    o = oracle.Oracle(I, J, K, phis=st["phis"])
    ref = o.step(st, dt, n)
    d0, dr = o.diagnostics(st), o.diagnostics(ref)
    report = {"grid": [I, J, K], "steps": n, "dt_s": dt,
              "oracle": {"mass_drift": dr["mass"] / d0["mass"] - 1, "energy_drift": dr["energy"] / d0["energy"] - 1}}
    for prec, tag in ((agcm.AGCM_FP64, "fp64"), (agcm.AGCM_FP32, "fp32")):
        s = agcm.State(g, prec)
        s.load(st)
        a = s.diagnostics()
        s.step(n, dt)
        b = s.diagnostics()
        out = to_np(s.store())
        err = {f: float(np.abs(out[f] - ref[f]).max() / np.abs(ref[f]).max()) for f in FIELDS}
        report[tag] = {"error_vs_oracle": err, "mass_drift": b["mass"] / a["mass"] - 1,
                       "energy_drift": b["energy"] / a["energy"] - 1, "finite": b["finite"]}
        s.close()
    print("\nCONFIG2_REPORT " + json.dumps(report))
    assert max(report["fp64"]["error_vs_oracle"].values()) <= 1e-9
    assert max(report["fp32"]["error_vs_oracle"].values()) <= 1e-2
    assert abs(report["fp64"]["mass_drift"]) < 1e-13 and abs(report["fp32"]["mass_drift"]) < 1e-6
    assert abs(report["fp64"]["energy_drift"] - report["oracle"]["energy_drift"]) <= 1e-6 * abs(
        report["oracle"]["energy_drift"]) + 1e-14


def test_config5_1000_steps_fp32_drift():
    I, J, K, n = 1440, 720, 30, 1000
    st = inputs.baroclinic_jet(I, J, K, seed=5, noise=1e-3, terrain_seed=2)
    g = agcm.Grid(I, J, K, phis=st["phis"])
    dt = g.dt(100.0)
    s = agcm.State(g, agcm.AGCM_FP32)
    s.load(st)
    a = s.diagnostics()
    drifts = []
    for chunk in range(10):
        s.step(n // 10, dt)
        b = s.diagnostics()
        drifts.append((b["mass"] / a["mass"] - 1, b["energy"] / a["energy"] - 1))
    report = {"grid": [I, J, K], "steps": n, "dt_s": dt, "simulated_hours": n * dt / 3600,
              "mass_drift": drifts[-1][0], "energy_drift": drifts[-1][1],
              "energy_drift_every_100": [d[1] for d in drifts], "finite": b["finite"],
              "max_u": b["max_u"], "max_v": b["max_v"]}
    print("\nCONFIG5_REPORT " + json.dumps(report))
    assert b["finite"] == 1
    assert abs(report["mass_drift"]) < 1e-5
    assert report["energy_drift"] < 0  # the three-stage step only removes energy


def test_full_model_options_300_split_steps_fp32():
    """1440 x 720 x 30 FP32 with every option the library has on at once: the
    lapse-rate standard atmosphere with the delta kappa Phi/P term, split
    stepping (adaptation sub-steps under the gravity-wave dt) and the
    low-latitude filters after every step; 300 steps (about 10.7 simulated
    hours).  Reports mass and energy drift; the run must stay finite and keep
    its mass."""
    I, J, K, n = 1440, 720, 30, 300
    th = dict(profile=1, Ts0=288.15, lapse=6.5e-3, Ttrop=216.65, delta=1.0)
    st = inputs.baroclinic_jet(I, J, K, seed=5, noise=1e-3, terrain_seed=2)
    g = agcm.Grid(I, J, K, phis=st["phis"], thermo=th)
    dt, msub = g.dt_split(100.0)
    s = agcm.State(g, agcm.AGCM_FP32)
    s.load(st)
    a = s.diagnostics()
    for _ in range(n):
        s.step_split(1, dt, msub)
        s.filter(0.25)
    b = s.diagnostics()
    report = {"grid": [I, J, K], "steps": n, "dt_s": dt, "msub": msub, "simulated_hours": n * dt / 3600,
              "mass_drift": b["mass"] / a["mass"] - 1, "energy_drift": b["energy"] / a["energy"] - 1,
              "finite": b["finite"], "max_u": b["max_u"], "max_v": b["max_v"]}
    print("\nFULL_OPTIONS_REPORT " + json.dumps(report))
    assert b["finite"] == 1
    assert abs(report["mass_drift"]) < 1e-5
    assert b["max_u"] < 200.0


def test_fp32_column_means_over_one_long_call():
    """FP32 keeps the FP64 column means within a call by adding FP32 sums of
    each stage's increments, and recomputes them exactly at the start of every
    call: 2000 steps in one call end where 20 calls of 100 steps end, to within
    the FP32 precision of the fields."""
    I, J, K, n = 256, 128, 30, 2000
    st = inputs.baroclinic_jet(I, J, K, seed=3, noise=1e-3, terrain_seed=2)
    g = agcm.Grid(I, J, K, phis=st["phis"])
    dt = g.dt(100.0)
    a, b = agcm.State(g, agcm.AGCM_FP32), agcm.State(g, agcm.AGCM_FP32)
    a.load(st)
    b.load(st)
    a.step(n, dt)
    for _ in range(20):
        b.step(n // 20, dt)
    x, y = to_np(a.store()), to_np(b.store())
    err = {f: float(np.abs(x[f] - y[f]).max() / np.abs(y[f]).max()) for f in FIELDS}
    print("\nCOLUMN_MEANS_REPORT " + json.dumps({"steps": n, "one_call_vs_20_calls": err}))
    assert max(err.values()) < 1e-4, err
    a.close()
    b.close()
