"""Benchmark of the leap-format dynamical-core step on GB300.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload: 1440 x 720 x 30 (0.25 deg, the high-resolution case), FP32 state
with FP64 column integrals, jet + terrain + seeded noise.  A "step" is one
full three-stage time step.  The metric is grid-point-steps per second
(nlon*nlat*nlev*steps / s); for N > 1 each rank advances its own replica
(the path has no exchange step on one GPU) and the value is the sum over ranks.

The JSON line adds the roofline of the dominant kernel (algorithmic bytes over
its CUDA-event launch time, against the measured copy bandwidth, with the ncu
DRAM traffic of the same source), its instruction counters, the end-to-end
rate through the C ABI with host buffers, the oracle's CPU rate on one and on
all host cores, nvidia-smi clocks sampled during the timed region, and the
other forms (FP64, small grid, split stepping, thermodynamics, filters, the
64-member ensemble, the adjoint).

The reference arm (--impl reference) times the FP64 CPU oracle, as it stands,
on every host core, one sample of the same model per core per timed step
(360x180x30, or 180x90x30 when many steps are asked for).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = (1440, 720, 30)
BYTES_PER_POINT_STEP = {4: 96, 8: 192}  # 24 words: stages read/write 6 + 9 + 9 words

# DRAM traffic of the dominant kernel from an ncu capture of this workload,
# valid only while the kernel source is the one that was captured.
NCU_TRAFFIC = {
    # kernel bracket name: (sha1 of the stage-kernel sources at capture time,
    # DRAM bytes per stage summed over the stage's launches)
    "k_fused_stage": ("bdf6da56225021001f2b3994ea157acdfa68fd16", 943000000),
}

# Instruction counters of the dominant kernel (ncu per-opcode counts, this
# workload, a later stage's launches weighted by the points of their rows),
# valid while the kernel source is the one that was captured: FP32 flops per
# point and stage (fadd + fmul + 2 ffma), thread instructions per point, warp
# instructions issued per point.
NCU_OPS = {
    "k_fused_stage": ("bdf6da56225021001f2b3994ea157acdfa68fd16", 181.1, 312.6, 9.77),
}


# DRAM traffic of one FP32 adjoint step at 720x360x30 (all its launches: the
# forward recompute of the two stage states and three adjoint products), from
# an ncu capture, valid while the kernel sources are the captured ones.
NCU_ADJ = ("f69af5c5506a1652024ccb2750b972e976a7678a", 2752465920)


def kernel_source_hash(names=("agcm_row.cuh", "agcm_fused.cuh", "agcm_common.cuh")):
    """sha1 of kernel sources (by default the stage kernels: the row-segment
    and column kernels)."""
    import hashlib

    h = hashlib.sha1()
    for name in names:
        with open(os.path.join(ROOT, "paper_2103_10114_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


ADJ_SOURCES = ("agcm_adjoint.cuh", "agcm_phases.cuh", "agcm_row.cuh", "agcm_fused.cuh", "agcm_common.cuh")


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "samples": len(sm),
                "reasons": sorted(reasons)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
        return dist.get_rank(), ws, int(os.environ.get("LOCAL_RANK", "0"))
    return 0, 1, 0


def max_over_ranks(value, device):
    """Largest value over all ranks (timing is the slowest rank's); identity on one rank."""
    import torch

    if not torch.distributed.is_available() or not torch.distributed.is_initialized():
        return float(value)
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(points_per_rank, steps, ms_max, world):
    """Replicas: every rank advances its own state; the job's rate is the sum."""
    return world * points_per_rank * steps / (ms_max / 1e3)


def cpu_oracle_rate(nlon, nlat, nlev, steps=1, st=None):
    """Time the FP64 oracle on one grid; returns (gp-steps/s, seconds)."""
    import oracle
    from paper_2103_10114_gb300 import inputs

    if st is None:
        st = inputs.baroclinic_jet(nlon, nlat, nlev, seed=5, noise=1e-2, terrain_seed=2)
    o = oracle.Oracle(nlon, nlat, nlev, phis=st["phis"])
    dt = 60.0
    t0 = time.perf_counter()
    o.step(st, dt, steps)
    el = time.perf_counter() - t0
    return nlon * nlat * nlev * steps / el, el


_SAMPLE = {}


def _oracle_sample_step(arg):
    """One FP64 oracle step of a seeded sample grid in a worker process; the
    sample and the oracle's grid are kept per worker, and only the step is
    timed."""
    nlon, nlat, nlev, seed = arg
    key = (nlon, nlat, nlev, seed)
    if key not in _SAMPLE:
        import oracle
        from paper_2103_10114_gb300 import inputs

        _SAMPLE.clear()
        st = inputs.baroclinic_jet(nlon, nlat, nlev, seed=seed, noise=1e-2, terrain_seed=2)
        _SAMPLE[key] = (oracle.Oracle(nlon, nlat, nlev, phis=st["phis"]), st)
    o, st = _SAMPLE[key]
    t0 = time.perf_counter()
    o.step(st, 60.0, 1)
    return time.perf_counter() - t0


def cpu_oracle_rate_all_cores(nlon=360, nlat=180, nlev=30, steps=1, warmup=1):
    """The oracle as it stands, one sample step per host core at a time in
    spawned worker processes; returns (aggregate gp-steps/s, workers, mean
    seconds per step).  A step's time is that of its slowest worker."""
    import multiprocessing as mp

    import oracle

    oracle.build()  # compile once before the workers load it
    n = os.cpu_count() or 1
    task = [(nlon, nlat, nlev, 100)] * n
    ctx = mp.get_context("spawn")
    with ctx.Pool(n) as pool:
        for _ in range(max(1, warmup)):
            pool.map(_oracle_sample_step, task, chunksize=1)
        per_step = [max(pool.map(_oracle_sample_step, task, chunksize=1)) for _ in range(steps)]
    el = sum(per_step)
    return n * nlon * nlat * nlev * steps / el, n, el / steps


def run_reference(args):
    """The oracle on the machine's host cores: each timed step is one oracle step
    of a 360x180x30 sample of the workload on every core at once."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # a 360x180x30 sample step takes about 0.7 s on every core of the GB300
    # box; many timed steps use a quarter-size sample so the run stays near
    # two minutes
    sample = (360, 180, 30) if (args.steps + args.warmup) * 0.7 <= 150.0 else (180, 90, 30)
    value, cores, sec = cpu_oracle_rate_all_cores(*sample, steps=args.steps, warmup=args.warmup)
    line = {
        "impl": "reference", "metric": "grid-point-steps/s", "value": value, "unit": "gp-steps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "leap-format IAP step 1440x720x30 (0.25 deg) jet+terrain",
                   "sample": f"{sample[0]}x{sample[1]}x{sample[2]} per core, {cores} cores"},
        "cpu_baseline": {"value": value, "unit": "gp-steps/s", "cores": cores, "kind": "oracle",
                         "sample": f"one oracle step of a {sample[0]}x{sample[1]}x{sample[2]} sample on each of "
                                   f"{cores} cores per timed step"},
        "e2e": {"value": value, "unit": "gp-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--only", choices=["adjoint", "ensemble", "fp64", "fp32", "fp32_720", "split", "filter", "thermo",
                                       "gradient"],
                    help="measure one form alone and print its JSON (for profiling)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.only:
        return run_only(args.only)

    import numpy as np
    import torch

    from paper_2103_10114_gb300 import agcm, inputs

    rank, world, local = dist_setup()
    torch.cuda.set_device(local)
    agcm.build()
    agcm.lib()
    I, J, K = WORKLOAD
    pts = I * J * K
    st = inputs.baroclinic_jet(I, J, K, seed=5 + rank, noise=1e-2, terrain_seed=2)
    g = agcm.Grid(I, J, K, phis=st["phis"])
    dt = g.dt(100.0)
    s = agcm.State(g, agcm.AGCM_FP32)
    s.load(st)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    # warm-up
    s.step(args.warmup, dt)
    torch.cuda.synchronize()
    d0 = s.diagnostics()  # conservation reference at the start of the timed steps
    # timed region: device-resident inputs
    s.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        s.step(args.steps, dt)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
    ms = e0.elapsed_time(e1)
    prof = s.profile_read()
    s.profile(False)
    clocks = clk.summary()
    ms = max_over_ranks(ms, "cuda")
    value = whole_job_rate(pts, args.steps, ms, world)
    d = s.diagnostics()

    # end to end through the C ABI with pinned host buffers
    esz = 4
    host = {f: torch.from_numpy(np.ascontiguousarray(st[f], dtype=np.float32)).pin_memory() for f in agcm.FIELDS}
    hout = {f: torch.empty_like(host[f]).pin_memory() for f in agcm.FIELDS}
    nbytes = sum(h.numel() * esz for h in host.values())
    e2e_steps = max(3, args.steps // 2)
    torch.cuda.synchronize()
    barrier()
    e0.record(stream)
    for _ in range(e2e_steps):
        s.load_host(host)
        s.step(1, dt)
        s.store_host(hout)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_serial_ms = max_over_ranks(e0.elapsed_time(e1), "cuda")
    e2e_serial = whole_job_rate(pts, e2e_steps, e2e_serial_ms, world)
    # the same calls streamed: three device states on three streams, so the
    # host->device copy of one step, the step of the other state and the
    # device->host copy overlap (copy engines are full duplex)
    e2e, e2e_ok = e2e_streamed(agcm, torch, g, dt, host, hout, e2e_steps, world, barrier)

    peak, peak_kind = peaks()
    # dominant kernel and its algorithmic bytes (one stage: 6/9/9 words per point -> 8 on average)
    name, (kms, kn) = max(prof.items(), key=lambda kv: kv[1][0])
    stage_bytes = pts * 8 * esz
    # the profiler brackets each stage (the stride-1 row band and the other
    # rows, two concurrent launches) with one pair of events: the roofline's
    # unit is the stage
    n_stages = 3 * args.steps
    stage_ms = kms / n_stages
    achieved = stage_bytes / (stage_ms / 1e3) / 1e9 if name == "k_fused_stage" else None
    traffic, traffic_src = None, None
    rec = NCU_TRAFFIC.get(name)
    if rec and rec[0] == kernel_source_hash():
        traffic, traffic_src = rec[1], f"ncu dram read + write per stage, source sha1 {rec[0][:12]}"
    compute = None
    orec = NCU_OPS.get(name)
    if orec and orec[0] == kernel_source_hash():
        nsm = torch.cuda.get_device_properties(0).multi_processor_count
        fmax = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["sm_max_mhz"]) \
            if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 2070.0
        launch_s = stage_ms / 1e3
        fp32 = orec[1] * pts / launch_s / 1e12
        fp32_peak = nsm * 128 * 2 * fmax * 1e6 / 1e12
        issue = orec[3] * pts / launch_s
        issue_peak = nsm * 4 * fmax * 1e6
        compute = {"fp32_flops_per_point_stage": orec[1], "thread_inst_per_point_stage": orec[2],
                   "fp32_tflops": fp32, "fp32_peak_tflops": fp32_peak, "fp32_frac": fp32 / fp32_peak,
                   "warp_inst_per_point_stage": orec[3], "issue_frac": issue / issue_peak,
                   "peak_note": f"{nsm} SMs x 128 FP32 lanes x 2 x {fmax:.0f} MHz; issue: 4 warp-inst/SM/cycle",
                   "source": f"ncu per-opcode counts, this workload, source sha1 {orec[0][:12]}"}
    launches = sum(n for _, n in prof.values())
    line = {
        "metric": "grid-point-steps/s", "value": value, "unit": "gp-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "leap-format IAP step 1440x720x30 (0.25 deg), FP32 with FP64 column sums",
                   "ic": "jet+terrain+noise 1e-2", "dt_s": dt, "parallelism": "replicas" if world > 1 else "1 gpu",
                   "l2": "inputs larger than L2 (state 373 MB)"},
        "hbm_frac_step": value / world * BYTES_PER_POINT_STEP[esz] / (peak * 1e9),
        "roofline": {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": traffic, "peak_kind": peak_kind,
                     "traffic_source": traffic_src, "bytes_per_stage": stage_bytes, "avg_stage_ms": stage_ms,
                     "launches_per_stage": kn / n_stages,
                     "note": "peak = measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"},
        "compute": compute,
        "kernels": {k: {"ms_total": v[0], "launches": v[1], "share": v[0] / sum(x[0] for x in prof.values())}
                    for k, v in prof.items()},
        "e2e": {"value": e2e, "unit": "gp-steps/s", "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
                "how": "agcm_state_load (pinned host) + agcm_step + agcm_state_store (pinned host) per step; "
                       "three states on three streams so copies overlap compute",
                "serial_value": e2e_serial, "outputs_match_serial": e2e_ok},
        "gpu_launches": launches,
        "clocks": clocks,
        "sypd_equiv": (value / world / pts) * dt / 365.0,
        "finite": bool(d["finite"]),
        # relative change over the timed steps, from the FP64 diagnostics (mass:
        # area sum of the surface pressure; energy: the total effective energy)
        "drift": {"mass": (d["mass"] - d0["mass"]) / d0["mass"],
                  "energy": (d["energy"] - d0["energy"]) / d0["energy"], "steps": args.steps,
                  "simulated_hours": args.steps * dt / 3600.0},
    }
    if rank == 0 and not args.no_forms:
        line["forms"] = measure_forms(agcm, inputs, torch)
    if rank == 0 and not args.no_cpu_baseline:
        rate, el = cpu_oracle_rate(I, J, K, st=st)
        line["cpu_baseline"] = {"value": rate, "unit": "gp-steps/s", "cores": 1, "kind": "oracle",
                                "sample": f"one FP64 oracle step of the full {I}x{J}x{K} workload ({el:.1f} s)",
                                "host_cores": os.cpu_count()}
        try:
            arate, nw, sec = cpu_oracle_rate_all_cores(steps=2)
            line["cpu_baseline_all_cores"] = {
                "value": arate, "unit": "gp-steps/s", "cores": nw, "kind": "oracle",
                "sample": f"{nw} worker processes, one FP64 oracle step of a 360x180x30 sample each, "
                          f"2 timed steps ({sec:.2f} s per step)"}
        except Exception as e:  # reported, not hidden
            line["cpu_baseline_all_cores"] = {"error": repr(e)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def e2e_streamed(agcm, torch, g, dt, host, hout_serial, steps, world, barrier, nstates=3):
    """End-to-end rate through the C ABI with host buffers: per step one
    host->device load, one step and one device->host store, issued round-robin
    on `nstates` states and streams.  Returns (rate, outputs equal to the
    serial run's)."""
    states = [agcm.State(g, agcm.AGCM_FP32) for _ in range(nstates)]
    houts = [{f: torch.empty_like(host[f]).pin_memory() for f in agcm.FIELDS} for _ in range(nstates)]
    streams = [torch.cuda.Stream() for _ in range(nstates)]
    main = torch.cuda.current_stream()

    def issue(n):
        q = n % nstates
        states[q].load_host(host, stream=streams[q])
        states[q].step(1, dt, stream=streams[q])
        states[q].store_host(houts[q], stream=streams[q])

    for n in range(nstates):  # warm-up
        issue(n)
    torch.cuda.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(main)
    for q in streams:
        q.wait_stream(main)
    for n in range(steps):
        issue(n)
    for q in streams:
        main.wait_stream(q)
    e1.record(main)
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), "cuda")
    ok = all(bool(torch.equal(h[f], hout_serial[f])) for h in houts for f in agcm.FIELDS)
    for s_ in states:
        s_.close()
    return whole_job_rate(g.points(), steps, ms, world), ok


def run_only(form):
    import torch

    from paper_2103_10114_gb300 import agcm, inputs

    agcm.build()
    agcm.lib()
    if form == "adjoint":
        out = measure_adjoint(agcm, inputs, torch, steps=3)
    elif form == "ensemble":
        out = measure_ensemble(agcm, inputs, torch, steps=3, per_member=False)
    elif form == "split":
        out = measure_split(agcm, inputs, torch, steps=3)
    elif form == "filter":
        out = measure_filter(agcm, inputs, torch, reps=3)
    elif form == "thermo":
        out = measure_thermo(agcm, inputs, torch, steps=3)
    elif form == "gradient":
        out = measure_gradient(agcm, inputs, torch)
    else:  # fp64 / fp32: the plain FP64 / FP32 step at the bench size; fp32_720: FP32 at 720x360x30
        I, J, K = (720, 360, 30) if form == "fp32_720" else WORKLOAD
        st = inputs.baroclinic_jet(I, J, K, seed=6, noise=1e-2, terrain_seed=2)
        g = agcm.Grid(I, J, K, phis=st["phis"])
        s = agcm.State(g, agcm.AGCM_FP64 if form == "fp64" else agcm.AGCM_FP32)  # noqa: E501
        s.load(st)
        s.step(1, g.dt(100.0))
        ms = _time(torch, lambda: s.step(2, g.dt(100.0)), 1) / 2
        out = {"value": I * J * K / (ms / 1e3), "unit": "gp-steps/s", "ms_per_step": ms}
    print(json.dumps({"form": form, **out}), flush=True)


def _time(torch, fn, reps):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def measure_forms(agcm, inputs, torch, steps=5):
    """gp-steps/s of the other forms on the same GPU: plain FP64 at the same size,
    FP32 at 256x128x30, the 64-member ensemble (one persistent launch, autotuned,
    replayed from a CUDA graph) against per-member FP64 launches, and the
    adjoint step at 720x360x30."""
    out = {}
    I, J, K = WORKLOAD
    st = inputs.baroclinic_jet(I, J, K, seed=6, noise=1e-2, terrain_seed=2)
    g = agcm.Grid(I, J, K, phis=st["phis"])
    dt = g.dt(100.0)
    s = agcm.State(g, agcm.AGCM_FP64)
    s.load(st)
    s.step(2, dt)
    ms = _time(torch, lambda: s.step(steps, dt), 1) / steps
    out["fp64_1440x720x30"] = {"value": I * J * K / (ms / 1e3), "unit": "gp-steps/s", "ms_per_step": ms,
                               "bound": "fp64 pipe (GB300 runs FP64 at 2 lanes/SM/cycle)"}
    s.close()
    # FP32 at the precision-comparison size (state fits in L2)
    I2, J2, K2 = 256, 128, 30
    st2 = inputs.baroclinic_jet(I2, J2, K2, seed=3, terrain_seed=2)
    g2 = agcm.Grid(I2, J2, K2, phis=st2["phis"])
    for prec, tag in ((agcm.AGCM_FP32, "fp32"), (agcm.AGCM_FP64, "fp64")):
        s2 = agcm.State(g2, prec)
        s2.load(st2)
        s2.step(3, g2.dt(100.0))
        ms = _time(torch, lambda: s2.step(20, g2.dt(100.0)), 1) / 20
        out[f"{tag}_256x128x30"] = {"value": I2 * J2 * K2 / (ms / 1e3), "unit": "gp-steps/s", "ms_per_step": ms,
                                    "note": "state fits in L2"}
        if prec == agcm.AGCM_FP32:  # the same 20 steps replayed from a CUDA graph
            graph = s2.capture(20, g2.dt(100.0))
            graph.replay()
            gms = _time(torch, graph.replay, 3) / 20
            out[f"{tag}_256x128x30"]["graph"] = {"value": I2 * J2 * K2 / (gms / 1e3), "ms_per_step": gms}
        s2.close()
    try:
        out["split_1440x720x30"] = measure_split(agcm, inputs, torch)
    except Exception as e:
        out["split_1440x720x30"] = {"error": repr(e)}
    try:
        out["thermo_1440x720x30"] = measure_thermo(agcm, inputs, torch)
    except Exception as e:
        out["thermo_1440x720x30"] = {"error": repr(e)}
    try:
        out["filter_1440x720x30"] = measure_filter(agcm, inputs, torch)
    except Exception as e:
        out["filter_1440x720x30"] = {"error": repr(e)}
    try:
        out["ensemble_64"] = measure_ensemble(agcm, inputs, torch)
    except Exception as e:  # reported, not hidden
        out["ensemble_64"] = {"error": repr(e)}
    try:
        out["gradient_config3"] = measure_gradient(agcm, inputs, torch)
    except Exception as e:
        out["gradient_config3"] = {"error": repr(e)}
    try:
        out["adjoint_720x360x30"] = measure_adjoint(agcm, inputs, torch)
    except Exception as e:
        out["adjoint_720x360x30"] = {"error": repr(e)}
    return out


def measure_split(agcm, inputs, torch, steps=5):
    """Split stepping at 1440x720x30 FP32: msub adaptation steps of dt/msub and
    one advection step of dt per step (dt from the flow speed alone)."""
    I, J, K = WORKLOAD
    st = inputs.baroclinic_jet(I, J, K, seed=6, noise=1e-2, terrain_seed=2)
    g = agcm.Grid(I, J, K, phis=st["phis"])
    dt, msub = g.dt_split(100.0)
    s = agcm.State(g, agcm.AGCM_FP32)
    s.load(st)
    s.step_split(1, dt, msub)
    ms = _time(torch, lambda: s.step_split(steps, dt, msub), 1) / steps
    pts = I * J * K
    words = 24 * msub + 24
    res = {"value": pts / (ms / 1e3), "unit": "gp-steps/s", "ms_per_step": ms, "dt_s": dt, "msub": msub,
           "bytes_per_point_step": words * 4,
           "hbm_frac_step": pts / (ms / 1e3) * words * 4 / (peaks()[0] * 1e9),
           "sypd_equiv": pts / (ms / 1e3) / pts * dt / 365.0,
           "finite": bool(s.diagnostics()["finite"])}
    s.close()
    return res


THERMO_FULL = dict(profile=1, Ts0=288.15, lapse=6.5e-3, Ttrop=216.65, delta=1.0, delta_c=0.0, delta_p=0.0)


def measure_thermo(agcm, inputs, torch, steps=5):
    """The step at 1440x720x30 FP32 with Eq. 1's thermodynamics on: a
    lapse-rate standard atmosphere (per-level b) and the nonlinear
    delta kappa Phi/P term."""
    I, J, K = WORKLOAD
    st = inputs.baroclinic_jet(I, J, K, seed=6, noise=1e-2, terrain_seed=2)
    g = agcm.Grid(I, J, K, phis=st["phis"], thermo=THERMO_FULL)
    dt = g.dt(100.0)
    s = agcm.State(g, agcm.AGCM_FP32)
    s.load(st)
    s.step(2, dt)
    ms = _time(torch, lambda: s.step(steps, dt), 1) / steps
    res = {"value": I * J * K / (ms / 1e3), "unit": "gp-steps/s", "ms_per_step": ms, "dt_s": dt,
           "thermo": THERMO_FULL, "finite": bool(s.diagnostics()["finite"])}
    s.close()
    return res


def measure_filter(agcm, inputs, torch, reps=20):
    """The low-latitude filters at 1440x720x30 FP32: the filter alone (bytes:
    one read and one write of every row it changes) and a step followed by the
    filter."""
    I, J, K = WORKLOAD
    st = inputs.baroclinic_jet(I, J, K, seed=6, noise=1e-2, terrain_seed=2)
    g = agcm.Grid(I, J, K, phis=st["phis"])
    dt = g.dt(100.0)
    s = agcm.State(g, agcm.AGCM_FP32)
    s.load(st)
    s.filter()
    ms_f = _time(torch, s.filter, reps)
    dth = math.pi / J

    def changed(colat):  # rows the filter rewrites: |latitude| <= 70 degrees (nlon even)
        return abs(90.0 - math.degrees(colat)) <= 70.0

    nu = sum(1 for j in range(J) if changed((j + 0.5) * dth))
    nv = sum(1 for j in range(J - 1) if changed((j + 1.0) * dth))
    rows = (2 * K + 1) * nu + K * nv
    bytes_ = rows * I * 4 * 2
    s.step(1, dt)

    def both():
        s.step(1, dt)
        s.filter()

    ms_s = _time(torch, both, 5)
    res = {"filter_ms": ms_f, "filter_gbs": bytes_ / (ms_f / 1e3) / 1e9,
           "filter_hbm_frac": bytes_ / (ms_f / 1e3) / 1e9 / peaks()[0], "filtered_rows": rows,
           "value": I * J * K / (ms_s / 1e3), "unit": "gp-steps/s (step + filter)", "ms_per_step": ms_s,
           "finite": bool(s.diagnostics()["finite"])}
    s.close()
    return res


def measure_ensemble(agcm, inputs, torch, steps=10, per_member=True):
    """Config 4: 32 @ 256x128x30 + 24 @ 360x180x30 + 8 @ 720x360x30, FP32,
    advanced in the autotuned way (one persistent launch, or the members'
    single-state launches forked over streams) and replayed from a CUDA graph;
    the best persistent shape is reported beside it, and both against 64
    per-member launches of the plain FP64 step."""
    from paper_2103_10114_gb300.ensemble import Ensemble

    terr = {}
    states, grids, dts = [], [], []
    for (I, J, K), seed, noise in inputs.ensemble_members():
        if (I, J) not in terr:
            terr[(I, J)] = inputs.terrain_phis(I, J, seed=2)
        st = inputs.baroclinic_jet(I, J, K, seed=seed, noise=noise, terrain_seed=None)
        st["phis"] = terr[(I, J)]
        g = agcm.Grid(I, J, K, phis=st["phis"])
        s = agcm.State(g, agcm.AGCM_FP32)
        s.load(st)
        grids.append((g, st))
        states.append(s)
        dts.append(g.dt(100.0))
    pts = sum(g.points() for g, _ in grids)
    ens = Ensemble(states)
    shape, times = ens.autotune(dts, steps=2, graph=True)  # the ensemble is replayed from a graph

    def graph_ms(shp):
        ens.configure(*shp)
        graph = ens.capture(steps, dts)
        graph.replay()
        t = _time(torch, graph.replay, 1) / steps
        ens.status()
        return t

    ms = graph_ms(shape)
    res = {"value": pts / (ms / 1e3), "unit": "gp-steps/s", "ms_per_step": ms, "points": pts,
           "shape": list(shape), "tuned_ms": {"x".join(map(str, k)): round(t, 4) for k, t in times.items()},
           "hbm_frac_step": pts / (ms / 1e3) * 96 / (peaks()[0] * 1e9)}
    persistent = [k for k in times if not str(k[0]).startswith("streams")]
    if persistent:
        best_p = min(persistent, key=times.get)
        pms = ms if best_p == shape else graph_ms(best_p)
        res["persistent"] = {"shape": list(best_p), "ms_per_step": pms, "value": pts / (pms / 1e3),
                             "hbm_frac_step": pts / (pms / 1e3) * 96 / (peaks()[0] * 1e9)}
    ens.close()
    for s in states:
        s.close()
    if not per_member:
        return res
    # per-member launches of the plain FP64 step
    s64 = []
    for (g, st) in grids:
        s = agcm.State(g, agcm.AGCM_FP64)
        s.load(st)
        s64.append(s)
    for s, d in zip(s64, dts):
        s.step(1, d)

    def one():
        for s, d in zip(s64, dts):
            s.step(1, d)

    ms64 = _time(torch, one, 3)
    res["per_member_fp64"] = {"value": pts / (ms64 / 1e3), "unit": "gp-steps/s", "ms_per_step": ms64,
                              "launches_per_step": 3 * len(s64)}
    res["speedup_vs_per_member_fp64"] = ms64 / ms
    for s in s64:
        s.close()
    return res


def measure_gradient(agcm, inputs, torch):
    """Config 3 end to end: the gradient of J = mean pi^2 over a 20 x 20 deg box
    after 50 FP32 steps at 720x360x30 with respect to the initial state,
    through torch.autograd with 8 checkpointed states (forward, then the
    binomial reverse sweep of adjoint steps and recomputation)."""
    from paper_2103_10114_gb300 import autograd as ag

    I, J, K, n = 720, 360, 30, 50
    st = inputs.baroclinic_jet(I, J, K, seed=3, noise=1e-2, terrain_seed=2)
    g = agcm.Grid(I, J, K, phis=st["phis"])
    dt = g.dt(100.0)
    s = agcm.State(g, agcm.AGCM_FP32)
    mask = ag.box_mask(I, J)
    x0 = {f: torch.as_tensor(st[f], dtype=torch.float32, device="cuda").requires_grad_(True)
          for f in agcm.FIELDS}
    times = []
    for rep in range(2):  # the first run warms up
        for v in x0.values():
            v.grad = None
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = ag.run(s, x0, n, dt, snaps=8)
        jval = ag.box_objective(out["pi"], mask)
        jval.backward()
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    stats = getattr(ag.AgcmSteps, "last_stats", {})
    res = {"seconds": times[-1], "steps": n, "snapshots": 8, "grid": [I, J, K],
           "forward_steps_in_sweep": stats.get("forward_steps"), "max_snapshots": stats.get("max_snapshots"),
           "grad_finite": bool(all(torch.isfinite(v.grad).all() for v in x0.values()))}
    s.close()
    return res


def measure_adjoint(agcm, inputs, torch, steps=5):
    """Config 3 grid 720x360x30: adjoint steps per second (each recomputes its
    two stage states) in FP32 and FP64."""
    I, J, K = 720, 360, 30
    st = inputs.baroclinic_jet(I, J, K, seed=3, noise=1e-2, terrain_seed=2)
    g = agcm.Grid(I, J, K, phis=st["phis"])
    dt = g.dt(100.0)
    res = {}
    for prec, tag in ((agcm.AGCM_FP32, "fp32"), (agcm.AGCM_FP64, "fp64")):
        s = agcm.State(g, prec)
        s.load(st)
        lam = s.store()
        s.step_adjoint(lam, dt)
        ms = _time(torch, lambda: s.step_adjoint(lam, dt), steps)
        s.profile(True)
        s.step_adjoint(lam, dt)
        torch.cuda.synchronize()
        kern = {k: round(v[0], 4) for k, v in s.profile_read().items()}
        s.profile(False)
        s.step(1, dt)
        fms = _time(torch, lambda: s.step(1, dt), steps)
        # bytes model of one adjoint step: the forward recompute (24 words)
        # plus about 30 words of adjoint stages per point
        esz = 4 if prec == agcm.AGCM_FP32 else 8
        rate = I * J * K / (ms / 1e3)
        res[tag] = {"value": rate, "unit": "gp-steps/s", "ms_per_adjoint_step": ms,
                    "ms_per_forward_step": fms, "adjoint_over_forward": ms / fms,
                    "bytes_per_point_step": 54 * esz, "hbm_frac_step": rate * 54 * esz / (peaks()[0] * 1e9),
                    "kernel_ms_per_step": kern}
        if prec == agcm.AGCM_FP32 and NCU_ADJ[0] and NCU_ADJ[0] == kernel_source_hash(ADJ_SOURCES):
            res[tag]["ncu_dram_bytes_per_step"] = NCU_ADJ[1]
            res[tag]["ncu_traffic_over_model"] = NCU_ADJ[1] / (54 * esz * I * J * K)
        s.close()
    return res


if __name__ == "__main__":
    main()
