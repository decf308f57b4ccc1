"""Ensembles of members of uneven resolution: one persistent launch per call,
an autotuner for its launch shape, and CUDA-graph replay.

Two ways to advance the members, both captured whole in one CUDA graph:

* "persistent": one launch of the ensemble kernel (agcm_ensemble_step), in
  one of two forms: one-warp blocks running the column body on items of 32
  columns of 1, 2 or 4 consecutive rows (its launch shape: how many blocks are
  resident per SM, and the row tile); or 256-thread blocks (warps_per_block
  8) running the row-segment body on (member, row segment) items, with the
  rows near the poles on the column body;
* "streams": each member stepped by the single-state kernel (agcm_step) with
  the members spread round-robin over N CUDA streams, so small members run
  side by side.  The single-state kernel reads its grid tables from the launch
  parameters and fits in 80-96 registers, where the persistent kernel, which
  reads each member's tables through a descriptor, needs 168.  "streams-row"
  does the same with every member on the row-segment stage kernel
  (agcm_state_set_stage_kernel 2): a small member alone would not fill the
  GPU with row segments and takes the column kernel, but side by side with
  the others its row segments are the cheaper work per point.

The best choice depends on the member mix and the GPU, so `autotune` times
each candidate on the ensemble itself and keeps the fastest (cached per
member mix and device name for the life of the process).
"""
from __future__ import annotations

import ctypes

from . import agcm

_TUNE_CACHE: dict = {}


class Ensemble:
    def __init__(self, states):
        self.states = list(states)
        arr = (ctypes.c_void_p * len(self.states))(*[s.handle for s in self.states])
        h = ctypes.c_void_p()
        agcm.check(agcm.lib().agcm_ensemble_create(arr, len(self.states), ctypes.byref(h)))
        self._h = h
        self.shape = (1, 0, 1)
        self._streams = []

    @property
    def handle(self):
        return self._h

    def points(self):
        return sum(s.grid.points() for s in self.states)

    def configure(self, warps_per_block, blocks_per_sm=0, rows_per_item=1):
        """Persistent launch: (warps per block, blocks per SM, rows per item).
        Streams: configure("streams", n) steps the members on n streams, each
        member on the stage kernel its own grid calls for; configure("streams-row",
        n) with every member on the row-segment kernel.  Configuring sets the
        members' stage-kernel choice (agcm_state_set_stage_kernel)."""
        if warps_per_block in ("streams", "streams-row"):
            import torch

            n = int(blocks_per_sm)
            if n < 1:
                raise ValueError("need at least one stream")
            self._streams = [torch.cuda.Stream() for _ in range(n)]
            for s in self.states:
                s.set_stage_kernel(2 if warps_per_block == "streams-row" else 0)
            self.shape = (warps_per_block, n)
            return
        for s in self.states:
            s.set_stage_kernel(0)
        agcm.check(agcm.lib().agcm_ensemble_configure(self._h, int(warps_per_block), int(blocks_per_sm)))
        agcm.check(agcm.lib().agcm_ensemble_tile(self._h, int(rows_per_item)))
        self.shape = (int(warps_per_block), int(blocks_per_sm), int(rows_per_item))

    def set_timeout(self, seconds, test_missing_blocks=0):
        agcm.check(agcm.lib().agcm_ensemble_set_timeout(self._h, float(seconds), int(test_missing_blocks)))

    def step(self, nsteps, dts, stream=None):
        if self.shape[0] in ("streams", "streams-row"):
            self._step_streams(nsteps, dts, stream)
            return
        arr = (ctypes.c_double * len(self.states))(*[float(d) for d in dts])
        agcm.check(agcm.lib().agcm_ensemble_step(self._h, int(nsteps), arr, agcm._stream_ptr(stream)))

    def _step_streams(self, nsteps, dts, stream=None):
        """Fork the members over the streams after `stream`, join them back."""
        import torch

        if nsteps == 0:
            return
        main = stream if stream is not None else torch.cuda.current_stream()
        for q in self._streams:
            q.wait_stream(main)
        for k, (s, dt) in enumerate(zip(self.states, dts)):
            s.step(int(nsteps), float(dt), stream=self._streams[k % len(self._streams)])
        for q in self._streams:
            main.wait_stream(q)

    def status(self, stream=None):
        """Synchronises; raises AgcmError(AGCM_ETIMEOUT) if a barrier gave up."""
        agcm.check(agcm.lib().agcm_ensemble_status(self._h, agcm._stream_ptr(stream)))

    def profile(self, enable=True):
        agcm.check(agcm.lib().agcm_ensemble_profile(self._h, 1 if enable else 0, None, None))

    def profile_read(self):
        ms, n = ctypes.c_double(), ctypes.c_int64()
        agcm.check(agcm.lib().agcm_ensemble_profile(self._h, -1, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def signature(self):
        import torch

        return (torch.cuda.get_device_name(), tuple((s.grid.nlon, s.grid.nlat, s.grid.nlev, s.precision)
                                                    for s in self.states))

    def autotune(self, dts, steps=2, candidates=None, verbose=False, graph=False):
        """Time each launch shape on this ensemble (the states are restored
        afterwards) and keep the fastest.  Returns (shape, {shape: ms/step}).
        graph=True times each shape replayed from a CUDA graph of `steps`
        steps (for an ensemble that will be replayed so: the host's launch
        cost, which differs between the shapes, is then not part of a step),
        else called eagerly."""
        import torch

        key = self.signature() + (bool(graph),)
        if key in _TUNE_CACHE:
            self.configure(*_TUNE_CACHE[key])
            return _TUNE_CACHE[key], {}
        if candidates is None:
            candidates = [(1, b, r) for r in (1, 2, 4) for b in (0, 8, 16)]
            candidates += [(8, b, 1) for b in (0, 2)]
            candidates += [("streams", n) for n in (4, 8, 16)]
            candidates += [("streams-row", n) for n in (8, 16)]
        saved = [s.store() for s in self.states]
        times = {}
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for shape in candidates:
            self.configure(*shape)
            self.step(1, dts)
            torch.cuda.synchronize()
            if graph:
                g = self.capture(steps, dts)
                g.replay()
                torch.cuda.synchronize()
                e0.record()
                g.replay()
                e1.record()
            else:
                e0.record()
                self.step(steps, dts)
                e1.record()
            torch.cuda.synchronize()
            self.status()
            times[shape] = e0.elapsed_time(e1) / steps
            if verbose:
                print("ensemble shape", shape, f"{times[shape]:.3f} ms/step")
        best = min(times, key=times.get)
        for s, x in zip(self.states, saved):
            s.load(x)
        self.configure(*best)
        _TUNE_CACHE[key] = best
        return best, times

    def capture(self, nsteps, dts):
        """A CUDA graph of `nsteps` ensemble steps (the persistent launch, or
        the members' launches forked over the streams); replay it with
        graph.replay()."""
        import torch

        self.step(0, dts)  # uploads dt and the vertical means outside the capture
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                self.step(nsteps, dts, stream=s)
        torch.cuda.current_stream().wait_stream(s)
        return g

    def close(self):
        if getattr(self, "_h", None):
            agcm.check(agcm.lib().agcm_ensemble_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
