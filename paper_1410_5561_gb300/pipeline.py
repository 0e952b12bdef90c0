"""Independent problems streamed through one grid with host transfers overlapping the sweeps.

Each job is one initial field on the host, advanced by T steps, with u_T read back to the
host. The host link is far slower than HBM (about 200 GB/s per direction against 6.8 TB/s),
so moving a 1024^3 FP32 field in and out costs close to a third of a 100-step sweep when
the phases run one after another. Here the copy engines move dense fields between the host
and two dense device staging arrays on their own streams, while the sweep of the previous
job runs; the grid's own kernels scatter the staged field into the padded layout before a
sweep and gather u_T out of it afterwards (a device-to-device pass of a few milliseconds).
Per job, ordered by events:

    h2d(i):     host input i -> staging_in       after load(i - 1) has read staging_in
    compute(i): load(i) = set_field(staging_in); run(T);
                store(i) = get_field(staging_out) after d2h(i - 1) has emptied staging_out
    d2h(i):     staging_out -> host output i     after store(i)

so the compute stream holds only the sweeps and the two short device passes, and the link
transfers of jobs i + 1 and i - 1 proceed beside the sweep of job i. Results are identical
to running the jobs one by one (the same kernels on the same values).

The three streams must reach the GPU through different hardware work queues, or the queue
serialises them (a sweep then waits for an unrelated copy out: measured 515-549 GLUP/s at
1024^3 with CUDA's default of 8 queues in a process with many streams, 614-638 with 32).
Processes that create many streams should set CUDA_DEVICE_MAX_CONNECTIONS (e.g. 32) before
CUDA starts; ``bench.py`` does.

The copy engines' rate to page-locked host memory differs between machines of the same kind
(measured 200 GB/s per direction on some GB300 machines, 40-70 GB/s on others), while the
library's copy kernel, which keeps many SM loads in flight, held about 200 GB/s on all of
them. Three modes:

- "staged": the staging scheme above with the copy engines (DMA) moving the host data, each
  transfer split over ``dma_chunks`` streams so that several copy engines can serve it (where
  one engine already reaches the link's rate, 211 GB/s in and 193 out on a GB300 machine, the split
  changes nothing; on a box with slower engines it cut a job from 195 to 173 ms; the
  calibration tries one and ``dma_chunks`` streams);
- "overlap": the same scheme with the library's SM copy (``stencil_copy``) on the transfer
  streams, limited to ``copy_ctas`` CTAs so that it runs on the SMs the persistent sweep
  leaves free (a 1024^3 sweep places 15 clusters of 9 CTAs on 135 of the 152 SMs). Four CTAs
  move a 1024^3 FP32 field in about 30 ms; the host traffic they drive slows the sweep beside
  them by about 18 % (116 -> 137 ms, measured with 4 to 24 CTAs), which the copy engines do not,
  so this mode wins only where the copy engines are slow;
- "direct": the jobs one by one, set_field / run / get_field from and to the host with the
  library's copy kernel on all SMs.

With ``mode="auto"`` the first call times the three on its first input (three staged or
overlapped jobs, whose steady-state cost per job is the distance between consecutive sweeps,
against one direct job) and keeps the fastest; ``calibration`` records the figures.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib as C
from .stencil import Stencil


class Pipeline:
    MODES = ("auto", "staged", "overlap", "direct")

    def __init__(self, grid: Stencil, T: int, halo: float = 0.0, mode: str = "auto", copy_ctas: int = 4,
                 dma_chunks: int = 4):
        if mode not in self.MODES:
            raise ValueError(f"mode must be one of {self.MODES}")
        self.grid = grid
        self.T = int(T)
        self.halo = float(halo)
        self.mode = mode
        self.copy_ctas = int(copy_ctas)
        self.dma_chunks = max(1, int(dma_chunks))
        self._aux = {}  # per transfer stream: the streams its chunks run on
        self.calibration = None
        self._trace = None
        dev = grid.device
        self.staging_in = self.staging_out = None  # dense device arrays of the staged mode
        self.compute = torch.cuda.Stream(dev)
        self.h2d = torch.cuda.Stream(dev)
        self.d2h = torch.cuda.Stream(dev)

    def run(self, inputs: list[torch.Tensor], outputs: list[torch.Tensor], trace: bool = False) -> torch.cuda.Event:
        """Advance every ``inputs[i]`` (page-locked host, (nz, ny, nx)) by T steps into
        ``outputs[i]`` (page-locked host; a buffer listed twice ends up holding the later job's
        result). Returns the event recorded after the last copy out; the outputs are valid once
        it has completed. ``trace``: also record timing events at every phase boundary; after
        completion ``timeline()`` gives each job's phases in milliseconds from the start."""
        if len(inputs) != len(outputs):
            raise ValueError("one output per input")
        g = self.grid
        for t in list(inputs) + list(outputs):
            if t.device.type != "cpu" or not t.is_pinned() or t.dtype != g.dtype or not t.is_contiguous():
                raise ValueError("inputs and outputs must be contiguous page-locked host tensors of the "
                                 "grid's dtype")
        if not inputs:
            return None
        if self.mode == "auto":
            self._calibrate(inputs[0], outputs[0])
        if self.mode == "direct":
            return self._run_direct(inputs, outputs, trace)
        return self._run_staged(inputs, outputs, trace, sm_copies=self.mode == "overlap")

    def _calibrate(self, src: torch.Tensor, dst: torch.Tensor):
        import time
        dev = self.grid.device
        cost = {}
        chunks = self.dma_chunks
        staged = {}
        for k in sorted({1, chunks}):
            self.dma_chunks = k
            self._run_staged([src] * 3, [dst] * 3, trace=True).synchronize()
            tl = self.timeline()
            staged[k] = (tl[2]["run"] - tl[0]["run"]) / 2
        self.dma_chunks = min(staged, key=staged.get)
        cost["staged"] = staged[self.dma_chunks]
        self._run_staged([src] * 3, [dst] * 3, trace=True, sm_copies=True).synchronize()
        tl = self.timeline()
        cost["overlap"] = (tl[2]["run"] - tl[0]["run"]) / 2
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        self._run_direct([src], [dst], False).synchronize()
        cost["direct"] = 1e3 * (time.perf_counter() - t0)
        self.mode = min(cost, key=cost.get)
        self.calibration = {f"{m}_ms_per_job": v for m, v in cost.items()}
        self.calibration["staged_ms_per_job_by_dma_chunks"] = staged
        self.calibration["dma_chunks"] = self.dma_chunks
        self.calibration["chosen"] = self.mode
        if self.mode == "direct":  # the staging arrays are not needed any more
            self.staging_in = self.staging_out = None

    def _run_direct(self, inputs, outputs, trace: bool):
        """One job at a time on the grid's stream; the library's copy kernel moves the host data."""
        g = self.grid
        self._trace = [] if trace else None
        t0 = self._mark(g.stream)
        for src, dst in zip(inputs, outputs):
            ev = {"h2d": self._mark(g.stream)}
            g.set_field(src, halo=self.halo)
            ev["h2d_end"] = ev["set"] = ev["run"] = self._mark(g.stream)
            g.run(self.T)
            ev["run_end"] = ev["d2h"] = self._mark(g.stream)
            g.get_field(dst)
            ev["end"] = self._mark(g.stream)
            if self._trace is not None:
                self._trace.append(ev)
        self._t0 = t0
        return g.stream.record_event()

    def _copy(self, dst: torch.Tensor, src: torch.Tensor, stream, sm_copies: bool):
        """dst <- src (same shape) on `stream`: the library's SM copy with copy_ctas CTAs, or the
        copy engines (also for sizes the SM copy does not take: not a multiple of 16 bytes)."""
        nbytes = src.numel() * src.element_size()
        if sm_copies and nbytes % 16 == 0 and dst.data_ptr() % 16 == 0 and src.data_ptr() % 16 == 0:
            C.call("stencil_copy", ctypes.c_void_p(dst.data_ptr()), ctypes.c_void_p(src.data_ptr()),
                   ctypes.c_size_t(nbytes), self.copy_ctas, ctypes.c_void_p(stream.cuda_stream))
        elif self.dma_chunks == 1 or src.numel() < self.dma_chunks:
            with torch.cuda.stream(stream):
                dst.copy_(src, non_blocking=True)
        else:
            aux = self._aux.get(stream.cuda_stream)
            if aux is None:
                aux = self._aux[stream.cuda_stream] = [torch.cuda.Stream(self.grid.device)
                                                       for _ in range(self.dma_chunks)]
            start = stream.record_event()
            d, s_ = dst.view(-1), src.view(-1)
            n = s_.numel()
            ch = -(-n // len(aux))
            for i, st in enumerate(aux):
                st.wait_event(start)
                with torch.cuda.stream(st):
                    d[i * ch:min(n, (i + 1) * ch)].copy_(s_[i * ch:min(n, (i + 1) * ch)], non_blocking=True)
                stream.wait_event(st.record_event())

    def _run_staged(self, inputs, outputs, trace: bool, sm_copies: bool = False):
        g = self.grid
        if self.staging_in is None:
            shape = (g.nz, g.ny, g.nx)
            self.staging_in = torch.empty(shape, dtype=g.dtype, device=g.device)
            self.staging_out = torch.empty(shape, dtype=g.dtype, device=g.device)
        saved = g.stream
        cur = torch.cuda.current_stream(g.device)
        start = cur.record_event()
        for st in (self.h2d, self.compute, self.d2h):
            st.wait_event(start)
        consumed = emptied = last = None
        g.set_stream(self.compute)
        self._trace = [] if trace else None
        t0 = self._mark(cur)

        for src, dst in zip(inputs, outputs):
            ev = {}
            with torch.cuda.stream(self.h2d):
                if consumed is not None:
                    self.h2d.wait_event(consumed)
                ev["h2d"] = self._mark(self.h2d)
                self._copy(self.staging_in, src, self.h2d, sm_copies)
                ev["h2d_end"] = self._mark(self.h2d)
                loaded = self.h2d.record_event()
            self.compute.wait_event(loaded)
            ev["set"] = self._mark(self.compute)
            g.set_field(self.staging_in, halo=self.halo)
            consumed = self.compute.record_event()
            ev["run"] = self._mark(self.compute)
            g.run(self.T)
            ev["run_end"] = self._mark(self.compute)
            if emptied is not None:
                self.compute.wait_event(emptied)
            g.get_field(self.staging_out)
            ready = self.compute.record_event()
            with torch.cuda.stream(self.d2h):
                self.d2h.wait_event(ready)
                ev["d2h"] = self._mark(self.d2h)
                self._copy(dst, self.staging_out, self.d2h, sm_copies)
                ev["end"] = self._mark(self.d2h)
                emptied = last = self.d2h.record_event()
            if self._trace is not None:
                self._trace.append(ev)
        self._t0 = t0
        for st in (self.h2d, self.compute, self.d2h):
            cur.wait_stream(st)
        g.set_stream(saved)
        saved.wait_stream(cur)
        return last

    def _mark(self, stream):
        if self._trace is None:
            return None
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream)
        return e

    def timeline(self) -> list[dict]:
        """Per job of the last traced run: start and end of its copy in, load, sweep, end of sweep,
        start and end of its copy out, in ms from the start of the run (events must have
        completed)."""
        if not self._trace:
            return []
        return [{k: self._t0.elapsed_time(e) for k, e in ev.items()} for ev in self._trace]
