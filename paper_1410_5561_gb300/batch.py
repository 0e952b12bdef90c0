"""Many independent grids advanced by one persistent launch (stencil_batch_* in the C ABI).

The launch can be captured in a CUDA graph (torch.cuda.CUDAGraph); after graph
replays call :meth:`Batch.sync_parity` so the grids know which array holds
their current time level.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib as C
from .stencil import Stencil, Tuning


class Batch:
    def __init__(self, grids: list[Stencil], T: list[int], tuning: Tuning, stream: torch.cuda.Stream | None = None):
        assert len(grids) == len(T) and len(grids) > 0
        self.grids = list(grids)
        self.T = [int(t) for t in T]
        self.tuning = tuning
        hs = (ctypes.c_void_p * len(grids))(*[g._h.value for g in grids])
        ts = (ctypes.c_int * len(grids))(*self.T)
        tn = tuning.c()
        h = ctypes.c_void_p()
        C.call("stencil_batch_create", ctypes.byref(h), hs, ts, len(grids), ctypes.byref(tn))
        self._h = h
        nbytes = int(C.lib().stencil_batch_workspace_bytes(h))
        dev = grids[0].device
        self.workspace = torch.empty(max(nbytes, 16), dtype=torch.uint8, device=dev)
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        C.call("stencil_batch_bind", h, ctypes.c_void_p(self.workspace.data_ptr()),
               ctypes.c_void_p(self.stream.cuda_stream))

    @property
    def items(self) -> int:
        return C.call("stencil_batch_item_count", self._h)

    @property
    def lups(self) -> int:
        return sum(g.nx * g.ny * g.nz * t for g, t in zip(self.grids, self.T))

    def launch(self, stream: torch.cuda.Stream | None = None):
        s = stream if stream is not None else torch.cuda.current_stream(self.grids[0].device)
        C.call("stencil_batch_launch", self._h, ctypes.c_void_p(s.cuda_stream))

    def capture(self) -> torch.cuda.CUDAGraph:
        """A CUDA graph holding one launch (the grids are not advanced by capturing)."""
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream(self.grids[0].device)
        s.wait_stream(torch.cuda.current_stream(self.grids[0].device))
        with torch.cuda.graph(g, stream=s):
            self.launch(s)
        self.sync_parity()  # capturing did not run the launch
        return g

    @property
    def launches(self) -> int:
        n = ctypes.c_longlong(0)
        C.call("stencil_batch_launch_count", self._h, ctypes.byref(n))
        return int(n.value)

    def status(self) -> int:
        v = ctypes.c_int(0)
        C.call("stencil_batch_status", self._h, ctypes.byref(v))
        return int(v.value)

    def sync_parity(self):
        C.call("stencil_batch_sync_parity", self._h)

    def set_wait_limit(self, spins: int):
        C.call("stencil_batch_set_wait_limit", self._h, ctypes.c_uint(spins))

    def inject_stall(self, item: int):
        C.call("stencil_batch_inject_stall", self._h, int(item))

    def close(self):
        if getattr(self, "_h", None):
            C.lib().stencil_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
