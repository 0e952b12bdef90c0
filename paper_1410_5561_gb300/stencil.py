"""Python face of the C ABI: one :class:`Stencil` per grid, torch tensors as device memory.

Every compute step runs in the CUDA library; this module only allocates the
arrays the library asks for (through torch), passes pointers and sizes, and
builds strided views of the padded layout.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from . import _lib as C

KINDS = {"7pt_const": C.STENCIL_7PT_CONST, "7pt_var": C.STENCIL_7PT_VAR,
         "25pt_var": C.STENCIL_25PT_VAR}
RADIUS = {C.STENCIL_7PT_CONST: 1, C.STENCIL_7PT_VAR: 1, C.STENCIL_25PT_VAR: 4}
NCOEF = {C.STENCIL_7PT_CONST: 0, C.STENCIL_7PT_VAR: 7, C.STENCIL_25PT_VAR: 13}
DTYPES = {torch.float32: C.STENCIL_F32, torch.float64: C.STENCIL_F64, torch.bfloat16: C.STENCIL_BF16}
SCHEMES = {"plain": C.STENCIL_PLAIN, "blocked": C.STENCIL_BLOCKED, "auto": C.STENCIL_AUTO,
           "wavefront": C.STENCIL_WAVEFRONT}


def kind_id(kind) -> int:
    return KINDS[kind] if isinstance(kind, str) else int(kind)


@dataclass(frozen=True)
class Tuning:
    """Blocked-schedule tunables: diamond width D_w, frontlines N_F, warps per CTA
    (the thread group sharing one extruded diamond), x columns per CTA."""
    dw: int
    nf: int = 1
    warps: int = 8
    xtile: int = 128

    def c(self) -> C.stencil_tuning:
        return C.stencil_tuning(self.dw, self.nf, self.warps, self.xtile)


def _ptr(t: torch.Tensor) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


def probe_fma_peak(dtype=torch.float32, iters: int = 4096, device=None) -> float:
    """Measured vector FMA throughput in flop/s (two flops per FMA) on the current device."""
    scratch = torch.empty(65536, dtype=torch.uint8, device=device or "cuda")
    stream = torch.cuda.current_stream(scratch.device)
    sec = ctypes.c_double(0.0)
    fl = ctypes.c_double(0.0)
    C.call("stencil_probe_fma", DTYPES[dtype], int(iters), _ptr(scratch),
           ctypes.c_void_p(stream.cuda_stream), ctypes.byref(sec), ctypes.byref(fl))
    return fl.value / sec.value


class Stencil:
    """One grid: two field arrays (ping-pong), coefficient arrays, workspace."""

    def __init__(self, kind, nx: int, ny: int, nz: int, dtype=torch.float32, coef_dtype=None,
                 device=None, stream: torch.cuda.Stream | None = None, workspace: bool = True):
        self.kind = kind_id(kind)
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.dtype = dtype
        self.coef_dtype = coef_dtype if coef_dtype is not None else dtype
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        C.call("stencil_create", ctypes.byref(h), self.kind, self.nx, self.ny, self.nz,
               DTYPES[dtype], DTYPES[self.coef_dtype], ctypes.c_void_p(self.stream.cuda_stream))
        self._h = h
        self.layout = self._layout(C.STENCIL_FIELD_ARRAY)
        lay = self.layout
        n = lay.bytes // lay.elem_bytes
        self.fields = [torch.empty(n, dtype=dtype, device=self.device) for _ in range(2)]
        self.ncoef = NCOEF[self.kind]
        self.coefs = []
        if self.ncoef:
            cl = self._layout(C.STENCIL_COEF_ARRAY)
            self.coefs = [torch.empty(cl.bytes // cl.elem_bytes, dtype=self.coef_dtype, device=self.device)
                          for _ in range(self.ncoef)]
        wsb = int(C.lib().stencil_workspace_bytes(self._h)) if workspace else 0
        self.workspace = torch.empty(max(wsb, 16), dtype=torch.uint8, device=self.device) if wsb else None
        carr = (ctypes.c_void_p * 13)(*[c.data_ptr() for c in self.coefs])
        C.call("stencil_bind", self._h, _ptr(self.fields[0]), _ptr(self.fields[1]),
               carr if self.ncoef else None,
               _ptr(self.workspace) if self.workspace is not None else None)

    # ------------------------------------------------------------ layout
    def _layout(self, which) -> C.stencil_layout:
        out = C.stencil_layout()
        C.call("stencil_layout_of", self._h, which, ctypes.byref(out))
        return out

    def padded(self, t: torch.Tensor) -> torch.Tensor:
        lay = self.layout
        return t.view(lay.planes, lay.pitch_y, lay.pitch_x)

    def interior(self, t: torch.Tensor) -> torch.Tensor:
        lay = self.layout
        r, xo = lay.radius, lay.x_offset
        return self.padded(t)[r:r + self.nz, r:r + self.ny, xo:xo + self.nx]

    @property
    def parity(self) -> int:
        return C.call("stencil_parity", self._h)

    @property
    def current(self) -> torch.Tensor:
        """Interior view (no copy) of the array holding the current time level."""
        return self.interior(self.fields[self.parity])

    # ------------------------------------------------------------ data
    def set_coeffs(self, scalars=None, arrays=None):
        if self.kind == C.STENCIL_7PT_CONST:
            sc = (ctypes.c_double * 2)(*[float(v) for v in scalars])
            C.call("stencil_set_coeffs", self._h, sc, None, C.STENCIL_HOST)
            return
        arrs = [a.to(self.coef_dtype).contiguous() for a in arrays]
        assert len(arrs) == self.ncoef
        for a in arrs:
            assert tuple(a.shape) == (self.nz, self.ny, self.nx), a.shape
        where = C.STENCIL_HOST if arrs[0].device.type == "cpu" else C.STENCIL_DEVICE
        ptrs = (ctypes.c_void_p * self.ncoef)(*[a.data_ptr() for a in arrs])
        C.call("stencil_set_coeffs", self._h, None, ptrs, where)
        if where == C.STENCIL_HOST:
            self.sync()
        self._keep = arrs  # device sources stay alive until the copies are done

    def set_field(self, u0: torch.Tensor, halo: float = 0.0, async_host: bool = False):
        """Initial field from a dense (nz, ny, nx) tensor on the host or the device.

        ``async_host``: ``u0`` is page-locked host memory copied by the copy engines on this
        grid's stream without waiting (STENCIL_HOST_ASYNC); the caller keeps it unchanged until
        the stream has passed the copy."""
        u = u0.to(self.dtype).contiguous()
        assert tuple(u.shape) == (self.nz, self.ny, self.nx), u.shape
        if async_host:
            assert u.device.type == "cpu" and u.is_pinned() and u.data_ptr() == u0.data_ptr()
            where = C.STENCIL_HOST_ASYNC
        else:
            where = C.STENCIL_HOST if u.device.type == "cpu" else C.STENCIL_DEVICE
        C.call("stencil_set_field", self._h, _ptr(u), float(halo), where)
        if where == C.STENCIL_HOST:
            self.sync()
        self._keep_u = u

    def get_field(self, out: torch.Tensor | None = None, async_host: bool = False) -> torch.Tensor:
        """Dense interior copy of the current field (into ``out`` if given; host or device).

        ``async_host``: ``out`` is page-locked host memory filled by the copy engines on this
        grid's stream; the call returns at once and ``out`` is valid once the stream has passed
        the copy (STENCIL_HOST_ASYNC)."""
        if out is None:
            out = torch.empty((self.nz, self.ny, self.nx), dtype=self.dtype, device=self.device)
        assert out.is_contiguous() and out.dtype == self.dtype
        if async_host:
            assert out.device.type == "cpu" and out.is_pinned()
            where = C.STENCIL_HOST_ASYNC
        else:
            where = C.STENCIL_HOST if out.device.type == "cpu" else C.STENCIL_DEVICE
        C.call("stencil_get_field", self._h, _ptr(out), where)
        return out

    def set_stream(self, stream: torch.cuda.Stream):
        """Enqueue this grid's later calls on ``stream`` (ordering with earlier work is the
        caller's, through events)."""
        C.call("stencil_set_stream", self._h, ctypes.c_void_p(stream.cuda_stream))
        self.stream = stream

    # ------------------------------------------------------------ schedule
    def set_tuning(self, scheme: str = "plain", tuning: Tuning | None = None):
        t = tuning.c() if tuning is not None else None
        C.call("stencil_set_tuning", self._h, SCHEMES[scheme], ctypes.byref(t) if t is not None else None)

    def blocked_smem_bytes(self, tuning: Tuning) -> int:
        t = tuning.c()
        return int(C.lib().stencil_blocked_smem_bytes(self._h, ctypes.byref(t)))

    def run(self, T: int):
        C.call("stencil_run", self._h, int(T))

    def capture(self, T: int) -> torch.cuda.CUDAGraph:
        """A CUDA graph holding stencil_run(T) (not executed by capturing). Each replay
        advances the field by T steps from the array that was current at capture time, so
        replays chain when T is even; the handle's parity is left as before capturing."""
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream(self.device)
        side.wait_stream(self.stream)
        old, par = self.stream, self.parity
        self.set_stream(side)
        try:
            with torch.cuda.graph(g, stream=side):
                self.run(T)
        finally:
            self.set_stream(old)
        if self.parity != par:
            raise RuntimeError("capture of an odd step count: replays would not chain")
        return g

    # ------------------------------------------------------------ adjoint
    def adjoint_workspace(self, T: int, ckpt_every: int = 0) -> torch.Tensor:
        """Device workspace for run_checkpointed / run_adjoint (reused when large enough)."""
        need = int(C.lib().stencil_adjoint_workspace_bytes(self._h, int(T), int(ckpt_every)))
        ws = getattr(self, "_adj_ws", None)
        if ws is None or ws.numel() < need:
            ws = torch.empty(max(need, 16), dtype=torch.uint8, device=self.device)
            self._adj_ws = ws
        return ws

    def run_checkpointed(self, T: int, ckpt_every: int, workspace: torch.Tensor):
        C.call("stencil_run_checkpointed", self._h, int(T), int(ckpt_every), _ptr(workspace),
               ctypes.c_size_t(workspace.numel() * workspace.element_size()))

    def run_adjoint(self, T: int, ckpt_every: int, lam_T: torch.Tensor, g_u0: torch.Tensor, g_coef,
                    workspace: torch.Tensor):
        """lam_T, g_u0: field-layout tensors (self.padded shape); g_coef: FP64 gradient-layout tensors."""
        arr = (ctypes.c_void_p * 13)(*[g.data_ptr() for g in g_coef])
        C.call("stencil_run_adjoint", self._h, int(T), int(ckpt_every), _ptr(lam_T), _ptr(g_u0), arr,
               _ptr(workspace), ctypes.c_size_t(workspace.numel() * workspace.element_size()))

    def new_field_array(self, zero: bool = True) -> torch.Tensor:
        n = self.layout.bytes // self.layout.elem_bytes
        return torch.zeros(n, dtype=self.dtype, device=self.device) if zero else \
            torch.empty(n, dtype=self.dtype, device=self.device)

    def new_grad_array(self) -> torch.Tensor:
        return torch.empty(self.layout.bytes // self.layout.elem_bytes, dtype=torch.float64, device=self.device)

    def interior_of(self, t: torch.Tensor) -> torch.Tensor:
        """Interior view of any array in this grid's element layout (field, coefficient or gradient)."""
        lay = self.layout
        r, xo = lay.radius, lay.x_offset
        return t.view(lay.planes, lay.pitch_y, lay.pitch_x)[r:r + self.nz, r:r + self.ny, xo:xo + self.nx]

    def coef_interior(self, m: int) -> torch.Tensor:
        """Interior view (no copy) of coefficient array m, in the coefficient layout (whose
        pitch differs from the field's when the coefficients are stored in BF16)."""
        cl = self._layout(C.STENCIL_COEF_ARRAY)
        r, xo = cl.radius, cl.x_offset
        v = self.coefs[m].view(cl.planes, cl.pitch_y, cl.pitch_x)
        return v[r:r + self.nz, r:r + self.ny, xo:xo + self.nx]

    @property
    def launches(self) -> int:
        """Kernels this grid has launched so far."""
        n = ctypes.c_longlong(0)
        C.call("stencil_launch_count", self._h, ctypes.byref(n))
        return int(n.value)

    def tile_copy_passes(self) -> int:
        """Wavefront passes run with tile copies into shared memory (tuning xtile = 4)."""
        n = ctypes.c_longlong(0)
        C.call("stencil_tile_copy_passes", self._h, ctypes.byref(n))
        return int(n.value)

    def sync(self):
        """Wait for the grid's stream; raises on a CUDA error or a device-side timeout."""
        C.call("stencil_sync", self._h)

    def status(self) -> int:
        """The device error/timeout word (waits for the stream): 0, or a negative status."""
        return int(C.lib().stencil_status(self._h))

    def set_wait_limit(self, spins: int):
        """Bound on the spin iterations of one dependency wait of the persistent schedule."""
        C.call("stencil_set_wait_limit", self._h, ctypes.c_uint(int(spins)))

    def inject_stall(self, tile: int):
        """Test hook: tile ``tile`` of later persistent launches waits on a flag no tile sets
        (-1 removes it)."""
        C.call("stencil_inject_stall", self._h, int(tile))

    def close(self):
        if getattr(self, "_h", None):
            C.lib().stencil_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
