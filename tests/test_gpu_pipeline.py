"""Host transfers overlapped with sweeps: the staged pipeline, asynchronous copy-engine
transfers, the stream switch and the halo kept between jobs, each against the plain
one-job-at-a-time path (bit for bit: the same kernels on the same values)."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1410_5561_gb300 import _lib as C
from paper_1410_5561_gb300.pipeline import Pipeline
from paper_1410_5561_gb300.stencil import Tuning
from tests._util import Problem

pytestmark = pytest.mark.gpu


def _sequential(p, jobs, T, scheme, tn, halo):
    s = p.make()
    s.set_tuning(scheme, tn)
    out = []
    for u in jobs:
        s.set_field(u, halo=halo)
        s.run(T)
        out.append(s.get_field().cpu())
    return out


@pytest.mark.parametrize("kind,shape,fdt,cdt,scheme,tn", [
    ("7pt_const", (70, 33, 29), "f32", None, "blocked", Tuning(8, 2, 16, 56)),
    ("7pt_var", (45, 26, 31), "f32", "bf16", "auto", None),
    ("25pt_var", (29, 24, 22), "f64", None, "plain", None),
])
@pytest.mark.parametrize("T", [1, 8])
@pytest.mark.parametrize("mode", ["staged", "overlap", "direct", "auto"])
def test_pipeline_equals_jobs_one_by_one(kind, shape, fdt, cdt, scheme, tn, T, mode):
    p = Problem(kind, *shape, fdt=fdt, cdt=cdt, seed=21, halo=0.25)
    tdt = {"f32": torch.float32, "f64": torch.float64}[fdt]
    g = torch.Generator().manual_seed(5)
    jobs = [(torch.rand(shape[::-1], generator=g, dtype=torch.float64) * 2 - 1).to(tdt).pin_memory()
            for _ in range(5)]
    want = _sequential(p, jobs, T, scheme, tn, p.halo)
    s = p.make()
    s.set_tuning(scheme, tn)
    outs = [torch.empty_like(u).pin_memory() for u in jobs]
    pipe = Pipeline(s, T, halo=p.halo, mode=mode)
    pipe.run(jobs, outs).synchronize()
    if mode == "auto":  # calibrated once on the first input, then one of the three modes
        assert pipe.mode in ("staged", "overlap", "direct") and pipe.calibration["chosen"] == pipe.mode
    for a, b in zip(outs, want):
        assert torch.equal(a, b)
    # a second pass through the same pipeline (halo kept, grid reused) gives the same
    outs2 = [torch.empty_like(u).pin_memory() for u in jobs]
    pipe.run(jobs[::-1], outs2, trace=True).synchronize()
    for a, b in zip(outs2, want[::-1]):
        assert torch.equal(a, b)
    # the traced phases are ordered as the events that link the streams require
    tl = pipe.timeline()
    assert len(tl) == len(jobs)
    for i, j in enumerate(tl):
        assert j["h2d"] <= j["h2d_end"] <= j["set"] <= j["run"] <= j["run_end"] <= j["d2h"] <= j["end"]
        if i:
            assert j["run"] >= tl[i - 1]["run_end"] and j["h2d"] >= tl[i - 1]["set"]
    # the grid is back on its own stream and usable one job at a time
    s.set_field(jobs[0], halo=p.halo)
    s.run(T)
    assert torch.equal(s.get_field().cpu(), want[0])
    with pytest.raises(ValueError):
        pipe.run([jobs[0].clone()], [outs[0]])  # pageable input


def test_async_host_transfers_and_halo_changes():
    p = Problem("7pt_var", 40, 21, 17, fdt="f32", seed=22, halo=0.0)
    s = p.make()
    s.set_tuning("blocked", Tuning(8, 1, 8, 16))
    u = torch.from_numpy(p.u0).float().pin_memory()
    ref = {}
    for halo in (0.0, 0.5):
        q = Problem("7pt_var", 40, 21, 17, fdt="f32", seed=22, halo=halo)
        ref[halo] = _sequential(q, [u], 6, "plain", None, halo)[0]
    out = torch.empty_like(u).pin_memory()
    # the halo follows each call's value; unchanged values keep the arrays' halo
    for halo in (0.5, 0.5, 0.0, 0.0, 0.5):
        s.set_field(u, halo=halo, async_host=True)
        s.run(6)
        s.get_field(out, async_host=True)
        s.sync()
        assert torch.equal(out, ref[halo]), halo
    # a stream switch moves later work to the new stream
    side = torch.cuda.Stream()
    s.set_stream(side)
    s.set_field(u, halo=0.0, async_host=True)
    s.run(6)
    s.get_field(out, async_host=True)
    side.synchronize()
    assert torch.equal(out, ref[0.0])


def test_async_host_transfer_rejects_pageable_and_device_memory():
    p = Problem("7pt_const", 12, 10, 8, fdt="f32", seed=23)
    s = p.make()
    pageable = torch.zeros((8, 10, 12), dtype=torch.float32)
    dev = torch.zeros((8, 10, 12), dtype=torch.float32, device="cuda")
    for t in (pageable, dev):
        with pytest.raises(C.StencilError) as e:
            C.call("stencil_set_field", s._h, ctypes.c_void_p(t.data_ptr()), 0.0, C.STENCIL_HOST_ASYNC)
        assert e.value.status == -1
        with pytest.raises(C.StencilError) as e:
            C.call("stencil_get_field", s._h, ctypes.c_void_p(t.data_ptr()), C.STENCIL_HOST_ASYNC)
        assert e.value.status == -1
    # set_coeffs has no asynchronous form
    c = (ctypes.c_double * 2)(0.4, 0.1)
    with pytest.raises(C.StencilError):
        C.call("stencil_set_coeffs", s._h, c, None, C.STENCIL_HOST_ASYNC)
    assert np.isfinite(s.get_field().cpu().numpy()).all()


def test_sm_copy_between_host_and_device():
    """stencil_copy moves bytes between page-locked host and device memory in both directions
    and device to device, with any CTA count, and rejects unaligned pointers or sizes."""
    import ctypes
    from paper_1410_5561_gb300 import _lib as C
    from paper_1410_5561_gb300._lib import StencilError
    g = torch.Generator().manual_seed(9)
    n = 3 * 1024 * 1024 + 12  # not a multiple of the copy's unrolled stride
    host = torch.randint(-2**31, 2**31 - 1, (n,), generator=g, dtype=torch.int32).pin_memory()
    dev = torch.empty(n, dtype=torch.int32, device="cuda")
    back = torch.empty(n, dtype=torch.int32).pin_memory()
    st = torch.cuda.current_stream()
    for ctas in (1, 7, 64):
        dev.zero_()
        back.zero_()
        C.call("stencil_copy", ctypes.c_void_p(dev.data_ptr()), ctypes.c_void_p(host.data_ptr()),
               ctypes.c_size_t(4 * n), ctas, ctypes.c_void_p(st.cuda_stream))
        dev2 = torch.empty_like(dev)
        C.call("stencil_copy", ctypes.c_void_p(dev2.data_ptr()), ctypes.c_void_p(dev.data_ptr()),
               ctypes.c_size_t(4 * n), ctas, ctypes.c_void_p(st.cuda_stream))
        C.call("stencil_copy", ctypes.c_void_p(back.data_ptr()), ctypes.c_void_p(dev2.data_ptr()),
               ctypes.c_size_t(4 * n), ctas, ctypes.c_void_p(st.cuda_stream))
        torch.cuda.synchronize()
        assert torch.equal(back, host)
    pageable = torch.empty(64, dtype=torch.int32)  # not page-locked: refused before any access
    for dst, src, nbytes, ctas in [(dev.data_ptr(), pageable.data_ptr(), 64, 4),
                                   (pageable.data_ptr(), dev.data_ptr(), 64, 4),
                                   (dev.data_ptr() + 4, host.data_ptr(), 16, 4),   # unaligned destination
                                   (dev.data_ptr(), host.data_ptr(), 20, 4),       # size not a multiple of 16
                                   (dev.data_ptr(), host.data_ptr(), 16, 0)]:      # no CTA
        with pytest.raises(StencilError):
            C.call("stencil_copy", ctypes.c_void_p(dst), ctypes.c_void_p(src), ctypes.c_size_t(nbytes), ctas,
                   ctypes.c_void_p(st.cuda_stream))
