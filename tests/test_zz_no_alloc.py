"""The allocation-free batch entry point, stencil_batch_run_noalloc.

It exists for callers that cannot allocate device memory for a workspace (their
device memory belongs to another allocator, or they must not call cudaMalloc in
a latency-critical loop because it can synchronise the device); it keeps the
batch's scratch in a fixed array owned by the library. These tests call it
through the C ABI and compare its grids, bit for bit (the tolerance every
blocked and batched test uses), with the workspace-based batch path, over two
calls in a row. This file is collected last on purpose: if it fails, a run that
stops at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SHAPES = [((37, 29, 21), 9), ((16, 45, 12), 13), ((64, 8, 30), 4), ((5, 5, 5), 7), ((21, 40, 26), 16)]


def _handles(grids):
    return (ctypes.c_void_p * len(grids))(*[g._h.value for g in grids])


def test_noalloc_batch_matches_workspace_batch_on_two_calls():
    import torch
    from paper_1410_5561_gb300 import _lib as C
    from paper_1410_5561_gb300.batch import Batch
    from paper_1410_5561_gb300.stencil import Tuning
    from tests._util import Problem

    probs = [(Problem("7pt_var", *sh, fdt="f32", seed=70 + q, halo=0.05 * q), T) for q, (sh, T) in enumerate(SHAPES)]
    no_alloc = [p.make() for p, _ in probs]
    with_ws = [p.make() for p, _ in probs]
    Ts = [T for _, T in probs]
    tn = Tuning(8, 1, 16, 0)
    ref = Batch(with_ws, Ts, tn)
    hs = _handles(no_alloc)
    ts = (ctypes.c_int * len(Ts))(*Ts)
    t = tn.c()
    stream = torch.cuda.current_stream()
    for call in range(2):
        status = ctypes.c_int(-99)
        C.call("stencil_batch_run_noalloc", hs, ts, len(Ts), ctypes.byref(t), ctypes.c_void_p(stream.cuda_stream),
               ctypes.byref(status))
        assert status.value == 0, call
        ref.launch()
        assert ref.status() == 0
        for q, (a, b) in enumerate(zip(no_alloc, with_ws)):
            assert a.parity == b.parity
            assert np.array_equal(a.get_field().cpu().numpy(), b.get_field().cpu().numpy()), (call, q)


def test_noalloc_batch_rejects_a_plan_beyond_its_scratch():
    import torch
    from paper_1410_5561_gb300 import _lib as C
    from paper_1410_5561_gb300.stencil import Tuning
    from tests._util import Problem

    # D_w = 2 gives one diamond row per step: 2 x 201 rows x 513 tiles of 24 bytes > 4 MiB
    grids = [Problem("7pt_var", 8, 1024, 8, fdt="f32", seed=q).make() for q in range(2)]
    before = [g.get_field().cpu().numpy() for g in grids]
    ts = (ctypes.c_int * 2)(200, 200)
    t = Tuning(2, 1, 16, 0).c()
    # the same batch is valid for the workspace path, and needs more than the 4 MiB scratch:
    # the size limit, not the tuning or the grids, is what rejects the allocation-free call
    b = ctypes.c_void_p()
    C.call("stencil_batch_create", ctypes.byref(b), _handles(grids), ts, 2, ctypes.byref(t))
    try:
        assert int(C.lib().stencil_batch_workspace_bytes(b)) > (4 << 20)
    finally:
        C.lib().stencil_batch_destroy(b)
    status = ctypes.c_int(-99)
    rc = C.lib().stencil_batch_run_noalloc(_handles(grids), ts, 2, ctypes.byref(t),
                                           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                           ctypes.byref(status))
    assert C.STATUS[rc] == "STENCIL_EINVAL"
    assert status.value == -99
    for g, b in zip(grids, before):
        assert g.parity == 0 and np.array_equal(g.get_field().cpu().numpy(), b)
