"""Wavefront temporal blocking through L2 (STENCIL_WAVEFRONT).

Each unit of the schedule updates its cells with the plain sweep's column code,
so the result must equal the plain sweep bit for bit on any shape, step count
and tuning: a missed dependency (a unit reading a neighbour's plane before it
was written, or overwriting a cell a lower level still reads) shows up as a
changed bit. Oracle parity is checked as well, and the bounded waits are made to
run out on purpose (a stall hook) to check that the timeout is reported.
"""
import numpy as np
import pytest

import oracle
from paper_1410_5561_gb300.stencil import Tuning
from tests._util import Problem, step_tol

pytestmark = pytest.mark.gpu


def _run(p, T, scheme, tuning=None):
    s = p.make()
    s.set_tuning(scheme, tuning)
    s.run(T)
    s.sync()
    return s.get_field().cpu().numpy()


# Tuning(D_w = 2R h, z-chunk planes, rows per tile, coefficient planes prefetched into shared memory)
R1_WAVE = [Tuning(4, 1, 4, 0), Tuning(6, 3, 8, 2), Tuning(8, 2, 16, 0), Tuning(2, 5, 4, 2)]
R4_WAVE = [Tuning(16, 4, 4, 0), Tuning(24, 5, 8, 2), Tuning(8, 8, 16, 0), Tuning(32, 4, 8, 0),
           Tuning(16, 4, 16, 2)]


@pytest.mark.parametrize("tn", R1_WAVE, ids=lambda t: f"dw{t.dw}zc{t.nf}by{t.warps}")
@pytest.mark.parametrize("kind,shape,fdt,cdt", [
    ("7pt_const", (150, 37, 23), "f32", None),
    ("7pt_var", (133, 29, 19), "f32", None),
    ("7pt_var", (40, 43, 17), "f32", "bf16"),
    ("7pt_const", (70, 21, 12), "f64", None),
    ("7pt_var", (33, 19, 14), "f64", None),
])
@pytest.mark.parametrize("T", [1, 5, 8])
def test_wavefront_bitwise_equals_plain_r1(kind, shape, fdt, cdt, tn, T):
    p = Problem(kind, *shape, fdt=fdt, cdt=cdt, seed=21, halo=0.125)
    assert np.array_equal(_run(p, T, "plain"), _run(p, T, "wavefront", tn))


@pytest.mark.parametrize("tn", R4_WAVE, ids=lambda t: f"dw{t.dw}zc{t.nf}by{t.warps}")
@pytest.mark.parametrize("shape,fdt,cdt", [((141, 35, 27), "f32", None), ((38, 25, 30), "f64", None),
                                           ((27, 33, 19), "f32", "bf16")])
@pytest.mark.parametrize("T", [1, 3, 9])
def test_wavefront_bitwise_equals_plain_r4(shape, fdt, cdt, tn, T):
    p = Problem("25pt_var", *shape, fdt=fdt, cdt=cdt, seed=22, halo=-0.25)
    assert np.array_equal(_run(p, T, "plain"), _run(p, T, "wavefront", tn))


@pytest.mark.parametrize("kind,shape,fdt,cdt,T,tn", [
    ("25pt_var", (70, 61, 45), "f32", None, 8, Tuning(16, 8, 8, 0)),
    ("25pt_var", (40, 33, 30), "f32", "bf16", 6, Tuning(24, 4, 8, 0)),
    ("25pt_var", (26, 31, 23), "f64", None, 5, Tuning(16, 4, 4, 0)),
    ("7pt_var", (50, 47, 31), "f32", None, 10, Tuning(8, 4, 8, 0)),
    ("7pt_const", (64, 64, 64), "f64", None, 8, Tuning(4, 8, 8, 0)),
])
def test_wavefront_matches_oracle(kind, shape, fdt, cdt, T, tn):
    p = Problem(kind, *shape, fdt=fdt, cdt=cdt, seed=23)
    got = _run(p, T, "wavefront", tn).astype(np.float64)
    ref = p.oracle(T)
    assert oracle.step_normalised_l2(got, ref, T) <= step_tol(fdt)
    assert np.max(np.abs(got - ref)) <= p.elementwise_tol(T)


def test_wavefront_degenerate_shapes_and_successive_runs():
    for shape in [(1, 1, 1), (5, 2, 3), (9, 3, 40), (300, 1, 5), (3, 70, 2)]:
        p = Problem("25pt_var", *shape, fdt="f32", seed=24, halo=0.5)
        assert np.array_equal(_run(p, 7, "plain"), _run(p, 7, "wavefront", Tuning(16, 4, 4, 0))), shape
    p = Problem("7pt_var", 45, 40, 33, fdt="f32", seed=25)
    s = p.make()
    s.set_tuning("wavefront", Tuning(6, 2, 8, 0))
    for T in (3, 4, 0, 6):
        s.run(T)
    assert s.parity == 13 % 2
    assert np.array_equal(s.get_field().cpu().numpy(), _run(p, 13, "plain"))


def test_wavefront_rejects_malformed_tunings():
    from paper_1410_5561_gb300._lib import StencilError
    s = Problem("25pt_var", 40, 40, 40, fdt="f32", seed=1).make()
    for tn in [Tuning(12, 4, 8, 0),   # D_w not a multiple of 2R
               Tuning(16, 3, 8, 0),   # chunk thinner than R
               Tuning(16, 4, 2, 0),   # tile rows fewer than R
               Tuning(16, 4, 12, 0),   # rows per tile not 4, 8 or 16
               Tuning(16, 4, 8, 3)]:   # coefficient prefetch other than 0 or 2 planes
        with pytest.raises(StencilError):
            s.set_tuning("wavefront", tn)
    w = Problem("7pt_const", 20, 20, 20, fdt="f32", seed=1).make(workspace=False)
    with pytest.raises(StencilError):
        w.set_tuning("wavefront", None)  # needs a workspace


def test_wavefront_timeout_is_reported_not_hung():
    """A unit made to wait on a flag that no unit sets, with a short wait limit, ends the
    launch with the status word set; a new field clears it and the next run is exact."""
    from paper_1410_5561_gb300._lib import STATUS, StencilError
    p = Problem("25pt_var", 60, 40, 36, fdt="f32", seed=26)
    s = p.make()
    s.set_tuning("wavefront", Tuning(16, 4, 8, 0))
    s.set_wait_limit(2000)
    s.inject_stall(9)
    s.run(6)
    assert STATUS[s.status()] == "STENCIL_ETIMEOUT"
    with pytest.raises(StencilError):
        s.sync()
    s.inject_stall(-1)
    s.set_wait_limit(1 << 24)
    u0, _ = p.torch_inputs("cuda")
    s.set_field(u0, halo=p.halo)
    s.run(6)
    assert s.status() == 0
    assert np.array_equal(s.get_field().cpu().numpy(), _run(p, 6, "plain"))


def test_wavefront_run_captured_in_a_cuda_graph():
    import torch
    p = Problem("25pt_var", 41, 37, 29, fdt="f32", seed=27, halo=0.25)
    s = p.make()
    s.set_tuning("wavefront", Tuning(16, 4, 8, 0))
    s.run(2)
    torch.cuda.synchronize()
    g = s.capture(4)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    assert s.status() == 0
    assert np.array_equal(s.get_field().cpu().numpy(), _run(p, 10, "plain"))


def test_wavefront_unit_form_when_streams_outnumber_resident_ctas():
    """With more (level, tile) pairs than CTAs that can be resident, each pass runs as units
    popped in wave order instead of one CTA per (level, tile); both forms must give the
    plain sweep's result, and a stall in the unit form is reported as a timeout."""
    from paper_1410_5561_gb300._lib import STATUS
    p = Problem("7pt_const", 520, 1030, 6, fdt="f32", seed=28, halo=0.5)
    tn = Tuning(4, 1, 4, 0)  # h = 2, 5 x 258 tiles: 2580 streams
    assert np.array_equal(_run(p, 5, "plain"), _run(p, 5, "wavefront", tn))
    s = p.make()
    s.set_tuning("wavefront", tn)
    s.set_wait_limit(2000)
    s.inject_stall(3000)
    s.run(2)
    assert STATUS[s.status()] == "STENCIL_ETIMEOUT"


# Tile copies (xtile = 4): the 25-point stencil with an FP32 field, 8-row tiles, whole tile
# planes staged in shared memory by tensor copies (one CTA per level and tile).
TILE_WAVE = [Tuning(16, 4, 8, 4), Tuning(16, 8, 8, 4), Tuning(24, 5, 8, 4), Tuning(8, 16, 8, 4)]


@pytest.mark.parametrize("tn", TILE_WAVE, ids=lambda t: f"dw{t.dw}zc{t.nf}")
@pytest.mark.parametrize("shape,cdt", [((141, 35, 27), None), ((27, 33, 19), "bf16"), ((256, 16, 12), None),
                                       ((130, 9, 5), "bf16"), ((300, 20, 17), None)])
@pytest.mark.parametrize("T", [1, 3, 9])
def test_tile_copy_wavefront_bitwise_equals_plain(shape, cdt, tn, T):
    p = Problem("25pt_var", *shape, fdt="f32", cdt=cdt, seed=28, halo=-0.375)
    assert np.array_equal(_run(p, T, "plain"), _run(p, T, "wavefront", tn))


@pytest.mark.parametrize("cdt", [None, "bf16"])
def test_tile_copy_wavefront_runs_the_tile_copy_kernel(cdt):
    """The tile-copy pass is the kernel that runs when every (level, tile) CTA fits (and
    not the column walk it falls back to otherwise)."""
    p = Problem("25pt_var", 200, 40, 24, fdt="f32", cdt=cdt, seed=29)
    s = p.make()
    s.set_tuning("wavefront", Tuning(16, 8, 8, 4))
    s.run(4)
    assert s.tile_copy_passes() == 2  # two passes of two levels
    assert np.array_equal(s.get_field().cpu().numpy(), _run(p, 4, "plain"))
    # a tiling with more (level, tile) CTAs than fit at once falls back to the column walk
    q = Problem("25pt_var", 1024, 400, 6, fdt="f32", cdt=cdt, seed=29)
    w = q.make()
    w.set_tuning("wavefront", Tuning(16, 4, 8, 4))
    w.run(2)
    assert w.tile_copy_passes() == 0
    assert np.array_equal(w.get_field().cpu().numpy(), _run(q, 2, "plain"))


@pytest.mark.parametrize("cdt", [None, "bf16"])
def test_tile_copy_wavefront_matches_oracle(cdt):
    p = Problem("25pt_var", 150, 29, 22, fdt="f32", cdt=cdt, seed=30)
    got = _run(p, 6, "wavefront", Tuning(16, 4, 8, 4)).astype(np.float64)
    ref = p.oracle(6)
    assert oracle.step_normalised_l2(got, ref, 6) <= step_tol("f32")
    assert np.max(np.abs(got - ref)) <= p.elementwise_tol(6)


def test_tile_copy_wavefront_degenerate_shapes():
    for shape in [(1, 1, 1), (5, 2, 3), (9, 3, 40), (300, 1, 5), (3, 70, 2), (129, 8, 1)]:
        p = Problem("25pt_var", *shape, fdt="f32", seed=31, halo=0.5)
        assert np.array_equal(_run(p, 5, "plain"), _run(p, 5, "wavefront", Tuning(16, 4, 8, 4))), shape


def test_tile_copy_wavefront_timeout_reported_and_graph_captured():
    """A level-0 CTA made to wait on a flag nothing sets ends the pass with the status word set;
    after a new field the same tuning runs exactly, also replayed from a CUDA graph."""
    import torch
    from paper_1410_5561_gb300._lib import STATUS, StencilError
    p = Problem("25pt_var", 200, 40, 36, fdt="f32", seed=32, halo=0.25)
    s = p.make()
    s.set_tuning("wavefront", Tuning(16, 4, 8, 4))
    s.set_wait_limit(2000)
    s.inject_stall(3)
    s.run(2)
    assert STATUS[s.status()] == "STENCIL_ETIMEOUT"
    with pytest.raises(StencilError):
        s.sync()
    s.inject_stall(-1)
    s.set_wait_limit(1 << 24)
    u0, _ = p.torch_inputs("cuda")
    s.set_field(u0, halo=p.halo)
    s.run(2)
    torch.cuda.synchronize()
    g = s.capture(4)
    g.replay()
    torch.cuda.synchronize()
    assert s.status() == 0
    assert np.array_equal(s.get_field().cpu().numpy(), _run(p, 6, "plain"))


def test_tile_copy_option_only_for_the_25_point_fp32_field():
    from paper_1410_5561_gb300._lib import StencilError
    for kind, fdt in [("7pt_var", "f32"), ("25pt_var", "f64"), ("7pt_const", "f32")]:
        s = Problem(kind, 40, 40, 40, fdt=fdt, seed=1).make()
        with pytest.raises(StencilError):
            s.set_tuning("wavefront", Tuning(16 if kind == "25pt_var" else 4, 4, 8, 4))
