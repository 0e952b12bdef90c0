"""Temporally blocked (diamond / wavefront) sweeps on the GPU.

The blocked kernel evaluates every update with the same device function and the
same operand values as the plain sweep, so the two must agree bit for bit on
any shape, step count and tuning; that is the sharpest detector of tiling
mistakes (a wrong parity array, a missing boundary row, a stale ring slot).
Oracle parity of the blocked path is checked as well.
"""
import numpy as np
import pytest

import oracle
from paper_1410_5561_gb300.stencil import Tuning
from tests._util import Problem, step_tol

pytestmark = pytest.mark.gpu


def _run(p, T, scheme, tuning=None, workspace=True):
    s = p.make(workspace=workspace)
    s.set_tuning(scheme, tuning)
    s.run(T)
    return s.get_field().cpu().numpy()


# Tuning(D_w, N_F, warps, xtile); small x tiles force several x-tiles per diamond
R1_TUNINGS = [Tuning(4, 1, 4, 16), Tuning(8, 1, 8, 8), Tuning(8, 2, 8, 12), Tuning(10, 1, 16, 8),
              Tuning(6, 2, 8, 20), Tuning(2, 1, 2, 4), Tuning(10, 2, 16, 16)]
R4_TUNINGS = [Tuning(8, 1, 8, 8), Tuning(16, 1, 8, 12), Tuning(8, 2, 8, 16), Tuning(8, 2, 4, 20)]


@pytest.mark.parametrize("tn", R1_TUNINGS, ids=lambda t: f"dw{t.dw}nf{t.nf}w{t.warps}x{t.xtile}")
@pytest.mark.parametrize("kind,shape,fdt,cdt", [
    ("7pt_const", (45, 37, 23), "f32", None),
    ("7pt_var", (33, 29, 19), "f32", None),
    ("7pt_var", (40, 13, 17), "f32", "bf16"),
    ("7pt_const", (30, 21, 12), "f64", None),
])
@pytest.mark.parametrize("T", [1, 6, 13])
def test_blocked_bitwise_equals_plain_r1(kind, shape, fdt, cdt, tn, T):
    p = Problem(kind, *shape, fdt=fdt, cdt=cdt, seed=11, halo=0.125)
    a = _run(p, T, "plain")
    b = _run(p, T, "blocked", tn)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("kind,shape,fdt,cdt,tn", [
    ("7pt_const", (128, 30, 22), "f32", None, Tuning(8, 2, 16, 28)),
    ("7pt_const", (128, 30, 22), "f32", None, Tuning(6, 1, 8, 60)),
    ("7pt_const", (256, 19, 16), "f32", None, Tuning(8, 2, 16, 100)),
    ("7pt_var", (96, 26, 18), "f32", None, Tuning(8, 2, 16, 20)),
    ("7pt_var", (96, 26, 18), "f32", "bf16", Tuning(4, 2, 8, 44)),
    ("7pt_const", (64, 20, 14), "f64", None, Tuning(6, 2, 16, 24)),
])
@pytest.mark.parametrize("T", [2, 9])
def test_blocked_steady_state_path_bitwise(kind, shape, fdt, cdt, tn, T):
    """x sizes that are multiples of the vector width, so that whole warps take the
    radius-1 steady-state path (no lane straddles the grid's x boundary)."""
    p = Problem(kind, *shape, fdt=fdt, cdt=cdt, seed=15, halo=0.75)
    a = _run(p, T, "plain")
    b = _run(p, T, "blocked", tn)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("tn", R4_TUNINGS, ids=lambda t: f"dw{t.dw}nf{t.nf}w{t.warps}x{t.xtile}")
@pytest.mark.parametrize("shape,fdt,cdt", [((29, 35, 21), "f32", None), ((18, 25, 14), "f64", None),
                                           ((27, 33, 19), "f32", "bf16")])
@pytest.mark.parametrize("T", [1, 5, 9])
def test_blocked_bitwise_equals_plain_r4(shape, fdt, cdt, tn, T):
    p = Problem("25pt_var", *shape, fdt=fdt, cdt=cdt, seed=12, halo=-0.25)
    a = _run(p, T, "plain")
    b = _run(p, T, "blocked", tn)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("kind,shape,fdt,cdt,tn", [
    ("7pt_const", (245, 26, 20), "f32", None, Tuning(8, 2, 16, 116)),
    ("7pt_var", (233, 18, 15), "f32", None, Tuning(8, 1, 16, 116)),
    ("7pt_var", (240, 21, 13), "f32", "bf16", Tuning(8, 2, 16, 116)),
    ("7pt_const", (251, 22, 17), "f32", None, Tuning(4, 1, 4, 124)),
    ("7pt_const", (110, 20, 12), "f64", None, Tuning(8, 2, 16, 52)),
])
@pytest.mark.parametrize("T", [1, 7, 13])
def test_blocked_wide_x_tiles_bitwise(kind, shape, fdt, cdt, tn, T):
    """x tiles at and just past the width one 32-vector chunk holds (tile rows of one and
    of two chunks), several tiles per row, a partial last tile."""
    p = Problem(kind, *shape, fdt=fdt, cdt=cdt, seed=14, halo=0.5)
    a = _run(p, T, "plain")
    b = _run(p, T, "blocked", tn)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("kind,shape,fdt,cdt,T,tn", [
    ("7pt_const", (64, 64, 64), "f64", None, 8, Tuning(8, 1, 8, 48)),
    ("7pt_const", (64, 64, 64), "f64", None, 8, Tuning(10, 1, 16, 16)),
    ("7pt_var", (50, 47, 31), "f32", None, 10, Tuning(8, 1, 8, 16)),
    ("7pt_var", (50, 47, 31), "f32", "bf16", 10, Tuning(8, 2, 16, 24)),
    ("7pt_var", (36, 41, 22), "f64", None, 9, Tuning(6, 1, 8, 12)),
    ("25pt_var", (40, 33, 30), "f32", None, 6, Tuning(16, 1, 8, 20)),
    ("25pt_var", (40, 33, 30), "f32", "bf16", 6, Tuning(16, 1, 8, 20)),
    ("25pt_var", (26, 31, 23), "f64", None, 5, Tuning(8, 2, 8, 12)),
])
def test_blocked_matches_oracle(kind, shape, fdt, cdt, T, tn):
    p = Problem(kind, *shape, fdt=fdt, cdt=cdt, seed=13)
    got = _run(p, T, "blocked", tn).astype(np.float64)
    ref = p.oracle(T)
    assert oracle.step_normalised_l2(got, ref, T) <= step_tol(fdt)
    assert np.max(np.abs(got - ref)) <= p.elementwise_tol(T)


def test_blocked_small_and_degenerate_shapes():
    for shape in [(1, 1, 1), (5, 2, 3), (9, 3, 40), (64, 1, 5), (3, 70, 2)]:
        p = Problem("7pt_var", *shape, fdt="f32", seed=14, halo=0.5)
        for tn in [Tuning(4, 1, 4, 4), Tuning(8, 2, 8, 16)]:
            a = _run(p, 7, "plain")
            b = _run(p, 7, "blocked", tn)
            assert np.array_equal(a, b), (shape, tn)


def test_blocked_successive_runs_and_parity():
    p = Problem("7pt_const", 40, 40, 40, fdt="f32", seed=15)
    s = p.make()
    s.set_tuning("blocked", Tuning(8, 1, 8, 16))
    s.run(3)
    s.run(4)
    s.run(0)
    s.run(6)
    a = s.get_field().cpu().numpy()
    assert s.parity == 13 % 2
    b = _run(p, 13, "plain")
    assert np.array_equal(a, b)


def test_infeasible_tuning_rejected():
    from paper_1410_5561_gb300._lib import StencilError
    p = Problem("7pt_const", 64, 64, 64, fdt="f32", seed=1)
    s = p.make()
    with pytest.raises(StencilError):
        s.set_tuning("blocked", Tuning(7, 1, 8, 1))    # D_w not a multiple of 2R
    with pytest.raises(StencilError):
        s.set_tuning("blocked", Tuning(64, 8, 8, 64))  # rings far beyond shared memory
    with pytest.raises(StencilError):
        s.set_tuning("blocked", Tuning(8, 1, 8, 6))    # x tile not a multiple of 4 floats
    with pytest.raises(StencilError):
        s.set_tuning("blocked", Tuning(8, 1, 8, 4100))  # x tile wider than the 4096-column limit
    with pytest.raises(StencilError):
        s.set_tuning("blocked", Tuning(8, 3, 8, 64))   # more than two frontlines
    with pytest.raises(StencilError):
        s.set_tuning("blocked", Tuning(24, 1, 8, 64))   # 288 rows exceed 8 warps x 4 two-row items
    with pytest.raises(StencilError):
        s.set_tuning("blocked", Tuning(8, 1, 8, 2))    # x tile narrower than one vector


@pytest.mark.parametrize("kind,shape,fdt,tn", [
    ("7pt_const", (45, 37, 23), "f32", Tuning(8, 2, 8, 12)),
    ("7pt_var", (33, 29, 19), "f32", Tuning(6, 1, 8, 8)),
    ("25pt_var", (29, 35, 21), "f32", Tuning(16, 1, 8, 12)),
    ("7pt_const", (30, 21, 12), "f64", Tuning(8, 1, 8, 16)),
])
@pytest.mark.parametrize("T", [3, 11])
def test_row_launches_and_persistent_clusters_agree(kind, shape, fdt, tn, T):
    """Without a workspace the blocked schedule runs one launch per diamond row; with one
    it is a single persistent launch over the dependency-ordered tile list."""
    p = Problem(kind, *shape, fdt=fdt, seed=16, halo=0.2)
    a = _run(p, T, "blocked", tn, workspace=False)
    b = _run(p, T, "blocked", tn, workspace=True)
    c = _run(p, T, "plain")
    assert np.array_equal(a, b) and np.array_equal(a, c)


def test_persistent_plan_larger_than_workspace_is_split():
    """D_w = 2 gives one diamond row per step: 301 rows x 1025 tiles do not fit the
    4 MiB workspace, so the run is split into parts; the result must not change."""
    p = Problem("7pt_var", 4, 2048, 4, fdt="f32", seed=17)
    a = _run(p, 300, "plain")
    b = _run(p, 300, "blocked", Tuning(2, 1, 4, 4))
    assert np.array_equal(a, b)


def test_auto_scheme_and_default_tuning():
    """STENCIL_AUTO: the plain sweep for FP64 and the 25-point stencil, the default blocked
    tuning otherwise (N_F = 2 where it fits); both give the plain sweep's result."""
    for kind, fdt, cdt, blocked in [("7pt_const", "f32", None, True), ("7pt_var", "f32", "bf16", True),
                                    ("7pt_const", "f64", None, False), ("25pt_var", "f32", None, False)]:
        p = Problem(kind, 70, 23, 19, fdt=fdt, cdt=cdt, seed=16)
        s = p.make()
        s.set_tuning("auto")
        n0 = s.launches
        s.run(9)
        launches = s.launches - n0
        assert (launches == 1) == blocked, (kind, fdt, launches)  # persistent blocked: one launch
        assert np.array_equal(s.get_field().cpu().numpy(), _run(p, 9, "plain")), (kind, fdt)
        d = p.make()
        d.set_tuning("blocked")  # library default tuning
        d.run(9)
        assert np.array_equal(d.get_field().cpu().numpy(), _run(p, 9, "plain")), (kind, fdt)


def test_persistent_timeout_is_reported_not_hung():
    """A dependency wait of the single-grid persistent launch that runs out (a tile made to
    wait on a flag no tile sets, with a short limit) ends the launch with the status word
    set: stencil_status and stencil_sync report STENCIL_ETIMEOUT instead of returning
    invalid data silently. A new field clears it, and the next run is exact again."""
    from paper_1410_5561_gb300._lib import STATUS, StencilError
    p = Problem("7pt_const", 70, 64, 24, fdt="f32", seed=18)
    s = p.make()
    s.set_tuning("blocked", Tuning(8, 1, 8, 16))
    s.run(5)
    assert s.status() == 0
    s.set_wait_limit(2000)
    s.inject_stall(7)
    s.run(13)
    assert STATUS[s.status()] == "STENCIL_ETIMEOUT"
    with pytest.raises(StencilError):
        s.sync()
    s.inject_stall(-1)
    s.set_wait_limit(1 << 24)
    u0, _ = p.torch_inputs("cuda")
    s.set_field(u0, halo=p.halo)
    assert s.status() == 0
    s.run(13)
    s.sync()
    assert s.status() == 0
    assert np.array_equal(s.get_field().cpu().numpy(), _run(p, 13, "plain"))
    s.inject_stall(1 << 30)  # beyond the plan: no effect
    s.set_field(u0, halo=p.halo)
    s.run(13)
    assert s.status() == 0


@pytest.mark.parametrize("kind,fdt,cdt,tn", [
    ("7pt_const", "f32", None, Tuning(8, 2, 16, 16)),
    ("7pt_var", "f32", "bf16", Tuning(8, 1, 8, 16)),
    ("25pt_var", "f32", None, Tuning(16, 1, 8, 12)),
])
def test_persistent_run_captured_in_a_cuda_graph(kind, fdt, cdt, tn):
    """stencil_run of the persistent blocked schedule enqueues kernels and memsets only (no
    host copy of a plan, no wait), so it can be captured; two replays of run(6) give the
    plain sweep's 12 steps bit for bit."""
    import torch
    p = Problem(kind, 41, 37, 19, fdt=fdt, cdt=cdt, seed=19, halo=0.25)
    s = p.make()
    s.set_tuning("blocked", tn)
    s.run(2)  # first run after set_field (status word reset) outside the graph
    torch.cuda.synchronize()
    g = s.capture(6)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    assert s.status() == 0
    assert np.array_equal(s.get_field().cpu().numpy(), _run(p, 14, "plain"))


def test_model_guided_tuner_times_three_and_keeps_the_best():
    """The tuner predicts the first six candidates (Eq. 5 bytes at the kernel's streaming rate,
    useful columns, frontlines, register pressure), times at most three of them, and its
    choice is within 10 % of the best of all six timed exhaustively."""
    import torch
    from paper_1410_5561_gb300 import tuner
    p = Problem("7pt_const", 320, 320, 320, fdt="f32", seed=3)
    s = p.make()
    T = 24
    tn, table = tuner.best_blocked(s, T, reps=2, max_candidates=6, max_timed=3)
    assert 1 <= len(table) <= 3
    preds = tuner.last_predictions
    assert len(preds) >= len(table) and all(pr > 0 for _, pr, _ in preds)
    full, full_table = tuner.best_blocked(s, T, reps=2, max_candidates=6)
    best_full = min(t for _, t in full_table)
    s.set_tuning("blocked", tn)
    torch.cuda.synchronize()
    mine = tuner._time_run(s, T, 3)
    assert mine <= 1.10 * best_full, (tn, mine, full, best_full)
