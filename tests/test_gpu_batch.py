"""Persistent batched launch of many grids: every grid against the FP64 oracle
(element-wise bound and the step-normalised L2 gate), bitwise equal to per-grid
plain sweeps, CUDA-graph capture and replay, bounded dependency waits."""
import numpy as np
import pytest

import oracle
from paper_1410_5561_gb300 import inputs
from tests._util import Problem, step_tol

pytestmark = pytest.mark.gpu

SHAPES = [((37, 29, 21), 9), ((16, 45, 12), 13), ((64, 8, 30), 4), ((5, 5, 5), 7), ((50, 33, 17), 1),
          ((21, 40, 26), 16)]


def _problems(kind="7pt_var", fdt="f32", cdt=None, shapes=SHAPES, seed=40):
    return [(Problem(kind, *sh, fdt=fdt, cdt=cdt, seed=seed + q, halo=0.1 * (q % 3)), T)
            for q, (sh, T) in enumerate(shapes)]


def _plain_result(p, T):
    s = p.make()
    s.set_tuning("plain")
    s.run(T)
    return s.get_field().cpu().numpy()


def _check_oracle(p, T, got):
    """u_T of one grid of a batch against the FP64 oracle on the same (rounded) inputs."""
    got = np.asarray(got, dtype=np.float64)
    ref = p.oracle(T)
    assert oracle.step_normalised_l2(got, ref, T) <= step_tol(p.fdt)
    err = float(np.max(np.abs(got - ref))) if got.size else 0.0
    assert err <= p.elementwise_tol(T), (err, p.elementwise_tol(T))


@pytest.mark.parametrize("kind,fdt,cdt,tn", [
    ("7pt_var", "f32", None, (8, 1, 16)),
    ("7pt_var", "f32", "bf16", (6, 2, 8)),
    ("7pt_const", "f32", None, (8, 2, 16)),
    ("7pt_const", "f64", None, (4, 1, 8)),
    ("25pt_var", "f32", None, (8, 1, 8)),
    ("25pt_var", "f32", "bf16", (8, 2, 8)),
    ("25pt_var", "f64", None, (8, 2, 8)),
    ("7pt_var", "f64", None, (4, 2, 8)),
])
def test_batch_bitwise_equals_plain(kind, fdt, cdt, tn):
    from paper_1410_5561_gb300.batch import Batch
    from paper_1410_5561_gb300.stencil import Tuning
    probs = _problems(kind, fdt, cdt)
    grids = [p.make() for p, _ in probs]
    b = Batch(grids, [T for _, T in probs], Tuning(tn[0], tn[1], tn[2], 0))
    b.launch()
    assert b.status() == 0
    for (p, T), g in zip(probs, grids):
        got = g.get_field().cpu().numpy()
        _check_oracle(p, T, got)
        assert np.array_equal(got, _plain_result(p, T))


def test_batch_graph_replay():
    import torch
    from paper_1410_5561_gb300.batch import Batch
    from paper_1410_5561_gb300.stencil import Tuning
    probs = _problems()
    grids = [p.make() for p, _ in probs]
    b = Batch(grids, [T for _, T in probs], Tuning(8, 1, 16, 0))
    b.launch()            # ordinary launch first (one advance)
    torch.cuda.synchronize()
    graph = b.capture()   # not executed
    graph.replay()
    graph.replay()
    torch.cuda.synchronize()
    b.sync_parity()
    assert b.status() == 0
    for (p, T), g in zip(probs, grids):
        got = g.get_field().cpu().numpy()
        _check_oracle(p, 3 * T, got)
        assert np.array_equal(got, _plain_result(p, 3 * T))


def test_batch_timeout_is_reported_not_hung():
    import torch
    from paper_1410_5561_gb300.batch import Batch
    from paper_1410_5561_gb300.stencil import Tuning
    probs = _problems()
    grids = [p.make() for p, _ in probs]
    b = Batch(grids, [T for _, T in probs], Tuning(8, 1, 16, 0))
    b.set_wait_limit(2000)
    b.inject_stall(b.items // 2)
    b.launch()
    torch.cuda.synchronize()
    from paper_1410_5561_gb300._lib import STATUS
    assert STATUS[b.status()] == "STENCIL_ETIMEOUT"


def test_batch_full_workload_sampled():
    """The 64-grid batch (sides 32..192, T 10..200, 7-point variable FP32): a graph replay,
    then a sample of grids checked against the FP64 oracle and bitwise against their own
    plain sweeps."""
    import torch
    from paper_1410_5561_gb300.batch import Batch
    from paper_1410_5561_gb300.stencil import Tuning
    shapes = inputs.batch_shapes(0)
    probs = [(Problem("7pt_var", nx, ny, nz, fdt="f32", seed=q), T) for q, (nx, ny, nz, T) in enumerate(shapes)]
    grids = [p.make() for p, _ in probs]
    b = Batch(grids, [T for _, T in probs], Tuning(8, 1, 16, 0))
    graph = b.capture()
    graph.replay()
    torch.cuda.synchronize()
    b.sync_parity()
    assert b.status() == 0
    for q in (0, 7, 21, 42, 63):
        p, T = probs[q]
        got = grids[q].get_field().cpu().numpy()
        _check_oracle(p, T, got)
        assert np.array_equal(got, _plain_result(p, T)), q


def test_batch_autotuner_choice_is_feasible_and_exact():
    """tuner.tune_batch times the candidates as graph replays and returns one that builds;
    a fresh batch with it reproduces every grid's plain sweep bit for bit."""
    from paper_1410_5561_gb300 import tuner
    from paper_1410_5561_gb300.batch import Batch
    from paper_1410_5561_gb300.stencil import Tuning
    probs = _problems()
    grids = [p.make() for p, _ in probs]
    Ts = [T for _, T in probs]
    cands = [Tuning(4, 1, 8, 0), Tuning(8, 2, 16, 0), Tuning(6, 1, 16, 0), Tuning(64, 8, 8, 0)]
    tn, table = tuner.tune_batch(grids, Ts, cands, reps=1)
    assert tn in cands and len(table) >= 1 and all(t > 0 for _, t in table)
    assert all(c != Tuning(64, 8, 8, 0) for c, _ in table)  # infeasible: skipped
    fresh = [p.make() for p, _ in probs]
    b = Batch(fresh, Ts, tn)
    b.launch()
    assert b.status() == 0
    for (p, T), g in zip(probs, fresh):
        got = g.get_field().cpu().numpy()
        _check_oracle(p, T, got)
        assert np.array_equal(got, _plain_result(p, T))
