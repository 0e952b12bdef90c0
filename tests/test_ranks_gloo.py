"""The bench's multi-process plumbing (one process per GPU under torchrun, replicas only):
barrier, max over ranks and the whole-job aggregate, run as two gloo ranks on the CPU."""
import importlib.util
import json
import os
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out_dir: str):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "WORLD_SIZE": str(world),
                       "RANK": str(rank), "LOCAL_RANK": str(rank)})
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    r = bench.Ranks("gloo")
    r.barrier()
    t = r.maxall(1.0 + rank)                    # slowest rank's time
    v = r.aggregate(100.0, 2.0 + 3.0 * rank)    # 100 units per rank over the max time
    r.barrier()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"world": r.world, "root": r.root, "max": t, "value": v}, f)
    r.close()


def test_two_gloo_ranks(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"rank{i}.json")) for i in range(world)]
    assert [x["root"] for x in res] == [True, False]
    for x in res:
        assert x["world"] == 2
        assert x["max"] == 2.0
        assert x["value"] == pytest.approx(2 * 100.0 / 5.0)


def test_single_process_needs_no_process_group(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    spec = importlib.util.spec_from_file_location("bench_under_test1", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    r = bench.Ranks("gloo")
    assert r.world == 1 and r.root and r.dist is None
    r.barrier()
    assert r.maxall(3.5) == 3.5 and r.aggregate(10.0, 2.0) == 5.0


def test_pipeline_summary_of_a_timeline():
    """The e2e phase summary: mean sweep, gap between sweeps, copies, exposed ends."""
    jobs = []
    for i in range(3):
        r = 10.0 + 160.0 * i
        jobs.append({"h2d": r - 30.0, "h2d_end": r - 10.0, "set": r - 2.0, "run": r, "run_end": r + 150.0,
                     "d2h": r + 152.0, "end": r + 180.0})
    spec = importlib.util.spec_from_file_location("bench_summary", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    out = bench.pipeline_summary(jobs)
    assert out["sweep"] == 150.0
    assert out["gap_between_sweeps"] == 10.0
    assert out["copy_in"] == 20.0 and out["copy_out"] == 28.0
    assert out["first_sweep_start"] == 10.0 and out["after_last_sweep"] == 30.0
    assert out["total"] == jobs[-1]["end"]
    assert bench.pipeline_summary([]) is None
