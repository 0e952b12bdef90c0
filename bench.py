#!/usr/bin/env python3
"""GLUP/s and HBM bytes per LUP of the temporally blocked vs the plain sweep on GB300.

One step = one stencil_run(T = 100) of the 7-point constant-coefficient Jacobi
sweep (Listing 1, c0 = 0.4, c1 = 0.1) on a 1024^3 FP32 interior with a zero
Dirichlet halo, through the temporally blocked schedule with an autotuned
tuning; the plain one-step sweep is timed beside it, and (on one GPU) every
other stencil of the library is measured plain vs blocked as well.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank runs its own replica (the sweep does not
shard across GPUs here: replicas only); the reported value is the aggregate
GLUP/s over the max-over-ranks time. `--impl reference` times the FP64 CPU
oracle on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

# More hardware work queues than CUDA's default 8, so that the end-to-end pipeline's copy
# streams and its compute stream do not land on one queue and serialise (set before CUDA starts)
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GLUP/s and ncu HBM bytes/LUP, blocked vs plain sweep on one GB300, per stencil"
HEADLINE = dict(kind="7pt_const", n=1024, fdt="f32", cdt=None, T=100)
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "blocked_persist_kernel_7pt_const_f32_traffic.txt")
CPU_SAMPLE_N = 256
CPU_BASELINE_N = 512


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip the per-stencil table")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--case", default=None,
                    help="profiling helper: KIND:N:FIELD:COEF:SCHEME:T[:dw,nf,warps,xtile] runs that "
                         "case twice and exits (no JSON); also adjoint:KIND:N:FIELD:T and "
                         "batch[:dw,nf,warps]")
    return ap.parse_args()


def run_case(spec: str, seed: int):
    """Set up one grid and run it twice (used for ncu captures of single kernels).
    Also: adjoint:KIND:N:FIELD:T (forward with checkpoints + adjoint through autograd, twice)
    and batch[:dw,nf,warps] (the 64-grid 7-point variable FP32 batch, launched twice)."""
    import torch
    from paper_1410_5561_gb300.stencil import Tuning
    parts = spec.split(":")
    dev = torch.device("cuda", 0)
    if parts[0] == "adjoint":
        from paper_1410_5561_gb300 import inputs
        from paper_1410_5561_gb300.autograd import sweep
        kind, n, fdt, T = parts[1], int(parts[2]), parts[3], int(parts[4])
        s, u0 = make_grid(kind, n, fdt, None, seed, dev)
        coefs = torch.stack([s.interior_of(c).clone() for c in s.coefs])
        target = torch.empty_like(u0)
        inputs.fill_uniform_torch(target, seed, inputs.STREAM_TARGET, -1.0, 1.0)
        for _ in range(2):
            u = u0.clone().requires_grad_(True)
            c = coefs.clone().requires_grad_(True)
            (0.5 * ((sweep(u, c, s, T) - target) ** 2).sum()).backward()
        torch.cuda.synchronize(dev)
        print("case done", spec, flush=True)
        return 0
    if parts[0] == "batch":
        from paper_1410_5561_gb300 import inputs
        from paper_1410_5561_gb300.batch import Batch
        tn = Tuning(*[int(v) for v in parts[1].split(",")], 0) if len(parts) > 1 else Tuning(4, 1, 8, 0)
        shapes = inputs.batch_shapes(seed)
        grids = [make_grid_shape("7pt_var", nx, ny, nz, "f32", None, seed + q, dev)[0]
                 for q, (nx, ny, nz, T) in enumerate(shapes)]
        b = Batch(grids, [sh[3] for sh in shapes], tn)
        for _ in range(2):
            b.launch()
        torch.cuda.synchronize(dev)
        assert b.status() == 0
        print("case done", spec, flush=True)
        return 0
    kind, n, fdt, cdt, scheme, T = parts[0], int(parts[1]), parts[2], parts[3], parts[4], int(parts[5])
    tn = Tuning(*[int(v) for v in parts[6].split(",")]) if len(parts) > 6 else None
    s, _ = make_grid(kind, n, fdt, None if cdt in ("", "-") else cdt, seed, torch.device("cuda", 0))
    s.set_tuning(scheme, tn)
    s.run(T)
    s.sync()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s.stream)
    s.run(T)
    e1.record(s.stream)
    e1.synchronize()
    sec = e0.elapsed_time(e1) / 1e3
    print(f"case done {spec} {1e3 * sec:.3f} ms {float(n) ** 3 * T / sec / 1e9:.1f} GLUP/s", flush=True)
    return 0


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


# ----------------------------------------------------------------- CPU oracle arm

def host_description():
    """The host cores the CPU baseline runs on: logical CPUs, the ones this process may
    use (affinity), the CPU model and the clock the kernel reports."""
    info = {"nproc": os.cpu_count()}
    try:
        info["affinity_cpus"] = len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        info["affinity_cpus"] = None
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None and os.path.exists("/proc/cpuinfo"):
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
    info["cpu_model"] = model
    for key, fname in (("max_mhz", "cpuinfo_max_freq"), ("cur_mhz", "scaling_cur_freq")):
        p = f"/sys/devices/system/cpu/cpu0/cpufreq/{fname}"
        try:
            with open(p) as f:
                info[key] = int(f.read().strip()) / 1000.0
        except (OSError, ValueError):
            info[key] = None
    return info


def cpu_oracle_sample(budget_s: float = 15.0, n: int = CPU_BASELINE_N, seed: int = 0,
                      single_core_s: float = 5.0):
    """Time the FP64 oracle (7-point constant, Listing 1) on an n^3 sample on the host
    cores; T is chosen so the sample takes about ``budget_s`` seconds. A second, single-core
    run at reduced T (about ``single_core_s`` seconds) is reported beside it."""
    import oracle
    from paper_1410_5561_gb300 import inputs
    u0 = inputs.field_u0(seed, n, n, n)
    oracle.sweep("7pt_const", u0, 1)  # first call: thread pool start-up, page faults
    # per-step time from the difference of two runs (each call also pads and copies the grid)
    t0 = time.perf_counter()
    oracle.sweep("7pt_const", u0, 2)
    t2 = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.sweep("7pt_const", u0, 6)
    t6 = time.perf_counter() - t0
    t1 = max((t6 - t2) / 4, 1e-4)
    T = max(1, min(1000, int(max(budget_s - (t2 - 2 * t1), 1.0) / t1)))
    t0 = time.perf_counter()
    oracle.sweep("7pt_const", u0, T)
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    # one core, reduced T (stated)
    t0 = time.perf_counter()
    oracle.sweep("7pt_const", u0, 1, nthreads=1)
    t1s = max(time.perf_counter() - t0, 1e-3)
    T1 = max(1, min(50, int(single_core_s / t1s)))
    t0 = time.perf_counter()
    oracle.sweep("7pt_const", u0, T1, nthreads=1)
    dt1 = time.perf_counter() - t0
    return {"value": n ** 3 * T / dt / 1e9, "unit": "GLUP/s", "cores": cores, "kind": "oracle",
            "sample": f"7pt-const FP64 oracle, {n}^3 interior, T={T} steps ({dt:.1f} s), OpenMP over k",
            "host": host_description(),
            "single_core": {"value": n ** 3 * T1 / dt1 / 1e9, "unit": "GLUP/s", "cores": 1,
                            "sample": f"same grid, T={T1} steps ({dt1:.1f} s, reduced T), one thread"}}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    from paper_1410_5561_gb300 import inputs
    n = CPU_SAMPLE_N
    u0 = inputs.field_u0(args.seed, n, n, n)
    t0 = time.perf_counter()
    oracle.sweep("7pt_const", u0, 1)
    t1 = max(time.perf_counter() - t0, 1e-4)
    budget = 150.0 / max(1, args.steps + args.warmup)
    T = max(1, min(200, int(budget / t1)))
    for _ in range(args.warmup):
        oracle.sweep("7pt_const", u0, T)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.sweep("7pt_const", u0, T)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = n ** 3 * T * len(times) / tot / 1e9
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = f"7pt-const FP64 oracle, {n}^3 interior, T={T} steps per step, OpenMP over k"
    line = {
        "metric": METRIC, "value": value, "unit": "GLUP/s", "impl": "reference", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "7-point constant-coefficient Jacobi sweep (Listing 1), FP64 CPU oracle, "
                               f"bounded sample {n}^3 x T={T} of the 1024^3 T=100 workload",
                   "stencil": "7pt_const", "grid": [n, n, n], "T": T},
        "cpu_baseline": {"value": value, "unit": "GLUP/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "GLUP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------- GPU helpers

class ClockSampler:
    """nvidia-smi clock / throttle-reason samples every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.idx), "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except FileNotFoundError:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                c = [x.strip() for x in line.split(",")]
                if len(c) < 9:
                    continue
                try:
                    sm.append(float(c[1]))
                    mx.append(float(c[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, c[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if sm:
            out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                   "samples": len(sm)}
        return out


def make_grid(kind, n, fdt, cdt, seed, device):
    """A cubic Stencil with seeded inputs (see make_grid_shape)."""
    return make_grid_shape(kind, n, n, n, fdt, cdt, seed, device)


def make_grid_shape(kind, nx, ny, nz, fdt, cdt, seed, device):
    """A Stencil with seeded inputs generated on the device (the same values as the CPU
    recipe in paper_1410_5561_gb300.inputs, rounded once to the grid's precisions)."""
    import torch
    from paper_1410_5561_gb300 import inputs
    from paper_1410_5561_gb300.stencil import Stencil
    tdt = {"f32": torch.float32, "f64": torch.float64}[fdt]
    tcd = {"f32": torch.float32, "f64": torch.float64, "bf16": torch.bfloat16}[cdt or fdt]
    s = Stencil(kind, nx, ny, nz, dtype=tdt, coef_dtype=tcd, device=device)
    u0 = inputs.field_u0_torch(seed, nx, ny, nz, tdt, device)
    if kind == "7pt_const":
        s.set_coeffs(scalars=(0.4, 0.1))
    else:
        cs = inputs.coefs_torch(kind, seed, nx, ny, nz, tcd, device)
        s.set_coeffs(arrays=cs)
        del cs
    s.set_field(u0, halo=0.0)
    torch.cuda.synchronize(device)
    return s, u0


def pipeline_summary(tl):
    """Mean phase times (ms) of a traced pipeline run: sweeps, the gaps between consecutive
    sweeps, the copies in and out, and the exposed first copy in and last copy out."""
    if not tl:
        return None
    mean = lambda v: sum(v) / len(v) if v else None  # noqa: E731
    return {"sweep": mean([j["run_end"] - j["run"] for j in tl]),
            "gap_between_sweeps": mean([b["run"] - a["run_end"] for a, b in zip(tl, tl[1:])]),
            "copy_in": mean([j["h2d_end"] - j["h2d"] for j in tl]),
            "copy_out": mean([j["end"] - j["d2h"] for j in tl]),
            "first_sweep_start": tl[0]["run"], "after_last_sweep": tl[-1]["end"] - tl[-1]["run_end"],
            "total": tl[-1]["end"]}


def timed(s, T, steps, warmup, barrier=None):
    """Seconds for ``steps`` runs of T steps, CUDA events on the grid's stream."""
    import torch
    for _ in range(warmup):
        s.run(T)
    torch.cuda.synchronize(s.device)
    if barrier:
        barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s.stream)
    for _ in range(steps):
        s.run(T)
    e1.record(s.stream)
    e1.synchronize()
    torch.cuda.synchronize(s.device)
    if barrier:
        barrier()
    return e0.elapsed_time(e1) / 1e3


def traffic_from_profile(kernel_src_hash: str):
    """dram bytes per LUP recorded by the committed ncu summary, if it was taken on
    the current kernel source; else None."""
    if not os.path.exists(PROFILE_TRAFFIC):
        return None
    vals = {}
    with open(PROFILE_TRAFFIC) as f:
        for line in f:
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
    if vals.get("kernel_source_sha256") != kernel_src_hash:
        return None
    try:
        return float(vals["dram_bytes_per_lup"]), vals
    except (KeyError, ValueError):
        return None


def src_hash():
    h = hashlib.sha256()
    for name in ("blocked_impl.cuh", "blocked_launchers.h", "common.cuh", "internal.h"):
        with open(os.path.join(ROOT, "paper_1410_5561_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


class Ranks:
    """The processes of one launch (torchrun sets WORLD_SIZE, RANK, LOCAL_RANK, MASTER_*):
    one per GPU, each running its own replica of the workload. Only a barrier and the
    max-over-ranks of a time cross ranks; nothing of the sweep is exchanged."""

    def __init__(self, backend: str = "nccl"):
        import torch
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.backend = backend
        self.dist = None
        if backend == "nccl":
            if self.world > 1:
                torch.cuda.set_device(self.local)
            self.device = torch.device("cuda", self.local if self.world > 1 else torch.cuda.current_device())
        else:
            self.device = torch.device("cpu")
        if self.world > 1:
            import torch.distributed as dist
            dist.init_process_group(backend)
            self.dist = dist

    @property
    def root(self) -> bool:
        return self.rank == 0

    def barrier(self):
        if self.dist is None:
            return
        if self.backend == "nccl":
            self.dist.barrier(device_ids=[self.device.index])
        else:
            self.dist.barrier()

    def maxall(self, x: float) -> float:
        """max over ranks (a time: the job ends when its slowest rank does)"""
        if self.dist is None:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def aggregate(self, units_per_rank: float, seconds: float) -> float:
        """Whole-job throughput: the units all ranks processed over the max-over-ranks time."""
        return self.world * units_per_rank / self.maxall(seconds)

    def close(self):
        if self.dist is not None:
            self.dist.destroy_process_group()
            self.dist = None


def run_ours(args):
    import torch
    from paper_1410_5561_gb300 import model, tuner
    from paper_1410_5561_gb300.stencil import probe_fma_peak

    ranks = Ranks("nccl")
    world, rank, device = ranks.world, ranks.rank, ranks.device
    barrier, maxall = ranks.barrier, ranks.maxall

    hbm_peak, peak_src = peaks()
    fp32_peak = probe_fma_peak(torch.float32, device=device)
    fp64_peak = probe_fma_peak(torch.float64, iters=512, device=device)

    H = HEADLINE
    n, T = H["n"], H["T"]
    s, u0 = make_grid(H["kind"], n, H["fdt"], H["cdt"], args.seed, device)
    lups = float(n) ** 3 * T

    # autotune the blocked schedule on the real grid (model-guided: the six first candidates
    # are predicted, at most three timed), then reset the field
    tn, table = tuner.best_blocked(s, T, reps=1, max_candidates=6, max_timed=3, hbm_gbs=hbm_peak)
    preds = list(tuner.last_predictions)
    s.set_field(u0, halo=0.0)

    # headline: blocked
    for _ in range(args.warmup):
        s.run(T)
    clocks = ClockSampler(device.index)
    l0 = s.launches
    clocks.start()
    t_blk = timed(s, T, args.steps, 0, barrier)
    clk = clocks.stop()
    launches_timed = s.launches - l0
    t_blk = maxall(t_blk)
    value = world * lups * args.steps / t_blk / 1e9

    # plain beside it
    s.set_tuning("plain")
    ksteps = max(1, min(2, args.steps))
    t_plain = maxall(timed(s, T, ksteps, 1, barrier))
    plain_glups = lups * ksteps / t_plain / 1e9
    s.set_tuning("blocked", tn)

    # sampled error vs the FP64 oracle (rank 0, one GPU)
    err = None
    if rank == 0 and world == 1:
        import numpy as np
        import oracle
        s.set_field(u0, halo=0.0)
        s.run(T)
        got = s.current
        pts = [(1, 2, 3), (n // 2, n // 3, n // 5), (n - 1, n - 2, n // 2), (n // 7, n - 1, n - 3)]
        sc = (float(np.float32(0.4)), float(np.float32(0.1)))
        ref, g = [], []
        for (i, j, k) in pts:
            # the point depends on u0 within R*T cells; a crop with one more cell of margin,
            # clipped to the grid, keeps every value it depends on (the crop's own edges
            # are farther than R*T away unless they are the grid's Dirichlet faces)
            m = T + 1
            lo = [max(0, c - m) for c in (k, j, i)]
            hi = [min(n, c + m + 1) for c in (k, j, i)]
            crop = u0[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]].double().cpu().numpy()
            ref.append(oracle.points("7pt_const", crop, T, [(i - lo[2], j - lo[1], k - lo[0])], scalars=sc)[0])
            g.append(float(got[k, j, i]))
        ref, g = np.array(ref), np.array(g)
        err = float(np.max(np.abs(g - ref)) / max(np.max(np.abs(ref)), 1e-30))

    # end to end through the public API: host (pinned) in, host out, copies timed. One job per
    # step (H2D of u0, run(T), D2H of u_T). Pipelined: the copy engines move the next input
    # and the previous result through dense device staging arrays while a sweep runs
    # (paper_1410_5561_gb300.pipeline);
    # sequential: one grid, set_field / run / get_field one after another.
    e2e = e2e_seq = None
    if world >= 1:
        from paper_1410_5561_gb300.pipeline import Pipeline
        host_in = u0.cpu().pin_memory()
        host_out = [torch.empty_like(host_in).pin_memory() for _ in range(2)]
        nbytes = host_in.numel() * host_in.element_size()
        s.set_field(host_in, halo=0.0)
        s.run(T)
        s.get_field(host_out[0])
        barrier()
        ks = max(1, min(2, args.steps))
        t0 = time.perf_counter()
        for _ in range(ks):
            s.set_field(host_in, halo=0.0)
            s.run(T)
            s.get_field(host_out[0])
        te = maxall(time.perf_counter() - t0)
        e2e_seq = {"value": world * lups * ks / te / 1e9, "unit": "GLUP/s", "h2d_bytes_per_step": nbytes,
                   "d2h_bytes_per_step": nbytes, "steps": ks}
        pipe = Pipeline(s, T, halo=0.0, mode="auto")
        pipe.run([host_in] * 2, host_out).synchronize()  # warm-up and the mode's calibration
        kp = max(8, args.steps)  # jobs in flight amortise the first copy in and the last copy out
        passes, traces = [], []
        for _ in range(3):  # the host link is shared with the node's other work: median of 3 passes
            barrier()
            t0 = time.perf_counter()
            pipe.run([host_in] * kp, [host_out[i % 2] for i in range(kp)], trace=True).synchronize()
            passes.append(world * lups * kp / maxall(time.perf_counter() - t0) / 1e9)
            traces.append(pipeline_summary(pipe.timeline()))
        med = sorted(range(3), key=lambda i: passes[i])[1]
        e2e = {"value": passes[med], "unit": "GLUP/s", "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes, "steps": kp, "passes": passes, "timeline_ms": traces[med],
               "pipeline_mode": pipe.mode, "calibration": pipe.calibration,
               "how": "public API (pipeline.Pipeline), page-locked host buffers, one job (H2D u0, run(T), "
                      "D2H u_T) per step; staged mode: copy engines move the next input and the previous "
                      "result through dense device buffers while the sweep runs; overlap mode: the same "
                      "with the library's SM copy on the SMs the sweep leaves free; direct mode: one job at "
                      "a time with the library's copy kernel; the mode is calibrated once on this machine"}
        del host_in, host_out, pipe
        torch.cuda.empty_cache()

    # roofline of the blocked kernel (algorithmic bytes per LUP: Eq. 5 with FP32 sizes)
    bpl = model.bytes_per_lup("7pt_const", "f32", None, "blocked", tn.dw)
    achieved_gbs = bpl * lups * args.steps / t_blk / 1e9  # per GPU
    fp_time = model.FP_INSTR["7pt_const"] * 2 / fp32_peak
    hbm_time = bpl / (hbm_peak * 1e9)
    bound = "hbm" if hbm_time >= fp_time else "alu"
    prof = traffic_from_profile(src_hash())
    launches_per_step = max(1, launches_timed // max(1, args.steps))
    traffic = None
    if prof is not None:
        traffic = prof[0] * lups / launches_per_step
    if bound == "hbm":
        roof = {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved_gbs / hbm_peak, "traffic": traffic,
                "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)",
                "algorithmic_bytes_per_lup": bpl}
    else:
        ach = model.FLOPS["7pt_const"] * lups * args.steps / t_blk / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": fp32_peak / 1e12, "unit": "TFLOP/s",
                "frac": ach / (fp32_peak / 1e12), "traffic": traffic}

    line = {
        "metric": METRIC, "value": value, "unit": "GLUP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_blk / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"7-point constant-coefficient Jacobi sweep (Listing 1, c0=0.4, c1=0.1), "
                               f"{n}^3 interior FP32, zero Dirichlet halo, T={T} per step, temporally blocked "
                               f"(D_w={tn.dw}, N_F={tn.nf}, warps={tn.warps}, xtile={tn.xtile})",
                   "stencil": "7pt_const", "grid": [n, n, n], "T": T, "scheme": "blocked",
                   "tuning": {"dw": tn.dw, "nf": tn.nf, "warps": tn.warps, "xtile": tn.xtile},
                   "l2": f"inputs larger than L2 ({(n + 2) ** 3 * 4 / 1e9:.1f} GB per array)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "plain": {"value": plain_glups * world, "unit": "GLUP/s", "ms_per_step": 1e3 * t_plain / ksteps,
                  "algorithmic_bytes_per_lup": model.bytes_per_lup("7pt_const", "f32", None, "plain")},
        "blocked_over_plain": value / (plain_glups * world),
        "roofline": roof,
        "gpu_launches": int(launches_timed),
        "clocks": clk,
        "e2e": e2e,
        "e2e_sequential": e2e_seq,
        "err_vs_oracle_sampled": err,
        "fma_peaks_tflops": {"f32": fp32_peak / 1e12, "f64": fp64_peak / 1e12},
        "autotune": [{"tuning": f"dw={t.dw} nf={t.nf} warps={t.warps} xtile={t.xtile}",
                      "predicted_s": p, "measured_s": m} for t, p, m in preds],
    }
    del s, u0
    torch.cuda.empty_cache()

    if rank == 0 and world == 1:
        line["cpu_baseline"] = cpu_oracle_sample()
        if not args.no_extras:
            for key, fn in (("per_stencil", lambda: per_stencil(device, args.seed, hbm_peak, fp32_peak, fp64_peak)),
                            ("dw_sweep", lambda: dw_sweep(device, args.seed)),
                            ("energy", lambda: energy_table(device, args.seed)),
                            ("batched", lambda: batched(device, args.seed)),
                            ("adjoint", lambda: adjoint_timing(device, args.seed))):
                try:
                    line[key] = fn()
                except Exception as exc:  # report, never hide the headline
                    line[key + "_error"] = repr(exc)
                torch.cuda.empty_cache()
    if rank == 0:
        print(json.dumps(line), flush=True)
    ranks.barrier()
    ranks.close()
    return 0


PER_STENCIL = [
    ("7pt_const", 512, "f32", None, 100),
    ("7pt_const", 512, "f64", None, 100),
    ("7pt_var", 384, "f32", None, 50),
    ("7pt_var", 384, "f32", "bf16", 50),
    ("7pt_var", 384, "f64", None, 50),
    ("25pt_var", 256, "f32", None, 40),
    ("25pt_var", 256, "f32", "bf16", 40),
    ("25pt_var", 256, "f64", None, 40),
]


def sampled_oracle_error(s, kind, n, fdt, cdt, T, seed):
    """Error of the grid's current field (u_T from the seeded u0) against the FP64 oracle
    at a few sampled points: each point's u_T is evaluated by ``oracle.points`` on a crop of
    the host-drawn inputs reaching R*T + R cells past it (clipped at the grid's Dirichlet
    faces), in the precisions the device stores. Returns the step-normalised L2 over the
    points, ||g - ref|| / (||ref|| T), and the largest relative error; for BF16 coefficients
    also the "storage error": the same against the oracle on the unrounded FP64
    coefficients (stated, not gated)."""
    import numpy as np
    import oracle
    from paper_1410_5561_gb300 import inputs
    R = 4 if kind == "25pt_var" else 1
    m = R * T + R
    pts = [(0, 0, 0), (n - 1, n - 1, n - 1), (n - 1, 0, n // 2)]
    if 2 * m + 1 < n:
        pts.append((n // 2, n // 3, n // 5))
    sc = (0.4, 0.1)
    if fdt == "f32":
        sc = (float(np.float32(0.4)), float(np.float32(0.1)))
    got = s.current
    g, ref, ref_unrounded = [], [], []
    for (i, j, k) in pts:
        lo = tuple(max(0, c - m) for c in (k, j, i))
        hi = tuple(min(n, c + m + 1) for c in (k, j, i))
        u0 = inputs.field_u0_box(seed, n, n, n, lo, hi)
        if fdt == "f32":
            u0 = inputs.round_f32(u0)
        loc = [(i - lo[2], j - lo[1], k - lo[0])]
        coefs = c64 = None
        if kind != "7pt_const":
            c64 = inputs.coefs_box(kind, seed, n, n, n, lo, hi)
            st = cdt or fdt
            coefs = inputs.bf16_to_f64(inputs.bf16_bits(c64)) if st == "bf16" else (
                inputs.round_f32(c64) if st == "f32" else c64)
        ref.append(oracle.points(kind, u0, T, loc, coefs=coefs, scalars=sc)[0])
        if cdt == "bf16":
            ref_unrounded.append(oracle.points(kind, u0, T, loc, coefs=c64, scalars=sc)[0])
        g.append(float(got[k, j, i]))
    g, ref = np.array(g), np.array(ref)

    def errs(r):
        den = np.linalg.norm(r) * max(T, 1)
        return {"step_normalised_l2": float(np.linalg.norm(g - r) / den) if den > 0 else None,
                "max_rel": float(np.max(np.abs(g - r)) / max(float(np.max(np.abs(r))), 1e-300))}

    out = {"points": len(pts), **errs(ref),
           "gate": 1e-5 if fdt == "f32" else 1e-12}
    out["within_gate"] = out["step_normalised_l2"] is not None and out["step_normalised_l2"] <= out["gate"]
    if cdt == "bf16":
        out["storage_error_vs_unrounded_coefficients"] = errs(np.array(ref_unrounded))
    return out


def per_stencil(device, seed, hbm_peak, fp32_peak, fp64_peak):
    """Plain vs tuned blocked sweep (diamonds in shared memory, model-guided tuner) vs the
    wavefront schedule through L2, for every stencil and precision: GLUP/s, the model bytes per
    LUP, the roofline (the slower of the HBM bound at the model bytes and the FP-pipe bound)
    and the achieved fraction of it, and each result's error against the FP64 oracle on
    sampled points."""
    import torch
    from paper_1410_5561_gb300 import model, tuner
    from paper_1410_5561_gb300.stencil import Tuning
    rows = []
    for kind, n, fdt, cdt, T in PER_STENCIL:
        s, u0 = make_grid(kind, n, fdt, cdt, seed, device)
        lups = float(n) ** 3 * T
        bp = model.bytes_per_lup(kind, fdt, cdt, "plain")
        peak_fp = fp64_peak if fdt == "f64" else fp32_peak
        alu_glups = peak_fp / (model.FP_INSTR[kind] * 2) / 1e9
        s.set_tuning("plain")
        tp = timed(s, T, 2, 1) / 2
        s.set_field(u0, halo=0.0)
        s.run(T)
        err_plain = sampled_oracle_error(s, kind, n, fdt, cdt, T, seed)
        try:
            tn, _ = tuner.best_blocked(s, T, reps=1, max_candidates=6, max_timed=3, hbm_gbs=hbm_peak)
            tb = timed(s, T, 2, 1) / 2
            tun = {"dw": tn.dw, "nf": tn.nf, "warps": tn.warps, "xtile": tn.xtile}
            bb = model.bytes_per_lup(kind, fdt, cdt, "blocked", tn.dw)
            s.set_field(u0, halo=0.0)
            s.run(T)
            err_blk = sampled_oracle_error(s, kind, n, fdt, cdt, T, seed)
        except RuntimeError:
            tb, tun, bb, err_blk = None, None, None, None
        # wavefront through L2: the better of two tunings measured best on GB300 (25-point: 2 levels
        # with 16-plane chunks and loads copied ahead, or 3 levels; 7-point: 2 or 6 levels)
        R = 4 if kind == "25pt_var" else 1
        tw, tun_w, err_w = None, None, None
        wcands = (Tuning(16, 16, 8, 2), Tuning(24, 8, 4, 0)) if R == 4 else (Tuning(4, 4, 16, 0), Tuning(12, 8, 4, 0))
        for wt in wcands:
            try:
                s.set_tuning("wavefront", wt)
            except RuntimeError:
                continue
            t_ = timed(s, T, 2, 1) / 2
            if tw is None or t_ < tw:
                tw, tun_w = t_, wt
        if tun_w is not None:
            s.set_tuning("wavefront", tun_w)
            s.set_field(u0, halo=0.0)
            s.run(T)
            err_w = sampled_oracle_error(s, kind, n, fdt, cdt, T, seed)
        roof_p = min(hbm_peak / bp, alu_glups)
        roof_b = min(hbm_peak / bb, alu_glups) if bb else None
        gp = lups / tp / 1e9
        gb = lups / tb / 1e9 if tb else None
        rows.append({
            "stencil": kind, "grid": n, "field": fdt, "coef": cdt or fdt, "T": T,
            "plain_glups": gp,
            "blocked_glups": gb,
            "blocked_over_plain": gb / gp if gb else None,
            "blocked_tuning": tun,
            "wavefront_glups": lups / tw / 1e9 if tw else None,
            "wavefront_tuning": {"dw": tun_w.dw, "zchunk": tun_w.nf, "rows": tun_w.warps,
                                 "prefetch": tun_w.xtile} if tun_w else None,
            "autotune": [{"tuning": f"dw={t.dw} nf={t.nf} warps={t.warps} xtile={t.xtile}", "predicted_s": p_,
                          "measured_s": m_} for t, p_, m_ in tuner.last_predictions] if tun else None,
            "model_bytes_per_lup": {"plain": bp, "blocked": bb},
            "roofline_glups": {"hbm_plain": hbm_peak / bp, "hbm_blocked": hbm_peak / bb if bb else None,
                               "alu": alu_glups},
            "roofline_frac": {"plain": gp / roof_p, "blocked": gb / roof_b if gb else None,
                              "plain_bound": "hbm" if hbm_peak / bp <= alu_glups else "alu",
                              "blocked_bound": ("hbm" if hbm_peak / bb <= alu_glups else "alu") if bb else None},
            "err_vs_oracle": {"plain": err_plain, "blocked": err_blk, "wavefront": err_w},
        })
        del s, u0
        torch.cuda.empty_cache()
    return rows


DW_SWEEP = ("7pt_const", 512, "f32", None, 100)


def dw_sweep(device, seed, per_dw: int = 2):
    """Blocked GLUP/s at each feasible diamond width D_w (7-point constant FP32 512^3, T=100):
    the best of the first ``per_dw`` tuner candidates with that D_w, beside the Eq. 5 model code
    balance 2R(4 s_f)/D_w and the plain sweep."""
    import torch
    from paper_1410_5561_gb300 import model, tuner
    kind, n, fdt, cdt, T = DW_SWEEP
    s, _ = make_grid(kind, n, fdt, cdt, seed, device)
    lups = float(n) ** 3 * T
    s.set_tuning("plain")
    out = {"stencil": kind, "grid": n, "field": fdt, "T": T,
           "plain_glups": lups / (timed(s, T, 2, 1) / 2) / 1e9,
           "plain_model_bytes_per_lup": model.bytes_per_lup(kind, fdt, cdt, "plain"), "rows": []}
    cands = tuner.candidates(s)
    for dw in sorted({t.dw for t in cands}):
        best = None
        for tn in [t for t in cands if t.dw == dw][:per_dw]:
            try:
                s.set_tuning("blocked", tn)
            except Exception:
                continue
            sec = timed(s, T, 2, 1) / 2
            if best is None or sec < best[0]:
                best = (sec, tn)
        if best is None:
            continue
        sec, tn = best
        out["rows"].append({"dw": dw, "tuning": {"dw": tn.dw, "nf": tn.nf, "warps": tn.warps, "xtile": tn.xtile},
                            "glups": lups / sec / 1e9,
                            "model_bytes_per_lup": model.bytes_per_lup(kind, fdt, cdt, "blocked", dw)})
    del s
    torch.cuda.empty_cache()
    return out


ENERGY_CASES = [
    ("7pt_const", 1024, "f32", None, 100),
    ("7pt_const", 512, "f32", None, 100),
    ("7pt_const", 512, "f64", None, 100),
    ("7pt_var", 384, "f32", None, 50),
    ("7pt_var", 384, "f32", "bf16", 50),
]
# the wavefront tuning measured best per stencil and precision on GB300 (D_w, chunk planes, rows,
# copies ahead): six levels with 8-plane chunks and 4-row tiles, or two levels with 4-plane
# chunks and 16-row tiles for the 7-point variable FP32 sweep
ENERGY_WAVE = {("7pt_const", "f32"): (12, 8, 4, 0), ("7pt_const", "f64"): (12, 8, 4, 0),
               ("7pt_var", "f32"): (4, 4, 16, 0), ("7pt_var", "bf16"): (12, 8, 4, 0)}


def energy_table(device, seed, min_seconds: float = 2.0):
    """Board energy per LUP, plain vs blocked vs wavefront (the paper's Section IV question on the
    GPU): NVML's total-energy counter read around at least ``min_seconds`` of back-to-back runs
    of each schedule; the idle board power, read first over one second with nothing of ours
    running, gives the dynamic share. Blocked runs use the tuning the benchmark's autotuner
    chose for the grid (cached), else the tuner's first candidate."""
    import torch
    from paper_1410_5561_gb300 import energy, model, tuner
    from paper_1410_5561_gb300.stencil import Tuning
    meter = energy.EnergyMeter(energy.device_uuid(device))
    if not meter.available:
        return {"unavailable": meter.reason}
    torch.cuda.synchronize(device)
    idle = energy.idle_watts(meter, 1.0)
    rows = []
    sync = lambda: torch.cuda.synchronize(device)  # noqa: E731
    for kind, n, fdt, cdt, T in ENERGY_CASES:
        s, _ = make_grid(kind, n, fdt, cdt, seed, device)
        lups = float(n) ** 3 * T
        row = {"stencil": kind, "grid": n, "field": fdt, "coef": cdt or fdt, "T": T}
        for scheme in ("plain", "blocked", "wavefront"):
            if scheme == "plain":
                s.set_tuning("plain")
                bpl = model.bytes_per_lup(kind, fdt, cdt, "plain")
                tun = None
            elif scheme == "blocked":
                tn, _ = tuner.best_blocked(s, T, reps=1, max_candidates=6, max_timed=3)
                bpl = model.bytes_per_lup(kind, fdt, cdt, "blocked", tn.dw)
                tun = {"dw": tn.dw, "nf": tn.nf, "warps": tn.warps, "xtile": tn.xtile}
            else:
                wt = Tuning(*ENERGY_WAVE[(kind, cdt or fdt)])
                s.set_tuning("wavefront", wt)
                h = wt.dw // 2  # R = 1
                sf = 8 if fdt == "f64" else 4
                bpl = (model.bytes_per_lup(kind, fdt, cdt, "plain") + (h - 1) * sf) / h
                tun = {"dw": wt.dw, "zchunk": wt.nf, "rows": wt.warps}
            s.run(T)
            r = energy.measure(meter, lambda: s.run(T), lups, min_seconds=min_seconds, sync=sync)
            if r is None:
                row[scheme] = None
                continue
            dyn = None if idle is None else max(r["watts"] - idle, 0.0) * r["seconds"] / r["lups"] * 1e12
            row[scheme] = {"pj_per_lup": r["pj_per_lup"], "dynamic_pj_per_lup": dyn, "watts": r["watts"],
                           "glups": r["lups"] / r["seconds"] / 1e9, "model_bytes_per_lup": bpl,
                           "tuning": tun}
        if row.get("plain") and row.get("blocked"):
            row["blocked_over_plain_energy"] = row["blocked"]["pj_per_lup"] / row["plain"]["pj_per_lup"]
        if row.get("plain") and row.get("wavefront"):
            row["wavefront_over_plain_energy"] = row["wavefront"]["pj_per_lup"] / row["plain"]["pj_per_lup"]
        rows.append(row)
        del s
        torch.cuda.empty_cache()
    meter.close()
    return {"idle_watts": idle, "counter": "nvmlDeviceGetTotalEnergyConsumption (whole board)",
            "rows": rows}


def batched(device, seed):
    """64 independent 7-point variable FP32 grids (sides 32..192, T 10..200): one persistent
    CUDA-graph launch (autotuned diamond width, frontlines and warps) vs one launch per grid
    (plain sweeps, T launches per grid; and the blocked sweep with each grid's first tuner
    candidate)."""
    import torch
    from paper_1410_5561_gb300 import inputs, tuner
    from paper_1410_5561_gb300.batch import Batch
    shapes = inputs.batch_shapes(seed)
    grids = []
    for q, (nx, ny, nz, T) in enumerate(shapes):
        s, _ = make_grid_shape("7pt_var", nx, ny, nz, "f32", None, seed + q, device)
        grids.append(s)
    Ts = [sh[3] for sh in shapes]
    lups = sum(nx * ny * nz * T for (nx, ny, nz, T) in shapes)
    tn, table = tuner.tune_batch(grids, Ts)
    b = Batch(grids, Ts, tn)
    b.launch()
    torch.cuda.synchronize(device)
    g = b.capture()
    g.replay()
    torch.cuda.synchronize(device)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    reps = 3
    e0.record()
    for _ in range(reps):
        g.replay()
    e1.record()
    e1.synchronize()
    t_batch = e0.elapsed_time(e1) / 1e3 / reps
    b.sync_parity()
    status = b.status()
    stream = torch.cuda.current_stream(device)

    def per_grid(reps_):
        for s, T in zip(grids, Ts):
            s.run(T)
        torch.cuda.synchronize(device)
        e0.record(stream)
        for _ in range(reps_):
            for s, T in zip(grids, Ts):
                s.run(T)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / 1e3 / reps_

    for s in grids:  # one launch per grid and step
        s.set_tuning("plain")
    t_plain = per_grid(2)
    for s in grids:  # one persistent blocked launch per grid
        s.set_tuning("blocked", tuner.candidates(s)[0])
    t_blk = per_grid(1)
    return {"grids": len(shapes), "lups": lups, "tuning": {"dw": tn.dw, "nf": tn.nf, "warps": tn.warps},
            "graph_launch_glups": lups / t_batch / 1e9, "graph_ms": 1e3 * t_batch,
            "per_grid_plain_glups": lups / t_plain / 1e9, "per_grid_plain_ms": 1e3 * t_plain,
            "per_grid_blocked_glups": lups / t_blk / 1e9, "per_grid_blocked_ms": 1e3 * t_blk,
            "autotune": [{"tuning": f"dw={c.dw} nf={c.nf} warps={c.warps}", "ms": 1e3 * t} for c, t in table],
            "tiles": b.items, "status": status}


def adjoint_timing(device, seed):
    """25-point variable FP32 256^3, T=40: forward with sqrt(T) checkpoints + adjoint, with the
    grid on the plain sweep and on the wavefront schedule (whose backward pass recomputes the
    states and runs the transposed recursion as temporally blocked passes)."""
    import torch
    from paper_1410_5561_gb300 import inputs
    from paper_1410_5561_gb300.autograd import sweep
    from paper_1410_5561_gb300.stencil import Tuning
    n, T = 256, 40
    s, u0 = make_grid("25pt_var", n, "f32", None, seed, device)
    coefs = torch.stack([s.interior_of(c).clone() for c in s.coefs])
    target = torch.empty_like(u0)
    inputs.fill_uniform_torch(target, seed, inputs.STREAM_TARGET, -1.0, 1.0)

    def once():
        u = u0.clone().requires_grad_(True)
        c = coefs.clone().requires_grad_(True)
        uT = sweep(u, c, s, T)
        loss = 0.5 * ((uT - target) ** 2).sum()
        loss.backward()
        return loss

    out = {"stencil": "25pt_var", "grid": n, "T": T, "checkpoints": "ceil(sqrt(T)) = 7"}
    for label, scheme, tn in (("plain", "plain", None), ("wavefront", "wavefront", Tuning(16, 16, 8, 2))):
        s.set_tuning(scheme, tn)
        once()
        torch.cuda.synchronize(device)
        t0 = time.perf_counter()
        once()
        torch.cuda.synchronize(device)
        tt = time.perf_counter() - t0
        s.set_field(u0, halo=0.0)
        torch.cuda.synchronize(device)
        t0 = time.perf_counter()
        s.run(T)
        s.sync()
        tf = time.perf_counter() - t0
        out[label] = {"forward_plus_adjoint_s": tt, "forward_s": tf, "ratio": tt / tf,
                      "forward_plus_adjoint_glups": n ** 3 * T / tt / 1e9}
    # the plain-grid figures stay at the top level (the earlier report's fields)
    out.update(out["plain"])
    return out


def main():
    args = parse()
    if args.case:
        return run_case(args.case, args.seed)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
