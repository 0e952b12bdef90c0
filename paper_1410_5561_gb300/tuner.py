"""Model-guided autotuner for the blocked schedules.

Section II-A: the diamond width and the number of frontlines are chosen by
auto-tuning, with the search space pruned to blocks that fit the cache and
that give enough concurrency; Section VI asks for the tuning to be guided by
the models of Section III. Here:

* Capacity pruning (the GPU analog of Eq. 3): the "cache" is one CTA's shared
  memory (the library reports the exact ring footprint of a tuning, and tunings
  that do not fit the opt-in limit are dropped) and the register file (tunings
  that give a warp more than one item spill).
* Prediction before timing (Eq. 5): every candidate's time is predicted from its
  code balance at the streaming rate the schedule reaches, its useful share of
  computed columns, its frontlines and its register pressure (``predict``); the
  absolute scale is fixed by the first timed candidate, candidates predicted
  more than 1.5x slower than the best are dropped, and only the best few
  predictions are timed on the device with CUDA events (``autotune``).

Results are cached per (stencil, dtypes, shape, T).
"""
from __future__ import annotations

import math

import torch

from . import model
from .stencil import RADIUS, Stencil, Tuning

_CACHE: dict = {}
_KIND_NAME = {0: "7pt_const", 1: "7pt_var", 2: "25pt_var"}
_DT_NAME = {torch.float32: "f32", torch.float64: "f64", torch.bfloat16: "bf16"}


def one_warp_xtile(dw: int, r: int, v: int) -> int:
    """Widest x tile whose bottom-level row (tile plus trapezoid overlap) fits 32 vectors."""
    lt = dw // r - 1
    ov = math.ceil(r * (lt - 1) / v) if lt > 1 else 0
    return max(v, (32 - 2 * ov) * v)


def items_per_warp(t: Tuning, r: int, v: int) -> int:
    """Work items per warp of a blocked tuning, as the library splits a full diamond: D_w^2/(2R)
    row updates per level set, grouped in items of 2 rows (R = 1) or 1 row, each 32-vector
    chunk of the x-tile row (trapezoid overlap included) its own item."""
    lt = t.dw // r - 1
    ov = -(-r * (lt - 1) // v) if lt > 1 else 0
    nch = -(-(t.xtile // v + 2 * ov) // 32)
    items = (t.dw * t.dw // (2 * r)) // (2 if r == 1 else 1) * nch
    return -(-items // t.warps)


def x_tiles(nx: int, t: Tuning, r: int, v: int) -> int:
    """x tiles per row as the library cuts them: one if the row fits, else (R = 1) two edge
    tiles of xtile plus the one-sided trapezoid overlap around interior tiles of xtile, or
    (R = 4) equal tiles."""
    if nx <= t.xtile:
        return 1
    if r != 1:
        return -(-nx // t.xtile)
    lt = t.dw // r - 1
    ov = -(-r * (lt - 1) // v) if lt > 1 else 0
    xe = t.xtile + ov * v
    return 2 if nx <= 2 * xe else 2 + -(-(nx - 2 * xe) // t.xtile)


def candidates(s: Stencil, nfs=(1, 2), warps=(8, 16), max_dw=None) -> list[Tuning]:
    """Tunings that fit shared memory, best model code balance first."""
    r = RADIUS[s.kind]
    eb = torch.empty((), dtype=s.dtype).element_size()
    v = 16 // eb
    optin = torch.cuda.get_device_properties(s.device).shared_memory_per_block_optin
    max_dw = max_dw or 16 * r
    out = []
    for dw in range(2 * r, max_dw + 1, 2 * r):
        xt = one_warp_xtile(dw, r, v)
        xts = {xt, max(v, (xt // 2) // v * v)}
        ntile = -(-s.nx // xt)  # the same number of x tiles, evenly wide
        xts.add(max(v, -(-(-(-s.nx // ntile)) // v) * v))
        if r == 1 and s.nx > xt:  # the narrowest tiles that keep the uneven split's tile count
            nt = x_tiles(s.nx, Tuning(dw, 1, 16, xt), r, v)
            lt = dw // r - 1
            ov = -(-r * (lt - 1) // v) if lt > 1 else 0
            if nt > 2:
                xts.add(max(v, -(-(-(-(s.nx - 2 * ov * v) // nt)) // v) * v))
        for nclu in (2, 4, 8):  # x tiles splitting the row into portable cluster sizes
            xts.add(max(v, ((s.nx + nclu - 1) // nclu + v - 1) // v * v))
        for xtile in sorted(xts, reverse=True):
            for nf in nfs:
                for w in warps:
                    t = Tuning(dw, nf, w, xtile)
                    need = s.blocked_smem_bytes(t)
                    if 0 < need <= optin:
                        out.append(t)
    kind = _KIND_NAME[s.kind]
    fdt = _DT_NAME[s.dtype]
    cdt = _DT_NAME[s.coef_dtype]
    # measured order of merit on GB300: one item per warp, D_w near 8R (the largest width whose
    # rings leave room for 16 warps), 16 warps, the cheaper frontline count, then the share of computed x
    # columns that are useful (each x tile computes whole 32-vector chunks of its row, overlap
    # included); the model code balance (Eq. 5) breaks ties
    def chunks(t):
        lt = t.dw // r - 1
        ov = -(-r * (lt - 1) // v) if lt > 1 else 0
        return -(-(t.xtile // v + 2 * ov) // 32)

    def useful(t):
        return s.nx / (x_tiles(s.nx, t, r, v) * chunks(t) * 32 * v)

    def score(t):
        # register capacity first (the GPU analog of the paper's cache-size pruning with
        # Eq. 3): with R = 1 each warp keeps its items' z-windows in registers, and tunings
        # that give a warp more than one item spill under the 128-register cap of 512-thread
        # CTAs (measured 2.4-11x slower at 512^3; they stay as a last resort)
        return (r == 1 and items_per_warp(t, r, v) > 1, abs(t.dw - 8 * r), -t.warps, nf_cost(kind, fdt, cdt, t.nf),
                -round(useful(t), 3), chunks(t), -t.xtile, model.bytes_per_lup(kind, fdt, cdt, "blocked", t.dw))
    out.sort(key=score)
    return out


# Streaming rates (fraction of the HBM copy bandwidth) and per-schedule factors the model
# uses, measured on GB300 (2070 MHz): the plain sweep streams at 0.83 of the copy rate, the
# one-CTA-per-SM diamond kernel at 0.42 of it for every diamond width whose items fit one per
# warp (D_w = 4, 6, 8 at 512^3: 2.6-2.9 TB/s), and a warp with 2 or 4 items spills (3x and 7x
# slower); one frontline costs 23 % more per update than two (one CTA barrier per plane), except
# for the 7-point variable stencil with FP32 coefficients, whose two frontlines wait on their
# coefficient loads one after the other: there one frontline is 6 % cheaper (215 vs 201 GLUP/s
# at 384^3, T = 50).
PLAIN_STREAM = 0.83
BLOCKED_STREAM = 0.42
SPILL = {1: 1.0, 2: 3.0, 4: 7.0}
NF_COST = {1: 1.23, 2: 1.0}
NF_COST_7PT_VAR_F32 = {1: 0.94, 2: 1.0}


def nf_cost(kind: str, fdt: str, cdt: str, nf: int) -> float:
    """Measured cost factor of N_F frontlines per update (relative to two)."""
    table = NF_COST_7PT_VAR_F32 if (kind == "7pt_var" and fdt == "f32" and cdt == "f32") else NF_COST
    return table.get(nf, 1.0)
HBM_GBS = 6780.0  # GB300 copy bandwidth, used when the caller gives none
PRUNE = 1.5


def predict(s: Stencil, T: int, scheme: str, t: Tuning | None = None, hbm_gbs: float = HBM_GBS,
            fp_peak: float | None = None) -> float:
    """Predicted seconds (up to a common scale) of ``T`` steps of grid ``s`` under a schedule.

    plain: the slower of the algorithmic bytes (2 s_f + n_c s_c per LUP) at the plain sweep's
    streaming rate and the floating-point instructions at ``fp_peak`` FLOP/s (FP64 sweeps are
    bound by GB300's FP64 units); blocked: Eq. 5's code balance at the diamond kernel's
    streaming rate, divided by the useful share of computed x columns, times the register
    (items per warp) and frontline factors; wavefront: the plain sweep's rate, since every time
    level keeps pace with level 0, which has h^-1 of the CTAs (measured: the schedule cuts HBM
    bytes but not time)."""
    kind = _KIND_NAME[s.kind]
    fdt = _DT_NAME[s.dtype]
    cdt = _DT_NAME[s.coef_dtype]
    r = RADIUS[s.kind]
    v = 16 // torch.empty((), dtype=s.dtype).element_size()
    lups = float(s.nx) * s.ny * s.nz * T
    alu = 0.0
    if fp_peak:
        alu = lups * model.FP_INSTR[kind] * 2 / fp_peak
    if scheme in ("plain", "wavefront"):
        b = model.bytes_per_lup(kind, fdt, cdt, "plain")
        return max(lups * b / (PLAIN_STREAM * hbm_gbs * 1e9), alu)
    b = model.bytes_per_lup(kind, fdt, cdt, "blocked", t.dw)
    lt = t.dw // r - 1
    ov = -(-r * (lt - 1) // v) if lt > 1 else 0
    nch = -(-(t.xtile // v + 2 * ov) // 32)
    useful = s.nx / (x_tiles(s.nx, t, r, v) * nch * 32 * v)
    k = items_per_warp(t, r, v)
    k = 1 if k <= 1 else (2 if k <= 2 else 4)
    mem = lups * b / (BLOCKED_STREAM * hbm_gbs * 1e9)
    return max(mem, alu) / min(1.0, useful) * SPILL[k] * nf_cost(kind, fdt, cdt, t.nf)


def _time_run(s: Stencil, T: int, reps: int) -> float:
    s.run(T)
    torch.cuda.synchronize(s.device)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    best = float("inf")
    for _ in range(reps):
        e0.record(s.stream)
        s.run(T)
        e1.record(s.stream)
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    return best


def autotune(s: Stencil, T: int, reps: int = 2, max_candidates: int = 10, include_plain: bool = True,
             use_cache: bool = True, max_timed: int = 3, hbm_gbs: float = HBM_GBS, fp_peak: float | None = None,
             schemes=("plain", "blocked")):
    """Pick the fastest schedule for ``T`` steps of grid ``s``, guided by ``predict``.

    Candidates: the plain sweep, the first ``max_candidates`` blocked tunings of
    ``candidates`` (capacity-pruned) and, if asked, the library's default wavefront tuning.
    Each is predicted; the best prediction is timed first and fixes the model's absolute
    scale; candidates predicted more than 1.5x slower than the best are dropped; at most
    ``max_timed`` are timed, in predicted order. Returns (scheme, tuning or None, table), the
    table listing (label, predicted seconds, measured seconds or None) for every candidate.
    The grid's field advances while timing; callers reset it afterwards.
    """
    key = (s.kind, s.dtype, s.coef_dtype, s.nx, s.ny, s.nz, T, tuple(schemes), max_timed)
    if use_cache and key in _CACHE:
        scheme, tn, table = _CACHE[key]
        s.set_tuning(scheme, tn)
        return scheme, tn, table
    cands = []
    if include_plain and "plain" in schemes:
        cands.append(("plain", None))
    if "blocked" in schemes:
        cands += [("blocked", t) for t in candidates(s)[:max_candidates]]
    if "wavefront" in schemes:
        cands.append(("wavefront", None))
    pred = [(predict(s, T, sc, t, hbm_gbs, fp_peak), sc, t) for sc, t in cands]
    pred.sort(key=lambda x: x[0])
    table, best, scale = [], (float("inf"), "plain", None), None
    timed_n = 0
    for p, sc, t in pred:
        label = sc if t is None else f"{sc} dw={t.dw} nf={t.nf} warps={t.warps} xtile={t.xtile}"
        keep = timed_n < max_timed and (scale is None or p <= PRUNE * pred[0][0])
        meas = None
        if keep:
            try:
                s.set_tuning(sc, t)
            except Exception:
                keep = False
        if keep:
            meas = _time_run(s, T, reps)
            timed_n += 1
            if scale is None:
                scale = meas / p
            if meas < best[0]:
                best = (meas, sc, t)
        table.append((label, p * (scale or 1.0), meas))
    _, scheme, tn = best
    s.set_tuning(scheme, tn)
    _CACHE[key] = (scheme, tn, table)
    return scheme, tn, table


def best_blocked(s: Stencil, T: int, reps: int = 2, max_candidates: int = 10, max_timed: int | None = None,
                 hbm_gbs: float = HBM_GBS):
    """The fastest blocked tuning only (for reporting blocked against plain). With
    ``max_timed`` the candidates are ranked by ``predict``, those predicted more than 1.5x
    slower than the best are dropped and at most ``max_timed`` are timed; otherwise the first
    ``max_candidates`` of ``candidates`` are all timed. Returns (tuning, table of (tuning,
    seconds)); ``last_predictions`` keeps (tuning, predicted seconds, measured or None)."""
    global last_predictions
    key = ("blocked", max_timed) + (s.kind, s.dtype, s.coef_dtype, s.nx, s.ny, s.nz, T)
    if key in _CACHE:
        tn, table = _CACHE[key]
        s.set_tuning("blocked", tn)
        return tn, table
    cands = candidates(s)[:max_candidates]
    preds = {c: predict(s, T, "blocked", c, hbm_gbs) for c in cands}
    if max_timed is not None:
        p0 = min(preds.values()) if preds else 0.0
        order = sorted(cands, key=lambda c: preds[c])
        cands = [c for c in order if preds[c] <= PRUNE * p0][:max_timed]
    table = []
    best = (float("inf"), None)
    for tn in cands:
        try:
            s.set_tuning("blocked", tn)
        except Exception:
            continue
        t = _time_run(s, T, reps)
        table.append((tn, t))
        if t < best[0]:
            best = (t, tn)
    if best[1] is None:
        raise RuntimeError("no feasible blocked tuning")
    meas = dict(table)
    scale = (table[0][1] / preds[table[0][0]]) if table else 1.0
    last_predictions = [(c, preds[c] * scale, meas.get(c)) for c in sorted(preds, key=lambda c: preds[c])]
    s.set_tuning("blocked", best[1])
    _CACHE[key] = (best[1], table)
    return best[1], table


last_predictions: list = []


BATCH_CANDIDATES = [Tuning(dw, nf, w, 0) for dw in (4, 6, 8) for nf in (1, 2) for w in (8, 16)] + \
    [Tuning(4, 1, 4, 0), Tuning(2, 1, 4, 0), Tuning(2, 1, 8, 0)]


def tune_batch(grids: list[Stencil], T: list[int], candidates=None, reps: int = 2):
    """Fastest batch tuning (x tiles are whole rows in a batch) for advancing ``grids`` by ``T``.

    Each feasible candidate is built as a Batch, captured in a CUDA graph and replayed; the
    grids advance while timing (callers reset them). Returns (tuning, table of (tuning, seconds)).
    Section II-A: the paper tunes the diamond width and thread-group size per stencil and machine;
    here the small, uneven grids of a batch favour narrower diamonds than one large grid.
    """
    from .batch import Batch
    table = []
    best = (float("inf"), None)
    for tn in (candidates or BATCH_CANDIDATES):
        try:
            b = Batch(grids, T, tn)
        except Exception:
            continue
        g = b.capture()
        g.replay()
        torch.cuda.synchronize(grids[0].device)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            g.replay()
        e1.record()
        e1.synchronize()
        t = e0.elapsed_time(e1) / 1e3 / reps
        b.sync_parity()
        del g
        b.close()
        table.append((tn, t))
        if t < best[0]:
            best = (t, tn)
    if best[1] is None:
        raise RuntimeError("no feasible batch tuning")
    return best[1], table
