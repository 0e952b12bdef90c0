"""Oracle parity at the full workload sizes, in the launch configurations that are timed.

The FP64 oracle cannot sweep a 1024^3 grid, so each case samples output points
(corners, edges, faces, points beside x-tile seams, seeded interior points) and
evaluates u_T at each one with ``oracle.points`` on a crop of the inputs. The crop
reaches R*T + R cells beyond the sampled points (clipped at the grid's faces, which
are the real Dirichlet faces), so every value a point depends on is inside it and the
crop's own cut faces are out of reach. The crop is drawn on the host by the input
recipe itself; the device grid is drawn by the torch version of the same recipe, and
the test checks that the two agree bit for bit at the crop before comparing outputs.

Each case runs the plain sweep, the blocked schedule with every tuning the benchmark's
autotuner may pick (the first candidates in its order), the wavefront schedule with the
tunings the benchmark times, and STENCIL_AUTO, all on the same inputs; each result is checked against the oracle within the element-wise bound
of ``Problem.elementwise_tol`` (the weights of a row sum to at most 1, so each step
adds at most 2 x (roundings per update) x eps x max|u|).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1410_5561_gb300 import inputs, tuner
from paper_1410_5561_gb300.stencil import RADIUS, Stencil, Tuning
from tests._util import EPS, ROUNDINGS

pytestmark = pytest.mark.gpu

TDT = {"f32": torch.float32, "f64": torch.float64, "bf16": torch.bfloat16}

# (stencil, side, field, coefficient storage, T, blocked candidates the benchmark may pick)
FULL = [
    ("7pt_const", 1024, "f32", None, 100, 6),
    ("7pt_const", 512, "f32", None, 100, 4),
    ("7pt_const", 512, "f64", None, 100, 4),
    ("7pt_var", 384, "f32", None, 50, 4),
    ("7pt_var", 384, "f32", "bf16", 50, 4),
    ("7pt_var", 384, "f64", None, 50, 4),
    ("25pt_var", 256, "f32", None, 40, 4),
    ("25pt_var", 256, "f32", "bf16", 40, 4),
]
SEED = 0


def _points(n, seams, rng):
    pts = {(0, 0, 0), (n - 1, n - 1, n - 1), (n - 1, 0, n // 2), (0, n - 1, n - 1), (n // 2, n // 3, 0)}
    for x in seams:
        for i in (x - 1, x):
            if 0 <= i < n:
                pts.add((i, int(rng.integers(n)), int(rng.integers(n))))
    while len(pts) < len(seams) * 2 + 11:
        pts.add(tuple(int(v) for v in rng.integers(0, n, size=3)))
    return sorted(pts)


def _crop(kind, n, fdt, cdt, lo, hi):
    """Host-drawn inputs inside [lo, hi), rounded to the precisions the device stores."""
    u0 = inputs.field_u0_box(SEED, n, n, n, lo, hi)
    if fdt == "f32":
        u0 = inputs.round_f32(u0)
    coefs = None
    if kind != "7pt_const":
        c = inputs.coefs_box(kind, SEED, n, n, n, lo, hi)
        st = cdt or fdt
        coefs = inputs.bf16_to_f64(inputs.bf16_bits(c)) if st == "bf16" else (
            inputs.round_f32(c) if st == "f32" else c)
    return u0, coefs


def _oracle_at(kind, n, fdt, cdt, T, pts):
    """u_T at each point (i, j, k) from crops of the host-drawn inputs, FP64; points whose
    crops coincide (all of them, once R*T reaches across the grid) share one call."""
    r = RADIUS[{"7pt_const": 0, "7pt_var": 1, "25pt_var": 2}[kind]]
    m = r * T + r
    sc = (0.4, 0.1)
    if fdt == "f32":
        sc = (float(np.float32(0.4)), float(np.float32(0.1)))
    groups = {}
    for q, (i, j, k) in enumerate(pts):
        lo = tuple(max(0, c - m) for c in (k, j, i))
        hi = tuple(min(n, c + m + 1) for c in (k, j, i))
        groups.setdefault((lo, hi), []).append(q)
    out = np.empty(len(pts))
    crops = [None] * len(pts)
    for (lo, hi), qs in groups.items():
        u0, coefs = _crop(kind, n, fdt, cdt, lo, hi)
        local = [(pts[q][0] - lo[2], pts[q][1] - lo[1], pts[q][2] - lo[0]) for q in qs]
        out[qs] = oracle.points(kind, u0, T, local, coefs=coefs, scalars=sc)
        for q in qs:
            crops[q] = (lo, hi, u0, coefs)
    return out, crops


@pytest.mark.parametrize("kind,n,fdt,cdt,T,ncand", FULL,
                         ids=[f"{k}-{n}-{f}{'-' + c if c else ''}-T{T}" for k, n, f, c, T, _ in FULL])
def test_full_size_sampled_parity(kind, n, fdt, cdt, T, ncand):
    dev = torch.device("cuda")
    s = Stencil(kind, n, n, n, dtype=TDT[fdt], coef_dtype=TDT[cdt or fdt], device=dev)
    u0 = inputs.field_u0_torch(SEED, n, n, n, TDT[fdt], dev)
    if kind == "7pt_const":
        s.set_coeffs(scalars=(0.4, 0.1))
    else:
        cs = inputs.coefs_torch(kind, SEED, n, n, n, TDT[cdt or fdt], dev)
        s.set_coeffs(arrays=cs)
        del cs
    tunings = tuner.candidates(s)[:ncand]
    seams = sorted({t.xtile * q for t in tunings for q in (1, 2) if t.xtile * q < n})[:6]
    pts = _points(n, seams, np.random.default_rng(n * 7 + T))
    ref, crops = _oracle_at(kind, n, fdt, cdt, T, pts)

    # the device grid holds exactly the crop's inputs
    ii = torch.tensor([p[0] for p in pts], device=dev)
    jj = torch.tensor([p[1] for p in pts], device=dev)
    kk = torch.tensor([p[2] for p in pts], device=dev)
    for (i, j, k), (lo, hi, c0, cc) in zip(pts, crops):
        assert float(u0[k, j, i]) == c0[k - lo[0], j - lo[1], i - lo[2]]
        if cc is not None:
            dc = [float(s.coef_interior(m)[k, j, i]) for m in range(len(s.coefs))]
            assert dc == list(cc[:, k - lo[0], j - lo[1], i - lo[2]])

    scale = max(float(np.max(np.abs(c[2]))) for c in crops)
    tol = max(T, 1) * 2 * ROUNDINGS[kind] * EPS[fdt] * scale
    # the wavefront tunings the benchmark times (2 and 6 levels for R = 1; 2 levels with copies
    # ahead and 3 levels for R = 4)
    waves = [Tuning(16, 16, 8, 2), Tuning(24, 8, 4, 0)] if kind == "25pt_var" else \
        [Tuning(4, 4, 16, 0), Tuning(12, 8, 4, 0)]
    runs = [("plain", None)] + [("blocked", t) for t in tunings] + [("wavefront", t) for t in waves] + \
        [("auto", None)]
    for scheme, tn in runs:
        s.set_field(u0, halo=0.0)
        s.set_tuning(scheme, tn)
        s.run(T)
        got = s.current[kk, jj, ii].double().cpu().numpy()
        err = np.max(np.abs(got - ref))
        assert err <= tol, (scheme, tn, err, tol)
