"""Seeded synthetic inputs for the stencil sweeps.

This module is shared by the FP64 oracle tests and the GPU path, and holds none
of the method's arithmetic: it only draws numbers and shapes.

Generator (counter-based SplitMix64, written from its published definition by
Steele, Lea and Flood, "Fast splittable pseudorandom number generators", 2014):

    mix(z)  = z ^= z >> 30; z *= 0xBF58476D1CE4E5B9;
              z ^= z >> 27; z *= 0x94D049BB133111EB; z ^= z >> 31
    key     = mix(seed * G + stream)          (G = 0x9E3779B97F4A7C15, mod 2^64)
    x(n)    = mix(key + (n + 1) * G)
    u(n)    = (x(n) >> 11) * 2^-53            in [0, 1)

``n`` is the linear index over the interior with x fastest, then y, then z.
Streams: field u0 = 0, target = 1, coefficient array m = 2 + m, batch shapes
= 100 + (0: nx, 1: ny, 2: nz, 3: T).

Workload recipes (the paper's experiments use synthetic cubic grids, Section
IV; the sizes here are the ones this library is measured on):

* u0 and the adjoint target: uniform on [-1, 1].
* 7-point variable coefficients (Listing 2): r_m ~ U(0,1), m = 0..6;
  C_m = s * r_m / sum_m r_m, so the seven weights of every point sum to s.
* 25-point variable coefficients (Listing 3): r_m ~ U(0,1), m = 0..12;
  C00 = s * r_0 / S, C_m = s * r_m / S with S = r_0 + 2 * sum_{m>=1} r_m, so
  the operator's row sum (each axis coefficient weighs two points) is s.
* Reduced precisions are produced here by rounding the FP64 draws (round to
  nearest even); every consumer, the oracle included, takes the rounded values.
"""
from __future__ import annotations

import numpy as np

_G = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

STREAM_U0 = 0
STREAM_TARGET = 1
STREAM_COEF0 = 2
STREAM_SHAPES = 100

_CHUNK = 1 << 22


def _mix_np(z):
    with np.errstate(over="ignore"):
        z = z ^ (z >> np.uint64(30))
        z = z * _M1
        z = z ^ (z >> np.uint64(27))
        z = z * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def stream_key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * _G + np.uint64(stream)
    return _mix_np(np.array([z], dtype=np.uint64))[0]


def uniform01_range(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """u(n) for n in [start, start+count), float64 in [0, 1)."""
    key = stream_key(seed, stream)
    n = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        x = _mix_np(key + n * _G)
    return (x >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def fill_uniform(out: np.ndarray, seed: int, stream: int, lo: float, hi: float) -> np.ndarray:
    """Fill a C-contiguous array (any float dtype) with lo + (hi-lo)*u(n), n = flat index.

    Draws are made in FP64 and rounded once to ``out.dtype``.
    """
    flat = out.reshape(-1)
    total = flat.size
    for s in range(0, total, _CHUNK):
        c = min(_CHUNK, total - s)
        u = uniform01_range(seed, stream, s, c)
        flat[s:s + c] = lo + (hi - lo) * u
    return out


def _mix_torch(z):
    """SplitMix64 mix on int64 tensors (two's-complement wrap; logical shifts by masking)."""
    import torch
    def shr(x, k):
        return (x >> k) & ((1 << (64 - k)) - 1)
    z = z ^ shr(z, 30)
    z = z * _s64(0xBF58476D1CE4E5B9)
    z = z ^ shr(z, 27)
    z = z * _s64(0x94D049BB133111EB)
    z = z ^ shr(z, 31)
    return z


def _s64(u: int) -> int:
    u &= 0xFFFFFFFFFFFFFFFF
    return u - (1 << 64) if u >= (1 << 63) else u


def fill_uniform_torch(out, seed: int, stream: int, lo: float, hi: float, chunk: int = 1 << 24):
    """Same values as :func:`fill_uniform`, computed with torch ops on ``out``'s device."""
    import torch
    flat = out.view(-1)
    key = _s64(int(stream_key(seed, stream)))
    g = _s64(0x9E3779B97F4A7C15)
    for s0 in range(0, flat.numel(), chunk):
        c = min(chunk, flat.numel() - s0)
        n = torch.arange(s0 + 1, s0 + c + 1, dtype=torch.int64, device=out.device)
        x = _mix_torch(n * g + key)
        u = ((x >> 11) & ((1 << 53) - 1)).to(torch.float64) * (2.0 ** -53)
        flat[s0:s0 + c] = (lo + (hi - lo) * u).to(out.dtype)
    return out


def uniform(seed: int, stream: int, shape, lo: float = 0.0, hi: float = 1.0,
            dtype=np.float64) -> np.ndarray:
    out = np.empty(tuple(shape), dtype=dtype)
    return fill_uniform(out, seed, stream, lo, hi)


def field_u0(seed: int, nx: int, ny: int, nz: int, dtype=np.float64) -> np.ndarray:
    """Initial interior field, shape (nz, ny, nx), uniform on [-1, 1]."""
    return uniform(seed, STREAM_U0, (nz, ny, nx), -1.0, 1.0, dtype)


def field_target(seed: int, nx: int, ny: int, nz: int, dtype=np.float64) -> np.ndarray:
    """Adjoint target field u_target, shape (nz, ny, nx), uniform on [-1, 1]."""
    return uniform(seed, STREAM_TARGET, (nz, ny, nx), -1.0, 1.0, dtype)


def _normalise(kind: str, r, row_sum: float):
    """Coefficient arrays from raw draws r[m] (numpy or torch FP64, any shape).

    7-point: C_m = row_sum * r_m / (r_0 + ... + r_6), so the seven weights of a
    point sum to row_sum. 25-point: C_m = row_sum * r_m / (r_0 + 2 (r_1 + ... + r_12)),
    since C_1..C_12 each weigh two neighbours. The sums run left to right and the
    same operations are done on either array type, so host and device values agree
    bit for bit.
    """
    if kind == "7pt_var":
        s = r[0] + r[1]
        for m in range(2, 7):
            s = s + r[m]
    else:
        t = r[1] + r[2]
        for m in range(3, 13):
            t = t + r[m]
        s = r[0] + 2.0 * t
    return [row_sum * r[m] / s for m in range(len(r))]


def coefs_7pt_var(seed: int, nx: int, ny: int, nz: int, row_sum: float = 0.95) -> np.ndarray:
    """Seven coefficient arrays (C0..C6), shape (7, nz, ny, nx), FP64.

    Order and neighbour of each array follow Listing 2: C0 centre, C1 +x,
    C2 -x, C3 +y, C4 -y, C5 +z, C6 -z.
    """
    r = [uniform(seed, STREAM_COEF0 + m, (nz, ny, nx)) for m in range(7)]
    return np.stack(_normalise("7pt_var", r, row_sum))


def coefs_25pt_var(seed: int, nx: int, ny: int, nz: int, row_sum: float = 0.95) -> np.ndarray:
    """Thirteen coefficient arrays (C00..C12), shape (13, nz, ny, nx), FP64.

    C00 weighs the centre; C(3(d-1)+a+1) weighs the pair at distance d on axis
    a (x=0, y=1, z=2), as in Listing 3.
    """
    r = [uniform(seed, STREAM_COEF0 + m, (nz, ny, nx)) for m in range(13)]
    return np.stack(_normalise("25pt_var", r, row_sum))


def box_uniform(seed: int, stream: int, shape, lo, hi, a: float = 0.0, b: float = 1.0) -> np.ndarray:
    """The values of ``uniform(seed, stream, shape, a, b)`` inside the box [lo, hi) (index
    order (z, y, x)), drawn without materialising the whole array."""
    nz, ny, nx = shape
    k = np.arange(lo[0], hi[0], dtype=np.uint64)[:, None, None]
    j = np.arange(lo[1], hi[1], dtype=np.uint64)[None, :, None]
    i = np.arange(lo[2], hi[2], dtype=np.uint64)[None, None, :]
    n = (k * np.uint64(ny) + j) * np.uint64(nx) + i + np.uint64(1)  # counter of flat index
    key = stream_key(seed, stream)
    with np.errstate(over="ignore"):
        x = _mix_np(key + n * _G)
    return a + (b - a) * ((x >> np.uint64(11)).astype(np.float64) * (2.0 ** -53))


def field_u0_box(seed: int, nx: int, ny: int, nz: int, lo, hi) -> np.ndarray:
    """``field_u0(seed, nx, ny, nz)[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]]``."""
    return box_uniform(seed, STREAM_U0, (nz, ny, nx), lo, hi, -1.0, 1.0)


def coefs_box(kind: str, seed: int, nx: int, ny: int, nz: int, lo, hi, row_sum: float = 0.95) -> np.ndarray:
    """The coefficient arrays of ``coefs_7pt_var`` / ``coefs_25pt_var`` inside a box."""
    nc = 7 if kind == "7pt_var" else 13
    r = [box_uniform(seed, STREAM_COEF0 + m, (nz, ny, nx), lo, hi) for m in range(nc)]
    return np.stack(_normalise(kind, r, row_sum))


def field_u0_torch(seed: int, nx: int, ny: int, nz: int, dtype, device):
    """``field_u0`` drawn on a torch device, rounded once to ``dtype``."""
    import torch
    out = torch.empty((nz, ny, nx), dtype=dtype, device=device)
    return fill_uniform_torch(out, seed, STREAM_U0, -1.0, 1.0)


def coefs_torch(kind: str, seed: int, nx: int, ny: int, nz: int, dtype, device, row_sum: float = 0.95):
    """The coefficient arrays of ``coefs_7pt_var`` / ``coefs_25pt_var`` computed on a torch
    device in FP64 and rounded once to ``dtype``; a list of (nz, ny, nx) tensors."""
    import torch
    nc = 7 if kind == "7pt_var" else 13
    r = []
    for m in range(nc):
        t = torch.empty((nz, ny, nx), dtype=torch.float64, device=device)
        r.append(fill_uniform_torch(t, seed, STREAM_COEF0 + m, 0.0, 1.0))
    c = _normalise(kind, r, row_sum)
    del r
    if dtype == torch.bfloat16:  # bf16_bits' rounding: to FP32 first, then to bfloat16
        return [x.to(torch.float32).to(dtype) for x in c]
    return [x.to(dtype) for x in c]


def batch_shapes(seed: int, count: int = 64, side_lo: int = 32, side_hi: int = 192,
                 t_lo: int = 10, t_hi: int = 200):
    """Per-grid (nx, ny, nz, T) for the batched workload; bounds inclusive."""
    out = []
    cols = []
    for j, (lo, hi) in enumerate([(side_lo, side_hi)] * 3 + [(t_lo, t_hi)]):
        u = uniform01_range(seed, STREAM_SHAPES + j, 0, count)
        cols.append(lo + np.floor(u * (hi - lo + 1)).astype(np.int64))
    for i in range(count):
        out.append(tuple(int(c[i]) for c in cols))
    return out


def round_f32(a: np.ndarray) -> np.ndarray:
    """Round FP64 values to FP32 (nearest even) and return them as FP64."""
    return np.asarray(a, dtype=np.float64).astype(np.float32).astype(np.float64)


def bf16_bits(a: np.ndarray) -> np.ndarray:
    """Round to bfloat16 (nearest even, via FP32) and return the uint16 bit patterns."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float64).astype(np.float32))
    b = f.view(np.uint32).astype(np.uint64)
    lsb = (b >> np.uint64(16)) & np.uint64(1)
    r = (b + np.uint64(0x7FFF) + lsb) >> np.uint64(16)
    return r.astype(np.uint16)


def bf16_to_f64(bits: np.ndarray) -> np.ndarray:
    return (bits.astype(np.uint32) << np.uint32(16)).view(np.float32).astype(np.float64)


def round_bf16(a: np.ndarray) -> np.ndarray:
    """Round FP64 values to bfloat16 (nearest even) and return them as FP64."""
    return bf16_to_f64(bf16_bits(a))
