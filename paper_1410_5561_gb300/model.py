"""Cache-block-size and code-balance models of Section III, plus per-LUP work counts.

Section III-B, Eq. 2 (R = 1) and Eq. 3 (general R): bytes of the wavefront
cache block for diamond width D_w, frontlines N_F, leading-dimension tile of
N_xb bytes, N_D domain-sized streams:
    W_w = D_w - 2R + N_F
    C_S = N_xb * [N_D * D_w * (D_w/2 - R + N_F) + 2R (D_w + W_w)]
Section III-C, Eq. 4 (R = 1) and Eq. 5 (general R): double-precision code
balance of the blocked sweep,
    B_C = 16 R [(2 D_w - 2R) + (N_D D_w + 2R)] / D_w^2   bytes per LUP.
The "16" is 8 bytes per double times the 2 that turns the per-diamond counts
into per-LUP figures (the diamond holds N_z D_w^2 / (2R) LUPs). Written with
element sizes (field s_f, coefficient s_c, n_c coefficient arrays, N_D = 2 + n_c)
it reads 2R [s_f (2 D_w - 2R) + (2 s_f + n_c s_c) D_w + 2R s_f] / D_w^2.

The GPU kernel's shared-memory footprint is computed by the library itself
(stencil_blocked_smem_bytes); these functions serve the tuner's pruning and
the reported model code balance.
"""
from __future__ import annotations

RADIUS = {"7pt_const": 1, "7pt_var": 1, "25pt_var": 4}
NCOEF = {"7pt_const": 0, "7pt_var": 7, "25pt_var": 13}
# Flops per LUP counted as the listings write them: Listing 1 has 4 multiplications
# and 6 additions (10), Listing 2 has 7 multiplications and 6 additions (13),
# Listing 3 has 13 multiplications and 24 additions (37).
FLOPS = {"7pt_const": 10, "7pt_var": 13, "25pt_var": 37}
# Instructions on the floating-point pipe per LUP as the kernels issue them
# (a mul, an add or an fma is one each): 1 mul + 3 add + 3 fma, 1 mul + 6 fma,
# 1 mul + 12 add + 12 fma. The ALU roofline divides these by the measured FMA
# instruction rate.
FP_INSTR = {"7pt_const": 7, "7pt_var": 7, "25pt_var": 25}
DT_BYTES = {"f32": 4, "f64": 8, "bf16": 2}


def wavefront_width(dw: int, nf: int, r: int = 1) -> int:
    """W_w (Section III-B): D_w + N_F - 2 for R = 1, D_w - 2R + N_F in general."""
    return dw - 2 * r + nf


def cache_block_bytes_r1(dw: int, nf: int, nxb: float, nd: int) -> float:
    """Eq. 2 (R = 1)."""
    ww = wavefront_width(dw, nf, 1)
    return nxb * (nd * (dw * dw / 2 + dw * (nf - 1)) + 2 * (dw + ww))


def cache_block_bytes(dw: int, nf: int, nxb: float, nd: int, r: int = 1) -> float:
    """Eq. 3 (general R)."""
    ww = wavefront_width(dw, nf, r)
    return nxb * (nd * dw * (dw / 2 - r + nf) + 2 * r * (dw + ww))


def code_balance_dp(dw: int, nd: int, r: int = 1) -> float:
    """Eq. 5 (Eq. 4 at R = 1): double-precision bytes per LUP of the blocked sweep."""
    return 16 * r * ((2 * dw - 2 * r) + (nd * dw + 2 * r)) / (dw * dw)


def code_balance(dw: int, r: int, sf: int, nc: int, sc: int) -> float:
    """Eq. 5 with element sizes: field s_f bytes, n_c coefficient arrays of s_c bytes."""
    return 2 * r * (sf * (2 * dw - 2 * r) + (2 * sf + nc * sc) * dw + 2 * r * sf) / (dw * dw)


def plain_bytes_per_lup(sf: int, nc: int, sc: int) -> float:
    """One-step sweep: read u_t and the coefficients once, write u_{t+1} once."""
    return 2 * sf + nc * sc


def bytes_per_lup(kind: str, fdt: str, cdt: str | None, scheme: str, dw: int | None = None) -> float:
    """Algorithmic HBM bytes per LUP of a schedule (the per-unit figure the roofline uses)."""
    sf = DT_BYTES[fdt]
    nc = NCOEF[kind]
    sc = DT_BYTES[cdt or fdt]
    if scheme == "plain":
        return plain_bytes_per_lup(sf, nc, sc)
    return code_balance(dw, RADIUS[kind], sf, nc, sc)


def diamond_levels(dw: int, r: int) -> int:
    """Time levels one extruded diamond spans: D_w / R - 1."""
    return dw // r - 1
