"""Shared test helpers: seeded problems in the precision each path consumes.

Both sides of every parity test receive the same values: FP64 draws from
``paper_1410_5561_gb300.inputs``, rounded once to the GPU's storage precision;
the FP64 oracle consumes the rounded values.
"""
from __future__ import annotations

import numpy as np

from paper_1410_5561_gb300 import inputs

EPS = {"f32": 2.0 ** -24, "f64": 2.0 ** -53}
# roundings per update on the GPU (mul + adds + fmas), Listings 1-3
ROUNDINGS = {"7pt_const": 7, "7pt_var": 7, "25pt_var": 25}


class Problem:
    """u0, coefficients and scalars for one grid, as FP64 arrays holding the
    values the GPU stores (rounded to its field / coefficient precision)."""

    def __init__(self, kind, nx, ny, nz, fdt="f32", cdt=None, seed=0, halo=0.0, row_sum=0.95,
                 c0=0.4, c1=0.1):
        self.kind, self.nx, self.ny, self.nz = kind, nx, ny, nz
        self.fdt = fdt
        self.cdt = cdt or fdt
        self.halo = halo
        u0 = inputs.field_u0(seed, nx, ny, nz)
        self.u0 = inputs.round_f32(u0) if fdt == "f32" else u0
        if fdt == "f32":
            self.halo = float(np.float32(halo))
        self.scalars = (c0, c1)
        if fdt == "f32":
            self.scalars = (float(np.float32(c0)), float(np.float32(c1)))
        self.coefs = None
        self.coef_bits = None
        if kind == "7pt_var":
            c = inputs.coefs_7pt_var(seed, nx, ny, nz, row_sum)
        elif kind == "25pt_var":
            c = inputs.coefs_25pt_var(seed, nx, ny, nz, row_sum)
        else:
            c = None
        if c is not None:
            if self.cdt == "bf16":
                self.coef_bits = inputs.bf16_bits(c)
                self.coefs = inputs.bf16_to_f64(self.coef_bits)
            elif self.cdt == "f32":
                self.coefs = inputs.round_f32(c)
            else:
                self.coefs = c

    def torch_inputs(self, device):
        import torch
        tdt = {"f32": torch.float32, "f64": torch.float64}[self.fdt]
        u0 = torch.from_numpy(self.u0).to(device=device, dtype=tdt)
        coefs = None
        if self.coefs is not None:
            if self.cdt == "bf16":
                coefs = torch.from_numpy(self.coef_bits.view(np.int16)).view(torch.bfloat16).to(device)
            else:
                coefs = torch.from_numpy(self.coefs).to(device=device, dtype=tdt)
        return u0, coefs

    def make(self, device="cuda", workspace=True):
        import torch
        from paper_1410_5561_gb300.stencil import Stencil
        tdt = {"f32": torch.float32, "f64": torch.float64}[self.fdt]
        cdt = {"f32": torch.float32, "f64": torch.float64, "bf16": torch.bfloat16}[self.cdt]
        s = Stencil(self.kind, self.nx, self.ny, self.nz, dtype=tdt, coef_dtype=cdt, device=device,
                    workspace=workspace)
        u0, coefs = self.torch_inputs(device)
        if self.kind == "7pt_const":
            s.set_coeffs(scalars=self.scalars)
        else:
            s.set_coeffs(arrays=list(coefs))
        s.set_field(u0, halo=self.halo)
        return s

    def oracle(self, T):
        import oracle
        return oracle.sweep(self.kind, self.u0, T, coefs=self.coefs, scalars=self.scalars, halo=self.halo)

    def elementwise_tol(self, T):
        """Bound on |gpu - oracle|: with sum |weights| <= 1 per row, each step adds at
        most (2 * roundings) * eps * max|u| and earlier errors do not grow."""
        m = max(float(np.max(np.abs(self.u0))), abs(self.halo))
        return max(T, 1) * 2 * ROUNDINGS[self.kind] * EPS[self.fdt] * m


def step_tol(fdt):
    """Per-step-normalised L2 gate on u_T vs the FP64 oracle."""
    return 1e-5 if fdt == "f32" else 1e-12
