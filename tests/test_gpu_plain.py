"""Plain one-step-per-pass sweeps on the GPU vs the FP64 oracle (Listings 1-3)."""
import numpy as np
import pytest

import oracle
from tests._util import Problem, step_tol

pytestmark = pytest.mark.gpu

CASES = [
    # kind, (nx, ny, nz), field, coef, T, halo
    ("7pt_const", (64, 64, 64), "f64", None, 8, 0.0),    # the 64^3 FP64 T=8 workload
    ("7pt_const", (67, 45, 33), "f32", None, 7, 0.0),
    ("7pt_const", (130, 9, 17), "f64", None, 5, 0.3),
    ("7pt_var", (70, 37, 29), "f32", None, 6, 0.0),
    ("7pt_var", (70, 37, 29), "f32", "bf16", 6, 0.0),
    ("7pt_var", (33, 40, 21), "f64", None, 6, -0.2),
    ("25pt_var", (45, 41, 38), "f32", None, 5, 0.0),
    ("25pt_var", (37, 29, 26), "f64", None, 4, 0.1),
    ("25pt_var", (45, 20, 19), "f32", "bf16", 3, 0.0),
    ("7pt_var", (1, 1, 1), "f32", None, 3, 0.5),
    ("25pt_var", (3, 2, 5), "f32", None, 2, 0.0),
]


@pytest.mark.parametrize("kind,shape,fdt,cdt,T,halo", CASES)
def test_plain_matches_oracle(kind, shape, fdt, cdt, T, halo):
    p = Problem(kind, *shape, fdt=fdt, cdt=cdt, seed=3, halo=halo)
    s = p.make()
    s.set_tuning("plain")
    s.run(T)
    got = s.get_field().double().cpu().numpy()
    ref = p.oracle(T)
    err = oracle.step_normalised_l2(got, ref, T)
    assert err <= step_tol(fdt), err
    assert np.max(np.abs(got - ref)) <= p.elementwise_tol(T)


def test_plain_T0_and_split_runs():
    p = Problem("7pt_var", 40, 31, 22, fdt="f32", seed=5)
    s = p.make()
    s.run(0)
    assert np.array_equal(s.get_field().cpu().numpy().astype(np.float64), p.u0)
    s.run(2)
    s.run(3)
    a = s.get_field().cpu()
    s2 = p.make()
    s2.run(5)
    assert np.array_equal(a.numpy(), s2.get_field().cpu().numpy())


def test_halo_cells_never_written():
    import torch
    p = Problem("25pt_var", 21, 19, 17, fdt="f32", seed=6, halo=0.7)
    s = p.make()
    s.run(3)
    s.sync()
    for f in s.fields:
        pad = s.padded(f).clone()
        lay = s.layout
        r, xo = lay.radius, lay.x_offset
        pad[r:r + s.nz, r:r + s.ny, xo:xo + s.nx] = float(np.float32(0.7))
        assert torch.all(pad == float(np.float32(0.7)))


@pytest.mark.parametrize("fdt", ["f32", "f64"])
def test_constant_invariant_bitwise(fdt):
    import torch
    from paper_1410_5561_gb300.stencil import Stencil
    tdt = torch.float32 if fdt == "f32" else torch.float64
    for kind, nc, w0, w in [("7pt_const", 0, 0.25, 0.125), ("7pt_var", 7, 0.25, 0.125),
                            ("25pt_var", 13, 0.25, 1.0 / 32)]:
        s = Stencil(kind, 37, 23, 19, dtype=tdt)
        if nc:
            arrs = [torch.full((19, 23, 37), w0 if m == 0 else w, dtype=tdt) for m in range(nc)]
            s.set_coeffs(arrays=arrs)
        else:
            s.set_coeffs(scalars=(w0, w))
        s.set_field(torch.full((19, 23, 37), 0.75, dtype=tdt), halo=0.75)
        s.run(5)
        assert torch.all(s.get_field() == 0.75)


@pytest.mark.parametrize("shape", [(37, 29, 21), (64, 16, 8), (5, 3, 2)])
@pytest.mark.parametrize("fdt", ["f32", "f64"])
def test_set_and_get_field_through_every_memory_kind(shape, fdt):
    """set_field / get_field with device memory, page-locked host memory (moved by the
    library's copy kernel over the host link) and pageable host memory (pitched DMA): the
    same interior, bit for bit, the halo left at the Dirichlet value; row lengths that are and
    are not a multiple of 16 bytes."""
    import torch
    p = Problem("7pt_var", *shape, fdt=fdt, seed=31, halo=0.75)
    tdt = torch.float32 if fdt == "f32" else torch.float64
    ref = torch.from_numpy(p.u0).to(tdt)
    sources = {"device": ref.cuda(), "pinned": ref.clone().pin_memory(), "pageable": ref.clone()}
    for name, src in sources.items():
        s = p.make()
        s.set_field(src, halo=0.75)
        torch.cuda.synchronize()
        dense = s.get_field().cpu()
        assert torch.equal(dense, ref), name
        padded = s.padded(s.fields[s.parity]).cpu()
        lay = s.layout
        r, xo = lay.radius, lay.x_offset
        inner = torch.zeros_like(padded, dtype=torch.bool)
        inner[r:r + s.nz, r:r + s.ny, xo:xo + s.nx] = True
        halo = padded[~inner]
        assert torch.all(halo == 0.75), name
        for oname, out in {"device": torch.empty_like(ref, device="cuda"),
                           "pinned": torch.empty_like(ref).pin_memory(), "pageable": torch.empty_like(ref)}.items():
            s.get_field(out)
            torch.cuda.synchronize()
            assert torch.equal(out.cpu(), ref), (name, oname)


@pytest.mark.parametrize("kind,shape,fdt,cdt", [
    ("7pt_const", (150, 37, 29), "f32", None), ("7pt_const", (70, 21, 18), "f64", None),
    ("7pt_var", (133, 29, 19), "f32", None), ("7pt_var", (40, 43, 17), "f32", "bf16"),
    ("7pt_var", (33, 19, 14), "f64", None), ("25pt_var", (141, 35, 27), "f32", None),
    ("25pt_var", (27, 33, 19), "f32", "bf16"), ("25pt_var", (38, 25, 30), "f64", None),
])
@pytest.mark.parametrize("T", [1, 4])
def test_prefetched_plain_sweep_is_bitwise_equal(kind, shape, fdt, cdt, T):
    """The plain sweep with every load of a plane copied two planes ahead into shared memory
    (plain tuning nf = 2) runs the same update on the same operands: bit-identical results."""
    from paper_1410_5561_gb300.stencil import Tuning
    p = Problem(kind, *shape, fdt=fdt, cdt=cdt, seed=41, halo=0.375)
    a = p.make()
    a.set_tuning("plain", Tuning(0, 0, 0, 0))
    a.run(T)
    b = p.make()
    b.set_tuning("plain", Tuning(0, 2, 0, 0))
    b.run(T)
    assert np.array_equal(a.get_field().cpu().numpy(), b.get_field().cpu().numpy())
