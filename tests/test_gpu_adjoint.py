"""Adjoint sweep on the GPU: against the FP64 oracle adjoint, the dot-product
identity, finite differences, and independence from the checkpoint interval."""
import numpy as np
import pytest

import oracle
from paper_1410_5561_gb300 import inputs
from tests._util import Problem

pytestmark = pytest.mark.gpu


def _grid_and_inputs(kind, shape, fdt, cdt=None, seed=21, halo=0.0, tuning=None):
    import torch
    p = Problem(kind, *shape, fdt=fdt, cdt=cdt, seed=seed, halo=halo)
    s = p.make()
    if tuning is not None:
        s.set_tuning("blocked", tuning)
    u0, coefs = p.torch_inputs("cuda")
    target = inputs.field_target(seed, *shape)
    if fdt == "f32":
        target = inputs.round_f32(target)
    return p, s, u0, coefs, torch.from_numpy(target).to("cuda", dtype=u0.dtype)


def _autograd_grads(s, u0, coefs, target, T, k=0, halo=0.0):
    import torch
    from paper_1410_5561_gb300.autograd import sweep
    u = u0.clone().requires_grad_(True)
    c = coefs.clone().requires_grad_(True)
    uT = sweep(u, c, s, T, k, halo)
    loss = 0.5 * ((uT.double() - target.double()) ** 2).sum()
    loss.backward()
    return float(loss.detach()), u.grad.double().cpu().numpy(), s.last_coef_grad.cpu().numpy()


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


@pytest.mark.parametrize("kind,shape,fdt,cdt,T,tol", [
    ("7pt_var", (13, 11, 9), "f64", None, 6, 1e-12),
    ("25pt_var", (17, 15, 13), "f64", None, 4, 1e-12),
    ("7pt_var", (33, 20, 17), "f32", None, 8, 2e-5),
    ("7pt_var", (33, 20, 17), "f32", "bf16", 8, 2e-5),
    ("25pt_var", (24, 19, 18), "f32", None, 5, 2e-5),
])
def test_adjoint_matches_oracle(kind, shape, fdt, cdt, T, tol):
    p, s, u0, coefs, target = _grid_and_inputs(kind, shape, fdt, cdt, halo=0.0)
    loss, gu, gc = _autograd_grads(s, u0, coefs, target, T)
    tnp = target.double().cpu().numpy()
    rl, ru, rc = oracle.adjoint(kind, p.u0, p.coefs, tnp, T)
    assert abs(loss - rl) <= tol * max(1.0, abs(rl))
    assert _rel(gu, ru) <= tol
    assert _rel(gc, rc) <= tol


def test_adjoint_nonzero_halo_fp64():
    p, s, u0, coefs, target = _grid_and_inputs("7pt_var", (9, 10, 11), "f64", halo=0.3)
    loss, gu, gc = _autograd_grads(s, u0, coefs, target, 5, halo=0.3)
    rl, ru, rc = oracle.adjoint("7pt_var", p.u0, p.coefs, target.cpu().numpy(), 5, halo=0.3)
    assert _rel(gu, ru) <= 1e-12 and _rel(gc, rc) <= 1e-12


@pytest.mark.parametrize("k", [1, 2, 3, 7, 50])
def test_checkpoint_interval_does_not_change_result(k):
    p, s, u0, coefs, target = _grid_and_inputs("25pt_var", (20, 18, 16), "f32")
    _, gu0, gc0 = _autograd_grads(s, u0, coefs, target, 7, 0)
    _, gu, gc = _autograd_grads(s, u0, coefs, target, 7, k)
    assert np.array_equal(gu, gu0) and np.array_equal(gc, gc0)


def test_blocked_forward_checkpoints_match_plain():
    from paper_1410_5561_gb300.stencil import Tuning
    p, s, u0, coefs, target = _grid_and_inputs("7pt_var", (40, 33, 21), "f32")
    _, gu0, gc0 = _autograd_grads(s, u0, coefs, target, 9)
    s.set_tuning("blocked", Tuning(8, 2, 8, 16))
    _, gu, gc = _autograd_grads(s, u0, coefs, target, 9)
    assert np.array_equal(gu, gu0) and np.array_equal(gc, gc0)


def test_dot_product_identity_fp64():
    """<lambda, A^T... > : <y, lam> = <w, g_u0> with y = A^T w (linear, zero halo)."""
    import torch
    from paper_1410_5561_gb300.autograd import sweep
    p, s, u0, coefs, _ = _grid_and_inputs("25pt_var", (21, 22, 23), "f64")
    T = 6
    w = u0.clone().requires_grad_(True)
    y = sweep(w, coefs, s, T)
    lam = torch.from_numpy(inputs.uniform(77, 0, y.shape, -1, 1)).cuda()
    (y * lam).sum().backward()
    lhs = float((y.detach() * lam).sum())
    rhs = float((w.detach() * w.grad).sum())
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


def test_finite_differences_32cube_fp64():
    """Gradients at 32^3 against central differences of the GPU forward (FP64):
    exact in u0 (the loss is quadratic in u0), O(h^2) in the coefficients."""
    import torch
    from paper_1410_5561_gb300.autograd import sweep
    p, s, u0, coefs, target = _grid_and_inputs("25pt_var", (32, 32, 32), "f64")
    T = 4
    loss, gu, gc = _autograd_grads(s, u0, coefs, target, T)

    def L(u, c):
        with torch.no_grad():
            uT = sweep(u, c, s, T)
            return 0.5 * float(((uT - target) ** 2).sum())

    rng = np.random.default_rng(3)
    for _ in range(4):
        i, j, k = (int(v) for v in rng.integers(0, 32, 3))
        h = 1e-3
        up = u0.clone(); up[k, j, i] += h
        um = u0.clone(); um[k, j, i] -= h
        fd = (L(up, coefs) - L(um, coefs)) / (2 * h)
        assert abs(fd - gu[k, j, i]) <= 1e-8 * max(1.0, abs(fd))
    for _ in range(8):
        m = int(rng.integers(0, 13))
        i, j, k = (int(v) for v in rng.integers(0, 32, 3))
        # the loss is ~1e4 here: h must keep the rounding noise eps*L/h well below the gradient
        h = 1e-3 * max(abs(float(coefs[m, k, j, i])), 1e-3)
        cp = coefs.clone(); cp[m, k, j, i] += h
        cm = coefs.clone(); cm[m, k, j, i] -= h
        fd = (L(u0, cp) - L(u0, cm)) / (2 * h)
        assert abs(fd - gc[m, k, j, i]) <= 1e-6 * max(1.0, abs(fd))


def test_full_size_25pt_adjoint_dot_product_fp32():
    """256^3 FP32, T=40, sqrt(T) checkpoints: <y, lam> = <w, g_w> to FP32 accuracy."""
    import torch
    from paper_1410_5561_gb300.autograd import sweep
    from paper_1410_5561_gb300.stencil import Stencil
    n, T = 256, 40
    s = Stencil("25pt_var", n, n, n, dtype=torch.float32)
    r = []
    acc = None
    for m in range(13):
        x = torch.empty((n, n, n), dtype=torch.float64, device="cuda")
        inputs.fill_uniform_torch(x, 0, inputs.STREAM_COEF0 + m, 0.0, 1.0)
        acc = x.clone() if acc is None else acc.add_(x if m == 0 else 2 * x)
        r.append(x)
    coefs = torch.stack([(0.95 * x / acc).float() for x in r])
    del r, acc
    w = torch.empty((n, n, n), dtype=torch.float32, device="cuda")
    inputs.fill_uniform_torch(w, 0, inputs.STREAM_U0, -1.0, 1.0)
    w.requires_grad_(True)
    y = sweep(w, coefs, s, T)
    lam = torch.empty_like(y)
    inputs.fill_uniform_torch(lam, 0, inputs.STREAM_TARGET, -1.0, 1.0)
    (y * lam).sum().backward()
    lhs = float((y.detach().double() * lam.double()).sum())
    rhs = float((w.detach().double() * w.grad.double()).sum())
    assert abs(lhs - rhs) <= 1e-4 * (float(y.detach().double().norm()) * float(lam.double().norm()))
    assert s.last_coef_grad.shape == (13, n, n, n)
    assert torch.isfinite(s.last_coef_grad).all()


def test_single_step_gradient_is_exact_product_fp32():
    """T = 1: gC_m(p) = lambda_1(p) u_0(p + o_m), a product of two FP32 values and exact in
    FP64. Pins the FP32 -> FP64 conversion of the gradient update bit for bit, with
    subnormals, signed zeros and large values planted in both factors."""
    import torch
    p = Problem("7pt_var", 37, 9, 7, fdt="f32", seed=5)
    s = p.make()
    u0 = p.u0.astype(np.float32)
    f = u0.reshape(-1)
    f[::11] = np.float32(1e-40)
    f[3::17] = np.float32(-3e-42)
    f[5::23] = np.float32(0.0)
    f[7::29] = np.float32(-0.0)
    f[9::31] = np.float32(3e30)
    s.set_field(torch.from_numpy(u0).cuda(), halo=0.0)
    lam = inputs.uniform(9, 0, u0.shape, -1, 1).astype(np.float32)
    g = lam.reshape(-1)
    g[2::13] = np.float32(2e-39)
    g[4::19] = np.float32(-0.0)
    ws = s.adjoint_workspace(1, 1)
    s.run_checkpointed(1, 1, ws)
    lam_t = s.new_field_array(zero=True)
    s.interior_of(lam_t).copy_(torch.from_numpy(lam).cuda())
    gu = s.new_field_array(zero=False)
    gc = [s.new_grad_array() for _ in range(7)]
    s.run_adjoint(1, 1, lam_t, gu, gc, ws)
    torch.cuda.synchronize()
    up = np.zeros((u0.shape[0] + 2, u0.shape[1] + 2, u0.shape[2] + 2))
    up[1:-1, 1:-1, 1:-1] = u0.astype(np.float64)
    nz, ny, nx = u0.shape
    # neighbour weighed by C_m (Listing 2 order: centre, +x, -x, +y, -y, +z, -z), axes (z, y, x)
    offs = [(0, 0, 0), (0, 0, 1), (0, 0, -1), (0, 1, 0), (0, -1, 0), (1, 0, 0), (-1, 0, 0)]
    for m, (dz, dy, dx) in enumerate(offs):
        nb = up[1 + dz:1 + dz + nz, 1 + dy:1 + dy + ny, 1 + dx:1 + dx + nx]
        want = lam.astype(np.float64) * nb + 0.0  # accumulated onto +0: a -0 product reads +0
        got = s.interior_of(gc[m]).cpu().numpy()
        assert np.array_equal(got.view(np.uint64), want.view(np.uint64)), m


@pytest.mark.parametrize("kind,fdt,scheme", [("25pt_var", "f32", "plain"), ("7pt_var", "f32", "blocked"),
                                             ("25pt_var", "f32", "wavefront")])
def test_forward_and_backward_captured_in_one_cuda_graph(kind, fdt, scheme):
    """The differentiable sweep (checkpointed forward, recompute, transposed steps, gradient
    passes) enqueues only device work, so forward and backward together can be captured in
    one CUDA graph; each replay reproduces the eager gradients bit for bit."""
    import torch
    from paper_1410_5561_gb300.autograd import sweep
    p, s, u0, coefs, target = _grid_and_inputs(kind, (40, 29, 23), fdt, seed=31)
    s.set_tuning(scheme, None)
    T = 9
    loss_e, gu_e, gc_e = _autograd_grads(s, u0, coefs, target, T)
    u = u0.clone().requires_grad_(True)
    c = coefs.clone().requires_grad_(True)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):  # warm-up on the capture stream (workspace, autograd state)
        s.set_stream(side)
        (0.5 * ((sweep(u, c, s, T).double() - target.double()) ** 2).sum()).backward()
    torch.cuda.current_stream().wait_stream(side)
    u.grad, c.grad = None, None
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        loss = 0.5 * ((sweep(u, c, s, T).double() - target.double()) ** 2).sum()
        loss.backward()
    for _ in range(2):
        g.replay()
        torch.cuda.synchronize()
        assert float(loss.detach()) == loss_e
        assert np.array_equal(u.grad.double().cpu().numpy(), gu_e)
        assert np.array_equal(s.last_coef_grad.cpu().numpy(), gc_e)


@pytest.mark.parametrize("kind,shape,fdt,cdt,T,k", [
    ("25pt_var", (44, 31, 27), "f32", None, 11, 0), ("7pt_var", (70, 33, 25), "f32", None, 13, 5),
    ("25pt_var", (30, 26, 22), "f32", None, 9, 9), ("7pt_var", (41, 29, 23), "f64", None, 8, 0),
    ("25pt_var", (36, 28, 24), "f32", "bf16", 7, 0),
    ("7pt_var", (300, 520, 6), "f32", None, 8, 4),  # 390 tiles: more (level, tile) pairs than CTAs
])
def test_wavefront_backward_gives_the_plain_gradients(kind, shape, fdt, cdt, T, k):
    """With the grid tuned to the wavefront schedule, the backward pass runs temporally blocked:
    each checkpoint segment's states are recomputed by one wavefront pass that writes every time
    level to its own array, and the segment's cotangents by one wavefront pass of transposed
    steps, each level writing its own cotangent array. Both give the per-step results bit for
    bit, so the gradients equal the plain-tuned grid's, and they match the FP64 oracle adjoint."""
    from paper_1410_5561_gb300.stencil import Tuning
    p, s, u0, coefs, target = _grid_and_inputs(kind, shape, fdt, cdt, seed=33)
    loss_p, gu_p, gc_p = _autograd_grads(s, u0, coefs, target, T, k)
    R = 4 if kind == "25pt_var" else 1
    s.set_tuning("wavefront", Tuning(4 * R, R, 4, 0))
    loss_w, gu_w, gc_w = _autograd_grads(s, u0, coefs, target, T, k)
    assert loss_w == loss_p
    assert np.array_equal(gu_w, gu_p) and np.array_equal(gc_w, gc_p)
    tol = 1e-12 if fdt == "f64" else 2e-5
    rl, ru, rc = oracle.adjoint(kind, p.u0, p.coefs, target.double().cpu().numpy(), T)
    assert _rel(gu_w, ru) <= tol and _rel(gc_w, rc) <= tol
