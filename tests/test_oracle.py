"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each check is chosen so that a plausible slip in the oracle (a dropped term, a
sign or index error, a coefficient attached to the wrong neighbour, a missing
halo contribution, a transposed operand in the adjoint) fails at least one:

* closed form: Dirichlet sine modes are eigenvectors of the 7-point operators
  (Listings 1 and 2 with axis-wise constant weights); amplification
  c0 + 2*(cx cos a + cy cos b + cz cos c) per step;
* invariant: a constant field with operator row sum 1 and a matching halo
  stays constant, bit for bit, with dyadic weights;
* shift special cases: one coefficient array alone reduces each step to a
  weighted shift (or pair of shifts) of the padded array, written with numpy
  slicing; superposition over the arrays recovers the full step;
* dense brute force on tiny grids: the operator assembled as a matrix from a
  neighbour table, applied T times;
* adjoint: transpose identity <A^T l, w> = <l, A w>, the assembled matrix's
  transpose, and central finite differences (exact in u0, O(h^2) in C);
* point evaluation on the dependency box equals the full sweep.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1410_5561_gb300 import inputs

RNG_SEED = 7


def _rand(shape, seed, lo=-1.0, hi=1.0):
    return inputs.uniform(seed, 0, shape, lo, hi)


# ----------------------------------------------------------------- closed form

def _sine_mode(nx, ny, nz, p, q, r):
    i = np.arange(1, nx + 1)
    j = np.arange(1, ny + 1)
    k = np.arange(1, nz + 1)
    sx = np.sin(p * math.pi * i / (nx + 1))
    sy = np.sin(q * math.pi * j / (ny + 1))
    sz = np.sin(r * math.pi * k / (nz + 1))
    return sz[:, None, None] * sy[None, :, None] * sx[None, None, :]


@pytest.mark.parametrize("pqr", [(1, 1, 1), (2, 3, 1), (9, 1, 4), (9, 7, 8), (5, 6, 2)])
def test_sine_eigenmode_7pt_const(pqr):
    nx, ny, nz = 9, 7, 8
    p, q, r = pqr
    c0, c1 = 0.4, 0.1
    u0 = _sine_mode(nx, ny, nz, p, q, r)
    lam = c0 + 2 * c1 * (math.cos(p * math.pi / (nx + 1)) + math.cos(q * math.pi / (ny + 1))
                         + math.cos(r * math.pi / (nz + 1)))
    T = 12
    uT = oracle.sweep("7pt_const", u0, T, scalars=(c0, c1))
    ref = lam ** T * u0
    scale = max(abs(lam) ** T, 1e-300)
    assert np.max(np.abs(uT - ref)) <= 1e-14 * T * 8 + 1e-15 * scale
    # rounding of u0 excites other modes, so the bound is relative to |u0|;
    # where the mode is still large it must also hold relative to the mode
    if abs(lam) ** T > 1e-3:
        assert np.max(np.abs(uT - ref)) / np.max(np.abs(ref)) < 1e-12


@pytest.mark.parametrize("pqr", [(1, 2, 3), (6, 1, 9)])
def test_sine_eigenmode_7pt_var_axiswise(pqr):
    """Axis-wise weights (cx, cy, cz) pin which coefficient pair acts on which axis."""
    nx, ny, nz = 6, 8, 9
    p, q, r = pqr
    c0, cx, cy, cz = 0.3, 0.05, 0.12, 0.2
    shape = (nz, ny, nx)
    C = np.stack([np.full(shape, v) for v in (c0, cx, cx, cy, cy, cz, cz)])
    u0 = _sine_mode(nx, ny, nz, p, q, r)
    lam = c0 + 2 * (cx * math.cos(p * math.pi / (nx + 1)) + cy * math.cos(q * math.pi / (ny + 1))
                    + cz * math.cos(r * math.pi / (nz + 1)))
    T = 9
    uT = oracle.sweep("7pt_var", u0, T, coefs=C)
    ref = lam ** T * u0
    assert np.max(np.abs(uT - ref)) <= 1e-13 * max(np.max(np.abs(ref)), 1e-12) + 1e-15


# ------------------------------------------------------------------- invariant

@pytest.mark.parametrize("kind", ["7pt_const", "7pt_var", "25pt_var"])
def test_constant_field_invariant_bitwise(kind):
    nx, ny, nz = 11, 9, 10
    c = 0.75
    shape = (nz, ny, nx)
    u0 = np.full(shape, c)
    if kind == "7pt_const":
        kw = dict(scalars=(0.25, 0.125))
    elif kind == "7pt_var":
        kw = dict(coefs=np.stack([np.full(shape, 0.25)] + [np.full(shape, 0.125)] * 6))
    else:
        kw = dict(coefs=np.stack([np.full(shape, 0.25)] + [np.full(shape, 1.0 / 32)] * 12))
    uT = oracle.sweep(kind, u0, 6, halo=c, **kw)
    assert np.array_equal(uT, u0)
    # with a zero halo the boundary layer must drop (the halo really is read)
    uz = oracle.sweep(kind, u0, 1, halo=0.0, **kw)
    assert uz[0, 0, 0] < c and uz[nz // 2, ny // 2, nx // 2] == c


# ------------------------------------------------------- shift special cases

O7 = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]


def _shifted(up, h, di, dj, dk, shape):
    nz, ny, nx = shape
    return up[h + dk:h + dk + nz, h + dj:h + dj + ny, h + di:h + di + nx]


@pytest.mark.parametrize("m", range(7))
def test_7pt_var_single_array_is_weighted_shift(m):
    shape = (5, 6, 7)
    u0 = _rand(shape, 1)
    w = _rand(shape, 2, 0.0, 1.0)
    C = np.zeros((7,) + shape)
    C[m] = w
    halo = 0.3
    got = oracle.sweep("7pt_var", u0, 1, coefs=C, halo=halo)
    up = np.pad(u0, 1, constant_values=halo)
    di, dj, dk = O7[m]
    assert np.array_equal(got, w * _shifted(up, 1, di, dj, dk, shape))


@pytest.mark.parametrize("m", range(13))
def test_25pt_single_array_is_weighted_pair_shift(m):
    shape = (9, 10, 11)
    u0 = _rand(shape, 3)
    w = _rand(shape, 4, 0.0, 1.0)
    C = np.zeros((13,) + shape)
    C[m] = w
    halo = -0.2
    got = oracle.sweep("25pt_var", u0, 1, coefs=C, halo=halo)
    up = np.pad(u0, 4, constant_values=halo)
    if m == 0:
        ref = w * u0
    else:
        d = (m - 1) // 3 + 1
        a = (m - 1) % 3
        off = [0, 0, 0]
        off[a] = d
        plus = _shifted(up, 4, off[0], off[1], off[2], shape)
        minus = _shifted(up, 4, -off[0], -off[1], -off[2], shape)
        ref = w * (plus + minus)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("kind,nc", [("7pt_var", 7), ("25pt_var", 13)])
def test_superposition_over_coefficient_arrays(kind, nc):
    shape = (9, 9, 10)
    u0 = _rand(shape, 5)
    C = np.stack([_rand(shape, 10 + m, 0.0, 0.2) for m in range(nc)])
    full = oracle.sweep(kind, u0, 1, coefs=C)
    parts = np.zeros(shape)
    for m in range(nc):
        Cm = np.zeros_like(C)
        Cm[m] = C[m]
        parts += oracle.sweep(kind, u0, 1, coefs=Cm)
    assert np.max(np.abs(full - parts)) < 1e-14


def test_7pt_const_equals_7pt_var_with_constant_arrays():
    shape = (6, 7, 8)
    u0 = _rand(shape, 6)
    c0, c1 = 0.4, 0.1
    C = np.stack([np.full(shape, c0)] + [np.full(shape, c1)] * 6)
    a = oracle.sweep("7pt_const", u0, 4, scalars=(c0, c1))
    b = oracle.sweep("7pt_var", u0, 4, coefs=C)
    assert np.max(np.abs(a - b)) < 1e-14


# ------------------------------------------------------------- dense brute force

def _neighbour_table(kind):
    """(weight index, offset) pairs read by one point, from the stencil's definition."""
    if kind in ("7pt_const", "7pt_var"):
        return [(m, O7[m]) for m in range(7)]
    tab = [(0, (0, 0, 0))]
    for d in range(1, 5):
        for a in range(3):
            for s in (1, -1):
                off = [0, 0, 0]
                off[a] = s * d
                tab.append((3 * (d - 1) + a + 1, tuple(off)))
    return tab


def _dense_operator(kind, shape, C=None, c0=0.4, c1=0.1):
    nz, ny, nx = shape
    n = nx * ny * nz
    A = np.zeros((n, n))
    idx = lambda i, j, k: (k * ny + j) * nx + i
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                row = idx(i, j, k)
                for m, (di, dj, dk) in _neighbour_table(kind):
                    qi, qj, qk = i + di, j + dj, k + dk
                    if not (0 <= qi < nx and 0 <= qj < ny and 0 <= qk < nz):
                        continue  # zero halo contributes nothing
                    if kind == "7pt_const":
                        w = c0 if m == 0 else c1
                    else:
                        w = C[m, k, j, i]
                    A[row, idx(qi, qj, qk)] += w
    return A


@pytest.mark.parametrize("kind,shape,T", [
    ("7pt_const", (8, 8, 8), 4),
    ("7pt_var", (8, 8, 8), 3),
    ("7pt_var", (9, 7, 5), 3),
    ("25pt_var", (9, 9, 9), 2),
    ("25pt_var", (10, 9, 6), 2),
])
def test_dense_brute_force(kind, shape, T):
    u0 = _rand(shape, 21)
    nc = oracle.NCOEF[oracle.KINDS[kind]]
    C = np.stack([_rand(shape, 30 + m, 0.0, 0.15) for m in range(nc)]) if nc else None
    A = _dense_operator(kind, shape, C)
    v = u0.ravel()
    for _ in range(T):
        v = A @ v
    got = oracle.sweep(kind, u0, T, coefs=C)
    assert np.max(np.abs(got.ravel() - v)) < 1e-13
    # the transpose matches the assembled matrix's transpose
    lam = _rand(shape, 22)
    gt = oracle.step_transpose(kind, lam, coefs=C)
    assert np.max(np.abs(gt.ravel() - A.T @ lam.ravel())) < 1e-13


# ------------------------------------------------------------------- adjoint

@pytest.mark.parametrize("kind,shape", [("7pt_var", (7, 6, 5)), ("25pt_var", (9, 10, 9))])
def test_transpose_dot_product_identity(kind, shape):
    nc = oracle.NCOEF[oracle.KINDS[kind]]
    C = np.stack([_rand(shape, 40 + m, 0.0, 0.2) for m in range(nc)])
    w = _rand(shape, 50)
    lam = _rand(shape, 51)
    Aw = oracle.sweep(kind, w, 1, coefs=C)
    Atl = oracle.step_transpose(kind, lam, coefs=C)
    lhs = float(np.dot(Atl.ravel(), w.ravel()))
    rhs = float(np.dot(lam.ravel(), Aw.ravel()))
    assert abs(lhs - rhs) <= 1e-13 * max(1.0, abs(lhs))


def _loss(kind, u0, C, target, T):
    uT = oracle.sweep(kind, u0, T, coefs=C)
    return 0.5 * float(np.sum((uT - target) ** 2))


@pytest.mark.parametrize("kind,shape,T", [("7pt_var", (5, 6, 4), 4), ("25pt_var", (9, 9, 10), 2)])
def test_adjoint_matches_central_differences(kind, shape, T):
    nc = oracle.NCOEF[oracle.KINDS[kind]]
    u0 = _rand(shape, 60)
    target = _rand(shape, 61)
    C = np.stack([_rand(shape, 62 + m, 0.0, 0.15) for m in range(nc)])
    loss, gu, gc = oracle.adjoint(kind, u0, C, target, T)
    assert abs(loss - _loss(kind, u0, C, target, T)) < 1e-12 * max(1, loss)
    rng = np.random.default_rng(RNG_SEED)
    # u0: the loss is quadratic in u0, so central differences are exact up to rounding
    for _ in range(6):
        p = tuple(int(rng.integers(0, s)) for s in shape)
        h = 1e-3
        up = u0.copy(); up[p] += h
        um = u0.copy(); um[p] -= h
        fd = (_loss(kind, up, C, target, T) - _loss(kind, um, C, target, T)) / (2 * h)
        assert abs(fd - gu[p]) < 1e-9 * max(1.0, abs(fd))
    # coefficients: O(h^2) truncation
    for _ in range(8):
        m = int(rng.integers(0, nc))
        p = tuple(int(rng.integers(0, s)) for s in shape)
        h = 1e-5 * max(abs(C[(m,) + p]), 1e-3)
        Cp = C.copy(); Cp[(m,) + p] += h
        Cm = C.copy(); Cm[(m,) + p] -= h
        fd = (_loss(kind, u0, Cp, target, T) - _loss(kind, u0, Cm, target, T)) / (2 * h)
        assert abs(fd - gc[(m,) + p]) < 1e-7 * max(1.0, abs(fd))
    # one random direction over all coefficient arrays
    dC = _rand(C.shape, 99)
    h = 1e-6
    fd = (_loss(kind, u0, C + h * dC, target, T) - _loss(kind, u0, C - h * dC, target, T)) / (2 * h)
    assert abs(fd - float(np.sum(gc * dC))) < 1e-6 * max(1.0, abs(fd))


def test_adjoint_T0_is_residual():
    shape = (4, 5, 6)
    u0 = _rand(shape, 70)
    target = _rand(shape, 71)
    C = np.stack([_rand(shape, 72 + m, 0.0, 0.15) for m in range(7)])
    loss, gu, gc = oracle.adjoint("7pt_var", u0, C, target, 0)
    assert np.array_equal(gu, u0 - target)
    assert not gc.any()


# --------------------------------------------------------- point evaluation

@pytest.mark.parametrize("kind,shape,T", [
    ("7pt_const", (12, 10, 11), 5),
    ("7pt_var", (9, 12, 10), 4),
    ("25pt_var", (14, 13, 12), 2),
])
def test_points_match_full_sweep(kind, shape, T):
    nc = oracle.NCOEF[oracle.KINDS[kind]]
    u0 = _rand(shape, 80)
    C = np.stack([_rand(shape, 81 + m, 0.0, 0.15) for m in range(nc)]) if nc else None
    full = oracle.sweep(kind, u0, T, coefs=C, halo=0.1)
    nz, ny, nx = shape
    pts = [(0, 0, 0), (nx - 1, ny - 1, nz - 1), (nx // 2, 1, nz - 2), (3, ny // 2, 0)]
    got = oracle.points(kind, u0, T, pts, coefs=C, halo=0.1)
    ref = np.array([full[k, j, i] for (i, j, k) in pts])
    assert np.array_equal(got, ref)


def test_step_normalised_l2():
    a = np.ones((2, 2, 2))
    assert oracle.step_normalised_l2(a, a, 5) == 0.0
    b = a * (1 + 1e-3)
    assert abs(oracle.step_normalised_l2(b, a, 10) - 1e-4) < 1e-12
