"""FP64 CPU oracle for the stencil sweeps (arXiv:1410.5561, Listings 1-3).

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package. The product path (the
CUDA library and its Python binding) never calls it.

The C source ``stencil_oracle.c`` is compiled with gcc into
``oracle/_liboracle.so`` by :func:`build` (called from ``__graft_entry__.build``).
Every function here takes and returns dense interior arrays shaped
``(nz, ny, nx)``; padding with the Dirichlet halo (width R) happens here.

Parity status: every function is pinned by ``tests/test_oracle.py`` (closed
form, invariants, shift special cases, dense brute force, transpose and
finite-difference identities, box-restricted point evaluation vs full sweep).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "stencil_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None

KINDS = {"7pt_const": 0, "7pt_var": 1, "25pt_var": 2}
RADIUS = {0: 1, 1: 1, 2: 4}
NCOEF = {0: 0, 1: 7, 2: 13}


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, OpenMP, no FP contraction)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            i = ctypes.c_int
            lib.oracle_step.argtypes = [i, i, i, i, dp, dp, dp, dp, i]
            lib.oracle_sweep.argtypes = [i, i, i, i, i, dp, dp, dp, dp, i]
            lib.oracle_step_transpose.argtypes = [i, i, i, i, dp, dp, dp, dp]
            lib.oracle_adjoint.argtypes = [i, i, i, i, i, dp, dp, dp, dp, dp, dp]
            lib.oracle_points.argtypes = [i, i, i, i, i, dp, dp, dp, i, ip, dp, i]
            for f in (lib.oracle_step, lib.oracle_sweep, lib.oracle_step_transpose,
                      lib.oracle_adjoint, lib.oracle_points):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _kind(kind) -> int:
    return KINDS[kind] if isinstance(kind, str) else int(kind)


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def pad(a: np.ndarray, h: int, value: float = 0.0) -> np.ndarray:
    """Interior (nz, ny, nx) -> padded FP64 array with a halo of width h set to value."""
    a = np.asarray(a, dtype=np.float64)
    return np.ascontiguousarray(np.pad(a, h, mode="constant", constant_values=value))


def unpad(a: np.ndarray, h: int) -> np.ndarray:
    return np.ascontiguousarray(a[h:-h, h:-h, h:-h]) if h else a


def _coef_block(k: int, coefs, shape):
    nc = NCOEF[k]
    if nc == 0:
        return None
    coefs = np.asarray(coefs, dtype=np.float64)
    assert coefs.shape == (nc,) + tuple(shape), (coefs.shape, shape)
    h = RADIUS[k]
    return np.ascontiguousarray(np.stack([pad(c, h, 0.0) for c in coefs]))


def _scalars(k: int, scalars):
    if k != 0:
        return np.zeros(2)
    return np.ascontiguousarray(np.asarray(scalars, dtype=np.float64).reshape(2))


def sweep(kind, u0, T: int, coefs=None, scalars=(0.4, 0.1), halo: float = 0.0,
          nthreads: int = 0) -> np.ndarray:
    """u_T (interior, FP64) after T Jacobi steps from interior u0 with a constant halo."""
    lib = _load()
    k = _kind(kind)
    h = RADIUS[k]
    u0 = np.asarray(u0, dtype=np.float64)
    nz, ny, nx = u0.shape
    u = pad(u0, h, halo)
    work = np.empty_like(u)
    cb = _coef_block(k, coefs, u0.shape)
    sc = _scalars(k, scalars)
    rc = lib.oracle_sweep(k, nx, ny, nz, int(T), _ptr(sc), _ptr(cb), _ptr(u), _ptr(work),
                          int(nthreads))
    if rc:
        raise RuntimeError(f"oracle_sweep failed: {rc}")
    return unpad(u, h)


def step_transpose(kind, lam, coefs=None, scalars=(0.4, 0.1)) -> np.ndarray:
    """A^T lam over the interior (interior in, interior out)."""
    lib = _load()
    k = _kind(kind)
    h = RADIUS[k]
    lam = np.asarray(lam, dtype=np.float64)
    nz, ny, nx = lam.shape
    src = pad(lam, h, 0.0)
    dst = np.empty_like(src)
    cb = _coef_block(k, coefs, lam.shape)
    sc = _scalars(k, scalars)
    rc = lib.oracle_step_transpose(k, nx, ny, nz, _ptr(sc), _ptr(cb), _ptr(src), _ptr(dst))
    if rc:
        raise RuntimeError(f"oracle_step_transpose failed: {rc}")
    return unpad(dst, h)


def adjoint(kind, u0, coefs, target, T: int, halo: float = 0.0):
    """(loss, g_u0, g_coef) for L = 0.5*||u_T - target||^2; all FP64 interior arrays."""
    lib = _load()
    k = _kind(kind)
    h = RADIUS[k]
    u0 = np.asarray(u0, dtype=np.float64)
    nz, ny, nx = u0.shape
    up = pad(u0, h, halo)
    tp = pad(target, h, 0.0)
    cb = _coef_block(k, coefs, u0.shape)
    gu = np.empty_like(up)
    gc = np.empty_like(cb)
    loss = ctypes.c_double(0.0)
    rc = lib.oracle_adjoint(k, nx, ny, nz, int(T), _ptr(cb), _ptr(up), _ptr(tp), _ptr(gu),
                            _ptr(gc), ctypes.byref(loss))
    if rc:
        raise RuntimeError(f"oracle_adjoint failed: {rc}")
    return loss.value, unpad(gu, h), np.stack([unpad(g, h) for g in gc])


def points(kind, u0, T: int, pts, coefs=None, scalars=(0.4, 0.1), halo: float = 0.0,
           nthreads: int = 0) -> np.ndarray:
    """u_T at interior points pts = [(i, j, k), ...] (FP64), without a full sweep."""
    lib = _load()
    k = _kind(kind)
    h = RADIUS[k]
    u0 = np.asarray(u0, dtype=np.float64)
    nz, ny, nx = u0.shape
    up = pad(u0, h, halo)
    cb = _coef_block(k, coefs, u0.shape)
    sc = _scalars(k, scalars)
    p = np.ascontiguousarray(np.asarray(pts, dtype=np.int32).reshape(-1, 3))
    out = np.empty(p.shape[0])
    rc = lib.oracle_points(k, nx, ny, nz, int(T), _ptr(sc), _ptr(cb), _ptr(up), p.shape[0],
                           p.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _ptr(out),
                           int(nthreads))
    if rc:
        raise RuntimeError(f"oracle_points failed: {rc}")
    return out


def step_normalised_l2(u_test, u_ref, T: int) -> float:
    """||u_test - u_ref||_2 / (||u_ref||_2 * max(T, 1)): the per-step-normalised error."""
    u_test = np.asarray(u_test, dtype=np.float64)
    u_ref = np.asarray(u_ref, dtype=np.float64)
    den = np.linalg.norm(u_ref.ravel()) * max(int(T), 1)
    num = np.linalg.norm((u_test - u_ref).ravel())
    return float(num / den) if den > 0 else float(num)


# Cache-block-size and code-balance models of Section III (Eqs. 2-5) live in the
# product package (they drive the tuner); they are pinned by tests, not here.
