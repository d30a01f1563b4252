"""FP64 CPU oracle for the FTLE hot path (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package.  The library itself is ``oracle.c`` (plain C, FP64, OpenMP over nodes); this module
builds it in-tree with gcc and exposes it through ctypes on numpy arrays.

Every function cites the definition it follows in ``oracle.c``'s header: RK4 flowmap, Householder-QR
least-squares gradient, cyclic-Jacobi eigenvalues of C = F^T F and of C - I, FTLE =
log1p(mu) / (2|T|), and the forward-mode parameter derivative of a weighted FTLE sum.
"""
from __future__ import annotations

import ctypes
import fcntl
import os
import subprocess
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
SRC = HERE / "oracle.c"
LIB = HERE / "liboracle.so"

DOUBLE_GYRE, ABC, LINEAR, SADDLE = 0, 1, 2, 3

_lib = None


def build(force: bool = False) -> Path:
    """Compile ``liboracle.so`` (gcc, -O2, OpenMP when available, no FP contraction)."""
    with open(HERE / ".build.lock", "w") as lk:
        fcntl.flock(lk, fcntl.LOCK_EX)
        if force or not LIB.exists() or SRC.stat().st_mtime > LIB.stat().st_mtime:
            tmp = LIB.with_suffix(".so.tmp")
            base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-shared", "-fPIC", "-o", str(tmp),
                    str(SRC), "-lm"]
            proc = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True, text=True)
            if proc.returncode != 0:  # no OpenMP runtime: serial build, same arithmetic
                proc = subprocess.run(base, capture_output=True, text=True)
            if proc.returncode != 0:
                raise RuntimeError(f"oracle build failed:\n{proc.stderr}")
            os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(str(build()))
        dp = ctypes.POINTER(ctypes.c_double)
        i32p = ctypes.POINTER(ctypes.c_int32)
        c_i64, c_d, c_i = ctypes.c_int64, ctypes.c_double, ctypes.c_int
        lib.orc_velocity.argtypes = [c_i, dp, c_i, c_d, dp, dp]
        lib.orc_velocity.restype = c_i
        lib.orc_dg_derivs.argtypes = [dp, c_d, dp, dp, dp]
        lib.orc_dg_derivs.restype = c_i
        lib.orc_advect.argtypes = [c_i, dp, c_i, c_i64, dp, c_d, c_d, c_d, dp]
        lib.orc_advect.restype = ctypes.c_long
        lib.orc_advect_tangent.argtypes = [dp, c_i64, dp, c_d, c_d, c_d, dp, dp]
        lib.orc_advect_tangent.restype = ctypes.c_long
        lib.orc_jacobi.argtypes = [c_i, dp, dp, dp]
        lib.orc_jacobi.restype = c_i
        lib.orc_ftle.argtypes = [c_i, c_i64, dp, i32p, i32p, dp, c_d, dp, dp, dp, dp, i32p]
        lib.orc_ftle.restype = c_i64
        lib.orc_param_grad.argtypes = [c_i64, dp, i32p, i32p, dp, c_d, c_d, c_d, dp, dp, dp]
        lib.orc_param_grad.restype = c_i
        lib.orc_num_threads.argtypes = []
        lib.orc_num_threads.restype = c_i
        _lib = lib
    return _lib


def _d(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _params(p) -> np.ndarray:
    out = np.zeros(12)
    p = np.asarray(p, dtype=np.float64).reshape(-1)
    out[: p.size] = p
    return out


def num_threads() -> int:
    return int(_load().orc_num_threads())


def velocity(kind: int, params, t: float, x) -> np.ndarray:
    """Velocity u(x, t) of one point (see the field definitions in oracle.c)."""
    x = _f64(x)
    u = np.zeros_like(x)
    if _load().orc_velocity(kind, _d(_params(params)), x.size, t, _d(x), _d(u)) != 0:
        raise ValueError("bad flow kind / dimension")
    return u


def dg_derivs(params, t: float, x):
    """Double gyre Jacobian du/dx (2x2) and du/d(A, eps, omega) (2x3) at one point."""
    x = _f64(x)
    J = np.zeros(4)
    P = np.zeros(6)
    _load().orc_dg_derivs(_d(_params(params)), t, _d(x), _d(J), _d(P))
    return J.reshape(2, 2), P.reshape(2, 3)


def advect(kind: int, params, x0: np.ndarray, T: float, dt: float, t0: float = 0.0) -> np.ndarray:
    """RK4 flowmap of every node; ``x0`` SoA [dim][n] -> phi SoA [dim][n] (FP64)."""
    x0 = _f64(x0)
    dim, n = x0.shape
    phi = np.empty_like(x0)
    ns = _load().orc_advect(kind, _d(_params(params)), dim, n, _d(x0), t0, T, dt, _d(phi))
    if ns < 0:
        raise ValueError("bad advection arguments")
    return phi


def advect_tangent(params, x0: np.ndarray, T: float, dt: float, t0: float = 0.0):
    """Double gyre flowmap and d phi / d(A, eps, omega): returns (phi [2][n], dphi [3][2][n])."""
    x0 = _f64(x0)
    n = x0.shape[1]
    phi = np.empty_like(x0)
    dphi = np.empty((3, 2, n))
    if _load().orc_advect_tangent(_d(_params(params)), n, _d(x0), t0, T, dt, _d(phi), _d(dphi)) < 0:
        raise ValueError("bad advection arguments")
    return phi, dphi


def jacobi(A: np.ndarray):
    """Cyclic Jacobi eigen-decomposition of a symmetric 2x2 / 3x3 matrix: (w, V)."""
    A = _f64(A)
    d = A.shape[0]
    w = np.zeros(d)
    V = np.zeros(d * d)
    _load().orc_jacobi(d, _d(A), _d(w), _d(V))
    return w, V.reshape(d, d)


def ftle_field(x: np.ndarray, row_ptr: np.ndarray, col_idx: np.ndarray, phi: np.ndarray, T: float,
               want_F: bool = False) -> dict:
    """Per-row FTLE kernel; returns dict with ftle, lam, mu, flags (and F if asked)."""
    x = _f64(x)
    phi = _f64(phi)
    dim, n = x.shape
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
    ftle = np.empty(n)
    lam = np.empty(n)
    mu = np.empty(n)
    flags = np.empty(n, dtype=np.int32)
    F = np.empty((n, dim, dim)) if want_F else None
    ndeg = _load().orc_ftle(dim, n, _d(x), _i(row_ptr), _i(col_idx), _d(phi), T, _d(ftle), _d(lam),
                            _d(mu), _d(F), _i(flags))
    if ndeg < 0:
        raise ValueError("bad FTLE arguments")
    out = {"ftle": ftle, "lam": lam, "mu": mu, "flags": flags, "n_degenerate": int(ndeg)}
    if want_F:
        out["F"] = F
    return out


def ftle(kind: int, params, x0: np.ndarray, row_ptr, col_idx, T: float, dt: float, t0: float = 0.0,
         want_F: bool = False) -> dict:
    """Whole path on every node: RK4 flowmap, then the FTLE kernel."""
    phi = advect(kind, params, x0, T, dt, t0)
    out = ftle_field(x0, row_ptr, col_idx, phi, T, want_F)
    out["phi"] = phi
    return out


def param_grad(x0: np.ndarray, row_ptr, col_idx, params, T: float, dt: float, w: np.ndarray,
               t0: float = 0.0):
    """d(sum_i w_i FTLE_i)/d(A, eps, omega) for the double gyre, forward mode.  Returns (grad[3], ftle)."""
    x0 = _f64(x0)
    n = x0.shape[1]
    w = _f64(w)
    grad = np.zeros(3)
    ft = np.empty(n)
    rc = _load().orc_param_grad(n, _d(x0), _i(np.ascontiguousarray(row_ptr, dtype=np.int32)),
                                _i(np.ascontiguousarray(col_idx, dtype=np.int32)), _d(_params(params)), t0,
                                T, dt, _d(w), _d(grad), _d(ft))
    if rc < 0:
        raise ValueError("bad gradient arguments")
    if rc == 1:
        raise ValueError("a weighted node has a degenerate neighbourhood")
    return grad, ft


def submesh(coords: np.ndarray, row_ptr: np.ndarray, col_idx: np.ndarray, rows: np.ndarray):
    """Restrict a mesh to target rows and their neighbours.

    Returns (sub_coords, sub_row_ptr, sub_col_idx, n_rows): the first ``n_rows`` local nodes are
    ``rows`` (in order) and carry their full neighbour lists; the rest are the neighbours, with
    empty rows.  Used to evaluate the oracle on a sample of a mesh too large to run whole.
    """
    rows = np.asarray(rows, dtype=np.int64)
    starts = row_ptr[rows].astype(np.int64)
    ends = row_ptr[rows + 1].astype(np.int64)
    nb = np.concatenate([col_idx[s:e] for s, e in zip(starts, ends)]) if len(rows) else np.zeros(0, np.int64)
    extra = np.setdiff1d(np.unique(nb.astype(np.int64)), rows)
    nodes = np.concatenate([rows, extra])
    local = {int(g): l for l, g in enumerate(nodes)}
    sub_ci = np.array([local[int(g)] for g in nb], dtype=np.int32)
    counts = np.zeros(len(nodes), dtype=np.int64)
    counts[: len(rows)] = ends - starts
    sub_rp = np.zeros(len(nodes) + 1, dtype=np.int32)
    sub_rp[1:] = np.cumsum(counts)
    return np.ascontiguousarray(coords[:, nodes]), sub_rp, sub_ci, len(rows)


def ftle_sample(kind: int, params, coords, row_ptr, col_idx, rows, T: float, dt: float,
                t0: float = 0.0) -> dict:
    """Oracle FTLE (and lambda_max, mu) of the sampled ``rows`` of a mesh."""
    sc, srp, sci, m = submesh(np.asarray(coords), np.asarray(row_ptr), np.asarray(col_idx), rows)
    out = ftle(kind, params, sc.astype(np.float64), srp, sci, T, dt, t0)
    return {k: (v[:m] if isinstance(v, np.ndarray) and v.ndim == 1 else v) for k, v in out.items()}
