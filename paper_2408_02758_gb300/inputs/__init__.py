"""Seeded synthetic inputs: meshes with CSR neighbour lists, flow parameters, workload presets.

This module holds none of the FTLE arithmetic; the CUDA path and the FP64 oracle both read
what it produces.  Meshes come from ``meshgen.c`` (lattice coordinates, SplitMix64 jitter,
stencil neighbour lists); the presets below give the synthetic workloads the paper's method is
measured on (double gyre on 2D meshes, ABC flow on a 3D tetrahedral mesh, a batch of
uneven double-gyre instances, and the region-mean gradient problem).

Flow parameter layout (``FlowSpec.params``, 12 doubles; the same layout the C-ABI takes):
  DOUBLE_GYRE: [A, eps, omega]
  ABC:         [A, B, C]
  LINEAR:      velocity u = M x, M row-major d x d in params[0 : d*d]
  SADDLE:      no parameters; u = (x, -y) in 2D and (x, -y, 0) in 3D
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass, field

import numpy as np

from .. import _build

AXIS, TRI, KUHN = 0, 1, 2
STENCIL_NAMES = {"axis": AXIS, "tri": TRI, "kuhn": KUHN}

DOUBLE_GYRE, ABC, LINEAR, SADDLE = 0, 1, 2, 3

BASE_SEED = 240802758

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build_inputs()
        lib = ctypes.CDLL(str(path))
        i64p = ctypes.POINTER(ctypes.c_int64)
        dp = ctypes.POINTER(ctypes.c_double)
        i32p = ctypes.POINTER(ctypes.c_int32)
        lib.ftlein_coords.argtypes = [ctypes.c_int, i64p, dp, dp, ctypes.c_double, ctypes.c_uint64, dp]
        lib.ftlein_coords.restype = ctypes.c_int
        lib.ftlein_nnz.argtypes = [ctypes.c_int, i64p, ctypes.c_int]
        lib.ftlein_nnz.restype = ctypes.c_int64
        lib.ftlein_csr.argtypes = [ctypes.c_int, i64p, ctypes.c_int, i32p, i32p]
        lib.ftlein_csr.restype = ctypes.c_int64
        lib.ftlein_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        lib.ftlein_uniform.restype = ctypes.c_double
        _lib = lib
    return _lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def uniform(seed: int, k: int) -> float:
    """Draw ``k`` of the counter-based SplitMix64 stream ``seed`` as a double in [0, 1)."""
    return float(_load().ftlein_uniform(seed, k))


@dataclass
class Mesh:
    """Nodes (SoA ``coords[dim][N]``) and a symmetric CSR neighbour list (int32)."""

    dim: int
    shape: tuple
    coords: np.ndarray
    row_ptr: np.ndarray
    col_idx: np.ndarray
    lo: tuple = ()
    hi: tuple = ()
    meta: dict = field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        return int(self.coords.shape[1])

    @property
    def nnz(self) -> int:
        return int(self.col_idx.shape[0])


def lattice_coords(shape, lo, hi, jitter: float = 0.0, seed: int = BASE_SEED) -> np.ndarray:
    dim = len(shape)
    n = np.asarray(shape, dtype=np.int64)
    N = int(np.prod(n))
    out = np.empty((dim, N), dtype=np.float64)
    lo_a = np.asarray(lo, dtype=np.float64)
    hi_a = np.asarray(hi, dtype=np.float64)
    rc = _load().ftlein_coords(dim, _ptr(n, ctypes.c_int64), _ptr(lo_a, ctypes.c_double),
                               _ptr(hi_a, ctypes.c_double), float(jitter), int(seed) & (2**64 - 1),
                               _ptr(out, ctypes.c_double))
    if rc != 0:
        raise ValueError(f"bad lattice arguments shape={shape} lo={lo} hi={hi}")
    return out


def lattice_csr(shape, stencil: int):
    dim = len(shape)
    n = np.asarray(shape, dtype=np.int64)
    N = int(np.prod(n))
    lib = _load()
    nnz = lib.ftlein_nnz(dim, _ptr(n, ctypes.c_int64), stencil)
    if nnz < 0:
        raise ValueError(f"bad stencil {stencil} for dim {dim} or nnz beyond int32")
    row_ptr = np.empty(N + 1, dtype=np.int32)
    col_idx = np.empty(nnz, dtype=np.int32)
    got = lib.ftlein_csr(dim, _ptr(n, ctypes.c_int64), stencil, _ptr(row_ptr, ctypes.c_int32),
                         _ptr(col_idx, ctypes.c_int32))
    if got != nnz:
        raise RuntimeError("CSR construction failed")
    return row_ptr, col_idx


def lattice_elements(shape, stencil: int) -> np.ndarray:
    """Element connectivity (int32 [n_elem, verts]) of the lattice meshes whose mesh edges the TRI
    and KUHN stencils list: two triangles per cell split along the (i,j)-(i+1,j+1) diagonal, or the
    six Kuhn tetrahedra 0 -> e_a -> e_a + e_b -> (1,1,1) of each hex."""
    if stencil == TRI:
        nx, ny = shape
        i, j = np.meshgrid(np.arange(nx - 1), np.arange(ny - 1), indexing="xy")
        v00 = (i + nx * j).ravel()
        v10, v11, v01 = v00 + 1, v00 + 1 + nx, v00 + nx
        tri = np.concatenate([np.stack([v00, v10, v11], 1), np.stack([v00, v11, v01], 1)])
        return np.ascontiguousarray(tri, dtype=np.int32)
    if stencil == KUHN:
        nx, ny, nz = shape
        i, j, k = np.meshgrid(np.arange(nx - 1), np.arange(ny - 1), np.arange(nz - 1), indexing="ij")
        c = (i + nx * (j + ny * k)).ravel()
        e = [1, nx, nx * ny]
        out = []
        for a, b, cc in [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]:
            out.append(np.stack([c, c + e[a], c + e[a] + e[b], c + e[a] + e[b] + e[cc]], 1))
        return np.ascontiguousarray(np.concatenate(out), dtype=np.int32)
    raise ValueError("element lists exist for the TRI and KUHN stencils")


def make_mesh(shape, lo, hi, stencil: int, jitter: float = 0.0, seed: int = BASE_SEED,
              coord_dtype=np.float32) -> Mesh:
    """Lattice mesh with jittered nodes; coordinates rounded once to ``coord_dtype``.

    The rounded coordinates are the exact inputs of every consumer (the CUDA path and the
    oracle alike); nothing downstream re-derives them in another precision.
    """
    c = lattice_coords(shape, lo, hi, jitter, seed).astype(coord_dtype)
    rp, ci = lattice_csr(shape, stencil)
    return Mesh(dim=len(shape), shape=tuple(int(s) for s in shape), coords=np.ascontiguousarray(c),
                row_ptr=rp, col_idx=ci, lo=tuple(lo), hi=tuple(hi),
                meta={"stencil": stencil, "jitter": jitter, "seed": seed})


def mesh_from_arrays(coords: np.ndarray, row_ptr: np.ndarray, col_idx: np.ndarray) -> Mesh:
    coords = np.ascontiguousarray(coords)
    return Mesh(dim=coords.shape[0], shape=(coords.shape[1],), coords=coords,
                row_ptr=np.ascontiguousarray(row_ptr, dtype=np.int32),
                col_idx=np.ascontiguousarray(col_idx, dtype=np.int32))


@dataclass
class FlowSpec:
    kind: int
    params: np.ndarray  # float64[12]

    @staticmethod
    def double_gyre(A=0.1, eps=0.25, omega=2 * math.pi / 10):
        p = np.zeros(12)
        p[:3] = (A, eps, omega)
        return FlowSpec(DOUBLE_GYRE, p)

    @staticmethod
    def abc(A=math.sqrt(3.0), B=math.sqrt(2.0), C=1.0):
        p = np.zeros(12)
        p[:3] = (A, B, C)
        return FlowSpec(ABC, p)

    @staticmethod
    def linear(M):
        M = np.asarray(M, dtype=np.float64)
        p = np.zeros(12)
        p[: M.size] = M.reshape(-1)
        return FlowSpec(LINEAR, p)

    @staticmethod
    def saddle():
        return FlowSpec(SADDLE, np.zeros(12))


@dataclass
class Workload:
    """One FTLE problem: mesh, flow, horizon and step, and the arithmetic mode it runs in."""

    name: str
    mesh: Mesh
    flow: FlowSpec
    T: float
    dt: float
    precision: str  # "fp64" | "fp32" | "fp32c"
    t0: float = 0.0
    extra: dict = field(default_factory=dict)

    @property
    def n_steps(self) -> int:
        return int(round(abs(self.T) / self.dt))


PRESET_NAMES = ["dg2d_structured_256x128", "dg2d_tri_2048x1024", "abc3d_kuhn_256", "dg2d_batched_64",
                "dg2d_tri_1024x512_grad"]


def preset(index: int, scale: float = 1.0) -> Workload:
    """The five synthetic workloads (index 0..4).  ``scale`` < 1 shrinks each lattice axis
    (for tests that need the same structure at a size the oracle finishes quickly)."""
    seed = BASE_SEED + index

    def sz(n, lo=4):
        return max(lo, int(round(n * scale)))

    if index == 0:
        shape = (sz(256), sz(128))
        m = make_mesh(shape, (0.0, 0.0), (2.0, 1.0), AXIS, 0.0, seed, coord_dtype=np.float64)
        return Workload(PRESET_NAMES[0], m, FlowSpec.double_gyre(), 10.0, 0.01, "fp64")
    if index == 1:
        shape = (sz(2048), sz(1024))
        m = make_mesh(shape, (0.0, 0.0), (2.0, 1.0), TRI, 0.3, seed)
        return Workload(PRESET_NAMES[1], m, FlowSpec.double_gyre(), 15.0, 0.01, "fp32c")
    if index == 2:
        shape = (sz(256),) * 3
        two_pi = 2 * math.pi
        m = make_mesh(shape, (0.0,) * 3, (two_pi,) * 3, KUHN, 0.25, seed)
        return Workload(PRESET_NAMES[2], m, FlowSpec.abc(), 5.0, 0.01, "fp32c")
    if index == 4:
        shape = (sz(1024), sz(512))
        m = make_mesh(shape, (0.0, 0.0), (2.0, 1.0), TRI, 0.3, seed)
        x0 = m.coords[0].astype(np.float64)
        region = ((x0 >= 0.5) & (x0 <= 1.5)).astype(np.float64)
        w = region / max(region.sum(), 1.0)
        return Workload(PRESET_NAMES[4], m, FlowSpec.double_gyre(), 15.0, 0.01, "fp32c",
                        extra={"weights": w, "ckpt_every": 50})
    raise ValueError("preset 3 is a batch: use batched_preset()")


def batched_preset(n_inst: int = 64, scale: float = 1.0, seed: int = BASE_SEED + 3):
    """Uneven batch of double-gyre instances on structured 4-neighbour grids.

    Instance i takes draws 4i..4i+3 of the stream: size exponent k in {0..4}
    (nx = 64 * 2^k, ny = nx / 2), eps ~ U[0, 0.5], omega ~ U[pi/10, pi/2], T in {5,10,15,20};
    A = 0.1 and dt = 0.01 throughout.
    """
    out = []
    for i in range(n_inst):
        u = [uniform(seed, 4 * i + r) for r in range(4)]
        k = min(4, int(u[0] * 5))
        nx = 64 * 2 ** k
        nx = max(8, int(round(nx * scale)))
        ny = max(4, nx // 2)
        eps = 0.5 * u[1]
        omega = math.pi / 10 + u[2] * (math.pi / 2 - math.pi / 10)
        T = (5.0, 10.0, 15.0, 20.0)[min(3, int(u[3] * 4))]
        m = make_mesh((nx, ny), (0.0, 0.0), (2.0, 1.0), AXIS, 0.0, seed, coord_dtype=np.float32)
        out.append(Workload(f"batch{i}_{nx}x{ny}", m, FlowSpec.double_gyre(0.1, eps, omega), T, 0.01,
                            "fp32c"))
    return out
