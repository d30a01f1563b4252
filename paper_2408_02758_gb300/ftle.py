"""Python binding of libftle.so (``include/ftle.h``): the same entry points, argument marshalling only.

Device memory and streams come from PyTorch; every step of the path runs in the library's CUDA
kernels.  There is no CPU fallback: if the library cannot be built or loaded, or a call fails, an
exception is raised.

Typical use::

    from paper_2408_02758_gb300 import ftle, inputs
    w = inputs.preset(1)                       # 2048 x 1024 jittered triangle mesh, double gyre
    dm = ftle.DeviceMesh.from_mesh(w.mesh)     # coords / CSR to the GPU
    out = ftle.compute(dm, w.flow, w.T, w.dt, "fp32c")   # FTLE field (torch tensor on the GPU)
"""
from __future__ import annotations

import ctypes
from ctypes import POINTER, Structure, c_char_p, c_double, c_int, c_int32, c_int64, c_size_t, c_uint64, c_void_p

import numpy as np

from . import _build

PREC = {"fp64": 0, "fp32": 1, "fp32c": 2}
FTLE_OK, FTLE_EINVAL, FTLE_ECUDA, FTLE_EWORKSPACE, FTLE_EUNSUPPORTED, FTLE_ERANGE, FTLE_ENOMEM = 0, -1, -2, -3, -4, -5, -6
STENCIL_NONE, STENCIL_AXIS, STENCIL_TRI, STENCIL_KUHN = 0, 1, 2, 3  # ftle_stencil


class ftle_mesh(Structure):
    _fields_ = [("dim", c_int32), ("coord_fp64", c_int32), ("n_nodes", c_int64), ("nnz", c_int64),
                ("coords", c_void_p), ("row_ptr", c_void_p), ("col_idx", c_void_p), ("ell_width", c_int32),
                ("reserved", c_int32), ("ell_idx", c_void_p), ("stencil", c_int32), ("grid", c_int32 * 3)]


class ftle_flow(Structure):
    _fields_ = [("kind", c_int32), ("reserved", c_int32), ("p", c_double * 12)]


class ftle_counters(Structure):
    _fields_ = [("n_flagged", c_uint64), ("n_degenerate", c_uint64), ("n_readvected", c_uint64),
                ("reserved", c_uint64 * 4), ("n_wait_timeouts", c_uint64)]


class ftle_rotation_info(Structure):
    _fields_ = [("unchecked", c_int32), ("carried", c_int32), ("angle_bound", c_double), ("diff_bound", c_double),
                ("angle_limit", c_double), ("diff_limit", c_double)]


class ftle_options(Structure):
    _fields_ = [("refine_kappa", c_double), ("advect_block", c_int32), ("advect_blocks_per_sm", c_int32),
                ("grad_block", c_int32), ("grad_tile", c_int32), ("refine_lanes", c_int32),
                ("defer_fp64", c_int32), ("validate_mesh", c_int32), ("grad_staging", c_int32),
                ("abc_refresh", c_int32)]


class ftle_mesh_report(Structure):
    _fields_ = [("bad_row_ptr", c_int64), ("bad_col_idx", c_int64), ("bad_ell_idx", c_int64),
                ("first_bad_row", c_int64), ("first_bad_col", c_int64), ("first_bad_ell", c_int64)]


class FTLEError(RuntimeError):
    def __init__(self, fn: str, status: int, msg: str):
        super().__init__(f"{fn} failed with status {status}: {msg}")
        self.status = status


_LIB = None

# (name, restype, argtypes) of every entry point in include/ftle.h
_SIGS = [
    ("ftle_version", c_int, []),
    ("ftle_last_error", c_char_p, []),
    ("ftle_status_string", c_char_p, [c_int]),
    ("ftle_rotation_bounds", c_int, [POINTER(ftle_flow), c_double, POINTER(ftle_rotation_info)]),
    ("ftle_flowmap_bytes", c_size_t, [c_int32, c_int64, c_int32]),
    ("ftle_checkpoint_bytes", c_size_t, [c_int32, c_int64, c_int32]),
    ("ftle_workspace_bytes", c_size_t, [c_int64]),
    ("ftle_advect", c_int, [POINTER(ftle_mesh), POINTER(ftle_flow), c_double, c_double, c_double, c_int32,
                            c_void_p, c_void_p, c_int32, POINTER(ftle_options), c_void_p]),
    ("ftle_gradient_eig", c_int, [POINTER(ftle_mesh), c_void_p, c_int32, c_double, c_void_p, c_void_p,
                                  c_void_p, c_size_t, POINTER(ftle_options), c_void_p]),
    ("ftle_refine", c_int, [POINTER(ftle_mesh), POINTER(ftle_flow), c_double, c_double, c_double, c_int32,
                            c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, POINTER(ftle_options), c_void_p]),
    ("ftle_compute", c_int, [POINTER(ftle_mesh), POINTER(ftle_flow), c_double, c_double, c_double, c_int32,
                             c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, POINTER(ftle_options), c_void_p]),
    ("ftle_host_workspace_bytes", c_size_t, [c_int32, c_int64, c_int64, c_int32]),
    ("ftle_compute_host", c_int, [c_int32, c_int64, c_int64, c_void_p, c_void_p, c_void_p, POINTER(ftle_flow),
                                  c_double, c_double, c_double, c_int32, c_void_p, c_void_p, c_size_t,
                                  POINTER(ftle_options), c_void_p]),
    ("ftle_read_counters", c_int, [c_void_p, POINTER(ftle_counters), c_void_p]),
    ("ftle_validate_mesh", c_int, [POINTER(ftle_mesh), POINTER(ftle_mesh_report), c_void_p, c_size_t, c_void_p]),
    ("ftle_ell_from_csr", c_int, [POINTER(ftle_mesh), c_int32, c_void_p, c_void_p]),
    ("ftle_csr_workspace_bytes", c_size_t, [c_int64, c_int32]),
    ("ftle_csr_from_elements", c_int, [c_int64, c_int64, c_int32, c_void_p, c_int32, c_void_p, c_void_p, c_int64,
                                       POINTER(c_int64), c_void_p, c_size_t, c_void_p]),
    ("ftle_gradient_eig_noalloc", c_int, [POINTER(ftle_mesh), c_void_p, c_int32, c_double, c_void_p, c_void_p,
                                          POINTER(ftle_options), c_void_p]),
    ("ftle_batch_workspace_bytes", c_size_t, [c_int32, POINTER(ftle_mesh), c_int32]),
    ("ftle_batch", c_int, [c_int32, POINTER(ftle_mesh), POINTER(ftle_flow), POINTER(c_double), c_double, c_int32,
                           POINTER(c_void_p), c_void_p, c_size_t, POINTER(ftle_options), c_void_p]),
    ("ftle_batch_plan_create", c_int, [c_int32, POINTER(ftle_mesh), POINTER(ftle_flow), POINTER(c_double),
                                       c_double, c_int32, POINTER(c_void_p), c_void_p, c_size_t,
                                       POINTER(ftle_options), c_void_p, POINTER(c_void_p)]),
    ("ftle_batch_plan_launch", c_int, [c_void_p, c_void_p]),
    ("ftle_batch_plan_destroy", c_int, [c_void_p]),
    ("ftle_backward_workspace_bytes", c_size_t, [c_int64, c_int32]),
    ("ftle_backward", c_int, [POINTER(ftle_mesh), POINTER(ftle_flow), c_double, c_double, c_double, c_int32,
                              c_void_p, c_void_p, c_int32, c_void_p, c_void_p, c_void_p, c_size_t,
                              POINTER(ftle_options), c_void_p]),
]


def lib():
    """Load (building first if its sources changed) libftle.so; raise if that is impossible."""
    global _LIB
    if _LIB is None:
        path = _build.build_ftle()
        L = ctypes.CDLL(str(path))
        for name, res, args in _SIGS:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


def library_path() -> str:
    return str(_build.LIBFTLE)


def _check(fn: str, rc: int):
    if rc != FTLE_OK:
        msg = lib().ftle_last_error().decode(errors="replace")
        raise FTLEError(fn, rc, msg)


def _ptr(t) -> int | None:
    if t is None:
        return None
    return int(t.data_ptr())


def _stream(stream):
    import torch

    if stream is None:
        return int(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _prec(p) -> int:
    return PREC[p] if isinstance(p, str) else int(p)


def make_flow(flow) -> ftle_flow:
    """ftle_flow from an ``inputs.FlowSpec`` (or anything with ``kind`` and ``params``)."""
    f = ftle_flow()
    f.kind = int(flow.kind)
    f.reserved = 0
    p = np.zeros(12)
    src = np.asarray(flow.params, dtype=np.float64).reshape(-1)
    p[: src.size] = src
    for q in range(12):
        f.p[q] = float(p[q])
    return f


def make_options(refine_kappa: float = 0.0, advect_block: int = 0, advect_blocks_per_sm: int = 0,
                 grad_block: int = 0, grad_tile: int = 0, refine_lanes: int = 0,
                 defer_fp64: bool = False, validate_mesh: bool = False, grad_staging: int = 0,
                 abc_refresh: int = 0) -> ftle_options:
    o = ftle_options()
    o.abc_refresh = abc_refresh
    o.grad_staging = grad_staging
    o.refine_lanes = refine_lanes
    o.defer_fp64 = int(bool(defer_fp64))
    o.validate_mesh = int(bool(validate_mesh))
    o.refine_kappa = refine_kappa
    o.advect_block = advect_block
    o.advect_blocks_per_sm = advect_blocks_per_sm
    o.grad_block = grad_block
    o.grad_tile = grad_tile
    return o


class DeviceMesh:
    """Mesh arrays resident on the GPU plus the ``ftle_mesh`` descriptor that points at them."""

    def __init__(self, coords, row_ptr, col_idx):
        import torch

        assert coords.is_cuda and row_ptr.is_cuda and col_idx.is_cuda
        assert coords.dtype in (torch.float32, torch.float64)
        assert row_ptr.dtype == torch.int32 and col_idx.dtype == torch.int32
        self.coords = coords.contiguous()
        self.row_ptr = row_ptr.contiguous()
        self.col_idx = col_idx.contiguous()
        d = ftle_mesh()
        d.dim = int(self.coords.shape[0])
        d.coord_fp64 = 1 if self.coords.dtype == torch.float64 else 0
        d.n_nodes = int(self.coords.shape[1])
        d.nnz = int(self.col_idx.numel())
        d.coords = _ptr(self.coords)
        d.row_ptr = _ptr(self.row_ptr)
        d.col_idx = _ptr(self.col_idx) if d.nnz else None
        self.desc = d

    @staticmethod
    def from_mesh(mesh, device="cuda"):
        import torch

        return DeviceMesh(torch.from_numpy(np.ascontiguousarray(mesh.coords)).to(device),
                          torch.from_numpy(mesh.row_ptr).to(device), torch.from_numpy(mesh.col_idx).to(device))

    def attach_ell(self, width: int | None = None, stream=None):
        """Build the fixed-width (-1 padded) neighbour list on the device and let the float gradient
        kernel use it.  width defaults to the largest row length."""
        import torch

        if width is None:
            width = int((self.row_ptr[1:] - self.row_ptr[:-1]).max().item()) if self.n_nodes else 1
        self.ell = torch.empty((width, self.n_nodes), dtype=torch.int32, device=self.coords.device)
        _check("ftle_ell_from_csr", lib().ftle_ell_from_csr(ctypes.byref(self.desc), width, _ptr(self.ell),
                                                            _stream(stream)))
        self.desc.ell_width = width
        self.desc.ell_idx = _ptr(self.ell)
        return self

    def attach_stencil(self, stencil: int, shape):
        """Let the float gradient kernel take the neighbours implied by a structured lattice of
        `shape` nodes (x fastest) instead of reading them: stencil is STENCIL_AXIS, STENCIL_TRI or
        STENCIL_KUHN, and the CSR rows must list the same neighbours."""
        shape = tuple(int(v) for v in shape)
        self.desc.stencil = int(stencil)
        for a in range(3):
            self.desc.grid[a] = shape[a] if a < len(shape) else 1
        return self

    def detach_stencil(self):
        self.desc.stencil = STENCIL_NONE
        for a in range(3):
            self.desc.grid[a] = 0
        return self

    def detach_ell(self):
        self.desc.ell_width = 0
        self.desc.ell_idx = None
        return self

    @property
    def dim(self) -> int:
        return self.desc.dim

    @property
    def n_nodes(self) -> int:
        return self.desc.n_nodes


# ------------------------------------------------------------------------------ raw entry points


def ftle_version() -> int:
    return int(lib().ftle_version())


def ftle_rotation_bounds(flow, dt: float) -> dict:
    """Host-side bounds behind the advection's unchecked rotated steps (no device work)."""
    f = make_flow(flow)
    info = ftle_rotation_info()
    _check("ftle_rotation_bounds", lib().ftle_rotation_bounds(ctypes.byref(f), dt, ctypes.byref(info)))
    return {"unchecked": bool(info.unchecked), "carried": bool(info.carried), "angle_bound": info.angle_bound,
            "diff_bound": info.diff_bound, "angle_limit": info.angle_limit, "diff_limit": info.diff_limit}


def ftle_flowmap_bytes(dim: int, n_nodes: int, precision) -> int:
    return int(lib().ftle_flowmap_bytes(dim, n_nodes, _prec(precision)))


def ftle_workspace_bytes(n_nodes: int) -> int:
    return int(lib().ftle_workspace_bytes(n_nodes))


def ftle_advect(mesh: DeviceMesh, flow, t0: float, T: float, dt: float, precision, flowmap, checkpoints=None,
                ckpt_every: int = 0, options: ftle_options | None = None, stream=None):
    f = make_flow(flow)
    _check("ftle_advect", lib().ftle_advect(ctypes.byref(mesh.desc), ctypes.byref(f), t0, T, dt, _prec(precision),
                                            _ptr(flowmap), _ptr(checkpoints), ckpt_every,
                                            ctypes.byref(options) if options else None, _stream(stream)))


def ftle_gradient_eig(mesh: DeviceMesh, flowmap, precision, T: float, ftle_out, lambda_out, workspace,
                      options: ftle_options | None = None, stream=None):
    _check("ftle_gradient_eig",
           lib().ftle_gradient_eig(ctypes.byref(mesh.desc), _ptr(flowmap), _prec(precision), T, _ptr(ftle_out),
                                   _ptr(lambda_out), _ptr(workspace), workspace.numel() * workspace.element_size(),
                                   ctypes.byref(options) if options else None, _stream(stream)))


NOALLOC_MAX_NODES = 1048576


def ftle_gradient_eig_noalloc(mesh: DeviceMesh, flowmap, precision, T: float, ftle_out, lambda_out,
                              options: ftle_options | None = None, stream=None):
    """FTLE core without a workspace: the scratch lives in a static device array of the library
    (at most NOALLOC_MAX_NODES nodes; calls that overlap on the GPU race on it)."""
    _check("ftle_gradient_eig_noalloc",
           lib().ftle_gradient_eig_noalloc(ctypes.byref(mesh.desc), _ptr(flowmap), _prec(precision), T,
                                           _ptr(ftle_out), _ptr(lambda_out),
                                           ctypes.byref(options) if options else None, _stream(stream)))


def ftle_refine(mesh: DeviceMesh, flow, t0: float, T: float, dt: float, precision, flowmap, ftle_out, lambda_out,
                workspace, options: ftle_options | None = None, stream=None):
    f = make_flow(flow)
    _check("ftle_refine",
           lib().ftle_refine(ctypes.byref(mesh.desc), ctypes.byref(f), t0, T, dt, _prec(precision), _ptr(flowmap),
                             _ptr(ftle_out), _ptr(lambda_out), _ptr(workspace),
                             workspace.numel() * workspace.element_size(),
                             ctypes.byref(options) if options else None, _stream(stream)))


def ftle_compute(mesh: DeviceMesh, flow, t0: float, T: float, dt: float, precision, flowmap, ftle_out, lambda_out,
                 workspace, options: ftle_options | None = None, stream=None):
    f = make_flow(flow)
    _check("ftle_compute",
           lib().ftle_compute(ctypes.byref(mesh.desc), ctypes.byref(f), t0, T, dt, _prec(precision), _ptr(flowmap),
                              _ptr(ftle_out), _ptr(lambda_out), _ptr(workspace),
                              workspace.numel() * workspace.element_size(),
                              ctypes.byref(options) if options else None, _stream(stream)))


def ftle_host_workspace_bytes(dim: int, n_nodes: int, nnz: int, precision) -> int:
    return int(lib().ftle_host_workspace_bytes(dim, n_nodes, nnz, _prec(precision)))


def ftle_compute_host(coords_host, row_ptr_host, col_idx_host, flow, t0: float, T: float, dt: float, precision,
                      ftle_host, device_ws, options: ftle_options | None = None, stream=None):
    """End-to-end call on HOST (preferably pinned) torch tensors; synchronises the stream."""
    f = make_flow(flow)
    dim, n = int(coords_host.shape[0]), int(coords_host.shape[1])
    nnz = int(col_idx_host.numel())
    _check("ftle_compute_host",
           lib().ftle_compute_host(dim, n, nnz, _ptr(coords_host), _ptr(row_ptr_host), _ptr(col_idx_host),
                                   ctypes.byref(f), t0, T, dt, _prec(precision), _ptr(ftle_host), _ptr(device_ws),
                                   device_ws.numel() * device_ws.element_size(),
                                   ctypes.byref(options) if options else None, _stream(stream)))


def ftle_read_counters(workspace, stream=None) -> dict:
    c = ftle_counters()
    _check("ftle_read_counters", lib().ftle_read_counters(_ptr(workspace), ctypes.byref(c), _stream(stream)))
    return {"n_flagged": int(c.n_flagged), "n_degenerate": int(c.n_degenerate), "n_readvected": int(c.n_readvected),
            "n_wait_timeouts": int(c.n_wait_timeouts)}


def ftle_validate_mesh(mesh: DeviceMesh, workspace=None, stream=None, check: bool = True) -> dict:
    """Device pass over the mesh's neighbour indices (row_ptr, col_idx, ell_idx); returns the
    report as a dict.  With check=True a bad index raises FTLEError (FTLE_EINVAL)."""
    ws = workspace if workspace is not None else workspace_empty(256, device=mesh.coords.device)
    r = ftle_mesh_report()
    rc = lib().ftle_validate_mesh(ctypes.byref(mesh.desc), ctypes.byref(r), _ptr(ws),
                                  ws.numel() * ws.element_size(), _stream(stream))
    if check:
        _check("ftle_validate_mesh", rc)
    elif rc not in (FTLE_OK, FTLE_EINVAL):
        _check("ftle_validate_mesh", rc)
    return {k: int(getattr(r, k)) for k, _ in ftle_mesh_report._fields_} | {"status": int(rc)}


# ------------------------------------------------------------------------------ buffer helpers


def ftle_checkpoint_bytes(dim: int, n_nodes: int, precision) -> int:
    return int(lib().ftle_checkpoint_bytes(dim, n_nodes, _prec(precision)))


def flowmap_empty(dim: int, n_nodes: int, precision, device="cuda"):
    """Uninitialised flowmap buffer in the layout of ``precision``: (dim, n) float64 / float32, or
    for fp32c a flat float32 buffer holding the (hi, lo) pairs and the gradient records (see
    flowmap_pairs)."""
    import torch

    p = _prec(precision)
    if p == PREC["fp64"]:
        return torch.empty((dim, n_nodes), dtype=torch.float64, device=device)
    if p == PREC["fp32"]:
        return torch.empty((dim, n_nodes), dtype=torch.float32, device=device)
    return torch.empty(ftle_flowmap_bytes(dim, n_nodes, p) // 4, dtype=torch.float32, device=device)


def flowmap_pairs(phi, dim: int, n_nodes: int):
    """(dim, n, 2) view of the (hi, lo) pairs at the start of an fp32c flowmap buffer."""
    return phi[: dim * n_nodes * 2].view(dim, n_nodes, 2)


def workspace_empty(nbytes: int, device="cuda"):
    """Device byte buffer (torch's allocator returns 256-byte aligned blocks)."""
    import torch

    t = torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)
    assert t.data_ptr() % 256 == 0
    return t


def ftle_out_empty(n_nodes: int, precision, device="cuda"):
    import torch

    return torch.empty(n_nodes, dtype=torch.float64 if _prec(precision) == PREC["fp64"] else torch.float32,
                       device=device)


def compute(mesh: DeviceMesh, flow, T: float, dt: float, precision="fp32c", t0: float = 0.0, want_lambda=False,
            options: ftle_options | None = None, stream=None, return_all=False):
    """Whole path (advect, gradient/eigen, FP64 refinement) into fresh device tensors."""
    import torch

    phi = flowmap_empty(mesh.dim, mesh.n_nodes, precision)
    out = ftle_out_empty(mesh.n_nodes, precision)
    lam = torch.empty(mesh.n_nodes, dtype=torch.float64, device="cuda") if want_lambda else None
    ws = workspace_empty(ftle_workspace_bytes(mesh.n_nodes))
    ftle_compute(mesh, flow, t0, T, dt, precision, phi, out, lam, ws, options, stream)
    if return_all:
        return {"ftle": out, "lam": lam, "phi": phi, "workspace": ws}
    return out


# ------------------------------------------------------------------------------ batched


def _batch_arrays(meshes, flows, T, outs):
    n = len(meshes)
    if not (len(flows) == len(T) == len(outs) == n):
        raise ValueError("meshes, flows, T and outs must have the same length")
    M = (ftle_mesh * n)(*[m.desc for m in meshes])
    Fl = (ftle_flow * n)(*[make_flow(f) for f in flows])
    Ta = (c_double * n)(*[float(t) for t in T])
    Oa = (c_void_p * n)(*[_ptr(o) for o in outs])
    return n, M, Fl, Ta, Oa


def ftle_batch_workspace_bytes(meshes, precision) -> int:
    n = len(meshes)
    M = (ftle_mesh * n)(*[m.desc for m in meshes])
    return int(lib().ftle_batch_workspace_bytes(n, M, _prec(precision)))


def ftle_batch(meshes, flows, T, dt: float, precision, outs, workspace, options: ftle_options | None = None,
               stream=None):
    """FTLE of many independent problems in one launch sequence (instances share dt, precision,
    dimension and flow kind).  ``outs`` are device float tensors, one per instance."""
    n, M, Fl, Ta, Oa = _batch_arrays(meshes, flows, T, outs)
    _check("ftle_batch", lib().ftle_batch(n, M, Fl, Ta, dt, _prec(precision), Oa, _ptr(workspace),
                                          workspace.numel() * workspace.element_size(),
                                          ctypes.byref(options) if options else None, _stream(stream)))


def compute_pair(mesh: DeviceMesh, flow, T: float, dt: float, precision="fp32c", options: ftle_options | None = None,
                 stream=None):
    """Forward (horizon +|T|) and backward (-|T|) FTLE of one mesh from t = 0, as two instances of
    one batched launch sequence: ridges of the forward field mark repelling structures, ridges of
    the backward field attracting ones.  Returns (ftle_forward, ftle_backward), device float32."""
    import torch

    dev = mesh.coords.device
    outs = [torch.empty(mesh.n_nodes, dtype=torch.float32, device=dev) for _ in range(2)]
    ws = workspace_empty(ftle_batch_workspace_bytes([mesh, mesh], precision), device=dev)
    ftle_batch([mesh, mesh], [flow, flow], [abs(T), -abs(T)], dt, precision, outs, ws, options=options, stream=stream)
    return outs[0], outs[1]


class BatchPlan:
    """A batch captured once into a CUDA graph (ftle_batch_plan_create) and replayed with launch()."""

    def __init__(self, meshes, flows, T, dt: float, precision, outs, workspace,
                 options: ftle_options | None = None, stream=None):
        n, M, Fl, Ta, Oa = _batch_arrays(meshes, flows, T, outs)
        self._keep = (meshes, outs, workspace)
        h = c_void_p()
        _check("ftle_batch_plan_create",
               lib().ftle_batch_plan_create(n, M, Fl, Ta, dt, _prec(precision), Oa, _ptr(workspace),
                                            workspace.numel() * workspace.element_size(),
                                            ctypes.byref(options) if options else None, _stream(stream),
                                            ctypes.byref(h)))
        self.handle = h

    def launch(self, stream=None):
        _check("ftle_batch_plan_launch", lib().ftle_batch_plan_launch(self.handle, _stream(stream)))

    def destroy(self):
        if self.handle:
            lib().ftle_batch_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


# ------------------------------------------------------------------------------ differentiation


def ftle_backward_workspace_bytes(n_nodes: int, dim: int = 2) -> int:
    return int(lib().ftle_backward_workspace_bytes(n_nodes, dim))


def ftle_backward(mesh: DeviceMesh, flow, t0: float, T: float, dt: float, precision, flowmap, checkpoints,
                  ckpt_every: int, dL_dftle, dL_dparams, workspace, options: ftle_options | None = None,
                  stream=None):
    """d(sum_i dL_dftle[i] FTLE_i)/d(A, eps, omega) into dL_dparams (device float64 [3])."""
    f = make_flow(flow)
    _check("ftle_backward",
           lib().ftle_backward(ctypes.byref(mesh.desc), ctypes.byref(f), t0, T, dt, _prec(precision), _ptr(flowmap),
                               _ptr(checkpoints), ckpt_every, _ptr(dL_dftle), _ptr(dL_dparams), _ptr(workspace),
                               workspace.numel() * workspace.element_size(),
                               ctypes.byref(options) if options else None, _stream(stream)))


def checkpoints_empty(dim: int, n_nodes: int, n_steps: int, ckpt_every: int, precision, device="cuda"):
    """Checkpoint slots for ftle_advect: n_steps // ckpt_every + 1 flowmaps."""
    import torch

    slots = n_steps // ckpt_every + 1
    nbytes = ftle_checkpoint_bytes(dim, n_nodes, precision)
    dtype = torch.float64 if _prec(precision) == PREC["fp64"] else torch.float32
    return torch.empty((slots, nbytes // dtype.itemsize), dtype=dtype, device=device)


# ------------------------------------------------------------------------------ mesh preparation


def ftle_csr_from_elements(n_nodes: int, elems, max_row: int, nnz_cap: int | None = None, stream=None):
    """CSR neighbour lists (row_ptr, col_idx device int32 tensors) of the node adjacency of a
    device int32 element array [n_elem, verts_per_elem], built on the GPU."""
    import torch

    elems = elems.contiguous()
    n_elem, v = int(elems.shape[0]), int(elems.shape[1])
    cap = nnz_cap if nnz_cap is not None else n_elem * v * (v - 1)
    row_ptr = torch.empty(n_nodes + 1, dtype=torch.int32, device=elems.device)
    col_idx = torch.empty(max(cap, 1), dtype=torch.int32, device=elems.device)
    ws = workspace_empty(int(lib().ftle_csr_workspace_bytes(n_nodes, max_row)), device=elems.device)
    nnz = c_int64(0)
    _check("ftle_csr_from_elements",
           lib().ftle_csr_from_elements(n_nodes, n_elem, v, _ptr(elems), max_row, _ptr(row_ptr), _ptr(col_idx), cap,
                                        ctypes.byref(nnz), _ptr(ws), ws.numel(), _stream(stream)))
    return row_ptr, col_idx[: nnz.value]
