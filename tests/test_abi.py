"""The C-ABI library builds for sm_103a, loads, and exports every function include/ftle.h declares
(no GPU needed: nothing is called that touches a device)."""
import re
import subprocess
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent


def declared_functions():
    text = (ROOT / "include" / "ftle.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(ftle_[a-z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["ftle_advect", "ftle_gradient_eig", "ftle_batch", "ftle_backward", "ftle_compute",
                 "ftle_status_string", "ftle_workspace_bytes", "ftle_compute_host"]:
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2408_02758_gb300 import ftle

    L = ftle.lib()  # builds with nvcc for sm_103a if stale
    path = ftle.library_path()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\b(ftle_[a-z0-9_]+)\b", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    assert L.ftle_version() == 1


def test_binding_covers_every_declared_symbol():
    from paper_2408_02758_gb300 import ftle

    bound = {name for name, _, _ in ftle._SIGS}
    assert set(declared_functions()) <= bound


def test_status_strings_and_host_side_validation():
    """Argument errors are caught before any device work (no GPU is touched)."""
    import ctypes

    from paper_2408_02758_gb300 import ftle

    L = ftle.lib()
    assert L.ftle_status_string(0) == b"ok"
    assert L.ftle_status_string(-3).startswith(b"workspace")
    f = ftle.ftle_flow()
    f.kind = 0
    m = ftle.ftle_mesh()
    m.dim = 3  # double gyre is 2D only
    m.n_nodes = 0
    rc = L.ftle_advect(ctypes.byref(m), ctypes.byref(f), 0.0, 1.0, 0.01, 2, None, None, 0, None, None)
    assert rc == ftle.FTLE_EINVAL
    assert b"2D" in L.ftle_last_error()
    m.dim = 2
    rc = L.ftle_advect(ctypes.byref(m), ctypes.byref(f), 0.0, 0.0, 0.01, 2, None, None, 0, None, None)
    assert rc == ftle.FTLE_EINVAL  # T = 0
    rc = L.ftle_advect(None, ctypes.byref(f), 0.0, 1.0, 0.01, 2, None, None, 0, None, None)
    assert rc == ftle.FTLE_EINVAL
    rc = L.ftle_gradient_eig(ctypes.byref(m), None, 2, 1.0, None, None, None, 0, None, None)
    assert rc == ftle.FTLE_EWORKSPACE
    rc = L.ftle_advect(ctypes.byref(m), ctypes.byref(f), 0.0, 1e12, 1e-3, 2, None, None, 0, None, None)
    assert rc == ftle.FTLE_ERANGE
    # fp32c: (hi, lo) pairs, then 32-byte gradient records at the next 256-byte boundary
    # 2D fp32c: then 7 run-boundary states (float2 [2][n] each, 256-byte aligned)
    assert L.ftle_flowmap_bytes(2, 10, 2) == 256 + 512 + 7 * 256 and L.ftle_flowmap_bytes(3, 10, 1) == 120
    assert L.ftle_flowmap_bytes(3, 10, 2) == 256 + 32 * 10
    assert L.ftle_checkpoint_bytes(2, 10, 2) == 160 and L.ftle_checkpoint_bytes(3, 10, 0) == 240
    # implicit lattice neighbours: checked with the mesh, before any device work
    m3 = ftle.ftle_mesh()
    m3.dim, m3.n_nodes, m3.coords, m3.row_ptr = 3, 24, 256, 256  # pointers never dereferenced here
    for stencil, grid, what in [(4, (2, 3, 4), b"unknown stencil"), (ftle.STENCIL_TRI, (2, 3, 4), b"does not exist"),
                                (ftle.STENCIL_KUHN, (2, 3, 5), b"lattice has 30 nodes"),
                                (ftle.STENCIL_KUHN, (1, 4, 6), b"grid[0] = 1")]:
        m3.stencil = stencil
        m3.grid[:] = grid
        assert L.ftle_gradient_eig(ctypes.byref(m3), None, 2, 1.0, None, None, None, 0, None, None) == ftle.FTLE_EINVAL
        assert what in L.ftle_last_error(), L.ftle_last_error()
    m3.dim, m3.n_nodes, m3.stencil = 2, 6, ftle.STENCIL_TRI
    m3.grid[:] = (2, 3, 2)  # the unused axis must be 1
    assert L.ftle_gradient_eig(ctypes.byref(m3), None, 2, 1.0, None, None, None, 0, None, None) == ftle.FTLE_EINVAL
    assert b"grid[2] = 2" in L.ftle_last_error()
    m3.grid[:] = (2, 3, 1)  # a valid lattice: the call goes on and stops at the NULL flowmap
    assert L.ftle_gradient_eig(ctypes.byref(m3), None, 2, 1.0, None, None, None, 0, None, None) == ftle.FTLE_EINVAL
    assert b"flowmap" in L.ftle_last_error()
    assert L.ftle_workspace_bytes(1000) >= 8000


def test_validate_mesh_host_side_errors():
    """ftle_validate_mesh refuses a NULL mesh and a missing or misaligned workspace on the host,
    before any device work."""
    import ctypes

    from paper_2408_02758_gb300 import ftle

    L = ftle.lib()
    rep = ftle.ftle_mesh_report()
    assert L.ftle_validate_mesh(None, ctypes.byref(rep), None, 0, None) == ftle.FTLE_EINVAL
    m = ftle.ftle_mesh()
    m.dim = 2
    m.n_nodes = 0
    assert L.ftle_validate_mesh(ctypes.byref(m), ctypes.byref(rep), None, 0, None) == ftle.FTLE_EWORKSPACE
    assert L.ftle_validate_mesh(ctypes.byref(m), ctypes.byref(rep), 256 + 8, 4096, None) == ftle.FTLE_EWORKSPACE


def test_options_refuse_bad_staging_and_refresh():
    """grad_staging outside {0, 1} and abc_refresh that is not a power of two in [1, 1024] are
    refused on the host (the flow and mesh are checked first, then the options)."""
    import ctypes

    from paper_2408_02758_gb300 import ftle

    L = ftle.lib()
    f = ftle.ftle_flow()
    f.kind = 1  # ABC
    m = ftle.ftle_mesh()
    m.dim = 3
    m.n_nodes = 0
    for kw in ({"grad_staging": 2}, {"abc_refresh": 3}, {"abc_refresh": 2048}):
        o = ftle.make_options(**kw)
        rc = L.ftle_advect(ctypes.byref(m), ctypes.byref(f), 0.0, 1.0, 0.01, 2, None, None, 0, ctypes.byref(o), None)
        assert rc == ftle.FTLE_EINVAL, kw
