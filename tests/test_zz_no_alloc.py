"""The workspace-free FTLE core (ftle_gradient_eig_noalloc) against the workspace entry point.

Callers that may not allocate device memory (a plugin whose host owns all allocations, a
component under a fixed device-memory budget, a loop that must not call cudaMalloc/cudaFree)
use the variant whose scratch is a static device array inside the library.  This file is
collected last on purpose: it runs after every other test, and also passes alone in a fresh
process.
"""
import numpy as np
import pytest

from paper_2408_02758_gb300 import inputs as I

from _parity import compare

pytestmark = pytest.mark.gpu


def _mesh_for(ftle, w, prec):
    import torch

    m = w.mesh
    coords = m.coords.astype(np.float64) if prec == "fp64" else m.coords  # FP64 mode reads double coords
    return ftle.DeviceMesh(torch.from_numpy(np.ascontiguousarray(coords)).cuda(),
                           torch.from_numpy(m.row_ptr).cuda(), torch.from_numpy(m.col_idx).cuda())


@pytest.mark.parametrize("prec", ["fp32c", "fp32", "fp64"])
@pytest.mark.parametrize("preset,scale", [(1, 1 / 4), (2, 1 / 8)])
def test_noalloc_matches_workspace_entry_point_twice(preset, scale, prec):
    """Two calls in a row give the workspace entry point's FTLE (within the parity tolerance, and
    with the same NaN nodes) and lambda_max, in every precision: FP32 and FP32C run the float
    kernel and the FP64 pass over the flag list kept in the static array, FP64 the double kernel."""
    import torch

    from paper_2408_02758_gb300 import ftle

    w = I.preset(preset, scale=scale)  # 512 x 256 triangle mesh / 32^3 tet mesh
    assert w.mesh.n_nodes <= ftle.NOALLOC_MAX_NODES
    dm = _mesh_for(ftle, w, prec)
    n = w.mesh.n_nodes
    phi = ftle.flowmap_empty(w.mesh.dim, n, prec)
    ftle.ftle_advect(dm, w.flow, 0.0, w.T, w.dt, prec, phi)
    ref = ftle.ftle_out_empty(n, prec)
    ref_lam = torch.empty(n, dtype=torch.float64, device="cuda")
    ws = ftle.workspace_empty(ftle.ftle_workspace_bytes(n))
    ftle.ftle_gradient_eig(dm, phi, prec, w.T, ref, ref_lam, ws)
    torch.cuda.synchronize()
    if prec != "fp64" and w.mesh.dim == 2:
        assert ftle.ftle_read_counters(ws)["n_flagged"] > 0  # the FP64 pass over the static list runs
    r = ref.double().cpu().numpy()
    rl = ref_lam.cpu().numpy()
    for call in range(2):
        out = torch.full((n,), 123.0, dtype=ref.dtype, device="cuda")
        lam = torch.full((n,), 123.0, dtype=torch.float64, device="cuda")
        ftle.ftle_gradient_eig_noalloc(dm, phi, prec, w.T, out, lam)
        torch.cuda.synchronize()
        g = out.double().cpu().numpy()
        rep = compare(g, r, rl)
        assert rep["ok"], (call, rep)
        assert np.array_equal(np.isnan(g), np.isnan(r))
        assert np.allclose(lam.cpu().numpy(), rl, rtol=1e-12, atol=0, equal_nan=True)


@pytest.mark.parametrize("prec", ["fp32c", "fp32"])
def test_noalloc_without_lambda_equals_workspace_entry_point_bit_for_bit(prec):
    """lambda_out = NULL on a valid call: the FTLE equals ftle_gradient_eig's bit for bit (same
    kernels, same per-node arithmetic, the flag list merely kept elsewhere)."""
    import torch

    from paper_2408_02758_gb300 import ftle

    w = I.preset(1, scale=1 / 8)
    dm = _mesh_for(ftle, w, prec)
    n = w.mesh.n_nodes
    phi = ftle.flowmap_empty(2, n, prec)
    ftle.ftle_advect(dm, w.flow, 0.0, w.T, w.dt, prec, phi)
    ref = ftle.ftle_out_empty(n, prec)
    ws = ftle.workspace_empty(ftle.ftle_workspace_bytes(n))
    ftle.ftle_gradient_eig(dm, phi, prec, w.T, ref, None, ws)
    out = torch.full((n,), 123.0, dtype=ref.dtype, device="cuda")
    ftle.ftle_gradient_eig_noalloc(dm, phi, prec, w.T, out, None)
    torch.cuda.synchronize()
    a, b = ref.cpu().numpy(), out.cpu().numpy()
    assert np.array_equal(a, b, equal_nan=True)


def test_noalloc_refuses_a_deferred_fp64_pass():
    """The deferred FP64 pass would belong to an ftle_refine on a caller workspace, which cannot
    see the flag list kept in the static array: defer_fp64 = 1 is refused on the host."""
    import torch

    from paper_2408_02758_gb300 import ftle

    w = I.preset(1, scale=1 / 64)
    dm = ftle.DeviceMesh.from_mesh(w.mesh)
    phi = ftle.flowmap_empty(2, w.mesh.n_nodes, "fp32c")
    out = ftle.ftle_out_empty(w.mesh.n_nodes, "fp32c")
    with pytest.raises(ftle.FTLEError) as e:
        ftle.ftle_gradient_eig_noalloc(dm, phi, "fp32c", 1.0, out, None, options=ftle.make_options(defer_fp64=True))
    assert e.value.status == ftle.FTLE_EINVAL
    torch.cuda.synchronize()


def test_noalloc_rejects_meshes_beyond_its_static_limit():
    import torch

    from paper_2408_02758_gb300 import ftle

    w = I.preset(1, scale=1 / 64)
    dm = ftle.DeviceMesh.from_mesh(w.mesh)
    phi = ftle.flowmap_empty(2, w.mesh.n_nodes, "fp32c")
    out = ftle.ftle_out_empty(w.mesh.n_nodes, "fp32c")
    dm.desc.n_nodes = ftle.NOALLOC_MAX_NODES + 1  # checked on the host before any launch
    with pytest.raises(ftle.FTLEError) as e:
        ftle.ftle_gradient_eig_noalloc(dm, phi, "fp32c", 1.0, out, None)
    assert e.value.status == ftle.FTLE_ERANGE
    assert "static scratch limit" in str(e.value)
    torch.cuda.synchronize()
