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


@pytest.mark.parametrize("preset,scale", [(1, 1 / 4), (2, 1 / 8)])
def test_noalloc_matches_workspace_entry_point_twice(preset, scale):
    import torch

    from paper_2408_02758_gb300 import ftle

    w = I.preset(preset, scale=scale)  # 512 x 256 triangle mesh / 32^3 tet mesh
    assert w.mesh.n_nodes <= ftle.NOALLOC_MAX_NODES
    dm = ftle.DeviceMesh.from_mesh(w.mesh)
    n = w.mesh.n_nodes
    phi = ftle.flowmap_empty(w.mesh.dim, n, "fp32c")
    ftle.ftle_advect(dm, w.flow, 0.0, w.T, w.dt, "fp32c", phi)
    ref = ftle.ftle_out_empty(n, "fp32c")
    ref_lam = torch.empty(n, dtype=torch.float64, device="cuda")
    ws = ftle.workspace_empty(ftle.ftle_workspace_bytes(n))
    ftle.ftle_gradient_eig(dm, phi, "fp32c", w.T, ref, ref_lam, ws)
    torch.cuda.synchronize()
    r = ref.double().cpu().numpy()
    rl = ref_lam.cpu().numpy()
    for call in range(2):
        out = torch.full((n,), 123.0, dtype=torch.float32, device="cuda")
        lam = torch.full((n,), 123.0, dtype=torch.float64, device="cuda")
        ftle.ftle_gradient_eig_noalloc(dm, phi, "fp32c", w.T, out, lam)
        torch.cuda.synchronize()
        g = out.double().cpu().numpy()
        rep = compare(g, r, rl)
        assert rep["ok"], (call, rep)
        assert np.array_equal(np.isnan(g), np.isnan(r))
        assert np.allclose(lam.cpu().numpy(), rl, rtol=1e-12, atol=0, equal_nan=True)


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
