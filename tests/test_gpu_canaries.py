"""Every buffer a call writes sits between two guard regions filled with a known byte pattern:
after the call the guards must be untouched, so no kernel writes past the sizes the C-ABI
declares (flowmap, checkpoints, FTLE and lambda outputs, workspaces, the parameter gradient),
on meshes whose node counts leave ragged tails for every tile and vector width.  Together with
the mesh validation pass this stands in for a memory checker, which is not run here."""
import numpy as np
import pytest

from paper_2408_02758_gb300 import inputs as I

pytestmark = pytest.mark.gpu

GUARD = 4096      # bytes on each side (a multiple of 256, so the buffer keeps the alignment rules)
PATTERN = 0xA5


@pytest.fixture(scope="module")
def F():
    from paper_2408_02758_gb300 import ftle

    ftle.lib()
    return ftle


class Guarded:
    """A device (or pinned host) byte buffer with guard regions around the part handed out."""

    def __init__(self, nbytes, device="cuda"):
        import torch

        self.n = int(nbytes)
        size = GUARD + ((self.n + 255) // 256) * 256 + GUARD
        self.buf = torch.full((size,), PATTERN, dtype=torch.uint8, device=device if device != "pinned" else "cpu")
        if device == "pinned":
            self.buf = self.buf.pin_memory()
        self.tail_start = GUARD + self.n

    def view(self, dtype):
        return self.buf[GUARD:GUARD + self.n].view(dtype)

    def intact(self):
        import torch

        torch.cuda.synchronize()
        b = self.buf.cpu().numpy()
        return bool(np.all(b[:GUARD] == PATTERN) and np.all(b[self.tail_start:] == PATTERN))


def _meshes():
    return [("tri", I.make_mesh((13, 9), (0, 0), (2, 1), I.TRI, 0.3, 5), I.FlowSpec.double_gyre(), 2.0),
            ("kuhn", I.make_mesh((7, 5, 3), (0, 0, 0), (6.2832,) * 3, I.KUHN, 0.3, 6), I.FlowSpec.abc(), 1.5)]


@pytest.mark.parametrize("case", [0, 1])
@pytest.mark.parametrize("layout", ["csr", "ell"])
def test_device_entry_points_stay_inside_their_buffers(F, case, layout):
    import torch

    name, m, flow, T = _meshes()[case]
    dm = F.DeviceMesh.from_mesh(m)
    if layout == "ell":
        dm.attach_ell()
    n, dim = m.n_nodes, m.dim
    phi = Guarded(F.ftle_flowmap_bytes(dim, n, "fp32c"))
    out = Guarded(4 * n)
    lam = Guarded(8 * n)
    ws = Guarded(F.ftle_workspace_bytes(n))
    nsteps = int(round(T / 0.01))
    ck = Guarded(F.ftle_checkpoint_bytes(dim, n, "fp32c") * (nsteps // 7 + 1))
    opt = F.make_options(refine_kappa=5.0)  # a wide re-advection list
    F.ftle_advect(dm, flow, 0.0, T, 0.01, "fp32c", phi.view(torch.float32), ck.view(torch.float32), 7)
    F.ftle_gradient_eig(dm, phi.view(torch.float32), "fp32c", T, out.view(torch.float32), lam.view(torch.float64),
                        ws.view(torch.uint8), options=F.make_options(refine_kappa=5.0, defer_fp64=True))
    F.ftle_refine(dm, flow, 0.0, T, 0.01, "fp32c", phi.view(torch.float32), out.view(torch.float32),
                  lam.view(torch.float64), ws.view(torch.uint8), options=F.make_options(refine_kappa=5.0,
                                                                                       defer_fp64=True))
    F.ftle_compute(dm, flow, 0.0, T, 0.01, "fp32c", phi.view(torch.float32), out.view(torch.float32),
                   lam.view(torch.float64), ws.view(torch.uint8), options=opt)
    assert F.ftle_read_counters(ws.view(torch.uint8))["n_readvected"] > 0
    for g, what in ((phi, "flowmap"), (ck, "checkpoints"), (out, "ftle"), (lam, "lambda"), (ws, "workspace")):
        assert g.intact(), (name, layout, what)
    assert torch.isfinite(out.view(torch.float32)).all()


@pytest.mark.parametrize("case", [0, 1])
def test_host_path_and_batch_stay_inside_their_buffers(F, case):
    import torch

    name, m, flow, T = _meshes()[case]
    n, dim = m.n_nodes, m.dim
    hout = Guarded(4 * n, device="pinned")
    hws = Guarded(F.ftle_host_workspace_bytes(dim, n, m.nnz, "fp32c"))
    ch = torch.from_numpy(np.ascontiguousarray(m.coords)).pin_memory()
    rp = torch.from_numpy(m.row_ptr).pin_memory()
    ci = torch.from_numpy(m.col_idx).pin_memory()
    F.ftle_compute_host(ch, rp, ci, flow, 0.0, T, 0.01, "fp32c", hout.view(torch.float32), hws.view(torch.uint8))
    assert hout.intact() and hws.intact(), name
    meshes = [F.DeviceMesh.from_mesh(m), F.DeviceMesh.from_mesh(m)]
    outs = [Guarded(4 * n), Guarded(4 * n)]
    bws = Guarded(F.ftle_batch_workspace_bytes(meshes, "fp32c"))
    F.ftle_batch(meshes, [flow, flow], [T, -T], 0.01, "fp32c", [o.view(torch.float32) for o in outs],
                 bws.view(torch.uint8), options=F.make_options(refine_kappa=5.0))
    assert all(o.intact() for o in outs) and bws.intact(), name


def test_backward_stays_inside_its_buffers(F):
    import torch

    name, m, flow, T = _meshes()[0]
    dm = F.DeviceMesh.from_mesh(m)
    n = m.n_nodes
    nsteps = int(round(T / 0.01))
    phi = F.flowmap_empty(2, n, "fp32c")
    ck = F.checkpoints_empty(2, n, nsteps, 50, "fp32c")
    F.ftle_advect(dm, flow, 0.0, T, 0.01, "fp32c", phi, ck, 50)
    w = torch.full((n,), 1.0 / n, dtype=torch.float32, device="cuda")
    grad = Guarded(3 * 8)
    ws = Guarded(F.ftle_backward_workspace_bytes(n, 2))
    F.ftle_backward(dm, flow, 0.0, T, 0.01, "fp32c", phi, ck, 50, w, grad.view(torch.float64), ws.view(torch.uint8))
    assert grad.intact() and ws.intact()
    assert torch.isfinite(grad.view(torch.float64)).all()
