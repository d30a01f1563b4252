"""torch.autograd.Function for the FTLE field of the double gyre as a function of its parameters.

Forward: RK4 flowmap with checkpoints (libftle ftle_advect), the FTLE core and the refinement of
float-sensitive nodes.  Backward: the library's reverse-mode adjoint (ftle_backward): the FTLE-map
adjoint gathered over the mesh adjacency, then the discrete adjoint of the RK4 steps, recomputing
each checkpoint segment.  Every step runs in libftle's CUDA kernels; this module only moves
tensors.

    params = torch.tensor([0.1, 0.25, 2 * math.pi / 10], dtype=torch.float64, requires_grad=True)
    ftle_field = FTLEFunction.apply(params, dmesh, 15.0, 0.01)
    loss = (ftle_field.double() * weights).sum()      # e.g. a region mean
    loss.backward()                                   # params.grad = dL/d(A, eps, omega)
"""
from __future__ import annotations

import torch

from . import ftle
from .inputs import FlowSpec


class FTLEFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, mesh, T: float, dt: float, precision: str = "fp32c", ckpt_every: int = 50):
        if mesh.dim != 2:
            raise ValueError("the parameter derivative is defined for the 2D double gyre")
        p = [float(v) for v in params.detach().double().cpu().tolist()]
        flow = FlowSpec.double_gyre(*p)
        n = mesh.n_nodes
        n_steps = int(round(abs(T) / dt))
        phi = ftle.flowmap_empty(2, n, precision)
        ckpt = ftle.checkpoints_empty(2, n, n_steps, ckpt_every, precision)
        out = ftle.ftle_out_empty(n, precision)
        ws = ftle.workspace_empty(ftle.ftle_workspace_bytes(n))
        ftle.ftle_advect(mesh, flow, 0.0, T, dt, precision, phi, ckpt, ckpt_every)
        opt = ftle.make_options(defer_fp64=True)  # the FP64 pass runs once, after the re-advection
        ftle.ftle_gradient_eig(mesh, phi, precision, T, out, None, ws, options=opt)
        ftle.ftle_refine(mesh, flow, 0.0, T, dt, precision, phi, out, None, ws, options=opt)
        ctx.save_for_backward(phi, ckpt)
        ctx.mesh, ctx.flow, ctx.T, ctx.dt, ctx.precision, ctx.ckpt_every = mesh, flow, T, dt, precision, ckpt_every
        ctx.param_device, ctx.param_dtype = params.device, params.dtype
        return out

    @staticmethod
    def backward(ctx, grad_out):
        phi, ckpt = ctx.saved_tensors
        mesh = ctx.mesh
        g = grad_out.detach().float().contiguous()
        if not g.is_cuda:
            g = g.cuda()
        dparams = torch.empty(3, dtype=torch.float64, device="cuda")
        ws = ftle.workspace_empty(ftle.ftle_backward_workspace_bytes(mesh.n_nodes, 2))
        ftle.ftle_backward(mesh, ctx.flow, 0.0, ctx.T, ctx.dt, ctx.precision, phi, ckpt, ctx.ckpt_every, g, dparams,
                           ws)
        return dparams.to(device=ctx.param_device, dtype=ctx.param_dtype), None, None, None, None, None


def ftle_field(params, mesh, T: float, dt: float, precision: str = "fp32c", ckpt_every: int = 50):
    return FTLEFunction.apply(params, mesh, T, dt, precision, ckpt_every)
