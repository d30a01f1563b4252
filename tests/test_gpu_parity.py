"""GPU path (libftle.so through its C-ABI) against the FP64 oracle, element by element.

Small cases (the oracle finishes in seconds) span many tiles and a ragged tail; the full-size
workloads are checked on sampled nodes the oracle computes one by one through a sub-mesh.
Tolerance (tests/_parity.py): 1e-4 relative where lambda_max > 1 + 1e-3, otherwise
1e-4 * max|FTLE| absolute; NaN must coincide.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2408_02758_gb300 import inputs as I

from _parity import compare, compare_conditioned, float_sensitivity, report

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    import torch  # noqa: F401

    from paper_2408_02758_gb300 import ftle

    ftle.lib()
    return ftle


def run_gpu(F, mesh, flow, T, dt, prec, **kw):
    dm = F.DeviceMesh.from_mesh(mesh)
    out = F.compute(dm, flow, T, dt, prec, want_lambda=True, return_all=True, **kw)
    cnt = F.ftle_read_counters(out["workspace"])
    return out["ftle"].double().cpu().numpy(), out["lam"].cpu().numpy(), out["phi"], cnt


def rk4_poly(z):
    return 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24


# ----------------------------------------------------------------------------- closed forms


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32c"])
@pytest.mark.parametrize("dim", [2, 3])
def test_saddle_ftle_closed_form(F, prec, dim):
    if dim == 2:
        m = I.make_mesh((37, 19), (0, 0), (2, 1), I.TRI, 0.3, 5, coord_dtype=np.float64 if prec == "fp64" else np.float32)
    else:
        m = I.make_mesh((9, 7, 6), (0, 0, 0), (1, 1, 1), I.KUHN, 0.25, 6, coord_dtype=np.float64 if prec == "fp64" else np.float32)
    dt, T = 0.01, 2.0
    ft, lam, _, cnt = run_gpu(F, m, I.FlowSpec.saddle(), T, dt, prec)
    expect = math.log(rk4_poly(dt)) / dt
    tol = {"fp64": 1e-12, "fp32c": 2e-6, "fp32": 1e-4}[prec]  # plain fp32 rounds the state every step
    assert np.all(np.abs(ft - expect) <= tol * expect), (np.abs(ft - expect).max(), cnt)
    assert cnt["n_degenerate"] == 0


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
@pytest.mark.parametrize("dim", [2, 3])
def test_linear_flow_flowmap_and_ftle(F, prec, dim):
    rng = np.random.default_rng(20 + dim)
    M = np.triu(rng.normal(size=(dim, dim))) * 0.5
    shape = (41, 23) if dim == 2 else (11, 9, 7)
    m = I.make_mesh(shape, (0,) * dim, (1,) * dim, I.TRI if dim == 2 else I.KUHN, 0.3, 21,
                    coord_dtype=np.float64 if prec == "fp64" else np.float32)
    T, dt = 1.5, 0.01
    ft, lam, phi, _ = run_gpu(F, m, I.FlowSpec.linear(M), T, dt, prec)
    Z = dt * M
    P = np.eye(dim) + Z + Z @ Z / 2 + Z @ Z @ Z / 6 + Z @ Z @ Z @ Z / 24
    P = np.linalg.matrix_power(P, 150)
    x0 = m.coords.astype(np.float64)
    if prec == "fp32c":
        ph = F.flowmap_pairs(phi, dim, m.n_nodes).double().cpu().numpy()
        ph = ph[..., 0] + ph[..., 1]
    else:
        ph = phi.double().cpu().numpy()
    assert np.abs(ph - P @ x0).max() < (1e-12 if prec == "fp64" else 1e-6)
    smax = np.linalg.svd(P, compute_uv=False)[0]
    expect = math.log(smax) / T
    assert np.abs(ft - expect).max() <= (1e-10 if prec == "fp64" else 1e-5) * abs(expect)


# ----------------------------------------------------------------------------- oracle parity


def _oracle_full(mesh, flow, T, dt):
    return O.ftle(flow.kind, flow.params, mesh.coords, mesh.row_ptr, mesh.col_idx, T, dt)


def test_structured_double_gyre_fp64_full_size(F):
    """256 x 128 structured grid, 4-neighbour stencil, T = 10, everything in double."""
    w = I.preset(0)
    ft, lam, _, cnt = run_gpu(F, w.mesh, w.flow, w.T, w.dt, "fp64")
    o = _oracle_full(w.mesh, w.flow, w.T, w.dt)
    rep = compare(ft, o["ftle"], o["lam"], rel_tol=1e-9)
    report(w.name, rep, sample="every node", precision="fp64")
    assert rep["ok"], rep
    assert cnt["n_degenerate"] == 0


@pytest.mark.parametrize("eps,omega", [(0.5, math.pi / 2), (0.0, 0.0)])
def test_double_gyre_forcing_extremes(F, eps, omega):
    """The forcing range of the batched instances' ends: eps = 0.5, omega = pi/2 at dt = 0.01
    puts the stage-three angle differences above the bound the unchecked step's first-order turn
    accepts, so every node takes the checked steps; eps = 0 is the steady gyre, whose a(t)
    vanishes.  Both follow the FP64 oracle."""
    w = I.preset(1, scale=1 / 32)
    flow = I.FlowSpec.double_gyre(0.1, eps, omega)
    ft, lam, _, cnt = run_gpu(F, w.mesh, flow, 10.0, 0.01, "fp32c")
    o = _oracle_full(w.mesh, flow, 10.0, 0.01)
    rep = compare(ft, o["ftle"], o["lam"])
    assert rep["ok"], (rep, cnt)


@pytest.mark.parametrize("scale", [1 / 16, 3 / 64])
def test_triangle_double_gyre_fp32c_small(F, scale):
    """Jittered triangle mesh (128 x 64 and a ragged 96 x 48), double gyre T = 15, fp32c + FP64 path."""
    w = I.preset(1, scale=scale)
    ft, lam, _, cnt = run_gpu(F, w.mesh, w.flow, w.T, w.dt, "fp32c")
    o = _oracle_full(w.mesh, w.flow, w.T, w.dt)
    rep = compare(ft, o["ftle"], o["lam"])
    print(rep, cnt)
    assert rep["ok"], (rep, cnt)


def test_abc_kuhn_fp32c_small(F):
    """32^3 jittered Kuhn tetrahedral mesh (14 neighbours), ABC flow, T = 5."""
    w = I.preset(2, scale=1 / 8)
    ft, lam, _, cnt = run_gpu(F, w.mesh, w.flow, w.T, w.dt, "fp32c")
    o = _oracle_full(w.mesh, w.flow, w.T, w.dt)
    rep = compare(ft, o["ftle"], o["lam"])
    print(rep, cnt)
    assert rep["ok"], (rep, cnt)


def test_flowmap_parity_fp32c(F):
    w = I.preset(1, scale=1 / 32)
    dm = F.DeviceMesh.from_mesh(w.mesh)
    phi = F.flowmap_empty(2, w.mesh.n_nodes, "fp32c")
    F.ftle_advect(dm, w.flow, 0.0, w.T, w.dt, "fp32c", phi)
    ph = F.flowmap_pairs(phi, 2, w.mesh.n_nodes).double().cpu().numpy()
    ph = ph[..., 0] + ph[..., 1]
    ref = O.advect(w.flow.kind, w.flow.params, w.mesh.coords, w.T, w.dt)
    err = np.abs(ph - ref)
    # separatrix nodes amplify rounding by up to ~1e4; the bulk stays near float's resolution
    assert np.median(err) < 1e-6 and err.max() < 5e-3


@pytest.mark.parametrize("preset,scale,T,dt", [(1, 1 / 16, 5.0, 0.1), (2, 1 / 8, 2.0, 0.05)])
def test_large_steps_mix_rotated_and_full_stages(F, preset, scale, T, dt):
    """Steps long enough that the stage angles of fast nodes exceed the small-angle bound, so
    lanes of one warp take the rotated and the fully evaluated stages side by side; both agree
    with the FP64 oracle's RK4 at the same step."""
    w = I.preset(preset, scale=scale)
    ft, lam, phi, cnt = run_gpu(F, w.mesh, w.flow, T, dt, "fp32c")
    o = _oracle_full(w.mesh, w.flow, T, dt)
    rep = compare(ft, o["ftle"], o["lam"])
    assert rep["ok"], (rep, cnt)
    ph = F.flowmap_pairs(phi, w.mesh.dim, w.mesh.n_nodes).double().cpu().numpy()
    err = np.abs(ph[..., 0] + ph[..., 1] - o["phi"])
    assert err.max() < 1e-6, err.max()


_FULL = {}


def _full_size(idx, n_sample=3000):
    """A benchmark workload at full size (2.1M-node triangle mesh; 16.7M-node tet mesh), its device
    mesh, and the oracle on sampled nodes (computed once per workload, shared by the layouts)."""
    if idx not in _FULL:
        _FULL.clear()  # one full-size workload resident at a time
        from paper_2408_02758_gb300 import ftle

        w = I.preset(idx)
        rng = np.random.default_rng(100 + idx)
        rows = np.sort(rng.choice(w.mesh.n_nodes, n_sample, replace=False))
        # always include the first and last nodes (corners) and a boundary node
        rows = np.unique(np.concatenate([rows, [0, w.mesh.n_nodes - 1, w.mesh.shape[0] // 2]]))
        o = O.ftle_sample(w.flow.kind, w.flow.params, w.mesh.coords, w.mesh.row_ptr, w.mesh.col_idx, rows, w.T, w.dt)
        _FULL[idx] = (w, ftle.DeviceMesh.from_mesh(w.mesh), rows, o)
    return _FULL[idx]


@pytest.mark.parametrize("layout", ["ell", "csr", "stencil"])
@pytest.mark.parametrize("idx", [1, 2])
def test_full_size_workload_sampled(F, idx, layout):
    """The benchmark's workloads at full size through each neighbour layout of the float gradient:
    the paper's fixed-width -1-padded list (the layout the benchmark times, built by
    ftle_ell_from_csr), the CSR rows, and the lattice's implicit stencil.  The whole path
    (ftle_compute, the benchmark's launch configuration) is compared with the oracle on >= 3000
    sampled nodes at the stated tolerance."""
    w, dm, rows, o = _full_size(idx)
    dm.detach_ell().detach_stencil()
    if layout == "ell":
        dm.attach_ell()
        assert dm.desc.ell_width == int(np.diff(w.mesh.row_ptr).max())
    elif layout == "stencil":
        dm.attach_stencil({I.AXIS: F.STENCIL_AXIS, I.TRI: F.STENCIL_TRI, I.KUHN: F.STENCIL_KUHN}[
            w.mesh.meta["stencil"]], w.mesh.shape)
    out = F.compute(dm, w.flow, w.T, w.dt, w.precision, return_all=True)
    cnt = F.ftle_read_counters(out["workspace"])
    ft = out["ftle"].double().cpu().numpy()
    dm.detach_ell().detach_stencil()
    rep = compare(ft[rows], o["ftle"], o["lam"])
    report(w.name, rep, sample=f"{len(rows)} random nodes", precision=w.precision, neighbours=layout, **cnt)
    assert rep["ok"], (rep, cnt)
    assert np.isfinite(ft).all()
    assert cnt["n_degenerate"] == 0


def test_full_field_triangle_double_gyre(F):
    """Every node of the 2048 x 1024 triangle-mesh workload (the benchmark's layout) against the
    oracle's whole field: 1e-4 relative on gated nodes, or the oracle's own one-rounding
    sensitivity where that is larger."""
    w, dm, _, _ = _full_size(1)
    dm.detach_stencil().attach_ell()
    ft = F.compute(dm, w.flow, w.T, w.dt, w.precision).double().cpu().numpy()
    dm.detach_ell()
    ref = O.ftle(w.flow.kind, w.flow.params, w.mesh.coords, w.mesh.row_ptr, w.mesh.col_idx, w.T, w.dt)
    S = float_sensitivity(O, w.flow, w.mesh, w.T, w.dt, base=ref["ftle"])
    rep = compare_conditioned(ft, ref["ftle"], ref["lam"], S)
    report(w.name, rep, sample="every node", precision=w.precision, neighbours="ell")
    assert rep["ok"], rep


# ----------------------------------------------------------------------------- edge cases


def test_degenerate_rows_give_nan_and_are_counted(F):
    import torch

    # node 0: collinear neighbours; node 1: one neighbour; node 2: none; node 3: fine; node 4: none
    x = np.array([[0.0, 1.0, 2.0, 0.0, 1.0], [0.0, 0.0, 0.0, 1.0, 1.0]], dtype=np.float32)
    rp = np.array([0, 2, 3, 3, 6, 6], dtype=np.int32)
    ci = np.array([1, 2, 0, 0, 1, 4], dtype=np.int32)
    mesh = I.mesh_from_arrays(x, rp, ci)
    for prec in ("fp64", "fp32", "fp32c"):
        m2 = I.mesh_from_arrays(x.astype(np.float64) if prec == "fp64" else x, rp, ci)
        ft, lam, _, cnt = run_gpu(F, m2, I.FlowSpec.linear(np.array([[1.0, 0.0], [0.0, 1.0]])), 0.5, 0.01, prec)
        assert np.isnan(ft[[0, 1, 2, 4]]).all(), (prec, ft)
        assert cnt["n_degenerate"] == 4, (prec, cnt)
        expect = math.log(rk4_poly(0.01)) / 0.01
        assert abs(ft[3] - expect) < 1e-5
    del mesh, torch


def test_empty_mesh_is_a_no_op(F):
    import torch

    m = I.mesh_from_arrays(np.zeros((2, 0), np.float32), np.zeros(1, np.int32), np.zeros(0, np.int32))
    dm = F.DeviceMesh(torch.zeros((2, 0), device="cuda"), torch.zeros(1, dtype=torch.int32, device="cuda"),
                      torch.zeros(1, dtype=torch.int32, device="cuda"))
    dm.desc.nnz = 0
    out = F.compute(dm, I.FlowSpec.saddle(), 1.0, 0.01, "fp32c")
    assert out.numel() == 0
    del m


def test_single_node_and_ragged_tail(F):
    # 257 x 3 lattice: n = 771, not a multiple of the block size
    m = I.make_mesh((257, 3), (0, 0), (2, 1), I.TRI, 0.3, 31)
    ft, lam, _, cnt = run_gpu(F, m, I.FlowSpec.double_gyre(), 3.0, 0.01, "fp32c")
    o = _oracle_full(m, I.FlowSpec.double_gyre(), 3.0, 0.01)
    rep = compare(ft, o["ftle"], o["lam"])
    assert rep["ok"], rep
    one = I.mesh_from_arrays(np.zeros((2, 1), np.float32), np.zeros(2, np.int32), np.zeros(0, np.int32))
    import torch

    dm = F.DeviceMesh(torch.zeros((2, 1), device="cuda"), torch.zeros(2, dtype=torch.int32, device="cuda"),
                      torch.zeros(1, dtype=torch.int32, device="cuda"))
    dm.desc.nnz = 0
    out = F.compute(dm, I.FlowSpec.saddle(), 1.0, 0.01, "fp32c")
    assert torch.isnan(out).all()
    del one


def test_backward_time_horizon(F):
    w = I.preset(1, scale=1 / 32)
    ft, lam, _, cnt = run_gpu(F, w.mesh, w.flow, -5.0, w.dt, "fp32c")
    o = _oracle_full(w.mesh, w.flow, -5.0, w.dt)
    rep = compare(ft, o["ftle"], o["lam"])
    assert rep["ok"], rep


def test_deterministic(F):
    w = I.preset(2, scale=1 / 16)
    a = run_gpu(F, w.mesh, w.flow, 2.0, w.dt, "fp32c")[0]
    b = run_gpu(F, w.mesh, w.flow, 2.0, w.dt, "fp32c")[0]
    assert np.array_equal(a, b)


def test_host_entry_point_matches_device_entry_point(F):
    import torch

    w = I.preset(1, scale=1 / 16)
    dev = run_gpu(F, w.mesh, w.flow, w.T, w.dt, "fp32c")[0]
    ch = torch.from_numpy(w.mesh.coords).pin_memory()
    rp = torch.from_numpy(w.mesh.row_ptr).pin_memory()
    ci = torch.from_numpy(w.mesh.col_idx).pin_memory()
    out = torch.empty(w.mesh.n_nodes, dtype=torch.float32).pin_memory()
    ws = F.workspace_empty(F.ftle_host_workspace_bytes(2, w.mesh.n_nodes, w.mesh.nnz, "fp32c"))
    F.ftle_compute_host(ch, rp, ci, w.flow, 0.0, w.T, w.dt, "fp32c", out, ws)
    assert np.array_equal(out.double().numpy(), dev)


@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
def test_host_entry_point_pinned_in_place_equals_staged(F, prec):
    """Page-locked buffers are read and written in place by the kernels (coordinates in FP32C, the
    FTLE always); pageable buffers go through staging copies: the same field bit for bit, and the
    device path's field."""
    import torch

    w = I.preset(2, scale=1 / 16) if prec == "fp32c" else I.preset(1, scale=1 / 32)
    mesh = w.mesh
    coords = mesh.coords.astype(np.float64) if prec == "fp64" else mesh.coords
    dim, n = mesh.dim, mesh.n_nodes
    ws = F.workspace_empty(F.ftle_host_workspace_bytes(dim, n, mesh.nnz, prec))
    dt = torch.float64 if prec == "fp64" else torch.float32
    outs = []
    for pinned in (True, False):
        ch = torch.from_numpy(np.ascontiguousarray(coords))
        rp = torch.from_numpy(mesh.row_ptr)
        ci = torch.from_numpy(mesh.col_idx)
        out = torch.full((n,), 5.0, dtype=dt)
        if pinned:
            ch, rp, ci, out = ch.pin_memory(), rp.pin_memory(), ci.pin_memory(), out.pin_memory()
        F.ftle_compute_host(ch, rp, ci, w.flow, 0.0, w.T, w.dt, prec, out, ws)
        outs.append(out.numpy().copy())
    assert np.array_equal(outs[0], outs[1], equal_nan=True)
    dm = F.DeviceMesh(torch.from_numpy(np.ascontiguousarray(coords)).cuda(), torch.from_numpy(mesh.row_ptr).cuda(),
                      torch.from_numpy(mesh.col_idx).cuda())
    dev = F.compute(dm, w.flow, w.T, w.dt, prec).cpu().numpy()
    assert np.array_equal(outs[0], dev, equal_nan=True)


def test_invalid_arguments_raise(F):
    import torch

    w = I.preset(1, scale=1 / 64)
    dm = F.DeviceMesh.from_mesh(w.mesh)
    phi = F.flowmap_empty(2, w.mesh.n_nodes, "fp32c")
    out = F.ftle_out_empty(w.mesh.n_nodes, "fp32c")
    small = F.workspace_empty(256)
    with pytest.raises(F.FTLEError) as e:
        F.ftle_gradient_eig(dm, phi, "fp32c", 1.0, out, None, small)
    assert e.value.status == F.FTLE_EWORKSPACE
    with pytest.raises(F.FTLEError) as e:
        F.ftle_advect(dm, I.FlowSpec.abc(), 0.0, 1.0, 0.01, "fp32c", phi)
    assert e.value.status == F.FTLE_EINVAL
    with pytest.raises(F.FTLEError):
        F.ftle_advect(dm, w.flow, 0.0, 1.0, 0.0, "fp32c", phi)
    torch.cuda.synchronize()


def test_float_float_readvection_matches_fp64_flowmap(F):
    """The nodes ftle_refine re-advects (read back from the workspace's list) carry a flowmap
    that agrees with the FP64 oracle to ~1e-11, i.e. at float-float, not float, accuracy."""
    import torch

    w = I.preset(1, scale=1 / 16)
    dm = F.DeviceMesh.from_mesh(w.mesh)
    out = F.compute(dm, w.flow, w.T, w.dt, "fp32c", return_all=True)
    cnt = F.ftle_read_counters(out["workspace"])
    n = w.mesh.n_nodes
    assert cnt["n_readvected"] > 0
    # workspace layout: 256-byte counters, then int32 flag list [n], then int32 mark list [n]
    off = 256 + ((4 * n + 255) // 256) * 256
    ws = out["workspace"].cpu().numpy()
    marked = np.frombuffer(ws[off: off + 4 * cnt["n_readvected"]].tobytes(), dtype=np.int32)
    assert len(np.unique(marked)) == len(marked) and marked.min() >= 0 and marked.max() < n
    ph = F.flowmap_pairs(out["phi"], 2, n).double().cpu().numpy()
    ph = ph[..., 0] + ph[..., 1]
    ref = O.advect(w.flow.kind, w.flow.params, w.mesh.coords[:, marked], w.T, w.dt)
    err = np.abs(ph[:, marked] - ref).max()
    assert err < 1e-10, err
    torch.cuda.synchronize()


@pytest.mark.parametrize("T", [1.23, 0.09, -4.0, 25.0])
def test_run_parallel_readvection_matches_fp64_flowmap(F, T):
    """The re-advected nodes' flowmap agrees with the FP64 oracle at float-float accuracy for step
    counts that do not divide into the runs evenly (123), runs of one or two steps (9), a backward
    horizon, and a horizon past the run-parallel table (2500 steps: the sequential kernel)."""
    w = I.preset(1, scale=1 / 32)
    dm = F.DeviceMesh.from_mesh(w.mesh)
    opt = F.make_options(refine_kappa=0.05)  # a wide re-advection list
    out = F.compute(dm, w.flow, T, w.dt, "fp32c", return_all=True, options=opt)
    cnt = F.ftle_read_counters(out["workspace"])
    n = w.mesh.n_nodes
    assert cnt["n_readvected"] > 0
    off = 256 + ((4 * n + 255) // 256) * 256
    ws = out["workspace"].cpu().numpy()
    marked = np.frombuffer(ws[off: off + 4 * cnt["n_readvected"]].tobytes(), dtype=np.int32)
    ph = F.flowmap_pairs(out["phi"], 2, n).double().cpu().numpy()
    ph = ph[..., 0] + ph[..., 1]
    ref = O.advect(w.flow.kind, w.flow.params, w.mesh.coords[:, marked], T, w.dt)
    err = np.abs(ph[:, marked] - ref).max()
    assert err < 1e-10, err


@pytest.mark.parametrize("T,dt", [(5.0, 0.01), (1.23, 0.01), (0.17, 0.01), (-2.0, 0.01), (0.05, 0.01), (1.0, 0.02)])
def test_run_parallel_abc_readvection_matches_fp64_flowmap(F, T, dt):
    """The 3D ABC re-advection integrates a node's runs side by side (ten runs, three lanes each,
    boundary states from the compensated float step, joined through each run's tangent): the
    re-advected flowmap agrees with the FP64 oracle at float-float accuracy for the workload's 500
    steps, step counts that do not divide into the runs (123), runs of two steps with the last
    ones empty (17), a backward horizon, fewer steps than runs (5: the one-run kernel), and steps
    long enough that the boundary pass takes the checked step (dt = 0.02: angles past the
    unchecked turns' limit)."""
    w = I.preset(2, scale=1 / 16)  # 16^3 jittered Kuhn mesh
    dm = F.DeviceMesh.from_mesh(w.mesh)
    opt = F.make_options(refine_kappa=0.3)  # a wide re-advection list
    if dt != 0.01:
        assert not F.ftle_rotation_bounds(w.flow, dt)["unchecked"]
    out = F.compute(dm, w.flow, T, dt, "fp32c", return_all=True, options=opt)
    cnt = F.ftle_read_counters(out["workspace"])
    n = w.mesh.n_nodes
    assert cnt["n_readvected"] > 0
    off = 256 + ((4 * n + 255) // 256) * 256
    ws = out["workspace"].cpu().numpy()
    marked = np.frombuffer(ws[off: off + 4 * cnt["n_readvected"]].tobytes(), dtype=np.int32)
    ph = F.flowmap_pairs(out["phi"], 3, n).double().cpu().numpy()
    ph = ph[..., 0] + ph[..., 1]
    ref = O.advect(w.flow.kind, w.flow.params, w.mesh.coords[:, marked], T, dt)
    err = np.abs(ph[:, marked] - ref).max()
    assert err < 1e-10, (err, len(marked))


@pytest.mark.parametrize("preset,scale,kappa", [(1, 1 / 16, 0.01), (2, 1 / 8, 0.3)])
def test_readvection_independent_of_lanes_per_block(F, preset, scale, kappa):
    """How many nodes a block of the float-float re-advection takes (refine_lanes; the 2D double
    gyre uses two lanes per node) changes scheduling only: results are bit-identical."""
    w = I.preset(preset, scale=scale)
    dm = F.DeviceMesh.from_mesh(w.mesh)
    outs = []
    for lanes in (32, 7, 1):
        opt = F.make_options(refine_lanes=lanes, refine_kappa=kappa)  # a wide re-advection list
        o = F.compute(dm, w.flow, w.T, w.dt, "fp32c", return_all=True, options=opt)
        outs.append((o["ftle"].cpu().numpy(), F.flowmap_pairs(o["phi"], w.mesh.dim, w.mesh.n_nodes).cpu().numpy()))
        assert F.ftle_read_counters(o["workspace"])["n_readvected"] > 0
    for ft, ph in outs[1:]:
        assert np.array_equal(ft, outs[0][0], equal_nan=True) and np.array_equal(ph, outs[0][1])


@pytest.mark.parametrize("preset,scale,width", [(1, 1 / 16, None), (1, 1 / 16, 7), (2, 1 / 8, None), (0, 1 / 4, 4)])
def test_fixed_width_neighbour_list_matches_csr(F, preset, scale, width):
    """The paper's fixed-width, -1 padded neighbour list gives bit-identical FTLE to the CSR rows
    (same neighbour order, same arithmetic); width 7 exercises the run-time-width kernel."""
    import torch

    w = I.preset(preset, scale=scale)
    dm = F.DeviceMesh.from_mesh(w.mesh)
    a = F.compute(dm, w.flow, w.T, w.dt, w.precision).cpu()
    dm.attach_ell(width)
    assert dm.desc.ell_width == (width or int(np.diff(w.mesh.row_ptr).max()))
    ell = dm.ell.cpu().numpy()
    rp, ci = w.mesh.row_ptr, w.mesh.col_idx
    for i in (0, 1, w.mesh.n_nodes // 2, w.mesh.n_nodes - 1):
        row = ci[rp[i]:rp[i + 1]]
        assert np.array_equal(ell[: len(row), i], row) and np.all(ell[len(row):, i] == -1)
    b = F.compute(dm, w.flow, w.T, w.dt, w.precision).cpu()
    assert torch.equal(torch.isnan(a), torch.isnan(b)) and torch.equal(a[~torch.isnan(a)], b[~torch.isnan(b)])


@pytest.mark.parametrize("shape", [(64, 32), (100, 37), (33, 17), (24, 20, 18), (17, 13, 11)])
def test_staged_index_tiles_equal_direct_loads(F, shape):
    """The fixed-width-list gradient with each tile's index slices staged in shared memory by bulk
    copies (grad_staging = 0, the default) equals the plain-load kernel (grad_staging = 1) bit for
    bit: a full last tile, a ragged last tile (n a multiple of 4: 3700 and 8640 nodes), and meshes
    the staged kernel leaves to the plain one (n not a multiple of 4: 561, 2431 nodes)."""
    import torch

    dim = len(shape)
    m = I.make_mesh(shape, (0,) * dim, (2,) + (1,) * (dim - 1), I.TRI if dim == 2 else I.KUHN, 0.3, 5)
    flow = I.FlowSpec.double_gyre() if dim == 2 else I.FlowSpec.abc()
    T = 5.0 if dim == 2 else 1.0
    dm = F.DeviceMesh.from_mesh(m)
    dm.attach_ell()
    phi = F.flowmap_empty(dim, m.n_nodes, "fp32c")
    F.ftle_advect(dm, flow, 0.0, T, 0.01, "fp32c", phi)
    outs = []
    for staging in (0, 1):
        out = torch.full((m.n_nodes,), 9.0, device="cuda")
        lam = torch.full((m.n_nodes,), 9.0, dtype=torch.float64, device="cuda")
        ws = F.workspace_empty(F.ftle_workspace_bytes(m.n_nodes))
        F.ftle_gradient_eig(dm, phi, "fp32c", T, out, lam, ws, options=F.make_options(grad_staging=staging))
        cnt = F.ftle_read_counters(ws)
        assert cnt["n_wait_timeouts"] == 0
        outs.append((out.cpu(), lam.cpu(), cnt["n_flagged"]))
    (a, la, fa), (b, lb, fb) = outs
    assert fa == fb
    assert torch.equal(torch.isnan(a), torch.isnan(b)) and torch.equal(a[~torch.isnan(a)], b[~torch.isnan(b)])
    assert torch.equal(torch.isnan(la), torch.isnan(lb)) and torch.equal(la[~torch.isnan(la)], lb[~torch.isnan(lb)])


@pytest.mark.parametrize("refresh", [1, 2, 8, 16])
def test_abc_carried_stage_one_refresh(F, refresh):
    """The compensated ABC step carries stage one's sines and cosines from step to step (stage
    four's pairs turned by the rest of the step's increment) and evaluates them afresh every
    abc_refresh steps: every period follows the
    oracle at the parity tolerance (a ragged 500 steps against periods that do not divide it), and
    the batched kernel, carrying them the same way, gives the single kernel's flowmap bit for bit."""
    import torch

    w = I.preset(2, scale=3 / 32)  # 24^3 jittered Kuhn mesh
    opt = F.make_options(abc_refresh=refresh)
    ft, lam, phi, cnt = run_gpu(F, w.mesh, w.flow, w.T, w.dt, "fp32c", options=opt)
    o = _oracle_full(w.mesh, w.flow, w.T, w.dt)
    rep = compare(ft, o["ftle"], o["lam"])
    assert rep["ok"], (refresh, rep)
    dm = F.DeviceMesh.from_mesh(w.mesh)
    out = torch.full((w.mesh.n_nodes,), 3.0, device="cuda")
    ws = F.workspace_empty(F.ftle_batch_workspace_bytes([dm], "fp32c"))
    F.ftle_batch([dm], [w.flow], [w.T], w.dt, "fp32c", [out], ws, options=F.make_options(abc_refresh=refresh,
                                                                                            refine_kappa=-1.0))
    single = F.compute(dm, w.flow, w.T, w.dt, "fp32c", options=F.make_options(abc_refresh=refresh, refine_kappa=-1.0))
    torch.cuda.synchronize()
    a, b = out.cpu(), single.cpu()
    assert torch.equal(torch.isnan(a), torch.isnan(b)) and torch.equal(a[~torch.isnan(a)], b[~torch.isnan(b)])


@pytest.mark.parametrize("A,B,C,dt,T", [(1.0, 1.0, 1.0, 0.005, 3.0), (2.0, 0.5, 1.0, 0.01, 2.0),
                                         (math.sqrt(3.0), math.sqrt(2.0), 1.0, 0.011, 5.06)])
def test_abc_unchecked_step_other_parameters(F, A, B, C, dt, T):
    """The unchecked compensated ABC step (stage one carried from stage four, stage two's shorter
    turn) on other flow parameters and step sizes, each within the host's bounds for the
    unchecked step: the whole field of a 24^3 Kuhn mesh follows the oracle at the parity
    tolerance."""
    flow = I.FlowSpec.abc(A, B, C)
    assert F.ftle_rotation_bounds(flow, dt)["unchecked"]
    w = I.preset(2, scale=3 / 32)  # 24^3 jittered Kuhn mesh
    ft, lam, _, cnt = run_gpu(F, w.mesh, flow, T, dt, "fp32c")
    o = _oracle_full(w.mesh, flow, T, dt)
    rep = compare(ft, o["ftle"], o["lam"])
    report(w.name, rep, sample="every node", precision="fp32c", A=A, B=B, C=C, dt=dt, T=T)
    assert rep["ok"], rep
    assert cnt["n_degenerate"] == 0


@pytest.mark.parametrize("T", [5.0, 2.47, 23.0])
def test_abc_carried_steps_with_and_without_checkpoints(F, T):
    """The carried ABC steps run grouped between refreshes (a whole group of the default period
    unrolled) when no checkpoint is stored, and one at a time when checkpoints are: the flowmap
    is the same bit for bit, for step counts that end a group exactly, cut one short (247) and
    span two coefficient chunks of 2048 steps (2300)."""
    import torch

    w = I.preset(2, scale=1 / 32)  # 8^3 jittered Kuhn mesh
    dm = F.DeviceMesh.from_mesh(w.mesh)
    n = w.mesh.n_nodes
    nsteps = int(round(T / w.dt))
    a = F.flowmap_empty(3, n, "fp32c")
    b = F.flowmap_empty(3, n, "fp32c")
    ck = F.checkpoints_empty(3, n, nsteps, 37, "fp32c")
    F.ftle_advect(dm, w.flow, 0.0, T, w.dt, "fp32c", a)
    F.ftle_advect(dm, w.flow, 0.0, T, w.dt, "fp32c", b, ck, 37)
    torch.cuda.synchronize()
    pa, pb = F.flowmap_pairs(a, 3, n), F.flowmap_pairs(b, 3, n)
    assert torch.equal(pa, pb)
    last = ck[nsteps // 37].view(3, n, 2)
    assert torch.isfinite(last).all()


def test_abc_refresh_must_be_a_power_of_two(F):
    w = I.preset(2, scale=1 / 32)
    dm = F.DeviceMesh.from_mesh(w.mesh)
    phi = F.flowmap_empty(3, w.mesh.n_nodes, "fp32c")
    for bad in (3, 2048, -4):
        with pytest.raises(F.FTLEError) as e:
            F.ftle_advect(dm, w.flow, 0.0, 1.0, w.dt, "fp32c", phi, options=F.make_options(abc_refresh=bad))
        assert e.value.status == F.FTLE_EINVAL


def _hub_mesh():
    """A 128 x 64 triangle mesh whose node 0 also neighbours every other node (a row of 8191
    entries, so the first tile's stretch of col_idx is longer than a stage holds)."""
    m = I.make_mesh((128, 64), (0, 0), (2, 1), I.TRI, 0.3, 9)
    n = m.n_nodes
    rows = [set(m.col_idx[m.row_ptr[i]:m.row_ptr[i + 1]].tolist()) for i in range(n)]
    rows[0] |= set(range(1, n))
    for i in range(1, n):
        rows[i].add(0)
    rp = np.zeros(n + 1, np.int32)
    rp[1:] = np.cumsum([len(r) for r in rows])
    ci = np.concatenate([np.array(sorted(r), np.int32) for r in rows])
    return I.mesh_from_arrays(m.coords, rp, ci)


@pytest.mark.parametrize("case", ["tri", "kuhn", "ragged", "hub", "offset"])
def test_staged_csr_stretches_equal_direct_loads(F, case):
    """The CSR gradient with each tile's stretch of col_idx staged in shared memory
    (grad_staging = 0, the default) equals the plain-load kernel bit for bit: lattice meshes, a
    ragged last tile, a hub row longer than a stage (read from global memory), and col_idx not
    16-byte aligned (left to the plain kernel)."""
    import torch

    if case == "tri":
        m = I.make_mesh((64, 48), (0, 0), (2, 1), I.TRI, 0.3, 5)
    elif case == "kuhn":
        m = I.make_mesh((24, 20, 18), (0, 0, 0), (2, 1, 1), I.KUHN, 0.3, 5)
    elif case == "ragged":
        m = I.make_mesh((17, 13, 11), (0, 0, 0), (2, 1, 1), I.KUHN, 0.3, 5)
    else:
        m = _hub_mesh()
    dim = m.dim
    flow = I.FlowSpec.double_gyre() if dim == 2 else I.FlowSpec.abc()
    T = 3.0 if dim == 2 else 1.0
    if case == "offset":
        base = F.DeviceMesh.from_mesh(m)
        ci = torch.empty(m.nnz + 1, dtype=torch.int32, device="cuda")
        ci[1:] = base.col_idx
        dm = F.DeviceMesh(base.coords, base.row_ptr, ci[1:])  # 4 bytes past a 256-byte boundary
        assert dm.col_idx.data_ptr() % 16 == 4
    else:
        dm = F.DeviceMesh.from_mesh(m)
    phi = F.flowmap_empty(dim, m.n_nodes, "fp32c")
    F.ftle_advect(dm, flow, 0.0, T, 0.01, "fp32c", phi)
    outs = []
    for staging in (0, 1):
        out = torch.full((m.n_nodes,), 9.0, device="cuda")
        lam = torch.full((m.n_nodes,), 9.0, dtype=torch.float64, device="cuda")
        ws = F.workspace_empty(F.ftle_workspace_bytes(m.n_nodes))
        F.ftle_gradient_eig(dm, phi, "fp32c", T, out, lam, ws, options=F.make_options(grad_staging=staging))
        cnt = F.ftle_read_counters(ws)
        assert cnt["n_wait_timeouts"] == 0
        outs.append((out.cpu(), lam.cpu(), cnt["n_flagged"]))
    (a, la, fa), (b, lb, fb) = outs
    assert fa == fb
    assert torch.equal(torch.isnan(a), torch.isnan(b)) and torch.equal(a[~torch.isnan(a)], b[~torch.isnan(b)])
    assert torch.equal(torch.isnan(la), torch.isnan(lb)) and torch.equal(la[~torch.isnan(la)], lb[~torch.isnan(lb)])


def test_fixed_width_list_rejects_long_rows(F):
    w = I.preset(2, scale=1 / 32)
    dm = F.DeviceMesh.from_mesh(w.mesh)
    with pytest.raises(F.FTLEError) as e:
        dm.attach_ell(8)  # Kuhn rows have 14 neighbours
    assert e.value.status == F.FTLE_ERANGE


@pytest.mark.parametrize("preset,scale", [(1, 1 / 16), (2, 1 / 16)])
def test_gradient_records_match_flowmap_pairs(F, preset, scale):
    """The 32-byte gradient records after the (hi, lo) pairs hold the node's float coordinates,
    the hi parts exactly and the lo parts (two of them in bfloat16 in 3D) as documented."""
    w = I.preset(preset, scale=scale)
    dm = F.DeviceMesh.from_mesh(w.mesh)
    n, dim = w.mesh.n_nodes, w.mesh.dim
    phi = F.flowmap_empty(dim, n, "fp32c")
    F.ftle_advect(dm, w.flow, 0.0, 1.0, w.dt, "fp32c", phi)
    pairs = F.flowmap_pairs(phi, dim, n).cpu().numpy()
    off = (8 * dim * n + 255) // 256 * 256 // 4
    rec = phi[off: off + 8 * n].cpu().numpy().reshape(n, 8)
    assert np.array_equal(rec[:, :dim], w.mesh.coords.T)
    if dim == 2:
        assert np.array_equal(rec[:, 2:4], pairs[:, :, 0].T) and np.array_equal(rec[:, 4:6], pairs[:, :, 1].T)
    else:
        assert np.array_equal(rec[:, 3], pairs[0, :, 0]) and np.array_equal(rec[:, 4:6], pairs[1:, :, 0].T)
        assert np.array_equal(rec[:, 6], pairs[0, :, 1])
        words = rec[:, 7].view(np.uint32)
        ly = (words << 16).view(np.float32)
        lz = (words & 0xFFFF0000).view(np.float32)
        for got, ref in ((ly, pairs[1, :, 1]), (lz, pairs[2, :, 1])):
            assert np.all(np.abs(got - ref) <= np.abs(ref) * 2.0 ** -8 + 1e-45)


@pytest.mark.parametrize("shape,stencil,max_row", [((37, 23), I.TRI, 16), ((9, 8, 7), I.KUHN, 80), ((64, 64, 64), I.KUHN, 80)])
def test_gpu_csr_from_elements_matches_host_lists(F, shape, stencil, max_row):
    """Neighbour lists built on the GPU from triangles / tetrahedra equal the host lists exactly."""
    import torch

    m = I.make_mesh(shape, (0,) * len(shape), (1,) * len(shape), stencil, 0.2, 3)
    el = torch.from_numpy(I.lattice_elements(shape, stencil)).cuda()
    rp, ci = F.ftle_csr_from_elements(m.n_nodes, el, max_row)
    assert np.array_equal(rp.cpu().numpy(), m.row_ptr)
    assert np.array_equal(ci.cpu().numpy(), m.col_idx)


def test_gpu_csr_from_elements_rejects_bad_input(F):
    import torch

    el = torch.tensor([[0, 1, 2], [1, 2, 7]], dtype=torch.int32, device="cuda")  # vertex 7 >= n_nodes
    with pytest.raises(F.FTLEError) as e:
        F.ftle_csr_from_elements(4, el, 8)
    assert e.value.status == F.FTLE_EINVAL
    el = torch.tensor([[0, 1, 2], [0, 2, 3], [0, 3, 1]], dtype=torch.int32, device="cuda")
    with pytest.raises(F.FTLEError) as e:
        F.ftle_csr_from_elements(4, el, 3)  # node 0 has 6 raw entries
    assert e.value.status == F.FTLE_ERANGE


@pytest.mark.parametrize("preset,scale", [(1, 1 / 16), (2, 1 / 16)])
def test_deferred_fp64_pass_gives_the_whole_path(F, preset, scale):
    """With defer_fp64 the gradient call leaves its flagged nodes NaN for ftle_refine, which
    recomputes them after the re-advection: the staged calls then equal ftle_compute (which
    defers by itself) and the undeferred staged calls, bit for bit."""
    import torch

    w = I.preset(preset, scale=scale)
    dm = F.DeviceMesh.from_mesh(w.mesh)
    n = w.mesh.n_nodes
    kappa = 0.3 if w.mesh.dim == 3 else 0.0  # a small 3D mesh flags nodes only with a wide test
    outs = []
    for defer in (True, False):
        opt = F.make_options(defer_fp64=defer, refine_kappa=kappa)
        phi = F.flowmap_empty(w.mesh.dim, n, "fp32c")
        out = F.ftle_out_empty(n, "fp32c")
        ws = F.workspace_empty(F.ftle_workspace_bytes(n))
        F.ftle_advect(dm, w.flow, 0.0, w.T, w.dt, "fp32c", phi)
        F.ftle_gradient_eig(dm, phi, "fp32c", w.T, out, None, ws, options=opt)
        torch.cuda.synchronize()
        flagged = F.ftle_read_counters(ws)["n_flagged"]
        assert flagged > 0
        n_nan = int(torch.isnan(out).sum())
        assert (n_nan >= flagged) if defer else (n_nan < flagged)
        F.ftle_refine(dm, w.flow, 0.0, w.T, w.dt, "fp32c", phi, out, None, ws, options=opt)
        outs.append(out.cpu())
    whole = F.compute(dm, w.flow, w.T, w.dt, "fp32c", options=F.make_options(refine_kappa=kappa)).cpu()
    for o in outs:
        assert torch.equal(torch.isnan(o), torch.isnan(whole))
        assert torch.equal(o[~torch.isnan(o)], whole[~torch.isnan(whole)])


@pytest.mark.parametrize("shape,stencil", [((37, 19), I.TRI), ((33, 17), I.AXIS), ((9, 7, 6), I.KUHN), ((9, 7, 6), I.AXIS)])
@pytest.mark.parametrize("prec", ["fp32c", "fp32"])
def test_implicit_stencil_matches_csr(F, shape, stencil, prec):
    """Neighbours taken from the lattice (ftle_mesh.stencil, no index read) give the FTLE of the
    CSR rows bit for bit: same neighbours, same order, padding slots adding exact zeros."""
    import torch

    dim = len(shape)
    m = I.make_mesh(shape, (0,) * dim, (2,) + (1,) * (dim - 1), stencil, 0.3, 11)
    flow = I.FlowSpec.double_gyre() if dim == 2 else I.FlowSpec.abc()
    T = 5.0 if dim == 2 else 1.0
    dm = F.DeviceMesh.from_mesh(m)
    a = F.compute(dm, flow, T, 0.01, prec, want_lambda=True, return_all=True)
    kind = {I.AXIS: F.STENCIL_AXIS, I.TRI: F.STENCIL_TRI, I.KUHN: F.STENCIL_KUHN}[stencil]
    dm.attach_stencil(kind, shape)
    b = F.compute(dm, flow, T, 0.01, prec, want_lambda=True, return_all=True)
    for key in ("ftle", "lam"):
        x, y = a[key].cpu(), b[key].cpu()
        assert torch.equal(torch.isnan(x), torch.isnan(y)) and torch.equal(x[~torch.isnan(x)], y[~torch.isnan(y)]), key
    assert F.ftle_read_counters(a["workspace"]) == F.ftle_read_counters(b["workspace"])


def test_double_gyre_nodes_inside_and_outside_the_domain(F):
    """Nodes in [0, 2] x [0, 1] take the unchecked rotated steps, nodes outside the checked ones
    (warps mixing both run the two loops); both follow the FP64 oracle's RK4, and the batched
    kernel, deciding per node the same way, gives the same flowmap and FTLE bit for bit."""
    import torch

    m = I.make_mesh((45, 23), (-0.5, -0.25), (2.5, 1.25), I.TRI, 0.3, 17)
    inside = (m.coords[0] >= 0) & (m.coords[0] <= 2) & (m.coords[1] >= 0) & (m.coords[1] <= 1)
    assert 0 < inside.sum() < m.n_nodes
    flow, T = I.FlowSpec.double_gyre(), 5.0
    dm = F.DeviceMesh.from_mesh(m)
    phi = F.flowmap_empty(2, m.n_nodes, "fp32c")
    F.ftle_advect(dm, flow, 0.0, T, 0.01, "fp32c", phi)
    ph = F.flowmap_pairs(phi, 2, m.n_nodes).double().cpu().numpy()
    ph = ph[..., 0] + ph[..., 1]
    ref = O.advect(flow.kind, flow.params, m.coords, T, 0.01)
    err = np.abs(ph - ref) / np.maximum(1.0, np.abs(ref))
    assert np.median(err[:, inside]) < 1e-6 and np.median(err[:, ~inside]) < 1e-6 and err.max() < 5e-3
    res = F.compute(dm, flow, T, 0.01, "fp32c", return_all=True)
    single = res["ftle"].cpu().double().numpy()
    n_readvected = F.ftle_read_counters(res["workspace"])["n_readvected"]
    out = torch.full((m.n_nodes,), 7.0, dtype=torch.float32, device="cuda")
    ws = F.workspace_empty(F.ftle_batch_workspace_bytes([dm], "fp32c"))
    F.ftle_batch([dm], [flow], [T], 0.01, "fp32c", [out], ws)
    b = out.cpu().double().numpy()
    # identical except the time coefficients of re-advected nodes (as in the batch tests): those
    # agree to float-float accuracy, at most one rounding of the float output
    diff = ~((b == single) | (np.isnan(b) & np.isnan(single)))
    assert np.count_nonzero(diff) <= n_readvected
    assert np.all(np.abs(b - single)[diff] <= 2.0**-23 * np.abs(single)[diff])
