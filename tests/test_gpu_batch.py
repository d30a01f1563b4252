"""Batched execution (ftle_batch, ftle_batch_plan_*) on the GPU: every instance equals its
single-problem result (same kernels' arithmetic), the captured graph replays identically, and
instances match the FP64 oracle."""
import numpy as np
import pytest

import oracle as O
from paper_2408_02758_gb300 import inputs as I

from _parity import compare, compare_conditioned, float_sensitivity, report

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def batch():
    import torch

    from paper_2408_02758_gb300 import ftle

    ws_list = I.batched_preset(12, scale=1 / 8)  # 8x4 .. 128x64 grids, T in {5, 10, 15, 20}
    meshes = [ftle.DeviceMesh.from_mesh(w.mesh) for w in ws_list]
    outs = [torch.full((w.mesh.n_nodes,), 7.0, dtype=torch.float32, device="cuda") for w in ws_list]
    return ftle, torch, ws_list, meshes, outs


def _single(ftle, w, dm, options=None):
    out = ftle.compute(dm, w.flow, w.T, w.dt, "fp32c", return_all=True, options=options)
    return out["ftle"].double().cpu().numpy(), ftle.ftle_read_counters(out["workspace"])


@pytest.mark.parametrize("kappa", [0.0, 0.05])
def test_batch_equals_single_instances(batch, kappa):
    """kappa = 0 is the default flagging; 0.05 forces the re-advection path on many nodes."""
    ftle, torch, ws_list, meshes, outs = batch
    opt = ftle.make_options(refine_kappa=kappa)
    ws = ftle.workspace_empty(ftle.ftle_batch_workspace_bytes(meshes, "fp32c"))
    ftle.ftle_batch(meshes, [w.flow for w in ws_list], [w.T for w in ws_list], 0.01, "fp32c", outs, ws, options=opt)
    torch.cuda.synchronize()
    n_refined = 0
    for w, dm, o in zip(ws_list, meshes, outs):
        single, cnt = _single(ftle, w, dm, opt)
        got = o.double().cpu().numpy()
        # identical arithmetic except the time coefficients of re-advected nodes: the batched
        # re-advection turns (sin, cos)(omega t) per half step where the single one reads a table
        # of double sines, so those nodes agree to float-float accuracy, which can move the float
        # output by one rounding; every other node is bit-identical
        diff = got != single
        assert np.count_nonzero(diff) <= cnt["n_readvected"], w.name
        assert np.all(np.abs(got - single)[diff] <= 2.0**-23 * np.abs(single)[diff]), w.name
        n_refined += cnt["n_readvected"]
    if kappa > 0:
        assert n_refined > 0  # the refinement path ran


def test_batch_plan_graph_replays_identically(batch):
    ftle, torch, ws_list, meshes, outs = batch
    ws = ftle.workspace_empty(ftle.ftle_batch_workspace_bytes(meshes, "fp32c"))
    ftle.ftle_batch(meshes, [w.flow for w in ws_list], [w.T for w in ws_list], 0.01, "fp32c", outs, ws)
    torch.cuda.synchronize()
    ref = [o.clone() for o in outs]
    for o in outs:
        o.fill_(-1.0)
    plan = ftle.BatchPlan(meshes, [w.flow for w in ws_list], [w.T for w in ws_list], 0.01, "fp32c", outs, ws,
                          options=ftle.make_options(grad_tile=512))
    for _ in range(2):
        plan.launch()
        torch.cuda.synchronize()
        for o, r in zip(outs, ref):
            assert torch.equal(o, r)
        for o in outs:
            o.fill_(-1.0)
    plan.destroy()


def test_batch_instances_match_oracle(batch):
    ftle, torch, ws_list, meshes, outs = batch
    ws = ftle.workspace_empty(ftle.ftle_batch_workspace_bytes(meshes, "fp32c"))
    ftle.ftle_batch(meshes, [w.flow for w in ws_list], [w.T for w in ws_list], 0.01, "fp32c", outs, ws)
    torch.cuda.synchronize()
    for k in (0, 3, 7):
        w = ws_list[k]
        o = O.ftle(w.flow.kind, w.flow.params, w.mesh.coords, w.mesh.row_ptr, w.mesh.col_idx, w.T, w.dt)
        rep = compare(outs[k].double().cpu().numpy(), o["ftle"], o["lam"])
        assert rep["ok"], (w.name, rep)


def test_batch_rejects_mixed_dimensions(batch):
    ftle, torch, ws_list, meshes, outs = batch
    m3 = I.make_mesh((4, 4, 4), (0, 0, 0), (1, 1, 1), I.KUHN, 0.2, 3)
    d3 = ftle.DeviceMesh.from_mesh(m3)
    o3 = torch.empty(m3.n_nodes, device="cuda")
    ws = ftle.workspace_empty(ftle.ftle_batch_workspace_bytes([meshes[0], d3], "fp32c"))
    with pytest.raises(ftle.FTLEError) as e:
        ftle.ftle_batch([meshes[0], d3], [ws_list[0].flow, I.FlowSpec.abc()], [1.0, 1.0], 0.01, "fp32c",
                        [outs[0], o3], ws)
    assert e.value.status == ftle.FTLE_EINVAL


def test_autotuned_options_give_identical_results(batch):
    """Launch shapes change scheduling only: the tuned options reproduce the default result."""
    ftle, torch, ws_list, meshes, outs = batch
    from paper_2408_02758_gb300 import autotune

    w = I.preset(1, scale=1 / 16)
    dm = ftle.DeviceMesh.from_mesh(w.mesh)
    cache = autotune.Cache(autotune.cache_path().with_name("autotune_test.json"))
    opts = autotune.options_for_compute(dm, w.flow, w.T, w.dt, "fp32c", cache=cache, retune=True)
    a = ftle.compute(dm, w.flow, w.T, w.dt, "fp32c").cpu()
    b = ftle.compute(dm, w.flow, w.T, w.dt, "fp32c", options=opts).cpu()
    assert torch.equal(a, b)
    # the gradient's shape alone, tuned on these CSR rows (the host-buffer path's layout)
    phi = ftle.flowmap_empty(2, w.mesh.n_nodes, "fp32c")
    ftle.ftle_advect(dm, w.flow, 0.0, w.T, w.dt, "fp32c", phi)
    gp = autotune.params_for_gradient(dm, phi, "fp32c", w.T, cache=cache, retune=True)
    assert set(gp) <= {"grad_block", "grad_staging"}
    c = ftle.compute(dm, w.flow, w.T, w.dt, "fp32c", options=ftle.make_options(**gp)).cpu()
    assert torch.equal(a, c)
    bopt = autotune.options_for_batch(meshes, [x.flow for x in ws_list], [x.T for x in ws_list], 0.01, "fp32c",
                                      cache=cache, retune=True)
    ws = ftle.workspace_empty(ftle.ftle_batch_workspace_bytes(meshes, "fp32c"))
    ftle.ftle_batch(meshes, [x.flow for x in ws_list], [x.T for x in ws_list], 0.01, "fp32c", outs, ws)
    ref = [o.clone() for o in outs]
    ftle.ftle_batch(meshes, [x.flow for x in ws_list], [x.T for x in ws_list], 0.01, "fp32c", outs, ws, options=bopt)
    torch.cuda.synchronize()
    for o, r in zip(outs, ref):
        assert torch.equal(o, r)


@pytest.mark.parametrize("preset,T", [(1, 5.0), (2, 2.0)])
def test_forward_backward_pair_in_one_batch(preset, T):
    """compute_pair runs +T and -T as one batch: each field equals its single run and the FP64
    oracle at the same horizon."""
    import torch

    from paper_2408_02758_gb300 import ftle

    w = I.preset(preset, scale=1 / 32 if preset == 1 else 1 / 16)
    dm = ftle.DeviceMesh.from_mesh(w.mesh)
    fwd, bwd = ftle.compute_pair(dm, w.flow, T, w.dt, "fp32c")
    torch.cuda.synchronize()
    x0 = w.mesh.coords.astype(np.float64)
    for got, horizon in ((fwd, T), (bwd, -T)):
        got = got.double().cpu().numpy()
        single = ftle.compute(dm, w.flow, horizon, w.dt, "fp32c").double().cpu().numpy()
        assert np.all((got == single) | (np.abs(got - single) <= 1e-9 * np.abs(single)) | (np.isnan(got) & np.isnan(single)))
        o = O.ftle(w.flow.kind, w.flow.params, x0, w.mesh.row_ptr, w.mesh.col_idx, horizon, w.dt)
        rep = compare(got, o["ftle"], o["lam"])
        assert rep["ok"], rep


def test_full_batched_workload_every_instance_matches_oracle():
    """The 64-instance workload at full scale (lattices 64 x 32 to 1024 x 512, T in {5, 10, 15,
    20}, eps and omega over their whole ranges), replayed from the captured graph as the
    benchmark runs it: 200 sampled nodes of every instance against the oracle."""
    import torch

    from paper_2408_02758_gb300 import ftle

    wl = I.batched_preset(64)
    meshes = [ftle.DeviceMesh.from_mesh(w.mesh) for w in wl]
    outs = [torch.full((w.mesh.n_nodes,), 7.0, dtype=torch.float32, device="cuda") for w in wl]
    ws = ftle.workspace_empty(ftle.ftle_batch_workspace_bytes(meshes, "fp32c"))
    plan = ftle.BatchPlan(meshes, [w.flow for w in wl], [w.T for w in wl], 0.01, "fp32c", outs, ws)
    plan.launch()
    torch.cuda.synchronize()
    rng = np.random.default_rng(64)
    g, of, ol = [], [], []
    for q, (w, o) in enumerate(zip(wl, outs)):
        rows = np.sort(rng.choice(w.mesh.n_nodes, min(200, w.mesh.n_nodes), replace=False))
        ref = O.ftle_sample(w.flow.kind, w.flow.params, w.mesh.coords, w.mesh.row_ptr, w.mesh.col_idx, rows, w.T,
                            w.dt)
        got = o.double().cpu().numpy()
        rep = compare(got[rows], ref["ftle"], ref["lam"])
        assert rep["ok"], (q, w.name, rep)
        assert np.isfinite(got).all(), q
        g.append(got[rows])
        of.append(ref["ftle"])
        ol.append(ref["lam"])
    rep = compare(np.concatenate(g), np.concatenate(of), np.concatenate(ol))
    report("dg2d_batched_64", rep, sample="200 random nodes of each of the 64 instances", precision="fp32c",
           execution="captured graph replay")
    assert rep["ok"], rep
    # whole fields of the three instances with the most ill-conditioned ridge flanks (T = 20,
    # 512 x 256 lattices): every node within 1e-4, or within the oracle's own change under a
    # one-rounding change of a flow parameter
    for q in (24, 5, 8):
        w = wl[q]
        assert w.T == 20.0, (q, w.name, w.T)
        ref = O.ftle(w.flow.kind, w.flow.params, w.mesh.coords, w.mesh.row_ptr, w.mesh.col_idx, w.T, w.dt)
        S = float_sensitivity(O, w.flow, w.mesh, w.T, w.dt, base=ref["ftle"])
        rep = compare_conditioned(outs[q].double().cpu().numpy(), ref["ftle"], ref["lam"], S)
        report(w.name, rep, sample="every node", precision="fp32c", execution="captured graph replay",
               eps=float(w.flow.params[1]), omega=float(w.flow.params[2]), T=w.T)
        assert rep["ok"], (q, rep)
    plan.destroy()
