"""Mesh validation (ftle_validate_mesh and ftle_options.validate_mesh): bad neighbour indices are
found by a device pass that reads the index arrays without gathering through them, and come back
as FTLE_EINVAL before any kernel reads through a bad index.

Every bad mesh here is only ever validated (or handed to an entry point that validates before
its first gather); none reaches a gradient kernel.
"""
import numpy as np
import pytest

from paper_2408_02758_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    from paper_2408_02758_gb300 import ftle

    ftle.lib()
    return ftle


def _small():
    return I.make_mesh((13, 9), (0, 0), (2, 1), I.TRI, 0.3, 41)


def _device(F, m, rp=None, ci=None):
    import torch

    return F.DeviceMesh(torch.from_numpy(np.ascontiguousarray(m.coords)).cuda(),
                        torch.from_numpy(m.row_ptr if rp is None else rp).cuda(),
                        torch.from_numpy(m.col_idx if ci is None else ci).cuda())


def test_valid_meshes_pass(F):
    for m in (_small(), I.preset(2, scale=1 / 16).mesh):
        dm = _device(F, m)
        rep = F.ftle_validate_mesh(dm)
        assert rep["status"] == F.FTLE_OK
        assert rep["bad_row_ptr"] == rep["bad_col_idx"] == rep["bad_ell_idx"] == 0
        assert rep["first_bad_col"] == -1
        dm.attach_ell()
        assert F.ftle_validate_mesh(dm)["bad_ell_idx"] == 0


@pytest.mark.parametrize("bad", [lambda n: n, lambda n: -1, lambda n: 2 ** 31 - 1])
def test_col_idx_out_of_range(F, bad):
    m = _small()
    ci = m.col_idx.copy()
    e = int(m.row_ptr[37]) + 1
    ci[e] = bad(m.n_nodes)
    ci[e + 5] = bad(m.n_nodes)
    dm = _device(F, m, ci=ci)
    rep = F.ftle_validate_mesh(dm, check=False)
    assert rep["status"] == F.FTLE_EINVAL
    assert rep["bad_col_idx"] == 2 and rep["first_bad_col"] == e
    with pytest.raises(F.FTLEError) as err:
        F.ftle_validate_mesh(dm)
    assert err.value.status == F.FTLE_EINVAL and "col_idx" in str(err.value)


def test_row_ptr_decrease_start_and_end(F):
    m = _small()
    rp = m.row_ptr.copy()
    rp[20] = rp[21] + 1  # row 19 grows past row 20's end: a decrease at row 20
    rep = F.ftle_validate_mesh(_device(F, m, rp=rp), check=False)
    assert rep["status"] == F.FTLE_EINVAL and rep["bad_row_ptr"] == 1 and rep["first_bad_row"] == 20
    rp = m.row_ptr.copy()
    rp[0] = 1
    rep = F.ftle_validate_mesh(_device(F, m, rp=rp), check=False)
    assert rep["status"] == F.FTLE_EINVAL and rep["first_bad_row"] == 0
    dm = _device(F, m)
    dm.desc.nnz = m.nnz - 3  # row_ptr[n] != nnz (only the first nnz entries of col_idx are read)
    rep = F.ftle_validate_mesh(dm, check=False)
    assert rep["status"] == F.FTLE_EINVAL and rep["bad_row_ptr"] == 1 and rep["first_bad_row"] == m.n_nodes - 1


def test_ell_out_of_range(F):
    m = _small()
    dm = _device(F, m)
    dm.attach_ell()
    n = m.n_nodes
    dm.ell[2, 5] = n
    dm.ell[0, 7] = -2
    rep = F.ftle_validate_mesh(dm, check=False)
    assert rep["status"] == F.FTLE_EINVAL and rep["bad_ell_idx"] == 2 and rep["first_bad_ell"] == 7
    assert rep["bad_col_idx"] == 0


def test_entry_points_refuse_bad_meshes_before_any_gather(F):
    """ftle_compute and ftle_gradient_eig with validate_mesh = 1, the batch with the same option,
    and ftle_compute_host (always) return FTLE_EINVAL; a valid mesh still computes."""
    import torch

    m = _small()
    flow = I.FlowSpec.double_gyre()
    ci = m.col_idx.copy()
    ci[11] = m.n_nodes
    bad = _device(F, m, ci=ci)
    opt = F.make_options(validate_mesh=True)
    phi = F.flowmap_empty(2, m.n_nodes, "fp32c")
    out = torch.full((m.n_nodes,), 5.0, device="cuda")
    ws = F.workspace_empty(F.ftle_workspace_bytes(m.n_nodes))
    with pytest.raises(F.FTLEError) as e:
        F.ftle_compute(bad, flow, 0.0, 2.0, 0.01, "fp32c", phi, out, None, ws, options=opt)
    assert e.value.status == F.FTLE_EINVAL
    good = _device(F, m)
    F.ftle_advect(good, flow, 0.0, 2.0, 0.01, "fp32c", phi)
    with pytest.raises(F.FTLEError) as e:
        F.ftle_gradient_eig(bad, phi, "fp32c", 2.0, out, None, ws, options=opt)
    assert e.value.status == F.FTLE_EINVAL
    torch.cuda.synchronize()
    assert torch.all(out == 5.0)  # nothing ran
    bws = F.workspace_empty(F.ftle_batch_workspace_bytes([good, bad], "fp32c"))
    outs = [torch.empty(m.n_nodes, device="cuda") for _ in range(2)]
    with pytest.raises(F.FTLEError) as e:
        F.ftle_batch([good, bad], [flow, flow], [2.0, 2.0], 0.01, "fp32c", outs, bws, options=opt)
    assert e.value.status == F.FTLE_EINVAL and "instance 1" in str(e.value)
    ch = torch.from_numpy(m.coords).pin_memory()
    rp = torch.from_numpy(m.row_ptr).pin_memory()
    hws = F.workspace_empty(F.ftle_host_workspace_bytes(2, m.n_nodes, m.nnz, "fp32c"))
    oh = torch.empty(m.n_nodes, dtype=torch.float32).pin_memory()
    with pytest.raises(F.FTLEError) as e:
        F.ftle_compute_host(ch, rp, torch.from_numpy(ci).pin_memory(), flow, 0.0, 2.0, 0.01, "fp32c", oh, hws)
    assert e.value.status == F.FTLE_EINVAL
    # the valid mesh through the same validating calls
    F.ftle_compute(good, flow, 0.0, 2.0, 0.01, "fp32c", phi, out, None, ws, options=opt)
    ref = F.compute(good, flow, 2.0, 0.01, "fp32c")
    torch.cuda.synchronize()
    assert torch.equal(torch.isnan(out), torch.isnan(ref)) and torch.equal(out[~torch.isnan(out)], ref[~torch.isnan(ref)])
    F.ftle_compute_host(ch, rp, torch.from_numpy(m.col_idx).pin_memory(), flow, 0.0, 2.0, 0.01, "fp32c", oh, hws)
    assert np.array_equal(oh.numpy(), ref.cpu().numpy(), equal_nan=True)


@pytest.mark.parametrize("offset", [0, 1, 2, 3])
def test_bad_entries_in_unaligned_heads_bodies_and_tails(F, offset):
    """The pass reads the index lists as 16-byte vectors from their first 16-byte boundary and the
    few entries before and after it one by one: lists starting 0-3 entries past a boundary, with
    bad entries at the first entry, inside the vectors and at the last entry, are all found, and
    the first position is reported relative to the list's own start."""
    import torch

    m = I.make_mesh((23, 17), (0, 0), (2, 1), I.TRI, 0.3, 43)
    n, nnz = m.n_nodes, m.nnz
    for where, values in (([0, 1, nnz // 2, nnz - 1], [n, -1, 2 ** 31 - 1, -5]),
                          ([nnz - 1], [n]), ([nnz // 2 + 1], [-(2 ** 31)]), ([], [])):
        ci = m.col_idx.copy()
        for e, v in zip(where, values):
            ci[e] = v
        buf = torch.zeros(nnz + 4, dtype=torch.int32, device="cuda")
        buf[offset:offset + nnz] = torch.from_numpy(ci).cuda()
        dm = F.DeviceMesh(torch.from_numpy(np.ascontiguousarray(m.coords)).cuda(),
                          torch.from_numpy(m.row_ptr).cuda(), buf[offset:offset + nnz])
        assert (dm.col_idx.data_ptr() - buf.data_ptr()) == 4 * offset
        rep = F.ftle_validate_mesh(dm, check=False)
        assert rep["bad_col_idx"] == len(where), (offset, where, rep)
        assert rep["first_bad_col"] == (min(where) if where else -1), (offset, where, rep)
        assert rep["status"] == (F.FTLE_EINVAL if where else F.FTLE_OK)
    # the fixed-width list: -1 is allowed, -2 and n are not; a list starting off a boundary
    dm = _device(F, m)
    dm.attach_ell()
    w = dm.desc.ell_width
    flat = dm.ell.reshape(-1).clone()
    L = flat.numel()
    bad = [0, L // 3, L - 1]
    for e, v in zip(bad, [-2, n, -(2 ** 31)]):
        flat[e] = v
    buf = torch.zeros(L + 4, dtype=torch.int32, device="cuda")
    buf[offset:offset + L] = flat
    dm.ell = buf[offset:offset + L].view(w, n)
    dm.desc.ell_idx = dm.ell.data_ptr()
    rep = F.ftle_validate_mesh(dm, check=False)
    assert rep["bad_ell_idx"] == 3 and rep["first_bad_ell"] == 0 and rep["bad_col_idx"] == 0, rep
