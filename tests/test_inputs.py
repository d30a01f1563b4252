"""Seeded input generator: mesh structure and determinism (no GPU)."""
import math

import numpy as np
import pytest

from paper_2408_02758_gb300 import inputs as I


def _adjacency_ok(m):
    rp, ci = m.row_ptr, m.col_idx
    n = m.n_nodes
    assert rp[0] == 0 and rp[-1] == len(ci)
    assert np.all(np.diff(rp) >= 0)
    assert ci.min() >= 0 and ci.max() < n
    rows = np.repeat(np.arange(n), np.diff(rp))
    assert not np.any(rows == ci), "self loops"
    # ascending within rows
    same = rows[1:] == rows[:-1]
    assert np.all(ci[1:][same] > ci[:-1][same])
    # symmetric: set of (i, j) equals set of (j, i)
    a = rows.astype(np.int64) * n + ci
    b = ci.astype(np.int64) * n + rows
    assert np.array_equal(np.sort(a), np.sort(b))


@pytest.mark.parametrize("shape,stencil,kmax", [((7, 5), I.AXIS, 4), ((7, 5), I.TRI, 6), ((4, 5, 6), I.AXIS, 6),
                                               ((4, 5, 6), I.KUHN, 14)])
def test_csr_structure(shape, stencil, kmax):
    m = I.make_mesh(shape, (0,) * len(shape), (1,) * len(shape), stencil, 0.3, 5)
    _adjacency_ok(m)
    deg = np.diff(m.row_ptr)
    assert deg.max() == kmax
    assert deg.min() >= len(shape)


def test_kuhn_interior_offsets():
    shape = (5, 5, 5)
    m = I.make_mesh(shape, (0,) * 3, (1,) * 3, I.KUHN, 0.0, 5)
    c = 2 + 5 * 2 + 25 * 2
    nb = m.col_idx[m.row_ptr[c]:m.row_ptr[c + 1]] - c
    expect = []
    for o in [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, 0, 1), (0, 1, 1), (1, 1, 1)]:
        lin = o[0] + 5 * o[1] + 25 * o[2]
        expect += [lin, -lin]
    assert sorted(nb.tolist()) == sorted(expect)


def test_tri_interior_offsets():
    m = I.make_mesh((6, 6), (0, 0), (1, 1), I.TRI, 0.0, 5)
    c = 3 + 6 * 3
    nb = m.col_idx[m.row_ptr[c]:m.row_ptr[c + 1]] - c
    assert sorted(nb.tolist()) == sorted([1, -1, 6, -6, 7, -7])


def test_jitter_bounds_and_boundaries():
    shape = (33, 17)
    m = I.make_mesh(shape, (0, 0), (2, 1), I.TRI, 0.3, 99, coord_dtype=np.float64)
    x = m.coords.reshape(2, shape[1], shape[0])
    hx, hy = 2 / 32, 1 / 16
    gx = np.arange(shape[0]) * hx
    gy = np.arange(shape[1]) * hy
    assert np.all(np.abs(x[0] - gx[None, :]) <= 0.3 * hx + 1e-15)
    assert np.all(np.abs(x[1] - gy[:, None]) <= 0.3 * hy + 1e-15)
    assert np.all(x[0][:, 0] == 0) and np.all(x[0][:, -1] == 2)
    assert np.all(x[1][0, :] == 0) and np.all(x[1][-1, :] == 1)
    # interior nodes really move, and the draws look uniform
    d = (x[0][1:-1, 1:-1] - gx[None, 1:-1]) / (0.3 * hx)
    assert abs(d.mean()) < 0.1 and 0.25 < d.var() < 0.42


def test_determinism_and_seed_dependence():
    a = I.make_mesh((9, 9), (0, 0), (1, 1), I.TRI, 0.3, 1)
    b = I.make_mesh((9, 9), (0, 0), (1, 1), I.TRI, 0.3, 1)
    c = I.make_mesh((9, 9), (0, 0), (1, 1), I.TRI, 0.3, 2)
    assert np.array_equal(a.coords, b.coords)
    assert not np.array_equal(a.coords, c.coords)


def test_splitmix64_reference_values():
    """SplitMix64 with seed 0: first outputs as published with the generator's definition."""
    # mix64(0 + k * golden) for k = 1, 2, 3
    lib = I._load()
    lib.ftlein_draw.argtypes = [I.ctypes.c_uint64, I.ctypes.c_uint64]
    lib.ftlein_draw.restype = I.ctypes.c_uint64
    got = [lib.ftlein_draw(0, k) for k in range(3)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_presets_shapes():
    w = I.preset(1, scale=1 / 64)
    assert w.mesh.shape == (32, 16) and w.precision == "fp32c" and w.n_steps == 1500
    w0 = I.preset(0, scale=1 / 8)
    assert w0.mesh.coords.dtype == np.float64 and w0.n_steps == 1000
    w2 = I.preset(2, scale=1 / 32)
    assert w2.mesh.dim == 3 and np.diff(w2.mesh.row_ptr).max() == 14
    w4 = I.preset(4, scale=1 / 32)
    assert abs(w4.extra["weights"].sum() - 1) < 1e-12
    batch = I.batched_preset(64)
    sizes = {b.mesh.shape for b in batch}
    assert len(batch) == 64 and len(sizes) > 1
    for b in batch:
        assert b.mesh.shape[0] in (64, 128, 256, 512, 1024) and b.mesh.shape[1] == b.mesh.shape[0] // 2
        assert b.T in (5.0, 10.0, 15.0, 20.0)
        A, eps, om = b.flow.params[:3]
        assert A == 0.1 and 0 <= eps <= 0.5 and math.pi / 10 <= om <= math.pi / 2


@pytest.mark.parametrize("shape,stencil", [((7, 5), I.TRI), ((4, 5, 3), I.KUHN)])
def test_element_lists_span_the_stencil_edges(shape, stencil):
    """The element lists' edges are exactly the stencil's neighbour pairs (host check of the
    connectivity the GPU adjacency builder consumes)."""
    m = I.make_mesh(shape, (0,) * len(shape), (1,) * len(shape), stencil, 0.0, 1)
    el = I.lattice_elements(shape, stencil)
    pairs = set()
    for row in el:
        for a in row:
            for b in row:
                if a != b:
                    pairs.add((int(a), int(b)))
    rows = np.repeat(np.arange(m.n_nodes), np.diff(m.row_ptr))
    assert pairs == set(zip(rows.tolist(), m.col_idx.tolist()))


# The lattice neighbours of each stencil, as the C-ABI's ftle_stencil defines them (offsets in
# (x, y[, z]), x fastest); every CSR row must be exactly the in-range offsets in ascending order.
_STENCIL_OFFSETS = {
    (2, I.AXIS): [(1, 0), (-1, 0), (0, 1), (0, -1)],
    (2, I.TRI): [(1, 0), (-1, 0), (0, 1), (0, -1), (1, 1), (-1, -1)],
    (3, I.AXIS): [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)],
    (3, I.KUHN): [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1), (1, 1, 0), (-1, -1, 0),
                  (0, 1, 1), (0, -1, -1), (1, 0, 1), (-1, 0, -1), (1, 1, 1), (-1, -1, -1)],
}


@pytest.mark.parametrize("shape,stencil", [((5, 4), I.AXIS), ((5, 4), I.TRI), ((2, 2), I.TRI), ((4, 3, 3), I.AXIS),
                                           ((4, 3, 3), I.KUHN), ((2, 2, 2), I.KUHN)])
def test_csr_rows_are_the_implicit_stencil(shape, stencil):
    """The implicit-stencil gradient path (ftle_mesh.stencil) takes a node's neighbours from the
    lattice instead of the rows: the generated rows must be the in-range offsets, ascending."""
    rp, ci = I.lattice_csr(shape, stencil)
    dim = len(shape)
    strides = [1, shape[0], shape[0] * (shape[1] if dim > 1 else 1)]
    for i in range(int(np.prod(shape))):
        idx = [i % shape[0], (i // shape[0]) % shape[1]] + ([i // (shape[0] * shape[1])] if dim == 3 else [])
        want = sorted(sum(o[a] * strides[a] for a in range(dim)) + i for o in _STENCIL_OFFSETS[(dim, stencil)]
                      if all(0 <= idx[a] + o[a] < shape[a] for a in range(dim)))
        assert list(ci[rp[i]:rp[i + 1]]) == want, (i, idx)
