"""Pins of the FP64 oracle against what the mathematics fixes (no GPU).

Each test checks the oracle against something other than itself: closed forms of RK4 on linear
flows, brute-force central differences, library routines on special cases, high-precision
arithmetic (mpmath), an independent high-order integrator, the stream function / Beltrami
property of the flows, and finite differences.  A dropped term, wrong sign, wrong index or
transposed operand anywhere in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2408_02758_gb300 import inputs as I


def rk4_poly(z):
    """Stability polynomial of classic RK4 (exact one-step map of u' = lambda u)."""
    return 1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24


def rk4_matrix(M, h):
    Z = h * np.asarray(M, dtype=np.float64)
    E = np.eye(Z.shape[0])
    return E + Z + Z @ Z / 2 + Z @ Z @ Z / 6 + Z @ Z @ Z @ Z / 24


# ----------------------------------------------------------------------------- flows


def test_double_gyre_matches_stream_function():
    """u = -d psi/dy, v = d psi/dx with psi = A sin(pi f(x,t)) sin(pi y) (the flow's definition)."""
    A, eps, om = 0.1, 0.25, 2 * math.pi / 10
    rng = np.random.default_rng(3)

    def psi(x, y, t):
        s = math.sin(om * t)
        f = eps * s * x * x + (1 - 2 * eps * s) * x
        return A * math.sin(math.pi * f) * math.sin(math.pi * y)

    d = 1e-6
    for _ in range(20):
        x, y, t = rng.uniform(0, 2), rng.uniform(0, 1), rng.uniform(0, 20)
        u = O.velocity(O.DOUBLE_GYRE, [A, eps, om], t, [x, y])
        u_ref = -(psi(x, y + d, t) - psi(x, y - d, t)) / (2 * d)
        v_ref = (psi(x + d, y, t) - psi(x - d, y, t)) / (2 * d)
        assert abs(u[0] - u_ref) < 1e-8 and abs(u[1] - v_ref) < 1e-8


def test_double_gyre_boundaries_are_invariant():
    p = [0.1, 0.25, 2 * math.pi / 10]
    for t in (0.0, 1.3, 7.7):
        for s in np.linspace(0, 1, 7):
            assert abs(O.velocity(O.DOUBLE_GYRE, p, t, [0.0, s])[0]) < 1e-15
            assert abs(O.velocity(O.DOUBLE_GYRE, p, t, [2.0, s])[0]) < 1e-14
            assert abs(O.velocity(O.DOUBLE_GYRE, p, t, [2 * s, 0.0])[1]) < 1e-15
            assert abs(O.velocity(O.DOUBLE_GYRE, p, t, [2 * s, 1.0])[1]) < 1e-14


def _num_jac(fun, x, d=1e-6):
    x = np.asarray(x, dtype=np.float64)
    J = np.zeros((x.size, x.size))
    for b in range(x.size):
        e = np.zeros_like(x)
        e[b] = d
        J[:, b] = (fun(x + e) - fun(x - e)) / (2 * d)
    return J


def test_abc_is_beltrami_and_divergence_free():
    """The ABC flow satisfies curl u = u and div u = 0."""
    p = [math.sqrt(3), math.sqrt(2), 1.0]
    rng = np.random.default_rng(4)
    for _ in range(20):
        x = rng.uniform(-3, 9, size=3)
        J = _num_jac(lambda z: O.velocity(O.ABC, p, 0.0, z), x)
        curl = np.array([J[2, 1] - J[1, 2], J[0, 2] - J[2, 0], J[1, 0] - J[0, 1]])
        u = O.velocity(O.ABC, p, 0.0, x)
        assert np.allclose(curl, u, atol=1e-8)
        assert abs(np.trace(J)) < 1e-8


def test_double_gyre_divergence_free():
    p = [0.1, 0.25, 2 * math.pi / 10]
    rng = np.random.default_rng(5)
    for _ in range(20):
        x = np.array([rng.uniform(0, 2), rng.uniform(0, 1)])
        t = rng.uniform(0, 15)
        J = _num_jac(lambda z: O.velocity(O.DOUBLE_GYRE, p, t, z), x)
        assert abs(np.trace(J)) < 1e-8


def test_double_gyre_derivatives_match_finite_differences():
    """Analytic Jacobian and d/d(A, eps, omega) used by the tangent-linear gradient."""
    p = np.array([0.1, 0.25, 2 * math.pi / 10])
    rng = np.random.default_rng(6)
    d = 1e-6
    for _ in range(20):
        x = np.array([rng.uniform(0, 2), rng.uniform(0, 1)])
        t = rng.uniform(0, 15)
        J, P = O.dg_derivs(p, t, x)
        Jn = _num_jac(lambda z: O.velocity(O.DOUBLE_GYRE, p, t, z), x)
        assert np.allclose(J, Jn, atol=1e-8)
        for q in range(3):
            e = np.zeros(3)
            e[q] = d
            Pn = (O.velocity(O.DOUBLE_GYRE, p + e, t, x) - O.velocity(O.DOUBLE_GYRE, p - e, t, x)) / (2 * d)
            assert np.allclose(P[:, q], Pn, atol=1e-8)


# ----------------------------------------------------------------------------- RK4


@pytest.mark.parametrize("dim", [2, 3])
def test_linear_flow_flowmap_is_rk4_polynomial_power(dim):
    """For u = M x, n RK4 steps map x0 to p(hM)^n x0 exactly (up to rounding)."""
    rng = np.random.default_rng(7 + dim)
    M = rng.normal(size=(dim, dim)) * 0.4
    x0 = rng.uniform(-1, 1, size=(dim, 50))
    T, dt = 2.0, 0.01
    phi = O.advect(O.LINEAR, M.reshape(-1), x0, T, dt)
    P = np.linalg.matrix_power(rk4_matrix(M, dt), 200)
    assert np.allclose(phi, P @ x0, rtol=0, atol=1e-12)
    # backward time: steps of -dt
    phib = O.advect(O.LINEAR, M.reshape(-1), x0, -T, dt)
    Pb = np.linalg.matrix_power(rk4_matrix(M, -dt), 200)
    assert np.allclose(phib, Pb @ x0, rtol=0, atol=1e-12)


def test_linear_flow_close_to_matrix_exponential():
    """RK4 global error is O(T h^4): the flowmap approaches expm(M T)."""
    from scipy.linalg import expm

    M = np.array([[0.3, 1.2], [-0.4, -0.3]])
    x0 = np.array([[0.3, -0.7], [0.5, 0.2]])
    T = 3.0
    errs = []
    for dt in (0.1, 0.05):
        phi = O.advect(O.LINEAR, M.reshape(-1), x0, T, dt)
        errs.append(np.abs(phi - expm(M * T) @ x0).max())
    assert errs[0] < 1e-4
    assert 12 < errs[0] / errs[1] < 20  # fourth order


def test_rk4_stage_times_against_high_order_integrator():
    """Non-autonomous double gyre: converges at fourth order to DOP853 with tight tolerance.
    Wrong stage times (all at t_k, say) would make the scheme first or second order."""
    from scipy.integrate import solve_ivp

    p = [0.1, 0.25, 2 * math.pi / 10]
    rng = np.random.default_rng(8)
    x0 = np.stack([rng.uniform(0.1, 1.9, 6), rng.uniform(0.1, 0.9, 6)])
    T = 5.0
    ref = np.empty_like(x0)
    for i in range(x0.shape[1]):
        sol = solve_ivp(lambda t, z: O.velocity(O.DOUBLE_GYRE, p, t, z), (0, T), x0[:, i], method="DOP853",
                        rtol=1e-13, atol=1e-14)
        ref[:, i] = sol.y[:, -1]
    e1 = np.abs(O.advect(O.DOUBLE_GYRE, p, x0, T, 0.1) - ref).max()
    e2 = np.abs(O.advect(O.DOUBLE_GYRE, p, x0, T, 0.05) - ref).max()
    assert e1 < 1e-5
    assert 12 < e1 / e2 < 20


# ----------------------------------------------------------------------------- least squares


def _struct_mesh(shape, stencil=I.AXIS):
    lo = (0.0,) * len(shape)
    hi = tuple(float(s - 1) * 0.5 for s in shape)  # spacing 0.5
    return I.make_mesh(shape, lo, hi, stencil, 0.0, 1, coord_dtype=np.float64)


@pytest.mark.parametrize("shape", [(4, 4), (3, 3, 3)])
def test_gradient_is_central_difference_on_structured_grid(shape):
    """On an axis-stencil lattice the least-squares gradient is the central difference inside
    and the one-sided difference along an axis where one neighbour is missing (brute force)."""
    m = _struct_mesh(shape)
    dim = len(shape)
    rng = np.random.default_rng(9)
    phi = rng.normal(size=(dim, m.n_nodes))
    out = O.ftle_field(m.coords, m.row_ptr, m.col_idx, phi, 1.0, want_F=True)
    hsp = 0.5
    strides = [int(np.prod(shape[:d])) for d in range(dim)]
    for i in range(m.n_nodes):
        idx = [(i // strides[d]) % shape[d] for d in range(dim)]
        F = np.zeros((dim, dim))
        for d in range(dim):
            lo_ok, hi_ok = idx[d] > 0, idx[d] < shape[d] - 1
            if lo_ok and hi_ok:
                F[:, d] = (phi[:, i + strides[d]] - phi[:, i - strides[d]]) / (2 * hsp)
            elif hi_ok:
                F[:, d] = (phi[:, i + strides[d]] - phi[:, i]) / hsp
            else:
                F[:, d] = (phi[:, i] - phi[:, i - strides[d]]) / hsp
        assert np.allclose(out["F"][i], F, atol=1e-12), i


def test_gradient_matches_lstsq_on_jittered_neighbourhoods():
    m = I.make_mesh((5, 5, 5), (0, 0, 0), (1, 1, 1), I.KUHN, 0.25, 11)
    rng = np.random.default_rng(10)
    phi = rng.normal(size=(3, m.n_nodes))
    x = m.coords.astype(np.float64)
    out = O.ftle_field(x, m.row_ptr, m.col_idx, phi, 1.0, want_F=True)
    for i in range(m.n_nodes):
        nb = m.col_idx[m.row_ptr[i]:m.row_ptr[i + 1]]
        X = (x[:, nb] - x[:, [i]]).T
        P = (phi[:, nb] - phi[:, [i]]).T
        Ft, *_ = np.linalg.lstsq(X, P, rcond=None)
        assert np.allclose(out["F"][i], Ft.T, atol=1e-10)


@pytest.mark.parametrize("stencil,shape", [(I.TRI, (9, 7)), (I.KUHN, (5, 4, 4)), (I.AXIS, (6, 5))])
def test_linear_flowmap_gives_exact_gradient_and_ftle(stencil, shape):
    """For a linear flow the least-squares fit is exact on every rank-d neighbourhood (interior
    and boundary), so FTLE = ln sigma_max(p(hM)^n) / |T| on every node."""
    dim = len(shape)
    rng = np.random.default_rng(12)
    M = np.triu(rng.normal(size=(dim, dim))) * 0.5  # non-normal
    m = I.make_mesh(shape, (0,) * dim, (1,) * dim, stencil, 0.3, 13)
    T, dt = 1.5, 0.01
    out = O.ftle(O.LINEAR, M.reshape(-1), m.coords, m.row_ptr, m.col_idx, T, dt, want_F=True)
    P = np.linalg.matrix_power(rk4_matrix(M, dt), 150)
    smax = np.linalg.svd(P, compute_uv=False)[0]
    assert np.allclose(out["F"], P[None], atol=1e-9)
    assert np.allclose(out["ftle"], math.log(smax) / T, rtol=1e-10, atol=0)
    assert np.allclose(out["lam"], smax ** 2, rtol=1e-10)


@pytest.mark.parametrize("T", [3.0, -3.0])
def test_saddle_ftle_is_log_amplification_everywhere(T):
    """u = (x, -y): F = diag(r^n, s^n), lambda_max = p(|h|)^{2n}, FTLE = ln p(|h|) / |h| ~ 1."""
    m = I.make_mesh((16, 8), (0, 0), (2, 1), I.TRI, 0.3, 14)
    dt = 0.01
    out = O.ftle(O.SADDLE, [], m.coords, m.row_ptr, m.col_idx, T, dt)
    expect = math.log(rk4_poly(dt)) / dt
    assert np.allclose(out["ftle"], expect, rtol=1e-12, atol=0)
    assert abs(expect - 1.0) < 1e-9
    m3 = I.make_mesh((4, 4, 4), (0, 0, 0), (1, 1, 1), I.KUHN, 0.25, 15)
    out3 = O.ftle(O.SADDLE, [], m3.coords, m3.row_ptr, m3.col_idx, T, dt)
    assert np.allclose(out3["ftle"], expect, rtol=1e-12, atol=0)


# ----------------------------------------------------------------------------- eigenvalues


def test_jacobi_2x2_closed_form_and_random_3x3():
    rng = np.random.default_rng(16)
    for _ in range(50):
        a, b, c = rng.normal(size=3)
        w, V = O.jacobi(np.array([[a, b], [b, c]]))
        lmax = (a + c) / 2 + math.sqrt(((a - c) / 2) ** 2 + b * b)
        assert abs(max(w) - lmax) < 1e-13 * (1 + abs(lmax))
    for _ in range(50):
        B = rng.normal(size=(3, 3))
        A = B + B.T
        w, V = O.jacobi(A)
        assert np.allclose(np.sort(w), np.linalg.eigvalsh(A), atol=1e-12)
        assert np.allclose(A @ V, V * w[None, :], atol=1e-12)
        assert np.allclose(V.T @ V, np.eye(3), atol=1e-12)


def test_mu_keeps_relative_accuracy_near_isotropy():
    """mu = lambda_max(F^T F) - 1 for F = Q (I + delta S): compare with 50-digit arithmetic."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    rng = np.random.default_rng(17)
    for delta in (1e-3, 1e-6, 1e-9):
        th = rng.uniform(0, 2 * math.pi)
        Q = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
        S = rng.normal(size=(2, 2))
        F = Q @ (np.eye(2) + delta * S)
        # lay F out as a linear flowmap on a tiny star stencil: phi = F x
        x = np.array([[0.0, 1.0, -1.0, 0.0, 0.0, 0.5], [0.0, 0.0, 0.0, 1.0, -1.0, 0.5]])
        phi = F @ x
        rp = np.array([0, 5, 5, 5, 5, 5, 5], dtype=np.int32)
        ci = np.array([1, 2, 3, 4, 5], dtype=np.int32)
        out = O.ftle_field(x, rp, ci, phi, 1.0, want_F=True)
        Fo = out["F"][0]
        Fm = mpmath.matrix(Fo.tolist())
        Cm = Fm.T * Fm
        ev = mpmath.eigsy(Cm)[0]
        mu_ref = float(max(ev[0], ev[1]) - 1)
        # FP64 bound: a few ulp(1) absolute on C - I, i.e. ~1e-15, never relative to C itself
        assert abs(out["mu"][0] - mu_ref) <= 1e-9 * abs(mu_ref) + 1e-15
        assert abs(math.log1p(mu_ref) / 2 - out["ftle"][0]) <= 1e-9 * abs(math.log1p(mu_ref) / 2) + 1e-15


# ----------------------------------------------------------------------------- invariants


def test_incompressible_flowmap_has_unit_jacobian_determinant():
    """Double gyre is divergence-free, so det(d phi/d x0) = 1; on lattices the central-difference
    gradient approaches it at second order in the spacing."""
    p = [0.1, 0.25, 2 * math.pi / 10]
    errs = []
    for n in (17, 33):
        m = I.make_mesh((2 * n - 1, n), (0.5, 0.25), (1.5, 0.75), I.AXIS, 0.0, 1, coord_dtype=np.float64)
        out = O.ftle(O.DOUBLE_GYRE, p, m.coords, m.row_ptr, m.col_idx, 2.0, 0.01, want_F=True)
        det = np.linalg.det(out["F"])
        inner = [(2 * n - 1) * (n // 2) + (n - 1)]  # the centre node (1.0, 0.5)
        errs.append(abs(det[inner[0]] - 1))
    assert errs[1] < errs[0] / 3


def test_double_gyre_nodes_on_walls_stay_on_walls():
    p = [0.1, 0.25, 2 * math.pi / 10]
    x0 = np.array([[0.0, 2.0, 0.7, 1.3], [0.4, 0.6, 0.0, 1.0]])
    phi = O.advect(O.DOUBLE_GYRE, p, x0, 10.0, 0.01)
    assert phi[0, 0] == 0.0 and abs(phi[0, 1] - 2.0) < 1e-12
    assert phi[1, 2] == 0.0 and abs(phi[1, 3] - 1.0) < 1e-12


def test_degenerate_neighbourhoods_give_nan_and_flag():
    # node 0: collinear neighbours; node 1: single neighbour; node 2: none; node 3: fine
    x = np.array([[0.0, 1.0, 2.0, 0.0, 1.0], [0.0, 0.0, 0.0, 1.0, 1.0]])
    rp = np.array([0, 2, 3, 3, 6, 6], dtype=np.int32)
    ci = np.array([1, 2, 0, 0, 1, 4], dtype=np.int32)
    phi = 2.0 * x
    out = O.ftle_field(x, rp, ci, phi, 1.0)
    assert np.isnan(out["ftle"][:3]).all() and (out["flags"][:3] == 1).all()
    assert out["n_degenerate"] == 4  # node 4 has no neighbours either
    assert abs(out["ftle"][3] - math.log(2.0)) < 1e-14


# ----------------------------------------------------------------------------- gradient


def test_tangent_linear_gradient_matches_central_differences():
    m = I.make_mesh((24, 12), (0, 0), (2, 1), I.TRI, 0.3, 18)
    p = np.array([0.1, 0.25, 2 * math.pi / 10])
    x0 = m.coords.astype(np.float64)
    region = ((x0[0] >= 0.5) & (x0[0] <= 1.5)).astype(np.float64)
    w = region / region.sum()
    T, dt = 4.0, 0.02
    g, ft = O.param_grad(x0, m.row_ptr, m.col_idx, p, T, dt, w)
    def central(q, h):
        e = np.zeros(3)
        e[q] = h
        fp = O.ftle(O.DOUBLE_GYRE, p + e, x0, m.row_ptr, m.col_idx, T, dt)["ftle"]
        fm = O.ftle(O.DOUBLE_GYRE, p - e, x0, m.row_ptr, m.col_idx, T, dt)["ftle"]
        return (w @ fp - w @ fm) / (2 * h)

    for q in range(3):
        f1, f2 = central(q, 1e-4), central(q, 5e-5)
        # central differences carry an h^2 truncation term; Richardson removes it
        rich = (4 * f2 - f1) / 3
        assert abs(g[q] - f1) <= 1e-5 * max(1.0, abs(g[q])), (q, g[q], f1)
        assert abs(g[q] - rich) <= 1e-8 * max(1.0, abs(g[q])), (q, g[q], rich)
    f0 = O.ftle(O.DOUBLE_GYRE, p, x0, m.row_ptr, m.col_idx, T, dt)["ftle"]
    assert np.allclose(ft, f0, rtol=1e-13, atol=0)


def test_submesh_sampling_reproduces_full_field():
    w = I.preset(1, scale=1 / 64)  # 32 x 16 jittered triangle mesh, same structure
    m = w.mesh
    full = O.ftle(w.flow.kind, w.flow.params, m.coords, m.row_ptr, m.col_idx, 2.0, w.dt)["ftle"]
    rows = np.array([0, 5, 17, 100, m.n_nodes - 1])
    s = O.ftle_sample(w.flow.kind, w.flow.params, m.coords, m.row_ptr, m.col_idx, rows, 2.0, w.dt)
    assert np.array_equal(s["ftle"], full[rows])


# ----------------------------------------------------------------------------- regression


@pytest.mark.parametrize("name", ["dg_tri_32x16_T2", "abc_kuhn_8_T1", "dg_struct_32x16_T10_fp64"])
def test_oracle_reproduces_golden_fixture(name):
    """Guards the oracle against silent change: fixtures written by tests/golden/make_golden.py."""
    import json
    from pathlib import Path

    rec = json.loads((Path(__file__).parent / "golden" / f"{name}.json").read_text())
    w = I.preset(rec["preset"], scale=rec["scale"])
    out = O.ftle(w.flow.kind, w.flow.params, w.mesh.coords, w.mesh.row_ptr, w.mesh.col_idx, rec["T"], w.dt)
    ref = np.array([float.fromhex(v) for v in rec["ftle"]])
    assert np.allclose(out["ftle"], ref, rtol=1e-12, atol=1e-15)
