"""The host-side bounds behind the advection's unchecked rotated steps (ftle_rotation_bounds; no
GPU needed).  The kernels drop their per-step angle check when these bounds hold, so each bound
is checked here against the stage angles themselves, sampled in double precision straight from
the flows' definitions (no code of the CUDA path): every sampled angle and stage-three angle
difference must stay within the library's bound, and the bound must not be loose by more than a
factor of 2 for the angles and 10 for the differences (so the sampling reaches the regime the
bound describes; the difference bounds chain triangle inequalities and sit 2-6 times above the
sampled maxima)."""
import math

import numpy as np
import pytest

from paper_2408_02758_gb300 import inputs as I


@pytest.fixture(scope="module")
def F():
    from paper_2408_02758_gb300 import ftle

    ftle.lib()
    return ftle


def _dg_stage_angles(A, eps, om, h, x0, y0, t0):
    """Stage angles of one classic RK4 step of the double gyre from (x0, y0) at t0: for stages
    two to four, pi (f_ts(x_s) - f_t0(x0)) and pi (y_s - y0) (f_t(x) = a x^2 + (1 - 2a) x,
    a = eps sin(omega t); u = -pi A sin(pi f) cos(pi y), v = pi A cos(pi f) sin(pi y) df/dx)."""

    def a(t):
        return eps * np.sin(om * t)

    def f(t, x):
        return a(t) * x * x + (1.0 - 2.0 * a(t)) * x

    def vel(t, x, y):
        F_ = f(t, x)
        fx = 2.0 * a(t) * x + 1.0 - 2.0 * a(t)
        return (-math.pi * A * np.sin(math.pi * F_) * np.cos(math.pi * y),
                math.pi * A * np.cos(math.pi * F_) * np.sin(math.pi * y) * fx)

    u1, v1 = vel(t0, x0, y0)
    x2, y2 = x0 + 0.5 * h * u1, y0 + 0.5 * h * v1
    u2, v2 = vel(t0 + 0.5 * h, x2, y2)
    x3, y3 = x0 + 0.5 * h * u2, y0 + 0.5 * h * v2
    u3, v3 = vel(t0 + 0.5 * h, x3, y3)
    x4, y4 = x0 + h * u3, y0 + h * v3
    f0 = f(t0, x0)
    return {s: (math.pi * (f(ts, xs) - f0), math.pi * (ys - y0))
            for s, (ts, xs, ys) in {2: (t0 + 0.5 * h, x2, y2), 3: (t0 + 0.5 * h, x3, y3), 4: (t0 + h, x4, y4)}.items()}


def _abc_stage_increments(A, B, C, h, p0):
    """Stage increments of one classic RK4 step of the ABC flow (u = A sin z + C cos y,
    v = B sin x + A cos z, w = C sin y + B cos x): h/2 k1, h/2 k2 and h k3, the angles by which the
    step turns stage one's sines and cosines."""

    def vel(p):
        x, y, z = p
        return np.stack([A * np.sin(z) + C * np.cos(y), B * np.sin(x) + A * np.cos(z), C * np.sin(y) + B * np.cos(x)])

    d1 = 0.5 * h * vel(p0)
    d2 = 0.5 * h * vel(p0 + d1)
    d3 = h * vel(p0 + d2)
    return d1, d2, d3


@pytest.mark.parametrize("A,eps,om,dt", [
    (0.1, 0.25, 2 * math.pi / 10, 0.01),   # the 2D workloads' gyre
    (0.1, 0.5, math.pi / 2, 0.01),         # the batched instances' extreme forcing
    (0.1, 0.42177016, 0.98781958, 0.01),
    (0.1, 0.0, 0.0, 0.01),                 # steady gyre
    (0.1, 0.25, 2 * math.pi / 10, -0.02),  # backward time, longer step
    (0.2, 0.5, math.pi, 0.005),
])
def test_double_gyre_bounds_hold_for_sampled_stage_angles(F, A, eps, om, dt):
    b = F.ftle_rotation_bounds(I.FlowSpec.double_gyre(A, eps, om), abs(dt))
    rng = np.random.default_rng(240802758)
    n = 400_000
    x0 = rng.uniform(0.0, 2.0, n)
    y0 = rng.uniform(0.0, 1.0, n)
    x0[:5], y0[:5] = [0.0, 0.5, 1.0, 1.5, 2.0], [0.0, 1.0, 0.0, 1.0, 0.5]  # walls and corners
    t0 = rng.uniform(0.0, 40.0, n)
    ang = _dg_stage_angles(A, eps, om, dt, x0, y0, t0)
    worst_angle = max(np.abs(c).max() for s in ang for c in ang[s])
    worst_diff = max(np.abs(ang[3][q] - ang[2][q]).max() for q in range(2))
    assert worst_angle <= b["angle_bound"], (worst_angle, b)
    assert worst_diff <= b["diff_bound"], (worst_diff, b)
    assert worst_angle >= 0.5 * b["angle_bound"] and worst_diff >= 0.1 * b["diff_bound"], (worst_angle, worst_diff, b)


@pytest.mark.parametrize("A,B,C,dt", [
    (math.sqrt(3.0), math.sqrt(2.0), 1.0, 0.01),  # the 3D workload's flow
    (1.0, 1.0, 1.0, 0.02),
    (2.0, 0.5, 1.0, -0.005),
])
def test_abc_bounds_hold_for_sampled_stage_increments(F, A, B, C, dt):
    b = F.ftle_rotation_bounds(I.FlowSpec.abc(A, B, C), abs(dt))
    rng = np.random.default_rng(240802759)
    p0 = rng.uniform(0.0, 2 * math.pi, (3, 400_000))
    d1, d2, d3 = _abc_stage_increments(A, B, C, dt, p0)
    worst_angle = max(np.abs(d).max() for d in (d1, d2, d3))
    worst_diff = np.abs(d2 - d1).max()
    assert worst_angle <= b["angle_bound"], (worst_angle, b)
    assert worst_diff <= b["diff_bound"], (worst_diff, b)
    assert worst_angle >= 0.5 * b["angle_bound"] and worst_diff >= 0.1 * b["diff_bound"], (worst_angle, worst_diff, b)


def _abc_step_increment(A, B, C, h, p0):
    """The RK4 increment h/6 (k1 + 2 k2 + 2 k3 + k4) of one ABC step and the stage-four increment
    h k3."""

    def vel(p):
        x, y, z = p
        return np.stack([A * np.sin(z) + C * np.cos(y), B * np.sin(x) + A * np.cos(z), C * np.sin(y) + B * np.cos(x)])

    k1 = vel(p0)
    k2 = vel(p0 + 0.5 * h * k1)
    k3 = vel(p0 + 0.5 * h * k2)
    k4 = vel(p0 + h * k3)
    return h / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4), h * k3


@pytest.mark.parametrize("A,B,C,dt", [
    (math.sqrt(3.0), math.sqrt(2.0), 1.0, 0.01),
    (1.0, 1.0, 1.0, 0.02),
    (2.0, 0.5, 1.0, -0.005),
])
def test_abc_carried_turn_is_third_order_and_within_the_difference_bound(F, A, B, C, dt):
    """A carried ABC step takes the next step's stage-one pairs from stage four's, turned to first
    order by inc - h k3.  That angle is third order in h (its first- and second-order terms
    cancel), bounded by h^2 L U / 6 (1 + hL/2 + (hL)^2 / 8) with L = U the largest pair sum, and
    so stays within the stage-three difference bound the host already checks."""
    b = F.ftle_rotation_bounds(I.FlowSpec.abc(A, B, C), abs(dt))
    U = max(A + C, B + A, C + B)
    h = abs(dt)
    rng = np.random.default_rng(240802760)
    p0 = rng.uniform(0.0, 2 * math.pi, (3, 400_000))
    worst = []
    for scale in (1.0, 0.5):
        inc, d3 = _abc_step_increment(A, B, C, dt * scale, p0)
        worst.append(np.abs(inc - d3).max())
    hs = h
    bound = hs * hs * U * U / 6.0 * (1.0 + hs * U / 2.0 + (hs * U) ** 2 / 8.0)
    assert worst[0] <= bound <= b["diff_bound"], (worst, bound, b)
    assert worst[0] / worst[1] > 7.0, worst  # third order: halving h divides it by ~8
    assert worst[0] < 0.05 * b["diff_bound"], (worst, b)


def test_carry_decision(F):
    """The ABC step carries stage one's pairs only while the step's angle bound stays within
    0.032 rad (its shorter stage-four turn then drops less than 4.4e-8): the 3D workload's step
    carries, a longer unchecked step does not, and the double gyre never does."""
    d = F.ftle_rotation_bounds(I.FlowSpec.abc(), 0.01)
    assert d["unchecked"] and d["carried"] and d["angle_bound"] < 0.032
    longer = F.ftle_rotation_bounds(I.FlowSpec.abc(), 0.011)
    assert longer["unchecked"] and not longer["carried"] and longer["angle_bound"] > 0.032
    edge = F.ftle_rotation_bounds(I.FlowSpec.abc(2.0, 0.5, 1.0), 0.01)  # angle bound 0.03
    assert edge["unchecked"] and edge["carried"]
    assert not F.ftle_rotation_bounds(I.FlowSpec.abc(), 0.02)["carried"]  # checked step
    assert not F.ftle_rotation_bounds(I.FlowSpec.double_gyre(), 0.01)["carried"]


def test_unchecked_decision_and_validation(F):
    dg = F.ftle_rotation_bounds(I.FlowSpec.double_gyre(), 0.01)
    assert dg["unchecked"] and dg["angle_bound"] < dg["angle_limit"] and dg["diff_bound"] < dg["diff_limit"]
    # eps = 0.5, omega = pi/2: the stage-three differences (3.6e-4) exceed the first-order turn's limit
    strong = F.ftle_rotation_bounds(I.FlowSpec.double_gyre(0.1, 0.5, math.pi / 2), 0.01)
    assert not strong["unchecked"] and strong["diff_bound"] > strong["diff_limit"]
    assert F.ftle_rotation_bounds(I.FlowSpec.abc(), 0.01)["unchecked"]
    assert not F.ftle_rotation_bounds(I.FlowSpec.abc(), 0.02)["unchecked"]  # angles up to 0.063
    sad = F.ftle_rotation_bounds(I.FlowSpec.saddle(), 0.01)
    assert not sad["unchecked"] and math.isinf(sad["angle_bound"])
    assert 0.0499 < dg["angle_limit"] < 0.05 and 2.99e-4 < dg["diff_limit"] < 3e-4
    for bad_dt in (0.0, math.inf, math.nan):
        with pytest.raises(F.FTLEError):
            F.ftle_rotation_bounds(I.FlowSpec.abc(), bad_dt)
