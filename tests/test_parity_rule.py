"""The comparison rule itself (host only): plain tolerance, NaN agreement, and the conditioning
allowance, on synthetic fields with planted errors."""
import numpy as np

from _parity import compare, compare_conditioned


def test_compare_gates_relative_error_on_stretched_nodes():
    o = np.array([0.5, 0.2, 1e-6, np.nan])
    lam = np.array([3.0, 2.0, 1.0000001, np.nan])
    g = o * np.array([1 + 5e-5, 1 - 2e-4, 1 + 0.5, 1.0])
    rep = compare(g, o, lam)
    assert rep["n_gated"] == 2 and not rep["ok"] and abs(rep["max_rel"] - 2e-4) < 1e-12
    g[1] = o[1] * (1 - 5e-5)
    assert compare(g, o, lam)["ok"]  # the ungated node's absolute error is tiny
    g[3] = 0.1
    assert compare(g, o, lam)["nan_mismatch"] == 1


def test_conditioned_rule_allows_only_the_sensitivity():
    o = np.full(5, 0.3)
    lam = np.full(5, 10.0)
    S = np.array([1e-6, 1e-6, 5e-4, 5e-4, 1e-6])
    g = o * (1 + np.array([5e-5, -9e-5, 4e-4, -1e-4, 0.0]))
    rep = compare_conditioned(g, o, lam, S)
    assert rep["ok"] and rep["n_over_tol"] == 1 and rep["n_over_tol_beyond_S"] == 0
    assert abs(rep["max_rel_well_conditioned"] - 9e-5) < 1e-12
    g[2] = o[2] * (1 + 6e-4)  # past its own sensitivity
    rep = compare_conditioned(g, o, lam, S)
    assert not rep["ok"] and rep["n_over_tol_beyond_S"] == 1
    g[2] = o[2]
    g[0] = o[0] * (1 + 2e-4)  # a well-conditioned node past 1e-4
    assert not compare_conditioned(g, o, lam, S)["ok"]
