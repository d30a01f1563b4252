"""Comparison rule for FTLE fields against the FP64 oracle.

Tolerance: relative error <= 1e-4 on nodes where the oracle's lambda_max > 1 + 1e-3; on the other
nodes the absolute error must stay <= 1e-4 * max|FTLE_oracle|.  NaN (rank-deficient
neighbourhoods) must coincide exactly.

Conditioning (compare_conditioned): on long double-gyre horizons a few nodes sit on the steep
flanks of FTLE ridges, where the oracle's own FTLE moves by more than 1e-4 relative when a flow
parameter moves by one float rounding (2^-24 relative).  No computation whose data pass through
float can be held to 1e-4 there; such a node is held to its sensitivity S instead (the largest
relative change of the oracle's FTLE over the three one-rounding perturbations of A, eps and
omega), and every other node to 1e-4.
"""
import json
import os

import numpy as np

REL_TOL = 1e-4
LAM_GATE = 1e-3


def compare(gpu_ftle, orc_ftle, orc_lam, rel_tol=REL_TOL, abs_frac=1e-4):
    g = np.asarray(gpu_ftle, dtype=np.float64)
    o = np.asarray(orc_ftle, dtype=np.float64)
    lam = np.asarray(orc_lam, dtype=np.float64)
    nan_o, nan_g = np.isnan(o), np.isnan(g)
    rep = {"n": int(o.size), "nan_mismatch": int(np.sum(nan_o != nan_g))}
    ok = ~nan_o & ~nan_g
    gate = ok & (lam > 1 + LAM_GATE)
    rest = ok & ~gate
    rel = np.abs(g[gate] - o[gate]) / np.abs(o[gate]) if gate.any() else np.zeros(0)
    scale = np.nanmax(np.abs(o)) if ok.any() else 0.0
    absd = np.abs(g[rest] - o[rest]) if rest.any() else np.zeros(0)
    rep.update({
        "n_gated": int(gate.sum()),
        "max_rel": float(rel.max()) if rel.size else 0.0,
        "p99_rel": float(np.quantile(rel, 0.99)) if rel.size else 0.0,
        "pass_frac": float(np.mean(rel <= rel_tol)) if rel.size else 1.0,
        "max_abs": float(np.max(np.abs(g[ok] - o[ok]))) if ok.any() else 0.0,
        "max_abs_ungated": float(absd.max()) if absd.size else 0.0,
        "abs_limit": float(abs_frac * scale),
    })
    rep["ok"] = (rep["nan_mismatch"] == 0 and rep["max_rel"] <= rel_tol and rep["max_abs_ungated"] <= abs_frac * scale)
    return rep


def report(workload: str, rep: dict, **extra) -> None:
    """One line of the per-workload error table: printed (pytest -s shows it) and, when the
    FTLE_ERROR_TABLE environment variable names a file, appended to it as JSON."""
    keep = ("n", "n_gated", "max_abs", "max_rel", "p99_rel", "pass_frac", "max_abs_ungated", "abs_limit",
            "nan_mismatch", "ok")
    line = json.dumps({"workload": workload, **{k: rep[k] for k in keep if k in rep}, **extra},
                      default=lambda v: v.item() if hasattr(v, "item") else str(v))
    print("ERROR-TABLE", line)
    path = os.environ.get("FTLE_ERROR_TABLE")
    if path:
        with open(path, "a") as fh:
            fh.write(line + "\n")


def float_sensitivity(oracle, flow, mesh, T, dt, rows=None, base=None):
    """S per node (or per sampled row): the largest relative change of the oracle's FTLE when A,
    eps or omega is multiplied by 1 + 2^-24 (zero parameters are left alone)."""
    x0 = np.asarray(mesh.coords, dtype=np.float64)

    def field(params):
        if rows is None:
            return oracle.ftle(flow.kind, params, x0, mesh.row_ptr, mesh.col_idx, T, dt)["ftle"]
        return oracle.ftle_sample(flow.kind, params, mesh.coords, mesh.row_ptr, mesh.col_idx, rows, T, dt)["ftle"]

    f0 = field(flow.params) if base is None else base
    S = np.zeros_like(f0)
    for q in range(3):
        if flow.params[q] == 0.0:
            continue
        p = np.array(flow.params, dtype=np.float64)
        p[q] *= 1.0 + 2.0 ** -24
        S = np.maximum(S, np.abs(field(p) - f0) / np.abs(f0))
    return S


def compare_conditioned(gpu_ftle, orc_ftle, orc_lam, S, rel_tol=REL_TOL):
    """compare() with the gated nodes held to max(rel_tol, S) instead of rel_tol; adds how many
    nodes needed the conditioning allowance and how far past rel_tol they went."""
    rep = compare(gpu_ftle, orc_ftle, orc_lam, rel_tol)
    g = np.asarray(gpu_ftle, dtype=np.float64)
    o = np.asarray(orc_ftle, dtype=np.float64)
    lam = np.asarray(orc_lam, dtype=np.float64)
    gate = ~np.isnan(o) & ~np.isnan(g) & (lam > 1 + LAM_GATE)
    rel = np.where(gate, np.abs(g - o) / np.where(gate, np.abs(o), 1.0), 0.0)
    over = gate & (rel > rel_tol)
    rep["n_over_tol"] = int(over.sum())
    rep["n_over_tol_beyond_S"] = int((over & (rel > S)).sum())
    rep["S_at_over_tol_min"] = float(S[over].min()) if over.any() else None
    rep["max_rel_well_conditioned"] = float(rel[gate & (S <= rel_tol)].max()) if (gate & (S <= rel_tol)).any() else 0.0
    rep["ok"] = (rep["nan_mismatch"] == 0 and rep["n_over_tol_beyond_S"] == 0
                 and rep["max_abs_ungated"] <= rep["abs_limit"])
    return rep
