"""Comparison rule for FTLE fields against the FP64 oracle.

Tolerance: relative error <= 1e-4 on nodes where the oracle's lambda_max > 1 + 1e-3; on the other
nodes the absolute error must stay <= 1e-4 * max|FTLE_oracle|.  NaN (rank-deficient
neighbourhoods) must coincide exactly.
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
