"""Writes the regression fixtures in this folder from the FP64 oracle alone.

Run from the repository root:  python tests/golden/make_golden.py
Each fixture records its inputs (preset, scale, horizon) so the test can rebuild them with the
seeded input generator; the values are oracle outputs, never values from the CUDA path.
"""
import json
import sys
from pathlib import Path

HERE = Path(__file__).resolve().parent
sys.path.insert(0, str(HERE.parent.parent))

import numpy as np  # noqa: E402

import oracle as O  # noqa: E402
from paper_2408_02758_gb300 import inputs as I  # noqa: E402

CASES = [
    {"name": "dg_tri_32x16_T2", "preset": 1, "scale": 1 / 64, "T": 2.0},
    {"name": "abc_kuhn_8_T1", "preset": 2, "scale": 1 / 32, "T": 1.0},
    {"name": "dg_struct_32x16_T10_fp64", "preset": 0, "scale": 1 / 8, "T": 10.0},
]


def compute(case):
    w = I.preset(case["preset"], scale=case["scale"])
    m = w.mesh
    out = O.ftle(w.flow.kind, w.flow.params, m.coords, m.row_ptr, m.col_idx, case["T"], w.dt)
    return out


def main():
    for case in CASES:
        out = compute(case)
        rec = dict(case)
        rec["source"] = "oracle/oracle.c (FP64), written by tests/golden/make_golden.py"
        rec["ftle"] = [float(v).hex() for v in out["ftle"]]
        rec["lam"] = [float(v).hex() for v in out["lam"]]
        (HERE / f"{case['name']}.json").write_text(json.dumps(rec, indent=0))
        print(case["name"], len(rec["ftle"]))


if __name__ == "__main__":
    main()
