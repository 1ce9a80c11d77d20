"""Writes opcount_smooth2d.json: the oracle's operation counts per cell-stage for
the 2D smooth periodic workload (1024^2, the benchmark flow), by step of the
stage and kind of operation, from the op-counting build (opcount.cpp).

The counts are taken on the same flow at 32^2 and 64^2 and extrapolated in the
grid size (per-cell count = a + b / N: the halo of ghost nodes and cells the
oracle also evaluates shrinks as 1/N). "counted" operations are the first,
nontrivial evaluations; re-evaluations of a pure function with the same inputs
and operations with an exact 0 / +-1 operand are tallied apart (opcount.cpp).
Test infrastructure: calls only the oracle and the seeded input generators.

    python oracle/count_ops.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import oracle as O  # noqa: E402
from paper_2609_29081_b300 import workloads as W  # noqa: E402

N_TARGET = 1024
SIZES = (32, 64)


def per_cell_stage(n):
    w = W.smooth_2d(n)
    P = O.problem(2, n, n, lo=w.lo, hi=w.hi, mu=w.mu, Pr=w.Pr, bc=w.bc, gamma=w.gamma)
    step = O.opcount(P, w.state, "step")            # five residuals + combinations
    dt = O.opcount(P, w.state, "dt")                # the CFL bound, once per step
    cs = 5.0 * n * n
    return step / cs, dt / cs


def main():
    res = {n: per_cell_stage(n) for n in SIZES}
    (s1, d1), (s2, d2) = res[SIZES[0]], res[SIZES[1]]
    n1, n2 = SIZES

    def extrap(a, b):
        # per-cell count a + b / N through the two sizes, evaluated at N_TARGET
        slope = (a - b) / (1.0 / n1 - 1.0 / n2)
        return b + slope * (1.0 / N_TARGET - 1.0 / n2)

    # (a category absent at both sizes stays exactly zero; round-off of the
    # extrapolation is cut at zero)
    step = np.maximum(extrap(s1, s2) + extrap(d1, d2), 0.0)
    cats = O.OPC_CATEGORIES
    phases = {}
    for ph, name in O.OPC_PHASES.items():
        row = {c: float(step[ph, k, 0]) for k, c in enumerate(cats)}
        if sum(row.values()) == 0 and step[ph, :, 1:].sum() == 0:
            continue
        row["repeated_flops"] = float(step[ph, :5, 1].sum())
        row["trivial_flops"] = float(step[ph, :5, 2].sum())
        phases[name] = row
    flops = float(step[:, :5, 0].sum())   # add, mul, div, sqrt, transcendental
    out = {
        "workload": "2D smooth periodic NS (rho=1+0.2sin(x+y), (u,v)=(1,0.5)+8-mode perturbation, p=1, "
                    "mu=0.01, Pr=0.72), limiter s+pp, CFL step",
        "grid": N_TARGET,
        "sizes_counted": list(SIZES),
        "unit": "operations per cell-stage (one of the five SSP-RK54 stages of one cell, its 3 point "
                "values included; the CFL bound's share of a step spread over the five stages)",
        "flops_per_cell_stage": flops,
        "by_category": {c: float(step[:, k, 0].sum()) for k, c in enumerate(cats)},
        "repeated_flops_per_cell_stage": float(step[:, :5, 1].sum()),
        "trivial_flops_per_cell_stage": float(step[:, :5, 2].sum()),
        "by_phase": phases,
    }
    path = os.path.join(HERE, "opcount_smooth2d.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
    print(json.dumps({k: out[k] for k in ("flops_per_cell_stage", "by_category",
                                           "repeated_flops_per_cell_stage")}, indent=1))


if __name__ == "__main__":
    main()
