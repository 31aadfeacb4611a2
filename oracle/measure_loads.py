"""Run the FP64 oracle to convergence on the 128^3 diffusion workload and store the
number of block products (loads) it needed, for the CPU-baseline extrapolation of
bench.py. Test infrastructure: calls only the oracle and the input generators.

The refinement stops the way the library's FP64 path does: outer target 1e-8, inner
solves to max(1e-6, 1e-8 ||b|| / (2 ||r||)) (refined_solve with adaptive_inner), so
the oracle is charged the loads this method needs under the same stopping rule.

    python -m oracle.measure_loads   (about half an hour on eight cores)
"""
from __future__ import annotations

import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import bcg, direct, operators  # noqa: E402
from paper_2501_18717_gb300 import workloads as W  # noqa: E402


def main():
    seed, grid, l, mu, tol = W.BASE_SEED + 2, 128, 32, 1e-4, 1e-8
    rp, ci, va, d = W.diffusion_csr(seed, grid)
    b = W.normals(seed, W.STREAM_RHS, d)
    om = W.omega(W.BASE_SEED + 3, d, l)
    op = operators.CSR(rp, ci, va)
    t0 = time.time()
    out = bcg.refined_solve(op, mu, b, om, tol=tol, inner_tol=1e-6, max_loads=20000, adaptive_inner=True)
    res = direct.rel_residual(op, mu, out["x"], b)
    rec = {"workload": "diffusion 128^3, mu 1e-4, l 32, tol 1e-8",
           "stopping_rule": "outer 1e-8; inner max(1e-6, 1e-8 ||b|| / (2 ||r||)), at most 0.5",
           "loads_fp64_refined_1e-8": out["loads"], "inner_block_loads": out["inner_loads"],
           "residual_loads": out["loads"] - out["inner_loads"],
           "refinements": out["refinements"], "rel_residual": res, "seconds": time.time() - t0}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "loads_diffusion128.json"), "w") as fh:
        json.dump(rec, fh, indent=1)
    print(rec)


if __name__ == "__main__":
    main()
