"""Writes oracle/iteration_counts.json: the number of FGMRES iterations the
oracle's exact-L^+ Schur solve needs at rtol 1e-8 on the first step of a
workload.  The CPU-baseline timing in bench.py times a bounded sample of the
oracle (a fixed number of iterations) and scales the per-iteration cost by
this count.  TEST/BENCH INFRASTRUCTURE ONLY; calls nothing outside oracle/ and
the input generators.

Usage: python -m oracle.iteration_count [config ...]
"""
from __future__ import annotations

import json
import os
import sys
from pathlib import Path

OUT = Path(__file__).resolve().parent / "iteration_counts.json"


def count(cfg: int, secondary: bool = True, rtol: float = 1e-8) -> int:
    from paper_2501_15314_gb300 import workloads as wl
    from . import helmholtz, mac, schur
    W = wl.config(cfg, secondary)
    g = mac.Grid(W.n)
    sys_ = schur.SchurSystem(g, W.X)
    a = 1.5 / W.dt
    workers = os.cpu_count()
    us = helmholtz.solve(g, W.f_body * g.interior_face_mask_packed(), a, 1.0 / W.Re,
                         workers=workers)
    rhs_F = a * (sys_.R.T @ us - W.U_gamma.ravel())
    b = sys_.rhs_scalar(a * mac.apply_GT(g, us), rhs_F)
    _, it, rel, _ = schur.solve_schur(sys_, b, rtol=rtol, workers=workers)
    return int(it)


if __name__ == "__main__":
    cfgs = [int(c) for c in sys.argv[1:]] or [3]
    data = json.loads(OUT.read_text()) if OUT.exists() else {}
    for c in cfgs:
        data[f"config{c}_stated_markers_rtol1e-8"] = count(c)
        print(c, data[f"config{c}_stated_markers_rtol1e-8"], flush=True)
    OUT.write_text(json.dumps(data, indent=1) + "\n")
