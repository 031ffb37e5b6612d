"""bench.py's comparison of a GPU step result with the oracle's: relative
2-norm, largest element difference over the largest oracle element, and the
same restricted to the shell cells (cells next to a face in the support of R)
and shell faces (the support of R).  An error planted only on one shell cell
must show in the shell figure at full size while the 2-norm dilutes it."""
import sys
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent.parent


def _bench():
    sys.path.insert(0, str(ROOT))
    import bench
    return bench


def _ref():
    from oracle import mac, step
    from paper_2501_15314_gb300 import workloads as wl
    W = wl.spheres_workload("t", 16, 100, 0.01, [[0.5] * 3], [0.25], None, 5)
    g = mac.Grid(16)
    return g, step.step(g, W.Re, W.dt, W.X, W.U_gamma, W.f_body)


def test_identical_results_give_zero_errors():
    bench = _bench()
    g, ref = _ref()
    err = bench.oracle_errors(ref, {k: ref[k].copy() for k in ("u", "p", "F")})
    for key in ("u", "p", "F"):
        assert all(v == 0.0 for v in err[key].values()), err
    assert "shell_max_abs_rel" in err["u"] and "shell_max_abs_rel" in err["p"]


def test_shell_cells_are_the_neighbours_of_the_support_of_R():
    # a perturbation on a cell far from the sphere leaves the shell figure at
    # zero; one on a cell next to a support face shows in it undiluted
    bench = _bench()
    g, ref = _ref()
    sysm = ref["sys"]
    got = {k: ref[k].copy() for k in ("u", "p", "F")}
    pmax = np.abs(ref["p"]).max()
    corner = 0                                     # cell (0, 0, 0): far from r = 0.25 at the centre
    got["p"][corner] += 1e-3 * pmax
    err = bench.oracle_errors(ref, got)
    assert err["p"]["shell_max_abs_rel"] == 0.0
    assert abs(err["p"]["max_abs_rel"] - 1e-3) < 1e-12
    # a cell next to the first face in R's support (an x-face: its two cells)
    f = int(np.unique(sysm.R.tocoo().row)[0])
    nxf = (g.nx + 1) * g.ny * g.nz
    assert f < nxf
    k, rem = divmod(f, (g.nx + 1) * g.ny)
    j, i = divmod(rem, g.nx + 1)
    cell = (k * g.ny + j) * g.nx + min(i, g.nx - 1)
    got = {k_: ref[k_].copy() for k_ in ("u", "p", "F")}
    got["p"][cell] += 1e-3 * pmax
    err = bench.oracle_errors(ref, got)
    assert abs(err["p"]["shell_max_abs_rel"] - 1e-3) < 1e-12
    assert err["p"]["rel_l2"] < 1e-3
