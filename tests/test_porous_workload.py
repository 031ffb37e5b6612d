"""The porous-sphere workload of Sec. 6.1.2 (Table 1, label spheresCenters):
the transcribed sub-sphere centres against the porosities and packing the
paper states, and grid-independent oracle iteration counts for the 7- and
14-sphere arrays (the claim of Sec. 6.2 behind Table 4, label 3dPorous)."""
import numpy as np
import pytest

from oracle import mac, schur
from paper_2501_15314_gb300 import workloads as wl


@pytest.mark.parametrize("n_sub,eps", [(7, 0.598), (14, 0.526)])
def test_table1_centres_give_the_stated_porosity_and_packing(n_sub, eps):
    r, cents = wl.POROUS_CENTRES[n_sub]
    c = 0.1 * np.asarray(cents)          # units of D, bounding centre at 0
    # porosity = 1 - n (r / (D/2))^3 as printed with each configuration
    assert abs((1.0 - n_sub * (r / 0.5) ** 3) - eps) < 0.01
    # packed without overlap inside the bounding sphere (radius 1/2)
    d = np.sqrt(((c[:, None] - c[None]) ** 2).sum(-1))
    np.fill_diagonal(d, np.inf)
    assert d.min() >= 2 * r - 2e-3
    assert (np.sqrt((c ** 2).sum(-1)) + r).max() <= 0.5 + 2e-3
    # several sub-spheres touch (gap below the table's rounding)
    assert d.min() < 2 * r + 2e-3


def test_workload_radius_reduction_and_velocity():
    W = wl.porous_sphere(64, 7)
    h = 1.0 / 64
    assert np.allclose(W.radii, 0.193 * 0.3 - 0.5 * h)
    assert np.allclose(W.U_gamma[:2], 0.0) and np.allclose(W.U_gamma[2], np.sin(1.0))
    k = W.body_id == 3
    rr = np.sqrt(((W.X[:, k] - W.centers[3][:, None]) ** 2).sum(0))
    assert np.allclose(rr, W.radii[3])


def _iters(W, rtol=1e-10):
    g = mac.Grid(W.n)
    sysm = schur.SchurSystem(g, W.X)
    rng = np.random.default_rng(0)
    b = sysm.rhs_scalar(mac.apply_GT(g, rng.standard_normal(g.n_faces)),
                        rng.standard_normal(3 * W.n_markers))
    return schur.solve_schur(sysm, b, rtol=rtol, workers=4)[1]


def test_oracle_iterations_grid_independent_for_porous_arrays():
    counts = {k: [_iters(wl.porous_sphere(n, k)) for n in (24, 40, 64)] for k in (7, 14)}
    single = [_iters(wl.oscillating_sphere(n, None)) for n in (24, 40, 64)]
    allc = sum(counts.values(), []) + single
    assert max(allc) - min(allc) <= 3, (counts, single)
