"""Pins of oracle.schur: brute-force block solves, the spectral theorem of
Sec. 5, Table 2 (PrecResults)'s behaviour of the scalar approximation, and the
grid-independent iteration counts of Sec. 6.2."""
import numpy as np
import pytest

from oracle import mac, schur
from paper_2501_15314_gb300 import workloads as wl
from conftest import load_golden


def _system(n, r=0.25, ratio=1.0, center=(0.5, 0.5, 0.5)):
    W = wl.spheres_workload("t", n, 100, 0.01, [center], [r], None, 0, spacing_ratio=ratio)
    return schur.SchurSystem(mac.Grid(n), W.X), W


def _mean_zero_basis(m):
    # orthonormal basis of the complement of the constants
    Q, _ = np.linalg.qr(np.eye(m) - 1.0 / m)
    return Q[:, : m - 1]


def test_fgmres_matches_dense_bruteforce():
    sys, _ = _system(10, r=0.27)
    rng = np.random.default_rng(0)
    b = sys.apply_S_tilde(rng.standard_normal(sys.g.m))
    x_dense = schur.solve_dense(sys.dense_S_tilde(), b)
    x, it, rel, _ = schur.solve_schur(sys, b, rtol=1e-14)
    assert rel <= 1e-13
    np.testing.assert_allclose(x, x_dense, rtol=0, atol=1e-11 * np.abs(x_dense).max())


def test_schur_elimination_matches_block_saddle_solve():
    # Eqs. (SchurPrimalP), (SchurPrimalF) against a direct solve of Eq. (Saddle)
    sys, _ = _system(8, r=0.22)
    m, k = sys.g.m, sys.k
    rng = np.random.default_rng(1)
    rp = sys.G.T @ rng.standard_normal(sys.g.n_faces)     # orthogonal to constants
    rF = rng.standard_normal(k)
    K = sys.saddle_matrix()
    # fix the pressure constant with an extra row enforcing mean(p) = 0
    A = np.vstack([K, np.concatenate([np.ones(m), np.zeros(k)])[None, :]])
    sol = np.linalg.lstsq(A, np.concatenate([rp, rF, [0.0]]), rcond=None)[0]
    p_ref, F_ref = sol[:m], sol[m:]
    p = schur.solve_dense(sys.dense_S_exact(), sys.rhs_exact(rp, rF))
    F = sys.force_exact(p, rF)
    np.testing.assert_allclose(p, p_ref, atol=1e-9 * np.abs(p_ref).max())
    np.testing.assert_allclose(F, F_ref, atol=1e-9 * np.abs(F_ref).max())


@pytest.mark.parametrize("n", [6, 8])
def test_theorem_spectrum_in_1_2(n):
    # Sec. 5: spec(L^{-1} S_p) within [1, 2] on the complement of the constants
    sys, _ = _system(n, r=0.2)
    Q = _mean_zero_basis(sys.g.m)
    Lq = Q.T @ sys.L.toarray() @ Q
    Sq = Q.T @ sys.dense_S_exact() @ Q
    ev = np.linalg.eigvals(np.linalg.solve(Lq, Sq)).real
    assert ev.min() >= 1.0 - 1e-9 and ev.max() <= 2.0 + 1e-9
    assert ev.max() > 1.9     # the upper bound is nearly attained (Table 2, PrecResults)


def test_scalar_approximation_spectrum_like_table2():
    # Table 2 (PrecResults): spec(L^{-1} S~_p) starts at 1 and reaches close to 2
    tab = load_golden("table2_spectrum.txt")
    sys, _ = _system(8, r=0.25)
    Q = _mean_zero_basis(sys.g.m)
    Lq = Q.T @ sys.L.toarray() @ Q
    Sq = Q.T @ sys.dense_S_tilde() @ Q
    ev = np.linalg.eigvals(np.linalg.solve(Lq, Sq)).real
    assert abs(ev.min() - tab[:, 3].min()) < 1e-9          # lower end exactly 1
    assert 1.8 < ev.max() < tab[:, 4].max() + 0.05


def test_no_markers_gives_laplacian_pinv():
    g = mac.Grid(12)
    sys = schur.SchurSystem(g, np.zeros((3, 0)))
    b = mac.remove_mean(np.random.default_rng(2).standard_normal(g.m))
    x, it, rel, _ = schur.solve_schur(sys, b, rtol=1e-14)
    np.testing.assert_allclose(x, mac.laplacian_pinv(g, b), atol=1e-12 * np.abs(x).max())
    assert it <= 2


def test_iterations_grid_independent():
    # Sec. 6.2: few iterations, nearly constant in the grid size
    its = []
    for n in (16, 32):
        W = wl.spheres_workload("t", n, 100, 0.01, [[0.5] * 3], [0.2], None, 0)
        sys = schur.SchurSystem(mac.Grid(n), W.X)
        b = sys.apply_S_tilde(np.random.default_rng(3).standard_normal(sys.g.m))
        _, it, rel, _ = schur.solve_schur(sys, b, rtol=1e-8)
        its.append(it)
    assert max(its) <= 14 and abs(its[0] - its[1]) <= 2, its


def test_unpreconditioned_needs_many_more_iterations():
    # Sec. 6.2, second experiment: without L^{-1} the count grows sharply
    W = wl.spheres_workload("t", 16, 100, 0.01, [[0.5] * 3], [0.2], None, 0)
    sys = schur.SchurSystem(mac.Grid(16), W.X)
    b = sys.apply_S_tilde(np.random.default_rng(4).standard_normal(sys.g.m))
    _, it_p, _, _ = schur.solve_schur(sys, b, rtol=1e-8)
    _, it_u, _, _ = schur.fgmres(sys.apply_S_tilde, b, lambda r: r, rtol=1e-8, restart=200,
                                 maxit=400)
    assert it_u > 8 * it_p

