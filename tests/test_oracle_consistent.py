"""Pins of the sign-consistent form of the correction system in
oracle.schur / oracle.step: [[L, -B^T], [B, -C]], whose update of
Eq. (u_n_plus_1) is divergence-free and satisfies the no-slip condition
exactly."""
import numpy as np
import pytest

from oracle import mac, schur, step
from paper_2501_15314_gb300 import workloads as wl
from test_oracle_schur import _mean_zero_basis, _system


def test_elimination_matches_block_solve():
    sys, _ = _system(8, r=0.22)
    m, k = sys.g.m, sys.k
    rng = np.random.default_rng(3)
    rp = sys.G.T @ rng.standard_normal(sys.g.n_faces)
    rF = rng.standard_normal(k)
    K = sys.saddle_matrix_consistent()
    A = np.vstack([K, np.concatenate([np.ones(m), np.zeros(k)])[None, :]])
    sol = np.linalg.lstsq(A, np.concatenate([rp, rF, [0.0]]), rcond=None)[0]
    p_ref, F_ref = sol[:m], sol[m:]
    p = schur.solve_dense(sys.dense_S_consistent(), sys.rhs_consistent(rp, rF))
    F = sys.force_exact(p, rF)
    np.testing.assert_allclose(p, p_ref, atol=1e-9 * np.abs(p_ref).max())
    np.testing.assert_allclose(F, F_ref, atol=1e-9 * np.abs(F_ref).max())


@pytest.mark.parametrize("n", [6, 8])
def test_spectrum_in_0_1(n):
    # S_c = G^T (I - P) G with P = R C^{-1} R^T an orthogonal projection
    sys, _ = _system(n, r=0.2)
    Q = _mean_zero_basis(sys.g.m)
    Lq = Q.T @ sys.L.toarray() @ Q
    Sq = Q.T @ sys.dense_S_consistent() @ Q
    ev = np.linalg.eigvals(np.linalg.solve(Lq, Sq)).real
    assert ev.min() >= -1e-9 and ev.max() <= 1.0 + 1e-9
    assert ev.min() < 0.1          # far from bounded below, unlike S_p
    P = sys.R @ np.linalg.solve(sys.C.toarray(), sys.R.T.toarray())
    np.testing.assert_allclose(P @ P, P, atol=1e-10)


def test_step_is_divergence_free_and_no_slip():
    W = wl.spheres_workload("t", 10, 100, 0.01, [[0.5, 0.48, 0.52]], [0.22], None, 7)
    g = mac.Grid(10)
    out = step.step(g, W.Re, W.dt, W.X, W.U_gamma, W.f_body, mode="consistent", rtol=1e-13)
    sys = out["sys"]
    div = sys.G.T @ out["u"]
    scale = np.abs(sys.G.T @ out["u_star"]).max()
    assert np.abs(div).max() < 1e-10 * scale
    slip = sys.R.T @ out["u"] - W.U_gamma.ravel()
    assert np.abs(slip).max() < 1e-10 * np.abs(W.U_gamma).max()
    # the paper's literal form leaves both at the size of the identities of
    # Eq. (Saddle) (oracle.step): a different solution
    lit = step.step(g, W.Re, W.dt, W.X, W.U_gamma, W.f_body, mode="exact", rtol=1e-13)
    assert np.abs(sys.G.T @ lit["u"]).max() > 1e3 * np.abs(div).max()
