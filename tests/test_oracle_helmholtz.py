"""Pins of oracle.helmholtz (BDF2 predictor operator and exact solve)."""
import numpy as np
import scipy.sparse.linalg as spla

from oracle import helmholtz, mac


def test_apply_matches_assembled_matrix():
    g = mac.Grid(4, 5, 6, h=0.25)
    a, nu = 37.0, 0.3
    A = helmholtz.matrix(g, a, nu)
    u = np.random.default_rng(0).standard_normal(g.n_faces) * g.interior_face_mask_packed()
    np.testing.assert_allclose(A @ u, helmholtz.apply(g, u, a, nu), rtol=1e-13, atol=1e-12)


def test_solve_matches_sparse_direct():
    g = mac.Grid(5, 4, 6, h=0.2)
    a, nu = 15.0, 0.7
    A = helmholtz.matrix(g, a, nu).tocsc()
    mask = g.interior_face_mask_packed()
    rhs = np.random.default_rng(1).standard_normal(g.n_faces) * mask
    idx = np.flatnonzero(mask)
    ref = np.zeros(g.n_faces)
    ref[idx] = spla.spsolve(A[idx][:, idx], rhs[idx])
    np.testing.assert_allclose(helmholtz.solve(g, rhs, a, nu), ref, atol=1e-12)


def test_second_order_on_manufactured_field():
    # u_d = sin(pi x) sin(pi y) sin(pi z) vanishes on every wall; -Lap u = 3 pi^2 u
    a, nu = 10.0, 0.5
    errs = []
    for n in (16, 32):
        g = mac.Grid(n)
        exact = []
        for d in range(3):
            x, y, z = g.face_coords(d)
            exact.append(np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z))
        ue = g.pack_faces(*exact) * g.interior_face_mask_packed()
        rhs = (a + 3 * nu * np.pi ** 2) * ue
        u = helmholtz.solve(g, rhs, a, nu)
        errs.append(np.abs(u - ue).max())
    order = np.log2(errs[0] / errs[1])
    assert 1.8 < order < 2.3, errs
