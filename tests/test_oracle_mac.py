"""Pins of oracle.mac (MAC grid operators, exact Neumann pseudo-inverse)."""
import numpy as np

from oracle import mac


def _div_loops(g, u):
    """Flux-form divergence written out cell by cell (wall faces carry 0)."""
    ux, uy, uz = g.split_faces(u)
    ux = ux.copy(); uy = uy.copy(); uz = uz.copy()
    ux[:, :, 0] = ux[:, :, -1] = 0.0
    uy[:, 0, :] = uy[:, -1, :] = 0.0
    uz[0, :, :] = uz[-1, :, :] = 0.0
    out = np.zeros(g.cell_shape)
    for k in range(g.nz):
        for j in range(g.ny):
            for i in range(g.nx):
                out[k, j, i] = ((ux[k, j, i + 1] - ux[k, j, i]) + (uy[k, j + 1, i] - uy[k, j, i])
                                + (uz[k + 1, j, i] - uz[k, j, i])) / g.h
    return out.ravel()


def _lap_loops(g, v):
    v3 = v.reshape(g.cell_shape)
    out = np.zeros(g.cell_shape)
    for k in range(g.nz):
        for j in range(g.ny):
            for i in range(g.nx):
                s = 0.0
                for dk, dj, di in ((0, 0, 1), (0, 0, -1), (0, 1, 0), (0, -1, 0), (1, 0, 0),
                                   (-1, 0, 0)):
                    kk, jj, ii = k + dk, j + dj, i + di
                    if 0 <= kk < g.nz and 0 <= jj < g.ny and 0 <= ii < g.nx:
                        s += v3[k, j, i] - v3[kk, jj, ii]
                out[k, j, i] = s / g.h ** 2
    return out.ravel()


def test_gradient_kills_constants():
    g = mac.Grid(5, 6, 7)
    G = mac.gradient_matrix(g)
    assert np.abs(G @ np.ones(g.m)).max() == 0.0


def test_gradient_transpose_is_minus_divergence():
    g = mac.Grid(5, 6, 7, h=0.1)
    G = mac.gradient_matrix(g)
    u = np.random.default_rng(0).standard_normal(g.n_faces)
    np.testing.assert_allclose(G.T @ u, -_div_loops(g, u), atol=1e-12)


def test_laplacian_is_7_point_neumann():
    g = mac.Grid(5, 4, 6, h=0.2)
    L = mac.laplacian_matrix(g)
    v = np.random.default_rng(1).standard_normal(g.m)
    np.testing.assert_allclose(L @ v, _lap_loops(g, v), atol=1e-11)
    assert abs(L - L.T).max() == 0.0


def test_pinv_matches_dense_pseudoinverse():
    g = mac.Grid(4, 5, 6, h=0.3)
    L = mac.laplacian_matrix(g).toarray()
    P = np.linalg.pinv(L)
    r = np.random.default_rng(2).standard_normal(g.m)
    np.testing.assert_allclose(mac.laplacian_pinv(g, r), P @ r, atol=1e-11)


def test_neumann_eigenvalues():
    g = mac.Grid(4, 3, 5, h=0.5)
    lam = np.sort(mac.neumann_eigenvalues(g).ravel())
    ev = np.sort(np.linalg.eigvalsh(mac.laplacian_matrix(g).toarray()))
    np.testing.assert_allclose(lam, ev, atol=1e-12)


def test_laplacian_second_order_on_cosine():
    # L = -Lap; cos(pi x) cos(pi y) cos(pi z) satisfies the Neumann condition
    errs = []
    for n in (16, 32):
        g = mac.Grid(n)
        c = (np.arange(n) + 0.5) / n
        Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
        f = np.cos(np.pi * X) * np.cos(np.pi * Y) * np.cos(np.pi * Z)
        Lf = mac.laplacian_matrix(g) @ f.ravel()
        errs.append(np.abs(Lf - 3 * np.pi ** 2 * f.ravel()).max())
    order = np.log2(errs[0] / errs[1])
    assert 1.8 < order < 2.2, errs


def test_matrix_free_operators_match_matrices():
    g = mac.Grid(6, 5, 7, h=0.3)
    rng = np.random.default_rng(5)
    p = rng.standard_normal(g.m)
    u = rng.standard_normal(g.n_faces)
    G = mac.gradient_matrix(g)
    np.testing.assert_allclose(mac.apply_G(g, p), G @ p, atol=1e-13)
    np.testing.assert_allclose(mac.apply_GT(g, u), G.T @ u, atol=1e-12)
    np.testing.assert_allclose(mac.apply_L(g, p), (G.T @ G) @ p, atol=1e-11)
