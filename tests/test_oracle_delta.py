"""Pins of oracle.delta (Roma delta, R, R^T) to closed forms, brute force and
the paper's Table A1 (RtR_spacing), and the O(h^2) accuracy of interpolation."""
import numpy as np
import pytest

from oracle import delta, mac
from paper_2501_15314_gb300 import workloads as wl
from conftest import load_golden


def test_phi_closed_form_values():
    # Eq. (delta): phi(0) = 2/3, phi(1/2) = 1/2, phi(1) = 1/6, phi(3/2) = 0
    v = delta.phi([0.0, 0.5, -0.5, 1.0, -1.0, 1.5, 2.0])
    np.testing.assert_allclose(v, [2 / 3, 0.5, 0.5, 1 / 6, 1 / 6, 0.0, 0.0], atol=1e-15)


@pytest.mark.parametrize("s", np.linspace(-0.5, 0.5, 23))
def test_phi_moments(s):
    # zeroth moment 1, first moment 0, sum of squares 1/2 for every shift
    j = np.arange(-4, 5)
    r = j - s
    p = delta.phi(r)
    assert abs(p.sum() - 1.0) < 1e-14
    assert abs((r * p).sum()) < 1e-14
    assert abs((p * p).sum() - 0.5) < 1e-14


def test_phi_continuous_c1_at_breakpoints():
    for x0, slope in ((0.5, -1.0), (1.5, 0.0)):
        e = 1e-7
        assert abs(delta.phi(x0 + e) - delta.phi(x0 - e)) < 1e-6
        d_left = (delta.phi(x0 - e) - delta.phi(x0 - 2 * e)) / e
        d_right = (delta.phi(x0 + 2 * e) - delta.phi(x0 + e)) / e
        assert abs(d_left - slope) < 1e-5 and abs(d_right - slope) < 1e-5


def _sphere(n, r, ratio=1.0, center=(0.5, 0.5, 0.5)):
    return wl.spheres_workload("t", n, 100, 0.01, [center], [r], None, 0, spacing_ratio=ratio)


def test_interp_matches_bruteforce_and_adjoint():
    g = mac.Grid(10, 12, 9)
    W = _sphere(10, 0.22, center=(0.5, 0.6, 0.45))
    rng = np.random.default_rng(0)
    u = rng.standard_normal(g.n_faces) * g.interior_face_mask_packed()
    R = delta.regularization_matrix(g, W.X)
    U_sparse = R.T @ u
    U_brute = delta.interp_bruteforce(g, W.X, u)
    np.testing.assert_allclose(U_sparse, U_brute, rtol=0, atol=1e-13)
    F = rng.standard_normal(R.shape[1])
    lhs = np.dot(R @ F, u)
    rhs = np.dot(F, U_brute)
    assert abs(lhs - rhs) <= 1e-13 * (abs(lhs) + 1)


def test_partition_of_unity_and_force_conservation():
    g = mac.Grid(16)
    W = _sphere(16, 0.3)
    R = delta.regularization_matrix(g, W.X)
    N = W.n_markers
    for d in range(3):
        u = np.zeros(g.n_faces)
        o, s = g.face_offsets[d], g.face_sizes[d]
        u[o:o + s] = 1.0
        U = (R.T @ u).reshape(3, N)
        np.testing.assert_allclose(U[d], 1.0, atol=1e-14)
        np.testing.assert_allclose(np.delete(U, d, axis=0), 0.0, atol=0)
    F = np.random.default_rng(1).standard_normal(3 * N)
    RF = R @ F
    for d in range(3):
        o, s = g.face_offsets[d], g.face_sizes[d]
        assert abs(RF[o:o + s].sum() - F[d * N:(d + 1) * N].sum()) < 1e-12


def test_linear_field_interpolated_exactly():
    # first-moment condition: linear fields are reproduced exactly
    g = mac.Grid(16)
    W = _sphere(16, 0.3)
    R = delta.regularization_matrix(g, W.X)
    for d in range(3):
        x, y, z = g.face_coords(d)
        field = 0.3 + 1.7 * x - 0.4 * y + 2.2 * z
        u = np.zeros(g.n_faces)
        o, s = g.face_offsets[d], g.face_sizes[d]
        u[o:o + s] = field.ravel()
        U = (R.T @ u).reshape(3, -1)[d]
        exact = 0.3 + 1.7 * W.X[0] - 0.4 * W.X[1] + 2.2 * W.X[2]
        np.testing.assert_allclose(U, exact, atol=1e-13)


def test_C_diagonal_is_one_eighth():
    # C_kk = (sum phi^2)^3 = 1/8 for every marker and component
    g = mac.Grid(16)
    W = _sphere(16, 0.3)
    R = delta.regularization_matrix(g, W.X)
    C = (R.T @ R).diagonal()
    np.testing.assert_allclose(C, 0.125, atol=1e-15)


def test_table_a1_rtr_row_sums():
    # Appendix A, Table A1 (RtR_spacing): average row sum of R^T R against spacing ratio
    table = load_golden("table_a1_rtr_rowsums.txt")
    g = mac.Grid(32)
    for ratio, lo, hi, avg in table:
        W = _sphere(32, 0.25, ratio=ratio)
        R = delta.regularization_matrix(g, W.X)
        rs = np.asarray((R.T @ R).sum(axis=1)).ravel()
        assert abs(rs.mean() - avg) <= 0.01 * avg, (ratio, rs.mean(), avg)
        assert abs(rs.min() - lo) <= 0.05 * lo and abs(rs.max() - hi) <= 0.05 * hi


def test_support_outside_interior_rejected():
    g = mac.Grid(16)
    X = np.array([[0.5], [0.5], [1.2 / 16]])   # z within 1.5h of the wall face
    with pytest.raises(ValueError):
        delta.regularization_matrix(g, X)


def test_smooth_field_interpolated_to_second_order():
    # zeroth and first moments vanish beyond order one, so interpolating a
    # smooth field leaves an O(h^2) error (Sec. 3.2: the kernel's moment
    # conditions); halving h divides the error by about 4
    errs = []
    for n in (16, 32, 64):
        g = mac.Grid(n)
        W = _sphere(n, 0.3, center=(0.48, 0.51, 0.53))
        R = delta.regularization_matrix(g, W.X)
        err = 0.0
        for d in range(3):
            x, y, z = g.face_coords(d)
            f = lambda a, b, c: np.sin(2 * np.pi * a + d) * np.cos(2 * np.pi * b) * np.cos(np.pi * c)  # noqa: E731
            u = np.zeros(g.n_faces)
            o, s = g.face_offsets[d], g.face_sizes[d]
            u[o:o + s] = f(x, y, z).ravel()
            U = (R.T @ u).reshape(3, -1)[d]
            err = max(err, np.abs(U - f(*W.X)).max())
        errs.append(err)
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all((orders > 1.8) & (orders < 2.3)), (errs, orders)
