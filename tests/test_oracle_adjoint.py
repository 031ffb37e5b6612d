"""Pins of the oracle's derivatives (oracle.delta.phi_prime,
regularization_derivative, oracle.adjoint) against things other than
themselves: the breakpoint values of Eq. (delta), the differentiated moment
identities, central differences, and exact linearity of the step in
U^Gamma."""
import numpy as np
import pytest

from oracle import adjoint, delta, mac, step
from paper_2501_15314_gb300 import workloads as wl


def test_phi_prime_breakpoints_and_centre():
    # C^1 join of the branches of Eq. (delta): slope -1 at 1/2, 0 at 3/2
    v = delta.phi_prime([0.0, 0.5, -0.5, 1.5, -1.5, 2.0])
    np.testing.assert_allclose(v, [0.0, -1.0, 1.0, 0.0, 0.0, 0.0], atol=1e-15)


def test_phi_prime_central_difference():
    rng = np.random.default_rng(3)
    r = rng.uniform(-1.6, 1.6, 400)
    r = r[np.min(np.abs(np.abs(r)[:, None] - np.array([0.5, 1.5])[None, :]), axis=1) > 1e-3]
    e = 1e-6
    fd = (delta.phi(r + e) - delta.phi(r - e)) / (2 * e)
    np.testing.assert_allclose(delta.phi_prime(r), fd, atol=1e-8)


@pytest.mark.parametrize("s", np.linspace(-0.5, 0.5, 17))
def test_phi_prime_moments(s):
    # d/ds of sum_j phi(j - s) = 1 and of sum_j (j - s) phi(j - s) = 0
    j = np.arange(-4, 5)
    r = j - s
    dp = delta.phi_prime(r)
    assert abs(dp.sum()) < 1e-13
    assert abs((r * dp).sum() + 1.0) < 1e-13


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_regularization_derivative_central_difference(axis):
    g = mac.Grid(10, 11, 12)
    W = wl.spheres_workload("t", 10, 100, 0.01, [[0.5213, 0.4731, 0.5077]], [0.2], None, 1)
    X = W.X.reshape(3, -1)
    e = 1e-6 * g.h
    # central differences are O(e) wrong where a tap sits within e of a
    # breakpoint of phi (|r| = 1/2, 3/2: phi'' jumps); keep clear of those
    for d in range(3):
        for ax in range(3):
            off = 0.0 if ax == d else 0.5
            r = X[ax] / g.h - off
            frac = np.abs(r - np.round(r * 2) / 2)
            assert frac.min() > 1e-4
    Xp, Xm = X.copy(), X.copy()
    Xp[axis] += e
    Xm[axis] -= e
    fd = (delta.regularization_matrix(g, Xp) - delta.regularization_matrix(g, Xm)) / (2 * e)
    dR = delta.regularization_derivative(g, X, axis)
    scale = np.abs(dR).max()
    assert np.abs((dR - fd).toarray()).max() < 1e-6 * scale


def _state(n, seed, second_step):
    """A small one-sphere problem; with second_step the forward step starts
    from the state after one step (u^n, p^n, F^n nonzero)."""
    W = wl.spheres_workload("t", n, 100, 0.01, [[0.5, 0.52, 0.48]], [0.15], None, seed)
    g = mac.Grid(n)
    X = W.X.reshape(3, -1)
    kw = dict(u_n=None, u_nm1=None, p_n=None, F_n=None)
    if second_step:
        first = step.step(g, W.Re, W.dt, X, W.U_gamma, W.f_body)
        kw = dict(u_n=first["u"], u_nm1=np.zeros(g.n_faces), p_n=first["p"], F_n=first["F"])
    body_id = np.zeros(X.shape[1], dtype=np.int32)
    centers = np.array([[0.5, 0.52, 0.48]])
    return W, g, X, kw, body_id, centers


def _loss(g, W, X, U, kw, body_id, centers, w):
    fw = step.step(g, W.Re, W.dt, X, U, W.f_body, **kw)
    out = step.body_force_torque(g, X, fw["F"], body_id, centers)
    return float((w * out).sum()), fw


def _vjp(g, W, X, U, kw, body_id, centers, w):
    J, fw = _loss(g, W, X, U, kw, body_id, centers, w)
    F_bar, X_lever, c_bar = adjoint.body_force_torque_vjp(g, X, fw["F"], body_id, centers, w)
    r = adjoint.step_vjp(g, W.Re, W.dt, X, fw, F_bar, F_n=kw["F_n"])
    return J, r, X_lever, c_bar


@pytest.mark.parametrize("second_step", [False, True])
def test_U_gradient_exact_by_linearity(second_step):
    W, g, X, kw, body_id, centers = _state(8, 11, second_step)
    w = adjoint.drag_torque_weights(1)
    U = W.U_gamma.ravel()
    J0, r, _, _ = _vjp(g, W, X, U, kw, body_id, centers, w)
    brute = np.empty_like(U)
    for j in range(U.size):
        Uj = U.copy()
        Uj[j] += 1.0
        brute[j] = _loss(g, W, X, Uj, kw, body_id, centers, w)[0] - J0
    np.testing.assert_allclose(r["U_bar"], brute, rtol=0, atol=1e-9 * np.abs(brute).max())


@pytest.mark.parametrize("second_step", [False, True])
def test_center_gradient_central_difference(second_step):
    """Rigid translation of the body (markers and centre) by +-1e-6 h."""
    W, g, X, kw, body_id, centers = _state(8, 12, second_step)
    w = adjoint.drag_torque_weights(1)
    U = W.U_gamma.ravel()
    _, r, X_lever, c_bar = _vjp(g, W, X, U, kw, body_id, centers, w)
    grad = (r["X_bar"] + X_lever).sum(axis=1) + c_bar[0]
    e = 1e-6 * g.h
    fd = np.empty(3)
    for ax in range(3):
        dX = np.zeros_like(X)
        dX[ax] = e
        dc = np.zeros_like(centers)
        dc[0, ax] = e
        Jp = _loss(g, W, X + dX, U, kw, body_id, centers + dc, w)[0]
        Jm = _loss(g, W, X - dX, U, kw, body_id, centers - dc, w)[0]
        fd[ax] = (Jp - Jm) / (2 * e)
    np.testing.assert_allclose(grad, fd, rtol=1e-6, atol=1e-6 * np.abs(fd).max())


def test_single_marker_gradient_central_difference():
    """Moving one marker alone (the centre fixed) checks the per-marker
    derivative including the lever arm, with u^n, F^n nonzero."""
    W, g, X, kw, body_id, centers = _state(8, 13, True)
    w = adjoint.drag_torque_weights(1)
    U = W.U_gamma.ravel()
    _, r, X_lever, _ = _vjp(g, W, X, U, kw, body_id, centers, w)
    grad = r["X_bar"] + X_lever
    e = 1e-6 * g.h
    for k in (0, X.shape[1] // 2):
        for ax in range(3):
            dX = np.zeros_like(X)
            dX[ax, k] = e
            Jp = _loss(g, W, X + dX, U, kw, body_id, centers, w)[0]
            Jm = _loss(g, W, X - dX, U, kw, body_id, centers, w)[0]
            fd = (Jp - Jm) / (2 * e)
            assert abs(grad[ax, k] - fd) <= 1e-6 * np.abs(grad).max()


def test_transposition_identity_random_directions():
    W = wl.spheres_workload("t", 16, 100, 0.01, [[0.5, 0.5, 0.5]], [0.25], None, 4)
    g = mac.Grid(16)
    X = W.X.reshape(3, -1)
    body_id = np.zeros(X.shape[1], dtype=np.int32)
    centers = np.array([[0.5, 0.5, 0.5]])
    rng = np.random.default_rng(5)
    w = rng.standard_normal((1, 6))
    U = W.U_gamma.ravel()
    kw = dict(u_n=None, u_nm1=None, p_n=None, F_n=None)
    _, r, _, _ = _vjp(g, W, X, U, kw, body_id, centers, w)
    for _ in range(2):
        dU = rng.standard_normal(U.size)
        Jp = _loss(g, W, X, U + dU, kw, body_id, centers, w)[0]
        Jm = _loss(g, W, X, U - dU, kw, body_id, centers, w)[0]
        d = (Jp - Jm) / 2
        assert abs(np.dot(r["U_bar"], dU) - d) <= 1e-9 * abs(d)


def test_body_force_torque_vjp_central_difference():
    g = mac.Grid(8)
    rng = np.random.default_rng(9)
    N, nb = 12, 2
    X = rng.uniform(0.3, 0.7, (3, N))
    F = rng.standard_normal((3, N))
    body_id = (np.arange(N) % nb).astype(np.int32)
    centers = rng.uniform(0.4, 0.6, (nb, 3))
    w = rng.standard_normal((nb, 6))

    def J(X_, F_, c_):
        return float((w * step.body_force_torque(g, X_, F_, body_id, c_)).sum())

    F_bar, X_bar, c_bar = adjoint.body_force_torque_vjp(g, X, F, body_id, centers, w)
    e = 1e-3   # J is bilinear: central differences are exact up to rounding
    for arr, grad in ((F, F_bar.reshape(3, N)), (X, X_bar), (centers, c_bar)):
        fd = np.zeros_like(arr)
        for idx in np.ndindex(arr.shape):
            p, m = arr.copy(), arr.copy()
            p[idx] += e
            m[idx] -= e
            args = {id(F): (X, p, centers), id(X): (p, F, centers),
                    id(centers): (X, F, p)}[id(arr)]
            argm = {id(F): (X, m, centers), id(X): (m, F, centers),
                    id(centers): (X, F, m)}[id(arr)]
            fd[idx] = (J(*args) - J(*argm)) / (2 * e)
        np.testing.assert_allclose(grad, fd, atol=1e-12 * max(1.0, np.abs(fd).max()))
