"""Pins of oracle.step: exact post-update identities implied by Eqs.
(Saddle), (ApproxSchurPrimalF) and (u_n_plus_1); energy conservation and
second-order accuracy of the convective term."""
import numpy as np
import pytest

from oracle import mac, step
from paper_2501_15314_gb300 import workloads as wl


def _curl_field(g, rng):
    """Discretely divergence-free face field with zero wall-normal flux: the
    discrete curl of a random edge potential that vanishes on the walls."""
    nx, ny, nz, h = g.nx, g.ny, g.nz, g.h
    Az = rng.standard_normal((nz, ny + 1, nx + 1))
    Az[:, 0, :] = Az[:, -1, :] = 0
    Az[:, :, 0] = Az[:, :, -1] = 0
    Ax = rng.standard_normal((nz + 1, ny + 1, nx))
    Ax[0] = Ax[-1] = 0
    Ax[:, 0, :] = Ax[:, -1, :] = 0
    Ay = rng.standard_normal((nz + 1, ny, nx + 1))
    Ay[0] = Ay[-1] = 0
    Ay[:, :, 0] = Ay[:, :, -1] = 0
    ux = (Az[:, 1:, :] - Az[:, :-1, :]) / h - (Ay[1:] - Ay[:-1]) / h
    uy = (Ax[1:] - Ax[:-1]) / h - (Az[:, :, 1:] - Az[:, :, :-1]) / h
    uz = (Ay[:, :, 1:] - Ay[:, :, :-1]) / h - (Ax[:, 1:, :] - Ax[:, :-1, :]) / h
    return g.pack_faces(ux, uy, uz)


@pytest.mark.parametrize("mode", ["scalar", "exact"])
def test_post_update_identities(mode):
    W = wl.spheres_workload("t", 12, 100, 0.01, [[0.5] * 3], [0.25], None, 5)
    g = mac.Grid(12)
    rng = np.random.default_rng(6)
    u_n = _curl_field(g, rng) * 0.1
    out = step.step(g, W.Re, W.dt, W.X, W.U_gamma, W.f_body, u_n=u_n, mode=mode)
    sys, dt = out["sys"], W.dt
    Fc = out["F_corr"]
    div = sys.G.T @ out["u"]
    # G^T u^{n+1} = (4 dt/3) B^T F'
    np.testing.assert_allclose(div, (4 * dt / 3) * (sys.B.T @ Fc),
                               atol=1e-10 * np.abs(sys.G.T @ out["u_star"]).max())
    slip = sys.R.T @ out["u"] - W.U_gamma.ravel()
    if mode == "scalar":   # (dt/3)(2C - I) F'
        expect = (dt / 3) * (2 * (sys.C @ Fc) - Fc)
    else:
        expect = np.zeros_like(slip)
    np.testing.assert_allclose(slip, expect, atol=1e-11 * max(1.0, np.abs(Fc).max() * dt))


def test_advection_conserves_energy_for_divergence_free_fields():
    g = mac.Grid(8, 9, 10)
    u = _curl_field(g, np.random.default_rng(0))
    assert np.abs(mac.gradient_matrix(g).T @ u).max() < 1e-10
    A = step.advection(g, u)
    assert abs(np.dot(u, A)) <= 1e-13 * np.abs(u).sum() * np.abs(A).max()


def test_advection_second_order():
    errs = []
    for n in (16, 32):
        g = mac.Grid(n)
        uu, ex = [], []
        for d in range(3):
            x, y, z = g.face_coords(d)
            s1, c1 = np.sin(np.pi * x), np.cos(np.pi * x)
            ux = s1 ** 2 * np.sin(2 * np.pi * y)
            uy = -np.sin(2 * np.pi * x) * np.sin(np.pi * y) ** 2
            if d == 0:
                uu.append(ux)
                ex.append(ux * 2 * np.pi * s1 * c1 * np.sin(2 * np.pi * y)
                          + uy * 2 * np.pi * s1 ** 2 * np.cos(2 * np.pi * y))
            elif d == 1:
                uu.append(uy)
                ex.append(ux * (-2 * np.pi * np.cos(2 * np.pi * x) * np.sin(np.pi * y) ** 2)
                          + uy * (-2 * np.pi * np.sin(2 * np.pi * x) * np.sin(np.pi * y)
                                  * np.cos(np.pi * y)))
            else:
                uu.append(0 * x)
                ex.append(0 * x)
        e = g.pack_faces(*ex) * g.interior_face_mask_packed()
        errs.append(np.abs(step.advection(g, g.pack_faces(*uu)) - e).max())
    order = np.log2(errs[0] / errs[1])
    assert 1.8 < order < 2.2, errs


def test_zero_forcing_zero_velocity_gives_zero_step():
    W = wl.spheres_workload("t", 12, 100, 0.01, [[0.5] * 3], [0.25], None, 5)
    g = mac.Grid(12)
    out = step.step(g, W.Re, W.dt, W.X, np.zeros_like(W.U_gamma), np.zeros(g.n_faces))
    assert np.abs(out["u"]).max() == 0.0 and np.abs(out["p"]).max() == 0.0


def test_body_force_torque_closed_form():
    # per body h^3 sum F_k and h^3 sum (X_k - X_c) x F_k (Eq. (IBM_force)),
    # written out for three markers with axis-aligned lever arms and forces
    g = mac.Grid(10)                                  # h^3 = 1e-3
    c = np.array([[0.5, 0.5, 0.5], [0.2, 0.3, 0.4]])
    X = np.array([[0.5, 0.5, 0.3],                    # columns: markers
                  [0.7, 0.5, 0.3],
                  [0.5, 0.6, 0.4]])
    F = np.array([[1.0, 0.0, 0.0],
                  [0.0, 2.0, 0.0],
                  [0.0, 0.0, 3.0]])
    body_id = np.array([0, 0, 1])
    out = step.body_force_torque(g, X, F, body_id, c)
    # body 0: r = (0, 0.2, 0) with F = (1, 0, 0), r = (0, 0, 0.1) with F = (0, 2, 0)
    # body 1: r = (0.1, 0, 0) with F = (0, 0, 3)
    expect = 1e-3 * np.array([[1.0, 2.0, 0.0, -0.2, 0.0, -0.2],
                              [0.0, 0.0, 3.0, 0.0, -0.3, 0.0]])
    np.testing.assert_allclose(out, expect, rtol=0, atol=1e-15)
