"""Reverse-mode derivatives of one one-way step with respect to the prescribed
marker velocities U^Gamma and the marker positions X, FP64, CPU.  TEST
INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper differentiates nothing; what is differentiated here is the step of
Sec. 3.1 exactly as ``oracle.step`` computes it (scalar C mode), and the loss
is the hydrodynamic force and torque on a body.  The body feels minus the IB
force on the fluid, so with the IB force h^3 sum_k F_k of Eq. (IBM_force) and
the IB torque h^3 sum_k (X_k - X_c) x F_k, the drag-plus-torque loss is
J = -e_z . force - e_z . torque, evaluated on F^{n+1} = F^n + F'.

``step_vjp`` runs the steps of ``oracle.step.step`` backwards, one adjoint
relation per forward relation (a = 3/(2 dt)):

  F'    = 2 (B p' - RHS_F)            (Eq. (ApproxSchurPrimalF))
  p'    = S~^+ b,  S~ = L + 2 B^T B   (Eqs. (tildeSp), (ApproxSchurPrimalP))
  b     = RHS_p + 2 G^T R RHS_F
  RHS_F = a (R^T u* - U^Gamma),  RHS_p = a G^T u*    (below Eq. (Saddle))
  H u*  = rhs_u(u^n, u^{n-1}, p^n, f) + R F^n        (Eq. (ustar))

Every place R appears contributes f^T (dR/dX) m for a face field f and a
marker field m; ``_dR_pairs`` turns such pairs into per-marker position
derivatives with ``delta.regularization_derivative``.  The solve adjoint uses
that S~ and the Helmholtz operator are symmetric (S~ = L + 2 G^T R R^T G;
the predictor operator is a diagonal shift of the symmetric no-slip
Laplacian), and that p' is the mean-zero solution, so lambda = S~^+ p'_bar.

``body_force_torque_vjp`` is the derivative of ``oracle.step.body_force_torque``
(linear in F, bilinear in X - X_c and F).

Pins (tests/test_oracle_adjoint.py): J is linear in U^Gamma, so
dJ/dU_j = J(U + e_j) - J(U) holds up to rounding and is checked for every j on
tiny grids; dJ/dX and dJ/dX_c against central differences of J with step 1e-6
cell widths; the transposition identity <U_bar, dU> = dJ[dU] on random
directions at larger sizes.
"""
from __future__ import annotations

import numpy as np

from . import delta, helmholtz, mac
from .schur import solve_schur


def drag_torque_weights(n_bodies: int, body: int = 0):
    """Weights w (n_bodies, 6) on [force | torque] of ``body_force_torque`` for
    J = -(force_z + torque_z) of one body (the body feels minus the IB
    force, Eq. (force_bal))."""
    w = np.zeros((n_bodies, 6))
    w[body, 2] = -1.0
    w[body, 5] = -1.0
    return w


def body_force_torque_vjp(g: mac.Grid, X, F, body_id, centers, w):
    """For J = sum_b w_b . out_b with out = body_force_torque(g, X, F, ...):
    returns (dJ/dF (3N,), dJ/dX (3, N) through the lever arms, dJ/dcenters
    (n_bodies, 3)).  With force_b = h^3 sum F_k and torque_b =
    h^3 sum (X_k - c_b) x F_k:  d/dF_k = h^3 (w_F + w_T x r_k),
    d/dX_k = h^3 F_k x w_T,  d/dc_b = -h^3 sum_k F_k x w_T."""
    X = np.asarray(X, dtype=np.float64).reshape(3, -1)
    F = np.asarray(F, dtype=np.float64).reshape(3, -1)
    centers = np.asarray(centers, dtype=np.float64).reshape(-1, 3)
    w = np.asarray(w, dtype=np.float64).reshape(-1, 6)
    body_id = np.asarray(body_id)
    h3 = g.h ** 3
    F_bar = np.zeros_like(F)
    X_bar = np.zeros_like(X)
    c_bar = np.zeros_like(centers)
    for b in range(centers.shape[0]):
        sel = body_id == b
        r = X[:, sel] - centers[b][:, None]
        wF, wT = w[b, :3], w[b, 3:]
        F_bar[:, sel] = h3 * (wF[:, None] + np.cross(wT, r.T).T)
        xb = h3 * np.cross(F[:, sel].T, wT).T
        X_bar[:, sel] = xb
        c_bar[b] = -xb.sum(axis=1)
    return F_bar.ravel(), X_bar, c_bar


def _dR_pairs(g: mac.Grid, X, pairs):
    """sum over (f, m) of f^T (dR/dX_e) m for each marker and axis e: returns
    (3, N).  f is a packed face field, m a (3N,) marker field."""
    X = np.asarray(X, dtype=np.float64).reshape(3, -1)
    N = X.shape[1]
    out = np.zeros((3, N))
    for e in range(3):
        dR = delta.regularization_derivative(g, X, e)
        for f, m in pairs:
            col = (dR.T @ f) * np.asarray(m, dtype=np.float64).ravel()
            out[e] += col.reshape(3, N).sum(axis=0)
    return out


def step_vjp(g: mac.Grid, Re: float, dt: float, X, fw: dict, F_bar, F_n=None,
             rtol=1e-13, workers=None):
    """Given the forward dict ``fw`` of ``oracle.step.step`` (scalar mode) and
    the cotangent F_bar = dJ/dF^{n+1}, returns dict(U_bar (3N,),
    X_bar (3, N) through R, lam = S~^+ (2 B^T F_bar), mu = H^{-1} u*_bar,
    iters)."""
    X = np.asarray(X, dtype=np.float64).reshape(3, -1)
    sys = fw["sys"]
    k = 3 * X.shape[1]
    F_n = np.zeros(k) if F_n is None else np.asarray(F_n, dtype=np.float64)
    F_bar = np.asarray(F_bar, dtype=np.float64).ravel()
    a = 3.0 / (2.0 * dt)
    nu = 1.0 / Re
    p_corr, u_star, rhs_F = fw["p_corr"], fw["u_star"], fw["rhs_F"]

    # F' = 2 (B p' - RHS_F)
    p_bar = 2.0 * sys.apply_BT(F_bar)
    rhsF_bar = -2.0 * F_bar
    pairs = [(mac.apply_G(g, p_corr), 2.0 * F_bar)]
    # p' = S~^+ b: lambda = S~^+ p_bar, b_bar = lambda;
    # dS~ = 2 G^T (dR R^T + R dR^T) G contributes -lambda^T dS~ p'
    lam, iters, _, _ = solve_schur(sys, p_bar, mode="scalar", rtol=rtol, workers=workers)
    Glam = mac.apply_G(g, lam)
    Gp = mac.apply_G(g, p_corr)
    pairs.append((Glam, -2.0 * sys.apply_B(p_corr)))
    pairs.append((Gp, -2.0 * sys.apply_B(lam)))
    # b = RHS_p + 2 G^T R RHS_F
    rhsp_bar = lam
    rhsF_bar = rhsF_bar + 2.0 * sys.apply_B(lam)
    pairs.append((Glam, 2.0 * rhs_F))
    # RHS_F = a (R^T u* - U)
    U_bar = -a * rhsF_bar
    ustar_bar = a * (sys.R @ rhsF_bar)
    pairs.append((u_star, a * rhsF_bar))
    # RHS_p = a G^T u*
    ustar_bar = ustar_bar + a * mac.apply_G(g, rhsp_bar)
    # H u* = rhs_u + R F^n (only interior faces are unknowns)
    mask = g.interior_face_mask_packed()
    mu = helmholtz.solve(g, np.where(mask, ustar_bar, 0.0), a, nu, workers=workers)
    if np.any(F_n != 0.0):
        pairs.append((mu, F_n))
    X_bar = _dR_pairs(g, X, pairs)
    return dict(U_bar=U_bar, X_bar=X_bar, lam=lam, mu=mu, iters=iters)
