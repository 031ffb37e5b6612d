"""One one-way SIMPLE-IBM time step, FP64, CPU.  TEST INFRASTRUCTURE ONLY (see
``oracle/__init__``).

Sec. 3.1, in the paper's order:

1. predictor, Eq. (ustar):
   (a - nu Lap) u* = (4 u^n - u^{n-1})/(2 dt) - G p^n + R F^n - A(u^n) + f
   with a = 3/(2 dt), nu = 1/Re, f a prescribed body force on the faces and
   A(u^n) the explicit convective term (``advection``; zero when u^n = 0);
2. correction right-hand sides below Eq. (Saddle):
   RHS_p = -(3/(2 dt)) div u* = a G^T u*,  RHS_F = a (R^T u* - U^Gamma);
3. Schur solve S~_p p' = RHS_p + 2 B^T RHS_F  (Eq. (ApproxSchurPrimalP)),
   or the exact S_p form (Eq. (SchurPrimalP)), or the sign-consistent form
   (``oracle.schur``; then div and slip of u^{n+1} vanish exactly);
4. force recovery F' = 2 (B p' - RHS_F)  (Eq. (ApproxSchurPrimalF)) or
   C^{-1}(B p' - RHS_F)  (Eq. (SchurPrimalF));
5. update, Eq. (u_n_plus_1) and the correction step that follows Eq. (divfree):
   u^{n+1} = u* + (2 dt/3)(-G p' + R F'),  p^{n+1} = p^n + p',
   F^{n+1} = F^n + F';
6. diagnostics: ||G^T u^{n+1}||, ||R^T u^{n+1} - U^Gamma||, and per body the
   IB force h^3 sum_k F_k (Eq. (IBM_force); the delta sums to one, so the sum
   over the Eulerian force field equals the Lagrangian sum) and torque
   h^3 sum_k (X_k - X_c) x F_k.

The exact identities G^T u^{n+1} = (4 dt/3) B^T F' (both C modes) and
R^T u^{n+1} - U^Gamma = (dt/3)(2C - I) F' (scalar mode; 0 in exact mode) follow
from steps 2-5 and pin the signs of this module (tests/test_oracle_step.py).
"""
from __future__ import annotations

import numpy as np

from . import helmholtz, mac
from .schur import SchurSystem, solve_schur


def advection(g: mac.Grid, u):
    """Explicit convective term (u.grad u)^n of Eq. (ustar) on the interior
    faces: the central finite-volume divergence form div(u u_d) on the MAC grid
    (Sec. 3.1: central differences for all spatial terms).  For component d the
    flux along e != d lives on the cell edges shared by a d-face and an e-face:
    (u_e averaged along d) * (u_d averaged along e); along e = d it is the square
    of u_d averaged to the cell centre.  Fluxes through walls vanish because the
    wall-normal velocity there is 0."""
    uc = [c.copy() for c in g.split_faces(np.asarray(u, dtype=np.float64))]
    for d in range(3):
        uc[d][~g.interior_face_mask(d)] = 0.0
    out = np.zeros(g.n_faces)
    oc = g.split_faces(out)
    h = g.h
    for d in range(3):
        ad = 2 - d                               # array axis of coordinate d
        ud = uc[d]
        acc = np.zeros_like(ud)
        for e in range(3):
            ae = 2 - e
            if e == d:
                lo = [slice(None)] * 3
                hi = [slice(None)] * 3
                lo[ad], hi[ad] = slice(0, -1), slice(1, None)
                cc = 0.5 * (ud[tuple(lo)] + ud[tuple(hi)])   # cell centres
                flux = cc * cc
                dst = [slice(None)] * 3
                dst[ad] = slice(1, -1)
                acc[tuple(dst)] += (flux[tuple(hi)] - flux[tuple(lo)]) / h
                continue
            ue = uc[e]
            # u_e averaged along d onto the interior d-face positions:
            # e-face array has cells along d; d-face k sits between cells k-1, k
            lo = [slice(None)] * 3
            hi = [slice(None)] * 3
            lo[ad], hi[ad] = slice(0, -1), slice(1, None)
            ue_d = 0.5 * (ue[tuple(lo)] + ue[tuple(hi)])
            # now indexed [.., e-face position 0..n_e, .., d-face 1..n_d-1]
            # u_d averaged along e onto e-face positions 1..n_e-1
            lo = [slice(None)] * 3
            hi = [slice(None)] * 3
            lo[ae], hi[ae] = slice(0, -1), slice(1, None)
            ud_e = 0.5 * (ud[tuple(lo)] + ud[tuple(hi)])
            sel = [slice(None)] * 3
            sel[ad] = slice(1, -1)
            ud_e = ud_e[tuple(sel)]
            # flux on edges, e positions 0..n_e; walls (0 and n_e) carry 0
            fshape = list(ue_d.shape)
            flux = np.zeros(fshape)
            inner = [slice(None)] * 3
            inner[ae] = slice(1, -1)
            flux[tuple(inner)] = ue_d[tuple(inner)] * ud_e
            lo = [slice(None)] * 3
            hi = [slice(None)] * 3
            lo[ae], hi[ae] = slice(0, -1), slice(1, None)
            dst = [slice(None)] * 3
            dst[ad] = slice(1, -1)
            acc[tuple(dst)] += (flux[tuple(hi)] - flux[tuple(lo)]) / h
        acc[~g.interior_face_mask(d)] = 0.0
        oc[d][...] = acc
    return out


def predictor_rhs(g: mac.Grid, dt: float, u_n, u_nm1, p_n, RF_n, f_body,
                  with_advection=True):
    """Right-hand side of the BDF2 momentum predictor, Eq. (ustar), on the
    interior faces (0 on the wall faces): moving the u^n and u^{n-1} parts of
    the BDF2 time derivative (3 u* - 4 u^n + u^{n-1})/(2 dt) to the right and
    keeping the explicit terms at time level n,

        rhs = (4 u^n - u^{n-1})/(2 dt) - G p^n + R F^n + f - A(u^n),

    with R F^n the spread force density (passed in as RF_n), f the prescribed
    body force on the faces and A the convective term (``advection``).  Shared
    by the one-way step and the two-way predictor of Eq. (ustar_two_way)."""
    rhs = (4.0 * u_n - u_nm1) / (2.0 * dt) - mac.apply_G(g, p_n) + RF_n + f_body
    if with_advection:
        rhs = rhs - advection(g, u_n)
    return np.where(g.interior_face_mask_packed(), rhs, 0.0)


def step(g: mac.Grid, Re: float, dt: float, X, U_gamma, f_body,
         u_n=None, u_nm1=None, p_n=None, F_n=None, mode="scalar",
         rtol=1e-13, with_advection=True, workers=None):
    """One step of Sec. 3.1; returns a dict of every intermediate."""
    X = np.asarray(X, dtype=np.float64).reshape(3, -1)
    nf, m, k = g.n_faces, g.m, 3 * X.shape[1]
    u_n = np.zeros(nf) if u_n is None else np.asarray(u_n, dtype=np.float64)
    u_nm1 = u_n if u_nm1 is None else np.asarray(u_nm1, dtype=np.float64)
    p_n = np.zeros(m) if p_n is None else np.asarray(p_n, dtype=np.float64)
    F_n = np.zeros(k) if F_n is None else np.asarray(F_n, dtype=np.float64)
    U_gamma = np.asarray(U_gamma, dtype=np.float64).ravel()
    a = 3.0 / (2.0 * dt)
    nu = 1.0 / Re
    sys = SchurSystem(g, X)

    rhs_u = predictor_rhs(g, dt, u_n, u_nm1, p_n, sys.R @ F_n,
                          np.asarray(f_body, dtype=np.float64), with_advection)
    u_star = helmholtz.solve(g, rhs_u, a, nu, workers=workers)

    rhs_p = a * mac.apply_GT(g, u_star)
    rhs_F = a * (sys.R.T @ u_star - U_gamma)
    if mode == "scalar":
        b = sys.rhs_scalar(rhs_p, rhs_F)
    elif mode == "exact":
        b = sys.rhs_exact(rhs_p, rhs_F)
    else:
        b = sys.rhs_consistent(rhs_p, rhs_F)
    p_corr, iters, relres, hist = solve_schur(sys, b, mode=mode, rtol=rtol,
                                              workers=workers)
    if mode == "scalar":
        F_corr = sys.force_scalar(p_corr, rhs_F)
    else:
        F_corr = sys.force_exact(p_corr, rhs_F)
    u_np1 = u_star + (2.0 * dt / 3.0) * (-mac.apply_G(g, p_corr) + sys.R @ F_corr)
    p_np1 = p_n + p_corr
    F_np1 = F_n + F_corr
    div = mac.apply_GT(g, u_np1)
    slip = sys.R.T @ u_np1 - U_gamma
    return dict(sys=sys, rhs_u=rhs_u, u_star=u_star, rhs_p=rhs_p, rhs_F=rhs_F,
                b=b, p_corr=p_corr, F_corr=F_corr, u=u_np1, p=p_np1, F=F_np1,
                iters=iters, relres=relres, hist=hist,
                div_l2=float(np.linalg.norm(div)),
                slip_l2=float(np.linalg.norm(slip)))


def body_force_torque(g: mac.Grid, X, F, body_id, centers):
    """Per body: IB force h^3 sum_k F_k (Eq. (IBM_force)) and torque
    h^3 sum_k (X_k - X_c) x F_k; returns array (n_bodies, 6)."""
    X = np.asarray(X, dtype=np.float64).reshape(3, -1)
    F = np.asarray(F, dtype=np.float64).reshape(3, -1)
    centers = np.asarray(centers, dtype=np.float64).reshape(-1, 3)
    body_id = np.asarray(body_id)
    out = np.zeros((centers.shape[0], 6))
    h3 = g.h ** 3
    for b in range(centers.shape[0]):
        sel = body_id == b
        r = X[:, sel] - centers[b][:, None]
        f = F[:, sel]
        out[b, :3] = h3 * f.sum(axis=1)
        out[b, 3:] = h3 * np.cross(r.T, f.T).sum(axis=0)
    return out
