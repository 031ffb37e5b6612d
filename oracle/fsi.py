"""Two-way coupled rigid spheres (Sec. 3.2), FP64, CPU.  TEST INFRASTRUCTURE
ONLY (see ``oracle/__init__``).

Per time step, in the paper's order (Sec. 3.2.1, a = 3/(2 dt)):

Step 1  explicit prediction of every sphere's position and orientation: the
        centre by the BDF2 form of Eq. (particle_position),
        X_c^{n+1} = (4 X_c^n - X_c^{n-1})/3 + (2/3) dt u_s^n, the orientation by
        the Rodrigues update (Eqs. (rotat_axis)-(next_time_step_matr)) with the
        Adams-Bashforth angle of Eq. (theta), and the markers at
        X_c^{n+1} + R^{n+1} L0 (L0: body-frame offsets).  Fixed for the step.
Step 2  the momentum predictor (Eq. (ustar_two_way)) at the new marker
        positions, giving u^{(0)}.
Step 3  corrections k = 0, 1, ...:
        * u_s^{(k)}, omega_s^{(k)} from the BDF2 forms of Newton's laws,
          Eqs. (bdy_linear_vel_iter), (bdy_angular_vel_iter), with the IB force
          and torque of F^{(n,k)} and the fluid momentum inside the sphere of
          Eq. (volume_integrals) (volume fractions alpha from the signed
          distance at the corners of each control volume, the linear
          reconstruction of Kempe & Froehlich 2012);
        * U^{(k)} = u_s^{(k)} + omega_s^{(k)} x (X_k - X_c)
          (Eq. (kinematic_constraint_iterative));
        * the correction system of Eq. (pressure_force_iterative_system) in
          its scalar Schur form (Eqs. (tildeSp)-(ApproxSchurPrimalF));
        * relaxed updates p += xi p', F += xi F',
          u += xi (1/a)(-G p' + R F'), until
          ||F'||_1 / ||F^{(n,k+1)}||_1 < tol (Eq. (convergence_criterion)).

Units: the paper writes Newton's laws for a sphere of diameter 1 (inertia
rho_f D^5).  Here lengths are those of the unit cube: a sphere of radius r
has volume V = 4 pi r^3 / 3 and moment of inertia theta J with J = 2 V r^2 / 5
(fluid density 1); with r = 1/2 the coefficients 6/(pi theta) and
60/(pi theta) of Eqs. (linear_momentum_sb_norm), (angular_momentum_sb_norm)
come back.  Gravity is a vector g (the paper's -Fr^{-2} e_z); the buoyancy-
corrected term is (theta - 1)/theta g.

The angular velocity is integrated in the inertial frame: for a sphere the
inertia is isotropic, so this equals the paper's body-frame solve; the
body-frame vector omega_cs = R^T omega_s feeds the Rodrigues update.  The
fluid angular momentum is taken about the sphere's centre at each time level.

Pins (tests/test_oracle_fsi.py): sum of the volume fractions against the
sphere volume (second order), the fluid momentum of uniform and rigidly
rotating fields against V u and J omega, the Rodrigues increment against a
rotation by gamma, the BDF2 rigid update reproducing free fall exactly, a step
with fixed bodies and one correction equal to ``oracle.step``, the converged
correction loop satisfying div u = 0 and the no-slip condition, and a free
heavy sphere falling slower than in vacuum.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import helmholtz, mac
from .schur import SchurSystem, solve_schur
from .step import predictor_rhs


@dataclass
class RigidSphere:
    radius: float
    theta: float                    # rho_p / rho_f
    xc: np.ndarray                  # centre at t^n
    xc_prev: np.ndarray             # centre at t^{n-1}
    us: np.ndarray = field(default_factory=lambda: np.zeros(3))
    us_prev: np.ndarray = field(default_factory=lambda: np.zeros(3))
    om: np.ndarray = field(default_factory=lambda: np.zeros(3))       # inertial frame
    om_prev: np.ndarray = field(default_factory=lambda: np.zeros(3))
    om_cs: np.ndarray = field(default_factory=lambda: np.zeros(3))    # body frame, t^n
    om_cs_prev: np.ndarray = field(default_factory=lambda: np.zeros(3))
    rot: np.ndarray = field(default_factory=lambda: np.eye(3))       # body -> inertial
    mom: np.ndarray = field(default_factory=lambda: np.zeros(3))      # int u dV, t^n
    mom_prev: np.ndarray = field(default_factory=lambda: np.zeros(3))
    amom: np.ndarray = field(default_factory=lambda: np.zeros(3))     # int r x u dV, t^n
    amom_prev: np.ndarray = field(default_factory=lambda: np.zeros(3))
    free: bool = True               # False: velocities held (prescribed motion)

    @property
    def volume(self):
        return 4.0 * np.pi * self.radius ** 3 / 3.0

    @property
    def inertia(self):               # per unit density: (2/5) V r^2
        return 0.4 * self.volume * self.radius ** 2


def volume_fraction(g: mac.Grid, d: int, center, radius):
    """alpha of the control volume of every d-face (the cell shifted by h/2
    along d): sum over its 8 corners of max(-phi, 0) divided by the sum of
    |phi|, phi = |x - c| - r the signed distance (Kempe & Froehlich 2012)."""
    x, y, z = g.face_coords(d)
    h = g.h
    c = np.asarray(center, dtype=np.float64)
    num = np.zeros(x.shape)
    den = np.zeros(x.shape)
    for sx in (-0.5, 0.5):
        for sy in (-0.5, 0.5):
            for sz in (-0.5, 0.5):
                phi = np.sqrt((x + sx * h - c[0]) ** 2 + (y + sy * h - c[1]) ** 2
                              + (z + sz * h - c[2]) ** 2) - radius
                num += np.maximum(-phi, 0.0)
                den += np.abs(phi)
    return np.where(den > 0.0, num / np.where(den > 0.0, den, 1.0), 0.0)


def fluid_momentum(g: mac.Grid, u, center, radius):
    """(int_{V_p} u dV, int_{V_p} (x - c) x u dV) by Eq. (volume_integrals):
    sum over the d-faces of alpha u_d h^3 (times the lever arm for the
    angular part)."""
    comps = g.split_faces(np.asarray(u, dtype=np.float64))
    c = np.asarray(center, dtype=np.float64)
    h3 = g.h ** 3
    lin = np.zeros(3)
    ang = np.zeros(3)
    for d in range(3):
        w = volume_fraction(g, d, c, radius) * comps[d] * h3
        w = np.where(g.interior_face_mask(d), w, 0.0)
        lin[d] = w.sum()
        x, y, z = g.face_coords(d)
        r = (x - c[0], y - c[1], z - c[2])
        e = np.zeros(3)
        e[d] = 1.0
        # r x (w e_d), summed
        ang[0] += np.sum(r[1] * w * e[2] - r[2] * w * e[1])
        ang[1] += np.sum(r[2] * w * e[0] - r[0] * w * e[2])
        ang[2] += np.sum(r[0] * w * e[1] - r[1] * w * e[0])
    return lin, ang


def skew(v):
    return np.array([[0.0, -v[2], v[1]], [v[2], 0.0, -v[0]], [-v[1], v[0], 0.0]])


def rodrigues_increment(om_cs, om_cs_prev, dt):
    """R_Delta of Eq. (incement_matr): axis om_cs / |om_cs| (Eq. (rotat_axis)),
    angle dt (3/2 |om_cs^n| - 1/2 |om_cs^{n-1}|) (Eq. (theta))."""
    nrm = float(np.linalg.norm(om_cs))
    if nrm == 0.0:
        return np.eye(3)
    W = skew(np.asarray(om_cs) / nrm)
    gam = dt * (1.5 * nrm - 0.5 * float(np.linalg.norm(om_cs_prev)))
    return np.eye(3) + np.sin(gam) * W + (1.0 - np.cos(gam)) * (W @ W)


def rigid_velocities(b: RigidSphere, dt, F_sum, T_sum, lin, ang, gravity):
    """(u_s^{(k)}, omega_s^{(k)}) of Eqs. (bdy_linear_vel_iter),
    (bdy_angular_vel_iter) for one sphere: F_sum, T_sum the IB force and
    torque (h^3 sum F_k, h^3 sum (X_k - X_c) x F_k), lin, ang the fluid
    momentum inside the sphere at the new position with the current iterate."""
    if not b.free:
        return b.us.copy(), b.om.copy()
    V, J, th = b.volume, b.inertia, b.theta
    g = np.asarray(gravity, dtype=np.float64)
    us = ((4.0 * b.us - b.us_prev) / 3.0 - (2.0 * dt / 3.0) * F_sum / (th * V)
          + (3.0 * lin - 4.0 * b.mom + b.mom_prev) / (3.0 * th * V)
          + (2.0 * dt / 3.0) * (th - 1.0) / th * g)
    om = ((4.0 * b.om - b.om_prev) / 3.0 - (2.0 * dt / 3.0) * T_sum / (th * J)
          + (3.0 * ang - 4.0 * b.amom + b.amom_prev) / (3.0 * th * J))
    return us, om


def fsi_step(g: mac.Grid, Re: float, dt: float, bodies, L0, body_id, u_n, u_nm1, p_n, F_n,
             f_body=None, gravity=(0.0, 0.0, 0.0), xi=1.0, tol=1e-3, max_inner=50,
             rtol=1e-13, with_advection=True, workers=None, criterion="lagrangian"):
    """One two-way step.  bodies: list of RigidSphere (updated in place to
    t^{n+1}); L0 (3, N) body-frame marker offsets; body_id (N,).  Returns a
    dict with u, p, F, X (markers at t^{n+1}), inner (correction count),
    iters (FGMRES iterations per correction), ratio (last ||F'||_1/||F||_1,
    or ||R F'||_1/||R F||_1 with criterion="eulerian": the stopping test of
    Eq. (convergence_criterion) on the force densities spread to the faces)."""
    L0 = np.asarray(L0, dtype=np.float64).reshape(3, -1)
    body_id = np.asarray(body_id)
    N = L0.shape[1]
    a = 3.0 / (2.0 * dt)
    nu = 1.0 / Re
    # Step 1: positions and orientations
    rot_new, xc_new = [], []
    X = np.zeros((3, N))
    for bi, b in enumerate(bodies):
        R1 = b.rot @ rodrigues_increment(b.om_cs, b.om_cs_prev, dt)
        x1 = (4.0 * b.xc - b.xc_prev) / 3.0 + (2.0 / 3.0) * dt * b.us
        sel = body_id == bi
        X[:, sel] = x1[:, None] + R1 @ L0[:, sel]
        rot_new.append(R1)
        xc_new.append(x1)
    lever = X - np.stack([xc_new[i] for i in body_id], axis=1) if N else X
    sys = SchurSystem(g, X)
    # Step 2: predictor
    u_n = np.asarray(u_n, dtype=np.float64)
    u_nm1 = np.asarray(u_nm1, dtype=np.float64)
    p = np.asarray(p_n, dtype=np.float64).copy()
    F = np.asarray(F_n, dtype=np.float64).ravel().copy()
    rhs = predictor_rhs(g, dt, u_n, u_nm1, p, sys.R @ F,
                        0.0 if f_body is None else np.asarray(f_body, dtype=np.float64),
                        with_advection)
    u = helmholtz.solve(g, rhs, a, nu, workers=workers)
    # Step 3: corrections
    h3 = g.h ** 3
    iters, ratio, inner = [], np.inf, 0
    vel = [(b.us.copy(), b.om.copy()) for b in bodies]
    for k in range(max_inner):
        Fk = F.reshape(3, -1)
        U = np.zeros((3, N))
        for bi, b in enumerate(bodies):
            sel = body_id == bi
            F_sum = h3 * Fk[:, sel].sum(axis=1)
            T_sum = h3 * np.cross(lever[:, sel].T, Fk[:, sel].T).sum(axis=0)
            lin, ang = fluid_momentum(g, u, xc_new[bi], b.radius)
            us, om = rigid_velocities(b, dt, F_sum, T_sum, lin, ang, gravity)
            vel[bi] = (us, om)
            U[:, sel] = us[:, None] + np.cross(om, lever[:, sel].T).T
        rhs_p = a * mac.apply_GT(g, u)
        rhs_F = a * (sys.R.T @ u - U.ravel())
        pc, it, _, _ = solve_schur(sys, sys.rhs_scalar(rhs_p, rhs_F), rtol=rtol, workers=workers)
        Fc = sys.force_scalar(pc, rhs_F)
        p = p + xi * pc
        F = F + xi * Fc
        u = u + xi * (1.0 / a) * (-mac.apply_G(g, pc) + sys.R @ Fc)
        iters.append(it)
        inner = k + 1
        # Eq. (convergence_criterion) on the marker force densities, or on
        # the force densities spread to the faces (what the fluid receives)
        if criterion == "eulerian":
            nF = np.abs(sys.R @ F).sum()
            ratio = np.abs(sys.R @ Fc).sum() / nF if nF > 0 else 0.0
        else:
            nF = np.abs(F).sum()
            ratio = np.abs(Fc).sum() / nF if nF > 0 else 0.0
        if ratio < tol:
            break
    # advance the bodies to t^{n+1}
    for bi, b in enumerate(bodies):
        us, om = vel[bi]
        lin, ang = fluid_momentum(g, u, xc_new[bi], b.radius)
        b.xc_prev, b.xc = b.xc.copy(), xc_new[bi]
        b.us_prev, b.us = b.us.copy(), us
        b.om_prev, b.om = b.om.copy(), om
        b.rot = rot_new[bi]
        b.om_cs_prev, b.om_cs = b.om_cs.copy(), rot_new[bi].T @ om
        b.mom_prev, b.mom = b.mom.copy(), lin
        b.amom_prev, b.amom = b.amom.copy(), ang
    return dict(u=u, p=p, F=F, X=X, inner=inner, iters=iters, ratio=ratio, sys=sys)
