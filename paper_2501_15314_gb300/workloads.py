"""Seeded synthetic inputs shared by the CUDA library's tests/bench and the CPU
oracle.  This module holds input generation only (marker placement, random
rigid motions, a smooth random body force); none of the solver's arithmetic.

The paper's workloads are rigid spheres in a box (Sec. 6.1); its marker
layouts (equal-area partitions) and experimental data are not reproduced.
Synthetic stand-ins:

* markers on a sphere: a Fibonacci lattice, z_i = 1 - (2i+1)/N,
  azimuth 2 pi i / golden-ratio, radius r, centre c;
* marker count at Lagrangian spacing h_L: round(4 pi r^2 / h_L^2); the paper
  uses spacing close to the cell width (Sec. 6.1, Appendix A);
* several spheres: centres drawn uniformly in [r + 3h, 1 - r - 3h]^3 with
  every pair at least 3h apart surface to surface (the delta support of
  Eq. (delta) is 1.5h; Appendix B keeps bodies two cells apart), rejection
  sampling with the workload's seed;
* prescribed marker velocity U = u_s + omega x (X - c) with u_s, omega drawn
  uniformly in [-1, 1]^3 per body (the rigid kinematic constraint of
  Eq. (kinematic_constraint));
* body force on the faces: for each component, a sum of 8 modes
  sin(2 pi k . x + phase), k with integer entries in 1..4, phase uniform in
  [0, 2 pi), amplitude 1; wall-normal boundary faces are 0.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

GOLDEN = (1.0 + 5.0 ** 0.5) / 2.0


def fibonacci_sphere(n_markers: int, radius: float, center) -> np.ndarray:
    """(3, N) marker coordinates on a sphere (Fibonacci lattice)."""
    i = np.arange(n_markers, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / n_markers
    rho = np.sqrt(np.maximum(1.0 - z * z, 0.0))
    th = 2.0 * np.pi * i / GOLDEN
    pts = np.stack([rho * np.cos(th), rho * np.sin(th), z]) * radius
    return pts + np.asarray(center, dtype=np.float64).reshape(3, 1)


def markers_for_spacing(radius: float, spacing: float) -> int:
    return int(round(4.0 * np.pi * radius * radius / (spacing * spacing)))


def place_spheres(n_bodies: int, r_lo: float, r_hi: float, h: float,
                  rng: np.random.Generator, max_tries: int = 100000):
    """Non-overlapping sphere centres and radii in the unit cube."""
    radii = rng.uniform(r_lo, r_hi, size=n_bodies)
    centers = np.zeros((n_bodies, 3))
    for b in range(n_bodies):
        r = radii[b]
        for _ in range(max_tries):
            c = rng.uniform(r + 3 * h, 1.0 - r - 3 * h, size=3)
            ok = all(np.linalg.norm(c - centers[q]) >= r + radii[q] + 3 * h
                     for q in range(b))
            if ok:
                centers[b] = c
                break
        else:
            raise RuntimeError("sphere placement failed")
    return centers, radii


def rigid_velocities(X, body_id, centers, rng: np.random.Generator):
    """(3, N) marker velocities of random rigid motions, one per body."""
    X = np.asarray(X).reshape(3, -1)
    nb = centers.shape[0]
    us = rng.uniform(-1.0, 1.0, size=(nb, 3))
    om = rng.uniform(-1.0, 1.0, size=(nb, 3))
    r = X - centers[body_id].T
    w = om[body_id].T
    cross = np.stack([w[1] * r[2] - w[2] * r[1],
                      w[2] * r[0] - w[0] * r[2],
                      w[0] * r[1] - w[1] * r[0]])
    return us[body_id].T + cross


def sine_body_force(nx: int, ny: int, nz: int, h: float,
                    rng: np.random.Generator, n_modes: int = 8) -> np.ndarray:
    """Packed face vector (u_x | u_y | u_z) of a smooth random forcing."""
    shapes = ((nz, ny, nx + 1), (nz, ny + 1, nx), (nz + 1, ny, nx))
    out = []
    for d in range(3):
        sh = shapes[d]
        k3, j3, i3 = np.meshgrid(np.arange(sh[0]), np.arange(sh[1]),
                                 np.arange(sh[2]), indexing="ij")
        x = (i3 + (0.0 if d == 0 else 0.5)) * h
        y = (j3 + (0.0 if d == 1 else 0.5)) * h
        z = (k3 + (0.0 if d == 2 else 0.5)) * h
        kv = rng.integers(1, 5, size=(n_modes, 3))
        ph = rng.uniform(0.0, 2.0 * np.pi, size=n_modes)
        f = np.zeros(sh)
        for q in range(n_modes):
            f += np.sin(2.0 * np.pi * (kv[q, 0] * x + kv[q, 1] * y + kv[q, 2] * z)
                        + ph[q])
        ax = 2 - d
        sl = [slice(None)] * 3
        sl[ax] = 0
        f[tuple(sl)] = 0.0
        sl[ax] = sh[ax] - 1
        f[tuple(sl)] = 0.0
        out.append(f.ravel())
    return np.concatenate(out)


@dataclass
class Workload:
    name: str
    n: int
    Re: float
    dt: float
    X: np.ndarray             # (3, N)
    body_id: np.ndarray       # (N,) int32
    centers: np.ndarray       # (n_bodies, 3)
    radii: np.ndarray
    U_gamma: np.ndarray       # (3, N)
    f_body: np.ndarray        # packed faces
    info: dict = field(default_factory=dict)

    @property
    def h(self):
        return 1.0 / self.n

    @property
    def n_markers(self):
        return self.X.shape[1]


def spheres_workload(name: str, n: int, Re: float, dt: float, centers, radii,
                     n_markers_total: int | None, seed: int,
                     spacing_ratio: float = 1.0, rng=None) -> Workload:
    """Markers on each sphere (count per sphere proportional to its area when
    a total is given, else at Lagrangian spacing h / spacing_ratio), random
    rigid velocities and a random sine body force."""
    rng = np.random.default_rng(seed) if rng is None else rng
    h = 1.0 / n
    centers = np.asarray(centers, dtype=np.float64).reshape(-1, 3)
    radii = np.asarray(radii, dtype=np.float64).ravel()
    area = 4.0 * np.pi * radii ** 2
    if n_markers_total is None:
        counts = [markers_for_spacing(r, h / spacing_ratio) for r in radii]
    else:
        counts = list(np.floor(n_markers_total * area / area.sum()).astype(int))
        counts[-1] += n_markers_total - sum(counts)
    Xs, ids = [], []
    for b, (c, r, nm) in enumerate(zip(centers, radii, counts)):
        Xs.append(fibonacci_sphere(nm, r, c))
        ids.append(np.full(nm, b, dtype=np.int32))
    X = np.concatenate(Xs, axis=1)
    body_id = np.concatenate(ids)
    U = rigid_velocities(X, body_id, centers, rng)
    f = sine_body_force(n, n, n, h, rng)
    lag_spacing = np.sqrt(area.sum() / X.shape[1])
    info = dict(spacing_ratio=h / lag_spacing, counts=counts)
    return Workload(name, n, Re, dt, X, body_id, centers, radii, U, f, info)


def config(index: int, secondary: bool = False) -> Workload:
    """The five sphere workloads, seeded by their index.

    1: 32^3, one sphere r = 0.2 at the centre, Re 100, dt 0.01
    2: 128^3, one sphere r = 0.15 at the centre, Re 100, dt 2e-3
    3: 256^3, eight spheres, radii uniform in [0.05, 0.1], Re 200, dt 1e-3
    4: 128^3, the transversely oscillating sphere of Sec. 6.1.1 (adjoint
       workload): r = 0.15 (D = 0.3), A/D = 1, at nondimensional time t = 1
       of Eq. (u_z_and_z): centre z = 0.5 - A cos(t), every marker moving
       with U = sin(t) e_z; Re 100, dt 2e-3, from rest, no body force
    5: 384^3, one sphere r = 0.08, Re 50, dt 5e-4
    Primary marker counts put markers at spacing h; ``secondary`` uses the
    stated totals (1000, 16000, 60000, 16000, 25000)."""
    rng = np.random.default_rng(index)
    if index == 1:
        return spheres_workload("sphere32", 32, 100.0, 0.01, [[0.5] * 3], [0.2],
                                1000 if secondary else None, index, rng=rng)
    if index == 2:
        return spheres_workload("sphere128", 128, 100.0, 2e-3, [[0.5] * 3], [0.15],
                                16000 if secondary else None, index, rng=rng)
    if index == 4:
        return oscillating_sphere(128, 16000 if secondary else None, t=1.0)
    if index == 3:
        n = 256
        centers, radii = place_spheres(8, 0.05, 0.1, 1.0 / n, rng)
        W = spheres_workload("spheres8_256", n, 200.0, 1e-3, centers, radii,
                             60000 if secondary else None, index, rng=rng)
        W.info["radius_law"] = "in [0.05,0.1]"
        return W
    if index == 5:
        return spheres_workload("sediment384", 384, 50.0, 5e-4,
                                [[0.5, 0.5, 0.7]], [0.08],
                                25000 if secondary else None, index, rng=rng)
    raise ValueError(index)


def oscillating_sphere(n: int, n_markers: int | None, t: float = 1.0, radius: float = 0.15,
                       amp_ratio: float = 1.0, Re: float = 100.0, dt: float = 2e-3) -> Workload:
    """One sphere of diameter D = 2 radius oscillating along z (Eq. (U_z) in
    the nondimensional form (u_z_and_z), lengths in units of D): at time t
    the centre sits at 0.5 - A cos(t D/A) and every marker moves with
    sin(t D/A) e_z, A = amp_ratio D.  Zero body force."""
    D = 2.0 * radius
    A = amp_ratio * D
    centre = np.array([[0.5, 0.5, 0.5 - A * np.cos(t * D / A)]])
    h = 1.0 / n
    nm = markers_for_spacing(radius, h) if n_markers is None else n_markers
    X = fibonacci_sphere(nm, radius, centre[0])
    body_id = np.zeros(nm, dtype=np.int32)
    U = np.zeros((3, nm))
    U[2] = np.sin(t * D / A)
    nf = 3 * n * n * (n + 1)
    lag_spacing = np.sqrt(4.0 * np.pi * radius ** 2 / nm)
    info = dict(spacing_ratio=h / lag_spacing, counts=[nm], t=t, amp_ratio=amp_ratio)
    return Workload(f"oscillating_sphere{n}", n, Re, dt, X, body_id, centre,
                    np.array([radius]), U, np.zeros(nf), info)


# Table 1 (label spheresCenters) of the paper: centres of the sub-spheres of
# the porous-sphere models of Sec. 6.1.2, in units of the bounding diameter D
# (the table prints 10x these values) relative to the bounding centre, and the
# sub-sphere radius in units of D.  The 14-sphere entry 1 prints y = -2.287;
# the symmetry of entries 1-4 gives -2.2875, used here.
POROUS_CENTRES = {
    7: (0.193, [(1.1140, -1.9296, -2.1126), (-2.2281, 0.0, -2.1126), (1.1140, 1.9296, -2.1126),
                (-1.5009, -2.5997, 0.64522), (3.0019, 0.0, 0.64522), (-1.5009, 2.5997, 0.64522),
                (0.0, 0.0, 3.0704)]),
    14: (0.161, [(0.0, -2.2875, -2.4917), (-2.2875, 0.0, -2.4917), (2.2875, 0.0, -2.4917),
                 (0.0, 2.2875, -2.4917), (-2.3820, -2.3820, -0.30478), (2.3820, -2.3820, -0.30478),
                 (-2.3820, 2.3820, -0.30478), (2.3820, 2.3820, -0.30478), (0.0, 0.0, 0.0),
                 (0.0, -2.8412, 1.8355), (-2.8412, 0.0, 1.8355), (2.8412, 0.0, 1.8355),
                 (0.0, 2.8412, 1.8355), (0.0, 0.0, 3.3825)]),
}


def porous_sphere(n: int, n_sub: int, t: float = 1.0, D: float = 0.3, amp_ratio: float = 1.0,
                  Re: float = 100.0, dt: float = 2e-3, spacing_ratio: float = 1.0) -> Workload:
    """The porous sphere of Sec. 6.1.2: n_sub (7 or 14) rigid sub-spheres
    packed in a bounding sphere of diameter D (Table 1), each radius reduced
    by half a cell width, the whole array oscillating along z like the sphere
    of Sec. 6.1.1 (Eq. (u_z_and_z), A = amp_ratio D, at time t): bounding
    centre (0.5, 0.5, 0.5 - A cos(t D/A)), every marker moving with
    sin(t D/A) e_z.  Markers at Lagrangian spacing h / spacing_ratio on every
    sub-sphere; zero body force."""
    r_unit, cents = POROUS_CENTRES[n_sub]
    h = 1.0 / n
    A = amp_ratio * D
    c0 = np.array([0.5, 0.5, 0.5 - A * np.cos(t * D / A)])
    centers = c0[None, :] + 0.1 * D * np.asarray(cents, dtype=np.float64)
    r_sub = r_unit * D - 0.5 * h
    Xs, ids = [], []
    for b, c in enumerate(centers):
        nm = markers_for_spacing(r_sub, h / spacing_ratio)
        Xs.append(fibonacci_sphere(nm, r_sub, c))
        ids.append(np.full(nm, b, dtype=np.int32))
    X = np.concatenate(Xs, axis=1)
    body_id = np.concatenate(ids)
    U = np.zeros_like(X)
    U[2] = np.sin(t * D / A)
    nf = 3 * n * n * (n + 1)
    area = 4.0 * np.pi * r_sub ** 2 * n_sub
    info = dict(spacing_ratio=h / np.sqrt(area / X.shape[1]), counts=[len(i) for i in ids],
                t=t, bounding_centre=c0.tolist(), D=D, r_sub=r_sub)
    return Workload(f"porous{n_sub}_{n}", n, Re, dt, X, body_id, centers,
                    np.full(n_sub, r_sub), U, np.zeros(nf), info)


def small_spheres(n: int, n_bodies: int, seed: int, r_lo: float, r_hi: float,
                  Re: float = 100.0, dt: float = 0.01,
                  spacing_ratio: float = 1.0) -> Workload:
    """A small multi-sphere workload for parity tests (several tiles, ragged
    marker counts)."""
    rng = np.random.default_rng(seed)
    centers, radii = place_spheres(n_bodies, r_lo, r_hi, 1.0 / n, rng)
    return spheres_workload(f"spheres{n_bodies}_{n}", n, Re, dt, centers, radii,
                            None, seed, spacing_ratio=spacing_ratio, rng=rng)
