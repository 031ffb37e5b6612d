"""Grid convergence of one oracle time step (TEST INFRASTRUCTURE ONLY: a
measurement on the oracle, run by hand with ``python -m oracle.step_convergence``).

One step from rest on 32^3, 64^3 and 128^3 (Re 1, dt 0.01, so the viscous
length sqrt(nu dt) = 0.1 spans at least 3 cells): a sphere of radius 0.2 at
the centre, markers at spacing h, moving rigidly (u_s = (0.3, -0.2, 0.1),
omega = e_z), and the body force (d+1) sin(2 pi x) sin(2 pi y) sin(2 pi z) on
component d.  The differences between successive grids (fine faces averaged
2 x 2 across onto the coarse faces they cover, fine cells 2 x 2 x 2 onto the
coarse cell) in the h^3-weighted L2 and the max norms give the observed
orders.  The paper states only the first-order accuracy of the regularised
delta (Sec. 2.3, footnote); after a single SIMPLE correction the velocity
also carries the step's constraint residual (Gᵀu = (4 dt/3) BᵀF',
Rᵀu - U = (dt/3)(2C - I) F'), which depends on the marker layout at each
grid, so these orders describe one step of the method, not its accuracy.
"""
from __future__ import annotations

import numpy as np

from . import mac, step


def fibonacci_sphere(n, r, c):
    i = np.arange(n) + 0.5
    zz = 1.0 - 2.0 * i / n
    rho = np.sqrt(1.0 - zz * zz)
    th = np.pi * (1.0 + 5.0 ** 0.5) * i
    return np.stack([c[0] + r * rho * np.cos(th), c[1] + r * rho * np.sin(th), c[2] + r * zz])


def run(n, r=0.2, Re=1.0, dt=0.01):
    g = mac.Grid(n)
    c = np.array([0.5, 0.5, 0.5])
    X = fibonacci_sphere(int(round(4.0 * np.pi * r * r * n * n)), r, c)
    us, om = np.array([0.3, -0.2, 0.1]), np.array([0.0, 0.0, 1.0])
    U = (us[:, None] + np.cross(om, (X - c[:, None]).T).T).ravel()
    parts = [np.zeros(sh) for sh in g.face_shapes]
    for d in range(3):
        x, y, z = g.face_coords(d)
        parts[d][...] = (d + 1) * np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y) * np.sin(2 * np.pi * z)
    f = g.pack_faces(*parts) * g.interior_face_mask_packed()
    return g, step.step(g, Re, dt, X, U, f, rtol=1e-12)


def restrict_faces(gf, gc, u):
    out = []
    for d, uf in enumerate(gf.split_faces(u)):
        ad = 2 - d
        sl = [slice(None)] * 3
        sl[ad] = slice(0, None, 2)
        v = uf[tuple(sl)]
        for ax in range(3):
            if ax != ad:
                v = 0.5 * (v.take(range(0, v.shape[ax], 2), axis=ax) +
                           v.take(range(1, v.shape[ax], 2), axis=ax))
        out.append(v)
    return gc.pack_faces(*out)


def restrict_cells(gf, p):
    a = p.reshape(gf.cell_shape)
    return a.reshape(a.shape[0] // 2, 2, a.shape[1] // 2, 2, a.shape[2] // 2, 2).mean(axis=(1, 3, 5))


def orders(ns=(32, 64, 128)):
    res = {n: run(n) for n in ns}
    out = {}
    for q in ("u", "p"):
        e2, einf = [], []
        for n in ns[:-1]:
            gc, oc = res[n]
            gf, of = res[2 * n]
            if q == "u":
                d = restrict_faces(gf, gc, of["u"]) - oc["u"]
            else:
                d = (restrict_cells(gf, of["p"]) - oc["p"].reshape(gc.cell_shape)).ravel()
            e2.append(np.sqrt(gc.h ** 3 * np.sum(d * d)))
            einf.append(np.max(np.abs(d)))
        out[q] = {"L2": [float(np.log2(a / b)) for a, b in zip(e2, e2[1:])],
                  "max": [float(np.log2(a / b)) for a, b in zip(einf, einf[1:])],
                  "L2_diffs": e2, "max_diffs": einf}
    return out


if __name__ == "__main__":
    import json
    print(json.dumps(orders(), indent=1))
