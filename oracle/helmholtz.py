"""BDF2 momentum predictor on the no-slip MAC grid, FP64, CPU.  TEST
INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Eq. (ustar): (3 u* - 4 u^n + u^{n-1})/(2 dt) = -grad p^n + (1/Re) Lap u*
+ R F^n - (u.grad u)^n, i.e. per velocity component

    (a I - nu Lap_h) u*_d = rhs_d,   a = 3/(2 dt),  nu = 1/Re,

with Lap_h the central 7-point Laplacian on the d-faces (Sec. 3.1).  Boundary
conditions (all walls no-slip, wall velocity 0): the wall-normal faces are not
unknowns and hold 0 (Dirichlet at the face); along the other two axes the ghost
value beyond a wall is minus the first interior value, so the velocity is 0 on
the wall midway between them.

``solve`` diagonalises the operator exactly, as the paper does with its
Kronecker-sum direct solver (Sec. 4.1, item 1): a type-I sine transform along
the face-normal axis (eigenvalues (2 - 2 cos(pi k/n))/h^2, k = 1..n-1) and a
type-II sine transform along the two cell-centred axes (eigenvalues
(2 - 2 cos(pi k/n))/h^2, k = 1..n).

``matrix`` assembles the same operator row by row from the stencil, for the
brute-force pin (tests/test_oracle_helmholtz.py), which also checks second-order
accuracy on a manufactured sine field.
"""
from __future__ import annotations

import numpy as np
import scipy.fft
import scipy.sparse as sp

from .mac import Grid


def _interior_slice(d):
    """Slice selecting the interior d-faces of a d-face array."""
    sl = [slice(None)] * 3
    sl[2 - d] = slice(1, -1)
    return tuple(sl)


def _eig_1d(n, h, face_axis):
    if face_axis:            # n-1 unknowns, Dirichlet at both end faces
        k = np.arange(1, n)
    else:                    # n unknowns, ghost = -interior at both ends
        k = np.arange(1, n + 1)
    return (2.0 - 2.0 * np.cos(np.pi * k / n)) / h ** 2


def solve(g: Grid, rhs, a: float, nu: float, workers=None):
    """u* (packed faces, wall faces 0) with (a - nu Lap_h) u* = rhs on the
    interior faces of each component."""
    out = np.zeros(g.n_faces)
    rhs_c = g.split_faces(np.asarray(rhs, dtype=np.float64))
    out_c = g.split_faces(out)
    ns = (g.nx, g.ny, g.nz)
    for d in range(3):
        r = rhs_c[d][_interior_slice(d)]
        lam = np.zeros(r.shape)
        for e in range(3):
            ax = 2 - e
            ev = _eig_1d(ns[e], g.h, face_axis=(e == d))
            shape = [1, 1, 1]
            shape[ax] = ev.size
            lam = lam + ev.reshape(shape)
            tp = 1 if e == d else 2
            r = scipy.fft.dst(r, type=tp, axis=ax, norm="ortho", workers=workers)
        r = r / (a + nu * lam)
        for e in range(3):
            tp = 1 if e == d else 2
            r = scipy.fft.idst(r, type=tp, axis=2 - e, norm="ortho", workers=workers)
        out_c[d][_interior_slice(d)] = r
    return out


def apply(g: Grid, u, a: float, nu: float):
    """(a - nu Lap_h) u on interior faces (0 on wall faces), by the stencil."""
    u_c = g.split_faces(np.asarray(u, dtype=np.float64))
    out = np.zeros(g.n_faces)
    out_c = g.split_faces(out)
    for d in range(3):
        v = u_c[d].copy()
        mask = g.interior_face_mask(d)
        v[~mask] = 0.0
        lap = np.zeros_like(v)
        for e in range(3):
            ax = 2 - e
            n = v.shape[ax]
            vp = np.zeros_like(v)
            vm = np.zeros_like(v)
            sl_to = [slice(None)] * 3
            sl_from = [slice(None)] * 3
            sl_to[ax], sl_from[ax] = slice(0, n - 1), slice(1, n)
            vp[tuple(sl_to)] = v[tuple(sl_from)]
            sl_to[ax], sl_from[ax] = slice(1, n), slice(0, n - 1)
            vm[tuple(sl_to)] = v[tuple(sl_from)]
            if e != d:      # ghost = -interior beyond the walls
                sl = [slice(None)] * 3
                sl[ax] = 0
                vm[tuple(sl)] = -v[tuple(sl)]
                sl[ax] = n - 1
                vp[tuple(sl)] = -v[tuple(sl)]
            lap += (vp - 2.0 * v + vm) / g.h ** 2
        res = a * v - nu * lap
        res[~mask] = 0.0
        out_c[d][...] = res
    return out


def matrix(g: Grid, a: float, nu: float) -> sp.csr_matrix:
    """The operator of ``apply`` assembled entry by entry from the stencil
    (rows and columns over all packed faces; wall rows/cols empty)."""
    rows, cols, vals = [], [], []
    ns = (g.nx, g.ny, g.nz)
    for d in range(3):
        sh = g.face_shapes[d]
        mask = g.interior_face_mask(d)
        for k in range(sh[0]):
            for j in range(sh[1]):
                for i in range(sh[2]):
                    if not mask[k, j, i]:
                        continue
                    row = g.face_offsets[d] + (k * sh[1] + j) * sh[2] + i
                    diag = a
                    idx = (i, j, k)
                    for e in range(3):
                        n_pts = sh[2 - e]
                        for step in (-1, 1):
                            q = list(idx)
                            q[e] += step
                            diag += 2.0 * nu / g.h ** 2 / 2.0
                            if 0 <= q[e] < n_pts:
                                qi, qj, qk = q
                                if e == d and (q[e] == 0 or q[e] == n_pts - 1):
                                    continue          # wall face: value 0
                                col = g.face_offsets[d] + (qk * sh[1] + qj) * sh[2] + qi
                                rows.append(row)
                                cols.append(col)
                                vals.append(-nu / g.h ** 2)
                            else:                       # ghost = -interior
                                diag += nu / g.h ** 2
                    rows.append(row)
                    cols.append(row)
                    vals.append(diag)
    return sp.csr_matrix((vals, (rows, cols)), shape=(g.n_faces, g.n_faces))
