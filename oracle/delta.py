"""Roma's discrete delta and the regularisation / interpolation operators,
FP64, CPU.  TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

* ``phi(r)``: Delta r * delta(r) of Eq. (delta), with r in units of the cell
  width: (1 + sqrt(1 - 3 r^2))/3 for |r| <= 1/2,
  (5 - 3|r| - sqrt(1 - 3 (1 - |r|)^2))/6 for 1/2 < |r| <= 3/2, else 0.
* ``phi_prime(r)``: d phi / dr, from differentiating the two branches of
  Eq. (delta): -r / sqrt(1 - 3 r^2) for |r| <= 1/2 and
  -sign(r) (1 + (1 - |r|)/sqrt(1 - 3 (1 - |r|)^2)) / 2 for 1/2 < |r| < 3/2.
* ``regularization_matrix``: R with (R F)_i = dx^3 sum_k F_k delta^3(x_i - X_k)
  (Eq. (regularization)).  dx^3 delta^3 = phi phi phi, so the entry for face i
  of component d and the d-component of marker k is
  phi((x_i-X_k)/h) phi((y_i-Y_k)/h) phi((z_i-Z_k)/h).  Columns are ordered
  component-major: column d*N + k.  Each component spreads only to its own
  face grid.  The interpolation operator of Eq. (interpolation) is its exact
  transpose R^T (same delta on both sides, Sec. 2.3).

The paper requires the delta's support to lie on grid points that exist
(Appendix B); with no-slip walls those are the interior faces.  A marker with a
nonzero weight on a wall-normal boundary face or outside the grid is rejected
with ``ValueError``.

Pins (tests/test_oracle_delta.py): closed-form values and the zeroth, first
and squared-sum moments of phi; R^T computed by an independent brute-force
double loop over all faces and markers; partition of unity; force
conservation; exact interpolation of linear fields and second-order
interpolation of a smooth field; the average row sum of R^T R against Table
A1 (RtR_spacing).  phi_prime
and ``regularization_derivative`` are pinned to central differences of phi
and R, the values -1 and 0 at the breakpoints and the differentiated moment
identities (tests/test_oracle_adjoint.py).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .mac import Grid


def phi(r):
    """Eq. (delta) times the cell width, r in cell widths."""
    r = np.abs(np.asarray(r, dtype=np.float64))
    out = np.zeros_like(r)
    inner = r <= 0.5
    outer = (r > 0.5) & (r <= 1.5)
    ri = r[inner]
    out[inner] = (1.0 + np.sqrt(np.maximum(1.0 - 3.0 * ri * ri, 0.0))) / 3.0
    ro = r[outer]
    out[outer] = (5.0 - 3.0 * ro
                  - np.sqrt(np.maximum(1.0 - 3.0 * (1.0 - ro) ** 2, 0.0))) / 6.0
    return out


def phi_prime(r):
    """Derivative of ``phi`` with respect to r (r in cell widths)."""
    r = np.asarray(r, dtype=np.float64)
    a = np.abs(r)
    out = np.zeros_like(r)
    inner = a <= 0.5
    outer = (a > 0.5) & (a < 1.5)
    ri = r[inner]
    out[inner] = -ri / np.sqrt(1.0 - 3.0 * ri * ri)
    q = 1.0 - a[outer]
    out[outer] = -np.sign(r[outer]) * 0.5 * (1.0 + q / np.sqrt(1.0 - 3.0 * q * q))
    return out


def _axis_candidates(s, offset, n_points):
    """Grid indices j with positions (j + offset) within two cells of s
    (s in cell widths); returns indices (N, 5) and distances (N, 5)."""
    base = np.floor(s - offset).astype(np.int64) - 2
    j = base[:, None] + np.arange(5)[None, :]
    dist = (j + offset) - s[:, None]
    return j, dist


def regularization_matrix(g: Grid, X) -> sp.csr_matrix:
    """R (n_faces x 3N) of Eq. (regularization); X has shape (3, N) (rows
    x, y, z of the markers).  Raises ValueError if any nonzero weight falls on
    a non-interior face."""
    return _regularization(g, X, None)


def regularization_derivative(g: Grid, X, axis: int) -> sp.csr_matrix:
    """dR/dX_axis: the entry of face i and marker column d*N + k is the
    derivative of R's entry with respect to coordinate ``axis`` of marker k,
    -(1/h) phi'((x_axis,i - X_axis,k)/h) times the other two phi factors."""
    return _regularization(g, X, axis)


def _regularization(g: Grid, X, deriv_axis):
    X = np.asarray(X, dtype=np.float64).reshape(3, -1)
    N = X.shape[1]
    h = g.h
    rows, cols, vals = [], [], []
    for d in range(3):
        shape = g.face_shapes[d]                  # (nz, ny, nx+...)
        n_pts = (shape[2], shape[1], shape[0])    # points along x, y, z
        mask = g.interior_face_mask(d)
        idx, w = [], []
        for e in range(3):
            offset = 0.0 if e == d else 0.5       # face axis vs centre axis
            j, dist = _axis_candidates(X[e] / h, offset, n_pts[e])
            idx.append(j)
            if e == deriv_axis:
                w.append(-phi_prime(dist) / h)
            else:
                w.append(phi(dist))
        # outer product of the three 1-D candidate sets: (N, 5, 5, 5)
        W = (w[2][:, :, None, None] * w[1][:, None, :, None]
             * w[0][:, None, None, :])
        I = np.broadcast_to(idx[0][:, None, None, :], W.shape)
        J = np.broadcast_to(idx[1][:, None, :, None], W.shape)
        K = np.broadcast_to(idx[2][:, :, None, None], W.shape)
        col = np.broadcast_to((d * N + np.arange(N))[:, None, None, None], W.shape)
        nz = W != 0.0
        I, J, K, col, Wv = I[nz], J[nz], K[nz], col[nz], W[nz]
        inside = ((I >= 0) & (I < n_pts[0]) & (J >= 0) & (J < n_pts[1])
                  & (K >= 0) & (K < n_pts[2]))
        if not np.all(inside):
            raise ValueError("marker delta support leaves the grid")
        if not np.all(mask[K, J, I]):
            raise ValueError("marker delta support touches a wall face")
        flat = g.face_offsets[d] + (K * shape[1] + J) * shape[2] + I
        rows.append(flat)
        cols.append(col)
        vals.append(Wv)
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    return sp.csr_matrix((vals, (rows, cols)), shape=(g.n_faces, 3 * N))


def interp_bruteforce(g: Grid, X, u):
    """(R^T u)_k of Eq. (interpolation) by a plain double loop over every face
    of every component and every marker (tiny grids only)."""
    X = np.asarray(X, dtype=np.float64).reshape(3, -1)
    N = X.shape[1]
    comps = g.split_faces(u)
    out = np.zeros((3, N))
    for d in range(3):
        x, y, z = g.face_coords(d)
        for k in range(N):
            w = (phi((x - X[0, k]) / g.h) * phi((y - X[1, k]) / g.h)
                 * phi((z - X[2, k]) / g.h))
            out[d, k] = np.sum(w * comps[d])
    return out.ravel()
