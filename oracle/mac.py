"""Staggered MAC grid operators, FP64, CPU.  TEST INFRASTRUCTURE ONLY (see
``oracle/__init__``).

Grid (Sec. 3.1, Fig. "cell"): uniform spacing h on [0, nx h] x [0, ny h] x
[0, nz h]; pressure at cell centres, u_d on the faces normal to axis d.
Array layout is C order [z][y][x] (x fastest):

* cells        (nz, ny, nx)      centre ((i+1/2)h, (j+1/2)h, (k+1/2)h)
* u_x faces    (nz, ny, nx+1)    at (i h, (j+1/2)h, (k+1/2)h)
* u_y faces    (nz, ny+1, nx)
* u_z faces    (nz+1, ny, nx)

A packed face vector is ravel(u_x) ++ ravel(u_y) ++ ravel(u_z).  All walls are
no-slip, so the wall-normal faces on the boundary are not unknowns: their rows
of G are zero and their values stay 0.

G is the central-difference gradient from cells to interior faces,
(G p)_f = (p_{c+} - p_{c-}) / h, G^T is its exact transpose (= -div, the
symmetry Sec. 5 requires) and L = G^T G is the Neumann 7-point Laplacian
(negated), the leading block of Eq. (Saddle).

Pins (tests/test_oracle_mac.py): G 1 = 0; G^T equals minus the flux-form
divergence written out cell by cell; L equals the 7-point stencil written out
by loops; ``laplacian_pinv`` equals numpy's dense pseudo-inverse on small grids;
second-order accuracy on a manufactured cosine field.
"""
from __future__ import annotations

import numpy as np
import scipy.fft
import scipy.sparse as sp


class Grid:
    """Uniform MAC grid with nx*ny*nz cells of width h."""

    def __init__(self, nx: int, ny: int | None = None, nz: int | None = None,
                 h: float | None = None):
        ny = nx if ny is None else ny
        nz = nx if nz is None else nz
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.h = 1.0 / self.nx if h is None else float(h)
        self.cell_shape = (self.nz, self.ny, self.nx)
        self.face_shapes = ((self.nz, self.ny, self.nx + 1),
                            (self.nz, self.ny + 1, self.nx),
                            (self.nz + 1, self.ny, self.nx))
        self.m = self.nx * self.ny * self.nz
        self.face_sizes = tuple(int(np.prod(s)) for s in self.face_shapes)
        self.face_offsets = (0, self.face_sizes[0],
                             self.face_sizes[0] + self.face_sizes[1])
        self.n_faces = sum(self.face_sizes)

    def split_faces(self, u):
        """Packed face vector -> (u_x, u_y, u_z) views in their array shapes."""
        u = np.asarray(u)
        return tuple(u[o:o + s].reshape(sh) for o, s, sh in
                     zip(self.face_offsets, self.face_sizes, self.face_shapes))

    def pack_faces(self, ux, uy, uz):
        return np.concatenate([np.ravel(ux), np.ravel(uy), np.ravel(uz)])

    def face_coords(self, d: int):
        """Coordinates (x, y, z) of the d-faces, each of that face array's shape."""
        h = self.h
        sh = self.face_shapes[d]
        kk, jj, ii = np.meshgrid(np.arange(sh[0]), np.arange(sh[1]),
                                 np.arange(sh[2]), indexing="ij")
        x = (ii + (0.0 if d == 0 else 0.5)) * h
        y = (jj + (0.0 if d == 1 else 0.5)) * h
        z = (kk + (0.0 if d == 2 else 0.5)) * h
        return x, y, z

    def interior_face_mask(self, d: int):
        """True on faces that are unknowns (not wall-normal boundary faces)."""
        sh = self.face_shapes[d]
        mask = np.ones(sh, dtype=bool)
        axis = 2 - d              # array axis of coordinate d
        sl = [slice(None)] * 3
        sl[axis] = 0
        mask[tuple(sl)] = False
        sl[axis] = sh[axis] - 1
        mask[tuple(sl)] = False
        return mask

    def interior_face_mask_packed(self):
        return self.pack_faces(*(self.interior_face_mask(d) for d in range(3)))


def gradient_matrix(g: Grid) -> sp.csr_matrix:
    """G: cells -> packed faces, (G p)_f = (p_{c+} - p_{c-})/h on interior
    faces, zero rows on wall faces (Sec. 3.1, central differences)."""
    rows, cols, vals = [], [], []
    cell_index = np.arange(g.m).reshape(g.cell_shape)
    for d in range(3):
        sh = g.face_shapes[d]
        face_index = g.face_offsets[d] + np.arange(g.face_sizes[d]).reshape(sh)
        axis = 2 - d
        n_ax = g.cell_shape[axis]
        # interior faces along axis d have index 1..n_ax-1; the cell on the
        # + side has the same index, the cell on the - side index-1
        sl_face = [slice(None)] * 3
        sl_face[axis] = slice(1, n_ax)
        sl_plus = [slice(None)] * 3
        sl_plus[axis] = slice(1, n_ax)
        sl_minus = [slice(None)] * 3
        sl_minus[axis] = slice(0, n_ax - 1)
        f = face_index[tuple(sl_face)].ravel()
        cp = cell_index[tuple(sl_plus)].ravel()
        cm = cell_index[tuple(sl_minus)].ravel()
        rows += [f, f]
        cols += [cp, cm]
        vals += [np.full(f.size, 1.0 / g.h), np.full(f.size, -1.0 / g.h)]
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    return sp.csr_matrix((vals, (rows, cols)), shape=(g.n_faces, g.m))


def apply_G(g: Grid, p):
    """G p on the packed faces (same definition as ``gradient_matrix``,
    written with array differences; used at sizes where the sparse matrix is
    too large)."""
    p3 = np.asarray(p, dtype=np.float64).reshape(g.cell_shape)
    out = []
    for d in range(3):
        axis = 2 - d
        f = np.zeros(g.face_shapes[d])
        sl = [slice(None)] * 3
        sl[axis] = slice(1, g.cell_shape[axis])
        f[tuple(sl)] = np.diff(p3, axis=axis) / g.h
        out.append(f.ravel())
    return np.concatenate(out)


def apply_GT(g: Grid, u):
    """G^T u (the transpose of ``apply_G``; wall faces do not contribute)."""
    comps = g.split_faces(np.asarray(u, dtype=np.float64))
    out = np.zeros(g.cell_shape)
    for d in range(3):
        axis = 2 - d
        n = g.cell_shape[axis]
        f = comps[d]
        inner = [slice(None)] * 3
        inner[axis] = slice(1, n)
        fi = f[tuple(inner)] / g.h           # interior faces 1..n-1
        plus = [slice(None)] * 3
        plus[axis] = slice(1, n)             # cell on the + side of face i is i
        minus = [slice(None)] * 3
        minus[axis] = slice(0, n - 1)        # cell on the - side is i-1
        out[tuple(plus)] += fi
        out[tuple(minus)] -= fi
    return out.ravel()


def apply_L(g: Grid, v):
    """L v = G^T (G v)."""
    return apply_GT(g, apply_G(g, v))


def laplacian_matrix(g: Grid) -> sp.csr_matrix:
    """L = G^T G, the (negated) Neumann Laplacian, leading block of
    Eq. (Saddle)."""
    G = gradient_matrix(g)
    return (G.T @ G).tocsr()


def neumann_eigenvalues(g: Grid) -> np.ndarray:
    """Eigenvalues of L in the cosine basis cos(pi k (i+1/2)/n) per axis:
    lambda = sum_d (2 - 2 cos(pi k_d / n_d)) / h^2, array of cell shape."""
    lam = []
    for n in (g.nz, g.ny, g.nx):
        k = np.arange(n)
        lam.append((2.0 - 2.0 * np.cos(np.pi * k / n)) / g.h ** 2)
    return lam[0][:, None, None] + lam[1][None, :, None] + lam[2][None, None, :]


def laplacian_pinv(g: Grid, r, workers: int | None = None):
    """Exact pseudo-inverse L^+ r (mean-zero result) by the orthonormal
    DCT-II diagonalisation of the Neumann Laplacian: the uniform-grid form of
    the Kronecker-sum fast diagonalisation of Sec. 4.2.  The zero eigenvalue
    (constant mode) is dropped."""
    r3 = np.asarray(r, dtype=np.float64).reshape(g.cell_shape)
    rh = scipy.fft.dctn(r3, type=2, norm="ortho", workers=workers)
    lam = neumann_eigenvalues(g)
    lam[0, 0, 0] = 1.0
    rh = rh / lam
    rh[0, 0, 0] = 0.0
    return scipy.fft.idctn(rh, type=2, norm="ortho", workers=workers).ravel()


def remove_mean(v):
    v = np.asarray(v, dtype=np.float64)
    return v - v.mean()
