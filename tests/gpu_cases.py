"""Seeded GPU test cases (grid + markers + inputs) and tensor helpers."""
import numpy as np

from paper_2501_15314_gb300 import workloads as wl


def dev(x, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


class Case:
    def __init__(self, name, nx, ny, nz, h, X, body_id=None, centers=None, Re=100.0, dt=0.01,
                 seed=0):
        self.name, self.nx, self.ny, self.nz, self.h = name, nx, ny, nz, h
        self.X = np.ascontiguousarray(np.asarray(X, dtype=np.float64).reshape(3, -1))
        self.N = self.X.shape[1]
        self.body_id = body_id if body_id is not None else np.zeros(self.N, dtype=np.int32)
        self.centers = centers
        self.Re, self.dt = Re, dt
        self.rng = np.random.default_rng(seed)

    def grid(self):
        from oracle import mac
        return mac.Grid(self.nx, self.ny, self.nz, self.h)


def sphere16():
    W = wl.spheres_workload("s16", 16, 100.0, 0.01, [[0.5, 0.47, 0.52]], [0.3], None, 11)
    return Case("sphere16", 16, 16, 16, 1 / 16, W.X, W.body_id, W.centers, seed=1)


def ragged_multi():
    """48 x 40 x 32 cells (ragged against the 32 x 8 thread tiles), three
    spheres of different sizes, marker counts not multiples of any block."""
    h = 1.0 / 48
    centers = np.array([[0.3, 0.4, 0.33], [0.7, 0.42, 0.35], [0.5, 0.62, 0.36]])
    radii = np.array([0.12, 0.1, 0.085])
    Xs, ids = [], []
    for b, (c, r) in enumerate(zip(centers, radii)):
        nm = wl.markers_for_spacing(r, h) + 7 * b
        Xs.append(wl.fibonacci_sphere(nm, r, c))
        ids.append(np.full(nm, b, dtype=np.int32))
    X = np.concatenate(Xs, axis=1)
    return Case("ragged48x40x32", 48, 40, 32, h, X, np.concatenate(ids), centers, Re=150.0,
                dt=0.004, seed=2)


def config_case(index, secondary=False):
    W = wl.config(index, secondary)
    c = Case(W.name, W.n, W.n, W.n, W.h, W.X, W.body_id, W.centers, Re=W.Re, dt=W.dt,
             seed=index)
    c.U_gamma = W.U_gamma.ravel()
    c.f_body = W.f_body
    return c


def wide_grid():
    """160 x 24 x 40 cells: two 128-face blocks along x (the second one
    ragged), ragged y and z tiles, one sphere of radius 0.03 at spacing h."""
    h = 1.0 / 160
    c = np.array([0.52, 0.075, 0.12])
    X = wl.fibonacci_sphere(wl.markers_for_spacing(0.03, h), 0.03, c)
    return Case("wide160x24x40", 160, 24, 40, h, X, None, c[None, :], Re=100.0, dt=0.004,
                seed=4)
