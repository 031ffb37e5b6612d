"""The seeded input generators shared by the oracle and the CUDA path: the
placement rule for several spheres (centres at least r + 3h from the walls,
surfaces at least 3h apart, so that the delta support of every marker stays
on interior faces and bodies stay two cells apart as in Appendix B), markers
on the sphere, rigid prescribed velocities, the sine body force, marker counts
and determinism under the seed."""
import numpy as np
import pytest

from paper_2501_15314_gb300 import workloads as wl


def test_eight_sphere_placement_rule():
    n = 256
    h = 1.0 / n
    rng = np.random.default_rng(3)                 # the 256^3 workload's seed
    centers, radii = wl.place_spheres(8, 0.05, 0.1, h, rng)
    assert np.all((radii >= 0.05) & (radii <= 0.1))
    for c, r in zip(centers, radii):
        assert np.all(c >= r + 3 * h) and np.all(c <= 1.0 - r - 3 * h)
    for a in range(8):
        for b in range(a):
            gap = np.linalg.norm(centers[a] - centers[b]) - radii[a] - radii[b]
            assert gap >= 3 * h, (a, b, gap / h)


def test_inputs_are_deterministic_under_the_seed():
    rng = np.random.default_rng(1)
    W = wl.spheres_workload("t", 32, 100.0, 0.01, [[0.5] * 3], [0.2], None, 0, rng=rng)
    W2 = wl.spheres_workload("t", 32, 100.0, 0.01, [[0.5] * 3], [0.2], None, 0,
                             rng=np.random.default_rng(1))
    for a, b in ((W.X, W2.X), (W.U_gamma, W2.U_gamma), (W.f_body, W2.f_body)):
        assert np.array_equal(a, b)
    W3 = wl.spheres_workload("t", 32, 100.0, 0.01, [[0.5] * 3], [0.2], None, 0,
                             rng=np.random.default_rng(2))
    assert not np.array_equal(W.U_gamma, W3.U_gamma)


def test_fibonacci_markers_lie_on_the_sphere():
    c = np.array([0.4, 0.55, 0.6])
    X = wl.fibonacci_sphere(2000, 0.17, c)
    d = X - c[:, None]
    np.testing.assert_allclose(np.linalg.norm(d, axis=0), 0.17, rtol=1e-14)
    # equal-area bands in z: z levels evenly spaced, centroid at the centre
    np.testing.assert_allclose(np.diff(d[2]), -2 * 0.17 / 2000, rtol=1e-9)
    assert np.linalg.norm(d.mean(axis=1)) < 1e-3 * 0.17
    # no two markers coincide; nearest-neighbour spacing near sqrt(area / N)
    sub = d[:, ::20]
    dist = np.linalg.norm(sub[:, :, None] - d[:, None, :], axis=0)
    dist[dist == 0] = np.inf
    nn = dist.min(axis=1)
    spacing = np.sqrt(4 * np.pi * 0.17 ** 2 / 2000)
    assert nn.min() > 0.5 * spacing and nn.max() < 1.5 * spacing


def test_rigid_velocities_preserve_distances():
    # a rigid motion keeps every pairwise distance on a body fixed:
    # (U_k - U_l) . (X_k - X_l) = 0 for markers k, l of the same body
    rng = np.random.default_rng(5)
    centers = np.array([[0.3, 0.3, 0.3], [0.7, 0.6, 0.65]])
    X = np.concatenate([wl.fibonacci_sphere(300, 0.1, centers[0]),
                        wl.fibonacci_sphere(200, 0.08, centers[1])], axis=1)
    body = np.concatenate([np.zeros(300, np.int32), np.ones(200, np.int32)])
    U = wl.rigid_velocities(X, body, centers, rng)
    assert U.shape == X.shape
    for b in (0, 1):
        Xb, Ub = X[:, body == b], U[:, body == b]
        dX = Xb[:, :, None] - Xb[:, None, :]
        dU = Ub[:, :, None] - Ub[:, None, :]
        assert np.abs((dX * dU).sum(axis=0)).max() < 1e-14
    # the two bodies move differently
    assert not np.allclose(U[:, 0] - U[:, 1], 0.0)


def test_sine_body_force_walls_and_modes():
    n = 12
    h = 1.0 / n
    f = wl.sine_body_force(n, n, n, h, np.random.default_rng(7))
    shapes = ((n, n, n + 1), (n, n + 1, n), (n + 1, n, n))
    off = 0
    for d, sh in enumerate(shapes):
        fd = f[off:off + int(np.prod(sh))].reshape(sh)
        off += fd.size
        ax = 2 - d
        assert np.all(np.take(fd, 0, axis=ax) == 0.0)
        assert np.all(np.take(fd, sh[ax] - 1, axis=ax) == 0.0)
        assert np.abs(fd).max() <= 8.0
        assert np.abs(fd).max() > 0.5
    assert off == f.size


@pytest.mark.parametrize("total", [None, 60000])
def test_marker_counts(total):
    rng = np.random.default_rng(3)
    n = 64
    centers, radii = wl.place_spheres(8, 0.05, 0.1, 1.0 / 256, rng)
    W = wl.spheres_workload("t", n, 200.0, 1e-3, centers, radii, total, 3, rng=rng)
    counts = np.array(W.info["counts"])
    assert counts.sum() == W.n_markers == W.body_id.size
    if total is None:
        expect = [int(round(4 * np.pi * r * r * n * n)) for r in radii]
        assert list(counts) == expect
        assert abs(W.info["spacing_ratio"] - 1.0) < 0.01
    else:
        assert W.n_markers == total
        share = 4 * np.pi * radii ** 2 / (4 * np.pi * radii ** 2).sum()
        assert np.all(np.abs(counts[:-1] - share[:-1] * total) < 1.0)
    for b in range(8):
        Xb = W.X[:, W.body_id == b]
        np.testing.assert_allclose(np.linalg.norm(Xb - centers[b][:, None], axis=0), radii[b],
                                   rtol=1e-13)
