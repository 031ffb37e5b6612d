"""The FP32 V-cycle against the FP64 V-cycle of the same algorithm.

The FP32 cycle runs the four-cell (float4) level kernels -- the first two
Chebyshev steps from zero fused, the further sweeps, the residual
restriction, the prolongation -- and the one-block coarse chain below 4096
cells; the FP64 cycle runs the one-cell kernels of the same operators.  The
two must agree to FP32 rounding on every grid shape: x-extents ragged
against the 128-cell rows of a warp, two x-tiles of which the second is
partial, ragged y and z tiles, different numbers of levels above the chain,
and one, two or three post-smoothing sweeps (the buffer alternation of the
last sweeps)."""
import numpy as np
import pytest

from gpu_cases import dev, host, rel

pytestmark = pytest.mark.gpu

GRIDS = [(48, 40, 32), (64, 64, 64), (160, 24, 40), (256, 16, 24), (128, 96, 48)]


@pytest.mark.parametrize("grid", GRIDS, ids=lambda g: "x".join(map(str, g)))
@pytest.mark.parametrize("post", [1, 2, 3])
def test_fp32_vcycle_matches_fp64_vcycle(cuda_device, grid, post):
    import torch
    from oracle import mac
    from paper_2501_15314_gb300.api import IBMSolver
    nx, ny, nz = grid
    s = IBMSolver(nx, ny, nz, 1.0 / nx, Re=100.0, dt=0.01)
    rng = np.random.default_rng(nx + 7 * ny + 31 * nz + post)
    b = mac.remove_mean(rng.standard_normal(nx * ny * nz))
    bd = dev(b)
    z32 = host(s.precond(bd, prec=1, pre=2, post=post))
    z64 = host(s.precond(bd, prec=0, pre=2, post=post))
    err = rel(z32, z64)
    print(f"{grid} post {post}: |z32 - z64| / |z64| = {err:.2e}")
    assert np.all(np.isfinite(z32))
    assert err < 2e-5, err
    s.close()
    torch.cuda.synchronize()


def test_fp32_vcycle_stationary_iteration_converges(cuda_device):
    # x += M (b - L x) with the FP32 cycle on a grid of two x-tiles
    import torch
    from oracle import mac
    from paper_2501_15314_gb300.api import IBMSolver
    nx, ny, nz = 160, 24, 40
    g = mac.Grid(nx, ny, nz, 1.0 / nx)
    s = IBMSolver(nx, ny, nz, 1.0 / nx, Re=100.0, dt=0.01)
    b = mac.remove_mean(np.random.default_rng(3).standard_normal(g.m))
    ref = mac.laplacian_pinv(g, b)
    bd, x = dev(b), dev(np.zeros(g.m))
    errs = []
    for _ in range(30):
        x = x + s.precond(bd - s.apply_laplacian(x), prec=1)
        xh = host(x)
        errs.append(rel(xh - xh.mean(), ref))
    assert errs[-1] < 1e-5 and errs[3] < 0.05 * errs[0], errs
    s.close()
    torch.cuda.synchronize()


def test_vcycle_on_vectors_off_the_16_byte_boundary(cuda_device):
    # r and z that start 8 bytes past an allocation's 16-byte boundary give
    # the same V-cycle as aligned ones (the FP32 cycle's four-cell kernels
    # move FP64 pairs; such vectors go through the level's own buffers)
    import torch
    from paper_2501_15314_gb300.api import IBMSolver
    nx, ny, nz = 48, 40, 32
    m = nx * ny * nz
    s = IBMSolver(nx, ny, nz, 1.0 / nx, Re=100.0, dt=0.01)
    b = np.random.default_rng(5).standard_normal(m)
    b -= b.mean()
    ra = dev(b)
    rb = torch.zeros(m + 1, dtype=torch.float64, device="cuda")
    rb[1:] = ra
    zb = torch.zeros(m + 1, dtype=torch.float64, device="cuda")
    assert rb[1:].data_ptr() % 16 == 8 and zb[1:].data_ptr() % 16 == 8
    za = host(s.precond(ra, prec=1))
    s.precond(rb[1:], prec=1, out=zb[1:])
    np.testing.assert_array_equal(host(zb[1:]), za)
    s.close()
    torch.cuda.synchronize()
