"""Parity of the CUDA operators (through the C ABI) with the FP64 oracle:
Laplacian, gradient and its transpose, interpolation R^T, spread R, the Schur
operator S~ = L + 2 B^T B, force recovery, and the V-cycle as an L^{-1}
approximation."""
import numpy as np
import pytest

import gpu_cases as gc
from gpu_cases import dev, host, rel

pytestmark = pytest.mark.gpu

CASES = [gc.sphere16, gc.ragged_multi]


@pytest.fixture(scope="module", params=CASES, ids=lambda f: f.__name__)
def setup(request, cuda_device):
    import torch
    from oracle import mac, schur
    from paper_2501_15314_gb300.api import IBMSolver
    case = request.param()
    g = case.grid()
    s = IBMSolver(case.nx, case.ny, case.nz, case.h, Re=case.Re, dt=case.dt)
    s.set_markers(dev(case.X))
    sysm = schur.SchurSystem(g, case.X)
    yield case, g, s, sysm
    s.close()
    torch.cuda.synchronize()


def test_laplacian(setup):
    from oracle import mac
    case, g, s, sysm = setup
    v = case.rng.standard_normal(g.m)
    out = host(s.apply_laplacian(dev(v)))
    assert rel(out, mac.apply_L(g, v)) < 1e-13


def test_gradient_and_transpose(setup):
    from oracle import mac
    case, g, s, sysm = setup
    p = case.rng.standard_normal(g.m)
    u = case.rng.standard_normal(g.n_faces)
    assert rel(host(s.gradient(dev(p))), mac.apply_G(g, p)) < 1e-14
    assert rel(host(s.gradient_t(dev(u))), mac.apply_GT(g, u)) < 1e-14


def test_interp_and_spread(setup):
    case, g, s, sysm = setup
    u = case.rng.standard_normal(g.n_faces)
    F = case.rng.standard_normal(3 * case.N)
    assert rel(host(s.interp(dev(u))), sysm.R.T @ u) < 1e-13
    assert rel(host(s.spread(dev(F))), sysm.R @ F) < 1e-13


def test_schur_apply(setup):
    case, g, s, sysm = setup
    v = case.rng.standard_normal(g.m)
    out = host(s.apply_schur(dev(v)))
    assert rel(out, sysm.apply_S_tilde(v)) < 1e-13
    # the marker term alone, which is ~1e-2 of the total, is also exact
    lap = host(s.apply_laplacian(dev(v)))
    mk_ref = sysm.apply_S_tilde(v) - sysm.apply_S_tilde(np.zeros_like(v))
    from oracle import mac
    assert rel(out - lap, 2.0 * sysm.apply_BT(sysm.apply_B(v))) < 1e-11


def test_force_correction(setup):
    case, g, s, sysm = setup
    p = case.rng.standard_normal(g.m)
    rF = case.rng.standard_normal(3 * case.N)
    out = host(s.force_correction(dev(p), dev(rF)))
    assert rel(out, sysm.force_scalar(p, rF)) < 1e-13


def test_schur_apply_deterministic(setup):
    import torch
    case, g, s, sysm = setup
    v = dev(case.rng.standard_normal(g.m))
    a = s.apply_schur(v)
    b = s.apply_schur(v)
    assert torch.equal(a, b)


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_vcycle_converges_to_pinv(setup, prec):
    # stationary iteration x += M (b - L x) with the V-cycle M converges to L^+ b
    from oracle import mac
    case, g, s, sysm = setup
    b = mac.remove_mean(case.rng.standard_normal(g.m))
    ref = mac.laplacian_pinv(g, b)
    bd = dev(b)
    x = dev(np.zeros(g.m))
    errs = []
    for it in range(30):
        r = bd - s.apply_laplacian(x)
        x = x + s.precond(r, prec=prec)
        xh = host(x)
        errs.append(rel(xh - xh.mean(), ref))
    if prec == 0:
        assert errs[-1] < 1e-11, errs
    else:
        assert errs[-1] < 1e-5, errs
    assert errs[3] < 0.05 * errs[0], errs     # contraction of a few V-cycles


def test_body_forces(setup):
    import torch
    from oracle import step
    case, g, s, sysm = setup
    F = case.rng.standard_normal(3 * case.N)
    centers = case.centers if case.centers is not None else np.array([[0.5, 0.5, 0.5]])
    nb = centers.shape[0]
    out = s.body_forces(dev(F), dev(case.X.ravel()), dev(case.body_id.astype(np.int32)), centers)
    ref = step.body_force_torque(g, case.X, F, case.body_id, centers)
    np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-15)
