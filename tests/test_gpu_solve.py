"""Parity of the GPU Schur solve (FGMRES + V-cycle, FP64 and mixed FP32
preconditioner) with the oracle's solve, plus the solver's edge cases."""
import numpy as np
import pytest

import gpu_cases as gc
from gpu_cases import dev, host, rel

pytestmark = pytest.mark.gpu

PARITY = 1e-10      # FP64 path vs FP64 oracle, both solved to 1e-13


@pytest.fixture(scope="module", params=[gc.sphere16, gc.ragged_multi,
                                        lambda: gc.config_case(1)],
                ids=["sphere16", "ragged48x40x32", "config1_32"])
def setup(request, cuda_device):
    import torch
    from oracle import schur
    from paper_2501_15314_gb300.api import IBMSolver
    case = request.param()
    g = case.grid()
    s = IBMSolver(case.nx, case.ny, case.nz, case.h, Re=case.Re, dt=case.dt)
    s.set_markers(dev(case.X))
    sysm = schur.SchurSystem(g, case.X)
    # a right-hand side of the form the step builds: RHS_p + 2 B^T RHS_F
    from oracle import mac
    u = case.rng.standard_normal(g.n_faces) * g.interior_face_mask_packed()
    b = sysm.rhs_scalar(mac.apply_GT(g, u), case.rng.standard_normal(sysm.k))
    ref, it_ref, rel_ref, _ = schur.solve_schur(sysm, b, rtol=1e-13)
    yield case, g, s, sysm, b, ref
    s.close()
    torch.cuda.synchronize()


MODES = [(0, 0), (1, 1), (1, 0), (1, 2)]
MODE_IDS = ["fp64_vcycle", "fp32_vcycle_ds_arnoldi", "fp32_vcycle_fp64_arnoldi",
            "fp32_vcycle_fp32_arnoldi"]


@pytest.mark.parametrize("prec,arnoldi", MODES, ids=MODE_IDS)
def test_solve_parity(setup, prec, arnoldi):
    case, g, s, sysm, b, ref = setup
    p, st = s.solve_schur(dev(b), rtol=1e-13, precond_prec=prec, arnoldi=arnoldi, maxit=300)
    assert st["relres_true"] <= 1e-13
    ph = host(p)
    assert abs(ph.mean()) < 1e-12 * np.abs(ph).max()
    assert rel(ph, ref) < PARITY, rel(ph, ref)
    # independent residual check with the oracle operator
    assert rel(sysm.apply_S_tilde(ph), b) < 2e-13


@pytest.mark.parametrize("arnoldi", [1, 2], ids=["ds_arnoldi", "fp32_arnoldi"])
def test_cycle_graphs_match_the_host_driven_loop(setup, arnoldi):
    """With cycle_graphs = 1 the FP32 and double-single Arnoldi cycles run as
    CUDA graph replays (Givens rotations and the stopping test on the device,
    the next iteration in a conditional node); by default, and while
    profiling, the host-driven loop runs.  Both take the same iterations to
    the same solution, also with a short restart (several cycles) and with a
    maxit that ends a cycle early."""
    case, g, s, sysm, b, ref = setup
    for kw in (dict(rtol=1e-13, maxit=300), dict(rtol=1e-13, restart=5, maxit=300),
               dict(rtol=1e-10, restart=7, maxit=9)):
        p_g, st_g = s.solve_schur(dev(b), precond_prec=1, arnoldi=arnoldi, cycle_graphs=1,
                                  raise_on_error=False, **kw)
        p_h, st_h = s.solve_schur(dev(b), precond_prec=1, arnoldi=arnoldi,
                                  raise_on_error=False, **kw)
        s.profile_enable(True)
        try:
            _, st_p = s.solve_schur(dev(b), precond_prec=1, arnoldi=arnoldi, cycle_graphs=1,
                                    raise_on_error=False, **kw)
        finally:
            s.profile_enable(False)
        assert st_g["graph_cycles"] >= 1 and st_g["graph_cycles"] == st_g["restarts"], st_g
        assert st_h["graph_cycles"] == 0 and st_p["graph_cycles"] == 0
        assert st_g["iters"] == st_h["iters"] and st_g["restarts"] == st_h["restarts"], (st_g, st_h)
        assert rel(host(p_g), host(p_h)) < 1e-12, kw
        n = min(st_g["iters"], len(st_g["relres_hist"]))
        # the estimates agree to the rounding of the rotations (the device's
        # hypot against the host's), far inside the stopping tests
        np.testing.assert_allclose(st_g["relres_hist"][:n], st_h["relres_hist"][:n], rtol=1e-6,
                                   atol=1e-13)
        if kw.get("maxit") == 9:
            assert st_g["iters"] <= 9


@pytest.mark.parametrize("prec,arnoldi", MODES, ids=MODE_IDS)
def test_solve_throughput_setting(setup, prec, arnoldi):
    case, g, s, sysm, b, ref = setup
    p, st = s.solve_schur(dev(b), rtol=1e-8, precond_prec=prec, arnoldi=arnoldi)
    ph = host(p)
    assert rel(sysm.apply_S_tilde(ph), b) <= 1e-8 * 1.001
    assert rel(ph, ref) < 1e-6
    assert st["iters"] <= 20, st["iters"]


def test_deterministic_and_restart_and_reorth(setup):
    import torch
    case, g, s, sysm, b, ref = setup
    bd = dev(b)
    p1, st1 = s.solve_schur(bd, rtol=1e-10)
    p2, st2 = s.solve_schur(bd, rtol=1e-10)
    assert torch.equal(p1, p2) and st1["iters"] == st2["iters"]
    p3, st3 = s.solve_schur(bd, rtol=1e-13, restart=4, maxit=400, precond_prec=0)
    assert st3["restarts"] > 1 and rel(host(p3), ref) < PARITY
    p4, st4 = s.solve_schur(bd, rtol=1e-13, reorth=1, precond_prec=0)
    assert rel(host(p4), ref) < PARITY


def test_initial_guess(setup):
    case, g, s, sysm, b, ref = setup
    x0 = dev(ref + 1e-3 * case.rng.standard_normal(g.m))
    p, st = s.solve_schur(dev(b), x0=x0, rtol=1e-13, precond_prec=0)
    assert rel(host(p), ref) < PARITY


def test_edge_cases(cuda_device):
    import torch
    from oracle import mac
    from paper_2501_15314_gb300 import _lib
    from paper_2501_15314_gb300.api import IBMSolver
    s = IBMSolver(16)
    g = mac.Grid(16)
    # no markers: S~ = L and the solution is L^+ b
    b = mac.remove_mean(np.random.default_rng(0).standard_normal(g.m))
    p, st = s.solve_schur(dev(b), rtol=1e-13, precond_prec=0)
    assert rel(host(p), mac.laplacian_pinv(g, b)) < PARITY
    # zero right-hand side gives zero
    p, st = s.solve_schur(dev(np.zeros(g.m)))
    assert st["iters"] == 0 and torch.count_nonzero(p) == 0
    # NaN right-hand side is reported, not propagated silently
    bad = b.copy()
    bad[5] = np.nan
    with pytest.raises(_lib.IBMError) as e:
        s.solve_schur(dev(bad))
    assert e.value.status == _lib.IBM_ERR_NAN
    # maxit reached
    p, st = s.solve_schur(dev(b), maxit=1, rtol=1e-14, raise_on_error=False)
    assert st["status"] == _lib.IBM_ERR_NOT_CONVERGED and st["iters"] == 1
    # invalid options
    with pytest.raises(_lib.IBMError):
        s.solve_schur(dev(b), restart=0)
    # markers whose delta support touches a wall face
    X = np.array([[0.5], [0.5], [1.2 / 16]])
    with pytest.raises(_lib.IBMError) as e:
        s.set_markers(dev(X))
    assert e.value.status == _lib.IBM_ERR_MARKER_DOMAIN
    X = np.array([[0.5], [np.nan], [0.5]])
    with pytest.raises(_lib.IBMError):
        s.set_markers(dev(X))
    s.close()
    # a grid that does not coarsen to <= 512 cells is rejected at creation
    with pytest.raises(_lib.IBMError):
        IBMSolver(50, 50, 75)


def test_fp32_arnoldi_request_with_nx_not_multiple_of_4(cuda_device):
    """FP32 Arnoldi requested on a 10 x 9 x 5 grid: nx is not a multiple of 4,
    so the float4 V-cycle and the single-precision Arnoldi forms do not apply
    and the solver runs the FP64 Arnoldi process with the scalar FP32 V-cycle
    (as the header states); parity with the oracle's solve at rtol 1e-13."""
    from oracle import mac, schur
    from paper_2501_15314_gb300 import workloads as wl
    from paper_2501_15314_gb300.api import IBMSolver
    nx, ny, nz, h = 10, 9, 5, 0.1
    g = mac.Grid(nx, ny, nz, h)
    X = wl.fibonacci_sphere(10, 0.06, [0.5, 0.45, 0.25])
    rng = np.random.default_rng(3)
    sysm = schur.SchurSystem(g, X)
    u = rng.standard_normal(g.n_faces) * g.interior_face_mask_packed()
    b = sysm.rhs_scalar(mac.apply_GT(g, u), rng.standard_normal(sysm.k))
    ref, _, _, _ = schur.solve_schur(sysm, b, rtol=1e-13)
    s = IBMSolver(nx, ny, nz, h)
    s.set_markers(dev(X))
    p, st = s.solve_schur(dev(b), rtol=1e-13, precond_prec=1, arnoldi=2, maxit=300)
    assert rel(host(p), ref) < PARITY, (rel(host(p), ref), st)
    s.close()
