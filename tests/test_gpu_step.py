"""Parity of one full GPU time step (predictor, RHS, Schur solve, force
recovery, update, diagnostics) with the oracle's step."""
import numpy as np
import pytest

import gpu_cases as gc
from gpu_cases import dev, host, rel

pytestmark = pytest.mark.gpu


def _run(case, u_n=None, u_nm1=None, p_n=None, F_n=None, prec=0, rtol=1e-13, helm_rtol=1e-14):
    from oracle import step
    from paper_2501_15314_gb300.api import IBMSolver
    g = case.grid()
    U = case.U_gamma
    f = case.f_body
    ref = step.step(g, case.Re, case.dt, case.X, U, f, u_n=u_n, u_nm1=u_nm1, p_n=p_n, F_n=F_n,
                    rtol=1e-13)
    s = IBMSolver(case.nx, case.ny, case.nz, case.h, Re=case.Re, dt=case.dt)
    s.set_markers(dev(case.X))
    z = lambda n: np.zeros(n)
    out, st = s.step(dev(u_n if u_n is not None else z(g.n_faces)),
                     dev(u_nm1 if u_nm1 is not None else (u_n if u_n is not None else z(g.n_faces))),
                     dev(p_n if p_n is not None else z(g.m)),
                     dev(F_n if F_n is not None else z(3 * case.N)), dev(U), dev(f),
                     precond_prec=prec, rtol=rtol, helm_rtol=helm_rtol, helm_maxit=12)
    s.close()
    return ref, {k: host(v) for k, v in out.items()}, st


def _with_inputs(case):
    g = case.grid()
    rng = np.random.default_rng(7)
    case.U_gamma = rng.uniform(-1, 1, 3 * case.N)
    case.f_body = rng.standard_normal(g.n_faces) * g.interior_face_mask_packed()
    return case


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_step_from_rest_config1(cuda_device, prec):
    case = gc.config_case(1)
    ref, out, st = _run(case, prec=prec)
    for k in ("u", "p", "F"):
        assert rel(out[k], ref[k]) < 1e-10, (k, rel(out[k], ref[k]))
    assert abs(st["div_l2"] - ref["div_l2"]) <= 1e-8 * ref["div_l2"] + 1e-12
    assert abs(st["slip_l2"] - ref["slip_l2"]) <= 1e-8 * ref["slip_l2"] + 1e-12


def test_step_with_history_ragged(cuda_device):
    # nonzero u^n, u^{n-1}, p^n, F^n exercise every term of Eq. (ustar),
    # including the convective term
    case = _with_inputs(gc.ragged_multi())
    g = case.grid()
    rng = np.random.default_rng(8)
    mask = g.interior_face_mask_packed()
    u_n = 0.3 * rng.standard_normal(g.n_faces) * mask
    u_nm1 = 0.3 * rng.standard_normal(g.n_faces) * mask
    p_n = rng.standard_normal(g.m)
    F_n = rng.standard_normal(3 * case.N)
    ref, out, st = _run(case, u_n, u_nm1, p_n, F_n)
    for k in ("u", "p", "F"):
        assert rel(out[k], ref[k]) < 1e-10, (k, rel(out[k], ref[k]))


def test_solver_on_its_own_stream_orders_against_caller(cuda_device):
    """A solver created on a stream other than the caller's: the inputs are
    written on the caller's stream behind a long busy kernel, the step runs
    on the solver's stream and the results are read back on the caller's
    stream.  The step must see the inputs and the caller the results: the
    same answer as a solver on the caller's stream."""
    import torch
    from paper_2501_15314_gb300.api import IBMSolver
    case = _with_inputs(gc.sphere16())
    g = case.grid()
    src = {k: dev(v) for k, v in dict(X=case.X, U=case.U_gamma, f=case.f_body).items()}
    outs = []
    for side in (False, True):
        s = IBMSolver(case.nx, case.ny, case.nz, case.h, Re=case.Re, dt=case.dt,
                      stream=torch.cuda.Stream() if side else None)
        torch.cuda.synchronize()
        inp = {k: torch.empty_like(v) for k, v in src.items()}
        torch.cuda._sleep(20_000_000)          # keeps the caller's stream busy for ~10 ms
        for k in inp:
            inp[k].copy_(src[k])
        s.set_markers(inp["X"])
        zf = torch.zeros(g.n_faces, dtype=torch.float64, device="cuda")
        out, st = s.step(zf, zf, torch.zeros(g.m, dtype=torch.float64, device="cuda"),
                         torch.zeros(3 * case.N, dtype=torch.float64, device="cuda"), inp["U"],
                         inp["f"], precond_prec=0, rtol=1e-12)
        outs.append({k: host(v) for k, v in out.items()})
        s.close()
    for k in ("u", "p", "F"):
        assert rel(outs[1][k], outs[0][k]) < 1e-13, (k, rel(outs[1][k], outs[0][k]))
        assert np.linalg.norm(outs[0][k]) > 0


def test_step_with_history_wide_grid(cuda_device):
    """A grid wider than one 128-face block of the predictor kernels along
    x (the second block ragged), with ragged y and z tiles: neighbours across
    every block edge.  FP64 form against the oracle, every term of
    Eq. (ustar) active."""
    case = _with_inputs(gc.wide_grid())
    g = case.grid()
    rng = np.random.default_rng(9)
    mask = g.interior_face_mask_packed()
    u_n = 0.3 * rng.standard_normal(g.n_faces) * mask
    u_nm1 = 0.3 * rng.standard_normal(g.n_faces) * mask
    p_n = rng.standard_normal(g.m)
    F_n = rng.standard_normal(3 * case.N)
    ref, out, st = _run(case, u_n, u_nm1, p_n, F_n)
    for k in ("u", "p", "F"):
        assert rel(out[k], ref[k]) < 1e-10, (k, rel(out[k], ref[k]))
    assert st["helm_iters"] >= 2, st


@pytest.mark.parametrize("helm_rtol,n_corr,tol", [(1e-4, 1, 5e-3), (1e-10, 2, 1e-8),
                                                   (1e-14, 3, 1e-10)])
def test_predictor_with_one_two_and_three_corrections(cuda_device, helm_rtol, n_corr, tol):
    """The predictor's first correction stays in FP32 until the second's last
    step writes u from both; alone, it is written by a pass of its own; a
    third one adds into u.  Each count gives the oracle's step to the
    accuracy its tolerance allows (every term of Eq. (ustar) active)."""
    case = _with_inputs(gc.ragged_multi())
    g = case.grid()
    rng = np.random.default_rng(11)
    mask = g.interior_face_mask_packed()
    u_n = 0.3 * rng.standard_normal(g.n_faces) * mask
    u_nm1 = 0.3 * rng.standard_normal(g.n_faces) * mask
    p_n = rng.standard_normal(g.m)
    F_n = rng.standard_normal(3 * case.N)
    ref, out, st = _run(case, u_n, u_nm1, p_n, F_n, helm_rtol=helm_rtol)
    assert st["helm_iters"] == n_corr if n_corr < 3 else st["helm_iters"] >= 3, st
    assert st["helm_relres"] <= helm_rtol, st
    for k in ("u", "p", "F"):
        assert np.all(np.isfinite(out[k]))
        assert rel(out[k], ref[k]) < tol, (k, rel(out[k], ref[k]))


def test_step_unchanged_by_concurrent_bulk_copies(cuda_device):
    """The scalars the host reads during a step (residual norms, Hessenberg
    entries, counts) come through mapped pinned memory, not copy-engine
    transfers: a step run while half a gigabyte moves between the host and
    the device on two other streams gives bit-for-bit the same result as a
    step run alone."""
    import torch
    from paper_2501_15314_gb300.api import IBMSolver
    case = _with_inputs(gc.ragged_multi())
    g = case.grid()
    s = IBMSolver(case.nx, case.ny, case.nz, case.h, Re=case.Re, dt=case.dt)
    args = (torch.zeros(g.n_faces, dtype=torch.float64, device="cuda"),) * 2 + (
        torch.zeros(g.m, dtype=torch.float64, device="cuda"),
        torch.zeros(3 * case.N, dtype=torch.float64, device="cuda"), dev(case.U_gamma),
        dev(case.f_body))
    X = dev(case.X)

    def run():
        s.set_markers(X)
        out, st = s.step(*args, precond_prec=1, rtol=1e-10)
        return {k: v.clone() for k, v in out.items()}, st["iters"]

    ref, it_ref = run()
    n = 64 * 1024 * 1024                       # 512 MB each way
    h_src = torch.ones(n, dtype=torch.float64).pin_memory()
    h_dst = torch.empty(n, dtype=torch.float64).pin_memory()
    d_buf = torch.empty(n, dtype=torch.float64, device="cuda")
    d_src = torch.ones(n, dtype=torch.float64, device="cuda")
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    for _ in range(3):
        with torch.cuda.stream(s_in):
            d_buf.copy_(h_src, non_blocking=True)
        with torch.cuda.stream(s_out):
            h_dst.copy_(d_src, non_blocking=True)
        out, it = run()
        assert it == it_ref
        for k in ref:
            assert torch.equal(out[k], ref[k]), k
    torch.cuda.synchronize()
    assert float(h_dst[-1]) == 1.0 and float(d_buf[0]) == 1.0
    s.close()


def _scaled_step(case, s_f, s_U):
    from paper_2501_15314_gb300.api import IBMSolver
    g = case.grid()
    s = IBMSolver(case.nx, case.ny, case.nz, case.h, Re=case.Re, dt=case.dt)
    s.set_markers(dev(case.X))
    z = lambda n: dev(np.zeros(n))  # noqa: E731
    out, _ = s.step(z(g.n_faces), z(g.n_faces), z(g.m), z(3 * case.N), dev(s_U * case.U_gamma),
                    dev(s_f * case.f_body), precond_prec=0, arnoldi=0, rtol=1e-13,
                    helm_rtol=1e-14, helm_maxit=12)
    s.close()
    return {k: host(v) for k, v in out.items()}


def test_predictor_input_range(cuda_device):
    # The step from rest is linear in (U^Gamma, f).  The predictor reads f as
    # FP32 pairs: above 2^-80 in magnitude the scaled inputs give the scaled
    # results (here 2^-40: every entry that matters stays above the floor);
    # every entry below 2^-80 is read as 0 (here 2^-100: the result is that of
    # the same step without body force).
    case = _with_inputs(gc.sphere16())
    base = _scaled_step(case, 1.0, 1.0)
    s = 2.0 ** -40
    small = _scaled_step(case, s, s)
    for k in ("u", "p", "F"):
        assert rel(small[k], s * base[k]) < 1e-10, (k, rel(small[k], s * base[k]))
    t = 2.0 ** -100
    assert np.abs(t * case.f_body).max() < 2.0 ** -80
    tiny = _scaled_step(case, t, 1.0)
    no_force = _scaled_step(case, 0.0, 1.0)
    for k in ("u", "p", "F"):
        np.testing.assert_array_equal(tiny[k], no_force[k])
