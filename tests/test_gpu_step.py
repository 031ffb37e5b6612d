"""Parity of one full GPU time step (predictor, RHS, Schur solve, force
recovery, update, diagnostics) with the oracle's step."""
import numpy as np
import pytest

import gpu_cases as gc
from gpu_cases import dev, host, rel

pytestmark = pytest.mark.gpu


def _run(case, u_n=None, u_nm1=None, p_n=None, F_n=None, prec=0, rtol=1e-13):
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
                     precond_prec=prec, rtol=rtol, helm_rtol=1e-14, helm_maxit=12)
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
