"""The exact (Eqs. (SchurPrimal)-(SchurPrimalF)) and sign-consistent forms of
the correction system on the GPU: C^{-1} by conjugate gradients on R^T R, the
Schur products, solves and whole steps against the oracle, and the bound of
the spectral theorem (Sec. 5) at 128^3."""
import numpy as np
import pytest

import gpu_cases as gc
from gpu_cases import dev, host, rel

pytestmark = pytest.mark.gpu

MODES = {"exact": 1, "consistent": 2}


def _solver(case):
    from paper_2501_15314_gb300.api import IBMSolver
    s = IBMSolver(case.nx, case.ny, case.nz, case.h, Re=case.Re, dt=case.dt)
    s.set_markers(dev(case.X))
    return s


@pytest.mark.parametrize("make", [gc.sphere16, gc.ragged_multi], ids=["sphere16", "ragged"])
def test_c_inverse_matches_oracle(cuda_device, make):
    from oracle import schur
    case = make()
    sysm = schur.SchurSystem(case.grid(), case.X)
    t = np.random.default_rng(1).standard_normal(3 * case.N)
    s = _solver(case)
    x, it = s.apply_c_inverse(dev(t), c_rtol=1e-14)
    ref = sysm.C_solve(t)
    assert rel(host(x), ref) < 1e-11, rel(host(x), ref)
    assert 0 < it < 500
    s.close()


@pytest.mark.parametrize("mode", list(MODES))
def test_schur_products_match_oracle(cuda_device, mode):
    from oracle import mac, schur
    case = gc.ragged_multi()
    sysm = schur.SchurSystem(case.grid(), case.X)
    v = mac.remove_mean(np.random.default_rng(2).standard_normal(case.grid().m))
    ref = sysm.apply_S_exact(v) if mode == "exact" else sysm.apply_S_consistent(v)
    s = _solver(case)
    out = s.apply_schur(dev(v), c_mode=MODES[mode], c_rtol=1e-14)
    assert rel(host(out), ref) < 1e-12, rel(host(out), ref)
    assert s.last_c_iters > 0
    s.close()


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32_ds"])
@pytest.mark.parametrize("mode", list(MODES))
def test_solve_matches_oracle(cuda_device, mode, prec):
    from oracle import mac, schur
    case = gc.sphere16()
    g = case.grid()
    sysm = schur.SchurSystem(g, case.X)
    rng = np.random.default_rng(3)
    b = sysm.rhs_exact(mac.apply_GT(g, rng.standard_normal(g.n_faces)),
                       rng.standard_normal(3 * case.N))
    ref, it_ref, _, _ = schur.solve_schur(sysm, b, mode=mode, rtol=1e-13)
    s = _solver(case)
    x, st = s.solve_schur(dev(b), precond_prec=prec, rtol=1e-13, maxit=400, restart=60,
                          c_mode=MODES[mode], c_rtol=1e-14)
    assert st["relres_true"] <= 1e-13
    assert rel(host(x), ref) < 1e-10, rel(host(x), ref)
    assert st["c_iters"] > 0
    print(f"{mode} prec {prec}: GPU iters {st['iters']} (oracle with exact L^+: {it_ref}), "
          f"inner CG iterations {st['c_iters']}")
    s.close()


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("make", [gc.sphere16, gc.ragged_multi], ids=["sphere16", "ragged"])
def test_step_matches_oracle(cuda_device, make, mode):
    from oracle import step
    case = make()
    g = case.grid()
    rng = np.random.default_rng(4)
    U = rng.uniform(-1, 1, 3 * case.N)
    f = rng.standard_normal(g.n_faces) * g.interior_face_mask_packed()
    ref = step.step(g, case.Re, case.dt, case.X, U, f, mode=mode, rtol=1e-13)
    s = _solver(case)
    z = lambda n: dev(np.zeros(n))  # noqa: E731
    out, st = s.step(z(g.n_faces), z(g.n_faces), z(g.m), z(3 * case.N), dev(U), dev(f),
                     precond_prec=0, rtol=1e-13, maxit=400, restart=60, helm_rtol=1e-14,
                     helm_maxit=12, c_mode=MODES[mode], c_rtol=1e-14)
    for k in ("u", "p", "F"):
        assert rel(host(out[k]), ref[k]) < 1e-10, (k, rel(host(out[k]), ref[k]))
    if mode == "consistent":
        # the sign-consistent update is divergence-free and no-slip exactly
        div_ustar = np.linalg.norm(ref["rhs_p"]) * (2.0 * case.dt / 3.0)   # ||G^T u*||
        assert st["div_l2"] < 1e-9 * div_ustar, (st["div_l2"], div_ustar)
        assert st["slip_l2"] < 1e-9 * np.linalg.norm(U)
    s.close()


def test_theorem_bound_rayleigh_quotients_128(cuda_device):
    """Sec. 5: spec(L^+ S_p) in [1, 2].  At 128^3 with one sphere at
    Lagrangian spacing h, the generalised Rayleigh quotient
    <v, S_p v> / <v, L v> of the GPU operators stays in [1, 2] for random
    vectors and for vectors concentrated on the marker shell, where the
    force term is largest; the scalar form's quotient is printed beside it."""
    import torch
    from paper_2501_15314_gb300 import workloads as wl
    from paper_2501_15314_gb300.api import IBMSolver
    W = wl.config(2)          # 128^3, r = 0.15, markers at spacing h
    s = IBMSolver(W.n, Re=W.Re, dt=W.dt)
    s.set_markers(dev(W.X))
    rng = np.random.default_rng(5)
    m = s.m
    # marker-concentrated vectors: B^T t for random t (supported on the shell)
    vs = [rng.standard_normal(m) for _ in range(2)]
    bt = []
    for _ in range(3):
        t = dev(rng.standard_normal(3 * W.n_markers))
        bt.append(host(s.gradient_t(s.spread(t))))
    vs += bt
    qs, qs_scalar = [], []
    for v in vs:
        v = v - v.mean()
        vd = dev(v)
        Lv = host(s.apply_laplacian(vd))
        Sv = host(s.apply_schur(vd, c_mode=1, c_rtol=1e-13))
        S2 = host(s.apply_schur(vd))
        den = float(np.dot(v, Lv))
        qs.append(float(np.dot(v, Sv)) / den)
        qs_scalar.append(float(np.dot(v, S2)) / den)
    print(f"Rayleigh quotients exact {qs} scalar {qs_scalar}")
    assert min(qs) >= 1.0 - 1e-12 and max(qs) <= 2.0 + 1e-12
    assert max(qs) > 1.2      # the shell vectors feel the force term
    s.close()
    torch.cuda.synchronize()
