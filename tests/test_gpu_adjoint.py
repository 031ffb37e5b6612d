"""The adjoint of one step on the GPU (ibm_adjoint_step,
ibm_body_forces_adjoint and the autograd wrappers): parity with the oracle's
reverse-mode derivative on small grids, and central differences of the GPU
forward step on the 128^3 oscillating sphere."""
import numpy as np
import pytest

import gpu_cases as gc
from gpu_cases import dev, host, rel

pytestmark = pytest.mark.gpu

FP64 = dict(precond_prec=0, rtol=1e-13, helm_rtol=1e-14, helm_maxit=12)


def _inputs(case, history, seed=7):
    g = case.grid()
    rng = np.random.default_rng(seed)
    mask = g.interior_face_mask_packed()
    U = rng.uniform(-1, 1, 3 * case.N)
    f = rng.standard_normal(g.n_faces) * mask
    if history:
        st = dict(u_n=0.3 * rng.standard_normal(g.n_faces) * mask,
                  u_nm1=0.3 * rng.standard_normal(g.n_faces) * mask,
                  p_n=rng.standard_normal(g.m), F_n=rng.standard_normal(3 * case.N))
    else:
        st = dict(u_n=np.zeros(g.n_faces), u_nm1=np.zeros(g.n_faces), p_n=np.zeros(g.m),
                  F_n=np.zeros(3 * case.N))
    return U, f, st


def _oracle(case, U, f, st, w):
    from oracle import adjoint, step
    g = case.grid()
    fw = step.step(g, case.Re, case.dt, case.X, U, f, rtol=1e-13, **st)
    F_bar, X_lever, c_bar = adjoint.body_force_torque_vjp(g, case.X, fw["F"], case.body_id,
                                                          case.centers, w)
    r = adjoint.step_vjp(g, case.Re, case.dt, case.X, fw, F_bar, F_n=st["F_n"])
    return dict(F_bar=F_bar, X_lever=X_lever.ravel(), c_bar=c_bar, U_bar=r["U_bar"],
                X_bar=r["X_bar"].ravel())


def _gpu(case, U, f, st, w, **opts):
    import torch
    from paper_2501_15314_gb300.api import IBMSolver
    s = IBMSolver(case.nx, case.ny, case.nz, case.h, Re=case.Re, dt=case.dt)
    X = dev(case.X)
    s.set_markers(X)
    F_n = dev(st["F_n"])
    out, _ = s.step(dev(st["u_n"]), dev(st["u_nm1"]), dev(st["p_n"]), F_n, dev(U), dev(f), **opts)
    bid = dev(case.body_id).to(torch.int32)
    loads = s.body_forces(out["F"], X, bid, case.centers)
    F_bar, X_lever, c_bar = s.body_forces_adjoint(out["F"], X, bid, case.centers, w, loads)
    U_bar, X_bar, ast = s.adjoint_step(out["u"], F_n, out["F"], F_bar, **opts)
    res = dict(F_bar=host(F_bar), X_lever=host(X_lever), c_bar=c_bar, U_bar=host(U_bar),
               X_bar=host(X_bar), stats=ast)
    s.close()
    return res


@pytest.mark.parametrize("history", [False, True], ids=["from_rest", "history"])
@pytest.mark.parametrize("make", [gc.sphere16, gc.ragged_multi], ids=["sphere16", "ragged"])
def test_adjoint_matches_oracle(cuda_device, make, history):
    case = make()
    nb = case.centers.shape[0]
    w = np.random.default_rng(3).standard_normal((nb, 6))
    U, f, st = _inputs(case, history)
    ref = _oracle(case, U, f, st, w)
    out = _gpu(case, U, f, st, w, **FP64)
    for k in ("F_bar", "X_lever", "U_bar", "X_bar"):
        assert rel(out[k], ref[k]) < 1e-10, (k, rel(out[k], ref[k]))
    assert rel(out["c_bar"], ref["c_bar"]) < 1e-10
    assert out["stats"]["relres_true"] <= 1e-13
    if history:
        assert out["stats"]["helm_iters"] >= 1   # the mu solve ran


def test_adjoint_mixed_precision_against_oracle(cuda_device):
    """Default options (FP32 V-cycle, double-single Arnoldi, rtol 1e-8): the
    adjoint solve reaches 1e-8 and the gradient error stays at that level."""
    case = gc.ragged_multi()
    w = np.random.default_rng(4).standard_normal((case.centers.shape[0], 6))
    U, f, st = _inputs(case, True, seed=8)
    ref = _oracle(case, U, f, st, w)
    out = _gpu(case, U, f, st, w, helm_rtol=1e-12)
    assert out["stats"]["relres_true"] <= 1e-8
    assert rel(out["U_bar"], ref["U_bar"]) < 1e-6
    assert rel(out["X_bar"], ref["X_bar"]) < 1e-6


def test_adjoint_no_markers(cuda_device):
    import torch
    from paper_2501_15314_gb300.api import IBMSolver
    s = IBMSolver(16)
    s.set_markers(torch.zeros((3, 0), dtype=torch.float64, device="cuda"))
    u = torch.zeros(s.nf, dtype=torch.float64, device="cuda")
    U_bar, X_bar, st = s.adjoint_step(u, None, None, None)
    assert U_bar.numel() == 0 and X_bar.numel() == 0 and st["iters"] == 0
    s.close()


def _loss_fn(s, X_rel, Xc, U, state, bid, opts):
    from paper_2501_15314_gb300.autograd import body_loads, ib_step
    X = X_rel + Xc.view(3, 1)
    F, _, _ = ib_step(s, X, U, state, **opts)
    loads = body_loads(s, F, X, bid, Xc.view(1, 3))
    return -(loads[0, 2] + loads[0, 5])   # drag_z + torque_z on the body


def test_autograd_matches_oracle_small(cuda_device):
    """X = X_rel + X_c with X_c and U^Gamma leaves: autograd's gradients equal
    the oracle's summed over the rigid translation."""
    import torch
    from oracle import adjoint
    from paper_2501_15314_gb300.api import IBMSolver
    case = gc.sphere16()
    U, f, st = _inputs(case, True, seed=9)
    w = adjoint.drag_torque_weights(1)
    ref = _oracle(case, U, f, st, w)
    grad_c_ref = (ref["X_bar"] + ref["X_lever"]).reshape(3, -1).sum(axis=1) + ref["c_bar"][0]
    s = IBMSolver(case.nx, case.ny, case.nz, case.h, Re=case.Re, dt=case.dt)
    c0 = case.centers[0]
    Xc = torch.tensor(c0, dtype=torch.float64, device="cuda", requires_grad=True)
    X_rel = dev(case.X - c0[:, None])
    Ut = dev(U).requires_grad_(True)
    state = {k: dev(v) for k, v in st.items()}
    state["f_body"] = dev(f)
    bid = dev(case.body_id).to(torch.int32)
    J = _loss_fn(s, X_rel, Xc, Ut, state, bid, FP64)
    J.backward()
    assert rel(host(Ut.grad), ref["U_bar"]) < 1e-10
    assert rel(host(Xc.grad), grad_c_ref) < 1e-10
    s.close()


def test_finite_differences_oscillating_sphere_128(cuda_device):
    """The 128^3 oscillating sphere (16000 markers, FP64, rtol 1e-13).

    Marker velocities: J is linear in U^Gamma, so central differences of step
    1e-6 along random directions agree to round-off.

    Centre coordinates: two things limit a central difference here.
    (i) phi of Eq. (delta) is only C^1 (phi'' jumps at |r| = 1/2, 3/2): every
    tap that crosses such a breakpoint within the step makes the quotient
    O(step) wrong, and the centre gradient (about 0.1) is a strongly
    cancelling sum over 16000 markers, so this truncation error is large
    (3e-5 at step 1e-6, 8e-7 at 1e-7, falling about as step^1.8).
    (ii) The FP64 forward step reproduces J (about 6) only to a few 1e-15, an
    error of about 3e-14 / step in the quotient.  The two balance near
    step 5e-8 at a few 1e-7; central differences at eight steps in
    [5e-8, 8.5e-8] share the truncation error but not the rounding, and
    their mean is compared with the adjoint gradient.  The single-step
    errors at 1e-6 and 1e-7 are printed for the record."""
    import torch
    from paper_2501_15314_gb300.api import IBMSolver
    case = gc.config_case(4, secondary=True)
    s = IBMSolver(case.nx, case.ny, case.nz, case.h, Re=case.Re, dt=case.dt)
    c0 = case.centers[0]
    X_rel = dev(case.X - c0[:, None])
    bid = dev(case.body_id).to(torch.int32)
    z = lambda n: torch.zeros(n, dtype=torch.float64, device="cuda")  # noqa: E731
    state = dict(u_n=z(s.nf), u_nm1=z(s.nf), p_n=z(s.m), F_n=z(3 * case.N),
                 f_body=dev(case.f_body))
    Xc = torch.tensor(c0, dtype=torch.float64, device="cuda", requires_grad=True)
    Ut = dev(case.U_gamma).requires_grad_(True)
    J = _loss_fn(s, X_rel, Xc, Ut, state, bid, FP64)
    J.backward()
    gc_ad, gU = host(Xc.grad), host(Ut.grad)
    assert s.last_adjoint_stats["relres_true"] <= 1e-13

    def J_at(Xc_v, U_v):
        with torch.no_grad():
            return float(_loss_fn(s, X_rel, Xc_v, U_v, state, bid, FP64))

    def fd_centre(e):
        fd = np.empty(3)
        for ax in range(3):
            d = torch.zeros(3, dtype=torch.float64, device="cuda")
            d[ax] = e
            fd[ax] = (J_at(Xc.detach() + d, Ut.detach())
                      - J_at(Xc.detach() - d, Ut.detach())) / (2 * e)
        return fd

    def err(fd):
        return float(np.linalg.norm(gc_ad - fd) / np.linalg.norm(fd))

    single = {e: err(fd_centre(e)) for e in (1e-6, 1e-7)}
    fd_mean = np.mean([fd_centre(5e-8 * (1 + 0.1 * i)) for i in range(8)], axis=0)
    err_mean = err(fd_mean)
    e = 1e-6
    rng = np.random.default_rng(4)
    errs_U = []
    for _ in range(3):
        dU = dev(rng.standard_normal(3 * case.N))
        fd = (J_at(Xc.detach(), Ut.detach() + e * dU)
              - J_at(Xc.detach(), Ut.detach() - e * dU)) / (2 * e)
        errs_U.append(abs(float(np.dot(gU, host(dU))) - fd) / abs(fd))
    print(f"J {float(J.detach()):.12g} centre gradient {gc_ad}; centre FD rel error: single steps "
          f"{single}, mean over steps 5e-8..8.5e-8 {err_mean:.3e}; "
          f"U directions rel error (step 1e-6) {errs_U}")
    assert err_mean < 1e-6
    assert max(errs_U) < 1e-6
    s.close()
