"""Ten consecutive one-way steps at 128^3 (one sphere r = 0.15, 4632
markers at Lagrangian spacing h, Re 100, dt 2e-3, sine-mode body force,
rigid marker velocities;
BDF2 history and the convective term active from the second step): the GPU
FP64 form and the mixed form (FP32 V-cycle) against the oracle, step by
step.  The sphere moves rigidly between steps (prescribed motion, the same
marker positions on both sides).  The stated count of 16000 markers (spacing
h/1.86) is not used here: with C^{-1} ~ 2 I the time integration diverges
for spacing ratios above about 1.58 (Table A1, RtR_spacing), and it does on
the GPU too (|F| reached 1e10 within eight steps)."""
import numpy as np
import pytest

from gpu_cases import dev, host, rel

pytestmark = pytest.mark.gpu


def _rotation(w, dt):
    """exp(dt [w]x) by the Rodrigues formula."""
    a = np.linalg.norm(w) * dt
    if a == 0.0:
        return np.eye(3)
    k = w / np.linalg.norm(w)
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + np.sin(a) * K + (1 - np.cos(a)) * K @ K


def test_ten_steps_128_against_oracle(cuda_device):
    from oracle import mac, step
    from paper_2501_15314_gb300 import workloads as wl
    from paper_2501_15314_gb300.api import IBMSolver
    W = wl.config(2)
    g = mac.Grid(W.n)
    rng = np.random.default_rng(20)
    us, om = rng.uniform(-1, 1, 3), rng.uniform(-1, 1, 3)
    c = W.centers[0].copy()
    X = W.X.copy()
    Rstep = _rotation(om, W.dt)
    solvers = {name: IBMSolver(W.n, Re=W.Re, dt=W.dt) for name in ("fp64", "mixed")}
    opts = {"fp64": dict(precond_prec=0, arnoldi=0, rtol=1e-12, helm_rtol=1e-13, helm_maxit=12),
            "mixed": dict(precond_prec=1, rtol=1e-8, helm_rtol=1e-10)}
    st_o = dict(u_n=np.zeros(g.n_faces), u_nm1=np.zeros(g.n_faces), p_n=np.zeros(g.m),
                F_n=np.zeros(3 * W.n_markers))
    st_g = {k: {kk: dev(v) for kk, v in st_o.items()} for k in solvers}
    f = dev(W.f_body)
    errs = []
    for n in range(10):
        U = us[:, None] + np.cross(om, (X - c[:, None]).T).T
        ref = step.step(g, W.Re, W.dt, X, U, W.f_body, rtol=1e-12, workers=8, **st_o)
        e = {}
        for name, s in solvers.items():
            sg = st_g[name]
            s.set_markers(dev(X))
            out, stat = s.step(sg["u_n"], sg["u_nm1"], sg["p_n"], sg["F_n"], dev(U.ravel()), f,
                               **opts[name])
            e[name] = {k: rel(host(out[k]), ref[k]) for k in ("u", "p", "F")}
            e[name]["iters"] = stat["iters"]
            sg["u_nm1"], sg["u_n"] = sg["u_n"], out["u"].clone()
            sg["p_n"], sg["F_n"] = out["p"].clone(), out["F"].clone()
        errs.append(e)
        st_o = dict(u_n=ref["u"], u_nm1=st_o["u_n"], p_n=ref["p"], F_n=ref["F"])
        # rigid motion to the next step
        X = (c + W.dt * us)[:, None] + Rstep @ (X - c[:, None])
        c = c + W.dt * us
    for s in solvers.values():
        s.close()
    for n, e in enumerate(errs):
        print(f"step {n + 1}: fp64 {e['fp64']}  mixed {e['mixed']}")
    for e in errs:
        for k in ("u", "p", "F"):
            assert e["fp64"][k] < 1e-10, errs
            assert e["mixed"][k] < 1e-6, errs
