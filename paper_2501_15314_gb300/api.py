"""Torch-facing wrapper of the C ABI (include/ibm_schur.h).

PyTorch provides device memory and the stream; every operation is one call
into libibmschur.  Tensors must be contiguous CUDA float64 (int32 for body
ids) in the layouts of the header: cells [nz][ny][nx] flattened, packed faces
u_x|u_y|u_z, marker arrays [3][N].
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _lib
from ._lib import IBM_PREC_FP32, IBM_PREC_FP64, check

__all__ = ["IBMSolver", "RigidSpheres", "IBM_PREC_FP32", "IBM_PREC_FP64"]


def _ptr(t: torch.Tensor, dtype=torch.float64, numel=None, name="tensor") -> int:
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.device.type != "cuda" or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, expected {numel}")
    return t.data_ptr()


def _stats_dict(st: _lib.ibm_solve_stats) -> dict:
    n = min(st.iters, _lib.HIST_MAX)
    return dict(iters=st.iters, restarts=st.restarts, relres_true=st.relres_true,
                relres_hist=list(st.relres_hist[:n]), helm_iters=st.helm_iters,
                helm_relres=st.helm_relres, div_l2=st.div_l2, slip_l2=st.slip_l2,
                c_iters=st.c_iters, graph_cycles=st.graph_cycles)


class RigidSpheres:
    """Host state of rigid spheres for ``IBMSolver.fsi_step`` (a ctypes array
    of ibm_rigid_sphere, advanced in place by every step)."""

    def __init__(self, radii, thetas, centers, velocities=None, omegas=None, free=True):
        import numpy as np
        centers = np.asarray(centers, dtype=np.float64).reshape(-1, 3)
        nb = centers.shape[0]
        radii = np.broadcast_to(np.asarray(radii, dtype=np.float64), (nb,))
        thetas = np.broadcast_to(np.asarray(thetas, dtype=np.float64), (nb,))
        vel = np.zeros((nb, 3)) if velocities is None else \
            np.asarray(velocities, dtype=np.float64).reshape(nb, 3)
        omg = np.zeros((nb, 3)) if omegas is None else \
            np.asarray(omegas, dtype=np.float64).reshape(nb, 3)
        free = np.broadcast_to(np.asarray(free), (nb,))
        self.arr = (_lib.ibm_rigid_sphere * nb)()
        for b in range(nb):
            s = self.arr[b]
            s.radius, s.theta = float(radii[b]), float(thetas[b])
            for e in range(3):
                s.xc[e] = s.xc_prev[e] = centers[b, e]
                s.us[e] = s.us_prev[e] = vel[b, e]
                s.om[e] = s.om_prev[e] = omg[b, e]
                s.om_cs[e] = s.om_cs_prev[e] = omg[b, e]
            for q in range(9):
                s.rot[q] = 1.0 if q % 4 == 0 else 0.0
            s.free_motion = 1 if free[b] else 0
        self.n = nb

    def get(self, name):
        """One field of every sphere: (n,) for a scalar field, (n, k) for an
        array field."""
        import numpy as np
        vals = [getattr(self.arr[b], name) for b in range(self.n)]
        return np.array([list(v) if hasattr(v, "__len__") else v for v in vals])


class IBMSolver:
    """One MAC grid (nx, ny, nz, h) with its workspace on the current device.

    The library runs on ``stream`` (default: the current stream at creation).
    Every call is ordered after the caller's current stream at the time of the
    call (where its inputs and freshly allocated outputs were written), and
    the caller's current stream after the call (where the results are read),
    so tensors can be produced and consumed on any stream.  Inputs are
    contiguous CUDA float64 tensors (int32 for body ids) in the layouts of
    include/ibm_schur.h."""

    def __init__(self, nx: int, ny: int | None = None, nz: int | None = None,
                 h: float | None = None, Re: float = 100.0, dt: float = 0.01,
                 stream: torch.cuda.Stream | None = None):
        self.lib = _lib.load()
        ny = nx if ny is None else ny
        nz = nx if nz is None else nz
        h = 1.0 / nx if h is None else h
        self.nx, self.ny, self.nz, self.h, self.Re, self.dt = nx, ny, nz, h, Re, dt
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        g = _lib.ibm_grid_desc(nx, ny, nz, h, Re, dt)
        ctx = C.c_void_p()
        st = self.lib.ibm_create(C.byref(g), C.c_void_p(self.stream.cuda_stream), C.byref(ctx))
        if st != _lib.IBM_OK:
            raise _lib.IBMError(st, "ibm_create failed")
        self.ctx = ctx
        self.m = self.lib.ibm_num_cells(ctx)
        self.nf = self.lib.ibm_num_faces(ctx)
        self.n_markers = 0

    # -- lifetime ---------------------------------------------------------
    def close(self):
        if getattr(self, "ctx", None):
            self.lib.ibm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _call(self, name, *args):
        """One library call on the solver's stream.  When the caller's current
        stream is another one, the call is ordered after it (where the inputs
        and the freshly allocated outputs were written) and the current
        stream after the call (where the results are read)."""
        cur = torch.cuda.current_stream()
        other = cur != self.stream
        if other:
            self.stream.wait_stream(cur)
        status = getattr(self.lib, name)(self.ctx, *args)
        if other:
            cur.wait_stream(self.stream)
        return status

    def _cells(self, **kw):
        return torch.empty(self.m, dtype=torch.float64, device="cuda", **kw)

    def _faces(self):
        return torch.empty(self.nf, dtype=torch.float64, device="cuda")

    # -- setup ------------------------------------------------------------
    def set_markers(self, X: torch.Tensor):
        X = X.reshape(3, -1) if X.numel() else X
        n = X.shape[1] if X.numel() else 0
        check(self._call("ibm_set_markers", n, _ptr(X, name="X") if n else None), self.ctx)
        self.n_markers = n
        self._X = X

    # -- operators --------------------------------------------------------
    def apply_laplacian(self, v, out=None):
        out = self._cells() if out is None else out
        check(self._call("ibm_apply_laplacian", _ptr(v, numel=self.m, name="v"),
                                           _ptr(out, numel=self.m, name="out")), self.ctx)
        return out

    def apply_schur(self, v, out=None, **kw):
        """S v: the scalar form S~ by default; with keyword options (c_mode,
        c_rtol, c_maxit) the form they select."""
        out = self._cells() if out is None else out
        if not kw:
            check(self._call("ibm_apply_schur", _ptr(v, numel=self.m, name="v"),
                                           _ptr(out, numel=self.m, name="out")), self.ctx)
            return out
        o = self.opts(**kw)
        it = C.c_int64(0)
        check(self._call("ibm_apply_schur_opts", _ptr(v, numel=self.m, name="v"),
                                            _ptr(out, numel=self.m, name="out"), C.byref(o),
                                            C.byref(it)), self.ctx)
        self.last_c_iters = it.value
        return out

    def apply_c_inverse(self, t, c_rtol=1e-14, c_maxit=500, out=None):
        """s = C^{-1} t, C = R^T R, by conjugate gradients; returns (s, iterations)."""
        nmk = 3 * self.n_markers
        out = torch.zeros(max(nmk, 1), dtype=torch.float64, device="cuda") if out is None else out
        it = C.c_int32(0)
        if nmk:
            check(self._call("ibm_apply_c_inverse", _ptr(t, numel=nmk, name="t"),
                                               _ptr(out, name="s"), c_rtol, c_maxit,
                                               C.byref(it)), self.ctx)
        return out[:nmk], it.value

    def precond(self, r, prec=IBM_PREC_FP32, pre=2, post=2, out=None):
        out = self._cells() if out is None else out
        check(self._call("ibm_apply_laplacian_precond",
            _ptr(r, numel=self.m, name="r"), _ptr(out, numel=self.m, name="z"),
            prec, pre, post), self.ctx)
        return out

    def interp(self, u, out=None):
        out = torch.zeros(3 * self.n_markers, dtype=torch.float64, device="cuda") \
            if out is None else out
        if self.n_markers:
            check(self._call("ibm_interp", _ptr(u, numel=self.nf, name="u"),
                                      _ptr(out, name="U")), self.ctx)
        return out

    def spread(self, F, out=None):
        out = self._faces() if out is None else out
        check(self._call("ibm_spread", _ptr(F, name="F") if self.n_markers else None,
                                  _ptr(out, numel=self.nf, name="u")), self.ctx)
        return out

    def gradient(self, p, out=None):
        out = self._faces() if out is None else out
        check(self._call("ibm_gradient", _ptr(p, numel=self.m, name="p"),
                                    _ptr(out, numel=self.nf, name="u")), self.ctx)
        return out

    def gradient_t(self, u, out=None):
        out = self._cells() if out is None else out
        check(self._call("ibm_gradient_t", _ptr(u, numel=self.nf, name="u"),
                                      _ptr(out, numel=self.m, name="out")), self.ctx)
        return out

    def force_correction(self, p, rhs_F, out=None):
        out = torch.zeros(3 * self.n_markers, dtype=torch.float64, device="cuda") \
            if out is None else out
        if self.n_markers:
            check(self._call("ibm_force_correction", _ptr(p, numel=self.m, name="p"),
                                                _ptr(rhs_F, name="rhs_F"),
                                                _ptr(out, name="F")), self.ctx)
        return out

    # -- solves -------------------------------------------------------------
    def opts(self, **kw) -> _lib.ibm_solve_opts:
        o = _lib.default_opts()
        for k, v in kw.items():
            if not hasattr(o, k):
                raise KeyError(k)
            setattr(o, k, v)
        return o

    def solve_schur(self, b, x0=None, raise_on_error=True, **kw):
        p = torch.zeros(self.m, dtype=torch.float64, device="cuda") if x0 is None \
            else x0.clone()
        o = self.opts(**kw)
        st = _lib.ibm_solve_stats()
        status = self._call("ibm_solve_schur", _ptr(b, numel=self.m, name="b"),
                                          _ptr(p, numel=self.m, name="p"), C.byref(o),
                                          C.byref(st))
        if raise_on_error:
            check(status, self.ctx)
        d = _stats_dict(st)
        d["status"] = status
        return p, d

    def step(self, u_n, u_nm1, p_n, F_n, U_gamma, f_body=None, out=None,
             raise_on_error=True, **kw):
        nmk = 3 * self.n_markers
        if out is None:
            out = dict(u=self._faces(), p=self._cells(),
                       F=torch.zeros(max(nmk, 1), dtype=torch.float64, device="cuda"))
        o = self.opts(**kw)
        st = _lib.ibm_solve_stats()
        status = self._call("ibm_step",
            _ptr(u_n, numel=self.nf, name="u_n"),
            _ptr(u_nm1, numel=self.nf, name="u_nm1"), _ptr(p_n, numel=self.m, name="p_n"),
            _ptr(F_n, name="F_n") if nmk else None,
            _ptr(U_gamma, name="U_gamma") if nmk else None,
            _ptr(f_body, numel=self.nf, name="f_body") if f_body is not None else None,
            _ptr(out["u"], numel=self.nf, name="u_np1"), _ptr(out["p"], numel=self.m, name="p_np1"),
            _ptr(out["F"], name="F_np1") if nmk else None, C.byref(o), C.byref(st))
        if raise_on_error:
            check(status, self.ctx)
        d = _stats_dict(st)
        d["status"] = status
        return out, d

    def fsi_step(self, spheres: "RigidSpheres", L0, body_id, u_n, u_nm1, p_n, F_n, f_body=None,
                 out=None, gravity=(0.0, 0.0, 0.0), xi=1.0, tol=1e-3, max_inner=50,
                 criterion=_lib.IBM_FSI_CRIT_LAGRANGIAN,
                 raise_on_error=True, **kw):
        """One two-way coupled step (Sec. 3.2); spheres advance in place.
        Returns (dict(X, u, p, F), stats)."""
        L0 = L0.reshape(3, -1)
        n = L0.shape[1]
        nmk = 3 * n
        if out is None:
            out = dict(X=torch.empty(nmk, dtype=torch.float64, device="cuda"), u=self._faces(),
                       p=self._cells(), F=torch.empty(nmk, dtype=torch.float64, device="cuda"))
        o = self.opts(**kw)
        fo = _lib.ibm_fsi_opts()
        self.lib.ibm_default_fsi_opts(C.byref(fo))
        for e in range(3):
            fo.gravity[e] = float(gravity[e])
        fo.xi, fo.tol, fo.max_inner = float(xi), float(tol), int(max_inner)
        fo.criterion = int(criterion)
        st = _lib.ibm_fsi_stats()
        status = self._call("ibm_fsi_step",
            spheres.n, spheres.arr, n, _ptr(L0, numel=nmk, name="L0"),
            _ptr(body_id, dtype=torch.int32, numel=n, name="body_id"),
            _ptr(u_n, numel=self.nf, name="u_n"), _ptr(u_nm1, numel=self.nf, name="u_nm1"),
            _ptr(p_n, numel=self.m, name="p_n"), _ptr(F_n, numel=nmk, name="F_n"),
            _ptr(f_body, numel=self.nf, name="f_body") if f_body is not None else None,
            _ptr(out["X"], numel=nmk, name="X"), _ptr(out["u"], numel=self.nf, name="u"),
            _ptr(out["p"], numel=self.m, name="p"), _ptr(out["F"], numel=nmk, name="F"),
            C.byref(o), C.byref(fo), C.byref(st))
        if raise_on_error:
            check(status, self.ctx)
        self.n_markers = n
        return out, dict(inner=st.inner, fgmres_iters=st.fgmres_iters, ratio=st.ratio,
                         helm_iters=st.helm_iters, helm_relres=st.helm_relres, status=status)

    def profile_enable(self, on=True):
        check(self._call("ibm_profile_enable", 1 if on else 0), self.ctx)

    def profile_read(self) -> dict:
        p = _lib.ibm_profile()
        check(self._call("ibm_profile_read", C.byref(p)), self.ctx)
        return {name: dict(ms=p.ms[i], launches=p.launches[i], bytes=p.bytes[i])
                for i, name in enumerate(_lib.PROF_NAMES)}

    def adjoint_step(self, u_np1, F_n, F_np1, F_bar, raise_on_error=True, **kw):
        """Adjoint of ``step`` (markers as last set, same options): returns
        (U_bar, X_bar, stats) for the cotangent F_bar = dJ/dF^{n+1}; X_bar is
        the part of dJ/dX that flows through R.  F_n may be None (zero)."""
        nmk = 3 * self.n_markers
        U_bar = torch.zeros(max(nmk, 1), dtype=torch.float64, device="cuda")
        X_bar = torch.zeros(max(nmk, 1), dtype=torch.float64, device="cuda")
        o = self.opts(**kw)
        st = _lib.ibm_solve_stats()
        status = self._call("ibm_adjoint_step",
            _ptr(u_np1, numel=self.nf, name="u_np1"),
            _ptr(F_n, numel=nmk, name="F_n") if (nmk and F_n is not None) else None,
            _ptr(F_np1, numel=nmk, name="F_np1") if nmk else None,
            _ptr(F_bar, numel=nmk, name="F_bar") if nmk else None,
            _ptr(U_bar, name="U_bar") if nmk else None,
            _ptr(X_bar, name="X_bar") if nmk else None, C.byref(o), C.byref(st))
        if raise_on_error:
            check(status, self.ctx)
        d = _stats_dict(st)
        d["status"] = status
        return U_bar[:nmk], X_bar[:nmk], d

    def body_forces_adjoint(self, F, X, body_id, centers, w, out):
        """Adjoint of ``body_forces`` for J = sum(w * out): returns
        (F_bar (device), X_bar through the lever arms (device),
        centers_bar (host numpy))."""
        import numpy as np
        centers = np.ascontiguousarray(np.asarray(centers, dtype=np.float64).reshape(-1, 3))
        nb = centers.shape[0]
        w = np.ascontiguousarray(np.asarray(w, dtype=np.float64).reshape(nb, 6))
        out = np.ascontiguousarray(np.asarray(out, dtype=np.float64).reshape(nb, 6))
        nmk = 3 * self.n_markers
        F_bar = torch.zeros(max(nmk, 1), dtype=torch.float64, device="cuda")
        X_bar = torch.zeros(max(nmk, 1), dtype=torch.float64, device="cuda")
        c_bar = np.zeros((nb, 3))
        dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))  # noqa: E731
        check(self._call("ibm_body_forces_adjoint",
            _ptr(F, name="F") if nmk else None, _ptr(X, name="X") if nmk else None,
            _ptr(body_id, dtype=torch.int32, name="body_id") if nmk else None, nb,
            dp(centers), dp(w), dp(out), _ptr(F_bar, name="F_bar") if nmk else None,
            _ptr(X_bar, name="X_bar") if nmk else None, dp(c_bar)), self.ctx)
        return F_bar[:nmk], X_bar[:nmk], c_bar

    def body_forces(self, F, X, body_id, centers):
        import numpy as np
        centers = np.ascontiguousarray(np.asarray(centers, dtype=np.float64).reshape(-1, 3))
        nb = centers.shape[0]
        out = np.zeros((nb, 6))
        check(self._call("ibm_body_forces",
            _ptr(F, name="F"), _ptr(X, name="X"),
            _ptr(body_id, dtype=torch.int32, name="body_id"), nb,
            centers.ctypes.data_as(C.POINTER(C.c_double)),
            out.ctypes.data_as(C.POINTER(C.c_double))), self.ctx)
        return out
