"""The pressure / force-density correction system and its primal Schur
complement, FP64, CPU.  TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

With B = R^T G and C = R^T R (Eq. (Saddle)):

* saddle matrix  [[L, B^T], [B, -C]] (Eq. (Saddle), read literally: the
  paper's Theorem 1, Table 2 (PrecResults) and every iteration count refer to this form);
* exact primal Schur complement S_p = L + B^T C^{-1} B (Eq. (SchurPrimal)),
  RHS  RHS_p + B^T C^{-1} RHS_F  (Eq. (SchurPrimalP)),
  force  F' = C^{-1}(B p' - RHS_F)  (Eq. (SchurPrimalF));
* scalar approximation C^{-1} ~ 2 I: S~_p = L + 2 B^T B (Eq. (tildeSp)),
  RHS  RHS_p + 2 B^T RHS_F  (Eq. (ApproxSchurPrimalP)),
  force  F' = 2 (B p' - RHS_F)  (Eq. (ApproxSchurPrimalF));
* the sign-consistent form ("consistent"): asking the update of
  Eq. (u_n_plus_1), u^{n+1} = u* + (1/a)(-G p' + R F'), to satisfy
  G^T u^{n+1} = 0 and R^T u^{n+1} = U^Gamma exactly gives
  [[L, -B^T], [B, -C]] [p'; F'] = [RHS_p; RHS_F] (the sign Eq.
  (modified_poisson) implies), Schur complement
  S_c = L - B^T C^{-1} B = G^T (I - R C^{-1} R^T) G, RHS
  RHS_p - B^T C^{-1} RHS_F and the same force formula as the exact form.
  R C^{-1} R^T is an orthogonal projection, so S_c is positive
  semi-definite with spec(L^+ S_c) in [0, 1]: it is not bounded below the
  way S_p is, which is why the paper's form is the one preconditioned by L.

L is singular (Neumann walls, constants in its null space); B 1 = R^T G 1 = 0,
so S~_p and S_p share that null space and every right-hand side built from
G^T (.) is orthogonal to it.  The oracle's p' is the unique mean-zero solution
(the paper pins a Dirichlet point instead, Sec. 5; a mean-zero projection keeps
L = G^T G exactly symmetric).

Solvers: ``solve_dense`` (pseudo-inverse on the mean-zero subspace, tiny
grids) and ``fgmres`` (right-preconditioned flexible GMRES, textbook modified
Gram-Schmidt Arnoldi with Givens rotations) preconditioned by the exact
``mac.laplacian_pinv``, i.e. the paper's single application of L^{-1} per
Krylov iteration (Sec. 4.2).

Pins (tests/test_oracle_schur.py): dense brute-force solve on small grids;
Theorem 1 (spec(L^+ S_p) in [1, 2]) by a dense generalised eigenproblem;
spec(L^+ S~_p) near [1, 2] as in Table 2 (PrecResults); the Schur elimination against a
direct block solve of Eq. (Saddle); no markers gives p' = L^+ b;
grid-independent FGMRES iteration counts and the large unpreconditioned count
(Sec. 6.2).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import mac
from .delta import regularization_matrix


class SchurSystem:
    """Matrices of Eq. (Saddle) for one grid and one marker set."""

    def __init__(self, g: mac.Grid, X):
        self.g = g
        self.X = np.asarray(X, dtype=np.float64).reshape(3, -1)
        self.R = regularization_matrix(g, self.X)
        self.C = (self.R.T @ self.R).tocsr()           # R^T R
        self.k = self.R.shape[1]
        self._G = None

    # sparse G, L, B for small grids (dense checks)
    @property
    def G(self):
        if self._G is None:
            self._G = mac.gradient_matrix(self.g)
        return self._G

    @property
    def L(self):
        return (self.G.T @ self.G).tocsr()

    @property
    def B(self):
        return (self.R.T @ self.G).tocsr()

    # --- operators -------------------------------------------------------
    def apply_B(self, v):
        """B v = R^T (G v)."""
        return self.R.T @ mac.apply_G(self.g, v)

    def apply_BT(self, t):
        """B^T t = G^T (R t)."""
        return mac.apply_GT(self.g, self.R @ np.asarray(t, dtype=np.float64))

    def apply_S_tilde(self, v):
        """S~_p v = L v + 2 B^T (B v), Eq. (tildeSp)."""
        v = np.asarray(v, dtype=np.float64)
        return mac.apply_L(self.g, v) + 2.0 * self.apply_BT(self.apply_B(v))

    def C_solve(self, t, tol=1e-15):
        """C^{-1} t for the exact Schur complement (Eq. (SchurPrimal))."""
        if self.k == 0:
            return np.zeros(0)
        return spla.spsolve(self.C.tocsc(), np.asarray(t, dtype=np.float64))

    def apply_S_exact(self, v):
        """S_p v = L v + B^T C^{-1} B v, Eq. (SchurPrimal)."""
        v = np.asarray(v, dtype=np.float64)
        return mac.apply_L(self.g, v) + self.apply_BT(self.C_solve(self.apply_B(v)))

    def apply_S_consistent(self, v):
        """S_c v = L v - B^T C^{-1} B v (sign-consistent form)."""
        v = np.asarray(v, dtype=np.float64)
        return mac.apply_L(self.g, v) - self.apply_BT(self.C_solve(self.apply_B(v)))

    def dense_S_consistent(self):
        Bd = self.B.toarray()
        Cd = self.C.toarray()
        return self.L.toarray() - Bd.T @ np.linalg.solve(Cd, Bd)

    def saddle_matrix_consistent(self):
        """[[L, -B^T], [B, -C]], dense."""
        return np.block([[self.L.toarray(), -self.B.T.toarray()],
                         [self.B.toarray(), -self.C.toarray()]])

    def rhs_consistent(self, rhs_p, rhs_F):
        """RHS_p - B^T C^{-1} RHS_F."""
        return np.asarray(rhs_p) - self.apply_BT(self.C_solve(rhs_F))

    def dense_S_tilde(self):
        B = self.B
        return (self.L + 2.0 * (B.T @ B)).toarray()

    def dense_S_exact(self):
        Bd = self.B.toarray()
        Cd = self.C.toarray()
        return self.L.toarray() + Bd.T @ np.linalg.solve(Cd, Bd)

    def saddle_matrix(self):
        """[[L, B^T], [B, -C]] of Eq. (Saddle), dense."""
        return np.block([[self.L.toarray(), self.B.T.toarray()],
                         [self.B.toarray(), -self.C.toarray()]])

    # --- right-hand sides and force recovery -----------------------------
    def rhs_scalar(self, rhs_p, rhs_F):
        """RHS_p + 2 B^T RHS_F, Eq. (ApproxSchurPrimalP)."""
        return np.asarray(rhs_p) + 2.0 * self.apply_BT(rhs_F)

    def rhs_exact(self, rhs_p, rhs_F):
        """RHS_p + B^T C^{-1} RHS_F, Eq. (SchurPrimalP)."""
        return np.asarray(rhs_p) + self.apply_BT(self.C_solve(rhs_F))

    def force_scalar(self, p, rhs_F):
        """F' = 2 (B p' - RHS_F), Eq. (ApproxSchurPrimalF)."""
        return 2.0 * (self.apply_B(p) - np.asarray(rhs_F))

    def force_exact(self, p, rhs_F):
        """F' = C^{-1} (B p' - RHS_F), Eq. (SchurPrimalF)."""
        return self.C_solve(self.apply_B(p) - np.asarray(rhs_F))


def solve_dense(A, b):
    """Mean-zero solution of a consistent singular symmetric system whose
    null space is the constants (pseudo-inverse, tiny grids)."""
    A = np.asarray(A, dtype=np.float64)
    m = A.shape[0]
    J = np.full((m, m), 1.0 / m)
    x = np.linalg.solve(A + J, np.asarray(b, dtype=np.float64))
    return x - x.mean()


def fgmres(apply_A, b, apply_M, rtol=1e-13, restart=60, maxit=600, x0=None):
    """Right-preconditioned flexible GMRES (textbook form): Arnoldi with
    modified Gram-Schmidt on A z_j, z_j = M(v_j), Givens rotations on the
    Hessenberg matrix, x = x0 + Z y.  Stops when the relative unpreconditioned
    residual ||b - A x|| / ||b|| is <= rtol (recomputed at every restart and
    at exit).  Returns (x, iterations, relative true residual, history)."""
    b = np.asarray(b, dtype=np.float64)
    n = b.size
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = np.linalg.norm(b)
    hist = []
    if bnorm == 0.0:
        return np.zeros(n), 0, 0.0, hist
    total = 0
    while True:
        r = b - apply_A(x)
        beta = np.linalg.norm(r)
        if beta / bnorm <= rtol or total >= maxit:
            return x, total, beta / bnorm, hist
        V = np.zeros((restart + 1, n))
        Z = np.zeros((restart, n))
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        gvec = np.zeros(restart + 1)
        gvec[0] = beta
        V[0] = r / beta
        j_used = 0
        for j in range(restart):
            Z[j] = apply_M(V[j])
            w = apply_A(Z[j])
            for i in range(j + 1):
                H[i, j] = np.dot(w, V[i])
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            denom = np.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / denom
            sn[j] = H[j + 1, j] / denom
            H[j, j] = denom
            H[j + 1, j] = 0.0
            gvec[j + 1] = -sn[j] * gvec[j]
            gvec[j] = cs[j] * gvec[j]
            total += 1
            j_used = j + 1
            hist.append(abs(gvec[j + 1]) / bnorm)
            if abs(gvec[j + 1]) / bnorm <= rtol or total >= maxit:
                break
        y = np.linalg.solve(np.triu(H[:j_used, :j_used]), gvec[:j_used])
        x = x + Z[:j_used].T @ y


def solve_schur(sys: SchurSystem, b, mode="scalar", rtol=1e-13, restart=60,
                maxit=600, workers=None):
    """Mean-zero p' solving S~_p p' = b (mode "scalar"), S_p p' = b (mode
    "exact") or S_c p' = b (mode "consistent") by FGMRES preconditioned with
    the exact L^+ (Sec. 4.1-4.2)."""
    A = {"scalar": sys.apply_S_tilde, "exact": sys.apply_S_exact,
         "consistent": sys.apply_S_consistent}[mode]
    M = lambda r: mac.laplacian_pinv(sys.g, r, workers=workers)
    x, it, rel, hist = fgmres(A, b, M, rtol=rtol, restart=restart, maxit=maxit)
    return mac.remove_mean(x), it, rel, hist
