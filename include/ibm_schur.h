/*
 * ibm_schur.h -- C ABI of the GB300 (sm_103a) Laplacian-preconditioned Schur
 * solver for the SIMPLE-based direct-forcing immersed boundary method
 * (Yovel, Treister & Feldman, arXiv 2501.15314).
 *
 * Problem (Sec. 3.1, Eq. (Saddle)): on a staggered MAC grid with pressure at
 * cell centres and velocity components on faces, with Lagrangian markers X_k
 * carrying forces F_k, the pressure / force-density corrections solve
 *
 *     [ L  B^T ] [p']   [RHS_p]      L = G^T G,  B = R^T G,  C = R^T R,
 *     [ B  -C  ] [F'] = [RHS_F],
 *
 * G the central-difference gradient (cells -> interior faces), G^T = -div,
 * R the regularisation (Eq. (regularization)) built from Roma's 3-point delta
 * (Eq. (delta)) and R^T the interpolation (Eq. (interpolation)).  With the
 * scalar approximation C^{-1} ~ 2I (Eq. (tildeSp)) the primal Schur complement
 * S~ = L + 2 B^T B is solved by a Krylov method preconditioned with the
 * Laplacian (Sec. 4.1-4.2): here right-preconditioned flexible GMRES in FP64
 * with one geometric-multigrid V-cycle (FP32 or FP64) standing in for L^{-1}.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Grid: nx*ny*nz cells of width h; domain [0,nx h]x[0,ny h]x[0,nz h]; all six
 *   walls no-slip.
 * Layout (C order, x fastest):
 *   cell field   [nz][ny][nx]                                 (m = nx ny nz)
 *   face vector  u_x [nz][ny][nx+1] ++ u_y [nz][ny+1][nx] ++ u_z [nz+1][ny][nx]
 *                packed contiguously in that order (n_faces values); the
 *                wall-normal faces on the walls are not unknowns, inputs there
 *                are ignored and outputs there are written as 0.
 *   marker data  structure-of-arrays [3][n_markers]: all x, then all y, then
 *                all z (positions, velocities, forces alike).
 * Memory: every field pointer is caller-owned DEVICE memory holding FP64
 *   (int32 where stated), contiguous, 8-byte aligned; the library never frees
 *   it.  The library owns only the workspace it allocates in ibm_create /
 *   ibm_set_markers and frees in ibm_destroy.
 * Streams: all work is enqueued on the stream given to ibm_create (the Schur
 *   product forks its marker interpolation onto an internal stream and joins
 *   it back before the product completes).  Entry points that return
 *   statistics or detect errors on the device synchronise that stream before
 *   returning (stated per call); the others are asynchronous.
 *   ibm_set_markers, ibm_solve_schur and ibm_step use no copy engine: their
 *   zeroing and device-to-device copies are kernels, and the scalars the host
 *   reads (residual norms, Hessenberg entries, counts, error flags) are
 *   written by kernels into mapped pinned host memory, so host transfers the
 *   caller queues on other streams run alongside without delaying them.
 * Errors: every call returns an ibm_status; ibm_last_error gives a message.
 *   No exception crosses the ABI and no kernel traps or asserts.  Arguments are
 *   validated before any work is enqueued.
 * Singular pressure: L (Neumann) and S~ have the constants as null space.  The
 *   solver returns the mean-zero solution (the paper pins a Dirichlet point
 *   instead, Sec. 5; a mean-zero projection keeps L = G^T G symmetric).
 */
#ifndef IBM_SCHUR_H
#define IBM_SCHUR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ibm_ctx ibm_ctx;

typedef enum {
  IBM_OK = 0,
  IBM_ERR_ARG = 1,            /* invalid argument (null pointer, bad size)   */
  IBM_ERR_CUDA = 2,           /* a CUDA runtime call failed                  */
  IBM_ERR_NOMEM = 3,          /* device allocation failed                    */
  IBM_ERR_NOT_CONVERGED = 4,  /* maxit reached; best iterate is returned     */
  IBM_ERR_BREAKDOWN = 5,      /* Krylov breakdown without convergence        */
  IBM_ERR_NAN = 6,            /* non-finite value in a residual or norm      */
  IBM_ERR_MARKER_DOMAIN = 7,  /* a marker's delta support leaves the interior */
  IBM_ERR_STATE = 8           /* call out of order (e.g. no markers set)     */
} ibm_status;

typedef enum { IBM_PREC_FP64 = 0, IBM_PREC_FP32 = 1 } ibm_precision;

/* Arithmetic of the Arnoldi process (Schur products, Gram-Schmidt, solution
 * update) inside FGMRES.  IBM_ARNOLDI_FP64: native FP64.  IBM_ARNOLDI_DS:
 * vectors held as pairs hi + lo of FP32 numbers (about 48 significant bits),
 * products and sums by error-free transformations on the FP32 pipes.
 * IBM_ARNOLDI_FP32: vectors held as single FP32 numbers (half the bytes of
 * the pairs; the Schur product still formed exactly and rounded once, the
 * sums compensated); a restart cycle ends once its residual estimate has
 * fallen by the FP32 limit (about 4e-6) and the next one starts from the FP64
 * residual, as mixed-precision iterative refinement.  DS and FP32 apply with
 * the FP32 V-cycle on grids with nx a multiple of 4 (otherwise FP64 is
 * used).  In all forms the residual b - S~ x that decides convergence and
 * starts every restart cycle is computed in native FP64. */
typedef enum { IBM_ARNOLDI_FP64 = 0, IBM_ARNOLDI_DS = 1, IBM_ARNOLDI_FP32 = 2 } ibm_arnoldi;

/* Treatment of C = R^T R (the (2,2) block of Eq. (Saddle)).
 * IBM_CMODE_SCALAR: C^{-1} ~ 2 I, the paper's production operator
 *   S~ = L + 2 B^T B (Eqs. (tildeSp)-(ApproxSchurPrimalF)).
 * IBM_CMODE_EXACT: S = L + B^T C^{-1} B, b = RHS_p + B^T C^{-1} RHS_F,
 *   F' = C^{-1}(B p' - RHS_F) (Eqs. (SchurPrimal)-(SchurPrimalF)), the
 *   operator of the spectral theorem of Sec. 5; C^{-1} by conjugate
 *   gradients on C (matrix-free R^T R) to c_rtol inside every product.
 * IBM_CMODE_CONSISTENT: the sign-consistent system [[L, -B^T], [B, -C]]
 *   that the update of Eq. (u_n_plus_1) implies when G^T u^{n+1} = 0 and
 *   R^T u^{n+1} = U^Gamma are imposed exactly: S = L - B^T C^{-1} B,
 *   b = RHS_p - B^T C^{-1} RHS_F, F' as in EXACT.  S is only positive
 *   semi-definite with spec(L^+ S) in [0, 1], so the Laplacian
 *   preconditioner does not bound its iteration count (offered to compare
 *   the two readings of the sign of Eq. (Saddle)). */
typedef enum { IBM_CMODE_SCALAR = 0, IBM_CMODE_EXACT = 1, IBM_CMODE_CONSISTENT = 2 } ibm_cmode;

/* Grid description: cell counts, cell width, Reynolds number and time step
 * (a = 3/(2 dt) and nu = 1/Re enter the BDF2 predictor, Eq. (ustar), and the
 * correction right-hand sides below Eq. (Saddle)). */
typedef struct {
  int32_t nx, ny, nz;
  double h;
  double Re;
  double dt;
} ibm_grid_desc;

/* Solver options (defaults from ibm_default_opts). */
typedef struct {
  int32_t precond_prec;  /* IBM_PREC_FP32: V-cycle stored and accumulated in
                            FP32 (mixed mode); IBM_PREC_FP64: V-cycle in FP64 */
  double rtol;           /* stop when ||b - S x|| / ||b|| <= rtol (FP64)     */
  int32_t maxit;         /* total FGMRES iterations over all restarts        */
  int32_t restart;       /* Krylov basis size (<= 64)                        */
  int32_t mg_pre;        /* Chebyshev degree of the pre-smoother  (0..4)     */
  int32_t mg_post;       /* Chebyshev degree of the post-smoother (0..4)     */
  int32_t reorth;        /* 1: classical Gram-Schmidt applied twice          */
  double helm_rtol;      /* predictor (Helmholtz) relative residual target   */
  int32_t helm_maxit;    /* predictor outer (FP64 defect) iterations         */
  int32_t with_advection;/* 1: include the explicit convective term of
                            Eq. (ustar) in the predictor                     */
  int32_t arnoldi;       /* ibm_arnoldi                                      */
  int32_t c_mode;        /* ibm_cmode                                        */
  double c_rtol;         /* inner CG on C: relative residual target          */
  int32_t c_maxit;       /* inner CG on C: iteration limit per solve         */
  int32_t cycle_graphs;  /* 1: run each FP32 / double-single Arnoldi cycle as
                            one CUDA graph replay (Givens rotations and the
                            stopping test on the device, the next iteration
                            in a conditional node; scalar C mode, profiling
                            off); 0 (default): the host-driven loop, which
                            launches ahead while the residual is far from
                            the target and measured faster on GB300       */
} ibm_solve_opts;

#define IBM_HIST_MAX 256

/* Solve statistics (host memory, filled by the call). */
typedef struct {
  int32_t iters;          /* FGMRES iterations (preconditioner applications) */
  int32_t restarts;       /* completed restart cycles                        */
  double relres_true;     /* ||b - S x|| / ||b|| recomputed in FP64 at exit  */
  double relres_hist[IBM_HIST_MAX]; /* Arnoldi residual estimate per iter   */
  int32_t helm_iters;     /* predictor outer iterations (ibm_step only)      */
  double helm_relres;     /* predictor relative residual (ibm_step only)     */
  double div_l2;          /* ||G^T u^{n+1}||_2            (ibm_step only)    */
  double slip_l2;         /* ||R^T u^{n+1} - U^Gamma||_2  (ibm_step only)    */
  int64_t c_iters;        /* inner CG iterations on C, summed (EXACT and
                             CONSISTENT modes)                               */
  int32_t graph_cycles;   /* restart cycles run as one CUDA graph replay
                             (FP32 / double-single Arnoldi, scalar C form,
                             profiling off): no host round trip inside them */
} ibm_solve_stats;

/* Fills *opts with defaults: FP32 V-cycle, rtol 1e-8, maxit 200, restart 40,
 * Chebyshev (2,2), single Gram-Schmidt pass, helm_rtol 1e-10, helm_maxit 8,
 * advection on, FP32 Arnoldi process with FP64 restarts, scalar C mode
 * (c_rtol 1e-14, c_maxit 500 for the other modes). */
void ibm_default_opts(ibm_solve_opts* opts);

/* Creates a context for one grid and allocates the grid-sized workspace
 * (multigrid hierarchy, temporaries); the Krylov bases are allocated by the
 * first solve for its restart length (grown when a later solve asks more).
 * stream: a cudaStream_t (may be NULL for the legacy default stream).
 * Requires nx, ny, nz >= 4 and h > 0, Re > 0, dt > 0.  Synchronises. */
ibm_status ibm_create(const ibm_grid_desc* grid, void* stream, ibm_ctx** out);

/* Frees the context and all workspace.  Safe on NULL. */
void ibm_destroy(ibm_ctx* ctx);

/* Message for the last error on this context ("" if none).  Valid until the
 * next call on the context. */
const char* ibm_last_error(const ibm_ctx* ctx);

/* Number of cells and packed faces of the context's grid. */
int64_t ibm_num_cells(const ibm_ctx* ctx);
int64_t ibm_num_faces(const ibm_ctx* ctx);

/* Sets the Lagrangian markers (Sec. 2.3): X is device [3][n_markers] FP64
 * positions.  Builds the per-marker Roma weights of Eq. (delta) for the three
 * velocity components and a cell-sorted marker list used by the deterministic
 * (atomic-free) spread.  n_markers == 0 is valid (then S~ = L).  Returns
 * IBM_ERR_MARKER_DOMAIN if a marker's 3x3x3 support for some component
 * touches a wall-normal boundary face or leaves the grid (Appendix B: the
 * support must lie on grid points that exist).  Synchronises. */
ibm_status ibm_set_markers(ibm_ctx* ctx, int64_t n_markers, const double* X);

/* out = L v = G^T G v (cells -> cells), the Neumann 7-point Laplacian of
 * Eq. (Saddle).  v and out must not alias.  Asynchronous. */
ibm_status ibm_apply_laplacian(ibm_ctx* ctx, const double* v, double* out);

/* out = S~ v = L v + 2 B^T B v, Eq. (tildeSp) (cells -> cells), the scalar
 * C mode (ibm_apply_schur_opts for the others).  v and out must not alias.
 * Asynchronous. */
ibm_status ibm_apply_schur(ibm_ctx* ctx, const double* v, double* out);

/* z = M^{-1} r: one multigrid V-cycle for the Neumann Laplacian (Chebyshev
 * smoothing, full-weighting restriction, trilinear prolongation, dense
 * pseudo-inverse on the coarsest level), the preconditioner of Sec. 4.1 (the
 * paper's own suggested replacement for its direct solver, Sec. 7).  prec
 * selects FP32 or FP64 storage/arithmetic inside the cycle; r and z are FP64.
 * The result is not mean-projected.  r and z must not alias.  Asynchronous. */
ibm_status ibm_apply_laplacian_precond(ibm_ctx* ctx, const double* r, double* z,
                                       int32_t prec, int32_t pre, int32_t post);

/* U = R^T u (faces -> markers, [3][n_markers]), Eq. (interpolation).
 * Asynchronous. */
ibm_status ibm_interp(ibm_ctx* ctx, const double* u, double* U);

/* u = R F (markers -> faces), Eq. (regularization); every face is written
 * (0 away from the markers).  Deterministic: each face sums its markers in a
 * fixed order, no atomics.  Asynchronous. */
ibm_status ibm_spread(ibm_ctx* ctx, const double* F, double* u);

/* u = G p (cells -> faces, 0 on wall faces) and out = G^T u (faces -> cells,
 * = -div u).  Asynchronous. */
ibm_status ibm_gradient(ibm_ctx* ctx, const double* p, double* u);
ibm_status ibm_gradient_t(ibm_ctx* ctx, const double* u, double* out);

/* Solves S~ p = b for the mean-zero p (Eq. (ApproxSchurPrimalP)) by
 * right-preconditioned FGMRES(restart) with one V-cycle per iteration.
 * p: in = initial guess x0, out = solution.  b must be orthogonal to the
 * constants (every b built from G^T(.) is).  stats may be NULL.  Synchronises
 * once per iteration (convergence test) and at exit.  Returns
 * IBM_ERR_NOT_CONVERGED if rtol is not met within maxit (p holds the last
 * iterate), IBM_ERR_NAN on a non-finite residual. */
ibm_status ibm_solve_schur(ibm_ctx* ctx, const double* b, double* p,
                           const ibm_solve_opts* opts, ibm_solve_stats* stats);

/* F' = 2 (B p - RHS_F), Eq. (ApproxSchurPrimalF) ([3][n_markers]), the
 * scalar C mode.  Asynchronous. */
ibm_status ibm_force_correction(ibm_ctx* ctx, const double* p,
                                const double* rhs_F, double* F_corr);

/* out = S v for the C mode of opts (c_mode, c_rtol, c_maxit; the other
 * fields are ignored): S~ v, (L + B^T C^{-1} B) v or (L - B^T C^{-1} B) v.
 * c_iters (may be NULL) receives the inner CG iterations.  Returns
 * IBM_ERR_NOT_CONVERGED if an inner CG missed c_rtol.  Synchronises in the
 * non-scalar modes (the CG checks its residual on the host). */
ibm_status ibm_apply_schur_opts(ibm_ctx* ctx, const double* v, double* out,
                                const ibm_solve_opts* opts, int64_t* c_iters);

/* s = C^{-1} t with C = R^T R ([3][n_markers] device vectors, t and s must
 * not alias): conjugate gradients on C, products matrix-free (spread to the
 * shell faces, interpolate back), to ||t - C s|| <= c_rtol ||t|| within
 * c_maxit iterations (IBM_ERR_NOT_CONVERGED otherwise, s holds the last
 * iterate).  iters may be NULL.  Synchronises. */
ibm_status ibm_apply_c_inverse(ibm_ctx* ctx, const double* t, double* s, double c_rtol,
                               int32_t c_maxit, int32_t* iters);

/* One one-way SIMPLE-IBM time step (Sec. 3.1) with the markers last set:
 *   1. predictor (Eq. (ustar)): (3/(2dt) - Lap/Re) u* = (4u^n - u^{n-1})/(2dt)
 *      - G p^n + R F^n - (u.grad u)^n + f_body, solved by FP64 defect
 *      correction around FP32 Chebyshev sweeps to helm_rtol;
 *   2. RHS_p = (3/(2dt)) G^T u*, RHS_F = (3/(2dt)) (R^T u* - U_gamma);
 *   3. ibm_solve_schur on b = RHS_p + 2 B^T RHS_F (scalar C mode;
 *      RHS_p +- B^T C^{-1} RHS_F in the EXACT / CONSISTENT modes);
 *   4. F' = 2 (B p' - RHS_F) (scalar; C^{-1}(B p' - RHS_F) otherwise);
 *   5. u^{n+1} = u* + (2dt/3)(-G p' + R F'), p^{n+1} = p^n + p',
 *      F^{n+1} = F^n + F'  (Eq. (u_n_plus_1) and the correction step);
 *   6. diagnostics ||G^T u^{n+1}||, ||R^T u^{n+1} - U_gamma|| into stats.
 * Inputs u_n, u_nm1 (faces), p_n (cells), F_n, U_gamma ([3][n_markers]),
 * f_body (faces; may be NULL for none).  Outputs u_np1, p_np1, F_np1 must not
 * alias the inputs.  Synchronises like ibm_solve_schur.
 * Input range: the predictor reads u_n, u_nm1, p_n and f_body as pairs of
 * FP32 numbers (hi + lo, within 2^-46 relative), split with integer
 * operations; an entry with |x| < 2^-80 (about 8.3e-25) is read as 0 and one
 * with |x| >= 2^101 (about 2.5e30) as +-infinity (then IBM_ERR_NAN).  So an
 * entry is lost only where it is below 2^-80 in absolute value: a field whose
 * entries that matter are all above that (any flow in units where velocities
 * and pressures are not below about 1e-20) is read to 2^-46 relative.  The
 * same holds for ibm_fsi_step and the predictor solve of ibm_adjoint_step. */
ibm_status ibm_step(ibm_ctx* ctx, const double* u_n, const double* u_nm1,
                    const double* p_n, const double* F_n, const double* U_gamma,
                    const double* f_body, double* u_np1, double* p_np1,
                    double* F_np1, const ibm_solve_opts* opts,
                    ibm_solve_stats* stats);

/* Per body b in [0, n_bodies): out[6b+0..2] = h^3 sum_{k in b} F_k (the IB
 * force sum of Eq. (IBM_force)) and out[6b+3..5] = h^3 sum (X_k - c_b) x F_k.
 * F, X: device [3][n_markers]; body_id: device int32 [n_markers] (values in
 * [0, n_bodies)); centers: host [n_bodies][3]; out: host [n_bodies][6].
 * Deterministic fixed-order reduction.  Synchronises. */
ibm_status ibm_body_forces(ibm_ctx* ctx, const double* F, const double* X,
                           const int32_t* body_id, int32_t n_bodies,
                           const double* centers, double* out);

/* Allocation-free variant of ibm_body_forces, for callers that cannot
 * allocate device memory: code running where cudaMalloc is unavailable or
 * forbidden (inside a caller's own fixed memory budget, under an allocator
 * that must not be re-entered, or in a host process that never creates an
 * ibm_ctx because creating one allocates the solver's workspace).  The paper
 * has no counterpart: it is a deployment convenience, not part of the method.
 *
 * Computes the same per-body force and torque sums as ibm_body_forces
 * (h^3 sum F_k and h^3 sum (X_k - c_b) x F_k) without a context: F, X are
 * device [3][n_markers], body_id device int32 [n_markers], centers host
 * [n_bodies][3], out host [n_bodies][6]; h the cell width; stream a
 * cudaStream_t (NULL = legacy default stream).  Synchronises the stream.
 *
 * Scratch: the device staging buffer (the centres going in, the sums coming
 * out) is a fixed array inside the library of IBM_NOALLOC_MAX_BODIES * 9
 * doubles (72 KiB) that every GPU loading the library holds until the process
 * exits.  No call allocates or frees memory.  A call looks up the current
 * device's address of that array (with the device current) the first time it
 * runs on that device, and again after the device's context has changed (for
 * example after cudaDeviceReset), so make the first call on a device outside
 * any stream capture.  All calls share the array and it keeps the last
 * call's contents: calls whose work overlaps on the GPU (different streams,
 * or different host threads on one device) race and must be serialised by
 * the caller.  Every centre and sum slot a call uses is written by that call,
 * so no clearing is needed between calls.  One kernel launch, one block per
 * body.  The call clears the calling thread's last CUDA runtime error before
 * it launches, so that its own check sees only its own launch.
 * Returns IBM_ERR_ARG when n_bodies < 1 or n_bodies > IBM_NOALLOC_MAX_BODIES,
 * h <= 0, a pointer is missing, F or X is not 8-byte aligned, body_id not
 * 4-byte aligned, or F, X or body_id is not device (or managed) memory of the
 * current device -- all before anything is launched; IBM_ERR_CUDA on a CUDA
 * failure. */
#define IBM_NOALLOC_MAX_BODIES 1024
ibm_status ibm_body_forces_noalloc(const double* F, const double* X, const int32_t* body_id,
                                   int64_t n_markers, int32_t n_bodies, const double* centers,
                                   double h, void* stream, double* out);

/* ---- Two-way coupled rigid spheres (Sec. 3.2) ---------------------------
 * Per sphere, the state at t^n and t^{n-1} that the BDF2 forms of Newton's
 * laws (Eqs. (bdy_linear_vel_iter), (bdy_angular_vel_iter)) and the
 * Rodrigues orientation update (Eqs. (rotat_axis)-(next_time_step_matr))
 * need.  Lengths are those of the grid (fluid density 1): a sphere of radius
 * r has volume V = 4 pi r^3/3 and moment of inertia theta J, J = 2 V r^2/5.
 * Host memory; ibm_fsi_step advances it to t^{n+1}. */
typedef struct {
  double radius;                  /* sphere radius                          */
  double theta;                   /* density ratio rho_p / rho_f            */
  double xc[3], xc_prev[3];       /* centre at t^n, t^{n-1}                 */
  double us[3], us_prev[3];       /* translational velocity                 */
  double om[3], om_prev[3];       /* angular velocity (inertial frame)      */
  double om_cs[3], om_cs_prev[3]; /* angular velocity (body frame)          */
  double rot[9];                  /* orientation R^n, row-major, maps body-
                                     frame vectors to the inertial frame    */
  double mom[3], mom_prev[3];     /* enclosed fluid momentum int_{V_p} u dV */
  double amom[3], amom_prev[3];   /* int_{V_p} (x - x_c) x u dV             */
  int32_t free_motion;            /* 1: Newton's laws; 0: velocities held
                                     (prescribed translation / rotation)   */
} ibm_rigid_sphere;

/* Norm of the stopping test of the two-way corrections,
 * Eq. (convergence_criterion):
 * IBM_FSI_CRIT_LAGRANGIAN: ||F'||_1 / ||F^{(n,k+1)}||_1 over the markers, as
 *   the equation is written;
 * IBM_FSI_CRIT_EULERIAN: ||R F'||_1 / ||R F^{(n,k+1)}||_1 over the faces, the
 *   force densities the fluid receives.  With C^{-1} ~ 2 I a correction damps
 *   the marker mode of eigenvalue lambda of C = R^T R by |1 - 2 lambda|; at
 *   marker spacing h many modes have lambda near 0 (C's smallest eigenvalue
 *   is about 2e-3), so ||F'||_1 stalls at a few 1e-3 of ||F||_1 while those
 *   modes, which R nearly annihilates, leave the flow and the bodies
 *   unchanged; the spread norm does not see them. */
typedef enum { IBM_FSI_CRIT_LAGRANGIAN = 0, IBM_FSI_CRIT_EULERIAN = 1 } ibm_fsi_criterion;

typedef struct {
  double gravity[3];   /* acceleration of gravity g (the paper's -Fr^-2 e_z);
                          the body feels (theta - 1)/theta g               */
  double xi;           /* relaxation of the corrections (0.6 .. 1.1)        */
  double tol;          /* stop when the ratio of the criterion < tol
                          (Eq. (convergence_criterion); 1e-3)              */
  int32_t max_inner;   /* correction limit per step                        */
  int32_t criterion;   /* ibm_fsi_criterion                                */
} ibm_fsi_opts;

typedef struct {
  int32_t inner;          /* corrections taken                             */
  int32_t fgmres_iters;   /* FGMRES iterations, summed over the corrections */
  double ratio;           /* last ratio of the stopping test (criterion)    */
  int32_t helm_iters;     /* predictor outer iterations                     */
  double helm_relres;
} ibm_fsi_stats;

/* Defaults: no gravity, xi 1, tol 1e-3, max_inner 50, Lagrangian criterion. */
void ibm_default_fsi_opts(ibm_fsi_opts* fopts);

/* One two-way coupled step (Sec. 3.2.1), scalar C mode:
 *   Step 1: each sphere's centre by (4 x^n - x^{n-1})/3 + (2/3) dt u_s^n and
 *     orientation R^{n+1} = R^n R_Delta (Rodrigues, Adams-Bashforth angle);
 *     markers X_k = x_c^{n+1} + R^{n+1} L0_k, written to X_np1 and set on
 *     the context (as ibm_set_markers);
 *   Step 2: the predictor of Eq. (ustar_two_way) (as ibm_step);
 *   Step 3: corrections k = 0, 1, ... : u_s, omega_s from Newton's laws with
 *     the IB force/torque of F^{(n,k)} and the enclosed-fluid momentum of
 *     Eq. (volume_integrals) (volume fractions from the signed distance at
 *     the corners of each face's control volume); U = u_s + omega x (X - x_c);
 *     the Schur solve of Eq. (pressure_force_iterative_system); relaxed
 *     updates p += xi p', F += xi F', u += xi (2dt/3)(-G p' + R F'); until
 *     ||F'||_1/||F||_1 < tol (||R F'||_1/||R F||_1 with the Eulerian
 *     criterion) or max_inner corrections.
 * bodies: host [n_bodies], advanced to t^{n+1} on success (left unchanged on
 * error).  L0: device [3][n_markers] body-frame offsets (X - x_c at R = I);
 * body_id: device int32 [n_markers] in [0, n_bodies).  u_n, u_nm1 (faces),
 * p_n (cells), F_n ([3][n_markers]), f_body (faces, may be NULL): device
 * inputs; X_np1, u_np1, p_np1, F_np1: device outputs, not aliasing inputs.
 * IBM_ERR_NOT_CONVERGED when max_inner is reached above tol (outputs and
 * bodies still advanced).  Synchronises. */
ibm_status ibm_fsi_step(ibm_ctx* ctx, int32_t n_bodies, ibm_rigid_sphere* bodies,
                        int64_t n_markers, const double* L0, const int32_t* body_id,
                        const double* u_n, const double* u_nm1, const double* p_n,
                        const double* F_n, const double* f_body, double* X_np1,
                        double* u_np1, double* p_np1, double* F_np1,
                        const ibm_solve_opts* opts, const ibm_fsi_opts* fopts,
                        ibm_fsi_stats* stats);

/* ---- Adjoint of one step ------------------------------------------------
 * The paper differentiates nothing; these calls give the exact derivative of
 * the one-way step above (scalar C mode, Eqs. (ustar)-(ApproxSchurPrimalF),
 * (u_n_plus_1)) so that gradients of the hydrodynamic force and torque on a
 * body can be taken with respect to the prescribed marker velocities U^Gamma
 * and the marker positions X.  With a = 3/(2 dt) and F_bar = dJ/dF^{n+1}:
 *   lambda = S~^+ (2 B^T F_bar)      (S~ symmetric: the transposed solve)
 *   U_bar  = 2a (F_bar - B lambda)
 *   X_bar  = (R F' - a u^{n+1})^T dR (U_bar / a) - (G lambda)^T dR F'
 *            + mu^T dR F^n,   H mu = a G lambda - R U_bar
 * where dR is the derivative of R's entries (products of Eq. (delta)'s phi)
 * with respect to each marker's own coordinates, H the predictor operator of
 * Eq. (ustar) and F' = F^{n+1} - F^n.  The mu term needs one predictor solve
 * and is skipped when F^n is zero.  */

/* Adjoint of ibm_step.  Inputs are the markers last set (the same as for the
 * forward step), the forward step's u^{n+1} (device packed faces), F^n and
 * F^{n+1} (device [3][n_markers]; F_n may be NULL for F^n = 0) and
 * F_bar = dJ/dF^{n+1} (device [3][n_markers]).  Outputs: U_bar = dJ/dU^Gamma
 * and X_bar = the part of dJ/dX that flows through R (both device
 * [3][n_markers], overwritten; a loss that also depends on X directly, like a
 * torque's lever arm, adds its own part, see ibm_body_forces_adjoint).  The
 * forward step must have run in scalar C mode (other modes: IBM_ERR_ARG)
 * with the same opts; the
 * adjoint solve uses opts (precond_prec, rtol, ...), and stats receives its
 * iteration count and true residual (helm_* for the mu solve).  Uses the
 * context's workspace: not concurrent with other calls on the same context.
 * Returns IBM_ERR_NOT_CONVERGED if the adjoint solve missed rtol (outputs
 * still written).  Synchronises. */
ibm_status ibm_adjoint_step(ibm_ctx* ctx, const double* u_np1, const double* F_n,
                            const double* F_np1, const double* F_bar, double* U_bar,
                            double* X_bar, const ibm_solve_opts* opts,
                            ibm_solve_stats* stats);

/* Adjoint of ibm_body_forces for J = sum_b w_b . out_b (w host
 * [n_bodies][6], weights on [force | torque]; out host [n_bodies][6] = the
 * forward result).  Writes F_bar = dJ/dF (device [3][n_markers]:
 * h^3 (w_F + w_T x (X_k - c_b))), X_bar_lever = dJ/dX through the lever arms
 * (device [3][n_markers]: h^3 F_k x w_T; may be NULL) and centers_bar
 * (host [n_bodies][3]: -force_b x w_T, from out).  Markers whose body_id is
 * outside [0, n_bodies) get zeros.  Synchronises. */
ibm_status ibm_body_forces_adjoint(ibm_ctx* ctx, const double* F, const double* X,
                                   const int32_t* body_id, int32_t n_bodies,
                                   const double* centers, const double* w, const double* out,
                                   double* F_bar, double* X_bar_lever, double* centers_bar);

/* Optional timing of kernel classes with CUDA events recorded on the
 * context's stream around the launches of each class (no effect on results).
 * ibm_profile_enable(ctx, 1) resets the counters and starts recording;
 * ibm_profile_read synchronises the stream and returns, per class, the summed
 * event-measured milliseconds and the number of timed launches. */
enum {
  IBM_PROF_LAPLACIAN_F64 = 0,  /* 7-point Laplacian inside S~ v (FP64, or
                                  double-single in the mixed Arnoldi)       */
  IBM_PROF_SCHUR_MARKERS = 1,  /* B v gather + B^T t shell gather in S~ v   */
  IBM_PROF_VCYCLE = 2,         /* one whole V-cycle (all levels)            */
  IBM_PROF_MULTIDOT = 3,       /* Gram-Schmidt multi-dot (+ final reduce)   */
  IBM_PROF_AXPY_NORM = 4,      /* Gram-Schmidt axpy + norm + normalisation  */
  IBM_PROF_PREDICTOR = 5,      /* whole predictor (Helmholtz) solve         */
  IBM_PROF_SOLVE = 6,          /* whole ibm_solve_schur / step solve        */
  IBM_PROF_STEP = 7,           /* whole ibm_step                            */
  IBM_PROF_MARKER_BUILD = 8,   /* ibm_set_markers                           */
  IBM_PROF_MG_SMOOTH_FINE = 9, /* one finest-level smoothing sweep kernel   */
  IBM_PROF_HELM_SWEEP = 10,    /* one inner FP32 Chebyshev step of the
                                  predictor (middle steps only)             */
  IBM_PROF_ADJOINT = 11,       /* whole ibm_adjoint_step                    */
  IBM_PROF_FSI = 12,           /* whole ibm_fsi_step                        */
  IBM_PROF_NCLASS = 16
};
typedef struct {
  double ms[IBM_PROF_NCLASS];
  int64_t launches[IBM_PROF_NCLASS];
  double bytes[IBM_PROF_NCLASS];   /* algorithmic DRAM bytes of the timed
                                      kernels (every array read or written
                                      once; 0 where not counted)            */
} ibm_profile;

ibm_status ibm_profile_enable(ibm_ctx* ctx, int32_t on);
/* Number of kernels this library has launched in the process so far (all
 * contexts); a difference of two reads counts the launches in between. */
int64_t ibm_kernel_launches(void);
ibm_status ibm_profile_read(ibm_ctx* ctx, ibm_profile* out);

#ifdef __cplusplus
}
#endif

#endif /* IBM_SCHUR_H */
