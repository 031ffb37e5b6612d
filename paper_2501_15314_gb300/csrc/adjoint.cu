// Adjoint of one one-way step (scalar C mode) and of the body force / torque
// sums, for gradients of the hydrodynamic load on a body with respect to the
// prescribed marker velocities and the marker positions.
//
// The step (Sec. 3.1; a = 3/(2 dt)) is
//   H u*  = rhs(u^n, u^{n-1}, p^n, f) + R F^n                   Eq. (ustar)
//   RHS_p = a G^T u*,  RHS_F = a (R^T u* - U^Gamma)             below Eq. (Saddle)
//   S~ p' = RHS_p + 2 G^T R RHS_F,  S~ = L + 2 B^T B            Eqs. (tildeSp), (ApproxSchurPrimalP)
//   F'    = 2 (B p' - RHS_F),  B = R^T G                        Eq. (ApproxSchurPrimalF)
//   u^{n+1} = u* + (1/a)(-G p' + R F')                          Eq. (u_n_plus_1)
// Running it backwards from F_bar = dJ/dF^{n+1}: S~ and H are symmetric and
// p' is the mean-zero solution, so one transposed solve
// lambda = S~^+ (2 B^T F_bar) gives U_bar = 2a (F_bar - B lambda).  Each use
// of R contributes f^T dR m for a face field f and a marker field m; after
// substituting the update equation the contributions collapse to three pairs:
//   (R F' - a u^{n+1}, U_bar / a),  (G lambda, -F'),  (mu, F^n)
// with H mu = a G lambda - R U_bar.  The position derivative of R is
// k_interp_dpos (markers.cu), built from phi' of Eq. (delta).
#include "ibm_internal.cuh"

namespace ibm {

namespace {

constexpr int TPB = 256;

// F_bar = h^3 (w_F + w_T x r), X_bar = h^3 F x w_T for the marker's body;
// wc holds per body [w_F(3) | w_T(3) | centre(3)].
__global__ void k_body_forces_adjoint(const double* __restrict__ F, const double* __restrict__ X,
                                      const int32_t* __restrict__ bid, int64_t n, int nb,
                                      const double* __restrict__ wc, double h3,
                                      double* __restrict__ F_bar, double* __restrict__ X_bar) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int b = bid[k];
  double fb[3] = {0.0, 0.0, 0.0}, xb[3] = {0.0, 0.0, 0.0};
  if (b >= 0 && b < nb) {
    const double* q = wc + 9 * b;
    const double wx = q[3], wy = q[4], wz = q[5];
    const double rx = X[k] - q[6], ry = X[n + k] - q[7], rz = X[2 * n + k] - q[8];
    fb[0] = h3 * (q[0] + (wy * rz - wz * ry));
    fb[1] = h3 * (q[1] + (wz * rx - wx * rz));
    fb[2] = h3 * (q[2] + (wx * ry - wy * rx));
    const double fx = F[k], fy = F[n + k], fz = F[2 * n + k];
    xb[0] = h3 * (fy * wz - fz * wy);
    xb[1] = h3 * (fz * wx - fx * wz);
    xb[2] = h3 * (fx * wy - fy * wx);
  }
  for (int e = 0; e < 3; ++e) {
    F_bar[e * n + k] = fb[e];
    if (X_bar) X_bar[e * n + k] = xb[e];
  }
}

}  // namespace

}  // namespace ibm

using namespace ibm;

extern "C" {

ibm_status ibm_adjoint_step(ibm_ctx* c, const double* u_np1, const double* F_n,
                            const double* F_np1, const double* F_bar, double* U_bar,
                            double* X_bar, const ibm_solve_opts* o, ibm_solve_stats* st) {
  if (check_ctx(c) != IBM_OK) return IBM_ERR_ARG;
  const int64_t n = c->mk.n;
  if (bad_ptr(u_np1)) return set_err(c, IBM_ERR_ARG, "bad u_np1");
  if (n > 0 && (bad_ptr(F_np1) || bad_ptr(F_bar) || bad_ptr(U_bar) || bad_ptr(X_bar) ||
                (F_n && bad_ptr(F_n))))
    return set_err(c, IBM_ERR_ARG, "bad marker pointer");
  if (n > 0 && (U_bar == X_bar || U_bar == F_bar || X_bar == F_bar || U_bar == F_np1 ||
                X_bar == F_np1 || (F_n && (U_bar == F_n || X_bar == F_n))))
    return set_err(c, IBM_ERR_ARG, "outputs must not alias inputs");
  ibm_status s = check_opts(c, o);
  if (s != IBM_OK) return s;
  if (o->c_mode != IBM_CMODE_SCALAR)
    return set_err(c, IBM_ERR_ARG, "the adjoint covers the scalar C mode only");
  if ((s = ensure_krylov(c, o->restart)) != IBM_OK) return s;
  set_cmode(c, o);
  ibm_solve_stats local;
  if (!st) st = &local;
  memset(st, 0, sizeof(*st));
  if (n == 0) return IBM_OK;   // no markers: J does not depend on U or X
  const int ph = prof_begin(c, IBM_PROF_ADJOINT);
  cudaStream_t str = c->stream;
  MarkerData& mk = c->mk;
  const double a = 1.5 / c->dt;
  const double inv_h = 1.0 / c->h;

  // lambda = S~^+ (2 B^T F_bar): the transposed (= same) Schur solve
  launch_zero(c->c2, sizeof(double) * c->m, str);
  launch_shell_gradt_spread(c, F_bar, 2.0, c->c2);
  double* lam = c->c3;
  launch_zero(lam, sizeof(double) * c->m, str);
  IBM_LAUNCH_CHECK(c);
  s = fgmres_solve(c, c->c2, lam, o, st, true);
  if (s != IBM_OK && s != IBM_ERR_NOT_CONVERGED) { prof_end(c, ph); return s; }
  const ibm_status solve_status = s;

  // U_bar = 2a (F_bar - B lambda)
  launch_marker_grad_interp(c, lam, 1.0, mk.t2);
  launch_axpby(F_bar, 2.0 * a, mk.t2, -2.0 * a, U_bar, 3 * n, str);
  // F' = F^{n+1} - F^n
  if (F_n)
    launch_axpby(F_np1, 1.0, F_n, -1.0, mk.t, 3 * n, str);
  else
    launch_copy(mk.t, F_np1, sizeof(double) * 3 * n, str);

  // X_bar = (R F' - a u^{n+1})^T dR (U_bar / a)
  launch_axpby(u_np1, -a, u_np1, 0.0, c->f1, c->nf, str);
  launch_shell_spread_faces(c, mk.t, 1.0, c->f1);
  launch_interp_dpos(c, c->f1, U_bar, 1.0 / a, false, X_bar);
  //        - (G lambda)^T dR F'
  launch_gradient(c->d, lam, c->f2, inv_h, str);
  launch_interp_dpos(c, c->f2, mk.t, -1.0, true, X_bar);
  IBM_LAUNCH_CHECK(c);

  //        + mu^T dR F^n,  H mu = a G lambda - R U_bar
  double fn2 = 0.0;
  if (F_n && (s = norm2_host(c, F_n, 3 * n, &fn2)) != IBM_OK) { prof_end(c, ph); return s; }
  if (fn2 > 0.0) {
    launch_axpby(c->f2, a, c->f2, 0.0, c->f1, c->nf, str);
    launch_shell_spread_faces(c, U_bar, -1.0, c->f1);
    IBM_LAUNCH_CHECK(c);
    s = helmholtz_solve(c, c->f1, c->f2, o, &st->helm_iters, &st->helm_relres);
    if (s != IBM_OK) { prof_end(c, ph); return s; }
    launch_interp_dpos(c, c->f2, F_n, 1.0, true, X_bar);
    IBM_LAUNCH_CHECK(c);
  }
  prof_end(c, ph);
  IBM_CUDA(c, cudaStreamSynchronize(str));
  return solve_status;
}

ibm_status ibm_body_forces_adjoint(ibm_ctx* c, const double* F, const double* X,
                                   const int32_t* body_id, int32_t n_bodies,
                                   const double* centers, const double* w, const double* out,
                                   double* F_bar, double* X_bar_lever, double* centers_bar) {
  if (check_ctx(c) != IBM_OK) return IBM_ERR_ARG;
  const int64_t n = c->mk.n;
  if (n_bodies < 1 || n_bodies > 4096 || !centers || !w || !out || !centers_bar)
    return set_err(c, IBM_ERR_ARG, "bad body arguments");
  if (n > 0 && (bad_ptr(F) || bad_ptr(X) || body_id == nullptr || bad_ptr(F_bar) ||
                (X_bar_lever && bad_ptr(X_bar_lever))))
    return set_err(c, IBM_ERR_ARG, "bad marker pointers");
  // d/dc_b of w_T . h^3 sum (X_k - c_b) x F_k = -(h^3 sum F_k) x w_T
  for (int b = 0; b < n_bodies; ++b) {
    const double* f = out + 6 * b;
    const double* wt = w + 6 * b + 3;
    centers_bar[3 * b + 0] = -(f[1] * wt[2] - f[2] * wt[1]);
    centers_bar[3 * b + 1] = -(f[2] * wt[0] - f[0] * wt[2]);
    centers_bar[3 * b + 2] = -(f[0] * wt[1] - f[1] * wt[0]);
  }
  if (n == 0) return IBM_OK;
  // per body [w_F | w_T | centre] staged in the reduction scratch
  // (9 * 4096 doubles fit in kRedBlocks * (kMaxRestart + 2))
  std::vector<double> wc((size_t)9 * n_bodies);
  for (int b = 0; b < n_bodies; ++b) {
    for (int q = 0; q < 6; ++q) wc[9 * b + q] = w[6 * b + q];
    for (int q = 0; q < 3; ++q) wc[9 * b + 6 + q] = centers[3 * b + q];
  }
  double* dwc = c->red_part;
  IBM_CUDA(c, cudaMemcpyAsync(dwc, wc.data(), sizeof(double) * wc.size(), cudaMemcpyHostToDevice,
                              c->stream));
  count_launch();
  k_body_forces_adjoint<<<div_up(n, TPB), TPB, 0, c->stream>>>(
      F, X, body_id, n, n_bodies, dwc, c->h * c->h * c->h, F_bar, X_bar_lever);
  IBM_LAUNCH_CHECK(c);
  IBM_CUDA(c, cudaStreamSynchronize(c->stream));
  return IBM_OK;
}

}  // extern "C"
