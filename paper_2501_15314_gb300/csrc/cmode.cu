// C^{-1} with C = R^T R, the (2,2) block of Eq. (Saddle), for the exact
// primal Schur complement S_p = L + B^T C^{-1} B (Eqs. (SchurPrimal)-
// (SchurPrimalF)) and the sign-consistent form L - B^T C^{-1} B.
//
// Conjugate gradients on C (symmetric positive definite when the markers'
// weight vectors are independent), matrix-free: C v = R^T (R v) spreads v onto
// the shell faces (written, not accumulated, so the rest of the face scratch is
// never read) and interpolates back.  The CG scalars live on the device (no
// host round trip per iteration); the host reads the residual every kCheck
// iterations.  C's diagonal is the same for every marker ((sum phi^2)^3 =
// 1/8 when no tap is cut off), so Jacobi scaling would not change anything.
// Its condition number grows quickly with the marker density (about 5e2 at
// Lagrangian spacing h, 2e5 at h / 1.38 for a sphere of radius 0.3 on 32^3),
// which is why the paper uses C^{-1} ~ 2 I in production.
#include "ibm_internal.cuh"

#include <cmath>

namespace ibm {

namespace {

constexpr int TPB = 256;
constexpr int kCheck = 4;

__global__ void k_cg_alpha(const double* __restrict__ rr, const double* __restrict__ pq,
                           double* __restrict__ alpha) {
  alpha[0] = pq[0] != 0.0 ? rr[0] / pq[0] : 0.0;
}

// s += alpha p, r -= alpha q
__global__ void k_cg_update(int64_t n, const double* __restrict__ alpha,
                            const double* __restrict__ p, const double* __restrict__ q,
                            double* __restrict__ s, double* __restrict__ r) {
  const double a = alpha[0];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    s[i] = fma(a, p[i], s[i]);
    r[i] = fma(-a, q[i], r[i]);
  }
}

// p = r + (rr_new / rr) p
__global__ void k_cg_direction(int64_t n, const double* __restrict__ rr,
                               const double* __restrict__ rr_new, const double* __restrict__ r,
                               double* __restrict__ p) {
  const double beta = rr[0] > 0.0 ? rr_new[0] / rr[0] : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = fma(beta, p[i], r[i]);
}

__global__ void k_copy_scalar(const double* __restrict__ a, double* __restrict__ b) { b[0] = a[0]; }

int small_grid(int64_t n) {
  const int64_t b = div_up(n, TPB);
  return (int)(b < 1216 ? (b < 1 ? 1 : b) : 1216);
}

}  // namespace

void apply_C(ibm_ctx* c, const double* v, double* out) {
  launch_shell_spread_faces_set(c, v, c->f4);
  launch_interp(c, c->f4, out);
}

ibm_status c_solve(ibm_ctx* c, const double* t, double* s, double rtol, int maxit,
                   int* iters_out) {
  MarkerData& mk = c->mk;
  const int64_t n = 3 * mk.n;
  cudaStream_t str = c->stream;
  if (iters_out) *iters_out = 0;
  if (n == 0) return IBM_OK;
  if (!c->cg_scal) {
    if (cudaMalloc(&c->cg_scal, sizeof(double) * 8) != cudaSuccess) {
      cudaGetLastError();
      return set_err(c, IBM_ERR_NOMEM, "CG scalar allocation failed");
    }
  }
  double* r = mk.cg;
  double* p = mk.cg + n;
  double* q = mk.cg + 2 * n;
  double* sc = c->cg_scal;   // [0] rr, [1] <p, q>, [2] alpha, [3] rr_new
  launch_zero(s, sizeof(double) * n, str);
  launch_copy(r, t, sizeof(double) * n, str);
  launch_copy(p, t, sizeof(double) * n, str);
  launch_dot(t, t, n, c->red_part, sc, str, c->host_red_dev);
  IBM_LAUNCH_CHECK(c);
  IBM_CUDA(c, cudaStreamSynchronize(str));
  const double tt = c->host_red[0];
  if (!std::isfinite(tt)) return set_err(c, IBM_ERR_NAN, "non-finite right-hand side of C s = t");
  if (tt == 0.0) return IBM_OK;
  const double target = rtol * rtol * tt;
  const int g = small_grid(n);
  int it = 0;
  double rr = tt;
  while (it < maxit) {
    apply_C(c, p, q);
    launch_dot(p, q, n, c->red_part, sc + 1, str);
    count_launch();
    k_cg_alpha<<<1, 1, 0, str>>>(sc, sc + 1, sc + 2);
    count_launch();
    k_cg_update<<<g, TPB, 0, str>>>(n, sc + 2, p, q, s, r);
    launch_dot(r, r, n, c->red_part, sc + 3, str);
    count_launch();
    k_cg_direction<<<g, TPB, 0, str>>>(n, sc, sc + 3, r, p);
    count_launch();
    k_copy_scalar<<<1, 1, 0, str>>>(sc + 3, sc);
    ++it;
    if (it % kCheck == 0 || it == maxit) {
      launch_to_host(sc, c->host_red_dev, sizeof(double), str);
      IBM_LAUNCH_CHECK(c);
      IBM_CUDA(c, cudaStreamSynchronize(str));
      rr = c->host_red[0];
      if (!std::isfinite(rr)) return set_err(c, IBM_ERR_NAN, "non-finite CG residual on C");
      if (rr <= target) break;
    }
  }
  if (iters_out) *iters_out = it;
  c->c_iters += it;
  if (rr > target) {
    char buf[160];
    snprintf(buf, sizeof buf, "CG on C = R^T R did not reach c_rtol %.3g in %d iterations (%.3g)",
             rtol, maxit, std::sqrt(rr / tt));
    return set_err(c, IBM_ERR_NOT_CONVERGED, buf);
  }
  return IBM_OK;
}

}  // namespace ibm

using namespace ibm;

extern "C" {

ibm_status ibm_apply_c_inverse(ibm_ctx* c, const double* t, double* s, double c_rtol,
                               int32_t c_maxit, int32_t* iters) {
  if (check_ctx(c) != IBM_OK) return IBM_ERR_ARG;
  const int64_t n = c->mk.n;
  if (n > 0 && (bad_ptr(t) || bad_ptr(s) || t == s))
    return set_err(c, IBM_ERR_ARG, "bad t/s");
  if (!(c_rtol > 0.0) || c_maxit < 1) return set_err(c, IBM_ERR_ARG, "need c_rtol > 0, c_maxit >= 1");
  int it = 0;
  const ibm_status st = c_solve(c, t, s, c_rtol, c_maxit, &it);
  if (iters) *iters = it;
  return st;
}

}  // extern "C"
