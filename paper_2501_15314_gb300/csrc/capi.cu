// C ABI of libibmschur (include/ibm_schur.h): context lifetime, argument
// validation, and the one-way SIMPLE-IBM time step of Sec. 3.1 composed from
// the stencil, marker, multigrid and Krylov kernels.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <new>

#include "ibm_internal.cuh"

namespace ibm {

ibm_status set_err(ibm_ctx* c, ibm_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

ibm_status cuda_err(ibm_ctx* c, cudaError_t e, const char* where) {
  char buf[256];
  snprintf(buf, sizeof buf, "CUDA error %s (%d) at %s", cudaGetErrorString(e), (int)e, where);
  return set_err(c, e == cudaErrorMemoryAllocation ? IBM_ERR_NOMEM : IBM_ERR_CUDA, buf);
}

static std::atomic<long long> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void add_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int prof_begin(ibm_ctx* c, int cls) {
  if (!c->prof_on) return -1;
  if (c->prof_used == c->prof.size()) {
    ibm_ctx::ProfRec r;
    r.cls = cls;
    if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) {
      cudaGetLastError();
      return -1;
    }
    c->prof.push_back(r);
  }
  const int h = (int)c->prof_used++;
  c->prof[h].cls = cls;
  cudaEventRecord(c->prof[h].a, c->stream);
  return h;
}

void prof_end(ibm_ctx* c, int h, double bytes) {
  if (h < 0) return;
  c->prof[h].bytes = bytes;
  c->prof_acc += bytes;
  cudaEventRecord(c->prof[h].b, c->stream);
}

void prof_note(ibm_ctx* c, double bytes) {
  if (c->prof_on) c->prof_acc += bytes;
}

double prof_mark(const ibm_ctx* c) { return c->prof_acc; }

void prof_end_span(ibm_ctx* c, int h, double mark) {
  if (h < 0) return;
  c->prof[h].bytes = c->prof_acc - mark;
  cudaEventRecord(c->prof[h].b, c->stream);
}

void prof_end_or_note(ibm_ctx* c, int h, double bytes) {
  if (h >= 0) prof_end(c, h, bytes);
  else prof_note(c, bytes);
}

namespace {

constexpr int TPB = 256;

// Per body b (block b): out[6b..6b+2] = h^3 sum_{k in b} F_k and
// out[6b+3..6b+5] = h^3 sum_{k in b} (X_k - c_b) x F_k (Eq. (IBM_force)),
// c_b = cen[3b..3b+2].  Each block scans every marker and keeps its body's;
// a fixed-order block reduction makes the sums reproducible.
__global__ void __launch_bounds__(TPB) k_body_sums(const double* __restrict__ F,
                                                   const double* __restrict__ X,
                                                   const int32_t* __restrict__ bid, int64_t n,
                                                   const double* __restrict__ cen, double h3,
                                                   double* __restrict__ out) {
  const int body = blockIdx.x;
  const double cx = cen[3 * body], cy = cen[3 * body + 1], cz = cen[3 * body + 2];
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t k = threadIdx.x; k < n; k += blockDim.x) {
    if (bid[k] != body) continue;
    const double fx = F[k], fy = F[n + k], fz = F[2 * n + k];
    const double rx = X[k] - cx, ry = X[n + k] - cy, rz = X[2 * n + k] - cz;
    acc[0] += fx; acc[1] += fy; acc[2] += fz;
    acc[3] += ry * fz - rz * fy;
    acc[4] += rz * fx - rx * fz;
    acc[5] += rx * fy - ry * fx;
  }
  __shared__ double sh[6][TPB];
  for (int q = 0; q < 6; ++q) sh[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int s = TPB / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
      for (int q = 0; q < 6; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < 6) out[6 * body + threadIdx.x] = h3 * sh[threadIdx.x][0];
}

__global__ void k_axpby_small(const double* __restrict__ x, double a, const double* __restrict__ y,
                              double b, double* __restrict__ out, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = a * x[i] + b * y[i];
}

}  // namespace

bool bad_ptr(const void* p) { return p == nullptr || (reinterpret_cast<uintptr_t>(p) & 7) != 0; }

void launch_body_sums(const double* F, const double* X, const int32_t* bid, int64_t n,
                      int n_bodies, const double* cen, double h3, double* out, cudaStream_t s) {
  count_launch();
  k_body_sums<<<n_bodies, TPB, 0, s>>>(F, X, bid, n, cen, h3, out);
}

ibm_status check_ctx(ibm_ctx* c) {
  if (!c) return IBM_ERR_ARG;
  c->err.clear();
  return IBM_OK;
}

ibm_status check_opts(ibm_ctx* c, const ibm_solve_opts* o) {
  if (!o) return set_err(c, IBM_ERR_ARG, "opts is null");
  if (o->precond_prec != IBM_PREC_FP32 && o->precond_prec != IBM_PREC_FP64)
    return set_err(c, IBM_ERR_ARG, "precond_prec must be IBM_PREC_FP32 or IBM_PREC_FP64");
  if (!(o->rtol > 0.0) || o->maxit < 1 || o->restart < 1 || o->restart > kMaxRestart)
    return set_err(c, IBM_ERR_ARG, "need rtol > 0, maxit >= 1, 1 <= restart <= 64");
  if (o->mg_pre < 0 || o->mg_pre > 4 || o->mg_post < 0 || o->mg_post > 4 ||
      o->mg_pre + o->mg_post == 0)
    return set_err(c, IBM_ERR_ARG, "mg_pre, mg_post in 0..4, not both 0");
  if (!(o->helm_rtol > 0.0) || o->helm_maxit < 1)
    return set_err(c, IBM_ERR_ARG, "need helm_rtol > 0 and helm_maxit >= 1");
  if (o->arnoldi != IBM_ARNOLDI_FP64 && o->arnoldi != IBM_ARNOLDI_DS &&
      o->arnoldi != IBM_ARNOLDI_FP32)
    return set_err(c, IBM_ERR_ARG, "arnoldi must be IBM_ARNOLDI_FP64, _DS or _FP32");
  if (o->c_mode != IBM_CMODE_SCALAR && o->c_mode != IBM_CMODE_EXACT &&
      o->c_mode != IBM_CMODE_CONSISTENT)
    return set_err(c, IBM_ERR_ARG, "c_mode must be IBM_CMODE_SCALAR, _EXACT or _CONSISTENT");
  if (o->c_mode != IBM_CMODE_SCALAR && (!(o->c_rtol > 0.0) || o->c_maxit < 1))
    return set_err(c, IBM_ERR_ARG, "need c_rtol > 0 and c_maxit >= 1");
  if (o->cycle_graphs != 0 && o->cycle_graphs != 1)
    return set_err(c, IBM_ERR_ARG, "cycle_graphs must be 0 or 1");
  return IBM_OK;
}

void set_cmode(ibm_ctx* c, const ibm_solve_opts* o) {
  c->cmode = o ? o->c_mode : IBM_CMODE_SCALAR;
  c->c_rtol = o ? o->c_rtol : 1e-14;
  c->c_maxit = o ? o->c_maxit : 500;
  c->c_iters = 0;
}

ibm_status ensure_krylov(ibm_ctx* c, int restart) {
  if (restart <= c->restart_cap) return IBM_OK;
  cudaFree(c->V);
  cudaFree(c->Z);
  c->V = c->Z = nullptr;
  c->restart_cap = 0;
  if (cudaMalloc(&c->V, sizeof(double) * (restart + 1) * c->m) != cudaSuccess ||
      cudaMalloc(&c->Z, sizeof(double) * restart * c->m) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(c->V);
    cudaFree(c->Z);
    c->V = c->Z = nullptr;
    return set_err(c, IBM_ERR_NOMEM, "Krylov basis allocation failed");
  }
  c->restart_cap = restart;
  return IBM_OK;
}

ibm_status norm2_host(ibm_ctx* c, const double* x, int64_t n, double* out) {
  launch_dot(x, x, n, c->red_part, c->red_out + 7 * (kMaxRestart + 2), c->stream,
             c->host_red_dev);
  IBM_LAUNCH_CHECK(c);
  IBM_CUDA(c, cudaStreamSynchronize(c->stream));
  *out = std::sqrt(c->host_red[0]);
  return IBM_OK;
}

ibm_status norm2_lead_host(ibm_ctx* c, const double* x, int64_t n, double* out) {
  launch_norm2_lead(x, n, c->red_part, c->red_out + 7 * (kMaxRestart + 2), c->stream,
                    c->host_red_dev);
  IBM_LAUNCH_CHECK(c);
  IBM_CUDA(c, cudaStreamSynchronize(c->stream));
  *out = std::sqrt(c->host_red[0]);
  if (std::isfinite(*out)) return IBM_OK;
  return norm2_host(c, x, n, out);   // values out of the leading parts' range
}

static void free_all(ibm_ctx* c) {
  cudaFree(c->cell_count); cudaFree(c->cell_start); cudaFree(c->cell_flag); cudaFree(c->scan_tmp);
  cudaFree(c->dev_flag); cudaFreeHost(c->host_flag);
  cudaFree(c->c1); cudaFree(c->c2); cudaFree(c->c3);
  cudaFree(c->f1); cudaFree(c->f2); cudaFree(c->f3); cudaFree(c->f4);
  cudaFree(c->g1); cudaFree(c->g2); cudaFree(c->g3); cudaFree(c->g4); cudaFree(c->g5); cudaFree(c->g6);
  cudaFree(c->red_part); cudaFree(c->red_out); cudaFreeHost(c->host_red); cudaFree(c->helm_part);
  cudaFree(c->V); cudaFree(c->Z);
  for (int l = 0; l < c->n_levels; ++l) {
    MGLevel& L = c->lv[l];
    cudaFree(L.x32); cudaFree(L.b32); cudaFree(L.t32);
    cudaFree(L.x64); cudaFree(L.b64); cudaFree(L.t64);
  }
  cudaFree(c->coarse_pinv64); cudaFree(c->coarse_pinv32); cudaFree(c->chain_tab);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  for (cudaEvent_t& e : c->ev_iter)
    if (e) cudaEventDestroy(e);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->cyc_exec) cudaGraphExecDestroy(c->cyc_exec);
  if (c->cyc_graph) cudaGraphDestroy(c->cyc_graph);
  if (c->cap) cudaStreamDestroy(c->cap);
  cudaFree(c->gstate); cudaFreeHost(c->host_gstate);
  MarkerData& m = c->mk;
  cudaFree(m.bf); cudaFree(m.bc); cudaFree(m.org); cudaFree(m.wf); cudaFree(m.wc); cudaFree(m.cw);
  cudaFree(m.t); cudaFree(m.t2); cudaFree(m.t32); cudaFree(m.dwf); cudaFree(m.dwc);
  cudaFree(m.wc32); cudaFree(m.cw32);
  cudaFree(m.cg);
  cudaFree(m.t3); cudaFree(c->cg_scal);
  cudaFree(m.entry_key); cudaFree(m.shell_cell); cudaFree(m.shell_off); cudaFree(m.ell_cell);
  cudaFree(m.ell_base); cudaFree(m.ell_len); cudaFree(m.ell_key); cudaFree(m.ell_coef);
  cudaFree(m.ell_coef32); cudaFree(m.ell_sw); cudaFree(m.ell_any);
  for (auto& r : c->prof) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  c->prof.clear();
}

// Predictor of Eq. (ustar): (a - nu Lap) u = rhs by defect correction.  Each
// correction solves A e = r^ with K FP32 Chebyshev steps on the exact
// spectral bounds [a, a + 12 nu / h^2] of A, where r^ = r / ||r|| is held in
// double-single (FP32 pair) arithmetic, and adds ||r|| e to the FP64 iterate;
// K is chosen for the reduction still needed (at most 1e-6 per correction,
// the FP32 limit).  The next residual is ||r|| (r^ - A e), formed in
// double-single on the FP32 pipes (k_helm_resid_ds) together with its norm:
// no FP64 residual pass, and the residual is as accurate as an FP64 one
// (about 2^-46 relative to the previous residual, plus the rounding of the
// FP64 iterate).
ibm_status helmholtz_solve(ibm_ctx* c, const double* rhs, double* u, const ibm_solve_opts* o,
                           int* iters, double* relres) {
  cudaStream_t s = c->stream;
  const int64_t nf = c->nf;
  const double a = 1.5 / c->dt;
  const double nu = 1.0 / c->Re;
  const double nu_h2 = nu / (c->h * c->h);
  const double lmin = a, lmax = a + 12.0 * nu_h2;
  const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin);
  const double sigma = theta / delta;
  double rnorm0;
  // the norm is the baseline of the stopping test only: the corrections
  // scale by the norms their own residual recursion carries
  ibm_status st = norm2_lead_host(c, rhs, nf, &rnorm0);
  if (st != IBM_OK) return st;
  if (!std::isfinite(rnorm0)) return set_err(c, IBM_ERR_NAN, "non-finite predictor RHS");
  *iters = 0;
  *relres = 0.0;
  if (rnorm0 == 0.0) {
    launch_zero(u, sizeof(double) * nf, s);
    return IBM_OK;
  }
  double* sdev = c->red_out + 7 * (kMaxRestart + 2) + 8;
  float* eK = nullptr;        // the last correction e (input of the next residual)
  double rn = rnorm0;         // ||r|| of the current residual
  double qn = rnorm0;         // norm of the stored (unnormalised) residual pair
  // The first correction stays in FP32 (g6, scale pend_s) until the last
  // step of the second writes u = pend_s e_1 + rn e_2 in one pass (the same
  // products and roundings as adding them one after the other); a later
  // correction adds into u.  When the first one is the only one, a flush
  // writes u.
  const float* pend = nullptr;
  double pend_s = 0.0;
  auto flush = [&]() {
    if (pend) launch_helm_flush(c->d, pend, pend_s, u, s);
    pend = nullptr;
  };
  for (int it = 0;; ++it) {
    if (it > 0) {
      // (g1, g5) = r^ - A e_K; ||r_new|| = ||r|| * ||r^ - A e_K||
      const int64_t nb = launch_helm_resid_ds(c->d, eK, c->g1, c->g5, a, nu_h2, c->helm_part,
                                              kMaxRestart + 2, s);
      launch_final_reduce(c->helm_part, (int)nb, sdev, s, c->host_red_dev);
      IBM_LAUNCH_CHECK(c);
      IBM_CUDA(c, cudaStreamSynchronize(s));
      qn = std::sqrt(c->host_red[0]);
      rn *= qn;
      if (!std::isfinite(rn)) return set_err(c, IBM_ERR_NAN, "non-finite predictor residual");
    }
    *relres = rn / rnorm0;
    if (*relres <= o->helm_rtol || rn == 0.0) {
      flush();
      IBM_LAUNCH_CHECK(c);
      return IBM_OK;
    }
    if (it >= o->helm_maxit) break;
    // reduction wanted from this correction (with a 3x margin), FP32-limited
    double want = o->helm_rtol / *relres / 3.0;
    if (want < 1e-6) want = 1e-6;
    int K = (int)std::ceil(std::acosh(1.0 / want) / std::acosh(sigma));
    K = K < 2 ? 2 : (K > 60 ? 60 : K);
    // e_old starts at zero (the first step after the normalisation takes it
    // as zero without reading it)
    float* eo = c->g2;
    float* e = c->g3;
    float* en = c->g4;
    // r^ = r / ||r||: from the FP64 right-hand side first, then from the pair
    launch_helm_cheb(c->d, nullptr, nullptr, c->g1, c->g5, it == 0 ? rhs : nullptr, 1.0 / qn,
                     (float)a, (float)nu_h2, (float)(1.0 / theta), 0.f, e, nullptr, 0.0, 0, s);
    double rho_prev = 1.0 / sigma;
    for (int q = 1; q < K; ++q) {
      const double rho = 1.0 / (2.0 * sigma - rho_prev);
      const int last = q == K - 1;
      // the first correction's last step keeps its output in g6; the
      // second's writes u from it and its own output; later ones add to u
      const bool keep = last && it == 0;
      const int mode = last && !keep ? 2 : 1;
      if (keep) en = c->g6;
      const int ph = mode == 2 ? -1 : prof_begin(c, IBM_PROF_HELM_SWEEP);
      const int flags = (q == 1 ? 1 : 0) | (mode == 2 && pend ? 2 : 0);
      launch_helm_cheb(c->d, e, eo, c->g1, nullptr, nullptr, 0.0, (float)a, (float)nu_h2,
                       (float)(2.0 * rho / delta), (float)(rho * rho_prev), en, u, rn, mode, s,
                       flags, mode == 2 ? pend : nullptr, pend_s);
      // e, e_old (not on the first step), r read; e_new written
      prof_end(c, ph, (q == 1 ? 12.0 : 16.0) * (double)c->nf);
      if (mode == 2) pend = nullptr;
      rho_prev = rho;
      float* t = eo; eo = e; e = en; en = t;
    }
    eK = e;   // after the rotation the last output is in e
    if (it == 0) {
      pend = eK;
      pend_s = rn;
    }
    IBM_LAUNCH_CHECK(c);
    *iters = it + 1;
  }
  flush();
  char buf[160];
  snprintf(buf, sizeof buf, "predictor did not reach helm_rtol %.3g (relres %.3g)", o->helm_rtol,
           *relres);
  return set_err(c, IBM_ERR_NOT_CONVERGED, buf);
}

}  // namespace ibm

using namespace ibm;

extern "C" {

void ibm_default_opts(ibm_solve_opts* o) {
  if (!o) return;
  o->precond_prec = IBM_PREC_FP32;
  o->rtol = 1e-8;
  o->maxit = 200;
  o->restart = 40;
  o->mg_pre = 2;
  o->mg_post = 2;
  o->reorth = 0;
  o->helm_rtol = 1e-10;
  o->helm_maxit = 8;
  o->with_advection = 1;
  o->arnoldi = IBM_ARNOLDI_FP32;
  o->c_mode = IBM_CMODE_SCALAR;
  o->c_rtol = 1e-14;
  o->c_maxit = 500;
  o->cycle_graphs = 0;
}

ibm_status ibm_create(const ibm_grid_desc* g, void* stream, ibm_ctx** out) {
  if (!out) return IBM_ERR_ARG;
  *out = nullptr;
  if (!g || g->nx < 4 || g->ny < 4 || g->nz < 4 || !(g->h > 0.0) || !(g->Re > 0.0) ||
      !(g->dt > 0.0))
    return IBM_ERR_ARG;
  if ((int64_t)g->nx * g->ny * g->nz * 4 > (int64_t)0x7fffffff) return IBM_ERR_ARG;
  ibm_ctx* c = new (std::nothrow) ibm_ctx();
  if (!c) return IBM_ERR_NOMEM;
  c->d = Dims{g->nx, g->ny, g->nz};
  c->h = g->h;
  c->Re = g->Re;
  c->dt = g->dt;
  c->m = cells_of(c->d);
  c->fd = face_dims(c->d);
  c->nf = c->fd.nfx + c->fd.nfy + c->fd.nfz;
  c->stream = static_cast<cudaStream_t>(stream);
  const int64_t m = c->m, nf = c->nf;
  // block sums of the scans: int32 per block, or a pair per block for the
  // marker lists' shell-cell pass (with the totals after them)
  const int64_t nscan = 2 * ((m + 4095) / 4096 + 2);
  bool ok = cudaMalloc(&c->cell_count, sizeof(int32_t) * m) == cudaSuccess &&
            cudaMalloc(&c->cell_start, sizeof(int32_t) * (m + 1)) == cudaSuccess &&
            cudaMalloc(&c->cell_flag, sizeof(int32_t) * (m + 1)) == cudaSuccess &&
            cudaMalloc(&c->scan_tmp, sizeof(int32_t) * nscan) == cudaSuccess &&
            cudaMalloc(&c->dev_flag, sizeof(int32_t) * 4) == cudaSuccess &&
            cudaHostAlloc(&c->host_flag, sizeof(int32_t) * 4, cudaHostAllocMapped) ==
                cudaSuccess &&
            cudaHostGetDevicePointer(&c->host_flag_dev, c->host_flag, 0) == cudaSuccess &&
            cudaMalloc(&c->c1, sizeof(double) * m) == cudaSuccess &&
            cudaMalloc(&c->c2, sizeof(double) * m) == cudaSuccess &&
            cudaMalloc(&c->c3, sizeof(double) * (m + 1)) == cudaSuccess &&
            cudaMalloc(&c->f1, sizeof(double) * nf) == cudaSuccess &&
            cudaMalloc(&c->f2, sizeof(double) * nf) == cudaSuccess &&
            cudaMalloc(&c->f3, sizeof(double) * nf) == cudaSuccess &&
            cudaMalloc(&c->f4, sizeof(double) * nf) == cudaSuccess &&
            cudaMalloc(&c->g1, sizeof(float) * helm_fp32_size(c->d)) == cudaSuccess &&
            cudaMalloc(&c->g2, sizeof(float) * helm_fp32_size(c->d)) == cudaSuccess &&
            cudaMalloc(&c->g3, sizeof(float) * helm_fp32_size(c->d)) == cudaSuccess &&
            cudaMalloc(&c->g4, sizeof(float) * helm_fp32_size(c->d)) == cudaSuccess &&
            cudaMalloc(&c->g5, sizeof(float) * helm_fp32_size(c->d)) == cudaSuccess &&
            cudaMalloc(&c->g6, sizeof(float) * helm_fp32_size(c->d)) == cudaSuccess &&
            cudaMalloc(&c->red_part, sizeof(double) * kRedBlocks * (kMaxRestart + 2)) ==
                cudaSuccess &&
            cudaMalloc(&c->red_out, sizeof(double) * 8 * (kMaxRestart + 2)) ==
                cudaSuccess &&
            cudaHostAlloc(&c->host_red, sizeof(double) * 8 * (kMaxRestart + 2),
                          cudaHostAllocMapped) == cudaSuccess &&
            cudaHostGetDevicePointer(&c->host_red_dev, c->host_red, 0) == cudaSuccess &&
            cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&c->ev_iter[0], cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&c->ev_iter[1], cudaEventDisableTiming) == cudaSuccess &&
            cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) == cudaSuccess &&
            cudaMalloc(&c->gstate, sizeof(double) * GState::kSize) == cudaSuccess &&
            cudaHostAlloc(&c->host_gstate, sizeof(double) * GState::kSize, cudaHostAllocMapped) ==
                cudaSuccess &&
            cudaHostGetDevicePointer(&c->host_gstate_dev, c->host_gstate, 0) == cudaSuccess;
  {
    // partial sums of the fused predictor residual norm (one per block)
    const int64_t nb = (int64_t)div_up(g->nx + 1, 32) * div_up(g->ny + 1, 8) * 3 *
                       div_up(g->nz + 1, 16);
    c->helm_part_n = nb * (kMaxRestart + 2);
    ok = ok && cudaMalloc(&c->helm_part, sizeof(double) * c->helm_part_n) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    free_all(c);
    delete c;
    return IBM_ERR_NOMEM;
  }
  // the predictor's FP32 arrays: wall faces beyond the launched x-range are
  // never written and must read as 0
  for (float* buf : {c->g1, c->g2, c->g3, c->g4, c->g5, c->g6})
    if (cudaMemset(buf, 0, sizeof(float) * helm_fp32_size(c->d)) != cudaSuccess) ok = false;
  ibm_status st = ok ? mg_setup(c) : IBM_ERR_CUDA;
  if (st == IBM_OK && cudaDeviceSynchronize() != cudaSuccess) st = IBM_ERR_CUDA;
  if (st != IBM_OK) {
    cudaGetLastError();
    free_all(c);
    delete c;
    return st;
  }
  c->markers_set = true;   // zero markers until ibm_set_markers
  *out = c;
  return IBM_OK;
}

void ibm_destroy(ibm_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  free_all(c);
  delete c;
}

const char* ibm_last_error(const ibm_ctx* c) { return c ? c->err.c_str() : "null context"; }

int64_t ibm_num_cells(const ibm_ctx* c) { return c ? c->m : 0; }
int64_t ibm_num_faces(const ibm_ctx* c) { return c ? c->nf : 0; }

ibm_status ibm_set_markers(ibm_ctx* c, int64_t n, const double* X) {
  if (check_ctx(c) != IBM_OK) return IBM_ERR_ARG;
  if (n < 0 || n > (int64_t)1 << 24) return set_err(c, IBM_ERR_ARG, "n_markers out of range");
  if (n > 0 && bad_ptr(X)) return set_err(c, IBM_ERR_ARG, "X is null or misaligned");
  const int ph = prof_begin(c, IBM_PROF_MARKER_BUILD);
  const ibm_status st = markers_build(c, n, X);
  prof_end(c, ph);
  return st;
}

ibm_status ibm_apply_laplacian(ibm_ctx* c, const double* v, double* out) {
  if (check_ctx(c) != IBM_OK) return IBM_ERR_ARG;
  if (bad_ptr(v) || bad_ptr(out) || v == out) return set_err(c, IBM_ERR_ARG, "bad v/out");
  launch_laplacian<double>(c->d, v, out, 1.0 / (c->h * c->h), c->stream);
  IBM_LAUNCH_CHECK(c);
  return IBM_OK;
}

ibm_status ibm_apply_schur(ibm_ctx* c, const double* v, double* out) {
  if (check_ctx(c) != IBM_OK) return IBM_ERR_ARG;
  if (bad_ptr(v) || bad_ptr(out) || v == out) return set_err(c, IBM_ERR_ARG, "bad v/out");
  set_cmode(c, nullptr);
  return schur_apply(c, v, out);
}

ibm_status ibm_apply_schur_opts(ibm_ctx* c, const double* v, double* out,
                                const ibm_solve_opts* o, int64_t* c_iters) {
  if (check_ctx(c) != IBM_OK) return IBM_ERR_ARG;
  if (bad_ptr(v) || bad_ptr(out) || v == out) return set_err(c, IBM_ERR_ARG, "bad v/out");
  const ibm_status s = check_opts(c, o);
  if (s != IBM_OK) return s;
  set_cmode(c, o);
  const ibm_status r = schur_apply(c, v, out);
  if (c_iters) *c_iters = c->c_iters;
  set_cmode(c, nullptr);
  return r;
}

ibm_status ibm_apply_laplacian_precond(ibm_ctx* c, const double* r, double* z, int32_t prec,
                                       int32_t pre, int32_t post) {
  if (check_ctx(c) != IBM_OK) return IBM_ERR_ARG;
  if (bad_ptr(r) || bad_ptr(z) || r == z) return set_err(c, IBM_ERR_ARG, "bad r/z");
  if ((prec != IBM_PREC_FP32 && prec != IBM_PREC_FP64) || pre < 0 || pre > 4 || post < 0 ||
      post > 4 || pre + post == 0)
    return set_err(c, IBM_ERR_ARG, "bad precision or smoothing degrees");
  return mg_vcycle(c, r, z, prec, pre, post);
}

ibm_status ibm_interp(ibm_ctx* c, const double* u, double* U) {
  if (check_ctx(c) != IBM_OK) return IBM_ERR_ARG;
  if (c->mk.n == 0) return IBM_OK;
  if (bad_ptr(u) || bad_ptr(U)) return set_err(c, IBM_ERR_ARG, "bad u/U");
  launch_interp(c, u, U);
  IBM_LAUNCH_CHECK(c);
  return IBM_OK;
}

ibm_status ibm_spread(ibm_ctx* c, const double* F, double* u) {
  if (check_ctx(c) != IBM_OK) return IBM_ERR_ARG;
  if (bad_ptr(u) || (c->mk.n > 0 && bad_ptr(F))) return set_err(c, IBM_ERR_ARG, "bad F/u");
  launch_zero(u, sizeof(double) * c->nf, c->stream);
  launch_shell_spread_faces(c, F, 1.0, u);
  IBM_LAUNCH_CHECK(c);
  return IBM_OK;
}

ibm_status ibm_gradient(ibm_ctx* c, const double* p, double* u) {
  if (check_ctx(c) != IBM_OK) return IBM_ERR_ARG;
  if (bad_ptr(p) || bad_ptr(u)) return set_err(c, IBM_ERR_ARG, "bad p/u");
  launch_gradient(c->d, p, u, 1.0 / c->h, c->stream);
  IBM_LAUNCH_CHECK(c);
  return IBM_OK;
}

ibm_status ibm_gradient_t(ibm_ctx* c, const double* u, double* out) {
  if (check_ctx(c) != IBM_OK) return IBM_ERR_ARG;
  if (bad_ptr(u) || bad_ptr(out)) return set_err(c, IBM_ERR_ARG, "bad u/out");
  launch_gradient_t(c->d, u, out, 1.0 / c->h, c->stream);
  IBM_LAUNCH_CHECK(c);
  return IBM_OK;
}

ibm_status ibm_solve_schur(ibm_ctx* c, const double* b, double* p, const ibm_solve_opts* o,
                           ibm_solve_stats* st) {
  if (check_ctx(c) != IBM_OK) return IBM_ERR_ARG;
  if (bad_ptr(b) || bad_ptr(p) || b == p) return set_err(c, IBM_ERR_ARG, "bad b/p");
  ibm_status s = check_opts(c, o);
  if (s != IBM_OK) return s;
  if ((s = ensure_krylov(c, o->restart)) != IBM_OK) return s;
  if (st) memset(st, 0, sizeof(*st));
  set_cmode(c, o);
  const double mk0 = prof_mark(c);
  const int ph = prof_begin(c, IBM_PROF_SOLVE);
  s = fgmres_solve(c, b, p, o, st);
  prof_end_span(c, ph, mk0);
  if (st) st->c_iters = c->c_iters;
  set_cmode(c, nullptr);
  return s;
}

ibm_status ibm_force_correction(ibm_ctx* c, const double* p, const double* rhs_F, double* Fc) {
  if (check_ctx(c) != IBM_OK) return IBM_ERR_ARG;
  const int64_t n = c->mk.n;
  if (n == 0) return IBM_OK;
  if (bad_ptr(p) || bad_ptr(rhs_F) || bad_ptr(Fc)) return set_err(c, IBM_ERR_ARG, "bad args");
  launch_marker_grad_interp(c, p, 1.0, c->mk.t);
  count_launch();
  k_axpby_small<<<div_up(3 * n, TPB), TPB, 0, c->stream>>>(c->mk.t, 2.0, rhs_F, -2.0, Fc, 3 * n);
  IBM_LAUNCH_CHECK(c);
  return IBM_OK;
}

static ibm_status step_impl(ibm_ctx* c, const double* u_n, const double* u_nm1, const double* p_n,
                    const double* F_n, const double* U_gamma, const double* f_body,
                    double* u_np1, double* p_np1, double* F_np1, const ibm_solve_opts* o,
                    ibm_solve_stats* st) {
  if (check_ctx(c) != IBM_OK) return IBM_ERR_ARG;
  const int64_t n = c->mk.n;
  if (bad_ptr(u_n) || bad_ptr(u_nm1) || bad_ptr(p_n) || bad_ptr(u_np1) || bad_ptr(p_np1) ||
      (f_body && bad_ptr(f_body)))
    return set_err(c, IBM_ERR_ARG, "bad field pointer");
  if (n > 0 && (bad_ptr(F_n) || bad_ptr(U_gamma) || bad_ptr(F_np1)))
    return set_err(c, IBM_ERR_ARG, "bad marker pointer");
  if (u_np1 == u_n || u_np1 == u_nm1 || p_np1 == p_n || (n > 0 && F_np1 == F_n))
    return set_err(c, IBM_ERR_ARG, "outputs must not alias inputs");
  ibm_status s = check_opts(c, o);
  if (s != IBM_OK) return s;
  if ((s = ensure_krylov(c, o->restart)) != IBM_OK) return s;
  ibm_solve_stats local;
  if (!st) st = &local;
  memset(st, 0, sizeof(*st));
  set_cmode(c, o);
  cudaStream_t str = c->stream;
  const double a = 1.5 / c->dt;
  const double inv_h = 1.0 / c->h;
  MarkerData& mk = c->mk;
  const bool scalar = o->c_mode == IBM_CMODE_SCALAR;
  const double csign = o->c_mode == IBM_CMODE_CONSISTENT ? -1.0 : 1.0;

  // 1. predictor (Eq. (ustar))
  launch_predictor_rhs_adv(c->d, u_n, u_nm1, p_n, f_body, o->with_advection, 1.0 / (2.0 * c->dt),
                           inv_h, c->f1, str);
  if (n > 0) launch_shell_spread_faces(c, F_n, 1.0, c->f1);
  IBM_LAUNCH_CHECK(c);
  double* u_star = c->f2;
  int ph = prof_begin(c, IBM_PROF_PREDICTOR);
  s = helmholtz_solve(c, c->f1, u_star, o, &st->helm_iters, &st->helm_relres);
  prof_end(c, ph);
  if (s != IBM_OK) return s;

  // 2. RHS_p = a G^T u*, RHS_F = a (R^T u* - U), b = RHS_p + 2 B^T RHS_F
  launch_gradt_axpby(c->d, u_star, a * inv_h, nullptr, 0.0, c->c2, str);
  if (n > 0) {
    launch_interp(c, u_star, mk.t2);
    count_launch();
    k_axpby_small<<<div_up(3 * n, TPB), TPB, 0, str>>>(mk.t2, a, U_gamma, -a, mk.t2, 3 * n);
    if (scalar) {
      launch_shell_gradt_spread(c, mk.t2, 2.0, c->c2);
    } else {
      // RHS_F kept in t3 (the Schur products use t and t2); b = RHS_p +- B^T C^{-1} RHS_F
      launch_copy(mk.t3, mk.t2, sizeof(double) * 3 * n, str);
      if ((s = c_solve(c, mk.t3, mk.t2, c->c_rtol, c->c_maxit, nullptr)) != IBM_OK) return s;
      launch_shell_gradt_spread(c, mk.t2, csign, c->c2);
    }
  }
  IBM_LAUNCH_CHECK(c);

  // 3. Schur solve for p' (into c3, zero initial guess)
  double* pc = c->c3;
  launch_zero(pc, sizeof(double) * c->m, str);
  const double mk0 = prof_mark(c);
  ph = prof_begin(c, IBM_PROF_SOLVE);
  // p' keeps its constant: only p^{n+1} depends on it, and it is removed
  // where p^{n+1} is formed (G p' and B p' are blind to it)
  double* psum = c->red_out + 7 * (kMaxRestart + 2) + 4;
  c->defer_mean = psum;
  s = fgmres_solve(c, c->c2, pc, o, st, true);
  c->defer_mean = nullptr;
  prof_end_span(c, ph, mk0);
  if (s != IBM_OK && s != IBM_ERR_NOT_CONVERGED) return s;
  const ibm_status solve_status = s;

  // 4.-5. F' = 2 (B p' - RHS_F); updates
  launch_axpy_shift(p_n, pc, psum, -1.0 / (double)c->m, p_np1, c->m, str);
  launch_grad_axpy(c->d, u_star, pc, -(2.0 * c->dt / 3.0) * inv_h, u_np1, str);
  if (n > 0) {
    launch_marker_grad_interp(c, pc, 1.0, mk.t);
    if (scalar) {
      count_launch();
      k_axpby_small<<<div_up(3 * n, TPB), TPB, 0, str>>>(mk.t, 2.0, mk.t2, -2.0, mk.t, 3 * n);
    } else {
      // F' = C^{-1} (B p' - RHS_F)
      count_launch();
      k_axpby_small<<<div_up(3 * n, TPB), TPB, 0, str>>>(mk.t, 1.0, mk.t3, -1.0, mk.t3, 3 * n);
      if ((s = c_solve(c, mk.t3, mk.t, c->c_rtol, c->c_maxit, nullptr)) != IBM_OK) return s;
    }
    count_launch();
    k_axpby_small<<<div_up(3 * n, TPB), TPB, 0, str>>>(F_n, 1.0, mk.t, 1.0, F_np1, 3 * n);
    launch_shell_spread_faces(c, mk.t, 2.0 * c->dt / 3.0, u_np1);
  }
  IBM_LAUNCH_CHECK(c);

  // 6. diagnostics: both squared norms go to the host mirror, one round trip
  double* dslot = c->red_out + 7 * (kMaxRestart + 2);
  // ||G^T u||^2 from per-block sums of squares (G^T u itself is not stored)
  if (gradt_norm2_blocks(c->d) <= c->helm_part_n) {
    const int64_t nb = launch_gradt_norm2(c->d, u_np1, inv_h, c->helm_part, str);
    launch_final_reduce(c->helm_part, (int)nb, dslot, str, c->host_red_dev, 1);
  } else {
    launch_gradient_t(c->d, u_np1, c->c1, inv_h, str);
    launch_dot(c->c1, c->c1, c->m, c->red_part, dslot, str, c->host_red_dev);
  }
  if (n > 0) {
    launch_interp(c, u_np1, mk.t2);
    count_launch();
    k_axpby_small<<<div_up(3 * n, TPB), TPB, 0, str>>>(mk.t2, 1.0, U_gamma, -1.0, mk.t2, 3 * n);
    launch_dot(mk.t2, mk.t2, 3 * n, c->red_part, dslot + 1, str, c->host_red_dev + 1);
  }
  IBM_LAUNCH_CHECK(c);
  IBM_CUDA(c, cudaStreamSynchronize(str));
  st->div_l2 = std::sqrt(c->host_red[0]);
  if (n > 0) st->slip_l2 = std::sqrt(c->host_red[1]);
  st->c_iters = c->c_iters;
  set_cmode(c, nullptr);
  return solve_status;
}

ibm_status ibm_step(ibm_ctx* c, const double* u_n, const double* u_nm1, const double* p_n,
                    const double* F_n, const double* U_gamma, const double* f_body,
                    double* u_np1, double* p_np1, double* F_np1, const ibm_solve_opts* o,
                    ibm_solve_stats* st) {
  const int ph = c ? prof_begin(c, IBM_PROF_STEP) : -1;
  const ibm_status s = step_impl(c, u_n, u_nm1, p_n, F_n, U_gamma, f_body, u_np1, p_np1, F_np1,
                                 o, st);
  if (c) prof_end(c, ph);
  return s;
}

int64_t ibm_kernel_launches(void) { return (int64_t)g_launches.load(); }

ibm_status ibm_profile_enable(ibm_ctx* c, int32_t on) {
  if (check_ctx(c) != IBM_OK) return IBM_ERR_ARG;
  IBM_CUDA(c, cudaStreamSynchronize(c->stream));
  c->prof_on = on != 0;
  c->prof_used = 0;
  c->prof_acc = 0.0;
  return IBM_OK;
}

ibm_status ibm_profile_read(ibm_ctx* c, ibm_profile* out) {
  if (check_ctx(c) != IBM_OK || !out) return IBM_ERR_ARG;
  IBM_CUDA(c, cudaStreamSynchronize(c->stream));
  memset(out, 0, sizeof(*out));
  for (size_t i = 0; i < c->prof_used; ++i) {
    float ms = 0.f;
    IBM_CUDA(c, cudaEventElapsedTime(&ms, c->prof[i].a, c->prof[i].b));
    const int k = c->prof[i].cls;
    if (k >= 0 && k < IBM_PROF_NCLASS) {
      out->ms[k] += ms;
      out->launches[k] += 1;
      out->bytes[k] += c->prof[i].bytes;
    }
  }
  return IBM_OK;
}

ibm_status ibm_body_forces(ibm_ctx* c, const double* F, const double* X, const int32_t* body_id,
                           int32_t n_bodies, const double* centers, double* out) {
  if (check_ctx(c) != IBM_OK) return IBM_ERR_ARG;
  const int64_t n = c->mk.n;
  if (n_bodies < 1 || n_bodies > 4096 || !centers || !out)
    return set_err(c, IBM_ERR_ARG, "bad body arguments");
  if (n > 0 && (bad_ptr(F) || bad_ptr(X) || body_id == nullptr))
    return set_err(c, IBM_ERR_ARG, "bad marker pointers");
  // sums, then the centres: n_bodies * 9 <= kRedBlocks * (kMaxRestart + 2)
  double* dout = c->red_part;
  double* dcen = c->red_part + 6 * (int64_t)n_bodies;
  const double h3 = c->h * c->h * c->h;
  if (n == 0) {
    for (int q = 0; q < 6 * n_bodies; ++q) out[q] = 0.0;
    return IBM_OK;
  }
  IBM_CUDA(c, cudaMemcpyAsync(dcen, centers, sizeof(double) * 3 * n_bodies,
                              cudaMemcpyHostToDevice, c->stream));
  launch_body_sums(F, X, body_id, n, n_bodies, dcen, h3, dout, c->stream);
  IBM_LAUNCH_CHECK(c);
  IBM_CUDA(c, cudaMemcpyAsync(out, dout, sizeof(double) * 6 * n_bodies, cudaMemcpyDeviceToHost,
                              c->stream));
  IBM_CUDA(c, cudaStreamSynchronize(c->stream));
  return IBM_OK;
}

}  // extern "C"
