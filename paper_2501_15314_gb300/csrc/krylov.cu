// Schur-complement operator S~ = L + 2 B^T B (Eq. (tildeSp)) and its
// Laplacian-preconditioned Krylov solve (Sec. 4.1-4.2): right-preconditioned
// flexible GMRES in FP64 with classical Gram-Schmidt done as one fused
// multi-dot pass and one fused axpy+norm pass per iteration.  The paper's own
// solver is left-preconditioned (BiCGStab/GMRES with an exact L^{-1}); the
// flexible right-preconditioned form is used here because the preconditioner
// (one FP32 V-cycle) is not an exact fixed linear map, and it measures the
// unpreconditioned residual directly.
//
// Reductions are two-stage with a fixed grid (kRedBlocks blocks, fixed-order
// tree inside each block, then one fixed-order tree per output): results are
// bitwise reproducible run to run.
#include <cmath>
#include <vector>

#include "ds.cuh"
#include "ibm_internal.cuh"

namespace ibm {

namespace {

constexpr int RT = kRedThreads;
constexpr int kOutStride = kMaxRestart + 2;

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Reduces NQ per-thread values across the block; thread q < nq of the block
// writes part[blockIdx.x * kOutStride + q].
template <int NQ>
__device__ __forceinline__ void block_reduce_store(double (&acc)[NQ], int nq, double* part) {
  __shared__ double sh[RT / 32][NQ];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const double v = warp_sum(acc[q]);
    if (lane == 0) sh[wid][q] = v;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < nq; q += RT) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < RT / 32; ++w) s += sh[w][q];
    part[(int64_t)blockIdx.x * kOutStride + q] = s;
  }
}

// part[b][q] = sum over this block's elements of w_i * V_q[i], q < nq <= NQ
template <int NQ>
__global__ void __launch_bounds__(RT) k_multidot(const double* __restrict__ w,
                                                 const double* __restrict__ V, int64_t ld, int nq,
                                                 int64_t n, double* __restrict__ part) {
  double acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT) {
    const double wi = __ldg(w + i);
#pragma unroll
    for (int q = 0; q < NQ; ++q)
      if (q < nq) acc[q] = fma(wi, __ldg(V + q * ld + i), acc[q]);
  }
  block_reduce_store<NQ>(acc, nq, part);
}

// w -= sum_q coef[q] V_q ; part[b][0] = sum of w_i^2 over this block
template <int NQ>
__global__ void __launch_bounds__(RT) k_axpy_norm(double* __restrict__ w,
                                                  const double* __restrict__ V, int64_t ld,
                                                  int nq, const double* __restrict__ coef,
                                                  int64_t n, double* __restrict__ part) {
  double cf[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) cf[q] = q < nq ? coef[q] : 0.0;
  double acc[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT) {
    double wi = w[i];
#pragma unroll
    for (int q = 0; q < NQ; ++q)
      if (q < nq) wi = fma(-cf[q], __ldg(V + q * ld + i), wi);
    w[i] = wi;
    acc[0] = fma(wi, wi, acc[0]);
  }
  block_reduce_store<1>(acc, 1, part);
}

// out[q] = sum_b part[b * stride + q], fixed-order tree (one block per q);
// with div != null also quot[q] = out[q] / div[q]; with hout != null also
// hout[q] = out[q] (the device address of the mapped host mirror)
__global__ void __launch_bounds__(RT) k_final_reduce(const double* __restrict__ part, int nb,
                                                     double* __restrict__ out,
                                                     const double* __restrict__ div = nullptr,
                                                     double* __restrict__ quot = nullptr,
                                                     double* hout = nullptr,
                                                     int stride = kOutStride) {
  const int q = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += RT) s += part[(int64_t)b * stride + q];
  __shared__ double sh[RT / 32];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < RT / 32; ++w) t += sh[w];
    out[q] = t;
    if (div) quot[q] = t / div[q];
    if (hout) hout[q] = t;
  }
}

// Zeroing and device-to-device copies by kernels, so that the copy engines
// serve only the caller's transfers: 16-byte words where both ends allow it,
// else 4-byte words.
template <typename W>
__global__ void k_zero_words(W* __restrict__ p, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = W{};
}
template <typename W>
__global__ void k_copy_words(W* __restrict__ dst, const W* __restrict__ src, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

// n 32-bit words from device memory to the mapped host mirror
__global__ void k_to_host(const uint32_t* __restrict__ src, uint32_t* dst, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

__global__ void k_dot(const double* __restrict__ a, const double* __restrict__ b, int64_t n,
                      double* __restrict__ part) {
  double acc[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT)
    acc[0] = fma(__ldg(a + i), b ? __ldg(b + i) : 1.0, acc[0]);
  block_reduce_store<1>(acc, 1, part);
}

// Sum of squares of an FP64 vector to about 1e-5 relative, for stopping
// baselines: each value's leading FP32 part (split_exact: sign, exponent and
// top fraction bits with integer operations) squared and summed in FP32 per
// thread, the threads' sums in FP64 (an FP64 dot is bound by the FP64 pipe).
__global__ void __launch_bounds__(RT) k_norm2_lead(const double* __restrict__ x, int64_t n,
                                                   double* __restrict__ part) {
  float acc = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT) {
    const float h = split_exact(__ldg(x + i)).hi;
    acc = fmaf(h, h, acc);
  }
  double a[1] = {(double)acc};
  block_reduce_store<1>(a, 1, part);
}

__global__ void k_axpby(const double* __restrict__ x, double a, const double* __restrict__ y,
                        double b, double* __restrict__ out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = fma(a, x[i], b * y[i]);
}

// x += sum_q y[q] Z_q  (y by value)
template <int NQ>
__global__ void __launch_bounds__(RT) k_gemv_acc(double* __restrict__ x,
                                                 const double* __restrict__ Z, int64_t ld, int nq,
                                                 const CoefF64 y, int64_t n) {
  double cf[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) cf[q] = q < nq ? y.v[q] : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT) {
    double xi = x[i];
#pragma unroll
    for (int q = 0; q < NQ; ++q)
      if (q < nq) xi = fma(cf[q], __ldg(Z + q * ld + i), xi);
    x[i] = xi;
  }
}

__global__ void k_axpy_shift(const double* __restrict__ x, const double* __restrict__ y,
                             const double* __restrict__ val, double scale,
                             double* __restrict__ out, int64_t n) {
  const double v = scale * (*val);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double yi = y[i] + v;
    out[i] = fma(1.0, x[i], 1.0 * yi);
  }
}

__global__ void k_add_scalar(double* __restrict__ x, int64_t n, const double* __restrict__ val,
                             double scale) {
  const double v = scale * (*val);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] += v;
}

#define IBM_NQ_DISPATCH(nq, KERNEL, ...)                          \
  do {                                                            \
    count_launch();                                               \
    if ((nq) <= 2) KERNEL<2><<<kRedBlocks, RT, 0, s>>>(__VA_ARGS__);        \
    else if ((nq) <= 4) KERNEL<4><<<kRedBlocks, RT, 0, s>>>(__VA_ARGS__);   \
    else if ((nq) <= 8) KERNEL<8><<<kRedBlocks, RT, 0, s>>>(__VA_ARGS__);   \
    else if ((nq) <= 12) KERNEL<12><<<kRedBlocks, RT, 0, s>>>(__VA_ARGS__); \
    else if ((nq) <= 16) KERNEL<16><<<kRedBlocks, RT, 0, s>>>(__VA_ARGS__); \
    else if ((nq) <= 24) KERNEL<24><<<kRedBlocks, RT, 0, s>>>(__VA_ARGS__); \
    else if ((nq) <= 32) KERNEL<32><<<kRedBlocks, RT, 0, s>>>(__VA_ARGS__); \
    else if ((nq) <= 48) KERNEL<48><<<kRedBlocks, RT, 0, s>>>(__VA_ARGS__); \
    else KERNEL<kMaxRestart + 1><<<kRedBlocks, RT, 0, s>>>(__VA_ARGS__);    \
  } while (0)

}  // namespace

void launch_multidot(const double* w, const double* V, int64_t ld, int nq, int64_t n,
                     double* part, double* out, cudaStream_t s, const double* div,
                     double* quot, double* hout) {
  IBM_NQ_DISPATCH(nq, k_multidot, w, V, ld, nq, n, part);
  count_launch();
  k_final_reduce<<<nq, RT, 0, s>>>(part, kRedBlocks, out, div, quot, hout);
}

void launch_axpy_norm(double* w, const double* V, int64_t ld, int nq, const double* coef,
                      int64_t n, double* part, double* out, cudaStream_t s, double* hout) {
  IBM_NQ_DISPATCH(nq, k_axpy_norm, w, V, ld, nq, coef, n, part);
  count_launch();
  k_final_reduce<<<1, RT, 0, s>>>(part, kRedBlocks, out, nullptr, nullptr, hout);
}

void launch_final_reduce(const double* part, int nb, double* out, cudaStream_t s,
                         double* hout, int stride) {
  count_launch();
  k_final_reduce<<<1, RT, 0, s>>>(part, nb, out, nullptr, nullptr, hout, stride);
}

void launch_dot(const double* a, const double* b, int64_t n, double* part, double* out,
                cudaStream_t s, double* hout) {
  count_launch();
  k_dot<<<kRedBlocks, RT, 0, s>>>(a, b, n, part);
  count_launch();
  k_final_reduce<<<1, RT, 0, s>>>(part, kRedBlocks, out, nullptr, nullptr, hout);
}

void launch_norm2_lead(const double* x, int64_t n, double* part, double* out, cudaStream_t s,
                       double* hout) {
  count_launch();
  k_norm2_lead<<<kRedBlocks, RT, 0, s>>>(x, n, part);
  count_launch();
  k_final_reduce<<<1, RT, 0, s>>>(part, kRedBlocks, out, nullptr, nullptr, hout);
}

namespace {
int word_blocks(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 4 * kRedBlocks ? 4 * kRedBlocks : b));
}
bool al16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
}  // namespace

void launch_zero(void* p, int64_t nbytes, cudaStream_t s) {
  if (nbytes <= 0) return;
  count_launch();
  if (al16(p) && nbytes % 16 == 0)
    k_zero_words<uint4><<<word_blocks(nbytes / 16), 256, 0, s>>>(static_cast<uint4*>(p),
                                                                 nbytes / 16);
  else
    k_zero_words<uint32_t><<<word_blocks(nbytes / 4), 256, 0, s>>>(static_cast<uint32_t*>(p),
                                                                   nbytes / 4);
}

void launch_copy(void* dst, const void* src, int64_t nbytes, cudaStream_t s) {
  if (nbytes <= 0) return;
  count_launch();
  if (al16(dst) && al16(src) && nbytes % 16 == 0)
    k_copy_words<uint4><<<word_blocks(nbytes / 16), 256, 0, s>>>(
        static_cast<uint4*>(dst), static_cast<const uint4*>(src), nbytes / 16);
  else
    k_copy_words<uint32_t><<<word_blocks(nbytes / 4), 256, 0, s>>>(
        static_cast<uint32_t*>(dst), static_cast<const uint32_t*>(src), nbytes / 4);
}

void launch_to_host(const void* src, void* dst_dev, int nbytes, cudaStream_t s) {
  count_launch();
  k_to_host<<<1, 64, 0, s>>>(static_cast<const uint32_t*>(src), static_cast<uint32_t*>(dst_dev),
                             nbytes / 4);
}

void launch_sum(const double* x, int64_t n, double* part, double* out, cudaStream_t s) {
  launch_dot(x, nullptr, n, part, out, s);
}

void launch_axpby(const double* x, double a, const double* y, double b, double* out, int64_t n,
                  cudaStream_t s) {
  count_launch();
  k_axpby<<<kRedBlocks, RT, 0, s>>>(x, a, y, b, out, n);
}

void launch_gemv_acc(double* x, const double* Z, int64_t ld, int nq, const double* y, int64_t n,
                     cudaStream_t s) {
  CoefF64 cy;
  for (int q = 0; q <= kMaxRestart; ++q) cy.v[q] = q < nq ? y[q] : 0.0;
  IBM_NQ_DISPATCH(nq, k_gemv_acc, x, Z, ld, nq, cy, n);
}

void launch_axpy_shift(const double* x, const double* y, const double* val, double scale,
                       double* out, int64_t n, cudaStream_t s) {
  count_launch();
  k_axpy_shift<<<kRedBlocks, RT, 0, s>>>(x, y, val, scale, out, n);
}

void launch_add_scalar_dev(double* x, int64_t n, const double* val, double scale,
                           cudaStream_t s) {
  count_launch();
  k_add_scalar<<<kRedBlocks, RT, 0, s>>>(x, n, val, scale);
}

// ---------------------------------------------------------------------------
ibm_status schur_apply(ibm_ctx* c, const double* v, double* out) {
  return schur_residual(c, nullptr, v, out);
}

ibm_status schur_residual(ibm_ctx* c, const double* b, const double* v, double* out) {
  // out = L v + 2 B^T (B v): t = 2 R^T G v per marker (on the side stream,
  // concurrently with out = L v), then the shell cells gather G^T R t.  With
  // b: out = b - S~ v, the Laplacian kernel writing b - L v and the gather
  // subtracting the marker term (no separate pass over the three vectors).
  const double sgn = b ? -1.0 : 1.0;
  const bool fork = c->cmode == IBM_CMODE_SCALAR && c->mk.n > 0;
  if (fork) {
    IBM_CUDA(c, cudaEventRecord(c->ev_fork, c->stream));
    IBM_CUDA(c, cudaStreamWaitEvent(c->side, c->ev_fork, 0));
    launch_marker_grad_interp(c, v, 2.0, c->mk.t, c->side);
    IBM_CUDA(c, cudaEventRecord(c->ev_join, c->side));
  }
  int ph = prof_begin(c, IBM_PROF_LAPLACIAN_F64);
  launch_laplacian_sub(c->d, v, b, out, 1.0 / (c->h * c->h), c->stream);
  prof_end(c, ph, (b ? 24.0 : 16.0) * (double)c->m);
  ph = prof_begin(c, IBM_PROF_SCHUR_MARKERS);
  if (fork) {
    IBM_CUDA(c, cudaStreamWaitEvent(c->stream, c->ev_join, 0));
    launch_shell_gradt_spread(c, c->mk.t, sgn, out);
  } else if (c->mk.n > 0) {
    // out +- B^T C^{-1} B v (exact / sign-consistent forms)
    launch_marker_grad_interp(c, v, 1.0, c->mk.t);
    const ibm_status s = c_solve(c, c->mk.t, c->mk.t2, c->c_rtol, c->c_maxit, nullptr);
    if (s != IBM_OK) { prof_end(c, ph); return s; }
    launch_shell_gradt_spread(c, c->mk.t2,
                              sgn * (c->cmode == IBM_CMODE_CONSISTENT ? -1.0 : 1.0), out);
  }
  prof_end(c, ph, c->mk.n > 0 ? marker_term_bytes(c, 8, 8) : 0.0);
  IBM_LAUNCH_CHECK(c);
  return IBM_OK;
}

namespace {

ibm_status fetch(ibm_ctx* c, const double* dev, int n) {
  launch_to_host(dev, c->host_red_dev, (int)sizeof(double) * n, c->stream);
  IBM_LAUNCH_CHECK(c);
  IBM_CUDA(c, cudaStreamSynchronize(c->stream));
  return IBM_OK;
}

}  // namespace

ibm_status fgmres_solve(ibm_ctx* c, const double* b, double* x, const ibm_solve_opts* o,
                        ibm_solve_stats* st, bool x_is_zero) {
  // The Arnoldi vectors are kept unnormalised: V_i with ||V_i||^2 = nrm2[i] on
  // the device.  The preconditioner is applied to V_j as stored (flexible
  // GMRES accepts any z_j; x = Z y uses the same z_j), the Gram-Schmidt
  // coefficients are <w, V_i> / nrm2[i] (formed on the device), and the
  // Hessenberg entries h_ij = <w, V_i> / ||V_i||, h_{j+1,j} = ||w|| on the host.
  if (o->precond_prec == IBM_PREC_FP32 &&
      (o->arnoldi == IBM_ARNOLDI_DS || o->arnoldi == IBM_ARNOLDI_FP32) && !o->reorth &&
      ds_supported(c))
    return fgmres_solve_ds(c, b, x, o, st, x_is_zero);
  cudaStream_t s = c->stream;
  const int64_t m = c->m;
  const int restart = o->restart;
  double* part = c->red_part;
  double* raw = c->red_out;                      // <w, V_i>
  double* coef = c->red_out + kOutStride;        // <w, V_i> / nrm2[i]
  double* raw2 = c->red_out + 2 * kOutStride;    // second Gram-Schmidt pass
  double* coef2 = c->red_out + 3 * kOutStride;
  double* nrm2 = c->red_out + 4 * kOutStride;    // ||V_i||^2
  double* sdev = c->red_out + 6 * kOutStride;    // scalars
  double* hr = c->host_red;                      // host mirror (same offsets)
  ibm_status stt;

  // ||b||
  launch_dot(b, b, m, part, sdev, s);
  prof_note(c, 8.0 * m);
  IBM_LAUNCH_CHECK(c);
  if ((stt = fetch(c, sdev, 1)) != IBM_OK) return stt;
  const double bnorm = std::sqrt(hr[0]);
  if (!std::isfinite(bnorm)) return set_err(c, IBM_ERR_NAN, "non-finite right-hand side");
  int total = 0, cycles = 0;
  double relres = 0.0;
  if (bnorm == 0.0) {
    launch_zero(x, sizeof(double) * m, s);
    if (st) { st->iters = 0; st->restarts = 0; st->relres_true = 0.0; st->graph_cycles = 0; }
    return IBM_OK;
  }
  std::vector<double> H((size_t)(restart + 1) * restart), cs(restart), sn(restart),
      g(restart + 1), y(restart), rn(restart + 1);
  auto Hm = [&](int i, int j) -> double& { return H[(size_t)i * restart + j]; };
  double* V = c->V;
  double* Z = c->Z;
  bool converged = false;
  ibm_status final_status = IBM_OK;
  bool first = true;
  while (true) {
    // V_0 = r0 = b - S x, nrm2[0] = ||r0||^2 (r0 = b for a zero first guess)
    double beta;
    if (first && x_is_zero) {
      launch_copy(V, b, sizeof(double) * m, s);
      launch_copy(nrm2, sdev, sizeof(double), s);
      prof_note(c, 16.0 * m);
      beta = bnorm;
    } else {
      if ((stt = schur_residual(c, b, x, V)) != IBM_OK) return stt;
      launch_dot(V, V, m, part, nrm2, s);
      prof_note(c, 8.0 * m);
      IBM_LAUNCH_CHECK(c);
      if ((stt = fetch(c, nrm2, 1)) != IBM_OK) return stt;
      beta = std::sqrt(hr[0]);
    }
    first = false;
    if (!std::isfinite(beta)) return set_err(c, IBM_ERR_NAN, "non-finite residual");
    relres = beta / bnorm;
    if (relres <= o->rtol) { converged = true; break; }
    if (total >= o->maxit) break;
    rn[0] = beta;
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int jused = 0;
    bool breakdown = false;
    for (int j = 0; j < restart && total < o->maxit; ++j) {
      double* vj = V + (int64_t)j * m;
      double* zj = Z + (int64_t)j * m;
      double* w = V + (int64_t)(j + 1) * m;
      const double mk0 = prof_mark(c);
      int ph = prof_begin(c, IBM_PROF_VCYCLE);
      if ((stt = mg_vcycle(c, vj, zj, o->precond_prec, o->mg_pre, o->mg_post)) != IBM_OK)
        return stt;
      prof_end_span(c, ph, mk0);
      if ((stt = schur_apply(c, zj, w)) != IBM_OK) return stt;
      ph = prof_begin(c, IBM_PROF_MULTIDOT);
      launch_multidot(w, V, m, j + 1, m, part, raw, s, nrm2, coef, hmirror(c, hr));
      prof_end(c, ph, 8.0 * (j + 2) * (double)m);
      ph = prof_begin(c, IBM_PROF_AXPY_NORM);
      launch_axpy_norm(w, V, m, j + 1, coef, m, part, nrm2 + j + 1, s,
                       hmirror(c, hr + 4 * kOutStride + j + 1));
      prof_end(c, ph, 8.0 * (j + 3) * (double)m);
      if (o->reorth) {
        launch_multidot(w, V, m, j + 1, m, part, raw2, s, nrm2, coef2,
                        hmirror(c, hr + 2 * kOutStride));
        launch_axpy_norm(w, V, m, j + 1, coef2, m, part, nrm2 + j + 1, s,
                         hmirror(c, hr + 4 * kOutStride + j + 1));
      }
      IBM_LAUNCH_CHECK(c);
      IBM_CUDA(c, cudaStreamSynchronize(s));
      for (int i = 0; i <= j; ++i)
        Hm(i, j) = (hr[i] + (o->reorth ? hr[2 * kOutStride + i] : 0.0)) / rn[i];
      const double hn = std::sqrt(hr[4 * kOutStride + j + 1]);
      if (!std::isfinite(hn)) return set_err(c, IBM_ERR_NAN, "non-finite Arnoldi vector");
      Hm(j + 1, j) = hn;
      rn[j + 1] = hn;
      for (int i = 0; i < j; ++i) {
        const double t = cs[i] * Hm(i, j) + sn[i] * Hm(i + 1, j);
        Hm(i + 1, j) = -sn[i] * Hm(i, j) + cs[i] * Hm(i + 1, j);
        Hm(i, j) = t;
      }
      const double den = std::hypot(Hm(j, j), Hm(j + 1, j));
      if (den == 0.0) { breakdown = true; break; }
      cs[j] = Hm(j, j) / den;
      sn[j] = Hm(j + 1, j) / den;
      Hm(j, j) = den;
      Hm(j + 1, j) = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++total;
      jused = j + 1;
      if (st && total - 1 < IBM_HIST_MAX) st->relres_hist[total - 1] = std::fabs(g[j + 1]) / bnorm;
      if (std::fabs(g[j + 1]) / bnorm <= o->rtol || hn == 0.0) break;
    }
    if (jused > 0) {
      for (int i = jused - 1; i >= 0; --i) {
        double acc = g[i];
        for (int q = i + 1; q < jused; ++q) acc -= Hm(i, q) * y[q];
        y[i] = acc / Hm(i, i);
      }
      launch_gemv_acc(x, Z, m, jused, y.data(), m, s);
      prof_note(c, 8.0 * (jused + 2) * (double)m);
      IBM_LAUNCH_CHECK(c);
    }
    ++cycles;
    if (breakdown && jused == 0) { final_status = IBM_ERR_BREAKDOWN; break; }
  }
  // mean-zero projection (S~ annihilates constants)
  if (c->defer_mean) {
    launch_sum(x, m, part, c->defer_mean, s);   // the caller removes the mean
    prof_note(c, 8.0 * m);
  } else {
    launch_sum(x, m, part, sdev, s);
    launch_add_scalar_dev(x, m, sdev, -1.0 / (double)m, s);
    prof_note(c, 24.0 * m);
  }
  IBM_LAUNCH_CHECK(c);
  if (st) {
    st->iters = total;
    st->restarts = cycles;
    st->graph_cycles = 0;
    st->relres_true = relres;
  }
  if (final_status != IBM_OK) return set_err(c, final_status, "FGMRES breakdown");
  if (!converged) {
    char buf[160];
    snprintf(buf, sizeof buf, "FGMRES did not reach rtol %.3g in %d iterations (relres %.3g)",
             o->rtol, total, relres);
    return set_err(c, IBM_ERR_NOT_CONVERGED, buf);
  }
  return IBM_OK;
}

}  // namespace ibm
