// Geometric-multigrid V-cycle for the Neumann Laplacian L = G^T G, used as the
// preconditioner "z ~ L^{-1} r" of Sec. 4.1.  The paper applies an exact
// direct solver (Sec. 4.2) and names a geometric-multigrid V-cycle as its
// replacement (Sec. 7); FGMRES tolerates the inexact, FP32 form.
//
// Cell-centred hierarchy (each level halves every axis), coarse operators
// re-discretised (7-point with width 2^l h), 8-cell averaging restriction,
// trilinear (3/4, 1/4 per axis) prolongation with reflection at the walls,
// Chebyshev-Richardson smoothing on D^{-1} L with the polynomial's roots on
// [0.3, 2] (the upper end is the Gershgorin bound of D^{-1} L), and a dense
// pseudo-inverse on the coarsest level (<= 512 cells).  Templates cover the
// FP32 (mixed) and FP64 forms; only the inputs/outputs at the finest level are
// FP64 in the mixed form.
#include <cmath>
#include <vector>

#include "ibm_internal.cuh"

namespace ibm {

namespace {

constexpr int BX = 32, BY = 8;
constexpr double kChebLo = 0.3, kChebHi = 2.0;

dim3 grid3(Dims d) { return dim3(div_up(d.nx, BX), div_up(d.ny, BY), d.nz); }

// Chebyshev-Richardson weights 1/lambda_i, lambda_i the roots of the degree-p
// Chebyshev polynomial mapped to [lo, hi].
void cheb_weights(int p, double* w) {
  for (int i = 0; i < p; ++i) {
    const double th = (2.0 * i + 1.0) * M_PI / (2.0 * p);
    const double lam = 0.5 * (kChebHi + kChebLo) + 0.5 * (kChebHi - kChebLo) * std::cos(th);
    w[i] = 1.0 / lam;
  }
}

// Neighbour sum and count of the Neumann 7-point stencil at cell (i, j, k).
template <typename T>
__device__ __forceinline__ T nb_sum(Dims d, const T* __restrict__ x, int64_t c, int i, int j, int k,
                                    int& nn) {
  const int64_t sy = d.nx, sz = (int64_t)d.nx * d.ny;
  T s = 0;
  nn = 0;
  if (i > 0) { s += __ldg(x + c - 1); ++nn; }
  if (i < d.nx - 1) { s += __ldg(x + c + 1); ++nn; }
  if (j > 0) { s += __ldg(x + c - sy); ++nn; }
  if (j < d.ny - 1) { s += __ldg(x + c + sy); ++nn; }
  if (k > 0) { s += __ldg(x + c - sz); ++nn; }
  if (k < d.nz - 1) { s += __ldg(x + c + sz); ++nn; }
  return s;
}

// x = w D^{-1} b   (first sweep from a zero iterate)
template <typename T>
__global__ void __launch_bounds__(BX * BY) k_cheb_first(Dims d, const T* __restrict__ b,
                                                        T* __restrict__ x, T w_h2) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= d.nx || j >= d.ny) return;
  const int nn = (i > 0) + (i < d.nx - 1) + (j > 0) + (j < d.ny - 1) + (k > 0) + (k < d.nz - 1);
  const int64_t c = ((int64_t)k * d.ny + j) * d.nx + i;
  x[c] = w_h2 * __ldg(b + c) / (T)nn;
}

// xo = x + w D^{-1} (b - L x),  D = nn / h^2, L x = (nn x_c - sum) / h^2
template <typename T>
__global__ void __launch_bounds__(BX * BY) k_cheb_sweep(Dims d, const T* __restrict__ x,
                                                        const T* __restrict__ b,
                                                        T* __restrict__ xo, T w, T h2) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= d.nx || j >= d.ny) return;
  const int64_t c = ((int64_t)k * d.ny + j) * d.nx + i;
  int nn;
  const T s = nb_sum(d, x, c, i, j, k, nn);
  const T xc = __ldg(x + c);
  // D^{-1}(b - Lx) = (h^2 b - nn xc + s) / nn
  const T r = fma(h2, __ldg(b + c), s - (T)nn * xc);
  xo[c] = fma(w, r / (T)nn, xc);
}

// bc = average over the 8 children of (b - L x); x == nullptr means x = 0.
template <typename T>
__global__ void __launch_bounds__(BX * BY) k_resid_restrict(Dims d, Dims dc,
                                                            const T* __restrict__ x,
                                                            const T* __restrict__ b,
                                                            T* __restrict__ bcoarse, T inv_h2) {
  const int I = blockIdx.x * BX + threadIdx.x;
  const int J = blockIdx.y * BY + threadIdx.y;
  const int K = blockIdx.z;
  if (I >= dc.nx || J >= dc.ny) return;
  T acc = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int i = 2 * I + (q & 1), j = 2 * J + ((q >> 1) & 1), k = 2 * K + (q >> 2);
    const int64_t c = ((int64_t)k * d.ny + j) * d.nx + i;
    T r = __ldg(b + c);
    if (x) {
      int nn;
      const T s = nb_sum(d, x, c, i, j, k, nn);
      r -= ((T)nn * __ldg(x + c) - s) * inv_h2;
    }
    acc += r;
  }
  bcoarse[((int64_t)K * dc.ny + J) * dc.nx + I] = acc * (T)0.125;
}

// x += P xc  (trilinear, weights 3/4 parent and 1/4 neighbour per axis; at a
// wall the neighbour is the parent itself).  x == nullptr-free form: if
// overwrite != 0 then x = P xc.
template <typename T>
__global__ void __launch_bounds__(BX * BY) k_prolong(Dims d, Dims dc, const T* __restrict__ xc,
                                                     T* __restrict__ x, int overwrite) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= d.nx || j >= d.ny) return;
  const int I = i >> 1, J = j >> 1, K = k >> 1;
  const int In = (i & 1) ? min(I + 1, dc.nx - 1) : max(I - 1, 0);
  const int Jn = (j & 1) ? min(J + 1, dc.ny - 1) : max(J - 1, 0);
  const int Kn = (k & 1) ? min(K + 1, dc.nz - 1) : max(K - 1, 0);
  const int64_t sy = dc.nx, sz = (int64_t)dc.nx * dc.ny;
  const T* p0 = xc + K * sz;
  const T* p1 = xc + Kn * sz;
  const T a00 = (T)0.75 * __ldg(p0 + J * sy + I) + (T)0.25 * __ldg(p0 + J * sy + In);
  const T a01 = (T)0.75 * __ldg(p0 + Jn * sy + I) + (T)0.25 * __ldg(p0 + Jn * sy + In);
  const T a10 = (T)0.75 * __ldg(p1 + J * sy + I) + (T)0.25 * __ldg(p1 + J * sy + In);
  const T a11 = (T)0.75 * __ldg(p1 + Jn * sy + I) + (T)0.25 * __ldg(p1 + Jn * sy + In);
  const T b0 = (T)0.75 * a00 + (T)0.25 * a01;
  const T b1 = (T)0.75 * a10 + (T)0.25 * a11;
  const T v = (T)0.75 * b0 + (T)0.25 * b1;
  const int64_t c = ((int64_t)k * d.ny + j) * d.nx + i;
  x[c] = overwrite ? v : x[c] + v;
}

// x = P b on the coarsest level: one block, dense pseudo-inverse.
template <typename T>
__global__ void k_coarse_solve(const T* __restrict__ P, const T* __restrict__ b,
                               T* __restrict__ x, int mc) {
  __shared__ T sb[kMaxCoarse];
  for (int q = threadIdx.x; q < mc; q += blockDim.x) sb[q] = b[q];
  __syncthreads();
  for (int r = threadIdx.x; r < mc; r += blockDim.x) {
    T acc = 0;
    for (int q = 0; q < mc; ++q) acc = fma(__ldg(P + (int64_t)r * mc + q), sb[q], acc);
    x[r] = acc;
  }
}

__global__ void k_d2f(const double* __restrict__ x, float* __restrict__ y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}
__global__ void k_f2d(const float* __restrict__ x, double* __restrict__ y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (double)x[i];
}

// Gauss-Jordan inverse with partial pivoting (host, n <= kMaxCoarse).
bool invert_dense(std::vector<double>& A, int n) {
  std::vector<double> inv((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0;
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (std::fabs(A[(size_t)r * n + col]) > std::fabs(A[(size_t)piv * n + col])) piv = r;
    if (A[(size_t)piv * n + col] == 0.0) return false;
    if (piv != col)
      for (int q = 0; q < n; ++q) {
        std::swap(A[(size_t)piv * n + q], A[(size_t)col * n + q]);
        std::swap(inv[(size_t)piv * n + q], inv[(size_t)col * n + q]);
      }
    const double dinv = 1.0 / A[(size_t)col * n + col];
    for (int q = 0; q < n; ++q) {
      A[(size_t)col * n + q] *= dinv;
      inv[(size_t)col * n + q] *= dinv;
    }
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      const double f = A[(size_t)r * n + col];
      if (f == 0.0) continue;
      for (int q = 0; q < n; ++q) {
        A[(size_t)r * n + q] -= f * A[(size_t)col * n + q];
        inv[(size_t)r * n + q] -= f * inv[(size_t)col * n + q];
      }
    }
  }
  A.swap(inv);
  return true;
}

template <typename T>
struct LevelPtrs {
  T* x;
  T* b;
  T* t;
};

template <typename T>
LevelPtrs<T> ptrs(MGLevel& L);
template <>
LevelPtrs<float> ptrs<float>(MGLevel& L) { return {L.x32, L.b32, L.t32}; }
template <>
LevelPtrs<double> ptrs<double>(MGLevel& L) { return {L.x64, L.b64, L.t64}; }

template <typename T>
const T* pinv_of(ibm_ctx* c);
template <>
const float* pinv_of<float>(ibm_ctx* c) { return c->coarse_pinv32; }
template <>
const double* pinv_of<double>(ibm_ctx* c) { return c->coarse_pinv64; }

// p Chebyshev sweeps on level l starting from *x (zero if from_zero); the
// result ends in *x (the sweep ping-pongs with *t and copies back if needed).
template <typename T>
void smooth(ibm_ctx* c, int l, const T* b, T* x, T* t, int p, bool from_zero, cudaStream_t s) {
  if (p <= 0) return;
  MGLevel& L = c->lv[l];
  double w[8];
  cheb_weights(p, w);
  const double h2 = L.h * L.h;
  T* cur = x;
  T* nxt = t;
  int q = 0;
  if (from_zero) {
    count_launch();
    k_cheb_first<T><<<grid3(L.d), dim3(BX, BY), 0, s>>>(L.d, b, x, (T)(w[0] * h2));
    q = 1;
  }
  for (; q < p; ++q) {
    const int ph = l == 0 ? prof_begin(c, IBM_PROF_MG_SMOOTH_FINE) : -1;
    count_launch();
    k_cheb_sweep<T><<<grid3(L.d), dim3(BX, BY), 0, s>>>(L.d, cur, b, nxt, (T)w[q], (T)h2);
    prof_end(c, ph);
    T* tmp = cur; cur = nxt; nxt = tmp;
  }
  if (cur != x) cudaMemcpyAsync(x, cur, sizeof(T) * L.m, cudaMemcpyDeviceToDevice, s);
}

// V-cycle on level l: x_l ~ L_l^{-1} b_l.
template <typename T>
void vcycle(ibm_ctx* c, int l, const T* b, T* x, T* t, int pre, int post, cudaStream_t s) {
  MGLevel& L = c->lv[l];
  if (l == c->n_levels - 1) {
    count_launch();
    k_coarse_solve<T><<<1, 256, 0, s>>>(pinv_of<T>(c), b, x, c->coarse_m);
    return;
  }
  MGLevel& C = c->lv[l + 1];
  LevelPtrs<T> cp = ptrs<T>(C);
  smooth<T>(c, l, b, x, t, pre, true, s);
  count_launch();
  k_resid_restrict<T><<<grid3(C.d), dim3(BX, BY), 0, s>>>(L.d, C.d, pre > 0 ? x : nullptr, b, cp.b,
                                                          (T)(1.0 / (L.h * L.h)));
  vcycle<T>(c, l + 1, cp.b, cp.x, cp.t, pre, post, s);
  count_launch();
  k_prolong<T><<<grid3(L.d), dim3(BX, BY), 0, s>>>(L.d, C.d, cp.x, x, pre > 0 ? 0 : 1);
  smooth<T>(c, l, b, x, t, post, false, s);
}

}  // namespace

ibm_status mg_setup(ibm_ctx* c) {
  // levels: halve while every axis is even and the level has > 64 cells
  Dims d = c->d;
  double h = c->h;
  int n = 0;
  while (true) {
    if (n >= kMaxLevels) return set_err(c, IBM_ERR_ARG, "too many multigrid levels");
    MGLevel& L = c->lv[n];
    L.d = d;
    L.h = h;
    L.m = cells_of(d);
    ++n;
    const bool can = (d.nx % 2 == 0) && (d.ny % 2 == 0) && (d.nz % 2 == 0) && d.nx >= 4 &&
                     d.ny >= 4 && d.nz >= 4 && L.m > 64;
    if (!can) break;
    d = Dims{d.nx / 2, d.ny / 2, d.nz / 2};
    h *= 2.0;
  }
  c->n_levels = n;
  MGLevel& Lc = c->lv[n - 1];
  if (Lc.m > kMaxCoarse)
    return set_err(c, IBM_ERR_ARG,
                   "grid must coarsen (halving all axes) to at most 512 cells; use dimensions "
                   "of the form q * 2^k with small q");
  for (int l = 0; l < n; ++l) {
    MGLevel& L = c->lv[l];
    if (cudaMalloc(&L.x32, sizeof(float) * L.m) != cudaSuccess ||
        cudaMalloc(&L.b32, sizeof(float) * L.m) != cudaSuccess ||
        cudaMalloc(&L.t32, sizeof(float) * L.m) != cudaSuccess ||
        cudaMalloc(&L.x64, sizeof(double) * L.m) != cudaSuccess ||
        cudaMalloc(&L.b64, sizeof(double) * L.m) != cudaSuccess ||
        cudaMalloc(&L.t64, sizeof(double) * L.m) != cudaSuccess) {
      cudaGetLastError();
      return set_err(c, IBM_ERR_NOMEM, "multigrid allocation failed");
    }
  }
  // dense pseudo-inverse of the coarsest Neumann Laplacian:
  // L^+ = (L + 1 1^T / mc)^{-1} - 1 1^T / mc
  const int mc = (int)Lc.m;
  c->coarse_m = mc;
  std::vector<double> A((size_t)mc * mc, 1.0 / mc);
  const double ih2 = 1.0 / (Lc.h * Lc.h);
  for (int k = 0; k < Lc.d.nz; ++k)
    for (int j = 0; j < Lc.d.ny; ++j)
      for (int i = 0; i < Lc.d.nx; ++i) {
        const int r = (k * Lc.d.ny + j) * Lc.d.nx + i;
        const int nb[6][3] = {{i - 1, j, k}, {i + 1, j, k}, {i, j - 1, k},
                              {i, j + 1, k}, {i, j, k - 1}, {i, j, k + 1}};
        for (auto& q : nb) {
          if (q[0] < 0 || q[0] >= Lc.d.nx || q[1] < 0 || q[1] >= Lc.d.ny || q[2] < 0 ||
              q[2] >= Lc.d.nz)
            continue;
          const int cq = (q[2] * Lc.d.ny + q[1]) * Lc.d.nx + q[0];
          A[(size_t)r * mc + r] += ih2;
          A[(size_t)r * mc + cq] -= ih2;
        }
      }
  if (!invert_dense(A, mc)) return set_err(c, IBM_ERR_ARG, "coarse operator is singular");
  for (auto& v : A) v -= 1.0 / mc;
  std::vector<float> A32(A.begin(), A.end());
  if (cudaMalloc(&c->coarse_pinv64, sizeof(double) * mc * mc) != cudaSuccess ||
      cudaMalloc(&c->coarse_pinv32, sizeof(float) * mc * mc) != cudaSuccess) {
    cudaGetLastError();
    return set_err(c, IBM_ERR_NOMEM, "coarse operator allocation failed");
  }
  IBM_CUDA(c, cudaMemcpy(c->coarse_pinv64, A.data(), sizeof(double) * mc * mc,
                         cudaMemcpyHostToDevice));
  IBM_CUDA(c, cudaMemcpy(c->coarse_pinv32, A32.data(), sizeof(float) * mc * mc,
                         cudaMemcpyHostToDevice));
  return IBM_OK;
}

ibm_status mg_vcycle(ibm_ctx* c, const double* r, double* z, int prec, int pre, int post) {
  cudaStream_t s = c->stream;
  MGLevel& L0 = c->lv[0];
  if (prec == IBM_PREC_FP32) {
    count_launch();
    k_d2f<<<kRedBlocks, 256, 0, s>>>(r, L0.b32, L0.m);
    vcycle<float>(c, 0, L0.b32, L0.x32, L0.t32, pre, post, s);
    count_launch();
    k_f2d<<<kRedBlocks, 256, 0, s>>>(L0.x32, z, L0.m);
  } else {
    vcycle<double>(c, 0, r, z, L0.t64, pre, post, s);
  }
  IBM_LAUNCH_CHECK(c);
  return IBM_OK;
}

}  // namespace ibm
