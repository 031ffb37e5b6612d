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
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "ibm_internal.cuh"

namespace ibm {

namespace {

constexpr int BX = 32, BY = 8;
constexpr double kChebLo = 0.3, kChebHi = 2.0;


// Chebyshev-Richardson weights 1/lambda_i, lambda_i the roots of the degree-p
// Chebyshev polynomial mapped to [lo, hi].
void cheb_weights(int p, double* w) {
  for (int i = 0; i < p; ++i) {
    const double th = (2.0 * i + 1.0) * M_PI / (2.0 * p);
    const double lam = 0.5 * (kChebHi + kChebLo) + 0.5 * (kChebHi - kChebLo) * std::cos(th);
    w[i] = 1.0 / lam;
  }
}

// All level kernels march along z: a block of 32 x 8 threads owns a 32 x 8
// column of cells over ZC consecutive planes, each thread keeps the planes
// below, at and above its cell in registers, and the in-plane neighbours come
// through L1.  One DRAM read per input array per cell, with several planes'
// loads in flight per thread.
constexpr int ZC = 16;

dim3 zm_grid(Dims d) { return dim3(div_up(d.nx, BX), div_up(d.ny, BY), div_up(d.nz, ZC)); }

// w / nn for nn = 0..6 (nn = number of existing neighbours of a cell).
template <typename T>
struct WOverN {
  T v[7];
};

template <typename T>
WOverN<T> w_over_n(double w) {
  WOverN<T> r;
  r.v[0] = (T)0;
  for (int q = 1; q < 7; ++q) r.v[q] = (T)(w / q);
  return r;
}

// w / nn from the table with static indices only (a dynamically indexed
// kernel-parameter array would be copied to local memory): interior cells
// (nn = 6) use the stored quotient, boundary cells divide.
template <typename T>
__device__ __forceinline__ T wn_of(const WOverN<T>& wn, int nn) {
  return nn == 6 ? wn.v[6] : wn.v[1] / (T)nn;
}

__device__ __forceinline__ int n_inplane(Dims d, int i, int j) {
  return (i > 0) + (i < d.nx - 1) + (j > 0) + (j < d.ny - 1);
}

template <typename T>
__device__ __forceinline__ T inplane_sum(const T* __restrict__ p, int64_t c, int i, int j, Dims d,
                                         int64_t sy) {
  T s = 0;
  if (i > 0) s += __ldg(p + c - 1);
  if (i < d.nx - 1) s += __ldg(p + c + 1);
  if (j > 0) s += __ldg(p + c - sy);
  if (j < d.ny - 1) s += __ldg(p + c + sy);
  return s;
}

// One Chebyshev-Richardson step: xo = x + w D^{-1} (b - L x), D = nn / h^2,
// L x = (nn x_c - sum of neighbours) / h^2.  b may be FP64 while T is FP32,
// and the output type TO may differ from T (FP64 result of the mixed cycle).
template <typename T, typename TB, typename TO>
__global__ void __launch_bounds__(BX * BY) k_sweep(Dims d, const T* __restrict__ x,
                                                   const TB* __restrict__ b, TO* __restrict__ xo,
                                                   WOverN<T> wn, T h2) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  if (i >= d.nx || j >= d.ny) return;
  const int z0 = blockIdx.z * ZC;
  const int z1 = min(z0 + ZC, d.nz);
  const int64_t sy = d.nx, sz = (int64_t)d.nx * d.ny;
  const int nip = n_inplane(d, i, j);
  int64_t c = (int64_t)z0 * sz + (int64_t)j * sy + i;
  T xp = z0 > 0 ? __ldg(x + c - sz) : (T)0;
  T xc = __ldg(x + c);
#pragma unroll 4
  for (int z = z0; z < z1; ++z, c += sz) {
    const T xn = (z + 1 < d.nz) ? __ldg(x + c + sz) : (T)0;
    const int nn = nip + (z > 0) + (z < d.nz - 1);
    const T s = inplane_sum(x, c, i, j, d, sy) + (xp + xn);
    const T r = fma(h2, (T)__ldg(b + c), s - (T)nn * xc);
    xo[c] = (TO)fma(wn_of(wn, nn), r, xc);
    xp = xc;
    xc = xn;
  }
}

// First smoothing step(s) from a zero iterate.  x1 = w0 D^{-1} b pointwise; with
// two != 0 also the second step xo = x1 + w1 D^{-1} (b - L x1), evaluating x1 at
// the neighbours from b on the fly (no x1 array).  bcopy (may be null) receives
// b rounded to T, for the later kernels of the level.
template <typename T, typename TB>
__global__ void __launch_bounds__(BX * BY) k_first(Dims d, const TB* __restrict__ b,
                                                   T* __restrict__ bcopy, T* __restrict__ xo,
                                                   WOverN<T> w0h2n, WOverN<T> w1n, T h2, int two) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  if (i >= d.nx || j >= d.ny) return;
  const int z0 = blockIdx.z * ZC;
  const int z1 = min(z0 + ZC, d.nz);
  const int64_t sy = d.nx, sz = (int64_t)d.nx * d.ny;
  const int nip = n_inplane(d, i, j);
  int64_t c = (int64_t)z0 * sz + (int64_t)j * sy + i;
  if (!two) {
    for (int z = z0; z < z1; ++z, c += sz) {
      const T bv = (T)__ldg(b + c);
      if (bcopy) bcopy[c] = bv;
      xo[c] = wn_of(w0h2n, nip + (z > 0) + (z < d.nz - 1)) * bv;
    }
    return;
  }
  // in-plane neighbour counts of the four in-plane neighbours
  const int nxm = i > 0 ? n_inplane(d, i - 1, j) : 0;
  const int nxp = i < d.nx - 1 ? n_inplane(d, i + 1, j) : 0;
  const int nym = j > 0 ? n_inplane(d, i, j - 1) : 0;
  const int nyp = j < d.ny - 1 ? n_inplane(d, i, j + 1) : 0;
  auto nzc = [&](int z) { return (z > 0) + (z < d.nz - 1); };
  // x1 below / at / above, carried along z
  T x1p = z0 > 0 ? wn_of(w0h2n, nip + nzc(z0 - 1)) * (T)__ldg(b + c - sz) : (T)0;
  T bcv = (T)__ldg(b + c);
  T x1c = wn_of(w0h2n, nip + nzc(z0)) * bcv;
#pragma unroll 2
  for (int z = z0; z < z1; ++z, c += sz) {
    T bnv = 0, x1n = 0;
    if (z + 1 < d.nz) {
      bnv = (T)__ldg(b + c + sz);
      x1n = wn_of(w0h2n, nip + nzc(z + 1)) * bnv;
    }
    const int zc = nzc(z);
    T s = x1p + x1n;
    if (i > 0) s += wn_of(w0h2n, nxm + zc) * (T)__ldg(b + c - 1);
    if (i < d.nx - 1) s += wn_of(w0h2n, nxp + zc) * (T)__ldg(b + c + 1);
    if (j > 0) s += wn_of(w0h2n, nym + zc) * (T)__ldg(b + c - sy);
    if (j < d.ny - 1) s += wn_of(w0h2n, nyp + zc) * (T)__ldg(b + c + sy);
    const int nn = nip + zc;
    if (bcopy) bcopy[c] = bcv;
    const T r = fma(h2, bcv, s - (T)nn * x1c);
    xo[c] = fma(wn_of(w1n, nn), r, x1c);
    x1p = x1c;
    x1c = x1n;
    bcv = bnv;
  }
}

// Residual restriction: bcoarse = average over the 8 children of (b - L x);
// x == nullptr means x = 0.  One thread per coarse cell; the children are read
// in x-pairs (2I, 2I+1).
template <typename T>
struct Pair;
template <>
struct Pair<float> {
  using type = float2;
};
template <>
struct Pair<double> {
  using type = double2;
};

template <typename T>
__device__ __forceinline__ void ld2(const T* p, T& a, T& b) {
  const typename Pair<T>::type v = __ldg(reinterpret_cast<const typename Pair<T>::type*>(p));
  a = v.x;
  b = v.y;
}

template <typename T>
__global__ void __launch_bounds__(BX * BY) k_restrict(Dims d, Dims dc, const T* __restrict__ x,
                                                      const T* __restrict__ b,
                                                      T* __restrict__ bcoarse, T inv_h2) {
  const int I = blockIdx.x * BX + threadIdx.x;
  const int J = blockIdx.y * BY + threadIdx.y;
  if (I >= dc.nx || J >= dc.ny) return;
  const int64_t sy = d.nx, sz = (int64_t)d.nx * d.ny;
  const int K0 = blockIdx.z * (ZC / 2);
  const int K1 = min(K0 + ZC / 2, dc.nz);
  for (int K = K0; K < K1; ++K) {
    T acc = 0;
#pragma unroll
    for (int dz = 0; dz < 2; ++dz) {
      const int k = 2 * K + dz;
#pragma unroll
      for (int dy = 0; dy < 2; ++dy) {
        const int j = 2 * J + dy;
        const int64_t c = (int64_t)k * sz + (int64_t)j * sy + 2 * I;
        T b0, b1;
        ld2(b + c, b0, b1);
        T r0 = b0, r1 = b1;
        if (x) {
          T x0, x1;
          ld2(x + c, x0, x1);
          // neighbours of the pair
          T s0 = x1, s1 = x0;
          int n0 = 1, n1 = 1;
          if (2 * I > 0) { s0 += __ldg(x + c - 1); ++n0; }
          if (2 * I + 2 < d.nx) { s1 += __ldg(x + c + 2); ++n1; }
          T a0, a1;
          if (j > 0) { ld2(x + c - sy, a0, a1); s0 += a0; s1 += a1; ++n0; ++n1; }
          if (j < d.ny - 1) { ld2(x + c + sy, a0, a1); s0 += a0; s1 += a1; ++n0; ++n1; }
          if (k > 0) { ld2(x + c - sz, a0, a1); s0 += a0; s1 += a1; ++n0; ++n1; }
          if (k < d.nz - 1) { ld2(x + c + sz, a0, a1); s0 += a0; s1 += a1; ++n0; ++n1; }
          r0 -= ((T)n0 * x0 - s0) * inv_h2;
          r1 -= ((T)n1 * x1 - s1) * inv_h2;
        }
        acc += r0 + r1;
      }
    }
    bcoarse[((int64_t)K * dc.ny + J) * dc.nx + I] = acc * (T)0.125;
  }
}

template <typename T, typename TO>
__global__ void k_convert(const T* __restrict__ x, TO* __restrict__ y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (TO)x[i];
}

// x (+)= P xc: trilinear, 3/4 parent and 1/4 neighbour per axis, the
// neighbour replaced by the parent at a wall.  One thread per fine x-pair
// (2I, 2I+1), which share the parent I; overwrite != 0 gives x = P xc.
template <typename T>
__global__ void __launch_bounds__(BX * BY) k_prolong(Dims d, Dims dc, const T* __restrict__ xc,
                                                     T* __restrict__ x, int overwrite) {
  const int I = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  if (I >= dc.nx || j >= d.ny) return;
  const int z0 = blockIdx.z * ZC;
  const int z1 = min(z0 + ZC, d.nz);
  const int J = j >> 1;
  const int Jn = (j & 1) ? min(J + 1, dc.ny - 1) : max(J - 1, 0);
  const int Im = max(I - 1, 0), Ip = min(I + 1, dc.nx - 1);
  const int64_t sy = dc.nx, sz = (int64_t)dc.nx * dc.ny;
  for (int k = z0; k < z1; ++k) {
    const int K = k >> 1;
    const int Kn = (k & 1) ? min(K + 1, dc.nz - 1) : max(K - 1, 0);
    // rows (J, K), (Jn, K), (J, Kn), (Jn, Kn); 3/4-1/4 in y and z first
    const T* r00 = xc + K * sz + J * sy;
    const T* r01 = xc + K * sz + Jn * sy;
    const T* r10 = xc + Kn * sz + J * sy;
    const T* r11 = xc + Kn * sz + Jn * sy;
    auto yz = [&](int q) {
      const T a = (T)0.75 * __ldg(r00 + q) + (T)0.25 * __ldg(r01 + q);
      const T bb = (T)0.75 * __ldg(r10 + q) + (T)0.25 * __ldg(r11 + q);
      return (T)0.75 * a + (T)0.25 * bb;
    };
    const T cm = yz(Im), c0 = yz(I), cp = yz(Ip);
    const T v0 = (T)0.75 * c0 + (T)0.25 * cm;   // fine 2I   (neighbour I-1)
    const T v1 = (T)0.75 * c0 + (T)0.25 * cp;   // fine 2I+1 (neighbour I+1)
    const int64_t f = ((int64_t)k * d.ny + j) * d.nx + 2 * I;
    typename Pair<T>::type* px = reinterpret_cast<typename Pair<T>::type*>(x + f);
    typename Pair<T>::type o;
    if (overwrite) {
      o.x = v0;
      o.y = v1;
    } else {
      o = *px;
      o.x += v0;
      o.y += v1;
    }
    *px = o;
  }
}

// ---------------------------------------------------------------------------
// FP32 kernels for levels whose x-extent is a multiple of 4: each thread owns
// four consecutive cells (one float4) of a row, a warp 128 cells, a block
// 128 x VY cells over zc planes.  x-neighbours come from the adjacent lanes by
// shuffles (scalar loads at the warp edges), z-neighbours from the registers
// of the march, y-neighbours from L1.  16-byte loads keep enough bytes in
// flight per SM to run near the DRAM bandwidth.
constexpr int VY = 8;
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float4 ld4(const float* p) {
  return __ldg(reinterpret_cast<const float4*>(p));
}
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ void st4(double* p, float4 v) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v.x, v.y);
  reinterpret_cast<double2*>(p)[1] = make_double2(v.z, v.w);
}
__device__ __forceinline__ float4 ld4_any(const float* p) { return ld4(p); }
__device__ __forceinline__ float4 ld4_any(const double* p) {
  const double2 a = __ldg(reinterpret_cast<const double2*>(p));
  const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
  return make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
}
// leading parts of four interleaved (hi, lo) pairs
__device__ __forceinline__ float4 ld4_any(const float2* p) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(p));
  const float4 b = __ldg(reinterpret_cast<const float4*>(p) + 1);
  return make_float4(a.x, a.z, b.x, b.z);
}
__device__ __forceinline__ float ld1_any(const float2* p) { return __ldg(p).x; }
__device__ __forceinline__ float ld1_any(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ld1_any(const double* p) { return (float)__ldg(p); }

// w / nn without division or dynamic indexing (nn in 1..6; 6 is the
// interior case): 1/nn by a chain of selects
__device__ __forceinline__ float inv_nn(int nn) {
  return nn >= 6 ? (1.f / 6.f)
                 : (nn == 5 ? 0.2f : (nn == 4 ? 0.25f : (nn == 3 ? (1.f / 3.f) : (nn == 2 ? 0.5f : 1.f))));
}
__device__ __forceinline__ float w_over(float w, int nn) { return w * inv_nn(nn); }

// Planes per thread of the four-cell kernels: about IBM_VEC_ZC_BLOCKS blocks
// per SM over the grid, at most kVecZcMax (each thread loads the planes
// above and below its first and last ones once more, and sets up its weights
// once).  With eight, levels of 128^3 cells and below get one plane per
// thread: there the kernels wait on memory latency rather than on bandwidth
// or instruction issue, and more blocks in flight hide more of it.
#ifndef IBM_VEC_ZC_MAX
#define IBM_VEC_ZC_MAX 4
#endif
constexpr int kVecZcMax = IBM_VEC_ZC_MAX;
#ifndef IBM_VEC_ZC_BLOCKS
#define IBM_VEC_ZC_BLOCKS 8
#endif
int vec_zc(Dims d) {
  const int64_t bxy = (int64_t)div_up(d.nx / 4, 32) * div_up(d.ny, VY);
  int64_t zc = (int64_t)d.nz * bxy / (152 * IBM_VEC_ZC_BLOCKS);
  zc = zc < 1 ? 1 : (zc > kVecZcMax ? kVecZcMax : zc);
  return (int)zc;
}

dim3 vec_grid(Dims d, int zc) {
  return dim3(div_up(d.nx / 4, 32), div_up(d.ny, VY), div_up(d.nz, zc));
}

bool vec_ok(Dims d) { return d.nx % 4 == 0; }

// xo = x + w D^{-1} (b - L x) for four cells per thread.  Rows and planes
// away from the y and z walls (a warp-uniform test) take a path whose
// weights and neighbour counts are per-thread constants and whose loads
// need no wall test.
// ZC > 0: exactly ZC planes per thread (the march unrolled at compile time;
// the launch's zc equals ZC); ZC = 0: zc planes at run time.
template <typename TO, int ZC = 0>
__global__ void __launch_bounds__(32 * VY) k_sweep_v4(Dims d, const float* __restrict__ x,
                                                      const float* __restrict__ b,
                                                      TO* __restrict__ xo, float w, float h2,
                                                      int zc) {
  pdl_wait();
  pdl_trigger();
  const int lane = threadIdx.x;
  const int i0 = 4 * (blockIdx.x * 32 + lane);
  const int j = blockIdx.y * VY + threadIdx.y;
  const bool act = i0 < d.nx && j < d.ny;
  const int z0 = blockIdx.z * zc;
  const int z1 = min(z0 + zc, d.nz);
  const int64_t sy = d.nx, sz = (int64_t)d.nx * d.ny;
  int64_t c = (int64_t)z0 * sz + (int64_t)j * sy + i0;
  const float4 Z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  // x-counts of the four cells; on rows/planes away from the y and z walls
  // the neighbour count is 4 + x-count and the weight w/nn is fixed per thread
  int ax[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) ax[q] = (i0 + q > 0) + (i0 + q < d.nx - 1);
  float wi[4], nni[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    wi[q] = w_over(w, ax[q] + 4);
    nni[q] = (float)(ax[q] + 4);
  }
  const int ny_c = (j > 0) + (j < d.ny - 1);
  const bool yin = ny_c == 2;
  float4 xp = (act && z0 > 0) ? ld4(x + c - sz) : Z4;
  float4 xc = act ? ld4(x + c) : Z4;
  constexpr int kUnroll = ZC > 0 ? ZC : 1;
#pragma unroll kUnroll
  for (int zz = 0; zz < (ZC > 0 ? ZC : zc); ++zz) {
    const int z = z0 + zz;
    if (z >= z1) break;
    const bool inner = yin && z > 0 && z < d.nz - 1;
    float4 xn = Z4, ym = Z4, yp = Z4, bb = Z4;
    if (inner) {
      if (act) {
        xn = ld4(x + c + sz);
        ym = ld4(x + c - sy);
        yp = ld4(x + c + sy);
        bb = ld4(b + c);
      }
    } else if (act) {
      if (z + 1 < d.nz) xn = ld4(x + c + sz);
      if (j > 0) ym = ld4(x + c - sy);
      if (j < d.ny - 1) yp = ld4(x + c + sy);
      bb = ld4(b + c);
    }
    float left = __shfl_up_sync(kFull, xc.w, 1);
    float right = __shfl_down_sync(kFull, xc.x, 1);
    if (lane == 0) left = (act && i0 > 0) ? __ldg(x + c - 1) : 0.f;
    if (lane == 31) right = (act && i0 + 4 < d.nx) ? __ldg(x + c + 4) : 0.f;
    const float xv[4] = {xc.x, xc.y, xc.z, xc.w};
    const float xl[4] = {left, xc.x, xc.y, xc.z};
    const float xr[4] = {xc.y, xc.z, xc.w, right};
    const float vym[4] = {ym.x, ym.y, ym.z, ym.w};
    const float vyp[4] = {yp.x, yp.y, yp.z, yp.w};
    const float vzp[4] = {xp.x, xp.y, xp.z, xp.w};
    const float vzn[4] = {xn.x, xn.y, xn.z, xn.w};
    const float vb[4] = {bb.x, bb.y, bb.z, bb.w};
    float o[4];
    if (inner) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float s = (xl[q] + xr[q]) + (vym[q] + vyp[q]) + (vzp[q] + vzn[q]);
        o[q] = fmaf(wi[q], fmaf(h2, vb[q], s - nni[q] * xv[q]), xv[q]);
      }
    } else {
      const int zn = (z > 0) + (z < d.nz - 1);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int nn = ax[q] + ny_c + zn;
        const float s = (xl[q] + xr[q]) + (vym[q] + vyp[q]) + (vzp[q] + vzn[q]);
        o[q] = fmaf(w_over(w, nn), fmaf(h2, vb[q], s - (float)nn * xv[q]), xv[q]);
      }
    }
    if (act) st4(xo + c, make_float4(o[0], o[1], o[2], o[3]));
    xp = xc;
    xc = xn;
    c += sz;
  }
}

// First smoothing step(s) from a zero iterate (see k_first), four cells per
// thread.  b may be FP64: each value is rounded once; x-neighbours move
// between lanes by shuffles, the block's rows (and the two y-halo rows) are
// staged as float4 in shared memory for the y-neighbours, z by the march.
template <typename TB, int ZC = 0>
__global__ void __launch_bounds__(32 * VY, 4) k_first_v4(Dims d, const TB* __restrict__ b,
                                                      float* __restrict__ bcopy,
                                                      float* __restrict__ xo, float w0h2,
                                                      float w1, float h2, int two, int zc) {
  pdl_wait();
  pdl_trigger();
  __shared__ float4 sb[VY + 2][32];
  const int lane = threadIdx.x, ty = threadIdx.y;
  const int i0 = 4 * (blockIdx.x * 32 + lane);
  const int j = blockIdx.y * VY + ty;
  const bool act = i0 < d.nx && j < d.ny;
  const int z0 = blockIdx.z * zc;
  const int z1 = min(z0 + zc, d.nz);
  const int64_t sy = d.nx, sz = (int64_t)d.nx * d.ny;
  int64_t c = (int64_t)z0 * sz + (int64_t)j * sy + i0;
  const float4 Z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  const int ny_c = (j > 0) + (j < d.ny - 1);
  if (!two) {
    const int n0 = ny_c + (i0 > 0) + 1, n3 = ny_c + 1 + (i0 + 3 < d.nx - 1);
    const int n12 = ny_c + 2;
    for (int z = z0; z < z1; ++z, c += sz) {
      if (!act) continue;
      const float4 bv = ld4_any(b + c);
      const int zn = (z > 0) + (z < d.nz - 1);
      float4 o;
      o.x = w_over(w0h2, n0 + zn) * bv.x;
      o.y = w_over(w0h2, n12 + zn) * bv.y;
      o.z = w_over(w0h2, n12 + zn) * bv.z;
      o.w = w_over(w0h2, n3 + zn) * bv.w;
      if (bcopy) st4(bcopy + c, bv);
      st4(xo + c, o);
    }
    return;
  }
  // Away from the y and z walls the two steps are one 7-point stencil on b
  // with per-thread weights: x1 = r b (r = w0 h^2 / nn), and with
  // nn x1 = w0 h^2 b,
  //   x2 = x1 + (w1/nn)(h^2 b - nn x1 + sum_nb x1)
  //      = c0 b + cl b_left + cr b_right + cy (b_y- + b_y+ + b_z- + b_z+),
  // c0 = r + (w1/nn) h^2 (1 - w0), cl = (w1/nn) r_left, cr = (w1/nn) r_right,
  // cy = (w1/nn) r (the y and z neighbours share the cell's x-count).  There
  // nn = 4 + x-count, the x-count is 2 except at an x-wall cell (1), so 1/nn
  // is 1/6 or 1/5.
  float k0[4], kl[4], kr[4], ky[4];
  {
    auto inv = [](bool two_x) { return two_x ? (1.f / 6.f) : 0.2f; };
    const float f0 = inv(i0 > 0), f3 = inv(i0 + 3 < d.nx - 1);
    const float fl = inv(i0 - 1 > 0), fr = inv(i0 + 4 < d.nx - 1);
    const float r_own[4] = {w0h2 * f0, w0h2 * (1.f / 6.f), w0h2 * (1.f / 6.f), w0h2 * f3};
    const float w1_own[4] = {w1 * f0, w1 * (1.f / 6.f), w1 * (1.f / 6.f), w1 * f3};
    const float rl4[4] = {w0h2 * fl, r_own[0], r_own[1], r_own[2]};
    const float rr4[4] = {r_own[1], r_own[2], r_own[3], w0h2 * fr};
    const float h2w = h2 - w0h2;   // h^2 (1 - w0)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      k0[q] = fmaf(w1_own[q], h2w, r_own[q]);
      kl[q] = w1_own[q] * rl4[q];
      kr[q] = w1_own[q] * rr4[q];
      ky[q] = w1_own[q] * r_own[q];
    }
  }
  const bool yin = j >= 2 && j <= d.ny - 3;
  float4 bp = (act && z0 > 0) ? ld4_any(b + c - sz) : Z4;
  float4 bc = act ? ld4_any(b + c) : Z4;
  constexpr int kUnroll = ZC > 0 ? ZC : 1;
#pragma unroll kUnroll
  for (int zz = 0; zz < (ZC > 0 ? ZC : zc); ++zz) {
    const int z = z0 + zz;
    if (z >= z1) break;
    // rows and planes two cells away from the y and z walls (warp-uniform)
    const bool inner = yin && z >= 2 && z <= d.nz - 3;
    float4 bn = Z4, ym = Z4, yp = Z4;
    if constexpr (std::is_same<TB, float>::value) {
      // FP32 input: the y-neighbour rows come straight through L1
      if (inner) {
        if (act) {
          bn = ld4_any(b + c + sz);
          ym = ld4_any(b + c - sy);
          yp = ld4_any(b + c + sy);
        }
      } else if (act) {
        if (z + 1 < d.nz) bn = ld4_any(b + c + sz);
        if (j > 0) ym = ld4_any(b + c - sy);
        if (j < d.ny - 1) yp = ld4_any(b + c + sy);
      }
    } else {
      bn = (act && z + 1 < d.nz) ? ld4_any(b + c + sz) : Z4;
      // rounded once, shared through shared memory
      sb[ty + 1][lane] = bc;
      if (ty == 0) sb[0][lane] = (act && j > 0) ? ld4_any(b + c - sy) : Z4;
      if (ty == VY - 1 || j == d.ny - 1)
        sb[ty + 2][lane] = (act && j < d.ny - 1) ? ld4_any(b + c + sy) : Z4;
      __syncthreads();
      ym = sb[ty][lane];
      yp = sb[ty + 2][lane];
    }
    float left = __shfl_up_sync(kFull, bc.w, 1);
    float right = __shfl_down_sync(kFull, bc.x, 1);
    if (lane == 0) left = (act && i0 > 0) ? ld1_any(b + c - 1) : 0.f;
    if (lane == 31) right = (act && i0 + 4 < d.nx) ? ld1_any(b + c + 4) : 0.f;
    const float bcv[4] = {bc.x, bc.y, bc.z, bc.w};
    const float bpv[4] = {bp.x, bp.y, bp.z, bp.w};
    const float bnv[4] = {bn.x, bn.y, bn.z, bn.w};
    const float ymv[4] = {ym.x, ym.y, ym.z, ym.w};
    const float ypv[4] = {yp.x, yp.y, yp.z, yp.w};
    float o[4];
    if (inner) {
      const float xl[4] = {left, bcv[0], bcv[1], bcv[2]};
      const float xr[4] = {bcv[1], bcv[2], bcv[3], right};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float s4 = (ymv[q] + ypv[q]) + (bpv[q] + bnv[q]);
        o[q] = fmaf(k0[q], bcv[q], fmaf(kl[q], xl[q], fmaf(kr[q], xr[q], ky[q] * s4)));
      }
    } else {
      // the two steps as written: x1 = w0 h^2 b / nn at the own cells, the
      // two x-halo cells and the y and z neighbours, then the second step
      auto nrow = [&](int jj, int q) {
        const int ii = i0 + q;
        return (ii > 0) + (ii < d.nx - 1) + (jj > 0) + (jj < d.ny - 1);
      };
      const int zn = (z > 0) + (z < d.nz - 1);
      const int znm = (z - 1 > 0) + (z - 1 < d.nz - 1);
      const int znp = (z + 1 > 0) + (z + 1 < d.nz - 1);
      const int cx_m = (i0 - 1 > 0) + 1 + ny_c;          // cell i0-1
      const int cx_p = 1 + (i0 + 4 < d.nx - 1) + ny_c;   // cell i0+4
      float x1[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) x1[q] = w_over(w0h2, nrow(j, q) + zn) * bcv[q];
      const float x1l = w_over(w0h2, cx_m + zn) * left;
      const float x1r = w_over(w0h2, cx_p + zn) * right;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int ii = i0 + q;
        const int nown = nrow(j, q);
        float s = 0.f;
        if (ii > 0) s += (q == 0) ? x1l : x1[q - 1];
        if (ii < d.nx - 1) s += (q == 3) ? x1r : x1[q + 1];
        if (j > 0) s += w_over(w0h2, nrow(j - 1, q) + zn) * ymv[q];
        if (j < d.ny - 1) s += w_over(w0h2, nrow(j + 1, q) + zn) * ypv[q];
        if (z > 0) s += w_over(w0h2, nown + znm) * bpv[q];
        if (z < d.nz - 1) s += w_over(w0h2, nown + znp) * bnv[q];
        const int nn = nown + zn;
        o[q] = fmaf(w_over(w1, nn), fmaf(h2, bcv[q], s - (float)nn * x1[q]), x1[q]);
      }
    }
    if (act) {
      st4(xo + c, make_float4(o[0], o[1], o[2], o[3]));
      if (bcopy) st4(bcopy + c, bc);
    }
    if constexpr (!std::is_same<TB, float>::value) __syncthreads();
    bp = bc;
    bc = bn;
    c += sz;
  }
}

// Residual restriction, four fine cells (two coarse cells) per thread and
// two fine rows (one coarse row); the march runs over fine planes.
__global__ void __launch_bounds__(32 * VY, 4) k_restrict_v4(Dims d, Dims dc,
                                                         const float* __restrict__ x,
                                                         const float* __restrict__ b,
                                                         float* __restrict__ bcoarse, float inv_h2,
                                                         int zcc) {
  pdl_wait();
  pdl_trigger();
  const int lane = threadIdx.x;
  const int i0 = 4 * (blockIdx.x * 32 + lane);
  const int J = blockIdx.y * VY + threadIdx.y;
  const bool act = i0 < d.nx && J < dc.ny;
  const int K0 = blockIdx.z * zcc;
  const int K1 = min(K0 + zcc, dc.nz);
  const int64_t sy = d.nx, sz = (int64_t)d.nx * d.ny;
  const float4 Z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  const int j0 = 2 * J;
  // rows j0 (r = 0) and j0 + 1 (r = 1); in-plane counts per row and cell
  int nin[2][4];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int ii = i0 + q, jj = j0 + r;
      nin[r][q] = (ii > 0) + (ii < d.nx - 1) + (jj > 0) + (jj < d.ny - 1);
    }
  const int zs = 2 * K0;
  int64_t c = (int64_t)zs * sz + (int64_t)j0 * sy + i0;
  float4 p0 = Z4, p1 = Z4, c0 = Z4, c1 = Z4;   // planes z-1 and z of rows r = 0, 1
  if (x && act) {
    if (zs > 0) { p0 = ld4(x + c - sz); p1 = ld4(x + c - sz + sy); }
    c0 = ld4(x + c);
    c1 = ld4(x + c + sy);
  }
  float acc0 = 0.f, acc1 = 0.f;
  for (int z = zs; z < 2 * K1; ++z, c += sz) {
    float4 b0 = act ? ld4(b + c) : Z4;
    float4 b1 = act ? ld4(b + c + sy) : Z4;
    if (x) {
      float4 n0 = Z4, n1 = Z4, ym = Z4, yp = Z4;
      if (act && z + 1 < d.nz) { n0 = ld4(x + c + sz); n1 = ld4(x + c + sz + sy); }
      if (act && j0 > 0) ym = ld4(x + c - sy);
      if (act && j0 + 2 < d.ny) yp = ld4(x + c + 2 * sy);
      float l0 = __shfl_up_sync(kFull, c0.w, 1), l1 = __shfl_up_sync(kFull, c1.w, 1);
      float r0 = __shfl_down_sync(kFull, c0.x, 1), r1 = __shfl_down_sync(kFull, c1.x, 1);
      if (lane == 0) {
        l0 = (act && i0 > 0) ? __ldg(x + c - 1) : 0.f;
        l1 = (act && i0 > 0) ? __ldg(x + c + sy - 1) : 0.f;
      }
      if (lane == 31) {
        r0 = (act && i0 + 4 < d.nx) ? __ldg(x + c + 4) : 0.f;
        r1 = (act && i0 + 4 < d.nx) ? __ldg(x + c + sy + 4) : 0.f;
      }
      const int zn = (z > 0) + (z < d.nz - 1);
      // row 0: y-neighbours ym (row j0-1) and c1 (row j0+1)
      b0.x -= ((float)(nin[0][0] + zn) * c0.x - ((l0 + c0.y) + (ym.x + c1.x) + (p0.x + n0.x))) * inv_h2;
      b0.y -= ((float)(nin[0][1] + zn) * c0.y - ((c0.x + c0.z) + (ym.y + c1.y) + (p0.y + n0.y))) * inv_h2;
      b0.z -= ((float)(nin[0][2] + zn) * c0.z - ((c0.y + c0.w) + (ym.z + c1.z) + (p0.z + n0.z))) * inv_h2;
      b0.w -= ((float)(nin[0][3] + zn) * c0.w - ((c0.z + r0) + (ym.w + c1.w) + (p0.w + n0.w))) * inv_h2;
      // row 1: y-neighbours c0 (row j0) and yp (row j0+2)
      b1.x -= ((float)(nin[1][0] + zn) * c1.x - ((l1 + c1.y) + (c0.x + yp.x) + (p1.x + n1.x))) * inv_h2;
      b1.y -= ((float)(nin[1][1] + zn) * c1.y - ((c1.x + c1.z) + (c0.y + yp.y) + (p1.y + n1.y))) * inv_h2;
      b1.z -= ((float)(nin[1][2] + zn) * c1.z - ((c1.y + c1.w) + (c0.z + yp.z) + (p1.z + n1.z))) * inv_h2;
      b1.w -= ((float)(nin[1][3] + zn) * c1.w - ((c1.z + r1) + (c0.w + yp.w) + (p1.w + n1.w))) * inv_h2;
      p0 = c0; p1 = c1; c0 = n0; c1 = n1;
    }
    acc0 += (b0.x + b0.y) + (b1.x + b1.y);
    acc1 += (b0.z + b0.w) + (b1.z + b1.w);
    if (z & 1) {
      if (act) {
        const int64_t cc = ((int64_t)(z >> 1) * dc.ny + J) * dc.nx + (i0 >> 1);
        *reinterpret_cast<float2*>(bcoarse + cc) = make_float2(acc0 * 0.125f, acc1 * 0.125f);
      }
      acc0 = acc1 = 0.f;
    }
  }
}

// x (+)= P xc for four fine cells per thread (parents I0 = 2q, I1 = 2q + 1).
__global__ void __launch_bounds__(32 * VY) k_prolong_v4(Dims d, Dims dc,
                                                        const float* __restrict__ xc,
                                                        float* __restrict__ x, int overwrite,
                                                        int zc) {
  pdl_wait();
  pdl_trigger();
  const int lane = threadIdx.x;
  const int q = blockIdx.x * 32 + lane;
  const int i0 = 4 * q;
  const int j = blockIdx.y * VY + threadIdx.y;
  if (i0 >= d.nx || j >= d.ny) return;
  const int z0 = blockIdx.z * zc;
  const int z1 = min(z0 + zc, d.nz);
  const int I0 = 2 * q, I1 = 2 * q + 1;
  const int Im = max(I0 - 1, 0), Ip = min(I1 + 1, dc.nx - 1);
  const int J = j >> 1;
  const int Jn = (j & 1) ? min(J + 1, dc.ny - 1) : max(J - 1, 0);
  const int64_t sy = dc.nx, sz = (int64_t)dc.nx * dc.ny;
  for (int k = z0; k < z1; ++k) {
    const int K = k >> 1;
    const int Kn = (k & 1) ? min(K + 1, dc.nz - 1) : max(K - 1, 0);
    const float* r00 = xc + K * sz + J * sy;
    const float* r01 = xc + K * sz + Jn * sy;
    const float* r10 = xc + Kn * sz + J * sy;
    const float* r11 = xc + Kn * sz + Jn * sy;
    auto yz = [&](int I) {
      const float a = 0.75f * __ldg(r00 + I) + 0.25f * __ldg(r01 + I);
      const float bb = 0.75f * __ldg(r10 + I) + 0.25f * __ldg(r11 + I);
      return 0.75f * a + 0.25f * bb;
    };
    const float cm = yz(Im), ca = yz(I0), cb = yz(I1), cp = yz(Ip);
    float4 v = make_float4(0.75f * ca + 0.25f * cm, 0.75f * ca + 0.25f * cb,
                           0.75f * cb + 0.25f * ca, 0.75f * cb + 0.25f * cp);
    const int64_t f = ((int64_t)k * d.ny + j) * d.nx + i0;
    if (!overwrite) {
      const float4 o = *reinterpret_cast<const float4*>(x + f);
      v.x += o.x; v.y += o.y; v.z += o.z; v.w += o.w;
    }
    st4(x + f, v);
  }
}

// ---------------------------------------------------------------------------
// The V-cycle below a level of at most kChainCells cells, in one CTA: every
// level's x, b and a ping-pong buffer live in shared memory, phases are
// separated by __syncthreads, so the five to eight launches per coarse level
// (each a few microseconds of latency for a few thousand cells) become one.
// The packed coordinates i | j << 10 | k << 20 and the masks of existing
// neighbours (bits x-, x+, y-, y+, z-, z+) of the chain's cells are built
// once at setup and copied into shared memory by each launch, so that no
// phase needs an integer division; the coarsest level's dense
// pseudo-inverse is staged in shared memory as well when it is small.
constexpr int kChainCells = 4096;
constexpr int kChainMax = 6;
constexpr int kChainThreads = 1024;
constexpr int kChainPinvStage = 128;   // largest coarsest level staged in shared memory

struct CoarseChain {
  int nlev;                    // levels in the chain (the last is the coarsest)
  Dims d[kChainMax];
  float h2[kChainMax];
  int off[kChainMax + 1];      // cell offsets of the levels in the smem arrays
  float wpre[8], wpost[8];     // Chebyshev-Richardson weights
  int pre, post;
  const float* pinv;           // dense pseudo-inverse of the coarsest level
  int mc;
  int stage_pinv;              // pinv copied into shared memory
  const uint32_t* pk;          // packed coordinates of the chain's cells
  const uint8_t* nb;           // neighbour masks of the chain's cells
};

__device__ __forceinline__ void unpack(uint32_t p, int& i, int& j, int& k) {
  i = p & 1023;
  j = (p >> 10) & 1023;
  k = p >> 20;
}

__device__ __forceinline__ float lap_nb(Dims d, const float* x, int c, uint32_t mask, int& nn) {
  const int sz = d.nx * d.ny;
  float s = 0.f;
  if (mask & 1u) s += x[c - 1];
  if (mask & 2u) s += x[c + 1];
  if (mask & 4u) s += x[c - d.nx];
  if (mask & 8u) s += x[c + d.nx];
  if (mask & 16u) s += x[c - sz];
  if (mask & 32u) s += x[c + sz];
  nn = __popc(mask);
  return s;
}

struct ChainSm {
  float* x;
  float* b;
  float* t;
  uint32_t* pk;
  uint8_t* nb;
  const float* pinv;
};

__host__ __device__ inline int round4(int n) { return (n + 3) & ~3; }
__host__ __device__ inline int round16(int n) { return (n + 15) & ~15; }

// floats of shared memory the chain needs: x, b, t and the coordinates
// (round4(tot) each, so that every array starts on a 16-byte boundary), the
// masks (round16(tot) bytes) and the staged pseudo-inverse
__host__ __device__ inline int chain_smem_floats(int tot, int mc, int stage) {
  return 4 * round4(tot) + round16(tot) / 4 + (stage ? round4(mc * mc) : 0);
}

__device__ ChainSm chain_layout(float* base, const CoarseChain& ch) {
  const int t4 = round4(ch.off[ch.nlev]);
  ChainSm S;
  S.x = base;
  S.b = base + t4;
  S.t = base + 2 * t4;
  S.pk = reinterpret_cast<uint32_t*>(base + 3 * t4);
  S.nb = reinterpret_cast<uint8_t*>(base + 4 * t4);
  S.pinv = ch.stage_pinv ? base + 4 * t4 + round16(ch.off[ch.nlev]) / 4 : ch.pinv;
  return S;
}

// Cells (or 16-byte words) a thread of the chain takes per round: their
// loads are issued together before their arithmetic or stores, so a round
// costs about one shared-memory (or L2) latency instead of four.
constexpr int kChainBatch = 4;

// Copies up to four arrays of 16-byte words from global to shared memory as
// one sequence: each thread loads its kChainBatch words of a round (from
// whichever array they fall in) before it stores them.
struct WordSegs {
  uint4* dst[4];
  const uint4* src[4];
  int end[4];   // running word counts; unused segments repeat the last end
};

__device__ void copy_segs(const WordSegs& w) {
  const int n = w.end[3];
  for (int base = threadIdx.x; base < n; base += kChainBatch * (int)blockDim.x) {
    uint4 v[kChainBatch];
    int seg[kChainBatch], off[kChainBatch];
#pragma unroll
    for (int q = 0; q < kChainBatch; ++q) {
      const int e = base + q * (int)blockDim.x;
      const int sg = (e >= w.end[0]) + (e >= w.end[1]) + (e >= w.end[2]);
      const int first = sg == 0 ? 0 : (sg == 1 ? w.end[0] : (sg == 2 ? w.end[1] : w.end[2]));
      const uint4* src = sg == 0 ? w.src[0] : (sg == 1 ? w.src[1] : (sg == 2 ? w.src[2] : w.src[3]));
      seg[q] = sg;
      off[q] = e - first;
      if (e < n) v[q] = __ldg(src + off[q]);
    }
#pragma unroll
    for (int q = 0; q < kChainBatch; ++q) {
      const int e = base + q * (int)blockDim.x;
      const int sg = seg[q];
      uint4* dst = sg == 0 ? w.dst[0] : (sg == 1 ? w.dst[1] : (sg == 2 ? w.dst[2] : w.dst[3]));
      if (e < n) dst[off[q]] = v[q];
    }
  }
}

// The coordinate and mask tables, the first level's b (m0 floats, a multiple
// of four) and the staged pseudo-inverse into shared memory in one sequence
// (the caller synchronises before they are used).  The tables are padded to
// whole 16-byte words at setup; the pseudo-inverse's last mc^2 mod 4 floats
// are copied one by one.
__device__ void chain_load(const CoarseChain& ch, const ChainSm& S, const float* b_in, int m0) {
  const int tot = ch.off[ch.nlev];
  WordSegs w;
  int e = 0;
  w.dst[0] = reinterpret_cast<uint4*>(S.pk);
  w.src[0] = reinterpret_cast<const uint4*>(ch.pk);
  w.end[0] = e += round4(tot) / 4;
  w.dst[1] = reinterpret_cast<uint4*>(S.nb);
  w.src[1] = reinterpret_cast<const uint4*>(ch.nb);
  w.end[1] = e += round16(tot) / 16;
  w.dst[2] = reinterpret_cast<uint4*>(S.b);
  w.src[2] = reinterpret_cast<const uint4*>(b_in);
  w.end[2] = e += m0 / 4;
  w.dst[3] = reinterpret_cast<uint4*>(const_cast<float*>(S.pinv));
  w.src[3] = reinterpret_cast<const uint4*>(ch.pinv);
  const int np = ch.stage_pinv ? ch.mc * ch.mc : 0;
  w.end[3] = e += np / 4;
  copy_segs(w);
  float* pv = const_cast<float*>(S.pinv);
  for (int q = (np & ~3) + (int)threadIdx.x; q < np; q += (int)blockDim.x) pv[q] = __ldg(ch.pinv + q);
}

// p Chebyshev steps on one level in shared memory; from_zero starts at x = 0.
// The steps alternate between x and t and the result ends in x: from zero
// the first step writes x or t so that the last one writes x; from x with an
// odd p the result is copied back.
__device__ void chain_smooth(const CoarseChain& ch, const ChainSm& S, int l, const float* w,
                             int p, bool from_zero) {
  if (p <= 0) return;
  const Dims d = ch.d[l];
  const int o = ch.off[l];
  const int m = d.nx * d.ny * d.nz;
  const float h2 = ch.h2[l];
  float* x = S.x + o;
  float* t = S.t + o;
  const float* b = S.b + o;
  const uint8_t* nb = S.nb + o;
  const int nt = (int)blockDim.x;
  float* cur = x;
  float* nxt = t;
  int q = 0;
  if (from_zero) {
    float* dst = (p & 1) ? x : t;
    for (int c = threadIdx.x; c < m; c += nt)
      dst[c] = w[0] * h2 * b[c] * inv_nn(__popc((uint32_t)nb[c]));
    __syncthreads();
    cur = dst;
    nxt = (p & 1) ? t : x;
    q = 1;
  }
  for (; q < p; ++q) {
    const float wq = w[q];
    for (int base = threadIdx.x; base < m; base += kChainBatch * nt) {
      float sn[kChainBatch], xv[kChainBatch], bv[kChainBatch];
      int nn[kChainBatch];
#pragma unroll
      for (int k = 0; k < kChainBatch; ++k) {
        const int c = base + k * nt;
        sn[k] = 0.f; xv[k] = 0.f; bv[k] = 0.f; nn[k] = 1;
        if (c < m) {
          sn[k] = lap_nb(d, cur, c, nb[c], nn[k]);
          xv[k] = cur[c];
          bv[k] = b[c];
        }
      }
#pragma unroll
      for (int k = 0; k < kChainBatch; ++k) {
        const int c = base + k * nt;
        if (c < m)
          nxt[c] = fmaf(wq * inv_nn(nn[k]), fmaf(h2, bv[k], sn[k] - (float)nn[k] * xv[k]), xv[k]);
      }
    }
    __syncthreads();
    float* tmp = cur; cur = nxt; nxt = tmp;
  }
  if (cur != x) {
    for (int c = threadIdx.x; c < m; c += nt) x[c] = cur[c];
    __syncthreads();
  }
}

// The cycle on the chain's levels: b of its first level in S.b, the tables
// loaded and synchronised; leaves x of its first level in S.x.
__device__ void chain_run(const CoarseChain& ch, const ChainSm& S) {
  const int nt = (int)blockDim.x;
  // descend
  for (int l = 0; l < ch.nlev - 1; ++l) {
    chain_smooth(ch, S, l, ch.wpre, ch.pre, true);
    const Dims d = ch.d[l], dc = ch.d[l + 1];
    const int mcl = dc.nx * dc.ny * dc.nz;
    const float ih2 = 1.f / ch.h2[l];
    const float* x = S.x + ch.off[l];
    const float* b = S.b + ch.off[l];
    const uint8_t* nb = S.nb + ch.off[l];
    const uint32_t* pkc = S.pk + ch.off[l + 1];
    float* bc = S.b + ch.off[l + 1];
    // eight threads per coarse cell (one child each), summed by shuffles;
    // the thread count is a multiple of 8, so a coarse cell's eight threads
    // are consecutive lanes of one warp in every round
    for (int base = 0; base < 8 * mcl; base += kChainBatch * nt) {
      float r[kChainBatch];
#pragma unroll
      for (int k = 0; k < kChainBatch; ++k) {
        const int tq = base + k * nt + (int)threadIdx.x;
        r[k] = 0.f;
        if (tq < 8 * mcl) {
          const int C = tq >> 3, q = tq & 7;
          int I, J, K;
          unpack(pkc[C], I, J, K);
          const int c =
              ((2 * K + (q >> 2)) * d.ny + 2 * J + ((q >> 1) & 1)) * d.nx + 2 * I + (q & 1);
          float v = b[c];
          if (ch.pre > 0) {
            int nn;
            const float sn = lap_nb(d, x, c, nb[c], nn);
            v -= ((float)nn * x[c] - sn) * ih2;
          }
          r[k] = v;
        }
      }
#pragma unroll
      for (int k = 0; k < kChainBatch; ++k) {
        const int tq = base + k * nt + (int)threadIdx.x;
        float v = r[k];
        v += __shfl_xor_sync(0xffffffffu, v, 1);
        v += __shfl_xor_sync(0xffffffffu, v, 2);
        v += __shfl_xor_sync(0xffffffffu, v, 4);
        if (tq < 8 * mcl && (tq & 7) == 0) bc[tq >> 3] = v * 0.125f;
      }
    }
    __syncthreads();
  }
  // coarsest: dense pseudo-inverse, one warp per row (lanes split the row,
  // summed by shuffles in a fixed order)
  {
    const int l = ch.nlev - 1;
    float* x = S.x + ch.off[l];
    const float* b = S.b + ch.off[l];
    const int lane = threadIdx.x & 31, nw = nt >> 5;
    for (int r = threadIdx.x >> 5; r < ch.mc; r += nw) {
      float acc = 0.f;
      for (int q = lane; q < ch.mc; q += 32) acc = fmaf(S.pinv[r * ch.mc + q], b[q], acc);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) x[r] = acc;
    }
    __syncthreads();
  }
  // ascend
  for (int l = ch.nlev - 2; l >= 0; --l) {
    float* x = S.x + ch.off[l];
    const float* xc = S.x + ch.off[l + 1];
    const uint32_t* pkf = S.pk + ch.off[l];
    const Dims d = ch.d[l], dc = ch.d[l + 1];
    const int m = d.nx * d.ny * d.nz;
    for (int base = threadIdx.x; base < m; base += kChainBatch * nt) {
      float v[kChainBatch], xo[kChainBatch];
#pragma unroll
      for (int k = 0; k < kChainBatch; ++k) {
        const int c = base + k * nt;
        v[k] = 0.f;
        xo[k] = 0.f;
        if (c < m) {
          int i, j, kk;
          unpack(pkf[c], i, j, kk);
          const int I = i >> 1, J = j >> 1, K = kk >> 1;
          const int In = (i & 1) ? min(I + 1, dc.nx - 1) : max(I - 1, 0);
          const int Jn = (j & 1) ? min(J + 1, dc.ny - 1) : max(J - 1, 0);
          const int Kn = (kk & 1) ? min(K + 1, dc.nz - 1) : max(K - 1, 0);
          auto X = [&](int a, int bb, int cc) { return xc[(cc * dc.ny + bb) * dc.nx + a]; };
          const float a00 = 0.75f * X(I, J, K) + 0.25f * X(In, J, K);
          const float a01 = 0.75f * X(I, Jn, K) + 0.25f * X(In, Jn, K);
          const float a10 = 0.75f * X(I, J, Kn) + 0.25f * X(In, J, Kn);
          const float a11 = 0.75f * X(I, Jn, Kn) + 0.25f * X(In, Jn, Kn);
          v[k] = 0.75f * (0.75f * a00 + 0.25f * a01) + 0.25f * (0.75f * a10 + 0.25f * a11);
          if (ch.pre > 0) xo[k] = x[c];
        }
      }
#pragma unroll
      for (int k = 0; k < kChainBatch; ++k) {
        const int c = base + k * nt;
        if (c < m) x[c] = ch.pre > 0 ? xo[k] + v[k] : v[k];
      }
    }
    __syncthreads();
    chain_smooth(ch, S, l, ch.wpost, ch.post, false);
  }
}

__global__ void __launch_bounds__(kChainThreads) k_coarse_chain(CoarseChain ch,
                                                                const float* __restrict__ b_in,
                                                                float* __restrict__ x_out) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ __align__(16) float sm[];
  const ChainSm S = chain_layout(sm, ch);
  const int m0 = ch.off[1];   // a multiple of 8 (the level has a level below it)
  chain_load(ch, S, b_in, m0);
  __syncthreads();
  chain_run(ch, S);
  for (int c = threadIdx.x; c < m0 / 4; c += blockDim.x)
    reinterpret_cast<float4*>(x_out)[c] = reinterpret_cast<const float4*>(S.x)[c];
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

// Pre-smoothing from a zero iterate: p Chebyshev steps on level l ending in x.
// The first two steps run as one kernel (k_first); b may be the FP64 input of
// the finest level, in which case bcopy receives its rounded copy.
template <typename T, typename TB>
void pre_smooth(ibm_ctx* c, int l, const TB* b, T* bcopy, T* x, T* t, int p, cudaStream_t s) {
  MGLevel& L = c->lv[l];
  double w[8];
  cheb_weights(p, w);
  const double h2 = L.h * L.h;
  const int two = p >= 2;
  const bool vec = std::is_same<T, float>::value && vec_ok(L.d);
  const int zc = vec_zc(L.d);
  const int ph = l == 0 ? prof_begin(c, IBM_PROF_MG_SMOOTH_FINE) : -1;
  count_launch();
  if constexpr (std::is_same<T, float>::value) {
    if (vec)
      launch_pdl(zc == 4 ? k_first_v4<TB, 4> : (zc == 1 ? k_first_v4<TB, 1> : k_first_v4<TB, 0>),
                 vec_grid(L.d, zc), dim3(32, VY), 0, s, L.d, b, bcopy, x, (float)(w[0] * h2),
                 (float)(two ? w[1] : 0.0), (float)h2, two, zc);
  }
  if constexpr (!std::is_same<TB, float2>::value) {
    if (!vec)
      k_first<T, TB><<<zm_grid(L.d), dim3(BX, BY), 0, s>>>(
          L.d, b, bcopy, x, w_over_n<T>(w[0] * h2), w_over_n<T>(two ? w[1] : 0.0), (T)h2, two);
  }
  prof_end_or_note(c, ph, (double)L.m * (sizeof(TB) + sizeof(T) + (bcopy ? sizeof(T) : 0)));
  const T* bb = bcopy ? bcopy : reinterpret_cast<const T*>(b);
  T* cur = x;
  T* nxt = t;
  for (int q = two ? 2 : 1; q < p; ++q) {
    count_launch();
    prof_note(c, (double)L.m * 3 * sizeof(T));
    if constexpr (std::is_same<T, float>::value) {
      if (vec)
        launch_pdl(zc == 4 ? k_sweep_v4<float, 4>
                           : (zc == 1 ? k_sweep_v4<float, 1> : k_sweep_v4<float, 0>),
                   vec_grid(L.d, zc), dim3(32, VY), 0, s, L.d,
                   (const float*)cur, (const float*)bb, nxt, (float)w[q], (float)h2, zc);
    }
    if (!vec)
      k_sweep<T, T, T><<<zm_grid(L.d), dim3(BX, BY), 0, s>>>(L.d, cur, bb, nxt,
                                                            w_over_n<T>(w[q]), (T)h2);
    T* tmp = cur; cur = nxt; nxt = tmp;
  }
  if (cur != x) {
    launch_copy(x, cur, sizeof(T) * L.m, s);
    prof_note(c, 2.0 * sizeof(T) * L.m);
  }
}

// one smoothing step src -> dst on level l
template <typename T, typename TO>
void sweep_step(ibm_ctx* c, int l, const T* src, const T* b, TO* dst, double w, cudaStream_t s) {
  MGLevel& L = c->lv[l];
  const double h2 = L.h * L.h;
  count_launch();
  if constexpr (std::is_same<T, float>::value) {
    if (vec_ok(L.d)) {
      const int zc = vec_zc(L.d);
      launch_pdl(zc == 4 ? k_sweep_v4<TO, 4> : (zc == 1 ? k_sweep_v4<TO, 1> : k_sweep_v4<TO, 0>),
                 vec_grid(L.d, zc), dim3(32, VY), 0, s, L.d, (const float*)src,
                 (const float*)b, dst, (float)w, (float)h2, zc);
      return;
    }
  }
  k_sweep<T, T, TO><<<zm_grid(L.d), dim3(BX, BY), 0, s>>>(L.d, src, b, dst, w_over_n<T>(w),
                                                         (T)h2);
}

// Post-smoothing: p Chebyshev steps from x; the last step writes out (which
// may be FP64 while T is FP32).  Intermediate iterates ping-pong between t and
// x; out never aliases the step's input.
template <typename T, typename TO>
void post_smooth(ibm_ctx* c, int l, const T* b, T* x, T* t, int p, TO* out, cudaStream_t s) {
  MGLevel& L = c->lv[l];
  if (p <= 0) {
    if ((const void*)out != (const void*)x) {
      count_launch();
      k_convert<T, TO><<<kRedBlocks, 256, 0, s>>>(x, out, L.m);
      prof_note(c, (double)L.m * (sizeof(T) + sizeof(TO)));
    }
    return;
  }
  double w[8];
  cheb_weights(p, w);
  const T* src = x;
  for (int q = 0; q < p; ++q) {
    const bool last = q == p - 1;
    const int ph = l == 0 ? prof_begin(c, IBM_PROF_MG_SMOOTH_FINE) : -1;
    if (last && (const void*)out != (const void*)src) {
      sweep_step<T, TO>(c, l, src, b, out, w[q], s);
      prof_end_or_note(c, ph, (double)L.m * (2 * sizeof(T) + sizeof(TO)));
      return;
    }
    T* dst = (src == x) ? t : x;
    sweep_step<T, T>(c, l, src, b, dst, w[q], s);
    prof_end_or_note(c, ph, (double)L.m * 3 * sizeof(T));
    src = dst;
  }
  // the last step landed in t or x while out aliases the other: copy
  if ((const void*)src != (const void*)out) {
    launch_copy(out, src, sizeof(T) * L.m, s);
    prof_note(c, 2.0 * sizeof(T) * L.m);
  }
}

// V-cycle on level l >= 1 (or level 0 in the FP64 form): x_l ~ L_l^{-1} b_l.
template <typename T>
void vcycle(ibm_ctx* c, int l, const T* b, T* x, T* t, int pre, int post, cudaStream_t s);

template <typename T>
void coarse_correct(ibm_ctx* c, int l, const T* b, T* x, int pre, int post, cudaStream_t s) {
  MGLevel& L = c->lv[l];
  MGLevel& C = c->lv[l + 1];
  LevelPtrs<T> cp = ptrs<T>(C);
  const T* xin = pre > 0 ? x : nullptr;
  bool done = false;
  count_launch();
  if constexpr (std::is_same<T, float>::value) {
    if (vec_ok(L.d)) {
      const int zcc = std::max(1, vec_zc(L.d) / 2);
      launch_pdl(k_restrict_v4,
                 dim3(div_up(L.d.nx / 4, 32), div_up(C.d.ny, VY), div_up(C.d.nz, zcc)),
                 dim3(32, VY), 0, s, L.d, C.d, (const float*)xin, (const float*)b, cp.b,
                 (float)(1.0 / (L.h * L.h)), zcc);
      done = true;
    }
  }
  if (!done)
    k_restrict<T><<<dim3(div_up(C.d.nx, BX), div_up(C.d.ny, BY), div_up(C.d.nz, ZC / 2)),
                    dim3(BX, BY), 0, s>>>(L.d, C.d, xin, b, cp.b, (T)(1.0 / (L.h * L.h)));
  prof_note(c, (double)L.m * ((xin ? 2 : 1) * sizeof(T)) + (double)C.m * sizeof(T));
  vcycle<T>(c, l + 1, cp.b, cp.x, cp.t, pre, post, s);
  done = false;
  count_launch();
  if constexpr (std::is_same<T, float>::value) {
    if (vec_ok(L.d)) {
      const int zc = vec_zc(L.d);
      launch_pdl(k_prolong_v4, vec_grid(L.d, zc), dim3(32, VY), 0, s, L.d, C.d,
                 (const float*)cp.x, x, pre > 0 ? 0 : 1, zc);
      done = true;
    }
  }
  if (!done)
    k_prolong<T><<<dim3(div_up(C.d.nx, BX), div_up(L.d.ny, BY), div_up(L.d.nz, ZC)),
                   dim3(BX, BY), 0, s>>>(L.d, C.d, cp.x, x, pre > 0 ? 0 : 1);
  prof_note(c, (double)C.m * sizeof(T) + (double)L.m * ((pre > 0 ? 2 : 1) * sizeof(T)));
}

constexpr size_t kChainSmemMax = 200 * 1024;

// The chain from level l (its first level, c->chain_l) down.
void chain_desc(ibm_ctx* c, int l, int pre, int post, CoarseChain& ch) {
  const int nlev = c->n_levels - l;
  ch.nlev = nlev;
  ch.off[0] = 0;
  for (int q = 0; q < nlev; ++q) {
    ch.d[q] = c->lv[l + q].d;
    ch.h2[q] = (float)(c->lv[l + q].h * c->lv[l + q].h);
    ch.off[q + 1] = ch.off[q] + (int)c->lv[l + q].m;
  }
  double w[8];
  cheb_weights(pre > 0 ? pre : 1, w);
  for (int q = 0; q < 8; ++q) ch.wpre[q] = q < pre ? (float)w[q] : 0.f;
  cheb_weights(post > 0 ? post : 1, w);
  for (int q = 0; q < 8; ++q) ch.wpost[q] = q < post ? (float)w[q] : 0.f;
  ch.pre = pre;
  ch.post = post;
  ch.pinv = c->coarse_pinv32;
  ch.mc = c->coarse_m;
  ch.stage_pinv = ch.mc <= kChainPinvStage;
  const int tot = ch.off[nlev];
  ch.pk = static_cast<const uint32_t*>(c->chain_tab);
  ch.nb = reinterpret_cast<const uint8_t*>(ch.pk + round4(tot));
}

size_t chain_smem_bytes(const CoarseChain& ch) {
  return sizeof(float) * (size_t)chain_smem_floats(ch.off[ch.nlev], ch.mc, ch.stage_pinv);
}

// Setup of the coarse end of the FP32 V-cycle: the chain's first level (the
// first level below the finest with at most kChainCells cells and a level
// below it) and the coordinate and mask tables of its cells.
ibm_status coarse_end_setup(ibm_ctx* c) {
  c->chain_l = -1;
  int l0 = -1;
  for (int l = 1; l < c->n_levels - 1; ++l)
    if (c->lv[l].m <= kChainCells) {
      l0 = l;
      break;
    }
  if (l0 < 0 || c->n_levels - l0 > kChainMax) return IBM_OK;
  CoarseChain ch;
  c->chain_tab = nullptr;
  chain_desc(c, l0, 2, 2, ch);
  if (chain_smem_bytes(ch) > kChainSmemMax) return IBM_OK;
  const int tot = ch.off[ch.nlev];
  // coordinates padded to whole 16-byte words, then the masks likewise
  std::vector<uint32_t> pk(round4(tot), 0u);
  std::vector<uint8_t> nb(round16(tot), 0u);
  for (int q = 0; q < ch.nlev; ++q) {
    const Dims d = ch.d[q];
    for (int k = 0; k < d.nz; ++k)
      for (int j = 0; j < d.ny; ++j)
        for (int i = 0; i < d.nx; ++i) {
          const int e = ch.off[q] + (k * d.ny + j) * d.nx + i;
          pk[e] = (uint32_t)i | ((uint32_t)j << 10) | ((uint32_t)k << 20);
          nb[e] = (uint8_t)((i > 0) | ((i < d.nx - 1) << 1) | ((j > 0) << 2) |
                            ((j < d.ny - 1) << 3) | ((k > 0) << 4) | ((k < d.nz - 1) << 5));
        }
  }
  if (cudaMalloc(&c->chain_tab, pk.size() * 4 + nb.size()) != cudaSuccess) {
    cudaGetLastError();
    c->chain_tab = nullptr;
    return set_err(c, IBM_ERR_NOMEM, "multigrid allocation failed");
  }
  IBM_CUDA(c, cudaMemcpy(c->chain_tab, pk.data(), pk.size() * 4, cudaMemcpyHostToDevice));
  IBM_CUDA(c, cudaMemcpy(static_cast<char*>(c->chain_tab) + pk.size() * 4, nb.data(),
                         nb.size(), cudaMemcpyHostToDevice));
  IBM_CUDA(c, cudaFuncSetAttribute(k_coarse_chain, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)kChainSmemMax));
  c->chain_l = l0;
  return IBM_OK;
}

// Launches the one-CTA cycle from level l down; false if it does not apply.
bool chain_vcycle(ibm_ctx* c, int l, const float* b, float* x, int pre, int post,
                  cudaStream_t s) {
  if (l != c->chain_l) return false;
  CoarseChain ch;
  chain_desc(c, l, pre, post, ch);
  count_launch();
  launch_pdl(k_coarse_chain, dim3(1), dim3(kChainThreads), chain_smem_bytes(ch), s, ch, b, x);
  prof_note(c, 8.0 * ch.off[1] + 4.0 * (double)ch.mc * ch.mc);
  return true;
}

template <typename T>
void vcycle(ibm_ctx* c, int l, const T* b, T* x, T* t, int pre, int post, cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value) {
    if (l > 0 && chain_vcycle(c, l, b, x, pre, post, s)) return;
  }
  if (l == c->n_levels - 1) {
    count_launch();
    k_coarse_solve<T><<<1, 256, 0, s>>>(pinv_of<T>(c), b, x, c->coarse_m);
    prof_note(c, (double)c->coarse_m * (c->coarse_m + 2) * sizeof(T));
    return;
  }
  if (pre > 0) pre_smooth<T, T>(c, l, b, nullptr, x, t, pre, s);
  coarse_correct<T>(c, l, b, x, pre, post, s);
  post_smooth<T, T>(c, l, b, x, t, post, x, s);
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
  return coarse_end_setup(c);
}

ibm_status mg_vcycle(ibm_ctx* c, const double* r, double* z, int prec, int pre, int post) {
  cudaStream_t s = c->stream;
  MGLevel& L0 = c->lv[0];
  if (c->n_levels == 1) {
    // the whole grid is the coarsest level: the cycle is the exact pseudo-inverse
    count_launch();
    k_coarse_solve<double><<<1, 256, 0, s>>>(c->coarse_pinv64, r, z, c->coarse_m);
    IBM_LAUNCH_CHECK(c);
    return IBM_OK;
  }
  auto al16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  if (prec == IBM_PREC_FP32 && vec_ok(L0.d) && (!al16(r) || !al16(z))) {
    // the four-cell kernels load and store FP64 pairs (16 bytes): a caller's
    // vector on an 8-byte boundary goes through the level's aligned buffers
    launch_copy(L0.b64, r, sizeof(double) * L0.m, s);
    ibm_status st = mg_vcycle(c, L0.b64, L0.t64, prec, pre, post);
    if (st != IBM_OK) return st;
    launch_copy(z, L0.t64, sizeof(double) * L0.m, s);
    IBM_LAUNCH_CHECK(c);
    return IBM_OK;
  }
  if (prec == IBM_PREC_FP32) {
    // finest level: FP64 in, FP32 inside, FP64 out
    if (pre > 0) {
      pre_smooth<float, double>(c, 0, r, L0.b32, L0.x32, L0.t32, pre, s);
    } else {
      // only the rounded copy of r is needed (the zero iterate is never read)
      count_launch();
      k_first<float, double><<<zm_grid(L0.d), dim3(BX, BY), 0, s>>>(
          L0.d, r, L0.b32, L0.t32, w_over_n<float>(0.0), w_over_n<float>(0.0), 0.f, 0);
    }
    coarse_correct<float>(c, 0, L0.b32, L0.x32, pre, post, s);
    post_smooth<float, double>(c, 0, L0.b32, L0.x32, L0.t32, post, z, s);
  } else {
    if (pre > 0) pre_smooth<double, double>(c, 0, r, nullptr, z, L0.t64, pre, s);
    coarse_correct<double>(c, 0, r, z, pre, post, s);
    post_smooth<double, double>(c, 0, r, z, L0.t64, post, z, s);
  }
  IBM_LAUNCH_CHECK(c);
  return IBM_OK;
}

// One V-cycle with FP32 input and output (the mixed Arnoldi process keeps
// its vectors as FP32 pairs and feeds the leading FP32 part).  r may be the
// level-0 right-hand-side array itself (it is only read); z must not alias
// the level-0 work arrays.
ibm_status mg_vcycle_f32(ibm_ctx* c, const float* r, float* z, int pre, int post) {
  cudaStream_t s = c->stream;
  MGLevel& L0 = c->lv[0];
  if (c->n_levels == 1 || !vec_ok(L0.d)) {
    // small or odd grids: through the FP64 cycle
    count_launch();
    k_convert<float, double><<<kRedBlocks, 256, 0, s>>>(r, L0.b64, L0.m);
    ibm_status st = mg_vcycle(c, L0.b64, L0.t64, IBM_PREC_FP32, pre, post);
    if (st != IBM_OK) return st;
    count_launch();
    k_convert<double, float><<<kRedBlocks, 256, 0, s>>>(L0.t64, z, L0.m);
    IBM_LAUNCH_CHECK(c);
    return IBM_OK;
  }
  if (pre > 0) pre_smooth<float, float>(c, 0, r, nullptr, L0.x32, L0.t32, pre, s);
  coarse_correct<float>(c, 0, r, L0.x32, pre, post, s);
  post_smooth<float, float>(c, 0, r, L0.x32, L0.t32, post, z, s);
  IBM_LAUNCH_CHECK(c);
  return IBM_OK;
}

ibm_status mg_vcycle_pair(ibm_ctx* c, const float2* r, float* z, int pre, int post) {
  cudaStream_t s = c->stream;
  MGLevel& L0 = c->lv[0];
  if (c->n_levels == 1 || !vec_ok(L0.d))
    return set_err(c, IBM_ERR_ARG, "pair V-cycle needs a multilevel grid with nx % 4 == 0");
  // the first kernel rounds nothing (the leading parts are FP32) and keeps a
  // contiguous copy of them for the level's later kernels
  const int zc = vec_zc(L0.d);
  if (pre > 0) {
    pre_smooth<float, float2>(c, 0, r, L0.b32, L0.x32, L0.t32, pre, s);
  } else {
    count_launch();
    k_first_v4<float2><<<vec_grid(L0.d, zc), dim3(32, VY), 0, s>>>(L0.d, r, L0.b32, L0.t32, 0.f,
                                                                   0.f, 0.f, 0, zc);
  }
  coarse_correct<float>(c, 0, L0.b32, L0.x32, pre, post, s);
  post_smooth<float, float>(c, 0, L0.b32, L0.x32, L0.t32, post, z, s);
  IBM_LAUNCH_CHECK(c);
  return IBM_OK;
}

}  // namespace ibm
