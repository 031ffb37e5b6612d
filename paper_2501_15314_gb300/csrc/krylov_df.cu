// Arnoldi process of the mixed-precision FGMRES in double-single arithmetic.
//
// GB300 executes FP64 (and FP64<->FP32 conversions) at about 1/58 of its FP32
// rate, which made the FP64 Schur product and Gram-Schmidt passes ALU-bound.
// In the mixed form (FP32 V-cycle) the Krylov vectors are therefore held as
// unevaluated sums hi + lo of two FP32 numbers ("double-single", about 48
// significant bits), and the Schur product L z (z = V-cycle output, exactly
// FP32), the multi-dot, the axpy + norm and the solution update run on the
// FP32 pipes with error-free transformations:
//   two_sum, two_prod and the double-single sums and products of ds.cuh.
// The marker term of S~ stays FP64 (it touches ~1% of the cells), the true
// residual b - S~ x that decides convergence (and restarts) is evaluated in
// native FP64, and dot products are reduced to FP64 per block.
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "ds.cuh"
#include "ibm_internal.cuh"

namespace ibm {

namespace {

constexpr int RT = kRedThreads;
constexpr int kOutStride = kMaxRestart + 2;
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ dsf d_to_ds(double x) {
  const float hi = (float)x;
  return {hi, (float)(x - (double)hi)};
}
__device__ __forceinline__ dsf ds_shfl_down(dsf a, int o) {
  return {__shfl_down_sync(kFull, a.hi, o), __shfl_down_sync(kFull, a.lo, o)};
}

// Reduces NQ double-single values across the block (warp shuffles, then the
// warps in order) and stores the block sums as FP64 in part[block][q].
template <int NQ>
__device__ __forceinline__ void block_reduce_ds(dsf (&acc)[NQ], int nq, double* part) {
  __shared__ float sh_hi[RT / 32][NQ];
  __shared__ float sh_lo[RT / 32][NQ];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    dsf v = acc[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = ds_add(v, ds_shfl_down(v, o));
    if (lane == 0) {
      sh_hi[wid][q] = v.hi;
      sh_lo[wid][q] = v.lo;
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < nq; q += RT) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < RT / 32; ++w) s += (double)sh_hi[w][q] + (double)sh_lo[w][q];
    part[(int64_t)blockIdx.x * kOutStride + q] = s;
  }
}

// hi/lo split of an FP64 vector into interleaved pairs; the leading parts
// are also written contiguously to hi (the next V-cycle's input)
__global__ void k_split(const double* __restrict__ x, float2* __restrict__ v,
                        float* __restrict__ hi, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const dsf d = d_to_ds(x[i]);
    v[i] = make_float2(d.hi, d.lo);
    hi[i] = d.hi;
  }
}

// w = L z for FP32 z in double-single: the 7-point difference
// nn z_c - sum of neighbours is summed exactly (two_sum chain), then scaled by
// 1/h^2 (split into hi + lo).  Four cells per thread, x-neighbours by
// shuffles, z by the march (as the FP32 smoothers).
constexpr int LVY = 8;

// Two cells at once: exact nn * zc as a pair, then each neighbour subtracted
// exactly (two_sum chain), then the scaling; paired FP32 instructions, bit
// for bit the two scalar evaluations.
__device__ __forceinline__ dsf2 lap_cell2(float2 zc, const float2 (&nb)[6], float2 nn, dsf ih2) {
  dsf2 acc = two_prod2(nn, zc);
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const dsf2 t = two_sum2(acc.hi, neg2(nb[q]));
    acc.hi = t.hi;
    acc.lo = __fadd2_rn(acc.lo, t.lo);
  }
  acc = fast_two_sum2(acc.hi, acc.lo);
  return ds_mul2(acc, ih2);
}

// (TW = float2: the pair; TW = float: rounded once to FP32)
template <typename TW>
__global__ void __launch_bounds__(32 * LVY) k_lap_ds(Dims d, const float* __restrict__ z,
                                                     TW* __restrict__ w, float ih2_hi,
                                                     float ih2_lo, int zc) {
  const int lane = threadIdx.x;
  const int i0 = 4 * (blockIdx.x * 32 + lane);
  const int j = blockIdx.y * LVY + threadIdx.y;
  const bool act = i0 < d.nx && j < d.ny;
  const int z0 = blockIdx.z * zc;
  const int z1 = min(z0 + zc, d.nz);
  const int64_t sy = d.nx, sz = (int64_t)d.nx * d.ny;
  int64_t c = (int64_t)z0 * sz + (int64_t)j * sy + i0;
  const float4 Z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  const dsf ih2 = {ih2_hi, ih2_lo};
  const int ny_c = (j > 0) + (j < d.ny - 1);
  const int nxq[4] = {(i0 > 0) + 1, 2, 2, 1 + (i0 + 3 < d.nx - 1)};
  auto ld4 = [&](const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); };
  float4 zp = (act && z0 > 0) ? ld4(z + c - sz) : Z4;
  float4 zcur = act ? ld4(z + c) : Z4;
  for (int zz = z0; zz < z1; ++zz, c += sz) {
    const float4 zn = (act && zz + 1 < d.nz) ? ld4(z + c + sz) : Z4;
    const float4 ym = (act && j > 0) ? ld4(z + c - sy) : Z4;
    const float4 yp = (act && j < d.ny - 1) ? ld4(z + c + sy) : Z4;
    float left = __shfl_up_sync(kFull, zcur.w, 1);
    float right = __shfl_down_sync(kFull, zcur.x, 1);
    if (lane == 0) left = (act && i0 > 0) ? __ldg(z + c - 1) : 0.f;
    if (lane == 31) right = (act && i0 + 4 < d.nx) ? __ldg(z + c + 4) : 0.f;
    const int zn_c = (zz > 0) + (zz < d.nz - 1);
    const float cv[4] = {zcur.x, zcur.y, zcur.z, zcur.w};
    const float xl[4] = {left, zcur.x, zcur.y, zcur.z};
    const float xr[4] = {zcur.y, zcur.z, zcur.w, right};
    const float vym[4] = {ym.x, ym.y, ym.z, ym.w};
    const float vyp[4] = {yp.x, yp.y, yp.z, yp.w};
    const float vzp[4] = {zp.x, zp.y, zp.z, zp.w};
    const float vzn[4] = {zn.x, zn.y, zn.z, zn.w};
    float ohi[4], olo[4];
    // cells (0, 1) and (2, 3) in pairs; missing neighbours contribute 0 and
    // are not counted
#pragma unroll
    for (int q = 0; q < 4; q += 2) {
      const float2 nb[6] = {make_float2(xl[q], xl[q + 1]),   make_float2(xr[q], xr[q + 1]),
                            make_float2(vym[q], vym[q + 1]), make_float2(vyp[q], vyp[q + 1]),
                            make_float2(vzp[q], vzp[q + 1]), make_float2(vzn[q], vzn[q + 1])};
      const float2 nn = make_float2((float)(nxq[q] + ny_c + zn_c), (float)(nxq[q + 1] + ny_c + zn_c));
      const dsf2 v = lap_cell2(make_float2(cv[q], cv[q + 1]), nb, nn, ih2);
      ohi[q] = v.hi.x;
      ohi[q + 1] = v.hi.y;
      olo[q] = v.lo.x;
      olo[q + 1] = v.lo.y;
    }
    if (act) {
      if constexpr (std::is_same<TW, float2>::value) {
        float4* wp = reinterpret_cast<float4*>(w + c);
        wp[0] = make_float4(ohi[0], olo[0], ohi[1], olo[1]);
        wp[1] = make_float4(ohi[2], olo[2], ohi[3], olo[3]);
      } else {
        *reinterpret_cast<float4*>(w + c) = make_float4(ohi[0], ohi[1], ohi[2], ohi[3]);
      }
    }
    zp = zcur;
    zcur = zn;
  }
}

// Shell cells: w[c] += scale * (G^T R t)[c] with the FP64 sum of the cell's
// entries (interleaved layout, as k_shell_gradt), added to the pair in FP64.
template <typename TW>
__global__ void k_shell_gradt_ds(int64_t n_shell, const int32_t* __restrict__ shell_cell,
                                 const int32_t* __restrict__ base, const int32_t* __restrict__ len,
                                 const int32_t* __restrict__ ekey,
                                 const double* __restrict__ ecoef, int64_t n_ell, int64_t nmk,
                                 const double* __restrict__ t, double scale,
                                 TW* __restrict__ wv) {
  const int64_t tq = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t g = tq >> 5;
  const int lane = (int)(tq & 31);
  const int64_t q = g * kEllCells + lane / kEllLanes;
  const bool live = g < ell_groups(n_shell) && q < n_shell;
  double acc = live ? ell_gradt_sum(ekey, ecoef, n_ell, nmk, t, base[g] + lane, len[g]) : 0.0;
  acc = ell_combine(acc);
  if (!live || lane % kEllLanes != 0) return;
  const int64_t c = shell_cell[q];
  if constexpr (std::is_same<TW, float2>::value) {
    const float2 wc = wv[c];
    const double v = (double)wc.x + (double)wc.y + scale * acc;
    const dsf r = d_to_ds(v);
    wv[c] = make_float2(r.hi, r.lo);
  } else {
    wv[c] = (float)((double)wv[c] + scale * acc);
  }
}

// The same gather for the FP32 Arnoldi cycles: FP32 coefficients and t, FP32
// FMAs, the cell's sum added to its FP32 value with one rounding.
__global__ void k_shell_gradt_f32(int64_t n_shell, const int32_t* __restrict__ shell_cell,
                                  const int32_t* __restrict__ base,
                                  const int32_t* __restrict__ len,
                                  const int32_t* __restrict__ ekey,
                                  const float* __restrict__ ecoef, int64_t n_ell, int64_t nmk,
                                  const float* __restrict__ t, float scale,
                                  float* __restrict__ wv) {
  const int64_t tq = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t g = tq >> 5;
  const int lane = (int)(tq & 31);
  const int64_t q = g * kEllCells + lane / kEllLanes;
  const bool live = g < ell_groups(n_shell) && q < n_shell;
  float acc = live ? ell_gradt_sum_f32(ekey, ecoef, n_ell, nmk, t, base[g] + lane, len[g]) : 0.f;
  acc = ell_combine_f32(acc);
  if (!live || lane % kEllLanes != 0) return;
  const int64_t c = shell_cell[q];
  wv[c] = fmaf(scale, acc, wv[c]);
}

// Compensated accumulation of products: the running FP32 sum S and an FP32
// accumulator E of everything S cannot hold (exact rounding errors of the
// leading products and of the additions, plus the hi*lo cross terms).  The
// value is S + E; E stays about 2^-24 |S|, so its own rounding is far below
// the 2^-48 level of the pair representation.
struct Comp {
  float s, e;
};

__device__ __forceinline__ void comp_add_prod(Comp& acc, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float e = __fmaf_rn(ah, bh, -p);         // exact error of the leading product
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
  const dsf t = two_sum(acc.s, p);
  acc.s = t.hi;
  acc.e = __fadd_rn(acc.e, __fadd_rn(e, t.lo));
}

__device__ __forceinline__ void comp_add_prod_f(Comp& acc, float ah, float al, float b) {
  const float p = __fmul_rn(ah, b);
  float e = __fmaf_rn(ah, b, -p);
  e = __fmaf_rn(al, b, e);
  const dsf t = two_sum(acc.s, p);
  acc.s = t.hi;
  acc.e = __fadd_rn(acc.e, __fadd_rn(e, t.lo));
}

// part[b][q] = <w, V_q> over the block's elements (compensated FP32 sums,
// block totals in FP64).
template <int NQ>
__global__ void __launch_bounds__(RT) k_multidot_ds(const float2* __restrict__ w,
                                                    const float2* __restrict__ V, int64_t ld,
                                                    int nq, int64_t n, double* __restrict__ part) {
  Comp acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) acc[q] = {0.f, 0.f};
  for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT) {
    const float2 wi = __ldg(w + i);
    float2 v[NQ];   // all loads first, then the arithmetic
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[q] = q < nq ? __ldg(V + q * ld + i) : make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < NQ; ++q)
      if (q < nq) comp_add_prod(acc[q], wi.x, wi.y, v[q].x, v[q].y);
  }
  dsf r[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) r[q] = fast_two_sum(acc[q].s, acc[q].e);
  block_reduce_ds<NQ>(r, nq, part);
}

// w -= sum_q coef[q] V_q (coef as pairs), part[b][0] = sum of w^2 (FP64)
template <int NQ>
__global__ void __launch_bounds__(RT) k_axpy_norm_ds(float2* __restrict__ w,
                                                     const float2* __restrict__ V, int64_t ld,
                                                     int nq, const float2* __restrict__ coef,
                                                     int64_t n, double* __restrict__ part,
                                                     float* __restrict__ hi) {
  float ch[NQ], cl[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const float2 v = q < nq ? coef[q] : make_float2(0.f, 0.f);
    ch[q] = v.x;
    cl[q] = v.y;
  }
  Comp nrm = {0.f, 0.f};
  for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT) {
    const float2 wi = w[i];
    float2 v[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[q] = q < nq ? __ldg(V + q * ld + i) : make_float2(0.f, 0.f);
    Comp t = {0.f, 0.f};
#pragma unroll
    for (int q = 0; q < NQ; ++q)
      if (q < nq) comp_add_prod(t, ch[q], cl[q], v[q].x, v[q].y);
    // w - (t.s + t.e) as a normalised pair
    const dsf d = two_sum(wi.x, -t.s);
    const dsf wn = fast_two_sum(d.hi, __fadd_rn(d.lo, __fsub_rn(wi.y, t.e)));
    w[i] = make_float2(wn.hi, wn.lo);
    hi[i] = wn.hi;
    comp_add_prod(nrm, wn.hi, wn.lo, wn.hi, wn.lo);
  }
  dsf r[1] = {fast_two_sum(nrm.s, nrm.e)};
  block_reduce_ds<1>(r, 1, part);
}

// out[q] = sum_b part[b][q] (fixed order); quot[q] = out[q] / div[q] as an
// FP64 value and as a hi/lo pair
__global__ void __launch_bounds__(RT) k_final_reduce_ds(const double* __restrict__ part, int nb,
                                                        double* __restrict__ out,
                                                        const double* __restrict__ div,
                                                        double* __restrict__ quot,
                                                        float2* __restrict__ quot_ds,
                                                        double* hout) {
  pdl_wait();
  pdl_trigger();
  const int q = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += RT) s += part[(int64_t)b * kOutStride + q];
  __shared__ double sh[RT / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(kFull, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < RT / 32; ++w) t += sh[w];
    out[q] = t;
    if (hout) hout[q] = t;   // mapped host mirror
    if (div) {
      const double qv = t / div[q];
      quot[q] = qv;
      const dsf p = d_to_ds(qv);
      quot_ds[q] = make_float2(p.hi, p.lo);
    }
  }
}

// x += sum_q y[q] Z_q for FP32 Z and double-single y, accumulated with the
// compensated scheme and added to the FP64 x once.
template <int NQ>
__global__ void __launch_bounds__(RT) k_gemv_ds(double* __restrict__ x,
                                                const float* __restrict__ Z, int64_t ld, int nq,
                                                const CoefDS y, int64_t n) {
  float yh[NQ], yl[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const float2 v = q < nq ? y.v[q] : make_float2(0.f, 0.f);
    yh[q] = v.x;
    yl[q] = v.y;
  }
  for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT) {
    float zq[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) zq[q] = q < nq ? __ldg(Z + q * ld + i) : 0.f;
    Comp acc = {0.f, 0.f};
#pragma unroll
    for (int q = 0; q < NQ; ++q)
      if (q < nq) comp_add_prod_f(acc, yh[q], yl[q], zq[q]);
    x[i] += (double)acc.s + (double)acc.e;
  }
}

// The same update four elements per thread (float4 loads of Z, two double2
// read-modify-writes of x), for m a multiple of 4 and nq <= 16; the FP32 sum
// and its error term are widened with integer operations, so the FP64 pipe
// only adds.
template <int NQ>
__global__ void __launch_bounds__(RT) k_gemv_ds4(double2* __restrict__ x,
                                                 const float4* __restrict__ Z, int64_t ld4,
                                                 int nq, const CoefDS y, int64_t n4) {
  pdl_wait();
  pdl_trigger();
  float yh[NQ], yl[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const float2 v = q < nq ? y.v[q] : make_float2(0.f, 0.f);
    yh[q] = v.x;
    yl[q] = v.y;
  }
  for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n4; i += (int64_t)gridDim.x * RT) {
    Comp a0 = {0.f, 0.f}, a1 = {0.f, 0.f}, a2 = {0.f, 0.f}, a3 = {0.f, 0.f};
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      if (q < nq) {
        const float4 zq = __ldg(Z + q * ld4 + i);
        comp_add_prod_f(a0, yh[q], yl[q], zq.x);
        comp_add_prod_f(a1, yh[q], yl[q], zq.y);
        comp_add_prod_f(a2, yh[q], yl[q], zq.z);
        comp_add_prod_f(a3, yh[q], yl[q], zq.w);
      }
    }
    double2 u0 = x[2 * i], u1 = x[2 * i + 1];
    u0.x += f2d_exact(a0.s) + f2d_exact(a0.e);
    u0.y += f2d_exact(a1.s) + f2d_exact(a1.e);
    u1.x += f2d_exact(a2.s) + f2d_exact(a2.e);
    u1.y += f2d_exact(a3.s) + f2d_exact(a3.e);
    x[2 * i] = u0;
    x[2 * i + 1] = u1;
  }
}

// FP32 Arnoldi process (IBM_ARNOLDI_FP32): the basis vectors are single FP32
// numbers (half the bytes of the pairs); dot products and the axpy are still
// accumulated with the compensated scheme, and each result is rounded once.

// part[b][q] = <w, V_q> for FP32 w and V
template <int NQ>
__global__ void __launch_bounds__(RT) k_multidot_sp(const float* __restrict__ w,
                                                    const float* __restrict__ V, int64_t ld,
                                                    int nq, int64_t n, double* __restrict__ part) {
  Comp acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) acc[q] = {0.f, 0.f};
  for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT) {
    const float wi = __ldg(w + i);
    float v[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[q] = q < nq ? __ldg(V + q * ld + i) : 0.f;
#pragma unroll
    for (int q = 0; q < NQ; ++q)
      if (q < nq) comp_add_prod_f(acc[q], wi, 0.f, v[q]);
  }
  dsf r[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) r[q] = fast_two_sum(acc[q].s, acc[q].e);
  block_reduce_ds<NQ>(r, nq, part);
}

// w -= sum_q coef[q] V_q (coef as pairs, the sum compensated, the result
// rounded once to FP32), part[b][0] = sum of w^2
template <int NQ>
__global__ void __launch_bounds__(RT) k_axpy_norm_sp(float* __restrict__ w,
                                                     const float* __restrict__ V, int64_t ld,
                                                     int nq, const float2* __restrict__ coef,
                                                     int64_t n, double* __restrict__ part) {
  float ch[NQ], cl[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const float2 v = q < nq ? coef[q] : make_float2(0.f, 0.f);
    ch[q] = v.x;
    cl[q] = v.y;
  }
  Comp nrm = {0.f, 0.f};
  for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT) {
    const float wi = w[i];
    float v[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[q] = q < nq ? __ldg(V + q * ld + i) : 0.f;
    Comp t = {0.f, 0.f};
#pragma unroll
    for (int q = 0; q < NQ; ++q)
      if (q < nq) comp_add_prod_f(t, ch[q], cl[q], v[q]);
    const dsf d = two_sum(wi, -t.s);
    const float wn = __fadd_rn(d.hi, __fsub_rn(d.lo, t.e));
    w[i] = wn;
    comp_add_prod_f(nrm, wn, 0.f, wn);
  }
  dsf r[1] = {fast_two_sum(nrm.s, nrm.e)};
  block_reduce_ds<1>(r, 1, part);
}

// The same two kernels on float4 (four consecutive elements per thread and
// array, 16-byte loads: more bytes in flight per thread), for m a multiple of
// 4 and nq <= 16.  Each element is accumulated exactly as in the scalar
// kernels; only the order of the additions within a thread differs.
template <int NQ>
__global__ void __launch_bounds__(RT) k_multidot_sp4(const float4* __restrict__ w,
                                                     const float4* __restrict__ V, int64_t ld4,
                                                     int nq, int64_t n4,
                                                     double* __restrict__ part) {
  pdl_wait();
  pdl_trigger();
  Comp acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) acc[q] = {0.f, 0.f};
  for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n4; i += (int64_t)gridDim.x * RT) {
    const float4 wi = __ldg(w + i);
    float4 v[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q)
      v[q] = q < nq ? __ldg(V + q * ld4 + i) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      if (q < nq) {
        comp_add_prod_f(acc[q], wi.x, 0.f, v[q].x);
        comp_add_prod_f(acc[q], wi.y, 0.f, v[q].y);
        comp_add_prod_f(acc[q], wi.z, 0.f, v[q].z);
        comp_add_prod_f(acc[q], wi.w, 0.f, v[q].w);
      }
    }
  }
  dsf r[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) r[q] = fast_two_sum(acc[q].s, acc[q].e);
  block_reduce_ds<NQ>(r, nq, part);
}

template <int NQ>
__device__ __forceinline__ float axpy_elem(float wi, const float (&ch)[NQ], const float (&cl)[NQ],
                                           const float (&v)[NQ], int nq) {
  Comp t = {0.f, 0.f};
#pragma unroll
  for (int q = 0; q < NQ; ++q)
    if (q < nq) comp_add_prod_f(t, ch[q], cl[q], v[q]);
  const dsf d = two_sum(wi, -t.s);
  return __fadd_rn(d.hi, __fsub_rn(d.lo, t.e));
}

template <int NQ>
__global__ void __launch_bounds__(RT) k_axpy_norm_sp4(float4* __restrict__ w,
                                                      const float4* __restrict__ V, int64_t ld4,
                                                      int nq, const float2* __restrict__ coef,
                                                      int64_t n4, double* __restrict__ part) {
  pdl_wait();
  pdl_trigger();
  float ch[NQ], cl[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const float2 c = q < nq ? coef[q] : make_float2(0.f, 0.f);
    ch[q] = c.x;
    cl[q] = c.y;
  }
  Comp nrm = {0.f, 0.f};
  for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n4; i += (int64_t)gridDim.x * RT) {
    const float4 wi = w[i];
    float4 v[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q)
      v[q] = q < nq ? __ldg(V + q * ld4 + i) : make_float4(0.f, 0.f, 0.f, 0.f);
    float vx[NQ], vy[NQ], vz[NQ], vw[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      vx[q] = v[q].x;
      vy[q] = v[q].y;
      vz[q] = v[q].z;
      vw[q] = v[q].w;
    }
    float4 o;
    o.x = axpy_elem<NQ>(wi.x, ch, cl, vx, nq);
    o.y = axpy_elem<NQ>(wi.y, ch, cl, vy, nq);
    o.z = axpy_elem<NQ>(wi.z, ch, cl, vz, nq);
    o.w = axpy_elem<NQ>(wi.w, ch, cl, vw, nq);
    w[i] = o;
    comp_add_prod_f(nrm, o.x, 0.f, o.x);
    comp_add_prod_f(nrm, o.y, 0.f, o.y);
    comp_add_prod_f(nrm, o.z, 0.f, o.z);
    comp_add_prod_f(nrm, o.w, 0.f, o.w);
  }
  dsf r[1] = {fast_two_sum(nrm.s, nrm.e)};
  block_reduce_ds<1>(r, 1, part);
}

// FP64 vector rounded to FP32
__global__ void k_round_f32(const double* __restrict__ x, float* __restrict__ v, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    v[i] = (float)x[i];
}

#define IBM_NQ_DISPATCH_DS(nq, KERNEL, ...)                                 \
  do {                                                                      \
    count_launch();                                                         \
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

// the float4 FP32 kernels, for nq <= 16
#define IBM_NQ_DISPATCH_SP4(nq, KERNEL, ...)                                       \
  do {                                                                             \
    count_launch();                                                                \
    const dim3 g_(kRedBlocks), b_(RT);                                             \
    if ((nq) <= 2) launch_pdl(KERNEL<2>, g_, b_, 0, s, __VA_ARGS__);               \
    else if ((nq) <= 4) launch_pdl(KERNEL<4>, g_, b_, 0, s, __VA_ARGS__);          \
    else if ((nq) <= 8) launch_pdl(KERNEL<8>, g_, b_, 0, s, __VA_ARGS__);          \
    else if ((nq) <= 12) launch_pdl(KERNEL<12>, g_, b_, 0, s, __VA_ARGS__);        \
    else launch_pdl(KERNEL<16>, g_, b_, 0, s, __VA_ARGS__);                        \
  } while (0)

int lap_zc(Dims d) {
  const int64_t bxy = (int64_t)div_up(d.nx / 4, 32) * div_up(d.ny, LVY);
  int64_t zc = (int64_t)d.nz * bxy / (152 * 4);
  zc = zc < 1 ? 1 : (zc > 16 ? 16 : zc);
  return (int)zc;
}

ibm_status fetch(ibm_ctx* c, const double* dev, int n) {
  launch_to_host(dev, c->host_red_dev, (int)sizeof(double) * n, c->stream);
  IBM_LAUNCH_CHECK(c);
  IBM_CUDA(c, cudaStreamSynchronize(c->stream));
  return IBM_OK;
}

}  // namespace

bool ds_supported(const ibm_ctx* c) { return c->d.nx % 4 == 0 && c->n_levels > 1; }

// w = S~ z for FP32 z, w as a hi/lo pair (double-single Laplacian, FP64
// marker term gathered from z and added on the shell cells) or, for the FP32
// Arnoldi cycles, one FP32 number (the Laplacian formed exactly and rounded
// once, the scalar-form marker term gathered in FP32).
template <typename TW>
ibm_status schur_apply_ds_t(ibm_ctx* c, const float* z, TW* w) {
  cudaStream_t s = c->stream;
  const double ih2 = 1.0 / (c->h * c->h);
  const float ih2_hi = (float)ih2;
  const float ih2_lo = (float)(ih2 - (double)ih2_hi);
  const int zc = lap_zc(c->d);
  const MarkerData& m = c->mk;
  // the marker gather t = 2 R^T G z runs on the side stream, concurrently
  // with the Laplacian; the shell scatter into w waits for both
  const bool fork = c->cmode == IBM_CMODE_SCALAR && m.n > 0 && m.n_shell > 0;
  if (fork) {
    IBM_CUDA(c, cudaEventRecord(c->ev_fork, s));
    IBM_CUDA(c, cudaStreamWaitEvent(c->side, c->ev_fork, 0));
    if constexpr (std::is_same<TW, float>::value)
      launch_marker_grad_interp_t32(c, z, 2.f, m.t32, c->side);
    else
      launch_marker_grad_interp_f32(c, z, 2.0, m.t, c->side);
    IBM_CUDA(c, cudaEventRecord(c->ev_join, c->side));
  }
  int ph = prof_begin(c, IBM_PROF_LAPLACIAN_F64);
  count_launch();
  k_lap_ds<TW><<<dim3(div_up(c->d.nx / 4, 32), div_up(c->d.ny, LVY), div_up(c->d.nz, zc)),
                 dim3(32, LVY), 0, s>>>(c->d, z, w, ih2_hi, ih2_lo, zc);
  prof_end(c, ph, (double)c->m * (4 + sizeof(TW)));
  if (m.n > 0 && m.n_shell > 0) {
    ph = prof_begin(c, IBM_PROF_SCHUR_MARKERS);
    const double* t = m.t;
    double sign = 1.0;
    if (fork) {
      IBM_CUDA(c, cudaStreamWaitEvent(s, c->ev_join, 0));
    } else {
      // +- B^T C^{-1} B z (exact / sign-consistent forms), C^{-1} in FP64
      launch_marker_grad_interp_f32(c, z, 1.0, m.t);
      const ibm_status st = c_solve(c, m.t, m.t2, c->c_rtol, c->c_maxit, nullptr);
      if (st != IBM_OK) { prof_end(c, ph); return st; }
      t = m.t2;
      sign = c->cmode == IBM_CMODE_CONSISTENT ? -1.0 : 1.0;
    }
    count_launch();
    if constexpr (std::is_same<TW, float>::value) {
      if (fork) {
        k_shell_gradt_f32<<<div_up(32 * ell_groups(m.n_shell), 256), 256, 0, s>>>(
            m.n_shell, m.ell_cell, m.ell_base, m.ell_len, m.ell_key, m.ell_coef32, m.n_ell, m.n,
            m.t32, 1.f, w);
        prof_end(c, ph, marker_term_bytes(c, 4, (int)sizeof(TW), 16));
        IBM_LAUNCH_CHECK(c);
        return IBM_OK;
      }
    }
    k_shell_gradt_ds<TW><<<div_up(32 * ell_groups(m.n_shell), 256), 256, 0, s>>>(
        m.n_shell, m.ell_cell, m.ell_base, m.ell_len, m.ell_key, m.ell_coef, m.n_ell, m.n, t,
        sign, w);
    prof_end(c, ph, marker_term_bytes(c, 4, (int)sizeof(TW)));
  }
  IBM_LAUNCH_CHECK(c);
  return IBM_OK;
}

ibm_status schur_apply_ds(ibm_ctx* c, const float* z, float2* w) {
  return schur_apply_ds_t<float2>(c, z, w);
}

// ---------------------------------------------------------------------------
// An Arnoldi cycle as one CUDA graph.  Iteration j's kernels (V-cycle, Schur
// product, Gram-Schmidt) are captured once, followed by k_givens, which
// applies the previous Givens rotations to the new Hessenberg column, forms
// the next rotation and the residual estimate, and decides whether the cycle
// goes on; iteration j + 1 sits in a conditional IF node whose condition
// k_givens sets, so the nodes nest as deep as the restart length and a cycle
// that stops early skips the rest.  The host launches the graph, reads the
// state once after it (GState layout) and forms the update as in the
// host-driven loop.  Opt-in (ibm_solve_opts.cycle_graphs): on GB300 the
// host-driven loop, which launches the next iteration before reading the
// current column while the residual is far from the target, measured
// faster (the one-thread Givens kernel and the conditional node add about
// 9 us per iteration on the critical path).  The host-driven loop also runs
// while profiling, for the exact and sign-consistent C forms (whose Schur
// product waits on the host) and when the graph cannot be built.

// g zeroed but g[0] = rn[0] = beta, and the cycle's scalars
__global__ void k_cycle_init(double* __restrict__ st, double beta, double bnorm, double rtol,
                             double cycle_stop, int rmax) {
  for (int i = threadIdx.x; i <= GState::R; i += blockDim.x) st[GState::kG + i] = 0.0;
  __syncthreads();
  if (threadIdx.x == 0) {
    st[GState::kG] = beta;
    st[GState::kRN] = beta;
    double* sc = st + GState::kSc;
    sc[GState::sBnorm] = bnorm;
    sc[GState::sRtol] = rtol;
    sc[GState::sStop] = cycle_stop;
    sc[GState::sRmax] = (double)rmax;
    sc[GState::sJused] = 0.0;
    sc[GState::sBreak] = 0.0;
    sc[GState::sNan] = 0.0;
  }
}

// Iteration j's Hessenberg column (raw[i] = <w, V_i>, nrm2[j + 1] = ||w||^2,
// the basis kept unnormalised with ||V_i|| = rn[i]) into the rotated
// triangular factor, as the host-driven loop does; one thread.
__global__ void k_givens(double* __restrict__ st, int j, const double* __restrict__ raw,
                         const double* __restrict__ nrm2, cudaGraphConditionalHandle next,
                         int has_next) {
  if (threadIdx.x != 0) return;
  constexpr int R = GState::R;
  double* H = st + GState::kH;
  double* cs = st + GState::kCS;
  double* sn = st + GState::kSN;
  double* g = st + GState::kG;
  double* rn = st + GState::kRN;
  double* sc = st + GState::kSc;
  auto Hm = [&](int i, int q) -> double& { return H[i * R + q]; };
  for (int i = 0; i <= j; ++i) Hm(i, j) = raw[i] / rn[i];
  const double hn = sqrt(nrm2[j + 1]);
  bool stop = true;
  if (!isfinite(hn)) {
    sc[GState::sNan] = 1.0;
  } else {
    Hm(j + 1, j) = hn;
    rn[j + 1] = hn;
    for (int i = 0; i < j; ++i) {
      const double t = cs[i] * Hm(i, j) + sn[i] * Hm(i + 1, j);
      Hm(i + 1, j) = -sn[i] * Hm(i, j) + cs[i] * Hm(i + 1, j);
      Hm(i, j) = t;
    }
    const double den = hypot(Hm(j, j), Hm(j + 1, j));
    if (den == 0.0) {
      sc[GState::sBreak] = 1.0;
    } else {
      cs[j] = Hm(j, j) / den;
      sn[j] = Hm(j + 1, j) / den;
      Hm(j, j) = den;
      Hm(j + 1, j) = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      sc[GState::sJused] = (double)(j + 1);
      const double res = fabs(g[j + 1]);
      const double bnorm = sc[GState::sBnorm];
      st[GState::kHist + j] = res / bnorm;
      stop = res / bnorm <= sc[GState::sRtol] || hn == 0.0 || res <= sc[GState::sStop] ||
             (double)(j + 1) >= sc[GState::sRmax];
    }
  }
  if (has_next) cudaGraphSetConditional(next, stop ? 0u : 1u);
}

// The part of the state the host reads after a cycle, copied to the mapped
// host copy at the same offsets: the scalars, g, the residual history and
// the upper triangle of the first jused columns of H.
__global__ void k_cycle_out(const double* __restrict__ st, double* __restrict__ hst) {
  constexpr int R = GState::R;
  const int ju = (int)st[GState::kSc + GState::sJused];
  for (int i = threadIdx.x; i < 16; i += blockDim.x) hst[GState::kSc + i] = st[GState::kSc + i];
  for (int i = threadIdx.x; i <= R; i += blockDim.x) hst[GState::kG + i] = st[GState::kG + i];
  for (int i = threadIdx.x; i < R; i += blockDim.x) hst[GState::kHist + i] = st[GState::kHist + i];
  for (int e = threadIdx.x; e < ju * ju; e += blockDim.x) {
    const int i = e / ju, q = e - i * ju;
    if (i <= q) hst[GState::kH + i * R + q] = st[GState::kH + i * R + q];
  }
}

// What a cycle graph depends on besides the context's fixed buffers.
void cycle_key(const ibm_ctx* c, const ibm_solve_opts* o, int restart,
               unsigned long long (&k)[16]) {
  const MarkerData& m = c->mk;
  const unsigned long long v[16] = {
      (unsigned long long)restart, (unsigned long long)o->mg_pre, (unsigned long long)o->mg_post,
      (unsigned long long)o->arnoldi, (unsigned long long)c->cmode, (unsigned long long)m.n,
      (unsigned long long)m.n_shell, (unsigned long long)m.n_ell,
      (unsigned long long)(uintptr_t)m.bf, (unsigned long long)(uintptr_t)m.ell_key,
      (unsigned long long)(uintptr_t)m.ell_base, (unsigned long long)c->m, 1ull, 0ull, 0ull, 0ull};
  for (int i = 0; i < 16; ++i) k[i] = v[i];
}

void drop_cycle_graph(ibm_ctx* c) {
  if (c->cyc_exec) cudaGraphExecDestroy(c->cyc_exec);
  if (c->cyc_graph) cudaGraphDestroy(c->cyc_graph);
  c->cyc_exec = nullptr;
  c->cyc_graph = nullptr;
  for (auto& v : c->cyc_key) v = 0;
}

// Captures iterations 0..restart-1 (launch_iter(j, true) on the capture
// stream) with their k_givens and the nested IF nodes; false (and the
// host-driven loop) if any step fails.  Kernels captured are not counted
// as launched; cyc_launches[j] holds iteration j's count for the replays.
template <typename F>
bool build_cycle_graph(ibm_ctx* c, int restart, F& launch_iter) {
  drop_cycle_graph(c);
  cudaGraph_t G = nullptr;
  if (cudaGraphCreate(&G, 0) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cudaStream_t saved = c->stream;
  c->stream = c->cap;
  const double* raw = c->red_out;
  const double* nrm2 = c->red_out + 4 * kOutStride;
  cudaGraph_t cur = G;
  bool ok = true;
  for (int j = 0; j < restart && ok; ++j) {
    if (cudaStreamBeginCaptureToGraph(c->cap, cur, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      ok = false;
      break;
    }
    const long long l0 = ibm_kernel_launches();
    ok = launch_iter(j, true) == IBM_OK;
    const bool has_next = j + 1 < restart;
    cudaGraphConditionalHandle h = 0;
    if (ok && has_next)
      ok = cudaGraphConditionalHandleCreate(&h, cur, 0, cudaGraphCondAssignDefault) == cudaSuccess;
    if (ok) {
      k_givens<<<1, 32, 0, c->cap>>>(c->gstate, j, raw, nrm2, h, has_next ? 1 : 0);
      ok = cudaGetLastError() == cudaSuccess;
    }
    cudaGraph_t next = nullptr;
    if (ok && has_next) {
      cudaStreamCaptureStatus cst;
      cudaGraph_t capg = nullptr;
      const cudaGraphNode_t* deps = nullptr;
      size_t nd = 0;
      ok = cudaStreamGetCaptureInfo(c->cap, &cst, nullptr, &capg, &deps, nullptr, &nd) ==
               cudaSuccess &&
           cst == cudaStreamCaptureStatusActive;
      cudaGraphNodeParams p = {};
      p.type = cudaGraphNodeTypeConditional;
      p.conditional.handle = h;
      p.conditional.type = cudaGraphCondTypeIf;
      p.conditional.size = 1;
      cudaGraphNode_t node = nullptr;
      if (ok) ok = cudaGraphAddNode(&node, capg, deps, nullptr, nd, &p) == cudaSuccess;
      if (ok)
        ok = cudaStreamUpdateCaptureDependencies(c->cap, &node, nullptr, 1,
                                                 cudaStreamSetCaptureDependencies) == cudaSuccess;
      if (ok) next = p.conditional.phGraph_out[0];
    }
    cudaGraph_t out = nullptr;
    if (cudaStreamEndCapture(c->cap, &out) != cudaSuccess) ok = false;
    const long long dl = ibm_kernel_launches() - l0;
    add_launches(-dl);
    c->cyc_launches[j] = (int)dl + 1;   // and k_givens
    cur = next;
  }
  c->stream = saved;
  cudaGraphExec_t exec = nullptr;
  if (ok) ok = cudaGraphInstantiate(&exec, G, 0) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    if (exec) cudaGraphExecDestroy(exec);
    cudaGraphDestroy(G);
    return false;
  }
  c->cyc_graph = G;
  c->cyc_exec = exec;
  return true;
}

ibm_status fgmres_solve_ds(ibm_ctx* c, const double* b, double* x, const ibm_solve_opts* o,
                           ibm_solve_stats* st, bool x_is_zero) {
  // Same flexible GMRES as fgmres_solve (unnormalised Arnoldi vectors with
  // squared norms nrm2[i] on the device), with the vectors as FP32 pairs
  // (Vhi/Vlo reuse the FP64 basis storage) or, for IBM_ARNOLDI_FP32, single
  // FP32 numbers; Z holds the FP32 V-cycle outputs.  A single-precision cycle
  // stops once its residual estimate has fallen by kSingleCycle (the FP32
  // basis cannot resolve more) and the next cycle starts from the FP64
  // residual.
  const bool single = o->arnoldi == IBM_ARNOLDI_FP32;
  // float4 Gram-Schmidt kernels: every basis vector starts on a 16-byte boundary
  const bool vec4 = single && c->m % 4 == 0;
  constexpr double kSingleCycle = 4e-6;
  cudaStream_t s = c->stream;
  const int64_t m = c->m;
  const int restart = o->restart;
  double* part = c->red_part;
  double* raw = c->red_out;
  double* coef = c->red_out + kOutStride;
  float2* coef_ds = reinterpret_cast<float2*>(c->red_out + 2 * kOutStride);
  double* nrm2 = c->red_out + 4 * kOutStride;
  double* sdev = c->red_out + 6 * kOutStride;
  double* hr = c->host_red;
  float2* V2 = reinterpret_cast<float2*>(c->V);
  float* V1 = reinterpret_cast<float*>(c->V);
  float* Zf = reinterpret_cast<float*>(c->Z);
  // leading parts of the newest basis vector, contiguous: the V-cycle input
  // (the vector itself in the single-precision form)
  float* vin = c->lv[0].b32;
  double* r64 = c->c1;
  ibm_status stt;

  launch_dot(b, b, m, part, sdev, s);
  prof_note(c, 8.0 * m);
  IBM_LAUNCH_CHECK(c);
  if ((stt = fetch(c, sdev, 1)) != IBM_OK) return stt;
  const double bnorm = std::sqrt(hr[0]);
  if (!std::isfinite(bnorm)) return set_err(c, IBM_ERR_NAN, "non-finite right-hand side");
  int total = 0, cycles = 0, graph_cycles = 0;
  double relres = 0.0;
  if (bnorm == 0.0) {
    launch_zero(x, sizeof(double) * m, s);
    if (st) { st->iters = 0; st->restarts = 0; st->relres_true = 0.0; st->graph_cycles = 0; }
    return IBM_OK;
  }
  std::vector<double> H((size_t)(restart + 1) * restart), cs(restart), sn(restart),
      g(restart + 1), y(restart), rn(restart + 1);
  auto Hm = [&](int i, int j) -> double& { return H[(size_t)i * restart + j]; };
  bool converged = false, first = true;
  ibm_status final_status = IBM_OK;
  while (true) {
    // FP64 residual r0 = b - S~ x (r0 = b for a zero first guess)
    double beta;
    const double* r0 = b;
    if (first && x_is_zero) {
      launch_copy(nrm2, sdev, sizeof(double), s);
      beta = bnorm;
    } else {
      if ((stt = schur_residual(c, b, x, r64)) != IBM_OK) return stt;
      launch_dot(r64, r64, m, part, nrm2, s);
      prof_note(c, 8.0 * m);
      IBM_LAUNCH_CHECK(c);
      if ((stt = fetch(c, nrm2, 1)) != IBM_OK) return stt;
      beta = std::sqrt(hr[0]);
      r0 = r64;
    }
    first = false;
    if (!std::isfinite(beta)) return set_err(c, IBM_ERR_NAN, "non-finite residual");
    relres = beta / bnorm;
    if (relres <= o->rtol) { converged = true; break; }
    if (total >= o->maxit) break;
    count_launch();
    if (single) {
      k_round_f32<<<kRedBlocks, RT, 0, s>>>(r0, V1, m);
      vin = V1;
      prof_note(c, 12.0 * m);
    } else {
      k_split<<<kRedBlocks, RT, 0, s>>>(r0, V2, vin, m);
      prof_note(c, 20.0 * m);
    }
    rn[0] = beta;
    const double cycle_stop = single ? kSingleCycle * beta : 0.0;
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int jused = 0;
    bool breakdown = false;
    // Iteration j's kernels: V-cycle, Schur product, Gram-Schmidt; the
    // Hessenberg column goes to the host mirror (raw part in one of two
    // buffers by the parity of j, apart from the scalar slot at the mirror's
    // start that other reads use) and an event marks the iteration's end.
    auto launch_iter = [&](int jj, bool graph) -> ibm_status {
      // graph: captured into a cycle graph (on the capture stream, which
      // c->stream names meanwhile; no host mirror, no end event)
      cudaStream_t s = c->stream;
      float* zj = Zf + (int64_t)jj * m;
      float2* w = V2 + (int64_t)(jj + 1) * m;
      float* w1 = V1 + (int64_t)(jj + 1) * m;
      const double mk0 = prof_mark(c);
      int ph = prof_begin(c, IBM_PROF_VCYCLE);
      ibm_status sv;
      if ((sv = mg_vcycle_f32(c, single ? V1 + (int64_t)jj * m : vin, zj, o->mg_pre,
                              o->mg_post)) != IBM_OK)
        return sv;
      prof_end_span(c, ph, mk0);
      if ((sv = single ? schur_apply_ds_t<float>(c, zj, w1) : schur_apply_ds_t<float2>(c, zj, w)) !=
          IBM_OK)
        return sv;
      const int nq = jj + 1;
      ph = prof_begin(c, IBM_PROF_MULTIDOT);
      if (vec4 && nq <= 16)
        IBM_NQ_DISPATCH_SP4(nq, k_multidot_sp4, reinterpret_cast<const float4*>(w1),
                            reinterpret_cast<const float4*>(V1), m / 4, nq, m / 4, part);
      else if (single)
        IBM_NQ_DISPATCH_DS(nq, k_multidot_sp, w1, V1, m, nq, m, part);
      else
        IBM_NQ_DISPATCH_DS(nq, k_multidot_ds, w, V2, m, nq, m, part);
      count_launch();
      launch_pdl(k_final_reduce_ds, dim3(nq), dim3(RT), 0, s, (const double*)part, kRedBlocks,
                 raw, (const double*)nrm2, coef, coef_ds,
                 graph ? nullptr : hmirror(c, hr + (2 + (jj & 1)) * kOutStride));
      prof_end(c, ph, (single ? 4.0 : 8.0) * (nq + 1) * (double)m);
      ph = prof_begin(c, IBM_PROF_AXPY_NORM);
      if (vec4 && nq <= 16)
        IBM_NQ_DISPATCH_SP4(nq, k_axpy_norm_sp4, reinterpret_cast<float4*>(w1),
                            reinterpret_cast<const float4*>(V1), m / 4, nq, coef_ds, m / 4, part);
      else if (single)
        IBM_NQ_DISPATCH_DS(nq, k_axpy_norm_sp, w1, V1, m, nq, coef_ds, m, part);
      else
        IBM_NQ_DISPATCH_DS(nq, k_axpy_norm_ds, w, V2, m, nq, coef_ds, m, part, vin);
      count_launch();
      launch_pdl(k_final_reduce_ds, dim3(1), dim3(RT), 0, s, (const double*)part, kRedBlocks,
                 nrm2 + jj + 1, (const double*)nullptr, (double*)nullptr, (float2*)nullptr,
                 graph ? nullptr : hmirror(c, hr + 4 * kOutStride + jj + 1));
      // V_0..V_j and w read, w written (and its leading parts for the pair form)
      prof_end(c, ph, single ? 4.0 * (nq + 2) * (double)m : (8.0 * (nq + 2) + 4.0) * (double)m);
      IBM_LAUNCH_CHECK(c);
      if (!graph) IBM_CUDA(c, cudaEventRecord(c->ev_iter[jj & 1], s));
      return IBM_OK;
    };
    // The host stays one iteration behind the device where that is safe:
    // iteration j+1 (which needs nothing from the host) is launched before
    // iteration j's column is read whenever the residual estimate, shrinking
    // at the fastest rate seen so far, cannot reach the stopping threshold at
    // iteration j; so the device does not idle during the host's read and
    // Givens update.  A wrong guess costs the unused iteration j+1; the
    // iterates and the iteration count do not depend on the guesses.  The
    // exact and sign-consistent forms, whose Schur product waits on the host
    // (inner conjugate gradients), run one iteration at a time.
    // the cycle as one graph replay where it applies
    const bool graph_form = o->cycle_graphs == 1 && !c->prof_on && c->cmode == IBM_CMODE_SCALAR &&
                            c->cap != nullptr && restart > 0 && restart <= kMaxRestart &&
                            total < o->maxit;
    if (graph_form) {
      unsigned long long key[16];
      cycle_key(c, o, restart, key);
      if (!std::equal(key, key + 16, c->cyc_key)) {
        // also kept when the build fails: the host-driven loop runs, and the
        // capture is not tried again for the same key
        build_cycle_graph(c, restart, launch_iter);
        std::copy(key, key + 16, c->cyc_key);
      }
    }
    if (graph_form && c->cyc_exec) {
      const int rmax = std::min(restart, o->maxit - total);
      count_launch();
      k_cycle_init<<<1, RT, 0, s>>>(c->gstate, beta, bnorm, o->rtol, cycle_stop, rmax);
      IBM_CUDA(c, cudaGraphLaunch(c->cyc_exec, s));
      count_launch();
      k_cycle_out<<<1, 256, 0, s>>>(c->gstate, c->host_gstate_dev);
      IBM_LAUNCH_CHECK(c);
      IBM_CUDA(c, cudaStreamSynchronize(s));
      const double* hs = c->host_gstate;
      const double* sc = hs + GState::kSc;
      const int ju = (int)sc[GState::sJused];
      const bool nan_col = sc[GState::sNan] != 0.0;
      breakdown = sc[GState::sBreak] != 0.0;
      const int ran = std::min(restart, (nan_col || breakdown) ? ju + 1 : ju);
      int64_t lsum = 0;
      for (int q = 0; q < ran; ++q) lsum += c->cyc_launches[q];
      add_launches(lsum);
      if (nan_col) return set_err(c, IBM_ERR_NAN, "non-finite Arnoldi vector");
      for (int q = 0; q < ju; ++q)
        for (int i = 0; i <= q; ++i) Hm(i, q) = hs[GState::kH + i * GState::R + q];
      for (int i = 0; i <= ju; ++i) g[i] = hs[GState::kG + i];
      for (int q = 0; q < ju; ++q)
        if (st && total + q < IBM_HIST_MAX) st->relres_hist[total + q] = hs[GState::kHist + q];
      total += ju;
      jused = ju;
      ++graph_cycles;
    } else {
      const double thresh = std::max(o->rtol * bnorm, cycle_stop);
      const bool ahead = c->cmode == IBM_CMODE_SCALAR;
      double prev = beta, rate = 0.05;   // assumed until a ratio has been seen
      bool have_rate = false;
      bool next_launched = false;
      if (restart > 0 && total < o->maxit) {
        if ((stt = launch_iter(0, false)) != IBM_OK) return stt;
        next_launched = true;
      }
      for (int j = 0; next_launched; ++j) {
        const bool can_next = j + 1 < restart && total + 1 < o->maxit;
        next_launched = false;
        if (ahead && can_next && prev * rate > 4.0 * thresh) {
          if ((stt = launch_iter(j + 1, false)) != IBM_OK) return stt;
          next_launched = true;
        }
        IBM_CUDA(c, cudaEventSynchronize(c->ev_iter[j & 1]));
        const double* hraw = hr + (2 + (j & 1)) * kOutStride;
        for (int i = 0; i <= j; ++i) Hm(i, j) = hraw[i] / rn[i];
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
        const double res = std::fabs(g[j + 1]);
        if (st && total - 1 < IBM_HIST_MAX) st->relres_hist[total - 1] = res / bnorm;
        if (res / bnorm <= o->rtol || hn == 0.0) break;
        if (res <= cycle_stop) break;   // FP32 basis exhausted
        if (prev > 0.0) {
          rate = have_rate ? std::min(rate, res / prev) : res / prev;
          have_rate = true;
        }
        prev = res;
        if (!next_launched && can_next) {
          if ((stt = launch_iter(j + 1, false)) != IBM_OK) return stt;
          next_launched = true;
        }
      }
    }
    if (jused > 0) {
      for (int i = jused - 1; i >= 0; --i) {
        double acc = g[i];
        for (int q = i + 1; q < jused; ++q) acc -= Hm(i, q) * y[q];
        y[i] = acc / Hm(i, i);
      }
      CoefDS cy;
      for (int i = 0; i <= kMaxRestart; ++i) {
        const double yi = i < jused ? y[i] : 0.0;
        const float yh = (float)yi;
        cy.v[i] = make_float2(yh, (float)(yi - (double)yh));
      }
      if (m % 4 == 0 && jused <= 16 && (reinterpret_cast<uintptr_t>(x) & 15u) == 0)
        IBM_NQ_DISPATCH_SP4(jused, k_gemv_ds4, reinterpret_cast<double2*>(x),
                            reinterpret_cast<const float4*>(Zf), m / 4, jused, cy, m / 4);
      else
        IBM_NQ_DISPATCH_DS(jused, k_gemv_ds, x, Zf, m, jused, cy, m);
      prof_note(c, (4.0 * jused + 16.0) * (double)m);
      IBM_LAUNCH_CHECK(c);
    }
    ++cycles;
    if (breakdown && jused == 0) { final_status = IBM_ERR_BREAKDOWN; break; }
  }
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
    st->relres_true = relres;
    st->graph_cycles = graph_cycles;
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
