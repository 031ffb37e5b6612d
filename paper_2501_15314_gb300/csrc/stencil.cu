// Staggered MAC-grid stencils (Sec. 3.1): the Neumann Laplacian L = G^T G of
// Eq. (Saddle), the gradient G and its transpose G^T = -div, and the pieces of
// the BDF2 momentum predictor of Eq. (ustar) (Helmholtz operator, explicit
// convective term, right-hand side).
//
// Thread layout: one thread per grid point, blocks of 32 x 8 in (x, y) and one
// z-plane per blockIdx.z, so that a warp reads 32 consecutive x values of each
// neighbour row (coalesced; the y/z neighbours hit L1/L2).
#include <algorithm>
#include <cstring>
#include <type_traits>

#include "ds.cuh"
#include "ibm_internal.cuh"

namespace ibm {

namespace {

constexpr int BX = 32, BY = 8;

// Geometry of the packed face vector: comp c has n[c][axis] points per axis.
struct FaceGeom {
  int n[3][3];
  int64_t off[3];
  int64_t sy[3], sz[3];
};

FaceGeom make_face_geom(Dims d) {
  FaceGeom g;
  FaceDims f = face_dims(d);
  int base[3] = {d.nx, d.ny, d.nz};
  for (int c = 0; c < 3; ++c) {
    for (int a = 0; a < 3; ++a) g.n[c][a] = base[a] + (a == c ? 1 : 0);
    g.sy[c] = g.n[c][0];
    g.sz[c] = (int64_t)g.n[c][0] * g.n[c][1];
  }
  g.off[0] = 0;
  g.off[1] = f.nfx;
  g.off[2] = f.nfx + f.nfy;
  return g;
}


dim3 cell_grid(Dims d) { return dim3(div_up(d.nx, BX), div_up(d.ny, BY), d.nz); }

// ---------------------------------------------------------------------------
// L v = G^T G v: sum over existing neighbours of (v_c - v_n) / h^2.
template <typename T>
__global__ void __launch_bounds__(BX * BY) k_laplacian(Dims d, const T* __restrict__ v,
                                                       T* __restrict__ out, T inv_h2) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= d.nx || j >= d.ny) return;
  const int64_t sy = d.nx, sz = (int64_t)d.nx * d.ny;
  const int64_t c = k * sz + j * sy + i;
  const T vc = __ldg(v + c);
  T r;
  if (i > 0 && i < d.nx - 1 && j > 0 && j < d.ny - 1 && k > 0 && k < d.nz - 1) {
    const T s = ((__ldg(v + c - 1) + __ldg(v + c + 1)) + (__ldg(v + c - sy) + __ldg(v + c + sy))) +
                (__ldg(v + c - sz) + __ldg(v + c + sz));
    r = fma((T)6, vc, -s);
  } else {
    T s = 0;
    int nn = 0;
    if (i > 0) { s += __ldg(v + c - 1); ++nn; }
    if (i < d.nx - 1) { s += __ldg(v + c + 1); ++nn; }
    if (j > 0) { s += __ldg(v + c - sy); ++nn; }
    if (j < d.ny - 1) { s += __ldg(v + c + sy); ++nn; }
    if (k > 0) { s += __ldg(v + c - sz); ++nn; }
    if (k < d.nz - 1) { s += __ldg(v + c + sz); ++nn; }
    r = fma((T)nn, vc, -s);
  }
  out[c] = r * inv_h2;
}

// ---------------------------------------------------------------------------
// FP64 Laplacian with the stencil sum formed exactly in integers.  GB300
// issues FP64 arithmetic at about 1/58 of its FP32 rate, so the seven-term
// FP64 sum bounds k_laplacian<double> far below the HBM rate.  Here each
// value v = m 2^(e - 1075) (m the signed 53-bit significand, e the biased
// exponent; a subnormal has e = 1 and no implicit bit) is aligned to the
// largest exponent E of the seven with kLapGuard extra low bits, and
// S = nn m_c - sum_nb m_nb is summed in 64-bit integers: the bits dropped
// below 2^(E - 1075 - kLapGuard) amount to at most 7 2^-kLapGuard units in
// the last place of the largest term, less than the rounding error of the
// FP64 sum.  Then out = (double)S 2^(E - 1075 - kLapGuard) / h^2 with two
// roundings (the conversion and one multiplication; the scale is 1/h^2 with
// E - 1080 added to its exponent field).  Non-finite values, and sums whose
// scale would leave the normal range, take the FP64 formula.
constexpr int kLapGuard = 5;

struct FxVal {
  int e;
  long long m;
};

__device__ __forceinline__ FxVal fx_unpack(double v) {
  const long long u = __double_as_longlong(v);
  int e = (int)((u >> 52) & 0x7ff);
  long long m = u & 0xFFFFFFFFFFFFFLL;
  if (e != 0)
    m |= 1LL << 52;
  else
    e = 1;
  return {e, u < 0 ? -m : m};
}

// m 2^kLapGuard shifted down to exponent E (|m| < 2^56, so no overflow)
__device__ __forceinline__ long long fx_align(long long m, int e, int E) {
  return (m * (1LL << kLapGuard)) >> min(E - e, 63);
}

// (nn v_c - sum of the six neighbour values) / h^2; an absent neighbour is 0
__device__ __forceinline__ double lap_fx(double vc, double xm, double xp, double ym, double yp,
                                         double zm, double zp, int nn, long long inv_h2_bits,
                                         int e_min, int e_max) {
  const FxVal c = fx_unpack(vc), a0 = fx_unpack(xm), a1 = fx_unpack(xp), a2 = fx_unpack(ym),
              a3 = fx_unpack(yp), a4 = fx_unpack(zm), a5 = fx_unpack(zp);
  const int E = max(max(max(c.e, a0.e), max(a1.e, a2.e)), max(max(a3.e, a4.e), a5.e));
  if (E < e_min || E > e_max) {
    const double s = ((xm + xp) + (ym + yp)) + (zm + zp);
    return fma((double)nn, vc, -s) * __longlong_as_double(inv_h2_bits);
  }
  long long S = fx_align(c.m * nn, c.e, E);
  S -= fx_align(a0.m, a0.e, E) + fx_align(a1.m, a1.e, E);
  S -= fx_align(a2.m, a2.e, E) + fx_align(a3.m, a3.e, E);
  S -= fx_align(a4.m, a4.e, E) + fx_align(a5.m, a5.e, E);
  const double scale =
      __longlong_as_double(inv_h2_bits + (long long)(E - 1075 - kLapGuard) * (1LL << 52));
  return __ll2double_rn(S) * scale;
}

// One cell per thread, blocks of 32 x 8 cells over zc z-planes: x-neighbours
// by shuffles (loads at the warp edges), z-neighbours from the registers of
// the march, y-neighbours through L1.
__global__ void __launch_bounds__(BX * BY) k_laplacian_fx(Dims d, const double* __restrict__ v,
                                                          const double* __restrict__ bsub,
                                                          double* __restrict__ out,
                                                          long long inv_h2_bits, int e_min,
                                                          int e_max, int zc) {
  const int lane = threadIdx.x;
  const int i = blockIdx.x * BX + lane;
  const int j = blockIdx.y * BY + threadIdx.y;
  const bool act = i < d.nx && j < d.ny;
  const int z0 = blockIdx.z * zc;
  const int z1 = min(z0 + zc, d.nz);
  const int64_t sy = d.nx, sz = (int64_t)d.nx * d.ny;
  int64_t c = (int64_t)z0 * sz + (int64_t)j * sy + i;
  const bool hxm = i > 0, hxp = i < d.nx - 1, hym = j > 0, hyp = j < d.ny - 1;
  const int nxy = (int)hxm + (int)hxp + (int)hym + (int)hyp;
  double vp = (act && z0 > 0) ? __ldg(v + c - sz) : 0.0;
  double vc = act ? __ldg(v + c) : 0.0;
  for (int z = z0; z < z1; ++z, c += sz) {
    double vn = 0.0, ym = 0.0, yp = 0.0;
    if (act) {
      if (z + 1 < d.nz) vn = __ldg(v + c + sz);
      if (hym) ym = __ldg(v + c - sy);
      if (hyp) yp = __ldg(v + c + sy);
    }
    double xm = __shfl_up_sync(0xffffffffu, vc, 1);
    double xp = __shfl_down_sync(0xffffffffu, vc, 1);
    if (lane == 0) xm = (act && hxm) ? __ldg(v + c - 1) : 0.0;
    if (lane == 31) xp = (act && hxp) ? __ldg(v + c + 1) : 0.0;
    if (!hxm) xm = 0.0;
    if (!hxp) xp = 0.0;
    const int nn = nxy + (z > 0) + (z < d.nz - 1);
    if (act) {
      const double lv = lap_fx(vc, xm, xp, ym, yp, vp, vn, nn, inv_h2_bits, e_min, e_max);
      out[c] = bsub ? __ldg(bsub + c) - lv : lv;   // b - L v for the true residual
    }
    vp = vc;
    vc = vn;
  }
}

// Scale limits for a fixed-point sum scaled by `scale` (as in lap_fx): the
// scale 2^(E - 1075 - kLapGuard) * scale is formed by adding E - 1075 -
// kLapGuard to the exponent field of `scale`, which must stay in [1, 2046];
// anything else (a non-finite value; a scale that is zero, subnormal or not
// finite) takes the FP64 formula.
struct FxLimits {
  long long bits;
  int e_min, e_max;
};

FxLimits fx_limits(double scale) {
  FxLimits L;
  std::memcpy(&L.bits, &scale, sizeof(L.bits));
  const int e_h = (int)((L.bits >> 52) & 0x7ff);
  L.e_min = std::max(1075 + kLapGuard + 1 - e_h, 1);
  L.e_max = std::min(2046 + 1075 + kLapGuard - e_h, 2046);
  if (e_h == 0 || e_h == 0x7ff) L.e_min = 2047;
  return L;
}

// alpha ((a0 - a1) + (a2 - a3) + (a4 - a5)) with the sum formed exactly in
// 64-bit integers as in lap_fx (|S| < 6 2^58)
__device__ __forceinline__ double div_fx(double a0, double a1, double a2, double a3, double a4,
                                         double a5, FxLimits L) {
  const FxVal v0 = fx_unpack(a0), v1 = fx_unpack(a1), v2 = fx_unpack(a2), v3 = fx_unpack(a3),
              v4 = fx_unpack(a4), v5 = fx_unpack(a5);
  const int E = max(max(max(v0.e, v1.e), max(v2.e, v3.e)), max(v4.e, v5.e));
  if (E < L.e_min || E > L.e_max)
    return __longlong_as_double(L.bits) * (((a0 - a1) + (a2 - a3)) + (a4 - a5));
  long long S = fx_align(v0.m, v0.e, E) - fx_align(v1.m, v1.e, E);
  S += fx_align(v2.m, v2.e, E) - fx_align(v3.m, v3.e, E);
  S += fx_align(v4.m, v4.e, E) - fx_align(v5.m, v5.e, E);
  const double scale =
      __longlong_as_double(L.bits + (long long)(E - 1075 - kLapGuard) * (1LL << 52));
  return __ll2double_rn(S) * scale;
}

// out = alpha * G^T u + beta * cin (cin may be null), (G^T u)_c = sum_d
// (u_{c-1/2} - u_{c+1/2}) over interior faces (wall faces read as 0), the
// sum formed exactly (div_fx).  One cell per thread, blocks of 32 x 8 cells
// over zc planes: the upper x-face from the next lane, the lower z-face from
// the march, the y-faces through L1.  NORM: instead of out, the block's sum
// of the squared values (FP64, fixed order) goes to sq_part[block].
template <bool NORM>
__global__ void __launch_bounds__(BX * BY) k_gradt_fx(Dims d, FaceGeom g,
                                                      const double* __restrict__ u, FxLimits L,
                                                      const double* __restrict__ cin,
                                                      double beta, double* __restrict__ out,
                                                      double* __restrict__ sq_part, int zc) {
  const int lane = threadIdx.x;
  const int i = blockIdx.x * BX + lane;
  const int j = blockIdx.y * BY + threadIdx.y;
  const bool act = i < d.nx && j < d.ny;
  const int z0 = blockIdx.z * zc;
  const int z1 = min(z0 + zc, d.nz);
  const double* ux = u + g.off[0];
  const double* uy = u + g.off[1];
  const double* uz = u + g.off[2];
  // interior faces: x-faces 1..nx-1, y-faces 1..ny-1, z-faces 1..nz-1
  const bool xlo = i > 0, xhi = i + 1 < d.nx, ylo = j > 0, yhi = j + 1 < d.ny;
  double zlo = (act && z0 > 0) ? __ldg(uz + (int64_t)z0 * g.sz[2] + (int64_t)j * g.sy[2] + i) : 0.0;
  double sq = 0.0;
  for (int z = z0; z < z1; ++z) {
    const int64_t fx = (int64_t)z * g.sz[0] + (int64_t)j * g.sy[0] + i;
    const int64_t fy = (int64_t)z * g.sz[1] + (int64_t)j * g.sy[1] + i;
    double a0 = 0.0, a2 = 0.0, a3 = 0.0, zhi = 0.0;
    if (act) {
      if (xlo) a0 = __ldg(ux + fx);
      if (ylo) a2 = __ldg(uy + fy);
      if (yhi) a3 = __ldg(uy + fy + g.sy[1]);
      if (z + 1 < d.nz) zhi = __ldg(uz + (int64_t)(z + 1) * g.sz[2] + (int64_t)j * g.sy[2] + i);
    }
    // the upper x-face of cell i is the lower one of cell i + 1
    double a1 = __shfl_down_sync(0xffffffffu, a0, 1);
    if (lane == 31) a1 = (act && xhi) ? __ldg(ux + fx + 1) : 0.0;
    if (!xhi) a1 = 0.0;
    if (act) {
      const double v = div_fx(a0, a1, a2, a3, zlo, zhi, L);
      if constexpr (NORM) {
        sq = fma(v, v, sq);
      } else {
        const int64_t c = ((int64_t)z * d.ny + j) * d.nx + i;
        out[c] = cin ? fma(beta, __ldg(cin + c), v) : v;
      }
    }
    zlo = zhi;
  }
  if constexpr (NORM) {
    __shared__ double sh[BY];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_down_sync(0xffffffffu, sq, o);
    if (lane == 0) sh[threadIdx.y] = sq;
    __syncthreads();
    if (lane == 0 && threadIdx.y == 0) {
      double t = 0.0;
#pragma unroll
      for (int w = 0; w < BY; ++w) t += sh[w];
      sq_part[((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = t;
    }
  }
}

// u = u_in + alpha * G p on interior faces, 0 on wall faces (u_in may be
// null; it may be u).  Thread (i, j) marches over the z-planes 0..nz and
// writes the x-, y- and z-faces at (i, j, k) that exist: p(i-1) comes from
// the previous lane, p(k-1) from the march, p(j-1) through L1.
__global__ void __launch_bounds__(BX * BY) k_grad_axpy(Dims d, FaceGeom g,
                                                       const double* __restrict__ u_in,
                                                       const double* __restrict__ p,
                                                       double alpha, double* __restrict__ u,
                                                       int zc) {
  const int lane = threadIdx.x;
  const int i = blockIdx.x * BX + lane;
  const int j = blockIdx.y * BY + threadIdx.y;
  const bool col = i <= d.nx && j <= d.ny;      // some face of this column exists
  const bool cell = i < d.nx && j < d.ny;       // the cell column exists
  const int z0 = blockIdx.z * zc;
  const int z1 = min(z0 + zc, d.nz + 1);
  const int64_t sy = d.nx, sz = (int64_t)d.nx * d.ny;
  auto pc_at = [&](int k) { return (int64_t)k * sz + (int64_t)j * sy + i; };
  double pzm = (cell && z0 > 0 && z0 - 1 < d.nz) ? __ldg(p + pc_at(z0 - 1)) : 0.0;
  for (int k = z0; k < z1; ++k) {
    const bool kin = k < d.nz;
    const double pc = (cell && kin) ? __ldg(p + pc_at(k)) : 0.0;
    double pxm = __shfl_up_sync(0xffffffffu, pc, 1);
    if (lane == 0) pxm = (i > 0 && i - 1 < d.nx && j < d.ny && kin) ? __ldg(p + pc_at(k) - 1) : 0.0;
    if (col) {
      // x-face (i, j, k): i in 0..nx, j < ny, k < nz
      if (j < d.ny && kin) {
        const int64_t f = g.off[0] + (int64_t)k * g.sz[0] + (int64_t)j * g.sy[0] + i;
        double val = 0.0;
        if (i > 0 && i < d.nx) {
          const double gp = pc - pxm;
          val = u_in ? fma(alpha, gp, __ldg(u_in + f)) : alpha * gp;
        }
        u[f] = val;
      }
      // y-face (i, j, k): i < nx, j in 0..ny, k < nz
      if (i < d.nx && kin) {
        const int64_t f = g.off[1] + (int64_t)k * g.sz[1] + (int64_t)j * g.sy[1] + i;
        double val = 0.0;
        if (j > 0 && j < d.ny) {
          const double gp = pc - __ldg(p + pc_at(k) - sy);
          val = u_in ? fma(alpha, gp, __ldg(u_in + f)) : alpha * gp;
        }
        u[f] = val;
      }
      // z-face (i, j, k): i < nx, j < ny, k in 0..nz
      if (cell) {
        const int64_t f = g.off[2] + (int64_t)k * g.sz[2] + (int64_t)j * g.sy[2] + i;
        double val = 0.0;
        if (k > 0 && k < d.nz) {
          const double gp = pc - pzm;
          val = u_in ? fma(alpha, gp, __ldg(u_in + f)) : alpha * gp;
        }
        u[f] = val;
      }
    }
    pzm = pc;
  }
}

// Predictor Helmholtz operator on the d-faces, A = a I - nu Lap_h with the
// no-slip ghosts: A e = diag e_c - (nu / h^2) * (sum of neighbours), where the
// face-normal axis reads the wall faces (which hold 0) and each cell-centred
// axis adds nu / h^2 to diag for every missing neighbour (ghost = -e_c).
// Kernels below march along z over ZH planes; blockIdx.z = comp * zchunks +
// chunk, so one launch covers the three face grids.
// x[c] for a runtime c in 0..2 without dynamic indexing (which would copy a
// kernel-parameter struct to local memory)
template <typename T>
__device__ __forceinline__ T sel3(int c, T a, T b, T d) {
  return c == 0 ? a : (c == 1 ? b : d);
}

constexpr int ZH = 16;

// u_E at (x, y, z) of its own face grid, split into an FP32 pair
template <int E>
__device__ __forceinline__ dsf ldu(const FaceGeom& g, const double* __restrict__ u, int x, int y,
                                   int z) {
  return split_exact(__ldg(u + g.off[E] + (int64_t)z * g.sz[E] + (int64_t)y * g.sy[E] + x));
}

// Convective flux on the edge between the C-face at (x, y, z) and the E-face
// index q along E (E != C): (sum of the two u_E adjacent along C) times
// (sum of the two u_C adjacent along E); 0 on the walls (q = 0 or the last
// E-face).  For an interior C-face every value read is an interior face.
template <int C, int E>
__device__ __forceinline__ dsf edge_flux_ds(const FaceGeom& g, const double* __restrict__ u,
                                            int x, int y, int z, int q) {
  if (q <= 0 || q >= g.n[E][E] - 1) return dsf{0.f, 0.f};
  const int ax = E == 0 ? q : x, ay = E == 1 ? q : y, az = E == 2 ? q : z;
  const dsf ue = ds_add_d(ldu<E>(g, u, ax - (C == 0), ay - (C == 1), az - (C == 2)),
                        ldu<E>(g, u, ax, ay, az));
  const dsf uc = ds_add_d(ldu<C>(g, u, ax - (E == 0), ay - (E == 1), az - (E == 2)),
                        ldu<C>(g, u, ax, ay, az));
  return ds_mul(ue, uc);
}

// The same flux in FP64 straight from the FP64 values (no splits): the
// kernel below forms one pair of fluxes per face this way, on the FP64
// pipe, which its double-single arithmetic leaves idle.
template <int C, int E>
__device__ __forceinline__ double edge_flux_f64(const FaceGeom& g, const double* __restrict__ u,
                                                int x, int y, int z, int q) {
  if (q <= 0 || q >= g.n[E][E] - 1) return 0.0;
  const int ax = E == 0 ? q : x, ay = E == 1 ? q : y, az = E == 2 ? q : z;
  auto at = [&](int e, int xx, int yy, int zz) {
    return __ldg(u + g.off[e] + (int64_t)zz * g.sz[e] + (int64_t)yy * g.sy[e] + xx);
  };
  const double ue = at(E, ax - (C == 0), ay - (C == 1), az - (C == 2)) + at(E, ax, ay, az);
  const double uc = at(C, ax - (E == 0), ay - (E == 1), az - (E == 2)) + at(C, ax, ay, az);
  return ue * uc;
}

// Right-hand side of the predictor, Eq. (ustar), with the convective term
// fused in, for the C-faces (one launch per velocity component):
//   rhs = (4 u^n - u^{n-1}) / (2 dt) - G p^n + f - A(u^n) on interior faces
// (0 on wall faces).  A is the central divergence form on the MAC grid (the
// cell-centred square of u_C averaged along C, and on the edges the product
// of u_E averaged along C with u_C averaged along E, 0 on walls) with the 1/2
// averages folded into one factor 1/4:
//   4 A = [ (u_+ + u_0)^2 - (u_0 + u_-)^2 ] along C
//       + sum over the two other axes of (flux at the upper edge - lower edge).
// The march runs along z; the flux through the lower z-edge (or, for u_z, the
// lower cell-centred square) is the previous face's upper one and is reused.
// The FP64 pipe of GB300 is ~58x slower than its FP32 pipes, so the FP64
// inputs are split into FP32 pairs (split_exact, integer operations, 2^-46
// relative) and the formula is evaluated in double-single arithmetic; its
// sums take Dekker's addition (ds_add_d), whose error, a few units of 2^-46
// of the operands, is of the order the inputs' splits already carry.  One
// pair of edge fluxes per face (the y-edges of u_x and u_z, the x-edges of
// u_y) is formed in FP64 from the FP64 values instead, which keeps the
// otherwise idle FP64 pipe busy and saves their splits; their difference
// joins the sum as a pair.  The FP64 result is the exact sum of the pair
// (one FP64 add).
// Templating on C makes every stride and boundary test a compile-time case.
template <int C>
__global__ void __launch_bounds__(BX * BY) k_predictor_rhs_ds(
    Dims d, FaceGeom g, const double* __restrict__ un, const double* __restrict__ unm1,
    const double* __restrict__ pn, const double* __restrict__ fb, int with_adv, dsf c4, dsf c1,
    dsf cp_h, dsf ca, double* __restrict__ rhs) {
  const int lane = threadIdx.x;
  const int i = blockIdx.x * BX + lane;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int n0 = g.n[C][0], n1 = g.n[C][1], n2 = g.n[C][2];
  const int z0 = blockIdx.z * ZH;
  // u_y and u_z faces share their x-edge fluxes between neighbouring lanes,
  // so lanes past the last face stay in the march (without loads or stores);
  // a row past the last one leaves as a whole warp
  const bool act = i < n0;
  if (j >= n1 || (C == 0 && !act)) return;
  const int z1 = min(z0 + ZH, n2);
  const int64_t sy = g.sy[C], sz = g.sz[C];
  int64_t f = g.off[C] + (int64_t)z0 * sz + (int64_t)j * sy + i;
  const bool col_wall = (C == 0 && (i == 0 || i == n0 - 1)) || (C == 1 && (j == 0 || j == n1 - 1));
  if (col_wall) {
    if (act)
      for (int z = z0; z < z1; ++z, f += sz) rhs[f] = 0.0;
    return;
  }
  const int64_t csy = d.nx, csz = (int64_t)d.nx * d.ny;
  const int64_t cstr = C == 0 ? 1 : (C == 1 ? csy : csz);
  const dsf Z = {0.f, 0.f};
  auto sq = [](dsf x) { return ds_mul(x, x); };
  // lower z-flux (C = 0, 1) or lower cell-centred square (C = 2)
  dsf carry = Z;
  if (with_adv && act) {
    if (C == 2) {
      const dsf lo = (z0 - 1 >= 1) ? ldu<2>(g, un, i, j, z0 - 1) : Z;
      const dsf mid = (z0 >= 1 && z0 <= n2 - 2) ? ldu<2>(g, un, i, j, z0) : Z;
      carry = sq(ds_add_d(lo, mid));
    } else {
      carry = edge_flux_ds<C, 2>(g, un, i, j, z0, z0);
    }
  }
  // the flux through the x-edge at q = i + 1 of this lane is the flux
  // through the x-edge at q = i of the next lane (the same values, the same
  // operations); lane 0 forms its lower one itself
  auto xflux_pair = [&](auto fn, dsf& lower) {
    const dsf up = act ? fn(i + 1) : Z;
    lower.hi = __shfl_up_sync(0xffffffffu, up.hi, 1);
    lower.lo = __shfl_up_sync(0xffffffffu, up.lo, 1);
    if (lane == 0) lower = act ? fn(i) : Z;
    return up;
  };
  for (int z = z0; z < z1; ++z, f += sz) {
    if (C == 2 && (z == 0 || z == n2 - 1)) {
      if (!act) continue;
      rhs[f] = 0.0;
      if (with_adv) {
        const dsf mid = (z >= 1 && z <= n2 - 2) ? ldu<2>(g, un, i, j, z) : Z;
        const dsf hi = (z + 1 <= n2 - 2) ? ldu<2>(g, un, i, j, z + 1) : Z;
        carry = sq(ds_add_d(mid, hi));
      }
      continue;
    }
    // x-edge fluxes (shared between lanes: every lane takes part); for u_y
    // in FP64 (its pair of fluxes on the FP64 pipe)
    dsf fx_lo = Z, fx_up = Z;
    double fx64_lo = 0.0, fx64_up = 0.0;
    if (with_adv && C == 2) {
      fx_up = xflux_pair([&](int q) { return edge_flux_ds<2, 0>(g, un, i, j, z, q); }, fx_lo);
    } else if (with_adv && C == 1) {
      fx64_up = act ? edge_flux_f64<1, 0>(g, un, i, j, z, i + 1) : 0.0;
      fx64_lo = __shfl_up_sync(0xffffffffu, fx64_up, 1);
      if (lane == 0) fx64_lo = act ? edge_flux_f64<1, 0>(g, un, i, j, z, i) : 0.0;
    }
    if (!act) continue;
    const int64_t cp = (int64_t)z * csz + (int64_t)j * csy + i;   // cell on the + side
    const dsf u0 = split_exact(__ldg(un + f));
    // 4/(2dt) u^n - 1/(2dt) u^{n-1} - (p_+ - p_-)/h (+ f)
    dsf v = ds_add_d(ds_mul(c4, u0), ds_neg(ds_mul(c1, split_exact(__ldg(unm1 + f)))));
    const dsf dp = ds_add_d(split_exact(__ldg(pn + cp)), ds_neg(split_exact(__ldg(pn + cp - cstr))));
    v = ds_add_d(v, ds_neg(ds_mul(cp_h, dp)));
    if (fb) v = ds_add_d(v, split_exact(__ldg(fb + f)));
    if (with_adv) {
      dsf acc;
      if (C == 2) {
        const dsf up = (z + 1 <= n2 - 2) ? ldu<2>(g, un, i, j, z + 1) : Z;
        const dsf up2 = sq(ds_add_d(u0, up));
        acc = ds_add_d(up2, ds_neg(carry));
        carry = up2;
        acc = ds_add_d(acc, ds_add_d(fx_up, ds_neg(fx_lo)));
        // y-edges in FP64
        acc = ds_add_d(acc, split_exact(edge_flux_f64<2, 1>(g, un, i, j, z, j + 1) -
                                        edge_flux_f64<2, 1>(g, un, i, j, z, j)));
      } else {
        // own axis: (u_+ - u_-)(u_+ + 2 u_0 + u_-), wall faces read as 0
        constexpr int O = 1 - C;   // the other in-plane axis
        const int pc = C == 0 ? i : j, nc = C == 0 ? n0 : n1;
        const dsf up = (pc + 1 <= nc - 2) ? ldu<C>(g, un, i + (C == 0), j + (C == 1), z) : Z;
        const dsf um = (pc - 1 >= 1) ? ldu<C>(g, un, i - (C == 0), j - (C == 1), z) : Z;
        const dsf two_u0 = {2.f * u0.hi, 2.f * u0.lo};
        acc = ds_mul(ds_add_d(up, ds_neg(um)), ds_add_d(ds_add_d(up, um), two_u0));
        // the other in-plane axis's pair of fluxes in FP64 (x for u_y, y for u_x)
        if (O == 0) {
          acc = ds_add_d(acc, split_exact(fx64_up - fx64_lo));
        } else {
          acc = ds_add_d(acc, split_exact(edge_flux_f64<C, O>(g, un, i, j, z, j + 1) -
                                          edge_flux_f64<C, O>(g, un, i, j, z, j)));
        }
        const dsf fz = edge_flux_ds<C, 2>(g, un, i, j, z, z + 1);
        acc = ds_add_d(acc, ds_add_d(fz, ds_neg(carry)));
        carry = fz;
      }
      v = ds_add_d(v, ds_neg(ds_mul(ca, acc)));
    }
    rhs[f] = f2d_exact(v.hi) + f2d_exact(v.lo);
  }
}

// FP32 work arrays of the predictor use a padded copy of the face layout:
// rows padded to a multiple of 4 values, so that every row starts on a
// 16-byte boundary and a thread can own four consecutive faces (one float4).
// Padding holds 0 and is never read as a neighbour.
struct FaceGeom32 {
  int n[3][3];
  int64_t off[3], sy[3], sz[3];
};

FaceGeom32 make_face_geom32(Dims d) {
  const FaceGeom g = make_face_geom(d);
  FaceGeom32 p;
  int64_t off = 0;
  for (int c = 0; c < 3; ++c) {
    for (int a = 0; a < 3; ++a) p.n[c][a] = g.n[c][a];
    p.sy[c] = (g.n[c][0] + 3) / 4 * 4;
    p.sz[c] = p.sy[c] * g.n[c][1];
    p.off[c] = off;
    off += p.sz[c] * g.n[c][2];
  }
  return p;
}

constexpr int HVY = 8;
constexpr unsigned kFullMask = 0xffffffffu;

// One FP32 Chebyshev step for A e = r on the padded layout, four faces per
// thread; x-neighbours by shuffles, z by the march, y through L1.
// mode 0: first step from e = 0: the normalised residual r^ = rs r is formed
// in double-single from r64 (FP64, split without FP64 arithmetic) or, when
// r64 is null, from the pair (r32, rlo) in place; r^ is kept in (r32, rlo)
// and e_new = alpha r^.hi.  mode 1: e_new = e + beta (e - e_old) +
// alpha (r - A e) with r = r32; mode 2: the same step, accumulated into the
// FP64 iterate, u += us * e_new, and stored in e_new (the next residual
// reads it).  The mode is a template parameter: each instance carries only
// its own registers (mode 2 loads the FP64 iterate with the plane's other
// inputs, so that its latency overlaps theirs).
template <int mode>
__global__ void __launch_bounds__(32 * HVY) k_helm_cheb_v4(
    FaceGeom g, FaceGeom32 p, int zchunks, const float* __restrict__ e,
    const float* __restrict__ eo, float* __restrict__ r32, float* __restrict__ rlo,
    const double* __restrict__ r64, float rs_hi, float rs_lo, float a, float nu_h2, float alpha,
    float beta, float* __restrict__ en, double* __restrict__ u, double us,
    const float* __restrict__ pe, double ps, int flags) {
  pdl_wait();
  pdl_trigger();
  // flags: 1 = e_old is zero (not read); 2 = the FP64 iterate is not read
  // (mode 2 writes u = us e_new + ps pe on every face, ps pe being a
  // correction not yet added (none when pe is null), 0 on the wall faces)
  const bool eo_zero = flags & 1, u_zero = flags & 2;
  const int c = blockIdx.z / zchunks;
  const int zc = blockIdx.z - c * zchunks;
  const int lane = threadIdx.x;
  const int x0 = 4 * (blockIdx.x * 32 + lane);
  const int j = blockIdx.y * HVY + threadIdx.y;
  const int n0 = sel3(c, p.n[0][0], p.n[1][0], p.n[2][0]);
  const int n1 = sel3(c, p.n[0][1], p.n[1][1], p.n[2][1]);
  const int n2 = sel3(c, p.n[0][2], p.n[1][2], p.n[2][2]);
  const int z0 = zc * ZH;
  if (z0 >= n2 || blockIdx.x * 128 >= n0 || blockIdx.y * HVY >= n1) return;   // block-uniform
  const int z1 = min(z0 + ZH, n2);
  const bool act = x0 < n0 && j < n1;
  const int64_t sy = sel3(c, p.sy[0], p.sy[1], p.sy[2]), sz = sel3(c, p.sz[0], p.sz[1], p.sz[2]);
  int64_t f = sel3(c, p.off[0], p.off[1], p.off[2]) + (int64_t)z0 * sz + (int64_t)j * sy + x0;
  const int64_t sy64 = sel3(c, g.sy[0], g.sy[1], g.sy[2]);
  const int64_t sz64 = sel3(c, g.sz[0], g.sz[1], g.sz[2]);
  int64_t f64 = sel3(c, g.off[0], g.off[1], g.off[2]) + (int64_t)z0 * sz64 + (int64_t)j * sy64 + x0;
  const float4 Z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  // per-element validity and x-wall status
  bool val[4], wallx[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    val[q] = act && (x0 + q < n0);
    wallx[q] = c == 0 && (x0 + q == 0 || x0 + q == n0 - 1);
  }
  const bool wally = c == 1 && (j == 0 || j == n1 - 1);
  if constexpr (mode == 0) {
    const dsf rs = {rs_hi, rs_lo};
    for (int z = z0; z < z1; ++z, f += sz, f64 += sz64) {
      const bool wallz = c == 2 && (z == 0 || z == n2 - 1);
      float h4[4] = {0.f, 0.f, 0.f, 0.f}, l4[4] = {0.f, 0.f, 0.f, 0.f};
      if (act && !r64) {
        const float4 a4 = *reinterpret_cast<const float4*>(r32 + f);
        const float4 b4 = *reinterpret_cast<const float4*>(rlo + f);
        h4[0] = a4.x; h4[1] = a4.y; h4[2] = a4.z; h4[3] = a4.w;
        l4[0] = b4.x; l4[1] = b4.y; l4[2] = b4.z; l4[3] = b4.w;
      }
      float rh[4], rl[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const bool live = val[q] && !wallx[q] && !wally && !wallz;
        dsf v = {0.f, 0.f};
        if (live) v = ds_mul(r64 ? split_exact(__ldg(r64 + f64 + q)) : dsf{h4[q], l4[q]}, rs);
        rh[q] = v.hi;
        rl[q] = v.lo;
      }
      if (act) {
        *reinterpret_cast<float4*>(r32 + f) = make_float4(rh[0], rh[1], rh[2], rh[3]);
        *reinterpret_cast<float4*>(rlo + f) = make_float4(rl[0], rl[1], rl[2], rl[3]);
        *reinterpret_cast<float4*>(en + f) =
            make_float4(alpha * rh[0], alpha * rh[1], alpha * rh[2], alpha * rh[3]);
      }
    }
    return;
  }
  // ghost counts along y and z (cell-centred axes only), x per element
  const int gy = (c != 1) ? ((j == 0) + (j == n1 - 1)) : 0;
  int gx[4];
#pragma unroll
  for (int q = 0; q < 4; ++q)
    gx[q] = (c != 0) ? ((x0 + q == 0) + (x0 + q == n0 - 1)) : 0;
  const bool has_ym = j > 0, has_yp = j < n1 - 1;
  float4 ep = (act && z0 > 0) ? *reinterpret_cast<const float4*>(e + f - sz) : Z4;
  float4 ec = act ? *reinterpret_cast<const float4*>(e + f) : Z4;
  for (int z = z0; z < z1; ++z, f += sz, f64 += sz64) {
    const float4 ez = (act && z + 1 < n2) ? *reinterpret_cast<const float4*>(e + f + sz) : Z4;
    const float4 ym = (act && has_ym) ? *reinterpret_cast<const float4*>(e + f - sy) : Z4;
    const float4 yp = (act && has_yp) ? *reinterpret_cast<const float4*>(e + f + sy) : Z4;
    const float4 rr = act ? *reinterpret_cast<const float4*>(r32 + f) : Z4;
    const float4 eold = (act && !eo_zero) ? *reinterpret_cast<const float4*>(eo + f) : Z4;
    float left = __shfl_up_sync(kFullMask, ec.w, 1);
    float right = __shfl_down_sync(kFullMask, ec.x, 1);
    if (lane == 0) left = (act && x0 > 0) ? e[f - 1] : 0.f;
    if (lane == 31) right = (act && x0 + 4 < n0) ? e[f + 4] : 0.f;
    const bool wallz = c == 2 && (z == 0 || z == n2 - 1);
    const int gz = (c != 2) ? ((z == 0) + (z == n2 - 1)) : 0;
    double uo[4] = {0.0, 0.0, 0.0, 0.0};
    float4 pv = Z4;
    if constexpr (mode == 2) {
      if (u_zero) {
        if (pe && act) pv = *reinterpret_cast<const float4*>(pe + f);
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (val[q] && !wallx[q] && !wally && !wallz) uo[q] = u[f64 + q];
      }
    }
    const float ev[4] = {ec.x, ec.y, ec.z, ec.w};
    const float evp[4] = {ep.x, ep.y, ep.z, ep.w};
    const float evn[4] = {ez.x, ez.y, ez.z, ez.w};
    const float vym[4] = {ym.x, ym.y, ym.z, ym.w};
    const float vyp[4] = {yp.x, yp.y, yp.z, yp.w};
    const float vr[4] = {rr.x, rr.y, rr.z, rr.w};
    const float vo[4] = {eold.x, eold.y, eold.z, eold.w};
    float out[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int x = x0 + q;
      float sx = 0.f;
      // x-neighbours exist inside the row; on a cell-centred x-axis the
      // missing ones are ghosts (counted in gx), on the face axis the wall
      // faces hold 0
      if (x > 0) sx += (q == 0) ? left : ev[q - 1];
      if (x < n0 - 1) sx += (q == 3) ? right : ev[q + 1];
      const float s = sx + (vym[q] + vyp[q]) + (evp[q] + evn[q]);
      const float diag = a + nu_h2 * (float)(6 + gx[q] + gy + gz);
      const float res = vr[q] - fmaf(diag, ev[q], -nu_h2 * s);
      const bool live = val[q] && !wallx[q] && !wally && !wallz;
      out[q] = live ? ev[q] + beta * (ev[q] - vo[q]) + alpha * res : 0.f;
    }
    if (act) *reinterpret_cast<float4*>(en + f) = make_float4(out[0], out[1], out[2], out[3]);
    if constexpr (mode == 2) {
      const float pq[4] = {pv.x, pv.y, pv.z, pv.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        // (the same products and roundings as adding ps pe first, then us e_new)
        if (u_zero && pe) uo[q] = ps * f2d_exact(pq[q]);
        if (val[q] && !wallx[q] && !wally && !wallz)
          u[f64 + q] = u_zero && !pe ? us * f2d_exact(out[q])
                                     : fma(us, f2d_exact(out[q]), uo[q]);   // widened without the FP64 pipe
        else if (u_zero && val[q])
          u[f64 + q] = 0.0;
      }
    }
    ep = ec;
    ec = ez;
  }
}

// Next normalised residual of the predictor's defect correction, in
// double-single arithmetic on the FP32 pipes: after a correction that solved
// A e = r^ (r^ = r / ||r|| held as the pair (rhi, rlo)) and added ||r|| e to
// the FP64 iterate, the new residual is ||r|| (r^ - A e).  This kernel forms
// q = r^ - A e exactly enough (A e of the FP32 e with error-free sums and
// products, the last two sums by Dekker's addition: a few units of 2^-46
// relative to r^) and writes it back to (rhi, rlo); the
// block's sum of q.hi^2 goes to part[block * stride] (every block writes
// one).  The FP64 pipe is not used.
__global__ void __launch_bounds__(32 * HVY) k_helm_resid_ds(
    FaceGeom32 p, int zchunks, const float* __restrict__ e, float* __restrict__ rhi,
    float* __restrict__ rlo, float a_hi, float a_lo, float nu_hi, float nu_lo,
    double* __restrict__ part, int stride) {
  const int c = blockIdx.z / zchunks;
  const int zc = blockIdx.z - c * zchunks;
  const int lane = threadIdx.x;
  const int x0 = 4 * (blockIdx.x * 32 + lane);
  const int j = blockIdx.y * HVY + threadIdx.y;
  const int n0 = sel3(c, p.n[0][0], p.n[1][0], p.n[2][0]);
  const int n1 = sel3(c, p.n[0][1], p.n[1][1], p.n[2][1]);
  const int n2 = sel3(c, p.n[0][2], p.n[1][2], p.n[2][2]);
  const int z0 = zc * ZH;
  const int64_t blk = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  if (z0 >= n2 || blockIdx.x * 128 >= n0 || blockIdx.y * HVY >= n1) {   // block-uniform
    if (threadIdx.x == 0 && threadIdx.y == 0) part[blk * stride] = 0.0;
    return;
  }
  const int z1 = min(z0 + ZH, n2);
  const bool act = x0 < n0 && j < n1;
  const int64_t sy = sel3(c, p.sy[0], p.sy[1], p.sy[2]), sz = sel3(c, p.sz[0], p.sz[1], p.sz[2]);
  int64_t f = sel3(c, p.off[0], p.off[1], p.off[2]) + (int64_t)z0 * sz + (int64_t)j * sy + x0;
  const float4 Z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  bool val[4], wallx[4];
  int gx[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    val[q] = act && (x0 + q < n0);
    wallx[q] = c == 0 && (x0 + q == 0 || x0 + q == n0 - 1);
    gx[q] = (c != 0) ? ((x0 + q == 0) + (x0 + q == n0 - 1)) : 0;
  }
  const bool wally = c == 1 && (j == 0 || j == n1 - 1);
  const int gy = (c != 1) ? ((j == 0) + (j == n1 - 1)) : 0;
  const bool has_ym = j > 0, has_yp = j < n1 - 1;
  const dsf A = {a_hi, a_lo}, NU = {nu_hi, nu_lo};
  const dsf D6 = ds_add(A, ds_mul_f(NU, 6.f));
  float acc = 0.f;
  float4 ep = (act && z0 > 0) ? *reinterpret_cast<const float4*>(e + f - sz) : Z4;
  float4 ec = act ? *reinterpret_cast<const float4*>(e + f) : Z4;
  for (int z = z0; z < z1; ++z, f += sz) {
    const float4 ez = (act && z + 1 < n2) ? *reinterpret_cast<const float4*>(e + f + sz) : Z4;
    const float4 ym = (act && has_ym) ? *reinterpret_cast<const float4*>(e + f - sy) : Z4;
    const float4 yp = (act && has_yp) ? *reinterpret_cast<const float4*>(e + f + sy) : Z4;
    const float4 rh = act ? *reinterpret_cast<const float4*>(rhi + f) : Z4;
    const float4 rl = act ? *reinterpret_cast<const float4*>(rlo + f) : Z4;
    float left = __shfl_up_sync(kFullMask, ec.w, 1);
    float right = __shfl_down_sync(kFullMask, ec.x, 1);
    if (lane == 0) left = (act && x0 > 0) ? e[f - 1] : 0.f;
    if (lane == 31) right = (act && x0 + 4 < n0) ? e[f + 4] : 0.f;
    const bool wallz = c == 2 && (z == 0 || z == n2 - 1);
    const int gz = (c != 2) ? ((z == 0) + (z == n2 - 1)) : 0;
    const float ev[4] = {ec.x, ec.y, ec.z, ec.w};
    const float evp[4] = {ep.x, ep.y, ep.z, ep.w};
    const float evn[4] = {ez.x, ez.y, ez.z, ez.w};
    const float vym[4] = {ym.x, ym.y, ym.z, ym.w};
    const float vyp[4] = {yp.x, yp.y, yp.z, yp.w};
    const float vrh[4] = {rh.x, rh.y, rh.z, rh.w};
    const float vrl[4] = {rl.x, rl.y, rl.z, rl.w};
    float oh[4], ol[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int x = x0 + q;
      const float xl = (x > 0) ? ((q == 0) ? left : ev[q - 1]) : 0.f;
      const float xr = (x < n0 - 1) ? ((q == 3) ? right : ev[q + 1]) : 0.f;
      dsf s = two_sum(xl, xr);
      s = ds_add_f(s, vym[q]);
      s = ds_add_f(s, vyp[q]);
      s = ds_add_f(s, evp[q]);
      s = ds_add_f(s, evn[q]);
      const int gh = gx[q] + gy + gz;
      const dsf diag = gh == 0 ? D6 : ds_add(A, ds_mul_f(NU, (float)(6 + gh)));
      const dsf Ae = ds_add_d(ds_mul_f(diag, ev[q]), ds_neg(ds_mul(NU, s)));
      dsf qv = ds_add_d(dsf{vrh[q], vrl[q]}, ds_neg(Ae));
      const bool live = val[q] && !wallx[q] && !wally && !wallz;
      if (!live) qv = dsf{0.f, 0.f};
      oh[q] = qv.hi;
      ol[q] = qv.lo;
      acc = fmaf(qv.hi, qv.hi, acc);
    }
    if (act) {
      *reinterpret_cast<float4*>(rhi + f) = make_float4(oh[0], oh[1], oh[2], oh[3]);
      *reinterpret_cast<float4*>(rlo + f) = make_float4(ol[0], ol[1], ol[2], ol[3]);
    }
    ep = ec;
    ec = ez;
  }
  // block reduction (FP64, fixed order)
  double v = (double)acc;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFullMask, v, o);
  __shared__ double sh[HVY];
  if (lane == 0) sh[threadIdx.y] = v;
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    double t = 0.0;
    for (int w = 0; w < HVY; ++w) t += sh[w];
    part[blk * stride] = t;
  }
}

}  // namespace

int march_zc(Dims d);

template <typename T>
void launch_laplacian(Dims d, const T* v, T* out, double inv_h2, cudaStream_t s) {
  count_launch();
  if constexpr (std::is_same<T, double>::value) {
    const int zc = march_zc(d);
    const FxLimits L = fx_limits(inv_h2);
    k_laplacian_fx<<<dim3(div_up(d.nx, BX), div_up(d.ny, BY), div_up(d.nz, zc)), dim3(BX, BY), 0,
                     s>>>(d, v, nullptr, out, L.bits, L.e_min, L.e_max, zc);
  } else {
    k_laplacian<T><<<cell_grid(d), dim3(BX, BY), 0, s>>>(d, v, out, (T)inv_h2);
  }
}
void launch_laplacian_sub(Dims d, const double* v, const double* b, double* out, double inv_h2,
                          cudaStream_t s) {
  count_launch();
  const int zc = march_zc(d);
  const FxLimits L = fx_limits(inv_h2);
  k_laplacian_fx<<<dim3(div_up(d.nx, BX), div_up(d.ny, BY), div_up(d.nz, zc)), dim3(BX, BY), 0,
                   s>>>(d, v, b, out, L.bits, L.e_min, L.e_max, zc);
}

template void launch_laplacian<float>(Dims, const float*, float*, double, cudaStream_t);
template void launch_laplacian<double>(Dims, const double*, double*, double, cudaStream_t);

dim3 grad_grid(Dims d, int zc) {
  return dim3(div_up(d.nx + 1, BX), div_up(d.ny + 1, BY), div_up(d.nz + 1, zc));
}

void launch_gradient(Dims d, const double* p, double* u, double inv_h, cudaStream_t s) {
  count_launch();
  const int zc = march_zc(d);
  k_grad_axpy<<<grad_grid(d, zc), dim3(BX, BY), 0, s>>>(d, make_face_geom(d), nullptr, p, inv_h,
                                                         u, zc);
}

void launch_grad_axpy(Dims d, const double* u_in, const double* p, double alpha, double* u_out,
                      cudaStream_t s) {
  count_launch();
  const int zc = march_zc(d);
  k_grad_axpy<<<grad_grid(d, zc), dim3(BX, BY), 0, s>>>(d, make_face_geom(d), u_in, p, alpha,
                                                         u_out, zc);
}

// planes per thread of the one-cell z-march kernels: about eight blocks per
// SM over the grid, at most 4
int march_zc(Dims d) {
  const int64_t bxy = (int64_t)div_up(d.nx, BX) * div_up(d.ny, BY);
  return (int)std::min<int64_t>(4, std::max<int64_t>(1, d.nz * bxy / (152 * 8)));
}

void launch_gradt_axpby(Dims d, const double* u, double alpha, const double* c, double beta,
                        double* out, cudaStream_t s) {
  count_launch();
  const int zc = march_zc(d);
  k_gradt_fx<false><<<dim3(div_up(d.nx, BX), div_up(d.ny, BY), div_up(d.nz, zc)), dim3(BX, BY),
                      0, s>>>(d, make_face_geom(d), u, fx_limits(alpha), c, beta, out, nullptr, zc);
}

int64_t gradt_norm2_blocks(Dims d) {
  const int zc = march_zc(d);
  return (int64_t)div_up(d.nx, BX) * div_up(d.ny, BY) * div_up(d.nz, zc);
}

int64_t launch_gradt_norm2(Dims d, const double* u, double alpha, double* part, cudaStream_t s) {
  count_launch();
  const int zc = march_zc(d);
  k_gradt_fx<true><<<dim3(div_up(d.nx, BX), div_up(d.ny, BY), div_up(d.nz, zc)), dim3(BX, BY), 0,
                     s>>>(d, make_face_geom(d), u, fx_limits(alpha), nullptr, 0.0, nullptr, part,
                          zc);
  return gradt_norm2_blocks(d);
}

void launch_gradient_t(Dims d, const double* u, double* out, double inv_h, cudaStream_t s) {
  launch_gradt_axpby(d, u, inv_h, nullptr, 0.0, out, s);
}

int helm_zchunks(Dims d) { return div_up(d.nz + 1, ZH); }

int64_t helm_fp32_size(Dims d) {
  const FaceGeom32 p = make_face_geom32(d);
  return p.off[2] + p.sz[2] * p.n[2][2];
}

// x-blocks cover the nx first points of every row (a multiple of 4 when
// rounded up); for u_x the remaining point x = nx is a wall face, never
// written and kept 0 since the arrays were cleared at creation
dim3 helm_v4_grid(Dims d) {
  return dim3(div_up(div_up(d.nx, 4), 32), div_up(d.ny + 1, HVY), 3 * helm_zchunks(d));
}

void launch_helm_cheb(Dims d, const float* e, const float* eo, float* r32, float* rlo,
                      const double* r64, double rs, float a, float nu_h2, float alpha, float beta,
                      float* en, double* u, double us, int mode, cudaStream_t s, int flags,
                      const float* pe, double ps) {
  const FaceGeom32 p = make_face_geom32(d);
  const float rs_hi = (float)rs, rs_lo = (float)(rs - (double)rs_hi);
  count_launch();
  const FaceGeom g = make_face_geom(d);
  const int zch = helm_zchunks(d);
  if (mode == 0)
    launch_pdl(k_helm_cheb_v4<0>, helm_v4_grid(d), dim3(32, HVY), 0, s, g, p, zch, e, eo, r32,
               rlo, r64, rs_hi, rs_lo, a, nu_h2, alpha, beta, en, u, us, pe, ps, flags);
  else if (mode == 1)
    launch_pdl(k_helm_cheb_v4<1>, helm_v4_grid(d), dim3(32, HVY), 0, s, g, p, zch, e, eo, r32,
               rlo, r64, rs_hi, rs_lo, a, nu_h2, alpha, beta, en, u, us, pe, ps, flags);
  else
    launch_pdl(k_helm_cheb_v4<2>, helm_v4_grid(d), dim3(32, HVY), 0, s, g, p, zch, e, eo, r32,
               rlo, r64, rs_hi, rs_lo, a, nu_h2, alpha, beta, en, u, us, pe, ps, flags);
}

// u = ps pe on the interior faces, 0 on the wall faces (a predictor
// correction kept in FP32 written to the FP64 iterate when no later
// correction's last step does it)
__global__ void __launch_bounds__(32 * HVY) k_helm_flush(FaceGeom g, FaceGeom32 p, int zchunks,
                                                         const float* __restrict__ pe, double ps,
                                                         double* __restrict__ u) {
  const int c = blockIdx.z / zchunks;
  const int zc = blockIdx.z - c * zchunks;
  const int x0 = 4 * (blockIdx.x * 32 + threadIdx.x);
  const int j = blockIdx.y * HVY + threadIdx.y;
  const int n0 = sel3(c, p.n[0][0], p.n[1][0], p.n[2][0]);
  const int n1 = sel3(c, p.n[0][1], p.n[1][1], p.n[2][1]);
  const int n2 = sel3(c, p.n[0][2], p.n[1][2], p.n[2][2]);
  const int z0 = zc * ZH;
  if (z0 >= n2 || x0 >= n0 || j >= n1) return;
  const int z1 = min(z0 + ZH, n2);
  const int64_t sy = sel3(c, p.sy[0], p.sy[1], p.sy[2]), sz = sel3(c, p.sz[0], p.sz[1], p.sz[2]);
  const int64_t sy64 = sel3(c, g.sy[0], g.sy[1], g.sy[2]);
  const int64_t sz64 = sel3(c, g.sz[0], g.sz[1], g.sz[2]);
  int64_t f = sel3(c, p.off[0], p.off[1], p.off[2]) + (int64_t)z0 * sz + (int64_t)j * sy + x0;
  int64_t f64 = sel3(c, g.off[0], g.off[1], g.off[2]) + (int64_t)z0 * sz64 + (int64_t)j * sy64 + x0;
  const bool wally = c == 1 && (j == 0 || j == n1 - 1);
  for (int z = z0; z < z1; ++z, f += sz, f64 += sz64) {
    const bool wallz = c == 2 && (z == 0 || z == n2 - 1);
    const float4 v = *reinterpret_cast<const float4*>(pe + f);
    const float vq[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (x0 + q >= n0) break;
      const bool wallx = c == 0 && (x0 + q == 0 || x0 + q == n0 - 1);
      u[f64 + q] = (wallx || wally || wallz) ? 0.0 : ps * f2d_exact(vq[q]);
    }
  }
}

void launch_helm_flush(Dims d, const float* pe, double ps, double* u, cudaStream_t s) {
  count_launch();
  k_helm_flush<<<helm_v4_grid(d), dim3(32, HVY), 0, s>>>(make_face_geom(d), make_face_geom32(d),
                                                          helm_zchunks(d), pe, ps, u);
}

int64_t launch_helm_resid_ds(Dims d, const float* e, float* rhi, float* rlo, double a,
                             double nu_h2, double* part, int stride, cudaStream_t s) {
  const dim3 gr = helm_v4_grid(d);
  const float a_hi = (float)a, a_lo = (float)(a - (double)a_hi);
  const float n_hi = (float)nu_h2, n_lo = (float)(nu_h2 - (double)n_hi);
  count_launch();
  k_helm_resid_ds<<<gr, dim3(32, HVY), 0, s>>>(make_face_geom32(d), helm_zchunks(d), e, rhi, rlo,
                                               a_hi, a_lo, n_hi, n_lo, part, stride);
  return (int64_t)gr.x * gr.y * gr.z;
}

// dsf of an FP64 constant (host)
dsf host_ds(double x) {
  const float hi = (float)x;
  return dsf{hi, (float)(x - (double)hi)};
}

void launch_predictor_rhs_adv(Dims d, const double* u_n, const double* u_nm1, const double* p_n,
                              const double* f_body, int with_adv, double inv_2dt, double inv_h,
                              double* rhs, cudaStream_t s) {
  const FaceGeom g = make_face_geom(d);
  const dsf c4 = host_ds(4.0 * inv_2dt), c1 = host_ds(inv_2dt), cph = host_ds(inv_h),
            ca = host_ds(0.25 * inv_h);
  const dim3 b(BX, BY);
  count_launch();
  k_predictor_rhs_ds<0><<<dim3(div_up(d.nx + 1, BX), div_up(d.ny, BY), div_up(d.nz, ZH)), b, 0,
                          s>>>(d, g, u_n, u_nm1, p_n, f_body, with_adv, c4, c1, cph, ca, rhs);
  count_launch();
  k_predictor_rhs_ds<1><<<dim3(div_up(d.nx, BX), div_up(d.ny + 1, BY), div_up(d.nz, ZH)), b, 0,
                          s>>>(d, g, u_n, u_nm1, p_n, f_body, with_adv, c4, c1, cph, ca, rhs);
  count_launch();
  k_predictor_rhs_ds<2><<<dim3(div_up(d.nx, BX), div_up(d.ny, BY), div_up(d.nz + 1, ZH)), b, 0,
                          s>>>(d, g, u_n, u_nm1, p_n, f_body, with_adv, c4, c1, cph, ca, rhs);
}

}  // namespace ibm
