// Staggered MAC-grid stencils (Sec. 3.1): the Neumann Laplacian L = G^T G of
// Eq. (Saddle), the gradient G and its transpose G^T = -div, and the pieces of
// the BDF2 momentum predictor of Eq. (ustar) (Helmholtz operator, explicit
// convective term, right-hand side).
//
// Thread layout: one thread per grid point, blocks of 32 x 8 in (x, y) and one
// z-plane per blockIdx.z, so that a warp reads 32 consecutive x values of each
// neighbour row (coalesced; the y/z neighbours hit L1/L2).
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

__device__ __forceinline__ int64_t fidx(const FaceGeom& g, int c, int i, int j, int k) {
  return g.off[c] + k * g.sz[c] + j * g.sy[c] + i;
}

// Value of component c at integer point (p[0], p[1], p[2]) of its own grid;
// wall-normal boundary faces (index 0 or n along c) read as 0.
__device__ __forceinline__ double face_val(const FaceGeom& g, const double* __restrict__ u,
                                           int c, int i, int j, int k) {
  int p[3] = {i, j, k};
  if (p[c] <= 0 || p[c] >= g.n[c][c] - 1) return 0.0;
  return __ldg(u + fidx(g, c, i, j, k));
}

dim3 cell_grid(Dims d) { return dim3(div_up(d.nx, BX), div_up(d.ny, BY), d.nz); }
dim3 face_grid(Dims d) { return dim3(div_up(d.nx + 1, BX), div_up(d.ny + 1, BY), d.nz + 1); }

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

// u = u_in + alpha * G p on interior faces, 0 on wall faces (u_in may be null).
__global__ void __launch_bounds__(BX * BY) k_grad_axpy(Dims d, FaceGeom g,
                                                       const double* __restrict__ u_in,
                                                       const double* __restrict__ p,
                                                       double alpha, double* __restrict__ u) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  const int64_t sy = d.nx, sz = (int64_t)d.nx * d.ny;
  const int p3[3] = {i, j, k};
  const int64_t cs[3] = {1, sy, sz};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (i >= g.n[c][0] || j >= g.n[c][1] || k >= g.n[c][2]) continue;
    const int64_t f = fidx(g, c, i, j, k);
    double val = 0.0;
    if (p3[c] > 0 && p3[c] < g.n[c][c] - 1) {
      const int64_t cp = k * sz + j * sy + i;   // cell on the + side
      const double gp = __ldg(p + cp) - __ldg(p + cp - cs[c]);
      val = u_in ? fma(alpha, gp, __ldg(u_in + f)) : alpha * gp;
    }
    u[f] = val;
  }
}

// out = alpha * G^T u + beta * cin: (G^T u)_c = sum_d (u_{c-1/2} - u_{c+1/2}),
// interior faces only (alpha carries the 1/h).
__global__ void __launch_bounds__(BX * BY) k_gradt_axpby(Dims d, FaceGeom g,
                                                         const double* __restrict__ u,
                                                         double alpha,
                                                         const double* __restrict__ cin,
                                                         double beta, double* __restrict__ out) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= d.nx || j >= d.ny) return;
  const double s = (face_val(g, u, 0, i, j, k) - face_val(g, u, 0, i + 1, j, k)) +
                   (face_val(g, u, 1, i, j, k) - face_val(g, u, 1, i, j + 1, k)) +
                   (face_val(g, u, 2, i, j, k) - face_val(g, u, 2, i, j, k + 1));
  const int64_t c = ((int64_t)k * d.ny + j) * d.nx + i;
  out[c] = cin ? fma(alpha, s, beta * __ldg(cin + c)) : alpha * s;
}

// Predictor Helmholtz operator on the d-faces, A = a I - nu Lap_h with the
// no-slip ghosts: A e = diag e_c - (nu / h^2) * (sum of neighbours), where the
// face-normal axis reads the wall faces (which hold 0) and each cell-centred
// axis adds nu / h^2 to diag for every missing neighbour (ghost = -e_c).
// Kernels below march along z over ZH planes; blockIdx.z = comp * zchunks +
// chunk, so one launch covers the three face grids.
constexpr int ZH = 16;

struct FaceThread {
  int c, i, j, z0, z1, n0, n1, n2;
  int64_t sy, sz, f0;
  bool wall;       // the whole column is a wall-normal face (c = 0 or 1)
  bool xm, xp, ym, yp;
  int ghosts_xy;
};

__device__ __forceinline__ bool face_thread(const FaceGeom& g, int zchunks, FaceThread& t) {
  t.c = blockIdx.z / zchunks;
  const int zc = blockIdx.z - t.c * zchunks;
  t.i = blockIdx.x * BX + threadIdx.x;
  t.j = blockIdx.y * BY + threadIdx.y;
  t.n0 = g.n[t.c][0];
  t.n1 = g.n[t.c][1];
  t.n2 = g.n[t.c][2];
  t.z0 = zc * ZH;
  if (t.i >= t.n0 || t.j >= t.n1 || t.z0 >= t.n2) return false;
  t.z1 = min(t.z0 + ZH, t.n2);
  t.sy = g.sy[t.c];
  t.sz = g.sz[t.c];
  t.f0 = g.off[t.c] + (int64_t)t.z0 * t.sz + (int64_t)t.j * t.sy + t.i;
  t.wall = (t.c == 0 && (t.i == 0 || t.i == t.n0 - 1)) || (t.c == 1 && (t.j == 0 || t.j == t.n1 - 1));
  t.xm = t.i > 0;
  t.xp = t.i < t.n0 - 1;
  t.ym = t.j > 0;
  t.yp = t.j < t.n1 - 1;
  t.ghosts_xy = 0;
  if (t.c != 0) t.ghosts_xy += (!t.xm) + (!t.xp);
  if (t.c != 1) t.ghosts_xy += (!t.ym) + (!t.yp);
  return true;
}

template <typename T>
__device__ __forceinline__ T face_inplane(const T* __restrict__ e, int64_t f, const FaceThread& t) {
  T s = 0;
  if (t.xm) s += __ldg(e + f - 1);
  if (t.xp) s += __ldg(e + f + 1);
  if (t.ym) s += __ldg(e + f - t.sy);
  if (t.yp) s += __ldg(e + f + t.sy);
  return s;
}

// Right-hand side of the predictor, Eq. (ustar), with the convective term
// fused in: rhs = (4 u^n - u^{n-1}) / (2 dt) - G p^n + f - A(u^n) on interior
// faces (0 on wall faces).  A is the central divergence form of k_advection
// with the 1/2 averages folded into one factor 1/4:
//   4 A = [ (u_+ + u_0)^2 - (u_0 + u_-)^2 ] along the component's own axis
//       + sum over the two other axes of (flux at the upper edge - lower edge),
//   flux = (u_e averaged pair sum) * (u_c averaged pair sum), 0 on walls.
// The march runs along z; the flux through the lower z-edge (or, for u_z, the
// lower cell-centred square) is the previous face's upper one and is reused.
__global__ void __launch_bounds__(BX * BY) k_predictor_rhs_adv(
    Dims d, FaceGeom g, int zchunks, const double* __restrict__ un,
    const double* __restrict__ unm1, const double* __restrict__ pn,
    const double* __restrict__ fb, int with_adv, double inv_2dt, double inv_h,
    double* __restrict__ rhs) {
  FaceThread t;
  if (!face_thread(g, zchunks, t)) return;
  const int c = t.c;
  int64_t f = t.f0;
  const int64_t csy = d.nx, csz = (int64_t)d.nx * d.ny;
  const int64_t cstride[3] = {1, csy, csz};
  // U(comp, x, y, z): face value, 0 on wall faces and outside the grid
  auto U = [&](int comp, int x, int y, int z) -> double {
    const int q[3] = {x, y, z};
    if (x < 0 || y < 0 || z < 0 || x >= g.n[comp][0] || y >= g.n[comp][1] || z >= g.n[comp][2])
      return 0.0;
    if (q[comp] == 0 || q[comp] == g.n[comp][comp] - 1) return 0.0;
    return __ldg(un + fidx(g, comp, x, y, z));
  };
  // flux on the edge between the c-face at p (p[c] = c-face index) and the
  // e-face index qe along e (other coordinate from p): 4 * (avg u_e)(avg u_c)
  auto eflux = [&](int e, int px, int py, int pz, int qe) -> double {
    const int ne = g.n[e][e] - 1;   // cells along e
    if (qe <= 0 || qe >= ne) return 0.0;
    int a[3] = {px, py, pz};
    a[e] = qe;
    int b0[3] = {a[0], a[1], a[2]}, b1[3] = {a[0], a[1], a[2]};
    b0[c] -= 1;   // u_e at the two cells adjacent along c
    const double ue = U(e, b0[0], b0[1], b0[2]) + U(e, b1[0], b1[1], b1[2]);
    int c0[3] = {a[0], a[1], a[2]}, c1[3] = {a[0], a[1], a[2]};
    c0[e] = qe - 1;
    const double uc = U(c, c0[0], c0[1], c0[2]) + U(c, c1[0], c1[1], c1[2]);
    return ue * uc;
  };
  const int i = t.i, j = t.j;
  double carry = 0.0;   // lower z-flux (c = 0, 1) or lower square (c = 2)
  if (with_adv && !t.wall) {
    if (c == 2) {
      const double s0 = U(2, i, j, t.z0 - 1) + U(2, i, j, t.z0);
      carry = s0 * s0;
    } else {
      carry = eflux(2, i, j, t.z0, t.z0);
    }
  }
  for (int z = t.z0; z < t.z1; ++z, f += t.sz) {
    const bool wall = t.wall || (c == 2 && (z == 0 || z == t.n2 - 1));
    if (wall) {
      rhs[f] = 0.0;
      if (with_adv) {
        if (c == 2) {
          const double s1 = U(2, i, j, z) + U(2, i, j, z + 1);
          carry = s1 * s1;
        } else {
          carry = eflux(2, i, j, z, z + 1);
        }
      }
      continue;
    }
    const int64_t cp = (int64_t)z * csz + (int64_t)j * csy + i;   // cell on the + side
    // (4 u^n - u^{n-1}) / (2 dt) - (p_+ - p_-) / h (+ f): two FMAs, one
    // multiply and one subtraction
    double v = fma(__ldg(un + f), 4.0 * inv_2dt, -inv_2dt * __ldg(unm1 + f));
    v = fma(-inv_h, __ldg(pn + cp) - __ldg(pn + cp - cstride[c]), v);
    if (fb) v += __ldg(fb + f);
    if (with_adv) {
      double acc;
      if (c == 2) {
        const double s1 = U(2, i, j, z) + U(2, i, j, z + 1);
        const double up2 = s1 * s1;
        acc = up2 - carry;
        carry = up2;
        acc += eflux(0, i, j, z, i + 1) - eflux(0, i, j, z, i);
        acc += eflux(1, i, j, z, j + 1) - eflux(1, i, j, z, j);
      } else {
        // own axis (x for u_x, y for u_y)
        int pp[3] = {i, j, z}, pm[3] = {i, j, z};
        pp[c] += 1;
        pm[c] -= 1;
        const double u0 = __ldg(un + f);
        const double up = U(c, pp[0], pp[1], pp[2]), um = U(c, pm[0], pm[1], pm[2]);
        acc = (up - um) * (up + 2.0 * u0 + um);
        const int o = 1 - c;   // the other in-plane axis
        const int po = o == 0 ? i : j;
        acc += eflux(o, i, j, z, po + 1) - eflux(o, i, j, z, po);
        const double fz = eflux(2, i, j, z, z + 1);
        acc += fz - carry;
        carry = fz;
      }
      v = fma(-0.25 * inv_h, acc, v);
    }
    rhs[f] = v;
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
// reads it).
__global__ void __launch_bounds__(32 * HVY) k_helm_cheb_v4(
    FaceGeom g, FaceGeom32 p, int zchunks, const float* __restrict__ e,
    const float* __restrict__ eo, float* __restrict__ r32, float* __restrict__ rlo,
    const double* __restrict__ r64, float rs_hi, float rs_lo, float a, float nu_h2, float alpha,
    float beta, float* __restrict__ en, double* __restrict__ u, double us, int mode) {
  const int c = blockIdx.z / zchunks;
  const int zc = blockIdx.z - c * zchunks;
  const int lane = threadIdx.x;
  const int x0 = 4 * (blockIdx.x * 32 + lane);
  const int j = blockIdx.y * HVY + threadIdx.y;
  const int n0 = p.n[c][0], n1 = p.n[c][1], n2 = p.n[c][2];
  const int z0 = zc * ZH;
  if (z0 >= n2 || blockIdx.x * 128 >= n0 || blockIdx.y * HVY >= n1) return;   // block-uniform
  const int z1 = min(z0 + ZH, n2);
  const bool act = x0 < n0 && j < n1;
  const int64_t sy = p.sy[c], sz = p.sz[c];
  int64_t f = p.off[c] + (int64_t)z0 * sz + (int64_t)j * sy + x0;
  const int64_t sy64 = g.sy[c], sz64 = g.sz[c];
  int64_t f64 = g.off[c] + (int64_t)z0 * sz64 + (int64_t)j * sy64 + x0;
  const float4 Z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  // per-element validity and x-wall status
  bool val[4], wallx[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    val[q] = act && (x0 + q < n0);
    wallx[q] = c == 0 && (x0 + q == 0 || x0 + q == n0 - 1);
  }
  const bool wally = c == 1 && (j == 0 || j == n1 - 1);
  if (mode == 0) {
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
    const float4 eold = act ? *reinterpret_cast<const float4*>(eo + f) : Z4;
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
    if (mode == 2) {
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (val[q] && !wallx[q] && !wally && !wallz) u[f64 + q] = fma(us, (double)out[q], u[f64 + q]);
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
// products, about 2^-46 relative to r^) and writes it back to (rhi, rlo); the
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
  const int n0 = p.n[c][0], n1 = p.n[c][1], n2 = p.n[c][2];
  const int z0 = zc * ZH;
  const int64_t blk = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  if (z0 >= n2 || blockIdx.x * 128 >= n0 || blockIdx.y * HVY >= n1) {   // block-uniform
    if (threadIdx.x == 0 && threadIdx.y == 0) part[blk * stride] = 0.0;
    return;
  }
  const int z1 = min(z0 + ZH, n2);
  const bool act = x0 < n0 && j < n1;
  const int64_t sy = p.sy[c], sz = p.sz[c];
  int64_t f = p.off[c] + (int64_t)z0 * sz + (int64_t)j * sy + x0;
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
      const dsf Ae = ds_add(ds_mul_f(diag, ev[q]), ds_neg(ds_mul(NU, s)));
      dsf qv = ds_add(dsf{vrh[q], vrl[q]}, ds_neg(Ae));
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

// Explicit convective term of Eq. (ustar): central finite-volume divergence
// form div(u u_c) on the MAC grid.  Along e == c the flux lives at cell
// centres (square of u_c averaged along c); along e != c on the edge shared by
// the c-face and the e-face: (u_e averaged along c) * (u_c averaged along e),
// zero on walls (wall-normal velocity 0).
__device__ __forceinline__ double edge_flux(const FaceGeom& g, const double* __restrict__ u,
                                            int c, int e, int pc[3]) {
  // pc: point with pc[c] = c-face index, pc[e] = e-face index (0..n_e).
  const int ne = g.n[e][e] - 1;   // cells along e
  if (pc[e] <= 0 || pc[e] >= ne) return 0.0;
  int q[3] = {pc[0], pc[1], pc[2]};
  // u_e at e-face pc[e], averaged over the two cells adjacent along c
  q[c] = pc[c] - 1;
  const double ue0 = face_val(g, u, e, q[0], q[1], q[2]);
  q[c] = pc[c];
  const double ue1 = face_val(g, u, e, q[0], q[1], q[2]);
  // u_c at c-face pc[c], averaged over the two cells adjacent along e
  int r[3] = {pc[0], pc[1], pc[2]};
  r[e] = pc[e] - 1;
  const double uc0 = face_val(g, u, c, r[0], r[1], r[2]);
  r[e] = pc[e];
  const double uc1 = face_val(g, u, c, r[0], r[1], r[2]);
  return 0.25 * (ue0 + ue1) * (uc0 + uc1);
}

__global__ void __launch_bounds__(BX * BY) k_advection(Dims d, FaceGeom g,
                                                       const double* __restrict__ u,
                                                       double inv_h, double* __restrict__ out) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
#pragma unroll 1
  for (int c = 0; c < 3; ++c) {
    if (i >= g.n[c][0] || j >= g.n[c][1] || k >= g.n[c][2]) continue;
    const int64_t f = fidx(g, c, i, j, k);
    int p[3] = {i, j, k};
    if (p[c] == 0 || p[c] == g.n[c][c] - 1) { out[f] = 0.0; continue; }
    double acc = 0.0;
    for (int e = 0; e < 3; ++e) {
      if (e == c) {
        int q[3] = {i, j, k};
        const double um = face_val(g, u, c, q[0], q[1], q[2]);
        q[c] = p[c] + 1;
        const double up = face_val(g, u, c, q[0], q[1], q[2]);
        q[c] = p[c] - 1;
        const double umm = face_val(g, u, c, q[0], q[1], q[2]);
        const double cp = 0.5 * (um + up), cm = 0.5 * (umm + um);
        acc += cp * cp - cm * cm;
      } else {
        int q[3] = {i, j, k};
        q[e] = p[e] + 1;
        const double fp = edge_flux(g, u, c, e, q);
        q[e] = p[e];
        const double fm = edge_flux(g, u, c, e, q);
        acc += fp - fm;
      }
    }
    out[f] = acc * inv_h;
  }
}

// rhs = (4 u^n - u^{n-1}) / (2 dt) - G p^n + f - adv on interior faces.
__global__ void __launch_bounds__(BX * BY) k_predictor_rhs(
    Dims d, FaceGeom g, const double* __restrict__ un, const double* __restrict__ unm1,
    const double* __restrict__ pn, const double* __restrict__ fb,
    const double* __restrict__ adv, double inv_2dt, double inv_h, double* __restrict__ rhs) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  const int64_t sy = d.nx, sz = (int64_t)d.nx * d.ny;
  const int p3[3] = {i, j, k};
  const int64_t cs[3] = {1, sy, sz};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (i >= g.n[c][0] || j >= g.n[c][1] || k >= g.n[c][2]) continue;
    const int64_t f = fidx(g, c, i, j, k);
    if (p3[c] == 0 || p3[c] == g.n[c][c] - 1) { rhs[f] = 0.0; continue; }
    const int64_t cp = k * sz + j * sy + i;
    double v = (4.0 * __ldg(un + f) - __ldg(unm1 + f)) * inv_2dt;
    v -= (__ldg(pn + cp) - __ldg(pn + cp - cs[c])) * inv_h;
    if (fb) v += __ldg(fb + f);
    if (adv) v -= __ldg(adv + f);
    rhs[f] = v;
  }
}

}  // namespace

template <typename T>
void launch_laplacian(Dims d, const T* v, T* out, double inv_h2, cudaStream_t s) {
  count_launch();
  k_laplacian<T><<<cell_grid(d), dim3(BX, BY), 0, s>>>(d, v, out, (T)inv_h2);
}
template void launch_laplacian<float>(Dims, const float*, float*, double, cudaStream_t);
template void launch_laplacian<double>(Dims, const double*, double*, double, cudaStream_t);

void launch_gradient(Dims d, const double* p, double* u, double inv_h, cudaStream_t s) {
  count_launch();
  k_grad_axpy<<<face_grid(d), dim3(BX, BY), 0, s>>>(d, make_face_geom(d), nullptr, p, inv_h, u);
}

void launch_grad_axpy(Dims d, const double* u_in, const double* p, double alpha, double* u_out,
                      cudaStream_t s) {
  count_launch();
  k_grad_axpy<<<face_grid(d), dim3(BX, BY), 0, s>>>(d, make_face_geom(d), u_in, p, alpha, u_out);
}

void launch_gradient_t(Dims d, const double* u, double* out, double inv_h, cudaStream_t s) {
  count_launch();
  k_gradt_axpby<<<cell_grid(d), dim3(BX, BY), 0, s>>>(d, make_face_geom(d), u, inv_h, nullptr,
                                                       0.0, out);
}

void launch_gradt_axpby(Dims d, const double* u, double alpha, const double* c, double beta,
                        double* out, cudaStream_t s) {
  count_launch();
  k_gradt_axpby<<<cell_grid(d), dim3(BX, BY), 0, s>>>(d, make_face_geom(d), u, alpha, c, beta,
                                                       out);
}

int helm_zchunks(Dims d) { return div_up(d.nz + 1, ZH); }

dim3 helm_grid(Dims d) {
  return dim3(div_up(d.nx + 1, BX), div_up(d.ny + 1, BY), 3 * helm_zchunks(d));
}

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
                      float* en, double* u, double us, int mode, cudaStream_t s) {
  const FaceGeom32 p = make_face_geom32(d);
  const float rs_hi = (float)rs, rs_lo = (float)(rs - (double)rs_hi);
  count_launch();
  k_helm_cheb_v4<<<helm_v4_grid(d), dim3(32, HVY), 0, s>>>(
      make_face_geom(d), p, helm_zchunks(d), e, eo, r32, rlo, r64, rs_hi, rs_lo, a, nu_h2, alpha,
      beta, en, u, us, mode);
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

void launch_advection(Dims d, const double* u, double inv_h, double* out, cudaStream_t s) {
  count_launch();
  k_advection<<<face_grid(d), dim3(BX, BY), 0, s>>>(d, make_face_geom(d), u, inv_h, out);
}

void launch_predictor_rhs_adv(Dims d, const double* u_n, const double* u_nm1, const double* p_n,
                              const double* f_body, int with_adv, double inv_2dt, double inv_h,
                              double* rhs, cudaStream_t s) {
  count_launch();
  k_predictor_rhs_adv<<<helm_grid(d), dim3(BX, BY), 0, s>>>(d, make_face_geom(d), helm_zchunks(d),
                                                             u_n, u_nm1, p_n, f_body, with_adv,
                                                             inv_2dt, inv_h, rhs);
}

void launch_predictor_rhs(Dims d, const double* u_n, const double* u_nm1, const double* p_n,
                          const double* f_body, const double* adv, double inv_2dt, double inv_h,
                          double* rhs, cudaStream_t s) {
  count_launch();
  k_predictor_rhs<<<face_grid(d), dim3(BX, BY), 0, s>>>(d, make_face_geom(d), u_n, u_nm1, p_n,
                                                         f_body, adv, inv_2dt, inv_h, rhs);
}

}  // namespace ibm
