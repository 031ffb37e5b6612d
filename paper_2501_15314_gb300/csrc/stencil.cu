// Staggered MAC-grid stencils (Sec. 3.1): the Neumann Laplacian L = G^T G of
// Eq. (Saddle), the gradient G and its transpose G^T = -div, and the pieces of
// the BDF2 momentum predictor of Eq. (ustar) (Helmholtz operator, explicit
// convective term, right-hand side).
//
// Thread layout: one thread per grid point, blocks of 32 x 8 in (x, y) and one
// z-plane per blockIdx.z, so that a warp reads 32 consecutive x values of each
// neighbour row (coalesced; the y/z neighbours hit L1/L2).
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

// Helmholtz residual of the predictor: res = rhs - (a u - nu Lap u) on
// interior faces.  Along the face-normal axis the wall faces hold 0; along the
// other axes the ghost beyond a wall is -u (no-slip at the wall midpoint).
__global__ void __launch_bounds__(BX * BY) k_helm_residual(Dims d, FaceGeom g,
                                                           const double* __restrict__ u,
                                                           double a, double nu_h2,
                                                           const double* __restrict__ rhs,
                                                           double* __restrict__ res) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  const int p3[3] = {i, j, k};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (i >= g.n[c][0] || j >= g.n[c][1] || k >= g.n[c][2]) continue;
    const int64_t f = fidx(g, c, i, j, k);
    if (p3[c] == 0 || p3[c] == g.n[c][c] - 1) { res[f] = 0.0; continue; }
    const double uc = __ldg(u + f);
    double s = 0.0, diag = a + 6.0 * nu_h2;
    const int64_t st[3] = {1, g.sy[c], g.sz[c]};
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      const int n_e = g.n[c][e];
      if (e == c) {   // neighbours are faces along their own normal
        if (p3[e] - 1 > 0) s += __ldg(u + f - st[e]);
        if (p3[e] + 1 < n_e - 1) s += __ldg(u + f + st[e]);
      } else {
        if (p3[e] > 0) s += __ldg(u + f - st[e]); else diag += nu_h2;
        if (p3[e] < n_e - 1) s += __ldg(u + f + st[e]); else diag += nu_h2;
      }
    }
    const double Au = fma(diag, uc, -nu_h2 * s);
    res[f] = __ldg(rhs + f) - Au;
  }
}

// One Chebyshev step for A e = r in FP32 (A the predictor's Helmholtz
// operator): e_new = e + beta (e - e_old) + alpha (r - A e); with first != 0
// the iterate is 0 and e_new = alpha r.
__global__ void __launch_bounds__(BX * BY) k_helm_cheb(Dims d, FaceGeom g,
                                                       const float* __restrict__ e,
                                                       const float* __restrict__ e_old,
                                                       const float* __restrict__ r, float a,
                                                       float nu_h2, float alpha, float beta,
                                                       float* __restrict__ e_new, int first) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  const int p3[3] = {i, j, k};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (i >= g.n[c][0] || j >= g.n[c][1] || k >= g.n[c][2]) continue;
    const int64_t f = fidx(g, c, i, j, k);
    if (p3[c] == 0 || p3[c] == g.n[c][c] - 1) { e_new[f] = 0.f; continue; }
    const float rc = __ldg(r + f);
    if (first) { e_new[f] = alpha * rc; continue; }
    const float ec = __ldg(e + f);
    float s = 0.f, diag = a + 6.f * nu_h2;
    const int64_t st[3] = {1, g.sy[c], g.sz[c]};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const int n_q = g.n[c][q];
      if (q == c) {
        if (p3[q] - 1 > 0) s += __ldg(e + f - st[q]);
        if (p3[q] + 1 < n_q - 1) s += __ldg(e + f + st[q]);
      } else {
        if (p3[q] > 0) s += __ldg(e + f - st[q]); else diag += nu_h2;
        if (p3[q] < n_q - 1) s += __ldg(e + f + st[q]); else diag += nu_h2;
      }
    }
    const float res = rc - fmaf(diag, ec, -nu_h2 * s);
    e_new[f] = ec + beta * (ec - __ldg(e_old + f)) + alpha * res;
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

void launch_helm_apply(Dims d, const double* u, double a, double nu_h2, const double* rhs,
                       double* res, cudaStream_t s) {
  count_launch();
  k_helm_residual<<<face_grid(d), dim3(BX, BY), 0, s>>>(d, make_face_geom(d), u, a, nu_h2, rhs,
                                                         res);
}

void launch_helm_cheb(Dims d, const float* e, const float* e_old, const float* r, float a,
                      float nu_h2, float alpha, float beta, float* e_new, int first,
                      cudaStream_t s) {
  count_launch();
  k_helm_cheb<<<face_grid(d), dim3(BX, BY), 0, s>>>(d, make_face_geom(d), e, e_old, r, a, nu_h2,
                                                     alpha, beta, e_new, first);
}

void launch_advection(Dims d, const double* u, double inv_h, double* out, cudaStream_t s) {
  count_launch();
  k_advection<<<face_grid(d), dim3(BX, BY), 0, s>>>(d, make_face_geom(d), u, inv_h, out);
}

void launch_predictor_rhs(Dims d, const double* u_n, const double* u_nm1, const double* p_n,
                          const double* f_body, const double* adv, double inv_2dt, double inv_h,
                          double* rhs, cudaStream_t s) {
  count_launch();
  k_predictor_rhs<<<face_grid(d), dim3(BX, BY), 0, s>>>(d, make_face_geom(d), u_n, u_nm1, p_n,
                                                         f_body, adv, inv_2dt, inv_h, rhs);
}

}  // namespace ibm
