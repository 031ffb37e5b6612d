// Two-way coupled rigid spheres (Sec. 3.2): one time step of the partitioned
// predictor-corrector of Sec. 3.2.1.
//
// Step 1 (host, per sphere): centre (4 x^n - x^{n-1})/3 + (2/3) dt u_s^n
//   (Eq. (particle_position)) and orientation R^{n+1} = R^n R_Delta with the
//   Rodrigues increment of Eqs. (rotat_axis)-(incement_matr); the markers
//   x_c + R L0 (k_rigid_positions) are set on the context once.
// Step 2: the momentum predictor of Eq. (ustar_two_way), as in ibm_step.
// Step 3, per correction: the IB force and torque per body (k_body_loads) and
//   the enclosed-fluid momentum of Eq. (volume_integrals) (k_sphere_momentum:
//   every face whose control volume can meet the sphere, volume fraction from
//   the signed distance at the 8 corners, Kempe & Froehlich 2012), both as
//   fixed-order per-block partials summed on the host; Newton's laws in the
//   BDF2 forms of Eqs. (bdy_linear_vel_iter), (bdy_angular_vel_iter) on the
//   host (a few scalars per body); U = u_s + omega x (X - x_c)
//   (k_rigid_velocity, Eq. (kinematic_constraint_iterative)); the scalar Schur
//   solve of Eq. (pressure_force_iterative_system); relaxed updates; the L1
//   ratio of Eq. (convergence_criterion) (k_asum2).
//
// Units: lengths of the grid, fluid density 1; a sphere of radius r has
// volume V = 4 pi r^3 / 3 and inertia theta J, J = 2 V r^2 / 5 (the paper's
// 6/(pi theta) and 60/(pi theta) for r = 1/2).  The angular velocity is
// integrated in the inertial frame (isotropic inertia); the body-frame vector
// R^T omega feeds the Rodrigues update.
#include "ibm_internal.cuh"

#include <cmath>
#include <vector>

namespace ibm {

namespace {

constexpr int TPB = 256;
constexpr int kLoadBlocks = 16;     // per body
constexpr int kMomBlocks = 32;      // per body and component
constexpr int kAsumBlocks = 256;
constexpr double kPi = 3.14159265358979323846;

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < TPB / 32; ++w) t += sh[w];
  return t;   // valid in thread 0
}

// X[e][k] = x_c[e] + sum_j R[e][j] L0[j][k]; pose per body: [x_c(3) | R(9)]
__global__ void k_rigid_positions(int64_t n, const double* __restrict__ L0,
                                  const int32_t* __restrict__ bid, const double* __restrict__ pose,
                                  int nb, double* __restrict__ X, int32_t* err) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int b = bid[k];
  if (b < 0 || b >= nb) {
    atomicOr(err, 1);
    for (int e = 0; e < 3; ++e) X[e * n + k] = 0.0;
    return;
  }
  const double* q = pose + 12 * b;
  const double l0 = L0[k], l1 = L0[n + k], l2 = L0[2 * n + k];
  for (int e = 0; e < 3; ++e)
    X[e * n + k] = q[e] + (q[3 + 3 * e] * l0 + q[4 + 3 * e] * l1 + q[5 + 3 * e] * l2);
}

// U[e][k] = u_s + omega x (X_k - x_c); vel per body: [x_c(3) | u_s(3) | omega(3)]
__global__ void k_rigid_velocity(int64_t n, const double* __restrict__ X,
                                 const int32_t* __restrict__ bid, const double* __restrict__ vel,
                                 double* __restrict__ U) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double* q = vel + 9 * bid[k];
  const double rx = X[k] - q[0], ry = X[n + k] - q[1], rz = X[2 * n + k] - q[2];
  U[k] = q[3] + (q[7] * rz - q[8] * ry);
  U[n + k] = q[4] + (q[8] * rx - q[6] * rz);
  U[2 * n + k] = q[5] + (q[6] * ry - q[7] * rx);
}

// partials of [h^3 sum F_k | h^3 sum (X_k - x_c) x F_k] over the markers of
// body blockIdx.y: part[(b * gridDim.x + blockIdx.x) * 6 + q]
__global__ void __launch_bounds__(TPB) k_body_loads(int64_t n, const double* __restrict__ F,
                                                    const double* __restrict__ X,
                                                    const int32_t* __restrict__ bid,
                                                    const double* __restrict__ xc, double h3,
                                                    double* __restrict__ part) {
  const int b = blockIdx.y;
  const double cx = xc[3 * b], cy = xc[3 * b + 1], cz = xc[3 * b + 2];
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t k = blockIdx.x * (int64_t)TPB + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * TPB) {
    if (bid[k] != b) continue;
    const double fx = F[k], fy = F[n + k], fz = F[2 * n + k];
    const double rx = X[k] - cx, ry = X[n + k] - cy, rz = X[2 * n + k] - cz;
    acc[0] += fx; acc[1] += fy; acc[2] += fz;
    acc[3] += ry * fz - rz * fy;
    acc[4] += rz * fx - rx * fz;
    acc[5] += rx * fy - ry * fx;
  }
  __shared__ double sh[TPB / 32];
  for (int q = 0; q < 6; ++q) {
    const double t = block_sum(acc[q], sh);
    if (threadIdx.x == 0) part[((int64_t)b * gridDim.x + blockIdx.x) * 6 + q] = h3 * t;
  }
}

// Enclosed-fluid momentum of Eq. (volume_integrals) for body y / 3 and
// velocity component y % 3 (y = blockIdx.y) over the face box
// box[y] = {i0, i1, j0, j1, k0, k1} (half-open, interior faces only):
// w = alpha u_d h^3 with alpha = sum_corners max(-phi, 0) / sum |phi| over the
// 8 corners of the face's control volume, phi = |x - x_c| - r.  Partials
// [lin(3) | ang(3)] at part[(y * gridDim.x + blockIdx.x) * 6 + q].
__global__ void __launch_bounds__(TPB) k_sphere_momentum(Dims d, double h,
                                                         const double* __restrict__ u,
                                                         const double* __restrict__ sph,
                                                         const int32_t* __restrict__ box,
                                                         double* __restrict__ part) {
  const int y = blockIdx.y;
  const int b = y / 3, dc = y % 3;
  const double cx = sph[4 * b], cy = sph[4 * b + 1], cz = sph[4 * b + 2], r = sph[4 * b + 3];
  const int32_t* bx = box + 6 * y;
  const int64_t ni = bx[1] - bx[0], nj = bx[3] - bx[2], nk = bx[5] - bx[4];
  const int64_t cnt = (ni > 0 && nj > 0 && nk > 0) ? ni * nj * nk : 0;
  const FaceDims fd = face_dims(d);
  const int64_t foff = dc == 0 ? 0 : (dc == 1 ? fd.nfx : fd.nfx + fd.nfy);
  const int64_t sy = d.nx + (dc == 0 ? 1 : 0);
  const int64_t sz = sy * (d.ny + (dc == 1 ? 1 : 0));
  const double ox = dc == 0 ? 0.0 : 0.5, oy = dc == 1 ? 0.0 : 0.5, oz = dc == 2 ? 0.0 : 0.5;
  const double h3 = h * h * h;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t t = blockIdx.x * (int64_t)TPB + threadIdx.x; t < cnt;
       t += (int64_t)gridDim.x * TPB) {
    const int i = bx[0] + (int)(t % ni);
    const int j = bx[2] + (int)((t / ni) % nj);
    const int k = bx[4] + (int)(t / (ni * nj));
    const double x = (i + ox) * h, yy = (j + oy) * h, z = (k + oz) * h;
    double num = 0.0, den = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const double px = x + ((q & 1) ? 0.5 : -0.5) * h - cx;
      const double py = yy + ((q & 2) ? 0.5 : -0.5) * h - cy;
      const double pz = z + ((q & 4) ? 0.5 : -0.5) * h - cz;
      const double phi = sqrt(px * px + py * py + pz * pz) - r;
      num += fmax(-phi, 0.0);
      den += fabs(phi);
    }
    if (num == 0.0) continue;
    const double w = (num / den) * u[foff + k * sz + j * sy + i] * h3;
    const double rv[3] = {x - cx, yy - cy, z - cz};
    acc[dc] += w;
    // r x (w e_dc): +r_{d2} w along d1, -r_{d1} w along d2 ((dc, d1, d2) cyclic)
    const int d1 = (dc + 1) % 3, d2 = (dc + 2) % 3;
    acc[3 + d1] += rv[d2] * w;
    acc[3 + d2] -= rv[d1] * w;
  }
  __shared__ double sh[TPB / 32];
  for (int q = 0; q < 6; ++q) {
    const double t = block_sum(acc[q], sh);
    if (threadIdx.x == 0) part[((int64_t)y * gridDim.x + blockIdx.x) * 6 + q] = t;
  }
}

// per-block partials of sum |a| and sum |b|: part[2 * blockIdx.x + {0, 1}]
__global__ void __launch_bounds__(TPB) k_asum2(int64_t n, const double* __restrict__ a,
                                               const double* __restrict__ b,
                                               double* __restrict__ part) {
  double sa = 0.0, sb = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)TPB + threadIdx.x; i < n; i += (int64_t)gridDim.x * TPB) {
    sa += fabs(a[i]);
    sb += fabs(b[i]);
  }
  __shared__ double sh[TPB / 32];
  const double ta = block_sum(sa, sh);
  const double tb = block_sum(sb, sh);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = ta;
    part[2 * blockIdx.x + 1] = tb;
  }
}

// ---- host-side rigid-body algebra ----
void matmul3(const double* A, const double* B, double* C) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      C[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
}

// R_Delta of Eq. (incement_matr) with axis om_cs/|om_cs| (Eq. (rotat_axis)) and
// angle dt (3/2 |om_cs^n| - 1/2 |om_cs^{n-1}|) (Eq. (theta))
void rodrigues(const double* om, const double* om_prev, double dt, double* Rd) {
  const double nrm = std::sqrt(om[0] * om[0] + om[1] * om[1] + om[2] * om[2]);
  for (int i = 0; i < 9; ++i) Rd[i] = (i % 4 == 0) ? 1.0 : 0.0;
  if (nrm == 0.0) return;
  const double np = std::sqrt(om_prev[0] * om_prev[0] + om_prev[1] * om_prev[1] +
                              om_prev[2] * om_prev[2]);
  const double a0 = om[0] / nrm, a1 = om[1] / nrm, a2 = om[2] / nrm;
  const double W[9] = {0.0, -a2, a1, a2, 0.0, -a0, -a1, a0, 0.0};
  double W2[9];
  matmul3(W, W, W2);
  const double g = dt * (1.5 * nrm - 0.5 * np);
  const double s = std::sin(g), c1 = 1.0 - std::cos(g);
  for (int i = 0; i < 9; ++i) Rd[i] += s * W[i] + c1 * W2[i];
}

// u_s, omega_s of Eqs. (bdy_linear_vel_iter), (bdy_angular_vel_iter)
void rigid_update(const ibm_rigid_sphere& b, double dt, const double* Fs, const double* Ts,
                  const double* lin, const double* ang, const double* g, double* us,
                  double* om) {
  if (!b.free_motion) {
    for (int e = 0; e < 3; ++e) { us[e] = b.us[e]; om[e] = b.om[e]; }
    return;
  }
  const double V = 4.0 * kPi * b.radius * b.radius * b.radius / 3.0;
  const double J = 0.4 * V * b.radius * b.radius;
  const double th = b.theta;
  for (int e = 0; e < 3; ++e) {
    us[e] = (4.0 * b.us[e] - b.us_prev[e]) / 3.0 - (2.0 * dt / 3.0) * Fs[e] / (th * V) +
            (3.0 * lin[e] - 4.0 * b.mom[e] + b.mom_prev[e]) / (3.0 * th * V) +
            (2.0 * dt / 3.0) * (th - 1.0) / th * g[e];
    om[e] = (4.0 * b.om[e] - b.om_prev[e]) / 3.0 - (2.0 * dt / 3.0) * Ts[e] / (th * J) +
            (3.0 * ang[e] - 4.0 * b.amom[e] + b.amom_prev[e]) / (3.0 * th * J);
  }
}

struct FsiScratch {
  double* dev = nullptr;     // [nb * 12] poses / velocities, then partials
  int32_t* box = nullptr;    // [nb * 3 * 6]
  size_t cap = 0, box_cap = 0;
};

}  // namespace

}  // namespace ibm

using namespace ibm;

extern "C" {

void ibm_default_fsi_opts(ibm_fsi_opts* f) {
  if (!f) return;
  f->gravity[0] = f->gravity[1] = f->gravity[2] = 0.0;
  f->xi = 1.0;
  f->tol = 1e-3;
  f->max_inner = 50;
  f->criterion = IBM_FSI_CRIT_LAGRANGIAN;
}

ibm_status ibm_fsi_step(ibm_ctx* c, int32_t nb, ibm_rigid_sphere* bodies, int64_t n,
                        const double* L0, const int32_t* body_id, const double* u_n,
                        const double* u_nm1, const double* p_n, const double* F_n,
                        const double* f_body, double* X_np1, double* u_np1, double* p_np1,
                        double* F_np1, const ibm_solve_opts* o, const ibm_fsi_opts* fo,
                        ibm_fsi_stats* fst) {
  if (check_ctx(c) != IBM_OK) return IBM_ERR_ARG;
  if (nb < 1 || nb > 4096 || !bodies || !fo) return set_err(c, IBM_ERR_ARG, "bad bodies/fopts");
  if (n < 1 || bad_ptr(L0) || body_id == nullptr || bad_ptr(X_np1) || bad_ptr(F_n) ||
      bad_ptr(F_np1))
    return set_err(c, IBM_ERR_ARG, "bad marker arguments");
  if (bad_ptr(u_n) || bad_ptr(u_nm1) || bad_ptr(p_n) || bad_ptr(u_np1) || bad_ptr(p_np1) ||
      (f_body && bad_ptr(f_body)))
    return set_err(c, IBM_ERR_ARG, "bad field pointer");
  if (u_np1 == u_n || u_np1 == u_nm1 || p_np1 == p_n || F_np1 == F_n || X_np1 == L0)
    return set_err(c, IBM_ERR_ARG, "outputs must not alias inputs");
  if (!(fo->xi > 0.0) || !(fo->tol >= 0.0) || fo->max_inner < 1 ||
      (fo->criterion != IBM_FSI_CRIT_LAGRANGIAN && fo->criterion != IBM_FSI_CRIT_EULERIAN))
    return set_err(c, IBM_ERR_ARG, "need xi > 0, tol >= 0, max_inner >= 1 and a known criterion");
  for (int b = 0; b < nb; ++b)
    if (!(bodies[b].radius > 0.0) || !(bodies[b].theta > 0.0))
      return set_err(c, IBM_ERR_ARG, "sphere radius and density ratio must be positive");
  ibm_status s = check_opts(c, o);
  if (s != IBM_OK) return s;
  if (o->c_mode != IBM_CMODE_SCALAR)
    return set_err(c, IBM_ERR_ARG, "the two-way step uses the scalar C mode");
  if ((s = ensure_krylov(c, o->restart)) != IBM_OK) return s;
  set_cmode(c, o);
  ibm_fsi_stats local;
  if (!fst) fst = &local;
  memset(fst, 0, sizeof(*fst));
  const int ph = prof_begin(c, IBM_PROF_FSI);
  cudaStream_t str = c->stream;
  const double dt = c->dt, h = c->h, a = 1.5 / dt, inv_h = 1.0 / h, h3 = h * h * h;

  // scratch: per-body parameters and the partial sums live in red_part
  // (kRedBlocks * (kMaxRestart + 2) doubles); the face boxes in cell_flag
  const size_t need = (size_t)nb * (12 + 6 * kLoadBlocks + 18 * kMomBlocks) + 2 * kAsumBlocks;
  if (need > (size_t)kRedBlocks * (kMaxRestart + 2) || (int64_t)nb * 18 > c->m + 1) {
    prof_end(c, ph);
    return set_err(c, IBM_ERR_ARG, "too many bodies for the reduction scratch");
  }
  double* d_par = c->red_part;                         // [nb][12]
  double* d_load = d_par + 12 * nb;                    // [nb][kLoadBlocks][6]
  double* d_mom = d_load + (size_t)6 * kLoadBlocks * nb;   // [nb*3][kMomBlocks][6]
  double* d_asum = d_mom + (size_t)18 * kMomBlocks * nb;   // [kAsumBlocks][2]
  int32_t* d_box = c->cell_flag;                       // [nb*3][6]

  // ---- Step 1: positions and orientations ----
  std::vector<double> pose(12 * nb), Rn(9 * nb), xn(3 * nb);
  for (int b = 0; b < nb; ++b) {
    const ibm_rigid_sphere& B = bodies[b];
    double Rd[9];
    rodrigues(B.om_cs, B.om_cs_prev, dt, Rd);
    matmul3(B.rot, Rd, &Rn[9 * b]);
    for (int e = 0; e < 3; ++e)
      xn[3 * b + e] = (4.0 * B.xc[e] - B.xc_prev[e]) / 3.0 + (2.0 / 3.0) * dt * B.us[e];
    for (int e = 0; e < 3; ++e) pose[12 * b + e] = xn[3 * b + e];
    for (int q = 0; q < 9; ++q) pose[12 * b + 3 + q] = Rn[9 * b + q];
  }
  IBM_CUDA(c, cudaMemcpyAsync(d_par, pose.data(), sizeof(double) * pose.size(),
                              cudaMemcpyHostToDevice, str));
  launch_zero(c->dev_flag, sizeof(int32_t), str);
  count_launch();
  k_rigid_positions<<<div_up(n, TPB), TPB, 0, str>>>(n, L0, body_id, d_par, nb, X_np1,
                                                     c->dev_flag);
  IBM_LAUNCH_CHECK(c);
  launch_to_host(c->dev_flag, c->host_flag_dev, sizeof(int32_t), str);
  IBM_LAUNCH_CHECK(c);
  IBM_CUDA(c, cudaStreamSynchronize(str));
  if (c->host_flag[0]) { prof_end(c, ph); return set_err(c, IBM_ERR_ARG, "body_id out of range"); }
  if ((s = ibm_set_markers(c, n, X_np1)) != IBM_OK) { prof_end(c, ph); return s; }
  MarkerData& mk = c->mk;

  // face boxes of every (body, component): control volumes within r + h/2
  std::vector<int32_t> box(18 * nb);
  const int ncell[3] = {c->d.nx, c->d.ny, c->d.nz};
  for (int b = 0; b < nb; ++b)
    for (int dc = 0; dc < 3; ++dc)
      for (int e = 0; e < 3; ++e) {
        const double off = (e == dc) ? 0.0 : 0.5;
        const double r = bodies[b].radius;
        int lo = (int)std::floor((xn[3 * b + e] - r) / h - off - 0.5) - 1;
        int hi = (int)std::ceil((xn[3 * b + e] + r) / h - off + 0.5) + 2;
        const int lo_lim = (e == dc) ? 1 : 0;
        const int hi_lim = (e == dc) ? ncell[e] : ncell[e];   // faces 1..n-1 or cells 0..n-1
        lo = lo < lo_lim ? lo_lim : lo;
        hi = hi > hi_lim ? hi_lim : hi;
        box[18 * b + 6 * dc + 2 * e] = lo;
        box[18 * b + 6 * dc + 2 * e + 1] = hi > lo ? hi : lo;
      }
  IBM_CUDA(c, cudaMemcpyAsync(d_box, box.data(), sizeof(int32_t) * box.size(),
                              cudaMemcpyHostToDevice, str));
  std::vector<double> sph(4 * nb);
  for (int b = 0; b < nb; ++b) {
    for (int e = 0; e < 3; ++e) sph[4 * b + e] = xn[3 * b + e];
    sph[4 * b + 3] = bodies[b].radius;
  }
  // enclosed-fluid momentum of u at the new positions -> lin[nb][3], ang[nb][3]
  std::vector<double> hpart((size_t)18 * kMomBlocks * nb);
  auto momentum = [&](const double* u, std::vector<double>& lin,
                      std::vector<double>& ang) -> ibm_status {
    IBM_CUDA(c, cudaMemcpyAsync(d_par, sph.data(), sizeof(double) * sph.size(),
                                cudaMemcpyHostToDevice, str));
    count_launch();
    k_sphere_momentum<<<dim3(kMomBlocks, 3 * nb), TPB, 0, str>>>(c->d, h, u, d_par, d_box, d_mom);
    IBM_LAUNCH_CHECK(c);
    IBM_CUDA(c, cudaMemcpyAsync(hpart.data(), d_mom, sizeof(double) * hpart.size(),
                                cudaMemcpyDeviceToHost, str));
    IBM_CUDA(c, cudaStreamSynchronize(str));
    lin.assign(3 * nb, 0.0);
    ang.assign(3 * nb, 0.0);
    for (int b = 0; b < nb; ++b)
      for (int dc = 0; dc < 3; ++dc)
        for (int blk = 0; blk < kMomBlocks; ++blk) {
          const double* q = &hpart[(((size_t)(3 * b + dc)) * kMomBlocks + blk) * 6];
          for (int e = 0; e < 3; ++e) {
            lin[3 * b + e] += q[e];
            ang[3 * b + e] += q[3 + e];
          }
        }
    return IBM_OK;
  };

  // ---- Step 2: predictor (Eq. (ustar_two_way)) into u_np1 ----
  launch_predictor_rhs_adv(c->d, u_n, u_nm1, p_n, f_body, o->with_advection, 1.0 / (2.0 * dt),
                           inv_h, c->f1, str);
  launch_shell_spread_faces(c, F_n, 1.0, c->f1);
  IBM_LAUNCH_CHECK(c);
  s = helmholtz_solve(c, c->f1, u_np1, o, &fst->helm_iters, &fst->helm_relres);
  if (s != IBM_OK) { prof_end(c, ph); return s; }
  launch_copy(p_np1, p_n, sizeof(double) * c->m, str);
  launch_copy(F_np1, F_n, sizeof(double) * 3 * n, str);

  // ---- Step 3: corrections ----
  std::vector<double> lin, ang, vel(9 * nb), loads((size_t)6 * kLoadBlocks * nb),
      us(3 * nb), om(3 * nb), asum(2 * kAsumBlocks), xc_dev(3 * nb);
  for (int q = 0; q < 3 * nb; ++q) xc_dev[q] = xn[q];
  for (int b = 0; b < nb; ++b)
    for (int e = 0; e < 3; ++e) { us[3 * b + e] = bodies[b].us[e]; om[3 * b + e] = bodies[b].om[e]; }
  double* Ugam = mk.t3;      // U^{(k)} (t3 is free in the scalar C mode)
  double* pc = c->c3;
  ibm_status solve_status = IBM_OK;
  double ratio = 1.0;
  int inner = 0;
  for (int k = 0; k < fo->max_inner; ++k) {
    // IB force and torque of F^{(n,k)} per body
    IBM_CUDA(c, cudaMemcpyAsync(d_par, xc_dev.data(), sizeof(double) * 3 * nb,
                                cudaMemcpyHostToDevice, str));
    count_launch();
    k_body_loads<<<dim3(kLoadBlocks, nb), TPB, 0, str>>>(n, F_np1, X_np1, body_id, d_par, h3,
                                                         d_load);
    IBM_LAUNCH_CHECK(c);
    IBM_CUDA(c, cudaMemcpyAsync(loads.data(), d_load, sizeof(double) * loads.size(),
                                cudaMemcpyDeviceToHost, str));
    if ((s = momentum(u_np1, lin, ang)) != IBM_OK) { prof_end(c, ph); return s; }
    for (int b = 0; b < nb; ++b) {
      double Fs[3] = {0, 0, 0}, Ts[3] = {0, 0, 0};
      for (int blk = 0; blk < kLoadBlocks; ++blk)
        for (int e = 0; e < 3; ++e) {
          Fs[e] += loads[((size_t)b * kLoadBlocks + blk) * 6 + e];
          Ts[e] += loads[((size_t)b * kLoadBlocks + blk) * 6 + 3 + e];
        }
      rigid_update(bodies[b], dt, Fs, Ts, &lin[3 * b], &ang[3 * b], fo->gravity, &us[3 * b],
                   &om[3 * b]);
      for (int e = 0; e < 3; ++e) {
        vel[9 * b + e] = xn[3 * b + e];
        vel[9 * b + 3 + e] = us[3 * b + e];
        vel[9 * b + 6 + e] = om[3 * b + e];
      }
    }
    IBM_CUDA(c, cudaMemcpyAsync(d_par, vel.data(), sizeof(double) * vel.size(),
                                cudaMemcpyHostToDevice, str));
    count_launch();
    k_rigid_velocity<<<div_up(n, TPB), TPB, 0, str>>>(n, X_np1, body_id, d_par, Ugam);
    // RHS_p = a G^T u, RHS_F = a (R^T u - U), b = RHS_p + 2 B^T RHS_F
    launch_gradt_axpby(c->d, u_np1, a * inv_h, nullptr, 0.0, c->c2, str);
    launch_interp(c, u_np1, mk.t2);
    launch_axpby(mk.t2, a, Ugam, -a, mk.t2, 3 * n, str);
    launch_shell_gradt_spread(c, mk.t2, 2.0, c->c2);
    launch_zero(pc, sizeof(double) * c->m, str);
    IBM_LAUNCH_CHECK(c);
    ibm_solve_stats sst;
    memset(&sst, 0, sizeof(sst));
    s = fgmres_solve(c, c->c2, pc, o, &sst, true);
    if (s != IBM_OK && s != IBM_ERR_NOT_CONVERGED) { prof_end(c, ph); return s; }
    if (s != IBM_OK) solve_status = s;
    fst->fgmres_iters += sst.iters;
    // F' = 2 (B p' - RHS_F); relaxed updates
    launch_marker_grad_interp(c, pc, 1.0, mk.t);
    launch_axpby(mk.t, 2.0, mk.t2, -2.0, mk.t, 3 * n, str);
    launch_axpby(p_np1, 1.0, pc, fo->xi, p_np1, c->m, str);
    launch_axpby(F_np1, 1.0, mk.t, fo->xi, F_np1, 3 * n, str);
    launch_grad_axpy(c->d, u_np1, pc, -fo->xi * (2.0 * dt / 3.0) * inv_h, u_np1, str);
    launch_shell_spread_faces(c, mk.t, fo->xi * (2.0 * dt / 3.0), u_np1);
    int nblk = kAsumBlocks;
    if (fo->criterion == IBM_FSI_CRIT_EULERIAN) {
      nblk = launch_shell_spread_asum2(c, mk.t, F_np1, d_asum);   // <= kAsumBlocks partials
      if (nblk > kAsumBlocks) { prof_end(c, ph); return set_err(c, IBM_ERR_ARG, "asum grid"); }
    } else {
      count_launch();
      k_asum2<<<kAsumBlocks, TPB, 0, str>>>(3 * n, mk.t, F_np1, d_asum);
    }
    IBM_LAUNCH_CHECK(c);
    IBM_CUDA(c, cudaMemcpyAsync(asum.data(), d_asum, sizeof(double) * 2 * nblk,
                                cudaMemcpyDeviceToHost, str));
    IBM_CUDA(c, cudaStreamSynchronize(str));
    double na = 0.0, nf = 0.0;
    for (int q = 0; q < nblk; ++q) { na += asum[2 * q]; nf += asum[2 * q + 1]; }
    if (!std::isfinite(na) || !std::isfinite(nf)) {
      prof_end(c, ph);
      return set_err(c, IBM_ERR_NAN, "non-finite force correction");
    }
    ratio = nf > 0.0 ? na / nf : 0.0;
    inner = k + 1;
    if (ratio < fo->tol) break;
  }
  // advance the bodies to t^{n+1}
  if ((s = momentum(u_np1, lin, ang)) != IBM_OK) { prof_end(c, ph); return s; }
  for (int b = 0; b < nb; ++b) {
    ibm_rigid_sphere& B = bodies[b];
    const double* R1 = &Rn[9 * b];
    for (int e = 0; e < 3; ++e) {
      B.xc_prev[e] = B.xc[e];
      B.xc[e] = xn[3 * b + e];
      B.us_prev[e] = B.us[e];
      B.us[e] = us[3 * b + e];
      B.om_prev[e] = B.om[e];
      B.om[e] = om[3 * b + e];
      B.om_cs_prev[e] = B.om_cs[e];
      B.mom_prev[e] = B.mom[e];
      B.mom[e] = lin[3 * b + e];
      B.amom_prev[e] = B.amom[e];
      B.amom[e] = ang[3 * b + e];
    }
    for (int e = 0; e < 3; ++e)   // om_cs = R^T om
      B.om_cs[e] = R1[e] * om[3 * b] + R1[3 + e] * om[3 * b + 1] + R1[6 + e] * om[3 * b + 2];
    for (int q = 0; q < 9; ++q) B.rot[q] = R1[q];
  }
  fst->inner = inner;
  fst->ratio = ratio;
  prof_end(c, ph);
  if (solve_status != IBM_OK) return solve_status;
  if (ratio >= fo->tol && fo->tol > 0.0) {
    char buf[160];
    snprintf(buf, sizeof buf, "two-way corrections stopped at ratio %.3g > tol %.3g (%s norm)",
             ratio, fo->tol, fo->criterion == IBM_FSI_CRIT_EULERIAN ? "spread" : "marker");
    return set_err(c, IBM_ERR_NOT_CONVERGED, buf);
  }
  return IBM_OK;
}

}  // extern "C"
