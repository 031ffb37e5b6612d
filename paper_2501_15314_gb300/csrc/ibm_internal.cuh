// Internal declarations shared by the CUDA translation units of libibmschur.
// Layout conventions are those of include/ibm_schur.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "ibm_schur.h"

namespace ibm {

constexpr int kMaxLevels = 16;
constexpr int kMaxRestart = 64;
constexpr int kMaxCoarse = 512;     // cells on the coarsest level (dense pinv)
constexpr int kRedBlocks = 1216;    // fixed grid of the two-stage reductions
constexpr int kRedThreads = 256;

struct Dims {
  int nx, ny, nz;
};

__host__ __device__ inline int64_t cells_of(Dims d) {
  return (int64_t)d.nx * d.ny * d.nz;
}

// Face-grid sizes of the packed face vector.
struct FaceDims {
  int64_t nfx, nfy, nfz;
};

__host__ __device__ inline FaceDims face_dims(Dims d) {
  FaceDims f;
  f.nfx = (int64_t)d.nz * d.ny * (d.nx + 1);
  f.nfy = (int64_t)d.nz * (d.ny + 1) * d.nx;
  f.nfz = (int64_t)(d.nz + 1) * d.ny * d.nx;
  return f;
}

// One multigrid level: cell counts, width, and FP32/FP64 buffers.
struct MGLevel {
  Dims d;
  double h;
  int64_t m;
  float* x32 = nullptr;
  float* b32 = nullptr;
  float* t32 = nullptr;   // ping-pong buffer for smoothing sweeps
  double* x64 = nullptr;
  double* b64 = nullptr;
  double* t64 = nullptr;
};

// Per-marker Roma data (Eq. (delta)).  For axis e: bf[e] is the first of the
// three face-type taps (positions i*h), bc[e] the first of the three
// centre-type taps (positions (i+1/2)h); wf/wc the 1-D weights; org[e] the
// origin of the 4x4x4 cell box covering every component's G^T R stencil.
struct MarkerData {
  int64_t n = 0, cap = 0;
  int32_t* bf = nullptr;    // [3][n]
  int32_t* bc = nullptr;    // [3][n]
  int32_t* org = nullptr;   // [3][n]
  double* wf = nullptr;     // [3 axes][3 taps][n]
  double* wc = nullptr;     // [3 axes][3 taps][n]
  double* cw = nullptr;     // [3 axes][4 cells][n] G^T-weighted face taps along
                            // the component's own axis: (w_{a-1} - w_a) / h
  double* dwf = nullptr;    // [3 axes][3 taps][n] phi' at the face taps
  double* dwc = nullptr;    // [3 axes][3 taps][n] phi' at the centre taps
  float* wc32 = nullptr;    // wc rounded to FP32 (the FP32 Arnoldi cycles' t = 2 B z)
  float* cw32 = nullptr;    // cw rounded to FP32
  double* cg = nullptr;     // [3][3n] conjugate-gradient work vectors for C^{-1}
  double* t3 = nullptr;     // [3][n] per-marker scratch (RHS_F in the C modes)
  // cell-sorted (marker, slot) list for the atomic-free gathers
  int64_t n_entries = 0, entries_cap = 0;
  int32_t* entry_key = nullptr;   // marker * 64 + slot, sorted within a cell
  // the same entries re-laid out for the B^T t gather: shell cells (in the
  // order of ell_cell) in groups of kEllCells (one warp, kEllLanes lanes per
  // cell), group w padded to its longest cell and stored interleaved, entry
  // kEllLanes r + j of the group's cell c at ell_base[w] + 32 r + kEllLanes c + j
  int64_t n_ell = 0, ell_cap = 0;
  int32_t* ell_key = nullptr;
  double* ell_coef = nullptr;     // [3][n_ell] G^T R coefficients (0 on padding)
  float* ell_coef32 = nullptr;    // [3][n_ell] their leading FP32 parts (FP32 Arnoldi cycles)
  // the spread R F onto the faces through the same layout: per entry and
  // component d the weight of F_{k,d} at the cell's lower d-face (0 on
  // padding and outside the support), and per shell cell (layout order) the
  // bits d of the faces inside some entry's support
  double* ell_sw = nullptr;       // [3][n_ell]
  uint8_t* ell_any = nullptr;     // [n_shell]
  int32_t* ell_base = nullptr;    // [n_groups + 1]
  int32_t* ell_len = nullptr;     // [n_groups] rounds (entries per lane)
  int64_t n_shell = 0;
  int32_t* shell_cell = nullptr;  // [n_shell] cells touched by any marker
  int32_t* shell_off = nullptr;   // [n_shell + 1] segment offsets
  // the shell cells in the order of the interleaved layout: within each
  // window of 1024 (128 groups) sorted by entry count, longest first, so that
  // the cells of a group have nearly equal counts and little padding
  int32_t* ell_cell = nullptr;    // [n_shell]
  double* t = nullptr;            // [3][n] per-marker scratch
  double* t2 = nullptr;           // [3][n] per-marker scratch
  float* t32 = nullptr;           // [3][n] t rounded to FP32 (FP32 Arnoldi cycles)
};

}  // namespace ibm

struct ibm_ctx {
  ibm::Dims d;
  double h, Re, dt;
  int64_t m, nf;
  ibm::FaceDims fd;
  cudaStream_t stream;
  // internal side stream and events: the marker gather of a Schur product
  // runs on it concurrently with the Laplacian
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaEvent_t ev_iter[2] = {nullptr, nullptr};   // ends of Krylov iterations (by parity)
  // FP32/double-single Arnoldi cycles replayed as one CUDA graph each
  // (krylov_df.cu): the capture stream, the graph and what it was built for,
  // the kernels each captured iteration launches, and the Givens state of a
  // cycle (device, and the mapped pinned copy the host reads after a cycle)
  cudaStream_t cap = nullptr;
  cudaGraph_t cyc_graph = nullptr;
  cudaGraphExec_t cyc_exec = nullptr;
  unsigned long long cyc_key[16] = {0};
  int cyc_launches[ibm::kMaxRestart] = {0};
  double* gstate = nullptr;
  double* host_gstate = nullptr;
  double* host_gstate_dev = nullptr;
  std::string err;

  // grid-sized scratch (FP64)
  int32_t* cell_count = nullptr;   // [m]
  int32_t* cell_start = nullptr;   // [m + 1]
  int32_t* cell_flag = nullptr;    // [m + 1]
  int32_t* scan_tmp = nullptr;     // block sums of the scans (int32 or int2 per block)
  int32_t* dev_flag = nullptr;     // device error word(s)
  int32_t* host_flag = nullptr;    // mapped pinned mirror (host address)
  int32_t* host_flag_dev = nullptr; // its device address
  double* c1 = nullptr;            // [m] cell temporaries
  double* c2 = nullptr;
  double* c3 = nullptr;
  double* f1 = nullptr;            // [nf] face temporaries
  double* f2 = nullptr;
  double* f3 = nullptr;
  double* f4 = nullptr;
  float* g1 = nullptr;             // [nf] FP32 face temporaries (predictor)
  float* g2 = nullptr;
  float* g3 = nullptr;
  float* g4 = nullptr;
  float* g5 = nullptr;             // low parts of the predictor's residual
  float* g6 = nullptr;             // the predictor's first correction, kept in FP32
  double* red_part = nullptr;      // [kRedBlocks][kMaxRestart + 2] partials
  double* red_out = nullptr;       // [8][kMaxRestart + 2] reduced values
  // set by the step around its solve: the solver leaves the constant of the
  // solution in place and writes the sum of its values here (device), which
  // the step subtracts where it forms p^{n+1} (G and B annihilate constants)
  double* defer_mean = nullptr;
  double* host_red = nullptr;      // mapped pinned mirror of red_out (host address)
  double* host_red_dev = nullptr;  // its device address
  double* helm_part = nullptr;     // per-block partials of the predictor norm
  int64_t helm_part_n = 0;         // its length (also holds the divergence norm's partials)

  // Krylov bases
  double* V = nullptr;             // [(kMaxRestart + 1)][m]
  double* Z = nullptr;             // [kMaxRestart][m]
  int restart_cap = 0;

  // multigrid hierarchy
  int n_levels = 0;
  ibm::MGLevel lv[ibm::kMaxLevels];
  double* coarse_pinv64 = nullptr; // dense [mc][mc]
  float* coarse_pinv32 = nullptr;
  int coarse_m = 0;
  // one-CTA chain of the coarse levels: its first level (-1: none), and the
  // packed coordinates and neighbour masks of its cells, built at setup
  int chain_l = -1;
  void* chain_tab = nullptr;

  ibm::MarkerData mk;
  bool markers_set = false;

  // C mode of the running call (set from the options at every entry point)
  int cmode = 0;
  double c_rtol = 1e-14;
  int c_maxit = 500;
  int64_t c_iters = 0;             // inner CG iterations since the call began
  double* cg_scal = nullptr;       // [8] device scalars of the CG on C

  // event timing of kernel classes (ibm_profile_enable)
  bool prof_on = false;
  double prof_acc = 0.0;   // algorithmic bytes counted while profiling
  struct ProfRec {
    int cls;
    cudaEvent_t a, b;
    double bytes;   // algorithmic bytes of the timed kernels
  };
  std::vector<ProfRec> prof;
  size_t prof_used = 0;
};

namespace ibm {

// Algorithmic bytes of the marker term of one Schur product (each array read
// or written once): per marker its tap bases, Roma weights and G-weighted
// weights (192 B), t written and read back (24 + 24 B; in the FP32 form t is
// written in FP64 and FP32 and read in FP32, the same 48 B); per cell-sorted
// entry its key and three G^T R coefficients (entry_bytes: 28 B, or 16 B
// from the FP32 copies); per shell cell the input value (sz_in), the cell
// index and the output read and written (2 sz_out).
inline double marker_term_bytes(const ibm_ctx* c, int sz_in, int sz_out, int entry_bytes = 28) {
  return (double)c->mk.n * 240.0 + (double)c->mk.n_entries * entry_bytes +
         (double)c->mk.n_shell * (sz_in + 4 + 2 * sz_out);
}

// ---- error helpers (host) ----
ibm_status set_err(ibm_ctx* c, ibm_status s, const std::string& msg);
ibm_status cuda_err(ibm_ctx* c, cudaError_t e, const char* where);

#define IBM_CUDA(ctx, call)                                           \
  do {                                                                \
    cudaError_t e_ = (call);                                          \
    if (e_ != cudaSuccess) return ::ibm::cuda_err((ctx), e_, #call);  \
  } while (0)

#define IBM_LAUNCH_CHECK(ctx)                                              \
  do {                                                                     \
    cudaError_t e_ = cudaGetLastError();                                   \
    if (e_ != cudaSuccess) return ::ibm::cuda_err((ctx), e_, "kernel launch"); \
  } while (0)

// argument and workspace helpers shared by the C entry points (capi.cu)
bool bad_ptr(const void* p);
ibm_status check_ctx(ibm_ctx* c);
ibm_status check_opts(ibm_ctx* c, const ibm_solve_opts* o);
ibm_status ensure_krylov(ibm_ctx* c, int restart);
ibm_status norm2_host(ibm_ctx* c, const double* x, int64_t n, double* out);
// the same to about 1e-5 relative without FP64 arithmetic per element (an
// exact FP64 dot when that is not finite): for stopping baselines
ibm_status norm2_lead_host(ibm_ctx* c, const double* x, int64_t n, double* out);
void launch_norm2_lead(const double* x, int64_t n, double* part, double* out, cudaStream_t s,
                       double* hout);
// (a - nu Lap) u = rhs of Eq. (ustar) to o->helm_rtol; uses g1..g6
ibm_status helmholtz_solve(ibm_ctx* c, const double* rhs, double* u, const ibm_solve_opts* o,
                           int* iters, double* relres);

// ---- stencils (stencil.cu) ----
// out = scale * L v  (Neumann 7-point, L = G^T G with h folded into scale)
template <typename T>
void launch_laplacian(Dims d, const T* v, T* out, double inv_h2, cudaStream_t s);
// out = b - L v in FP64 (b null: out = L v)
void launch_laplacian_sub(Dims d, const double* v, const double* b, double* out, double inv_h2,
                          cudaStream_t s);
void launch_gradient(Dims d, const double* p, double* u, double inv_h, cudaStream_t s);
void launch_gradient_t(Dims d, const double* u, double* out, double inv_h, cudaStream_t s);
// part[b] = the sums of squares of alpha G^T u over the blocks of one launch
// (returns their count, gradt_norm2_blocks(d))
int64_t gradt_norm2_blocks(Dims d);
int64_t launch_gradt_norm2(Dims d, const double* u, double alpha, double* part, cudaStream_t s);
// u_out = u_in + alpha * G p   (interior faces; wall faces 0)
void launch_grad_axpy(Dims d, const double* u_in, const double* p, double alpha,
                      double* u_out, cudaStream_t s);
// out = alpha * G^T u + beta * c   (c may be null)
void launch_gradt_axpby(Dims d, const double* u, double alpha, const double* c,
                        double beta, double* out, cudaStream_t s);
// predictor helpers
// (rhi, rlo) = (rhi, rlo) - A e in double-single (see k_helm_resid_ds) with
// per-block sums of the new hi^2 in part[b * stride]; returns the block count
int64_t launch_helm_resid_ds(Dims d, const float* e, float* rhi, float* rlo, double a,
                             double nu_h2, double* part, int stride, cudaStream_t s);
// number of floats of the predictor's padded FP32 face layout
int64_t helm_fp32_size(Dims d);
// one FP32 Chebyshev step of the predictor (see k_helm_cheb_v4)
void launch_helm_cheb(Dims d, const float* e, const float* eo, float* r32, float* rlo,
                      const double* r64, double rs, float a, float nu_h2, float alpha, float beta,
                      float* en, double* u, double us, int mode, cudaStream_t s,
                      int flags = 0, const float* pe = nullptr, double ps = 0.0);
// u = ps pe on the interior faces (pe on the predictor's padded FP32 layout)
void launch_helm_flush(Dims d, const float* pe, double ps, double* u, cudaStream_t s);   // 1: e_old is zero; 2: u is zero (mode 2 writes it)
// predictor RHS with the convective term of u_n fused in (with_adv != 0),
// evaluated in double-single arithmetic (see k_predictor_rhs_ds)
void launch_predictor_rhs_adv(Dims d, const double* u_n, const double* u_nm1,
                              const double* p_n, const double* f_body, int with_adv,
                              double inv_2dt, double inv_h, double* rhs, cudaStream_t s);

// ---- markers (markers.cu) ----
ibm_status markers_build(ibm_ctx* c, int64_t n, const double* X);
// t[d][k] = scale * (B v)_{k,d} = scale * (R^T G v)_{k,d}
// (on stream st when given, else the context's stream)
void launch_marker_grad_interp(ibm_ctx* c, const double* v, double scale, double* t,
                               cudaStream_t st = nullptr);
void launch_marker_grad_interp_f32(ibm_ctx* c, const float* v, double scale, double* t,
                                   cudaStream_t st = nullptr);
// t32[d][k] = scale * (B v)_{k,d} for FP32 v in FP32 arithmetic (FP32 copies of
// the weights): the FP32 Arnoldi cycles, whose Schur product is rounded to FP32
void launch_marker_grad_interp_t32(ibm_ctx* c, const float* v, float scale, float* t32,
                                   cudaStream_t st = nullptr);
// out[cell] += scale * (G^T R t)[cell] on the shell cells
void launch_shell_gradt_spread(ibm_ctx* c, const double* t, double scale, double* out);
// U[d][k] = (R^T u)_{k,d}
void launch_interp(ibm_ctx* c, const double* u, double* U);
// Xbar[e][k] (+)= scale * sum_d m[d][k] * sum_i f_d,i dR_{i,(d,k)}/dX_{e,k}
void launch_interp_dpos(ibm_ctx* c, const double* f, const double* m, double scale,
                        bool accumulate, double* Xbar);
// u[face] = beta * u[face] + scale * (R F)[face] on shell faces only
void launch_shell_spread_faces(ibm_ctx* c, const double* F, double scale, double* u);
// u = R F on the shell faces only (written, not accumulated)
void launch_shell_spread_faces_set(ibm_ctx* c, const double* F, double* u);
// Per-block partial L1 norms of R A and R B (2 doubles per block into part);
// returns the number of blocks (0 without markers).
int launch_shell_spread_asum2(ibm_ctx* c, const double* A, const double* B, double* part);
// ---- C = R^T R (cmode.cu) ----
void apply_C(ibm_ctx* c, const double* v, double* out);
ibm_status c_solve(ibm_ctx* c, const double* t, double* s, double rtol, int maxit, int* iters);
// the ctx's C mode from the options (and the CG counter reset)
void set_cmode(ibm_ctx* c, const ibm_solve_opts* o);

// ---- reductions and vector kernels (krylov.cu) ----
// red_out[q] = <w, V_q>, q < nq (two-stage, fixed order)
// (with div != null also quot[q] = out[q] / div[q])
// (with hout != null, the device address of a place in the mapped host
// mirror, the reduced values are also written there: the host reads them
// after synchronising the stream, with no copy-engine transfer that bulk
// copies queued by the caller on other streams could hold up)
void launch_multidot(const double* w, const double* V, int64_t ld, int nq, int64_t n,
                     double* part, double* out, cudaStream_t s, const double* div = nullptr,
                     double* quot = nullptr, double* hout = nullptr);
// w -= sum_q coef[q] V_q  (coef on device), out = ||w||^2 (two-stage)
void launch_axpy_norm(double* w, const double* V, int64_t ld, int nq, const double* coef,
                      int64_t n, double* part, double* out, cudaStream_t s,
                      double* hout = nullptr);
void launch_dot(const double* a, const double* b, int64_t n, double* part, double* out,
                cudaStream_t s, double* hout = nullptr);
// zero nbytes / copy nbytes device to device (multiples of 4), by kernels
void launch_zero(void* p, int64_t nbytes, cudaStream_t s);
void launch_copy(void* dst, const void* src, int64_t nbytes, cudaStream_t s);
// nbytes (a multiple of 4) from device memory to dst_dev, the device address
// of a place in a mapped host mirror (host_red_dev, host_flag_dev)
void launch_to_host(const void* src, void* dst_dev, int nbytes, cudaStream_t s);
void launch_axpby(const double* x, double a, const double* y, double b, double* out,
                  int64_t n, cudaStream_t s);
// x += sum_q y[q] Z_q, y = the first nq host values (passed by value)
void launch_gemv_acc(double* x, const double* Z, int64_t ld, int nq, const double* y,
                     int64_t n, cudaStream_t s);
// out[0] = sum of part[b * (kMaxRestart + 2)], b < nb (fixed order)
// out = sum of part[b * stride], b < nb (fixed order)
void launch_final_reduce(const double* part, int nb, double* out, cudaStream_t s,
                         double* hout = nullptr, int stride = kMaxRestart + 2);
void launch_sum(const double* x, int64_t n, double* part, double* out, cudaStream_t s);
// out = x + (y + scale * (*val)), in the operations of k_add_scalar then k_axpby
void launch_axpy_shift(const double* x, const double* y, const double* val, double scale,
                       double* out, int64_t n, cudaStream_t s);
void launch_add_scalar_dev(double* x, int64_t n, const double* val, double scale,
                           cudaStream_t s);

// ---- scans (markers.cu) ----
ibm_status exclusive_scan(ibm_ctx* c, const int32_t* in, int32_t* out, int64_t n);

// ---- multigrid (multigrid.cu) ----
ibm_status mg_setup(ibm_ctx* c);
ibm_status mg_vcycle(ibm_ctx* c, const double* r, double* z, int prec, int pre, int post);
ibm_status mg_vcycle_f32(ibm_ctx* c, const float* r, float* z, int pre, int post);
// V-cycle on the leading parts of an interleaved (hi, lo) pair vector
ibm_status mg_vcycle_pair(ibm_ctx* c, const float2* r, float* z, int pre, int post);

// ---- double-single Arnoldi process (krylov_df.cu) ----
bool ds_supported(const ibm_ctx* c);
ibm_status schur_apply_ds(ibm_ctx* c, const float* z, float2* w);
ibm_status fgmres_solve_ds(ibm_ctx* c, const double* b, double* x, const ibm_solve_opts* o,
                           ibm_solve_stats* st, bool x_is_zero);

// ---- solver (krylov.cu) ----
ibm_status schur_apply(ibm_ctx* c, const double* v, double* out);
// out = b - S~ v (the FP64 true residual), in the passes of schur_apply
ibm_status schur_residual(ibm_ctx* c, const double* b, const double* v, double* out);
// x_is_zero: the initial guess in x is known to be 0 (skips one S~ product)
ibm_status fgmres_solve(ibm_ctx* c, const double* b, double* x, const ibm_solve_opts* o,
                        ibm_solve_stats* st, bool x_is_zero = false);

// Counts one kernel launch (process-wide counter, ibm_kernel_launches).
void count_launch();
// adds n (which may be negative) to the launch counter: kernels captured into
// a graph are counted when the graph runs them, not when they are captured
void add_launches(int64_t n);

// Per-body force and torque sums (Eq. (IBM_force)) in one launch of n_bodies
// blocks: out[6b..6b+5] = h3 (sum F, sum (X - c_b) x F) over the markers with
// bid == b; cen: device [n_bodies][3].  Shared by ibm_body_forces and its
// allocation-free variant.
void launch_body_sums(const double* F, const double* X, const int32_t* bid, int64_t n,
                      int n_bodies, const double* cen, double h3, double* out, cudaStream_t s);

// Records a start event for class cls (returns a handle, -1 when off) and the
// matching end event.
int prof_begin(ibm_ctx* c, int cls);
// bytes: the algorithmic DRAM bytes of the timed kernels (each array read or
// written once), summed per class by ibm_profile_read
void prof_end(ibm_ctx* c, int handle, double bytes = 0.0);
// Algorithmic bytes of kernels outside any timed class (while profiling):
// they count towards the enclosing span (prof_end_span).
void prof_note(ibm_ctx* c, double bytes);
// prof_end for a class whose bytes are those counted (prof_end, prof_note)
// since prof_mark returned `mark`: the V-cycle, the solve, the step.
double prof_mark(const ibm_ctx* c);
void prof_end_span(ibm_ctx* c, int handle, double mark);
// prof_end when the class is timed (handle >= 0), else prof_note.
void prof_end_or_note(ibm_ctx* c, int handle, double bytes);

// Interleaved layout of the B^T t gather: a group (one warp) holds kEllCells
// shell cells, kEllLanes lanes per cell; lane l takes the entries
// p = kEllLanes r + l % kEllLanes of its cell, stored at base + 32 r + l.
#ifndef IBM_ELL_LANES
#define IBM_ELL_LANES 4
#endif
constexpr int kEllLanes = IBM_ELL_LANES;
constexpr int kEllCells = 32 / kEllLanes;
__host__ __device__ inline int64_t ell_groups(int64_t n_shell) {
  return (n_shell + kEllCells - 1) / kEllCells;
}

// Sum of the kEllLanes lanes of a cell, in a fixed order (all 32 lanes of
// the warp take part).
__device__ __forceinline__ double ell_combine(double v) {
#pragma unroll
  for (int o = 1; o < kEllLanes; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One lane's share of a shell cell's entries in the interleaved layout
// (round p at idx + 32 p): sum_p sum_e coef_e[p] t_e[marker(p)], FP64 FMAs
// in round order.  Four entries' loads are issued before their FMAs (the marker
// index of an entry must arrive before its t can be gathered, so one entry at
// a time leaves the thread waiting on two dependent loads per entry); the
// order of the FMAs, and so the result, is that of the plain loop.
__device__ __forceinline__ double ell_gradt_sum(const int32_t* __restrict__ ekey,
                                                const double* __restrict__ ecoef, int64_t n_ell,
                                                int64_t nmk, const double* __restrict__ t,
                                                int64_t idx, int L) {
  double acc = 0.0;
  int p = 0;
  for (; p + 4 <= L; p += 4, idx += 128) {
    int64_t k[4];
    double c0[4], c1[4], c2[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      k[u] = ekey[idx + 32 * u] >> 6;
      c0[u] = ecoef[idx + 32 * u];
      c1[u] = ecoef[n_ell + idx + 32 * u];
      c2[u] = ecoef[2 * n_ell + idx + 32 * u];
    }
    double t0[4], t1[4], t2[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      t0[u] = t[k[u]];
      t1[u] = t[nmk + k[u]];
      t2[u] = t[2 * nmk + k[u]];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      acc = fma(c0[u], t0[u], acc);
      acc = fma(c1[u], t1[u], acc);
      acc = fma(c2[u], t2[u], acc);
    }
  }
  for (; p < L; ++p, idx += 32) {
    const int64_t k = ekey[idx] >> 6;
    acc = fma(ecoef[idx], t[k], acc);
    acc = fma(ecoef[n_ell + idx], t[nmk + k], acc);
    acc = fma(ecoef[2 * n_ell + idx], t[2 * nmk + k], acc);
  }
  return acc;
}

// The same sum from the FP32 copies of the coefficients and of t, with FP32
// FMAs in the same order (the FP32 Arnoldi cycles round the Schur product to
// FP32; GB300 runs FP64 FMAs at about 1/58 of the FP32 rate).
__device__ __forceinline__ float ell_gradt_sum_f32(const int32_t* __restrict__ ekey,
                                                   const float* __restrict__ ecoef,
                                                   int64_t n_ell, int64_t nmk,
                                                   const float* __restrict__ t, int64_t idx,
                                                   int L) {
  float acc = 0.f;
  int p = 0;
  for (; p + 4 <= L; p += 4, idx += 128) {
    int64_t k[4];
    float c0[4], c1[4], c2[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      k[u] = ekey[idx + 32 * u] >> 6;
      c0[u] = ecoef[idx + 32 * u];
      c1[u] = ecoef[n_ell + idx + 32 * u];
      c2[u] = ecoef[2 * n_ell + idx + 32 * u];
    }
    float t0[4], t1[4], t2[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      t0[u] = t[k[u]];
      t1[u] = t[nmk + k[u]];
      t2[u] = t[2 * nmk + k[u]];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      acc = fmaf(c0[u], t0[u], acc);
      acc = fmaf(c1[u], t1[u], acc);
      acc = fmaf(c2[u], t2[u], acc);
    }
  }
  for (; p < L; ++p, idx += 32) {
    const int64_t k = ekey[idx] >> 6;
    acc = fmaf(ecoef[idx], t[k], acc);
    acc = fmaf(ecoef[n_ell + idx], t[nmk + k], acc);
    acc = fmaf(ecoef[2 * n_ell + idx], t[2 * nmk + k], acc);
  }
  return acc;
}

__device__ __forceinline__ float ell_combine_f32(float v) {
#pragma unroll
  for (int o = 1; o < kEllLanes; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Programmatic dependent launch: a kernel launched with launch_pdl may be
// scheduled while its predecessor in the stream is still finishing, and
// pdl_wait() (first statement of such a kernel) blocks until that
// predecessor has completed and its memory is visible; pdl_trigger() lets the
// next kernel be scheduled once every block of this one has started.  This
// hides the launch latency between the short dependent kernels of a V-cycle.
// Without the launch attribute both instructions have no effect.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}
template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  (void)cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);   // errors: last error
}

inline int div_up(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Solution coefficients of one FGMRES cycle, passed to the update kernel by
// value (kernel parameters need no host-to-device copy).
struct CoefF64 {
  double v[kMaxRestart + 1];
};
struct CoefDS {
  float2 v[kMaxRestart + 1];
};

// Givens state of one FP32 Arnoldi cycle run as a graph (doubles): H
// [(kMaxRestart + 1) x kMaxRestart, row-major as the host's], cs, sn, g, rn,
// the residual history of the cycle, and scalars.
struct GState {
  static constexpr int R = kMaxRestart;
  static constexpr int kH = 0, kCS = (R + 1) * R, kSN = kCS + R, kG = kSN + R, kRN = kG + R + 1,
                       kHist = kRN + R + 1, kSc = kHist + R, kSize = kSc + 16;
  // scalars: bnorm, rtol, cycle_stop, rmax (iterations allowed), jused,
  // breakdown flag, non-finite flag
  static constexpr int sBnorm = 0, sRtol = 1, sStop = 2, sRmax = 3, sJused = 4, sBreak = 5,
                       sNan = 6;
};

// Device address of a place in the mapped host mirror host_red (kernels write
// small results there; the host reads them after synchronising the stream).
inline double* hmirror(ibm_ctx* c, const double* hp) {
  return c->host_red_dev + (hp - c->host_red);
}

}  // namespace ibm
