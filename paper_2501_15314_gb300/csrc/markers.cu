// Lagrangian-marker transfer operators (Sec. 2.3): Roma's discrete delta
// (Eq. (delta)), interpolation R^T (Eq. (interpolation)), regularisation R
// (Eq. (regularization)) and the Schur-complement terms B = R^T G and
// B^T = G^T R of Eq. (Saddle), all matrix-free.
//
// Per marker and axis e only two tap bases exist: bf (positions i h, used by
// the component normal to e) and bc (positions (i+1/2) h, used by the other
// two components), each with three 1-D weights.  The cell footprint of
// G^T R e_{k,d} is 4 x 3 x 3 cells; the union over the three components is a
// 4 x 4 x 4 box with origin org.  A cell-sorted list of (marker, box slot)
// entries, each with its three G^T R coefficients, lets every shell cell (and
// every shell face) gather its markers in a fixed order: the spreads are
// deterministic and use no atomics.  The list is built once per marker set by
// a counting sort (atomics only in the counting, followed by a per-segment
// sort so that the final order does not depend on scheduling).
#include "ds.cuh"
#include "ibm_internal.cuh"

namespace ibm {

namespace {

constexpr int TPB = 256;

// Eq. (delta) times the cell width (phi) and its derivative d phi / dr
// (differentiated branch by branch; continuous, with value -sign(r) at
// |r| = 1/2 and 0 at |r| = 3/2), r in cell widths.  Both come from one
// reciprocal square root R = 1/sqrt(A) of the branch's A = 1 - 3 s^2: the
// square root is A R and the derivative's quotient s / sqrt(A) is s R (one
// FP64 rsqrt in place of a square root and a division).
struct RomaVal {
  double phi, dphi;
};

__device__ __forceinline__ RomaVal roma(double r) {
  const double a = fabs(r);
  if (a <= 0.5) {
    const double A = 1.0 - 3.0 * r * r;
    const double R = rsqrt(A);
    return {(1.0 + A * R) * (1.0 / 3.0), -r * R};
  }
  if (a < 1.5) {
    const double q = 1.0 - a;
    const double A = 1.0 - 3.0 * q * q;
    const double R = rsqrt(A);
    const double v = -0.5 * (1.0 + q * R);
    return {(5.0 - 3.0 * a - A * R) * (1.0 / 6.0), r > 0.0 ? v : -v};
  }
  return {0.0, 0.0};
}

struct MkView {
  int64_t n;
  const int32_t* bf;
  const int32_t* bc;
  const int32_t* org;
  const double* wf;
  const double* wc;
  const double* cw;
};

MkView view(const MarkerData& m) { return MkView{m.n, m.bf, m.bc, m.org, m.wf, m.wc, m.cw}; }

__global__ void k_marker_setup(Dims d, double inv_h, int64_t n, const double* __restrict__ X,
                               int32_t* bf, int32_t* bc, int32_t* org, double* wf, double* wc,
                               double* cw, double* dwf, double* dwc, float* wc32, float* cw32,
                               int32_t* err) {
  // one thread per (axis, marker): the three axes' Roma weights are
  // independent, and three times the threads hide the FP64 latency better
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= 3 * n) return;
  const int e = (int)(t / n);
  const int64_t k = t - (int64_t)e * n;
  const int ncell_e = e == 0 ? d.nx : (e == 1 ? d.ny : d.nz);
  bool bad = false;
  {
    const double s = X[e * n + k] * inv_h;
    const double fs = floor(s + 0.5);
    const double fc = floor(s);
    // guard the conversions against non-finite or huge inputs
    if (!(fs > -1e9 && fs < 1e9 && fc > -1e9 && fc < 1e9)) {
      bad = true;
      bf[e * n + k] = 1; bc[e * n + k] = 0; org[e * n + k] = 0;
      for (int q = 0; q < 3; ++q) {
        wf[(e * 3 + q) * n + k] = 0.0; wc[(e * 3 + q) * n + k] = 0.0;
        dwf[(e * 3 + q) * n + k] = 0.0; dwc[(e * 3 + q) * n + k] = 0.0;
      }
      for (int q = 0; q < 4; ++q) cw[(e * 4 + q) * n + k] = 0.0;
      for (int q = 0; q < 3; ++q) wc32[(e * 3 + q) * n + k] = 0.f;
      for (int q = 0; q < 4; ++q) cw32[(e * 4 + q) * n + k] = 0.f;
      atomicOr(err, 1);
      return;
    }
    const int b_f = (int)fs - 1;   // face taps b_f .. b_f+2 at positions i h
    const int b_c = (int)fc - 1;   // centre taps b_c .. b_c+2 at (i+1/2) h
    if (b_f < 1 || b_f + 2 > ncell_e - 1) bad = true;
    if (b_c < 0 || b_c + 2 > ncell_e - 1) bad = true;
    bf[e * n + k] = b_f;
    bc[e * n + k] = b_c;
    org[e * n + k] = min(b_f - 1, b_c);
    double W[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const RomaVal vf = roma((double)(b_f + q) - s);
      const RomaVal vc = roma((double)(b_c + q) + 0.5 - s);
      W[q] = vf.phi;
      wf[(e * 3 + q) * n + k] = vf.phi;
      wc[(e * 3 + q) * n + k] = vc.phi;
      dwf[(e * 3 + q) * n + k] = vf.dphi;
      dwc[(e * 3 + q) * n + k] = vc.dphi;
      wc32[(e * 3 + q) * n + k] = (float)vc.phi;
    }
    // cell b_f - 1 + q lies between faces b_f - 1 + q and b_f + q
    const double C[4] = {(0.0 - W[0]) * inv_h, (W[0] - W[1]) * inv_h, (W[1] - W[2]) * inv_h,
                         (W[2] - 0.0) * inv_h};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      cw[(e * 4 + q) * n + k] = C[q];
      cw32[(e * 4 + q) * n + k] = (float)C[q];
    }
  }
  if (bad) atomicOr(err, 1);
}

__device__ __forceinline__ int64_t cell_of(Dims d, int i, int j, int k) {
  return ((int64_t)k * d.ny + j) * d.nx + i;
}

__global__ void k_count(Dims d, MkView mk, int32_t* count) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= mk.n * 64) return;
  const int64_t k = t >> 6;
  const int s = (int)(t & 63);
  const int i = mk.org[k] + (s & 3), j = mk.org[mk.n + k] + ((s >> 2) & 3),
            l = mk.org[2 * mk.n + k] + (s >> 4);
  atomicAdd(count + cell_of(d, i, j, l), 1);
}

// Places each (marker, slot) pair in its cell's segment: the cell's count
// (left by k_count) is taken down by one per pair, and the value before the
// decrement gives a free position; the counts end at zero.  The order within
// a segment depends on the atomics' scheduling until k_sort_segments.
__global__ void k_fill(Dims d, MkView mk, const int32_t* __restrict__ start, int32_t* count,
                       int32_t* key) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= mk.n * 64) return;
  const int64_t k = t >> 6;
  const int s = (int)(t & 63);
  const int i = mk.org[k] + (s & 3), j = mk.org[mk.n + k] + ((s >> 2) & 3),
            l = mk.org[2 * mk.n + k] + (s >> 4);
  const int64_t c = cell_of(d, i, j, l);
  const int32_t pos = start[c] + atomicSub(count + c, 1) - 1;
  key[pos] = (int32_t)(k * 64 + s);
}

// Sorts each shell cell's segment (one warp per segment): the keys are
// distinct, so a key's place is the number of smaller keys in the segment;
// segments of up to 64 keys are ranked in registers (two keys per lane),
// longer ones by an insertion sort in lane 0.  Makes the entry order
// independent of the atomics' scheduling.
__global__ void k_sort_segments(int64_t n_shell, const int32_t* __restrict__ off, int32_t* key) {
  const int64_t q = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (q >= n_shell) return;   // whole warps leave together
  const int32_t a = off[q], L = off[q + 1] - off[q];
  if (L <= 1) return;
  if (L <= 64) {
    const int32_t k0 = lane < L ? key[a + lane] : 0x7fffffff;
    const int32_t k1 = lane + 32 < L ? key[a + 32 + lane] : 0x7fffffff;
    int r0 = 0, r1 = 0;
    for (int j = 0; j < L; ++j) {
      const int32_t kj = __shfl_sync(0xffffffffu, j < 32 ? k0 : k1, j & 31);
      r0 += kj < k0;
      r1 += kj < k1;
    }
    __syncwarp();
    if (lane < L) key[a + r0] = k0;
    if (lane + 32 < L) key[a + r1] = k1;
    return;
  }
  if (lane != 0) return;
  for (int32_t x = a + 1; x < a + L; ++x) {
    const int32_t v = key[x];
    int32_t y = x - 1;
    while (y >= a && key[y] > v) { key[y + 1] = key[y]; --y; }
    key[y + 1] = v;
  }
}

// Coefficients of G^T R e_{k,d} (d = 0, 1, 2) at global cell g: along d the
// G^T-weighted face taps cw (cell i lies between faces i and i+1), along the
// other two axes the centre-tap weights; zero outside the 4 x 3 x 3
// footprint.  Each axis's two factors are loaded once; coef_d = f_d P_d
// with f_d the cw factor along d and P_d the product of the centre weights
// along the other two axes (three pair products shared by the six weights:
// nine FP64 multiplications per entry, the FP64 pipe being this kernel's
// bound).
//
// With them the spread weights of the same entry: the weight of F_{k,d} at
// the cell's lower d-face, the face-tap weight wf along d times the same
// P_d, and in bit d whether that face lies inside the support.
__device__ __forceinline__ void gtr_coefs(const MkView& mk, int64_t k, const int g[3],
                                          double (&coef)[3], double (&sw)[3], int& in) {
  double fw[3], fc[3], ff[3];
  bool inw[3], inf[3];
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const int b_f = mk.bf[e * mk.n + k];
    const int qf = g[e] - (b_f - 1);
    fc[e] = (qf >= 0 && qf <= 3) ? mk.cw[(e * 4 + qf) * mk.n + k] : 0.0;
    inf[e] = qf >= 1 && qf <= 3;   // the face g[e] is face tap qf - 1 of 0..2
    ff[e] = inf[e] ? mk.wf[(e * 3 + qf - 1) * mk.n + k] : 0.0;
    const int qc = g[e] - mk.bc[e * mk.n + k];
    inw[e] = qc >= 0 && qc <= 2;
    fw[e] = inw[e] ? mk.wc[(e * 3 + qc) * mk.n + k] : 0.0;
  }
  const double p12 = fw[1] * fw[2], p02 = fw[0] * fw[2], p01 = fw[0] * fw[1];
  coef[0] = fc[0] * p12;
  coef[1] = fc[1] * p02;
  coef[2] = fc[2] * p01;
  sw[0] = ff[0] * p12;
  sw[1] = ff[1] * p02;
  sw[2] = ff[2] * p01;
  in = (inf[0] && inw[1] && inw[2] ? 1 : 0) | (inw[0] && inf[1] && inw[2] ? 2 : 0) |
       (inw[0] && inw[1] && inf[2] ? 4 : 0);
}

// FP32 values widened to FP64 with integer operations (the conversion
// instruction runs on the FP64 pipe, which this kernel also needs for its
// FMAs); FP64 values pass through.
__device__ __forceinline__ double widen(float x) { return f2d_exact(x); }
__device__ __forceinline__ double widen(double x) { return x; }

// t[d][k] = scale * (R^T G v)_{k,d} using the tensor-product form of the
// footprint: sum_a cw_d[a] sum_b w_e1[b] sum_c w_e2[c] v.  Four consecutive
// threads hold a = 0..3 of one (marker, component) and combine in a fixed
// order with warp shuffles.
template <typename TV>
__global__ void k_marker_grad_interp(Dims d, MkView mk, const TV* __restrict__ v,
                                     double scale, double* __restrict__ t) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nt = 12 * mk.n;
  double part = 0.0;
  int dc = 0;
  int64_t k = 0;
  if (tid < nt) {
    const int64_t pk = tid >> 2;
    const int a = (int)(tid & 3);
    dc = (int)(pk / mk.n);
    k = pk - dc * mk.n;
    const int e1 = dc == 0 ? 1 : 0;
    const int e2 = dc == 2 ? 1 : 2;
    int g[3];
    g[dc] = mk.bf[dc * mk.n + k] - 1 + a;
    const int b1 = mk.bc[e1 * mk.n + k], b2 = mk.bc[e2 * mk.n + k];
    const int64_t sy = d.nx, sz = (int64_t)d.nx * d.ny;
    double acc1 = 0.0;
#pragma unroll
    for (int q1 = 0; q1 < 3; ++q1) {
      g[e1] = b1 + q1;
      double acc2 = 0.0;
#pragma unroll
      for (int q2 = 0; q2 < 3; ++q2) {
        g[e2] = b2 + q2;
        const int64_t cell = g[0] + g[1] * sy + (int64_t)g[2] * sz;
        acc2 = fma(mk.wc[(e2 * 3 + q2) * mk.n + k], widen(__ldg(v + cell)), acc2);
      }
      acc1 = fma(mk.wc[(e1 * 3 + q1) * mk.n + k], acc2, acc1);
    }
    part = mk.cw[(dc * 4 + a) * mk.n + k] * acc1;
  }
  const int lane = threadIdx.x & 31;
  const int base = lane & ~3;
  const double p0 = __shfl_sync(0xffffffffu, part, base);
  const double p1 = __shfl_sync(0xffffffffu, part, base + 1);
  const double p2 = __shfl_sync(0xffffffffu, part, base + 2);
  const double p3 = __shfl_sync(0xffffffffu, part, base + 3);
  if (tid < nt && (lane & 3) == 0) t[dc * mk.n + k] = scale * ((p0 + p1) + (p2 + p3));
}

// The same for FP32 v with FP32 weights and FP32 FMAs (t32 only).
__global__ void k_marker_grad_interp_f32(Dims d, MkView mk, const float* __restrict__ wc32,
                                         const float* __restrict__ cw32,
                                         const float* __restrict__ v, float scale,
                                         float* __restrict__ t32) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nt = 12 * mk.n;
  float part = 0.f;
  int dc = 0;
  int64_t k = 0;
  if (tid < nt) {
    const int64_t pk = tid >> 2;
    const int a = (int)(tid & 3);
    dc = (int)(pk / mk.n);
    k = pk - dc * mk.n;
    const int e1 = dc == 0 ? 1 : 0;
    const int e2 = dc == 2 ? 1 : 2;
    int g[3];
    g[dc] = mk.bf[dc * mk.n + k] - 1 + a;
    const int b1 = mk.bc[e1 * mk.n + k], b2 = mk.bc[e2 * mk.n + k];
    const int64_t sy = d.nx, sz = (int64_t)d.nx * d.ny;
    float acc1 = 0.f;
#pragma unroll
    for (int q1 = 0; q1 < 3; ++q1) {
      g[e1] = b1 + q1;
      float acc2 = 0.f;
#pragma unroll
      for (int q2 = 0; q2 < 3; ++q2) {
        g[e2] = b2 + q2;
        const int64_t cell = g[0] + g[1] * sy + (int64_t)g[2] * sz;
        acc2 = fmaf(wc32[(e2 * 3 + q2) * mk.n + k], __ldg(v + cell), acc2);
      }
      acc1 = fmaf(wc32[(e1 * 3 + q1) * mk.n + k], acc2, acc1);
    }
    part = cw32[(dc * 4 + a) * mk.n + k] * acc1;
  }
  const int lane = threadIdx.x & 31;
  const int base = lane & ~3;
  const float p0 = __shfl_sync(0xffffffffu, part, base);
  const float p1 = __shfl_sync(0xffffffffu, part, base + 1);
  const float p2 = __shfl_sync(0xffffffffu, part, base + 2);
  const float p3 = __shfl_sync(0xffffffffu, part, base + 3);
  if (tid < nt && (lane & 3) == 0) t32[dc * mk.n + k] = scale * ((p0 + p1) + (p2 + p3));
}

// Order of the shell cells in the interleaved layout: each block sorts one
// window of 1024 consecutive shell cells by (entry count descending, index
// ascending) with a bitonic network in shared memory -- deterministic, and
// a window is 32 whole groups, so each group gets cells of nearly equal
// counts.  perm[q'] = q (position q' of the layout holds shell cell q),
// ell_cell[q'] = its cell.
constexpr int kOrderWin = 1024;
__global__ void __launch_bounds__(kOrderWin) k_ell_order(int64_t n_shell,
                                                         const int32_t* __restrict__ off,
                                                         const int32_t* __restrict__ shell_cell,
                                                         int32_t* perm, int32_t* ell_cell) {
  __shared__ unsigned long long key[kOrderWin];
  const int t = threadIdx.x;
  const int64_t q = (int64_t)blockIdx.x * kOrderWin + t;
  key[t] = q < n_shell ? ((unsigned long long)(0x7fffffff - (off[q + 1] - off[q])) << 32) |
                             (unsigned long long)(q - (int64_t)blockIdx.x * kOrderWin)
                       : ~0ull;
  __syncthreads();
  for (int k = 2; k <= kOrderWin; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      const int p = t ^ j;
      if (p > t) {
        const unsigned long long a = key[t], b = key[p];
        const bool up = (t & k) == 0;
        if (up ? (a > b) : (a < b)) {
          key[t] = b;
          key[p] = a;
        }
      }
      __syncthreads();
    }
  }
  if (q < n_shell) {
    const int64_t src = (int64_t)blockIdx.x * kOrderWin + (int64_t)(key[t] & 0xffffffffu);
    perm[q] = (int32_t)src;
    ell_cell[q] = shell_cell[src];
  }
}

// Group lengths of the interleaved layout.  A group is one warp: kEllCells
// shell cells (layout order) with kEllLanes lanes each; lane l of the group
// holds the entries p = kEllLanes r + (l % kEllLanes), r = 0, 1, ..., of cell
// l / kEllLanes at slot base[w] + 32 r + l.  len[w] = rounds of group w (the
// longest cell's count over kEllLanes, rounded up), cnt[w] = 32 * len[w].
__global__ void k_ell_len(int64_t n_shell, const int32_t* __restrict__ off,
                          const int32_t* __restrict__ perm, int32_t* len, int32_t* cnt) {
  const int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t ng = (n_shell + kEllCells - 1) / kEllCells;
  if (w >= ng) return;
  int32_t L = 0;
  for (int64_t q = kEllCells * w; q < min(kEllCells * w + kEllCells, n_shell); ++q) {
    const int32_t r = perm[q];
    L = max(L, off[r + 1] - off[r]);
  }
  const int32_t rounds = (L + kEllLanes - 1) / kEllLanes;
  len[w] = rounds;
  cnt[w] = 32 * rounds;
}

// Fills the interleaved layout with keys and G^T R coefficients (zero padding).
// One warp per group: round r, lane l fills slot base[w] + 32 r + l, entry
// p = kEllLanes r + l % kEllLanes of the group's cell l / kEllLanes (zeros
// past the cell's count or for a cell past the last shell cell).
__global__ void k_ell_fill(MkView mk, int64_t n_shell, const int32_t* __restrict__ off,
                           const int32_t* __restrict__ key, const int32_t* __restrict__ base,
                           const int32_t* __restrict__ len, const int32_t* __restrict__ perm,
                           const int32_t* __restrict__ ell_cell, Dims d, int64_t n_ell,
                           int32_t* ekey, double* ecoef, float* ecoef32, double* esw,
                           uint8_t* eany) {
  const int64_t tq = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t w = tq >> 5;
  if (w >= ell_groups(n_shell)) return;
  const int lane = (int)(tq & 31);
  const int64_t q = w * kEllCells + lane / kEllLanes;
  const bool live = q < n_shell;
  int32_t a = 0, nseg = 0;
  int g[3] = {0, 0, 0};
  if (live) {
    const int32_t r = perm[q];
    a = off[r];
    nseg = off[r + 1] - a;
    const int64_t c = ell_cell[q];
    g[0] = (int)(c % d.nx);
    g[1] = (int)((c / d.nx) % d.ny);
    g[2] = (int)(c / ((int64_t)d.nx * d.ny));
  }
  const int32_t rounds = len[w];
  int any = 0;
  for (int32_t rr = 0; rr < rounds; ++rr) {
    const int64_t dst = base[w] + (int64_t)rr * 32 + lane;
    const int p = kEllLanes * rr + lane % kEllLanes;
    if (live && p < nseg) {
      const int32_t kk = key[a + p];
      ekey[dst] = kk;
      const int64_t k = kk >> 6;
      double cf[3], sw[3];
      int in;
      gtr_coefs(mk, k, g, cf, sw, in);
      any |= in;
#pragma unroll
      for (int dc = 0; dc < 3; ++dc) {
        ecoef[dc * n_ell + dst] = cf[dc];
        // the FP32 copy is the leading part (integer operations; a
        // conversion would run on the FP64 pipe)
        ecoef32[dc * n_ell + dst] = split_exact(cf[dc]).hi;
        esw[dc * n_ell + dst] = sw[dc];
      }
    } else {
      ekey[dst] = 0;
#pragma unroll
      for (int dc = 0; dc < 3; ++dc) {
        ecoef[dc * n_ell + dst] = 0.0;
        ecoef32[dc * n_ell + dst] = 0.f;
        esw[dc * n_ell + dst] = 0.0;
      }
    }
  }
#pragma unroll
  for (int o = 1; o < kEllLanes; o <<= 1) any |= __shfl_xor_sync(0xffffffffu, any, o);
  if (live && lane % kEllLanes == 0) eany[q] = (uint8_t)any;
}

// u at the shell cells' lower faces += scale * (R F) (set: = scale * (R F)),
// faces outside every support left as they are: the spread through the
// interleaved layout, kEllLanes lanes per cell (each its share of the
// entries, summed by shuffles in a fixed order), the three components at
// once.  One warp per group: launch 32 threads per group.
__global__ void k_shell_spread_ell(Dims d, int64_t n_shell, const int32_t* __restrict__ ell_cell,
                                   const int32_t* __restrict__ base,
                                   const int32_t* __restrict__ len,
                                   const int32_t* __restrict__ ekey,
                                   const double* __restrict__ esw,
                                   const uint8_t* __restrict__ eany, int64_t n_ell, int64_t nmk,
                                   const double* __restrict__ F, double scale, int set,
                                   double* __restrict__ u) {
  const int64_t tq = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t g = tq >> 5;
  const int lane = (int)(tq & 31);
  const int64_t q = g * kEllCells + lane / kEllLanes;
  const bool live = g < ell_groups(n_shell) && q < n_shell;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
  if (live) {
    int64_t idx = base[g] + lane;
    const int L = len[g];
    int p = 0;
    for (; p + 4 <= L; p += 4, idx += 128) {
      int64_t k[4];
      double w0[4], w1[4], w2[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        k[v] = ekey[idx + 32 * v] >> 6;
        w0[v] = esw[idx + 32 * v];
        w1[v] = esw[n_ell + idx + 32 * v];
        w2[v] = esw[2 * n_ell + idx + 32 * v];
      }
      double f0[4], f1[4], f2[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        f0[v] = F[k[v]];
        f1[v] = F[nmk + k[v]];
        f2[v] = F[2 * nmk + k[v]];
      }
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        a0 = fma(w0[v], f0[v], a0);
        a1 = fma(w1[v], f1[v], a1);
        a2 = fma(w2[v], f2[v], a2);
      }
    }
    for (; p < L; ++p, idx += 32) {
      const int64_t k = ekey[idx] >> 6;
      a0 = fma(esw[idx], F[k], a0);
      a1 = fma(esw[n_ell + idx], F[nmk + k], a1);
      a2 = fma(esw[2 * n_ell + idx], F[2 * nmk + k], a2);
    }
  }
  a0 = ell_combine(a0);
  a1 = ell_combine(a1);
  a2 = ell_combine(a2);
  if (!live || lane % kEllLanes != 0) return;
  const int64_t c = ell_cell[q];
  const int ci = (int)(c % d.nx);
  const int cj = (int)((c / d.nx) % d.ny);
  const int ck = (int)(c / ((int64_t)d.nx * d.ny));
  const int any = eany[q];
  const FaceDims fd = face_dims(d);
  const double acc[3] = {a0, a1, a2};
#pragma unroll
  for (int dc = 0; dc < 3; ++dc) {
    if (!(any & (1 << dc))) continue;
    const int64_t foff = dc == 0 ? 0 : (dc == 1 ? fd.nfx : fd.nfx + fd.nfy);
    const int64_t sy = d.nx + (dc == 0 ? 1 : 0);
    const int64_t sz = sy * (d.ny + (dc == 1 ? 1 : 0));
    const int64_t f = foff + ck * sz + cj * sy + ci;
    u[f] = set ? scale * acc[dc] : fma(scale, acc[dc], u[f]);
  }
}

// out[c] += scale * sum over the entries of shell cell c of sum_d coef_d
// t[d][k]; coalesced loads through the interleaved layout, kEllLanes lanes
// per cell (each its own share of the entries), their sums combined in a
// fixed order.  One warp per group: launch 32 threads per group.
__global__ void k_shell_gradt(int64_t n_shell, const int32_t* __restrict__ shell_cell,
                              const int32_t* __restrict__ base, const int32_t* __restrict__ len,
                              const int32_t* __restrict__ ekey, const double* __restrict__ ecoef,
                              int64_t n_ell, int64_t nmk, const double* __restrict__ t,
                              double scale, double* __restrict__ out) {
  const int64_t tq = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t w = tq >> 5;
  const int lane = (int)(tq & 31);
  const int64_t q = w * kEllCells + lane / kEllLanes;
  const bool live = w < ell_groups(n_shell) && q < n_shell;
  double acc = live ? ell_gradt_sum(ekey, ecoef, n_ell, nmk, t, base[w] + lane, len[w]) : 0.0;
  acc = ell_combine(acc);
  if (live && lane % kEllLanes == 0) {
    const int64_t c = shell_cell[q];
    out[c] = fma(scale, acc, out[c]);
  }
}

// U[d][k] = sum over the 27 taps of component d of w * u_d  (R^T u)
__global__ void k_interp(Dims d, MkView mk, const double* __restrict__ u, double* __restrict__ U) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (tid >= 3 * mk.n) return;
  const int dc = (int)(tid / mk.n);
  const int64_t k = tid - dc * mk.n;
  const FaceDims fd = face_dims(d);
  const int64_t off = dc == 0 ? 0 : (dc == 1 ? fd.nfx : fd.nfx + fd.nfy);
  const int sx = 1;
  const int64_t sy = d.nx + (dc == 0 ? 1 : 0);
  const int64_t sz = sy * (d.ny + (dc == 1 ? 1 : 0));
  int b[3];
  const double* w[3];
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    b[e] = (e == dc) ? mk.bf[e * mk.n + k] : mk.bc[e * mk.n + k];
    w[e] = (e == dc) ? (mk.wf + e * 3 * mk.n + k) : (mk.wc + e * 3 * mk.n + k);
  }
  double acc = 0.0;
  for (int c2 = 0; c2 < 3; ++c2) {
    double acc1 = 0.0;
    for (int c1 = 0; c1 < 3; ++c1) {
      double acc0 = 0.0;
      const int64_t base = off + (int64_t)(b[2] + c2) * sz + (int64_t)(b[1] + c1) * sy + b[0];
      for (int c0 = 0; c0 < 3; ++c0) acc0 = fma(w[0][c0 * mk.n], __ldg(u + base + c0 * sx), acc0);
      acc1 = fma(w[1][c1 * mk.n], acc0, acc1);
    }
    acc = fma(w[2][c2 * mk.n], acc1, acc);
  }
  U[dc * mk.n + k] = acc;
}

// Face spread R F on the shell: every tap face of a marker is the lower face
// (along its own normal) of a cell of the marker's box, so one thread per
// (shell cell, component) owns that face and gathers its markers in order.
// spread_face: the gathered value (any = false when no tap of the cell's
// markers lands on that face) and the face's index in the packed vector.
__device__ __forceinline__ double spread_face(Dims d, const MkView& mk, int64_t n_shell,
                                              const int32_t* __restrict__ shell_cell,
                                              const int32_t* __restrict__ off,
                                              const int32_t* __restrict__ key,
                                              const double* __restrict__ F, int64_t tid,
                                              bool& any, int64_t& f) {
  const int dc = (int)(tid / n_shell);
  const int64_t q = tid - dc * n_shell;
  const int64_t c = shell_cell[q];
  const int ci = (int)(c % d.nx);
  const int cj = (int)((c / d.nx) % d.ny);
  const int ck = (int)(c / ((int64_t)d.nx * d.ny));
  const int g[3] = {ci, cj, ck};
  const int32_t a = off[q], b = off[q + 1];
  double acc = 0.0;
  any = false;
  for (int32_t x = a; x < b; ++x) {
    const int64_t k = key[x] >> 6;
    double w = 1.0;
    bool in = true;
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      const int base = (e == dc) ? mk.bf[e * mk.n + k] : mk.bc[e * mk.n + k];
      const int r = g[e] - base;
      if (r < 0 || r > 2) { in = false; break; }
      w *= (e == dc) ? mk.wf[(e * 3 + r) * mk.n + k] : mk.wc[(e * 3 + r) * mk.n + k];
    }
    if (in) { acc = fma(w, F[dc * mk.n + k], acc); any = true; }
  }
  const FaceDims fd = face_dims(d);
  const int64_t foff = dc == 0 ? 0 : (dc == 1 ? fd.nfx : fd.nfx + fd.nfy);
  const int64_t sy = d.nx + (dc == 0 ? 1 : 0);
  const int64_t sz = sy * (d.ny + (dc == 1 ? 1 : 0));
  f = foff + ck * sz + cj * sy + ci;
  return acc;
}

// L1 norms of the spread forces R A and R B over the faces (every face of the
// support is owned by one (shell cell, component) task): per block the sums
// of |(R A)_f| and |(R B)_f| over its tasks (fixed grid and order),
// part[2 blk], part[2 blk + 1].
constexpr int kSpreadAsumBlocks = 256;
__global__ void __launch_bounds__(TPB) k_shell_spread_asum2(
    Dims d, MkView mk, int64_t n_shell, const int32_t* __restrict__ shell_cell,
    const int32_t* __restrict__ off, const int32_t* __restrict__ key,
    const double* __restrict__ A, const double* __restrict__ B, double* __restrict__ part) {
  double sa = 0.0, sb = 0.0;
  for (int64_t tid = blockIdx.x * (int64_t)TPB + threadIdx.x; tid < 3 * n_shell;
       tid += (int64_t)kSpreadAsumBlocks * TPB) {
    bool any;
    int64_t f;
    sa += fabs(spread_face(d, mk, n_shell, shell_cell, off, key, A, tid, any, f));
    sb += fabs(spread_face(d, mk, n_shell, shell_cell, off, key, B, tid, any, f));
  }
  __shared__ double sh[2][TPB];
  sh[0][threadIdx.x] = sa;
  sh[1][threadIdx.x] = sb;
  __syncthreads();
  for (int w = TPB / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = sh[0][0];
    part[2 * blockIdx.x + 1] = sh[1][0];
  }
}

// ---- exclusive scan of int32 (three phases, 4096 elements per block) ----
constexpr int SCAN_T = 1024, SCAN_E = 4;

__device__ int32_t block_excl_scan(int32_t v, int32_t* sh, int32_t* total) {
  // warp-level inclusive scan then scan of warp totals
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int32_t w = sh[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    sh[lane] = w;
  }
  __syncthreads();
  const int32_t wprefix = wid > 0 ? sh[wid - 1] : 0;
  if (total) *total = sh[31];
  return wprefix + x - v;
}

// The same for pairs (.x and .y scanned independently).
__device__ int2 block_excl_scan2(int2 v, int2* sh, int2* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int2 x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int yx = __shfl_up_sync(0xffffffffu, x.x, o);
    const int yy = __shfl_up_sync(0xffffffffu, x.y, o);
    if (lane >= o) {
      x.x += yx;
      x.y += yy;
    }
  }
  if (lane == 31) sh[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int2 w = sh[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int yx = __shfl_up_sync(0xffffffffu, w.x, o);
      const int yy = __shfl_up_sync(0xffffffffu, w.y, o);
      if (lane >= o) {
        w.x += yx;
        w.y += yy;
      }
    }
    sh[lane] = w;
  }
  __syncthreads();
  const int2 wp = wid > 0 ? sh[wid - 1] : make_int2(0, 0);
  if (total) *total = sh[31];
  return make_int2(wp.x + x.x - v.x, wp.y + x.y - v.y);
}

// Shell cells of the marker lists, in two passes over the cell counts (each
// block SCAN_T * SCAN_E cells): k_cell_sums writes each block's (entries,
// shell cells); after the scan of those, k_shell_list writes, for every cell
// with entries, its segment start and its place in the shell list.
__global__ void k_cell_sums(const int32_t* __restrict__ count, int64_t n, int2* __restrict__ sums) {
  __shared__ int2 sh[32];
  const int64_t base = (int64_t)blockIdx.x * SCAN_T * SCAN_E + (int64_t)threadIdx.x * SCAN_E;
  int2 v = make_int2(0, 0);
#pragma unroll
  for (int q = 0; q < SCAN_E; ++q) {
    const int32_t k = (base + q < n) ? count[base + q] : 0;
    v.x += k;
    v.y += k > 0;
  }
  int2 total;
  block_excl_scan2(v, sh, &total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// exclusive scan of the nb block pairs in place (one block); the totals go
// to sums[nb]
__global__ void k_scan_sums2(int2* sums, int64_t nb) {
  __shared__ int2 sh[32];
  __shared__ int2 carry;
  if (threadIdx.x == 0) carry = make_int2(0, 0);
  __syncthreads();
  for (int64_t base = 0; base < nb; base += SCAN_T) {
    const int64_t i = base + threadIdx.x;
    const int2 v = i < nb ? sums[i] : make_int2(0, 0);
    int2 tot;
    const int2 ex = block_excl_scan2(v, sh, &tot);
    const int2 c0 = carry;
    if (i < nb) sums[i] = make_int2(ex.x + c0.x, ex.y + c0.y);
    __syncthreads();
    if (threadIdx.x == 0) carry = make_int2(c0.x + tot.x, c0.y + tot.y);
    __syncthreads();
  }
  if (threadIdx.x == 0) sums[nb] = carry;
}

__global__ void k_shell_list(const int32_t* __restrict__ count, int64_t n,
                             const int2* __restrict__ sums, int32_t* __restrict__ start,
                             int32_t* __restrict__ shell_cell, int32_t* __restrict__ shell_off,
                             int64_t nb) {
  __shared__ int2 sh[32];
  const int64_t base = (int64_t)blockIdx.x * SCAN_T * SCAN_E + (int64_t)threadIdx.x * SCAN_E;
  int32_t k[SCAN_E];
  int2 v = make_int2(0, 0);
#pragma unroll
  for (int q = 0; q < SCAN_E; ++q) {
    k[q] = (base + q < n) ? count[base + q] : 0;
    v.x += k[q];
    v.y += k[q] > 0;
  }
  const int2 ex = block_excl_scan2(v, sh, nullptr);
  const int2 b0 = sums[blockIdx.x];
  int32_t e = b0.x + ex.x, sidx = b0.y + ex.y;
#pragma unroll
  for (int q = 0; q < SCAN_E; ++q) {
    if (k[q] > 0) {
      start[base + q] = e;
      shell_cell[sidx] = (int32_t)(base + q);
      shell_off[sidx] = e;
      ++sidx;
    }
    e += k[q];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) shell_off[sums[nb].y] = sums[nb].x;
}

__global__ void k_scan_blocks(const int32_t* __restrict__ in, int64_t n, int32_t* __restrict__ out,
                              int32_t* __restrict__ block_sums) {
  __shared__ int32_t sh[32];
  const int64_t base = (int64_t)blockIdx.x * SCAN_T * SCAN_E + (int64_t)threadIdx.x * SCAN_E;
  int32_t v[SCAN_E];
  int32_t sum = 0;
#pragma unroll
  for (int q = 0; q < SCAN_E; ++q) {
    v[q] = (base + q < n) ? in[base + q] : 0;
    sum += v[q];
  }
  int32_t total;
  int32_t ex = block_excl_scan(sum, sh, &total);
#pragma unroll
  for (int q = 0; q < SCAN_E; ++q) {
    if (base + q < n) out[base + q] = ex;
    ex += v[q];
  }
  if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

// scans block_sums (nb entries) in place with a single block; writes the grand
// total to *total.
__global__ void k_scan_sums(int32_t* sums, int64_t nb, int32_t* total) {
  __shared__ int32_t sh[32];
  __shared__ int32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < nb; base += SCAN_T) {
    const int64_t i = base + threadIdx.x;
    const int32_t v = i < nb ? sums[i] : 0;
    int32_t tot;
    const int32_t ex = block_excl_scan(v, sh, &tot);
    const int32_t c0 = carry;
    if (i < nb) sums[i] = ex + c0;
    __syncthreads();
    if (threadIdx.x == 0) carry = c0 + tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scan_add(int32_t* out, int64_t n, const int32_t* __restrict__ sums,
                           const int32_t* __restrict__ total) {
  const int64_t base = (int64_t)blockIdx.x * SCAN_T * SCAN_E;
  const int32_t add = sums[blockIdx.x];
  for (int q = threadIdx.x; q < SCAN_T * SCAN_E; q += SCAN_T) {
    const int64_t i = base + q;
    if (i < n) out[i] += add;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = *total;
}

}  // namespace

// out[0..n] = exclusive scan of in[0..n-1] with out[n] = total.
ibm_status exclusive_scan(ibm_ctx* c, const int32_t* in, int32_t* out, int64_t n) {
  const int64_t nb = (n + SCAN_T * SCAN_E - 1) / (SCAN_T * SCAN_E);
  if (nb == 0) {
    launch_zero(out, sizeof(int32_t), c->stream);
    return IBM_OK;
  }
  int32_t* sums = c->scan_tmp;
  int32_t* total = c->scan_tmp + nb;
  count_launch();
  k_scan_blocks<<<(unsigned)nb, SCAN_T, 0, c->stream>>>(in, n, out, sums);
  count_launch();
  k_scan_sums<<<1, SCAN_T, 0, c->stream>>>(sums, nb, total);
  count_launch();
  k_scan_add<<<(unsigned)nb, SCAN_T, 0, c->stream>>>(out, n, sums, total);
  IBM_LAUNCH_CHECK(c);
  return IBM_OK;
}

static ibm_status grow_markers(ibm_ctx* c, int64_t n) {
  MarkerData& m = c->mk;
  if (n <= m.cap) return IBM_OK;
  cudaFree(m.bf); cudaFree(m.bc); cudaFree(m.org); cudaFree(m.wf); cudaFree(m.wc);
  cudaFree(m.cw); cudaFree(m.t); cudaFree(m.t2); cudaFree(m.t32); cudaFree(m.dwf);
  cudaFree(m.dwc); cudaFree(m.wc32); cudaFree(m.cw32);
  cudaFree(m.cg); cudaFree(m.t3);
  m.bf = m.bc = m.org = nullptr;
  m.wf = m.wc = m.cw = m.t = m.t2 = m.dwf = m.dwc = m.cg = m.t3 = nullptr;
  m.t32 = nullptr;
  m.wc32 = m.cw32 = nullptr;
  m.cap = 0;
  const size_t ni = sizeof(int32_t) * 3 * n, nd = sizeof(double) * 9 * n;
  if (cudaMalloc(&m.bf, ni) != cudaSuccess || cudaMalloc(&m.bc, ni) != cudaSuccess ||
      cudaMalloc(&m.org, ni) != cudaSuccess || cudaMalloc(&m.wf, nd) != cudaSuccess ||
      cudaMalloc(&m.wc, nd) != cudaSuccess || cudaMalloc(&m.dwf, nd) != cudaSuccess ||
      cudaMalloc(&m.dwc, nd) != cudaSuccess ||
      cudaMalloc(&m.cw, sizeof(double) * 12 * n) != cudaSuccess ||
      cudaMalloc(&m.t, sizeof(double) * 3 * n) != cudaSuccess ||
      cudaMalloc(&m.t32, sizeof(float) * 3 * n) != cudaSuccess ||
      cudaMalloc(&m.wc32, sizeof(float) * 9 * n) != cudaSuccess ||
      cudaMalloc(&m.cw32, sizeof(float) * 12 * n) != cudaSuccess ||
      cudaMalloc(&m.t2, sizeof(double) * 3 * n) != cudaSuccess ||
      cudaMalloc(&m.t3, sizeof(double) * 3 * n) != cudaSuccess ||
      cudaMalloc(&m.cg, sizeof(double) * 9 * n) != cudaSuccess) {
    cudaGetLastError();
    return set_err(c, IBM_ERR_NOMEM, "marker workspace allocation failed");
  }
  m.cap = n;
  return IBM_OK;
}

static ibm_status grow_entries(ibm_ctx* c, int64_t ne) {
  // shell cells never outnumber entries (each shell cell holds >= 1 entry)
  MarkerData& m = c->mk;
  if (ne <= m.entries_cap && m.entry_key) return IBM_OK;
  cudaFree(m.entry_key); cudaFree(m.shell_cell); cudaFree(m.shell_off); cudaFree(m.ell_base);
  cudaFree(m.ell_len); cudaFree(m.ell_cell); cudaFree(m.ell_any);
  m.entry_key = nullptr; m.shell_cell = nullptr; m.shell_off = nullptr; m.ell_base = nullptr;
  m.ell_len = nullptr; m.ell_cell = nullptr; m.ell_any = nullptr;
  m.entries_cap = 0;
  const int64_t cap = ne > 0 ? ne : 1;
  if (cudaMalloc(&m.entry_key, sizeof(int32_t) * cap) != cudaSuccess ||
      cudaMalloc(&m.ell_base, sizeof(int32_t) * (cap / kEllCells + 2)) != cudaSuccess ||
      cudaMalloc(&m.ell_len, sizeof(int32_t) * (cap / kEllCells + 2)) != cudaSuccess ||
      cudaMalloc(&m.shell_cell, sizeof(int32_t) * cap) != cudaSuccess ||
      cudaMalloc(&m.ell_cell, sizeof(int32_t) * cap) != cudaSuccess ||
      cudaMalloc(&m.ell_any, cap) != cudaSuccess ||
      cudaMalloc(&m.shell_off, sizeof(int32_t) * (cap + 1)) != cudaSuccess) {
    cudaGetLastError();
    return set_err(c, IBM_ERR_NOMEM, "marker entry list allocation failed");
  }
  m.entries_cap = cap;
  return IBM_OK;
}

static ibm_status grow_ell(ibm_ctx* c, int64_t n_ell) {
  MarkerData& m = c->mk;
  if (n_ell <= m.ell_cap && m.ell_key) return IBM_OK;
  cudaFree(m.ell_key);
  cudaFree(m.ell_coef);
  cudaFree(m.ell_coef32);
  cudaFree(m.ell_sw);
  m.ell_key = nullptr;
  m.ell_coef = nullptr;
  m.ell_coef32 = nullptr;
  m.ell_sw = nullptr;
  m.ell_cap = 0;
  const int64_t cap = n_ell > 0 ? n_ell : 1;
  if (cudaMalloc(&m.ell_key, sizeof(int32_t) * cap) != cudaSuccess ||
      cudaMalloc(&m.ell_coef, sizeof(double) * 3 * cap) != cudaSuccess ||
      cudaMalloc(&m.ell_coef32, sizeof(float) * 3 * cap) != cudaSuccess ||
      cudaMalloc(&m.ell_sw, sizeof(double) * 3 * cap) != cudaSuccess) {
    cudaGetLastError();
    return set_err(c, IBM_ERR_NOMEM, "marker gather layout allocation failed");
  }
  m.ell_cap = cap;
  return IBM_OK;
}

ibm_status markers_build(ibm_ctx* c, int64_t n, const double* X) {
  MarkerData& m = c->mk;
  c->markers_set = false;
  m.n = 0;
  m.n_entries = 0;
  m.n_shell = 0;
  if (n == 0) {
    c->markers_set = true;
    return IBM_OK;
  }
  ibm_status st = grow_markers(c, n);
  if (st != IBM_OK) return st;
  cudaStream_t s = c->stream;
  launch_zero(c->dev_flag, sizeof(int32_t), s);
  count_launch();
  k_marker_setup<<<div_up(3 * n, TPB), TPB, 0, s>>>(c->d, 1.0 / c->h, n, X, m.bf, m.bc, m.org,
                                                     m.wf, m.wc, m.cw, m.dwf, m.dwc, m.wc32,
                                                     m.cw32, c->dev_flag);
  IBM_LAUNCH_CHECK(c);
  launch_to_host(c->dev_flag, c->host_flag_dev, sizeof(int32_t), s);
  IBM_LAUNCH_CHECK(c);
  IBM_CUDA(c, cudaStreamSynchronize(s));
  if (c->host_flag[0] != 0)
    return set_err(c, IBM_ERR_MARKER_DOMAIN,
                   "a marker's delta support touches a wall face or leaves the grid");
  m.n = n;
  const MkView mv = view(m);
  // counting sort of (marker, slot) pairs by cell: counts, then one
  // reduction and one scan-and-list pass over the counts for the segment
  // starts and the shell-cell list, then the fill (which takes the counts
  // back to zero) and the per-segment sort
  launch_zero(c->cell_count, sizeof(int32_t) * c->m, s);
  count_launch();
  k_count<<<div_up(n * 64, TPB), TPB, 0, s>>>(c->d, mv, c->cell_count);
  const int64_t nb = (c->m + SCAN_T * SCAN_E - 1) / (SCAN_T * SCAN_E);
  int2* bsum = reinterpret_cast<int2*>(c->scan_tmp);
  count_launch();
  k_cell_sums<<<(unsigned)nb, SCAN_T, 0, s>>>(c->cell_count, c->m, bsum);
  count_launch();
  k_scan_sums2<<<1, SCAN_T, 0, s>>>(bsum, nb);
  launch_to_host(bsum + nb, c->host_flag_dev, sizeof(int2), s);
  IBM_LAUNCH_CHECK(c);
  IBM_CUDA(c, cudaStreamSynchronize(s));
  const int64_t ne = c->host_flag[0], ns = c->host_flag[1];
  st = grow_entries(c, ne);
  if (st != IBM_OK) return st;
  count_launch();
  k_shell_list<<<(unsigned)nb, SCAN_T, 0, s>>>(c->cell_count, c->m, bsum, c->cell_start,
                                               m.shell_cell, m.shell_off, nb);
  count_launch();
  k_fill<<<div_up(n * 64, TPB), TPB, 0, s>>>(c->d, mv, c->cell_start, c->cell_count, m.entry_key);
  count_launch();
  k_sort_segments<<<div_up(32 * ns, TPB), TPB, 0, s>>>(ns, m.shell_off, m.entry_key);
  IBM_LAUNCH_CHECK(c);
  // interleaved layout for the B^T t gather, in the order of ell_cell
  const int64_t ng = ell_groups(ns);
  int32_t* cnt = c->cell_count;   // back at zero after the fill: the group sizes
  int32_t* perm = c->cell_flag;   // scratch: the layout order
  count_launch();
  k_ell_order<<<div_up(ns, kOrderWin), kOrderWin, 0, s>>>(ns, m.shell_off, m.shell_cell, perm,
                                                          m.ell_cell);
  count_launch();
  k_ell_len<<<div_up(ng, TPB), TPB, 0, s>>>(ns, m.shell_off, perm, m.ell_len, cnt);
  IBM_LAUNCH_CHECK(c);
  st = exclusive_scan(c, cnt, m.ell_base, ng);
  if (st != IBM_OK) return st;
  launch_to_host(m.ell_base + ng, c->host_flag_dev, sizeof(int32_t), s);
  IBM_LAUNCH_CHECK(c);
  IBM_CUDA(c, cudaStreamSynchronize(s));
  const int64_t n_ell = c->host_flag[0];
  if ((st = grow_ell(c, n_ell)) != IBM_OK) return st;
  count_launch();
  k_ell_fill<<<div_up(32 * ng, TPB), TPB, 0, s>>>(mv, ns, m.shell_off, m.entry_key, m.ell_base,
                                             m.ell_len, perm, m.ell_cell, c->d, n_ell, m.ell_key,
                                             m.ell_coef, m.ell_coef32, m.ell_sw, m.ell_any);
  IBM_LAUNCH_CHECK(c);
  m.n_ell = n_ell;
  m.n_entries = ne;
  m.n_shell = ns;
  c->markers_set = true;
  return IBM_OK;
}

void launch_marker_grad_interp(ibm_ctx* c, const double* v, double scale, double* t,
                               cudaStream_t st) {
  const MarkerData& m = c->mk;
  if (m.n == 0) return;
  count_launch();
  k_marker_grad_interp<double><<<div_up(12 * m.n, TPB), TPB, 0, st ? st : c->stream>>>(
      c->d, view(m), v, scale, t);
}

void launch_marker_grad_interp_f32(ibm_ctx* c, const float* v, double scale, double* t,
                                   cudaStream_t st) {
  const MarkerData& m = c->mk;
  if (m.n == 0) return;
  count_launch();
  k_marker_grad_interp<float><<<div_up(12 * m.n, TPB), TPB, 0, st ? st : c->stream>>>(
      c->d, view(m), v, scale, t);
}

void launch_marker_grad_interp_t32(ibm_ctx* c, const float* v, float scale, float* t32,
                                   cudaStream_t st) {
  const MarkerData& m = c->mk;
  if (m.n == 0) return;
  count_launch();
  k_marker_grad_interp_f32<<<div_up(12 * m.n, TPB), TPB, 0, st ? st : c->stream>>>(
      c->d, view(m), m.wc32, m.cw32, v, scale, t32);
}

void launch_shell_gradt_spread(ibm_ctx* c, const double* t, double scale, double* out) {
  const MarkerData& m = c->mk;
  if (m.n == 0 || m.n_shell == 0) return;
  count_launch();
  k_shell_gradt<<<div_up(32 * ell_groups(m.n_shell), TPB), TPB, 0, c->stream>>>(
      m.n_shell, m.ell_cell, m.ell_base, m.ell_len, m.ell_key, m.ell_coef, m.n_ell, m.n, t,
      scale, out);
}

// Position derivative of the interpolation, contracted with a marker field:
// for marker k and axis e,
//   Xbar[e][k] (+)= scale sum_d m[d][k] sum_{taps i of component d}
//                   f_d,i d(phi phi phi)_i / dX_{e,k},
// d/dX_e of phi((x_e - X_e)/h) being -phi'/h.  Four lanes per marker (lanes
// d = 0, 1, 2 take the velocity components, lane 3 idles); the three
// components are combined by shuffles in a fixed order.
__global__ void k_interp_dpos(Dims d, MkView mk, const double* __restrict__ dwf,
                              const double* __restrict__ dwc, const double* __restrict__ f,
                              const double* __restrict__ mv, double scale, double inv_h,
                              int accumulate, double* __restrict__ Xbar) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t k = tid >> 2;
  const int dc = (int)(tid & 3);
  const bool act = k < mk.n && dc < 3;
  double g[3] = {0.0, 0.0, 0.0};
  if (act) {
    const FaceDims fd = face_dims(d);
    const int64_t off = dc == 0 ? 0 : (dc == 1 ? fd.nfx : fd.nfx + fd.nfy);
    const int64_t sy = d.nx + (dc == 0 ? 1 : 0);
    const int64_t sz = sy * (d.ny + (dc == 1 ? 1 : 0));
    int b[3];
    double w[3][3], dw[3][3];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      b[e] = (e == dc) ? mk.bf[e * mk.n + k] : mk.bc[e * mk.n + k];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        w[e][q] = (e == dc) ? mk.wf[(e * 3 + q) * mk.n + k] : mk.wc[(e * 3 + q) * mk.n + k];
        dw[e][q] = (e == dc) ? dwf[(e * 3 + q) * mk.n + k] : dwc[(e * 3 + q) * mk.n + k];
      }
    }
    for (int c2 = 0; c2 < 3; ++c2) {
      for (int c1 = 0; c1 < 3; ++c1) {
        const int64_t base = off + (int64_t)(b[2] + c2) * sz + (int64_t)(b[1] + c1) * sy + b[0];
#pragma unroll
        for (int c0 = 0; c0 < 3; ++c0) {
          const double v = __ldg(f + base + c0);
          g[0] = fma(v, dw[0][c0] * w[1][c1] * w[2][c2], g[0]);
          g[1] = fma(v, w[0][c0] * dw[1][c1] * w[2][c2], g[1]);
          g[2] = fma(v, w[0][c0] * w[1][c1] * dw[2][c2], g[2]);
        }
      }
    }
    const double mm = mv[dc * mk.n + k];
#pragma unroll
    for (int e = 0; e < 3; ++e) g[e] *= mm;
  }
  // lanes (d = 0, 1, 2, 3) of one marker are adjacent: sum in the order
  // (0 + 1) + (2 + 3)
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    g[e] += __shfl_xor_sync(0xffffffffu, g[e], 1);
    g[e] += __shfl_xor_sync(0xffffffffu, g[e], 2);
  }
  if (k < mk.n && dc == 0) {
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      const double v = -scale * inv_h * g[e];
      Xbar[e * mk.n + k] = accumulate ? Xbar[e * mk.n + k] + v : v;
    }
  }
}

void launch_interp(ibm_ctx* c, const double* u, double* U) {
  const MarkerData& m = c->mk;
  if (m.n == 0) return;
  count_launch();
  k_interp<<<div_up(3 * m.n, TPB), TPB, 0, c->stream>>>(c->d, view(m), u, U);
}

void launch_interp_dpos(ibm_ctx* c, const double* f, const double* mvec, double scale,
                        bool accumulate, double* Xbar) {
  const MarkerData& m = c->mk;
  if (m.n == 0) return;
  count_launch();
  k_interp_dpos<<<div_up(4 * m.n, TPB), TPB, 0, c->stream>>>(c->d, view(m), m.dwf, m.dwc, f, mvec,
                                                              scale, 1.0 / c->h,
                                                              accumulate ? 1 : 0, Xbar);
}

void launch_shell_spread_faces(ibm_ctx* c, const double* F, double scale, double* u) {
  const MarkerData& m = c->mk;
  if (m.n == 0 || m.n_shell == 0) return;
  count_launch();
  k_shell_spread_ell<<<div_up(32 * ell_groups(m.n_shell), TPB), TPB, 0, c->stream>>>(
      c->d, m.n_shell, m.ell_cell, m.ell_base, m.ell_len, m.ell_key, m.ell_sw, m.ell_any, m.n_ell,
      m.n, F, scale, 0, u);
}

int launch_shell_spread_asum2(ibm_ctx* c, const double* A, const double* B, double* part) {
  const MarkerData& m = c->mk;
  if (m.n == 0 || m.n_shell == 0) return 0;
  count_launch();
  k_shell_spread_asum2<<<kSpreadAsumBlocks, TPB, 0, c->stream>>>(
      c->d, view(m), m.n_shell, m.shell_cell, m.shell_off, m.entry_key, A, B, part);
  return kSpreadAsumBlocks;
}

void launch_shell_spread_faces_set(ibm_ctx* c, const double* F, double* u) {
  const MarkerData& m = c->mk;
  if (m.n == 0 || m.n_shell == 0) return;
  count_launch();
  k_shell_spread_ell<<<div_up(32 * ell_groups(m.n_shell), TPB), TPB, 0, c->stream>>>(
      c->d, m.n_shell, m.ell_cell, m.ell_base, m.ell_len, m.ell_key, m.ell_sw, m.ell_any, m.n_ell,
      m.n, F, 1.0, 1, u);
}

}  // namespace ibm
