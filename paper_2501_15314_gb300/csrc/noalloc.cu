// Allocation-free variant of ibm_body_forces for callers that cannot call
// cudaMalloc.  See include/ibm_schur.h for the contract.
//
// The device staging buffer the per-body sums are written to before the copy
// to the host is a file-scope __device__ array: it exists in every GPU that
// loads this library from module load until process exit, and no call
// allocates or frees anything.  Host code must not use the array's name as a
// device address (in host code it names a host-side shadow); the device
// address is looked up once per device with cudaGetSymbolAddress and cached.
#include <mutex>

#include "ibm_internal.cuh"

namespace ibm {
namespace {

constexpr int kNoallocThreads = 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_body_scratch[IBM_NOALLOC_MAX_BODIES * 6];

std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// Per body: sums of F and of (X - c) x F over its markers, times h^3, written
// to out[6b..6b+5].  One block per body, fixed-order block reduction; every
// output slot is overwritten, so nothing needs clearing between calls.
__global__ void k_body_forces_scratch(const double* __restrict__ F, const double* __restrict__ X,
                                      const int32_t* __restrict__ bid, int64_t n, double h3,
                                      double cx, double cy, double cz, int body,
                                      double* __restrict__ out) {
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t k = threadIdx.x; k < n; k += blockDim.x) {
    if (bid[k] != body) continue;
    const double fx = F[k], fy = F[n + k], fz = F[2 * n + k];
    const double rx = X[k] - cx, ry = X[n + k] - cy, rz = X[2 * n + k] - cz;
    acc[0] += fx; acc[1] += fy; acc[2] += fz;
    acc[3] += ry * fz - rz * fy;
    acc[4] += rz * fx - rx * fz;
    acc[5] += rx * fy - ry * fx;
  }
  __shared__ double sh[6][kNoallocThreads];
  for (int q = 0; q < 6; ++q) sh[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int s = kNoallocThreads / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
      for (int q = 0; q < 6; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < 6) out[threadIdx.x] = h3 * sh[threadIdx.x][0];
}

// Device address of g_body_scratch on the current device (looked up once).
cudaError_t scratch_address(double** ptr) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_body_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *ptr = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace ibm

extern "C" ibm_status ibm_body_forces_noalloc(const double* F, const double* X,
                                              const int32_t* body_id, int64_t n_markers,
                                              int32_t n_bodies, const double* centers, double h,
                                              void* stream, double* out) {
  if (n_bodies < 1 || n_bodies > IBM_NOALLOC_MAX_BODIES || !centers || !out || n_markers < 0 ||
      !(h > 0.0))
    return IBM_ERR_ARG;
  if (n_markers == 0) {
    for (int q = 0; q < 6 * n_bodies; ++q) out[q] = 0.0;
    return IBM_OK;
  }
  if (!F || !X || !body_id) return IBM_ERR_ARG;
  double* scratch = nullptr;
  if (ibm::scratch_address(&scratch) != cudaSuccess) return IBM_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const double h3 = h * h * h;
  for (int b = 0; b < n_bodies; ++b) {
    ibm::count_launch();
    ibm::k_body_forces_scratch<<<1, ibm::kNoallocThreads, 0, s>>>(
        F, X, body_id, n_markers, h3, centers[3 * b], centers[3 * b + 1],
        centers[3 * b + 2], b, scratch + 6 * b);
  }
  if (cudaGetLastError() != cudaSuccess) return IBM_ERR_CUDA;
  if (cudaMemcpyAsync(out, scratch, sizeof(double) * 6 * n_bodies, cudaMemcpyDeviceToHost, s) !=
      cudaSuccess)
    return IBM_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return IBM_ERR_CUDA;
  return IBM_OK;
}
