// Allocation-free variant of ibm_body_forces for callers that cannot call
// cudaMalloc.  See include/ibm_schur.h for the contract.
//
// The device staging buffer (the body centres going in, the per-body sums
// coming out) is a file-scope __device__ array: it exists in every GPU that
// loads this library from module load until process exit, and no call
// allocates or frees anything.  Host code must not use the array's name as a
// device address (in host code it names a host-side shadow); the device
// address is looked up with cudaGetSymbolAddress, with the device current,
// once per device and again whenever the device's context has changed (a
// cudaDeviceReset followed by new work creates a new context, in which the
// module and its array are loaded anew).
#include <cuda.h>

#include <cstdint>
#include <mutex>

#include "ibm_internal.cuh"

namespace ibm {
namespace {

constexpr int kMaxDevices = 64;
// centres [IBM_NOALLOC_MAX_BODIES][3], then the sums [IBM_NOALLOC_MAX_BODIES][6]
constexpr int kScratchDoubles = IBM_NOALLOC_MAX_BODIES * 9;

static __device__ __align__(256) double g_body_scratch[kScratchDoubles];

struct Cached {
  double* ptr = nullptr;
  unsigned long long ctx_id = 0;
};
std::mutex g_mu;
Cached g_cache[kMaxDevices];

using CtxGetCurrent = CUresult (*)(CUcontext*);
using CtxGetId = CUresult (*)(CUcontext, unsigned long long*);

// Identifier of the calling thread's current context (0 if it cannot be
// read).  The driver functions are found through the runtime, so the library
// does not link the driver library itself.
unsigned long long current_ctx_id() {
  static CtxGetCurrent get_current = nullptr;
  static CtxGetId get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    void* f0 = nullptr;
    void* f1 = nullptr;
    cudaDriverEntryPointQueryResult q0 = cudaDriverEntryPointSymbolNotFound, q1 = q0;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f0, 12000, cudaEnableDefault, &q0) ==
            cudaSuccess &&
        q0 == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrent>(f0);
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f1, 12000, cudaEnableDefault, &q1) ==
            cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetId>(f1);
    looked_up = true;
  }
  if (!get_current || !get_id) return 0;
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr || get_id(ctx, &id) != CUDA_SUCCESS)
    return 0;
  return id;
}

// Device address of g_body_scratch on the current device: looked up on the
// first call on a device and again after that device's context changed.
cudaError_t scratch_address(double** ptr) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  // makes the runtime's context current on this thread, so its id can be read
  if ((e = cudaFree(nullptr)) != cudaSuccess) return e;
  const unsigned long long id = current_ctx_id();
  std::lock_guard<std::mutex> lock(g_mu);
  Cached& c = g_cache[dev];
  if (!c.ptr || id == 0 || id != c.ctx_id) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_body_scratch);
    if (e != cudaSuccess) return e;
    c.ptr = static_cast<double*>(p);
    c.ctx_id = id;
  }
  *ptr = c.ptr;
  return cudaSuccess;
}

// Device (or managed) memory that the current device can address directly,
// aligned to `align` bytes.
bool device_ptr_ok(const void* p, uintptr_t align) {
  if (p == nullptr || (reinterpret_cast<uintptr_t>(p) & (align - 1)) != 0) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
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
  // misaligned pointers or memory this device cannot address are refused
  // before anything is launched
  if (!ibm::device_ptr_ok(F, 8) || !ibm::device_ptr_ok(X, 8) || !ibm::device_ptr_ok(body_id, 4))
    return IBM_ERR_ARG;
  // an error left by earlier, unrelated work on this thread is cleared here,
  // so that the check after the launch sees only this call's
  cudaGetLastError();
  double* scratch = nullptr;
  if (ibm::scratch_address(&scratch) != cudaSuccess) return IBM_ERR_CUDA;
  double* cen = scratch;
  double* sums = scratch + 3 * IBM_NOALLOC_MAX_BODIES;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // every centre and sum slot a call uses is written by that call
  if (cudaMemcpyAsync(cen, centers, sizeof(double) * 3 * n_bodies, cudaMemcpyHostToDevice, s) !=
      cudaSuccess)
    return IBM_ERR_CUDA;
  ibm::launch_body_sums(F, X, body_id, n_markers, n_bodies, cen, h * h * h, sums, s);
  if (cudaGetLastError() != cudaSuccess) return IBM_ERR_CUDA;
  if (cudaMemcpyAsync(out, sums, sizeof(double) * 6 * n_bodies, cudaMemcpyDeviceToHost, s) !=
      cudaSuccess)
    return IBM_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return IBM_ERR_CUDA;
  return IBM_OK;
}
