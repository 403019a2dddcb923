// A variant of the adjoint's parameter-gradient reduction that allocates
// nothing, for callers that cannot call cudaMalloc: code running inside a
// host framework that owns all device memory (a memory pool or arena it will
// not let libraries bypass), processes under a device-memory budget, or
// contexts where allocation is forbidden (for example between the set-up and
// the timed part of a real-time loop).  The paper has no counterpart; it is a
// convenience of this library.
//
// The per-block partial sums live in one file-scope __device__ array
// (g_partial, 256 KB: kBlocks blocks x 2 sums x at most kMaxSub substrates,
// FP64), which every GPU that loads the library holds until the process
// exits.  In host code `g_partial` names a host-side stand-in, not device
// memory, so its device address is looked up with cudaGetSymbolAddress, with
// the device current, and cached per device together with the unique id of
// the CUDA context it was looked up in: a call made in another context (after
// cudaDeviceReset, or from a context that is not the device's primary one)
// looks it up again instead of using an address of a context that is gone.
#include <cuda.h>  // CUcontext (type only; the two driver calls are fetched at run time)
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/biofvm.h"
#include "adjoint.cuh"

namespace {

constexpr int kBlocks = 512;
constexpr int kMaxSub = 32;
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_partial[kBlocks * 2 * kMaxSub];

std::mutex g_mutex;
double *g_addr[kMaxDevices] = {nullptr};
unsigned long long g_ctx[kMaxDevices] = {0};  // context id of each cached address (0: none)

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

// Unique id of the calling thread's current CUDA context (ids are never
// reused within a process), or 0 when there is none or it cannot be read.
unsigned long long current_context_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool tried = false;
  if (!tried) {  // called under g_mutex
    tried = true;
    void *p = nullptr, *q = nullptr;
    cudaDriverEntryPointQueryResult r1, r2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &r1) ==
            cudaSuccess &&
        r1 == cudaDriverEntryPointSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &q, 12000, cudaEnableDefault, &r2) ==
            cudaSuccess &&
        r2 == cudaDriverEntryPointSuccess) {
      get_current = reinterpret_cast<CtxGetCurrentFn>(p);
      get_id = reinterpret_cast<CtxGetIdFn>(q);
    }
  }
  CUcontext c = nullptr;
  unsigned long long id = 0;
  if (get_current && get_id && get_current(&c) == CUDA_SUCCESS && c &&
      get_id(c, &id) == CUDA_SUCCESS)
    return id;
  return 0;
}

biofvm_status fail(biofvm_status st, const char *msg) {
  bfv::set_error_message(msg);
  return st;
}

}  // namespace

extern "C" biofvm_status biofvm_param_grad_noalloc(const void *mu, const void *u, int nx, int ny,
                                                   int nz, int n_sub, int axis,
                                                   biofvm_precision prec, double dt, double h_axis,
                                                   double *dD, double *dlambda,
                                                   uintptr_t cuda_stream) {
  if (!mu || !u || !dD || !dlambda) return fail(BIOFVM_ERR_ARG, "NULL array argument");
  if (nx < 1 || ny < 1 || nz < 1) return fail(BIOFVM_ERR_ARG, "grid sizes must be >= 1");
  if (n_sub < 1 || n_sub > kMaxSub)
    return fail(BIOFVM_ERR_ARG, "n_sub must be in [1, 32]: the static scratch holds 32 substrates");
  if (axis < 0 || axis > 2) return fail(BIOFVM_ERR_ARG, "axis must be 0 (x), 1 (y) or 2 (z)");
  if (prec != BIOFVM_FP64 && prec != BIOFVM_FP32) return fail(BIOFVM_ERR_ARG, "unknown precision");
  if (!(dt > 0.0) || !(h_axis > 0.0) || !std::isfinite(dt) || !std::isfinite(h_axis))
    return fail(BIOFVM_ERR_ARG, "dt and h_axis must be finite and > 0");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return fail(BIOFVM_ERR_CUDA, "no usable CUDA device");
  double *partial;
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    const unsigned long long ctx = current_context_id();
    if (!g_addr[dev] || ctx == 0 || ctx != g_ctx[dev]) {
      // first call on this device, or in another context than the cached address's: look the
      // array's device address up (with no context id readable, on every call)
      void *p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_partial);
      if (e != cudaSuccess) return fail(BIOFVM_ERR_CUDA, "cudaGetSymbolAddress(g_partial) failed");
      g_addr[dev] = static_cast<double *>(p);
      g_ctx[dev] = current_context_id();  // the lookup made the device's context current
    }
    partial = g_addr[dev];
  }
  const long long S = n_sub;
  const long long nel = (long long)nx * ny * nz * S;
  const long long stride = axis == 0 ? S : axis == 1 ? (long long)nx * S : (long long)nx * ny * S;
  const int n_axis = axis == 0 ? nx : axis == 1 ? ny : nz;
  const long long used = (long long)kBlocks * bfv::kReduceThreads / S * S;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  if (prec == BIOFVM_FP64) {
    bfv::adj_reduce_kernel<double><<<kBlocks, bfv::kReduceThreads, 0, st>>>(
        static_cast<const double *>(mu), static_cast<const double *>(u), nel, n_sub, stride,
        n_axis, used, partial);
    bfv::adj_reduce_final_kernel<double><<<1, 32, 0, st>>>(partial, kBlocks, n_sub, -dt / 3.0,
                                                           -dt / (h_axis * h_axis), dlambda, dD);
  } else {
    bfv::adj_reduce_kernel<float><<<kBlocks, bfv::kReduceThreads, 0, st>>>(
        static_cast<const float *>(mu), static_cast<const float *>(u), nel, n_sub, stride, n_axis,
        used, partial);
    bfv::adj_reduce_final_kernel<float><<<1, 32, 0, st>>>(partial, kBlocks, n_sub, -dt / 3.0,
                                                          -dt / (h_axis * h_axis), dlambda, dD);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(BIOFVM_ERR_CUDA, cudaGetErrorString(e));
  return BIOFVM_OK;
}
