// FMA issue-rate probe: the arithmetic roof the benchmark reports the FP64
// sweeps against.  The Thomas recurrences of Sect. 2.1 (Eq. 2: per line, a
// forward axpy and division and a backward axpy per position) run as FMAs;
// on a GB300 the FP64 unit is narrow, so the FP64 step is bounded by its FMA
// rate rather than by HBM, and that rate is measured here, on the device the
// caller has current, rather than taken from a data sheet.
//
// Each thread runs kChains independent dependent chains x <- fma(x, a, b),
// enough to cover the pipe latency; the grid holds 32 warps per SM.  A
// calibration launch sizes the timed launches to about 25 ms; the best of
// three CUDA-event timings gives FMA/s.  The result is kept alive through a
// file-scope device word written only if the sum is an impossible value.
#include <cuda_runtime.h>

#include "../../include/biofvm.h"
#include "internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;
constexpr int kProbeCtasPerSm = 4;

__device__ double g_probe_sink;

template <typename T>
__global__ void __launch_bounds__(kProbeThreads) fma_probe_kernel(T a, T b, int iters) {
  T x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; k++) x[k] = T(threadIdx.x & 7) * T(0.125) + T(k) * T(0.01);
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int k = 0; k < kChains; k++) x[k] = fma(x[k], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < kChains; k++) s += x[k];
  if (s == T(-1.0e30)) g_probe_sink = (double)s;  // never true: x stays in (0, 1)
}

biofvm_status fail(biofvm_status st, const char *msg) {
  bfv::set_error_message(msg);
  return st;
}

template <typename T>
cudaError_t timed(int grid, int iters, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1,
                  float *ms) {
  cudaEventRecord(e0, st);
  fma_probe_kernel<T><<<grid, kProbeThreads, 0, st>>>(T(0.9999), T(1.0e-5), iters);
  cudaEventRecord(e1, st);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  return e;
}

template <typename T>
biofvm_status probe(cudaStream_t st, double *rate) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return fail(BIOFVM_ERR_CUDA, "no usable CUDA device");
  const int grid = sms * kProbeCtasPerSm;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return fail(BIOFVM_ERR_CUDA, "cudaEventCreate failed");
  }
  float ms = 0.f;
  int iters = 256;
  cudaError_t e = timed<T>(grid, iters, st, e0, e1, &ms);  // calibration (and warm-up)
  if (e == cudaSuccess) {
    const double want = 25.0;  // ms per timed launch
    const double scale = ms > 0.f ? want / ms : 64.0;
    const double it = (double)iters * (scale > 4096.0 ? 4096.0 : scale);
    iters = it < 256.0 ? 256 : it > 2.0e8 ? 200000000 : (int)it;
  }
  double best = 0.0;
  for (int rep = 0; rep < 3 && e == cudaSuccess; rep++) {
    e = timed<T>(grid, iters, st, e0, e1, &ms);
    if (e == cudaSuccess && ms > 0.f) {
      const double r = (double)grid * kProbeThreads * kChains * iters / (ms * 1e-3);
      if (r > best) best = r;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return fail(BIOFVM_ERR_CUDA, cudaGetErrorString(e));
  *rate = best;
  return BIOFVM_OK;
}

}  // namespace

extern "C" biofvm_status biofvm_probe_fma_rate(biofvm_precision prec, uintptr_t cuda_stream,
                                               double *fma_per_second) {
  if (!fma_per_second) return fail(BIOFVM_ERR_ARG, "fma_per_second is NULL");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  if (prec == BIOFVM_FP64) return probe<double>(st, fma_per_second);
  if (prec == BIOFVM_FP32) return probe<float>(st, fma_per_second);
  return fail(BIOFVM_ERR_ARG, "unknown precision");
}
