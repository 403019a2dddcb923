// FP32 instantiations of the persistent TMA-pipelined sweep kernels (pipe.cuh),
// a translation unit of their own so that the build compiles them in parallel
// with the other kernels.
#include "pipe.cuh"

namespace bfv {

cudaError_t allow_pipe_smem_f32(int maxm, size_t bytes) {
  switch (maxm) {
    case 8: return allow_pipe_smem<float, 8>(bytes);
    case 16: return allow_pipe_smem<float, 16>(bytes);
    case 24: return allow_pipe_smem<float, 24>(bytes);
    case 32: return allow_pipe_smem<float, 32>(bytes);
    case 48: return allow_pipe_smem<float, 48>(bytes);
    case 64: return allow_pipe_smem<float, 64>(bytes);
    case 96: return allow_pipe_smem<float, 96>(bytes);
    case 128: return allow_pipe_smem<float, 128>(bytes);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_pipe_f32(const CUtensorMap &map, const PipeArgs &a, int maxm, int grid,
                            size_t smem, cudaStream_t st) {
  switch (maxm) {
    case 8: return launch_pipe_one<float, 8>(map, a, grid, smem, st);
    case 16: return launch_pipe_one<float, 16>(map, a, grid, smem, st);
    case 24: return launch_pipe_one<float, 24>(map, a, grid, smem, st);
    case 32: return launch_pipe_one<float, 32>(map, a, grid, smem, st);
    case 48: return launch_pipe_one<float, 48>(map, a, grid, smem, st);
    case 64: return launch_pipe_one<float, 64>(map, a, grid, smem, st);
    case 96: return launch_pipe_one<float, 96>(map, a, grid, smem, st);
    case 128: return launch_pipe_one<float, 128>(map, a, grid, smem, st);
  }
  return cudaErrorInvalidValue;
}

namespace {
// Rows of `len` elements from a field with rows `spitch` apart into one with
// rows `dpitch` apart: one warp per row, lanes along the row (coalesced);
// T is a 4- or 2-byte element (the copy moves bits, no arithmetic).
template <typename T>
__global__ void __launch_bounds__(256) pitch_rows_kernel(const T *__restrict__ src,
                                                         T *__restrict__ dst, int64_t rows,
                                                         int len, int spitch, int dpitch) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < rows;
       r += warps) {
    const T *s = src + r * spitch;
    T *d = dst + r * dpitch;
    for (int i = lane; i < len; i += 32) d[i] = s[i];
  }
}
}  // namespace

cudaError_t launch_pitch_rows(const void *src, void *dst, int64_t rows, int len, int spitch,
                              int dpitch, size_t esz, int grid, cudaStream_t st) {
  if (rows <= 0 || len <= 0) return cudaSuccess;
  if (esz == 4)
    pitch_rows_kernel<uint32_t><<<grid, 256, 0, st>>>(static_cast<const uint32_t *>(src),
                                                     static_cast<uint32_t *>(dst), rows, len,
                                                     spitch, dpitch);
  else if (esz == 2)
    pitch_rows_kernel<uint16_t><<<grid, 256, 0, st>>>(static_cast<const uint16_t *>(src),
                                                     static_cast<uint16_t *>(dst), rows, len,
                                                     spitch, dpitch);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

int pipe_max_threads_f32(int maxm) {  // mirrors PipeBound<float, maxm>
  const int regs = maxm * 4 / 4 + 96;
  const int raw = 65536 / regs;
  return (raw >= 1024 ? 1024 : raw) / 32 * 32;
}

}  // namespace bfv
