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

int pipe_max_threads_f32(int maxm) {  // mirrors PipeBound<float, maxm>
  const int regs = maxm * 4 / 4 + 96;
  const int raw = 65536 / regs;
  return (raw >= 1024 ? 1024 : raw) / 32 * 32;
}

}  // namespace bfv
