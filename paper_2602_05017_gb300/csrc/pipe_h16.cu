// Instantiations of the persistent TMA-pipelined sweep (pipe.cuh) for fields
// stored in 16 bits -- bf16 or fp16 -- with FP32 arithmetic and FP32 constants:
// chunk capacities 32 and 64 (the planner rounds the chunk capacity of a 16-bit
// handle up to 32, and takes 16-line tiles rather than chunks above 64).
#include "pipe.cuh"

namespace bfv {

template <typename H>
cudaError_t allow_pipe_smem_h16(int maxm, size_t bytes) {
  switch (maxm) {
    case 32: return allow_pipe_smem<float, 32, H>(bytes);
    case 64: return allow_pipe_smem<float, 64, H>(bytes);
  }
  return cudaErrorInvalidValue;
}

template <typename H>
cudaError_t launch_pipe_h16(const CUtensorMap &map, const PipeArgs &a, int maxm, int grid,
                            size_t smem, cudaStream_t st) {
  switch (maxm) {
    case 32: return launch_pipe_one<float, 32, H>(map, a, grid, smem, st);
    case 64: return launch_pipe_one<float, 64, H>(map, a, grid, smem, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t allow_pipe_smem_bf16(int maxm, size_t bytes) {
  return allow_pipe_smem_h16<__nv_bfloat16>(maxm, bytes);
}
cudaError_t allow_pipe_smem_fp16(int maxm, size_t bytes) {
  return allow_pipe_smem_h16<__half>(maxm, bytes);
}
cudaError_t launch_pipe_bf16(const CUtensorMap &map, const PipeArgs &a, int maxm, int grid,
                             size_t smem, cudaStream_t st) {
  return launch_pipe_h16<__nv_bfloat16>(map, a, maxm, grid, smem, st);
}
cudaError_t launch_pipe_fp16(const CUtensorMap &map, const PipeArgs &a, int maxm, int grid,
                             size_t smem, cudaStream_t st) {
  return launch_pipe_h16<__half>(map, a, maxm, grid, smem, st);
}

}  // namespace bfv
