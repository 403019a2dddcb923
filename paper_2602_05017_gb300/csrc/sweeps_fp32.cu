// FP32 instantiations of the sweep kernels (element type float; the Thomas
// constants are computed in double on the host and rounded to float).
#include "adjoint.cuh"
#include "batch.cuh"
#include "stream.cuh"
#include "sweeps.cuh"

namespace bfv {

cudaError_t launch_x_f32(const XLaunch &a, cudaStream_t st) {
  switch (a.maxm) {
    case 8: return launch_x_one<float, 8>(a, st);
    case 16: return launch_x_one<float, 16>(a, st);
    case 24: return launch_x_one<float, 24>(a, st);
    case 32: return launch_x_one<float, 32>(a, st);
    case 48: return launch_x_one<float, 48>(a, st);
    case 64: return launch_x_one<float, 64>(a, st);
    case 96: return launch_x_one<float, 96>(a, st);
    case 128: return launch_x_one<float, 128>(a, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_col_f32(const ColLaunch &a, cudaStream_t st) {
  switch (a.maxm) {
    case 8: return launch_col_one<float, 8>(a, st);
    case 16: return launch_col_one<float, 16>(a, st);
    case 24: return launch_col_one<float, 24>(a, st);
    case 32: return launch_col_one<float, 32>(a, st);
    case 48: return launch_col_one<float, 48>(a, st);
    case 64: return launch_col_one<float, 64>(a, st);
    case 96: return launch_col_one<float, 96>(a, st);
    case 128: return launch_col_one<float, 128>(a, st);
  }
  return cudaErrorInvalidValue;
}


cudaError_t allow_x_smem_f32(int maxm, size_t bytes) {
  switch (maxm) {
    case 8: return allow_x_smem<float, 8>(bytes);
    case 16: return allow_x_smem<float, 16>(bytes);
    case 24: return allow_x_smem<float, 24>(bytes);
    case 32: return allow_x_smem<float, 32>(bytes);
    case 48: return allow_x_smem<float, 48>(bytes);
    case 64: return allow_x_smem<float, 64>(bytes);
    case 96: return allow_x_smem<float, 96>(bytes);
    case 128: return allow_x_smem<float, 128>(bytes);
  }
  return cudaErrorInvalidValue;
}


cudaError_t launch_nodes_f32(const NodeLaunch &a, cudaStream_t st) {
  return launch_nodes_one<float>(a, st);
}

cudaError_t launch_adj_reduce_f32(const ReduceLaunch &a, cudaStream_t st) {
  adj_reduce_kernel<float><<<a.nblocks, kReduceThreads, 0, st>>>(
      static_cast<const float *>(a.mu), static_cast<const float *>(a.u), a.nel, a.S, a.stride,
      a.n_axis, a.used, a.partial);
  adj_reduce_final_kernel<float><<<1, 32, 0, st>>>(a.partial, a.nblocks, a.S, a.scale_lambda, a.scale_D,
                                            a.dlambda, a.dD);
  return cudaGetLastError();
}

cudaError_t launch_src_adjoint_f32(const SrcAdjLaunch &a, cudaStream_t st) {
  if ((a.dsec || a.dupt) && a.n > 0)
    src_adjoint_agents_kernel<float><<<(unsigned)((a.n + 255) / 256), 256, 0, st>>>(
        static_cast<const float *>(a.gbar), static_cast<const float *>(a.u1), a.elem, a.entry,
        static_cast<const float *>(a.src_scale), a.weight, a.target, a.n, a.dt, a.S, a.dsec,
        a.dupt);
  if (a.n_entries > 0)
    src_adjoint_scale_kernel<float><<<(unsigned)((a.n_entries + 255) / 256), 256, 0, st>>>(
        static_cast<float *>(a.gbar), a.src_elem, static_cast<const float *>(a.src_scale),
        a.n_entries);
  return cudaGetLastError();
}


cudaError_t launch_batch_f32(const BatchArgs &a, int, int grid, cudaStream_t st) {
  return launch_batch_one<float>(a, grid, st);
}

cudaError_t batch_occupancy_f32(int maxm, int *out) { return batch_blocks_per_sm<float>(maxm, out); }

cudaError_t launch_stream_f32(const StreamArgs &a, int grid, cudaStream_t st) {
  return launch_stream_one<float, 0>(a, grid, st);
}

}  // namespace bfv
