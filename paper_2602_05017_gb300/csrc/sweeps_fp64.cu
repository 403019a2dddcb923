// FP64 instantiations of the sweep kernels (element type double).
#include "adjoint.cuh"
#include "batch.cuh"
#include "stream.cuh"
#include "sweeps.cuh"

namespace bfv {

cudaError_t launch_x_f64(const XLaunch &a, cudaStream_t st) {
  switch (a.maxm) {
    case 8: return launch_x_one<double, 8>(a, st);
    case 16: return launch_x_one<double, 16>(a, st);
    case 24: return launch_x_one<double, 24>(a, st);
    case 32: return launch_x_one<double, 32>(a, st);
    case 48: return launch_x_one<double, 48>(a, st);
    case 64: return launch_x_one<double, 64>(a, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_col_f64(const ColLaunch &a, cudaStream_t st) {
  switch (a.maxm) {
    case 8: return launch_col_one<double, 8>(a, st);
    case 16: return launch_col_one<double, 16>(a, st);
    case 24: return launch_col_one<double, 24>(a, st);
    case 32: return launch_col_one<double, 32>(a, st);
    case 48: return launch_col_one<double, 48>(a, st);
    case 64: return launch_col_one<double, 64>(a, st);
  }
  return cudaErrorInvalidValue;
}


cudaError_t allow_x_smem_f64(int maxm, size_t bytes) {
  switch (maxm) {
    case 8: return allow_x_smem<double, 8>(bytes);
    case 16: return allow_x_smem<double, 16>(bytes);
    case 24: return allow_x_smem<double, 24>(bytes);
    case 32: return allow_x_smem<double, 32>(bytes);
    case 48: return allow_x_smem<double, 48>(bytes);
    case 64: return allow_x_smem<double, 64>(bytes);
  }
  return cudaErrorInvalidValue;
}


cudaError_t launch_nodes_f64(const NodeLaunch &a, cudaStream_t st) {
  return launch_nodes_one<double>(a, st);
}

cudaError_t launch_adj_reduce_f64(const ReduceLaunch &a, cudaStream_t st) {
  adj_reduce_kernel<double><<<a.nblocks, kReduceThreads, 0, st>>>(
      static_cast<const double *>(a.mu), static_cast<const double *>(a.u), a.nel, a.S, a.stride,
      a.n_axis, a.used, a.partial);
  adj_reduce_final_kernel<double><<<1, 32, 0, st>>>(a.partial, a.nblocks, a.S, a.scale_lambda, a.scale_D,
                                            a.dlambda, a.dD);
  return cudaGetLastError();
}

cudaError_t launch_src_adjoint_f64(const SrcAdjLaunch &a, cudaStream_t st) {
  if ((a.dsec || a.dupt) && a.n > 0)
    src_adjoint_agents_kernel<double><<<(unsigned)((a.n + 255) / 256), 256, 0, st>>>(
        static_cast<const double *>(a.gbar), static_cast<const double *>(a.u1), a.elem, a.entry,
        static_cast<const double *>(a.src_scale), a.weight, a.target, a.n, a.dt, a.S, a.dsec,
        a.dupt);
  if (a.n_entries > 0)
    src_adjoint_scale_kernel<double><<<(unsigned)((a.n_entries + 255) / 256), 256, 0, st>>>(
        static_cast<double *>(a.gbar), a.src_elem, static_cast<const double *>(a.src_scale),
        a.n_entries);
  return cudaGetLastError();
}


cudaError_t launch_batch_f64(const BatchArgs &a, int, int grid, cudaStream_t st) {
  return launch_batch_one<double>(a, grid, st);
}

cudaError_t batch_occupancy_f64(int maxm, int *out) { return batch_blocks_per_sm<double>(maxm, out); }

cudaError_t allow_stream_smem_f64() { return allow_stream_smem<double>(); }

cudaError_t launch_stream_f64(const StreamArgs &a, int grid, cudaStream_t st) {
  switch (a.out) {
    case 1: return launch_stream_one<double, 1>(a, grid, st);
    case 2: return launch_stream_one<double, 2>(a, grid, st);
  }
  return launch_stream_one<double, 0>(a, grid, st);
}

}  // namespace bfv
