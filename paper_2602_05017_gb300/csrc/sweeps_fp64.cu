// FP64 instantiations of the sweep kernels (element type double).
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

}  // namespace bfv
