// FP32 instantiations of the sweep kernels (element type float; the Thomas
// constants are computed in double on the host and rounded to float).
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

}  // namespace bfv
