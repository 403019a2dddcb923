// Small grids (FP64): every step of a biofvm_step call in ONE cooperative,
// persistent launch.
//
// On a grid as small as 50^3 a step is latency-bound: each sweep kernel spends
// its time on the first loads of every line and on the serial Thomas chain,
// and three kernels per step add their launch and drain gaps.  Here one launch
// runs all the steps, with the same stages and arithmetic as the step kernels
// (Src, B, X^-1, B, Y^-1, B, Z^-1, B; Thomas of Algorithm 1 on the App. A
// system: forward g_i = d_i inv_i + mul_i g_{i-1}, backward x_i = g_i + mul_i
// x_{i+1}):
//
//   phase 1, per z-plane (CTA b takes planes b, b + G, ...): the plane is
//     loaded into shared memory, the source update and the Dirichlet
//     application before the x-solve are applied there, every x-line and every
//     y-line of the plane is solved in shared memory (one thread per line), each
//     followed by its Dirichlet application, and the plane is stored back;
//   grid barrier;
//   phase 2, per z-line (one thread each, spread over all CTAs): the streaming
//     line solver of the z-sweep (stream.cuh, unscaled output) with the
//     Dirichlet application after it;
//   grid barrier, next step.
//
// The grid barrier is a counter and a generation word in global memory; every
// wait on it is bounded (about two seconds): on expiry the status word is set,
// an abort word makes every CTA stop at its next barrier, and the launch
// returns (the field is then undefined).  All CTAs are co-resident: the
// launch goes through cudaLaunchCooperativeKernel, which refuses a grid that
// could not be.
#include <cuda_runtime.h>
#include <stdint.h>

#include "stream.cuh"

namespace bfv {

namespace {

constexpr int kSmallThreads = 256;

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Barrier of all CTAs; false when it gave up (timeout, or another CTA's).
// bar[0] arrivals, bar[1] generation, bar[2] abort.
__device__ bool grid_barrier(unsigned *bar, int *status) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = ld_acquire_u32(bar + 2) == 0;
    if (ok) {
      const unsigned gen = ld_acquire_u32(bar + 1);
      __threadfence();  // this block's writes (ordered by __syncthreads) before the arrival
      if (atomicAdd(bar, 1u) + 1 == gridDim.x) {
        atomicExch(bar, 0u);
        __threadfence();
        atomicAdd(bar + 1, 1u);  // release the others
      } else {
        const long long t0 = clock64();
        while (ld_acquire_u32(bar + 1) == gen) {
          if (ld_acquire_u32(bar + 2) != 0) {
            ok = 0;
            break;
          }
          if (clock64() - t0 > (1ll << 32)) {
            atomicExch(status, kStatusTimeout);
            atomicExch(bar + 2, 1u);
            ok = 0;
            break;
          }
          __nanosleep(32);
        }
      }
      __threadfence();
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Solve the lines of one plane in shared memory, one thread per line: AX 0 the
// x-lines (line l = (y, s), positions S apart), AX 1 the y-lines (line l =
// column (x, s), positions nx*S apart); inv/mul: the axis constants [n][S].
template <int AX>
__device__ __forceinline__ void solve_in_smem(double *plane, int nx, int ny, int S,
                                              const double *inv, const double *mul) {
  const int nlines = AX == 0 ? ny * S : nx * S;
  const int n = AX == 0 ? nx : ny, st = AX == 0 ? S : nx * S;
  for (int l = threadIdx.x; l < nlines; l += blockDim.x) {
    const int s = l % S;
    double *q = plane + (AX == 0 ? (l / S) * nx * S + s : l);
    double g = 0.0;
    for (int i = 0; i < n; i++) {
      g = fma(mul[i * S + s], g, q[i * st] * inv[i * S + s]);
      q[i * st] = g;
    }
    double x = g;
    for (int i = n - 2; i >= 0; i--) {
      x = fma(mul[i * S + s], x, q[i * st]);
      q[i * st] = x;
    }
  }
}

__global__ void __launch_bounds__(kSmallThreads, 1) small_steps_kernel(const SmallArgs a) {
  extern __shared__ __align__(16) double small_smem[];
  const int nx = a.nx, ny = a.ny, nz = a.nz, S = a.S;
  const int pl = nx * ny * S;  // elements of one z-plane
  double *plane = small_smem;
  double *xinv = plane + pl, *xmul = xinv + nx * S, *yinv = xmul + nx * S, *ymul = yinv + ny * S;
  for (int i = threadIdx.x; i < nx * S; i += blockDim.x) {
    xinv[i] = __ldg(a.tab[0] + i);
    xmul[i] = __ldg(a.tab[0] + (size_t)nx * S + i);
  }
  for (int i = threadIdx.x; i < ny * S; i += blockDim.x) {
    yinv[i] = __ldg(a.tab[1] + i);
    ymul[i] = __ldg(a.tab[1] + (size_t)ny * S + i);
  }
  __syncthreads();
  auto face_value = [&](int s, double &v) {
    if (!a.any_dir || !a.dir_on[s]) return false;
    v = __ldg(a.dir_val + s);
    return true;
  };
  // B on a plane in shared memory: the plane's face voxels of flagged substrates
  auto dirichlet_plane = [&](int z) {
    if (!a.any_dir) return;
    const bool zf = z == 0 || z == nz - 1;
    for (int e = threadIdx.x; e < pl; e += blockDim.x) {
      const int s = e % S, v = e / S, x = v % nx, y = v / nx;
      double val;
      if ((zf || x == 0 || x == nx - 1 || y == 0 || y == ny - 1) && face_value(s, val))
        plane[e] = val;
    }
    __syncthreads();
  };
  for (int step = 0; step < a.n_steps; step++) {
    // ---- phase 1: Src, B, X^-1, B, Y^-1, B on each z-plane in shared memory ----
    for (int z = blockIdx.x; z < nz; z += gridDim.x) {
      double *g = a.rho + (size_t)z * pl;
      for (int e = threadIdx.x; e < pl; e += blockDim.x) plane[e] = g[e];
      __syncthreads();
      if (a.has_src) {  // entries of the plane's rows: unique elements
        const long long e0 = a.src_row_off[(long long)z * ny];
        const long long e1 = a.src_row_off[(long long)z * ny + ny];
        for (long long k = e0 + threadIdx.x; k < e1; k += blockDim.x) {
          const long long off = a.src_elem[k] - (long long)z * pl;
          plane[off] = (plane[off] + __ldg(a.src_alpha + k)) * __ldg(a.src_scale + k);
        }
        __syncthreads();
      }
      dirichlet_plane(z);
      solve_in_smem<0>(plane, nx, ny, S, xinv, xmul);
      __syncthreads();
      dirichlet_plane(z);
      solve_in_smem<1>(plane, nx, ny, S, yinv, ymul);
      __syncthreads();
      dirichlet_plane(z);
      for (int e = threadIdx.x; e < pl; e += blockDim.x) g[e] = plane[e];
      __syncthreads();
    }
    if (!grid_barrier(a.bar, a.status)) return;
    // ---- phase 2: Z^-1 then B, one z-line per thread: a warp takes 32 adjacent lines (its
    // loads coalesce), the warps spread over the CTAs ----
    const int lane = threadIdx.x & 31, nwarps = gridDim.x * (blockDim.x >> 5);
    for (int w = blockIdx.x + gridDim.x * (threadIdx.x >> 5); w * 32 < pl; w += nwarps) {
      const int c = w * 32 + lane;
      if (c >= pl) continue;  // (the line solver has no warp-wide step)
      const int s = c % S, v = c / S, x = v % nx, y = v / nx;
      LineCoef<double> cf;
      cf.S = S;
      cf.k0 = a.zk0;
      cf.inv = a.ztab + s;
      cf.mul = a.ztab + (size_t)nz * S + s;
      cf.q = a.ztab + 2 * (size_t)nz * S + s;
      cf.c0 = __ldg(a.zint + s);
      cf.c1 = __ldg(a.zint + S + s);
      cf.om = 1.0;
      cf.clo = 0.0;
      double val = 0.0;
      LineDir dr;
      dr.before = false;
      dr.after = face_value(s, val);
      dr.face = x == 0 || x == nx - 1 || y == 0 || y == ny - 1;
      solve_lines_f64<0>(a.rho + c, nz, (long long)pl, true, cf, dr, 0.0, val);
    }
    if (!grid_barrier(a.bar, a.status)) return;
  }
}

}  // namespace

size_t small_smem_bytes(int nx, int ny, int S) {
  return ((size_t)nx * ny * S + 2 * (size_t)(nx + ny) * S) * sizeof(double);
}

cudaError_t small_max_blocks(int *blocks_per_sm, size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(small_steps_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, small_steps_kernel,
                                                       kSmallThreads, smem);
}

cudaError_t launch_small_f64(const SmallArgs &a, int grid, size_t smem, cudaStream_t st) {
  SmallArgs args = a;
  void *params[] = {&args};
  return cudaLaunchCooperativeKernel((const void *)small_steps_kernel, dim3(grid),
                                     dim3(kSmallThreads), params, smem, st);
}

}  // namespace bfv
