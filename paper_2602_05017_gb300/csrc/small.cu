// Small grids (FP64): every step of a biofvm_step call in ONE cooperative,
// persistent launch.
//
// On a grid as small as 50^3 a step is latency-bound: each sweep kernel spends
// its time on the first loads of every line and on the serial Thomas chain,
// and three kernels per step add their launch and drain gaps.  Here one launch
// runs all the steps, with the stages of a step (Src, B, X^-1, B, Y^-1, B,
// Z^-1, B) and Algorithm 1 on the App. A system in its partitioned form: a
// line of n positions is cut into T chunks of m, each solved by one thread
// from a zero carry, and the carries between chunks come from the chunk end
// values (the same arithmetic as the partitioned sweeps of sweeps.cuh, in
// FP64).  An FP64 warp instruction occupies its scheduler's FP64 pipe for many
// cycles, so a dependent chain is slow: chunks cut the chains and spread the
// lines over all the warps of a CTA.
//
//   phase 1, per z-plane (CTA b takes planes b, b + G, ...): the plane is
//     loaded into shared memory, the source update and the Dirichlet
//     application before the x-solve are applied there, every x-line and every
//     y-line of the plane is solved there (thread = (line, chunk)), each
//     followed by its Dirichlet application, and the plane is stored back;
//   grid barrier;
//   phase 2, per group of 32 adjacent z-lines (CTA b takes groups b, b + G,
//     ...): the group is staged in shared memory ([z][32], coalesced), solved
//     (thread = (line, chunk)), the Dirichlet application after it applied on
//     the way back to the field;
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

#include <algorithm>

#include "internal.h"

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

// One axis's tables staged in shared memory: inv, mul, pf, pb [n][S] (the
// layout of the host's axis tables) and the carry weights cw [T][T][S].
struct ChunkTab {
  const double *inv, *mul, *pf, *pb, *cw;
};

__device__ ChunkTab stage_tab(double *dst, const double *src, int n, int S, int T) {
  const int blk = 4 * n * S;
  for (int i = threadIdx.x; i < blk; i += blockDim.x) dst[i] = __ldg(src + i);
  const double *gcw = src + blk + (size_t)T * S + 2 * (size_t)S;
  for (int i = threadIdx.x; i < T * T * S; i += blockDim.x) dst[blk + i] = __ldg(gcw + i);
  ChunkTab t;
  t.inv = dst;
  t.mul = dst + n * S;
  t.pf = dst + 2 * n * S;
  t.pb = dst + 3 * n * S;
  t.cw = dst + blk;
  return t;
}

__host__ __device__ inline int chunk_tab_elems(int n, int S, int T) { return 4 * n * S + T * T * S; }

// Partitioned solve of L lines of n positions held in shared memory: line l
// starts at q + base(l), position i is i*stride further on, its substrate is
// sub(l).  Lines are taken in batches of Lb = blockDim/T; in a batch thread
// (l, t) solves chunk t = positions [t*m, t*m + m) of its line from a zero
// carry (forward g_i = inv_i d_i + mul_i g_{i-1}, backward x_i = g_i + mul_i
// x_{i+1}), and the carries into each chunk, sums of the other chunks' end
// values weighted by products of their pf / pb ends (cw), correct it:
// g_i += pf_i * carry_in, x_i += pb_i * carry_out.  Every thread of the CTA
// calls it (barriers inside); s_end, s_beg hold blockDim doubles each.
template <typename Base, typename Sub>
__device__ void solve_chunked(double *q, int L, int T, int m, int n, int S, int stride,
                              Base base, Sub sub, const ChunkTab tb, double *s_end, double *s_beg) {
  const int Lb = (int)blockDim.x / T;
  for (int l0 = 0; l0 < L; l0 += Lb) {
    const int tid = threadIdx.x;
    const int lb = tid % Lb, t = tid / Lb, l = l0 + lb;
    const bool act = t < T && l < L;
    const int s = act ? sub(l) : 0;
    const int lo = t * m, hi = min(n, lo + m) - 1;
    double *p = q + (act ? base(l) : 0);
    double g = 0.0;
    if (act) {
      for (int i = lo; i <= hi; i++) {
        g = fma(tb.mul[i * S + s], g, tb.inv[i * S + s] * p[i * stride]);
        p[i * stride] = g;
      }
      s_end[t * Lb + lb] = g;
    }
    __syncthreads();
    if (act && t > 0) {
      double c = 0.0;
      for (int u = t - 1; u >= 0; u--) c = fma(tb.cw[(u * T + t) * S + s], s_end[u * Lb + lb], c);
      for (int i = lo; i <= hi; i++) p[i * stride] = fma(tb.pf[i * S + s], c, p[i * stride]);
    }
    double x = 0.0;
    if (act) {
      for (int i = hi; i >= lo; i--) {
        x = fma(tb.mul[i * S + s], x, p[i * stride]);
        p[i * stride] = x;
      }
      s_beg[t * Lb + lb] = x;
    }
    __syncthreads();
    if (act && t + 1 < T) {
      double c = 0.0;
      for (int u = t + 1; u < T; u++) c = fma(tb.cw[(u * T + t) * S + s], s_beg[u * Lb + lb], c);
      for (int i = lo; i <= hi; i++) p[i * stride] = fma(tb.pb[i * S + s], c, p[i * stride]);
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kSmallThreads, 1) small_steps_kernel(const SmallArgs a) {
  extern __shared__ __align__(16) double small_smem[];
  const int nx = a.nx, ny = a.ny, nz = a.nz, S = a.S;
  const int pl = nx * ny * S;  // elements of one z-plane
  const int buf_elems = max(pl, 32 * nz);
  double *buf = small_smem;
  double *tx = buf + buf_elems;
  double *ty = tx + chunk_tab_elems(nx, S, a.T[0]);
  double *tz = ty + chunk_tab_elems(ny, S, a.T[1]);
  double *s_end = tz + chunk_tab_elems(nz, S, a.T[2]);
  double *s_beg = s_end + kSmallThreads;
  const ChunkTab xt = stage_tab(tx, a.tab[0], nx, S, a.T[0]);
  const ChunkTab yt = stage_tab(ty, a.tab[1], ny, S, a.T[1]);
  const ChunkTab zt = stage_tab(tz, a.tab[2], nz, S, a.T[2]);
  __syncthreads();
  auto dir_on = [&](int s) { return a.any_dir && a.dir_on[s]; };
  // B on a plane in shared memory: the plane's face voxels of flagged substrates
  auto dirichlet_plane = [&](int z) {
    if (!a.any_dir) return;
    const bool zf = z == 0 || z == nz - 1;
    for (int e = threadIdx.x; e < pl; e += blockDim.x) {
      const int s = e % S, v = e / S, x = v % nx, y = v / nx;
      if ((zf || x == 0 || x == nx - 1 || y == 0 || y == ny - 1) && dir_on(s))
        buf[e] = __ldg(a.dir_val + s);
    }
    __syncthreads();
  };
  const int ngroups = (pl + 31) / 32;
  for (int step = 0; step < a.n_steps; step++) {
    // ---- phase 1: Src, B, X^-1, B, Y^-1, B on each z-plane in shared memory ----
    for (int z = blockIdx.x; z < nz; z += gridDim.x) {
      double *g = a.rho + (size_t)z * pl;
      for (int e = threadIdx.x; e < pl; e += blockDim.x) buf[e] = g[e];
      __syncthreads();
      if (a.has_src) {  // entries of the plane's rows: unique elements
        const long long e0 = a.src_row_off[(long long)z * ny];
        const long long e1 = a.src_row_off[(long long)z * ny + ny];
        for (long long k = e0 + threadIdx.x; k < e1; k += blockDim.x) {
          const long long off = a.src_elem[k] - (long long)z * pl;
          buf[off] = (buf[off] + __ldg(a.src_alpha + k)) * __ldg(a.src_scale + k);
        }
        __syncthreads();
      }
      dirichlet_plane(z);
      // x-lines: line l = (y, s), positions S apart
      solve_chunked(buf, ny * S, a.T[0], a.m[0], nx, S, S,
                    [&](int l) { return (l / S) * nx * S + l % S; }, [&](int l) { return l % S; },
                    xt, s_end, s_beg);
      dirichlet_plane(z);
      // y-lines: line l = (x, s), positions nx*S apart
      solve_chunked(buf, nx * S, a.T[1], a.m[1], ny, S, nx * S, [&](int l) { return l; },
                    [&](int l) { return l % S; }, yt, s_end, s_beg);
      dirichlet_plane(z);
      for (int e = threadIdx.x; e < pl; e += blockDim.x) g[e] = buf[e];
      __syncthreads();
    }
    if (!grid_barrier(a.bar, a.status)) return;
    // ---- phase 2: Z^-1 then B on groups of 32 adjacent z-lines staged as [z][32] ----
    for (int gi = blockIdx.x; gi < ngroups; gi += gridDim.x) {
      const int c0 = gi * 32, ncol = min(32, pl - c0);
      for (int e = threadIdx.x; e < nz * 32; e += blockDim.x) {
        const int z = e >> 5, c = e & 31;
        buf[e] = c < ncol ? a.rho[(size_t)z * pl + c0 + c] : 0.0;
      }
      __syncthreads();
      solve_chunked(buf, 32, a.T[2], a.m[2], nz, S, 32, [&](int l) { return l; },
                    [&](int l) { return (c0 + l) % S; }, zt, s_end, s_beg);
      for (int e = threadIdx.x; e < nz * 32; e += blockDim.x) {
        const int z = e >> 5, c = e & 31;
        if (c >= ncol) continue;
        const int col = c0 + c, s = col % S, v = col / S, x = v % nx, y = v / nx;
        double val = buf[e];
        if (dir_on(s) && (z == 0 || z == nz - 1 || x == 0 || x == nx - 1 || y == 0 || y == ny - 1))
          val = __ldg(a.dir_val + s);
        a.rho[(size_t)z * pl + col] = val;
      }
      __syncthreads();
    }
    if (!grid_barrier(a.bar, a.status)) return;
  }
}

}  // namespace

// Chunks per axis for lines of n positions, L lines at once (x: ny*S, y: nx*S,
// z: 32 per group): as many as fit beside the lines in one CTA, at least two
// positions each.
int small_chunks(int n, int L) {
  const int fit = std::max(1, kSmallThreads / std::max(1, L));
  return std::max(1, std::min(fit, (n + 1) / 2));
}

size_t small_smem_bytes(int nx, int ny, int nz, int S, const int T[3]) {
  const size_t pl = (size_t)nx * ny * S;
  const size_t buf = std::max(pl, (size_t)32 * nz);
  return (buf + chunk_tab_elems(nx, S, T[0]) + chunk_tab_elems(ny, S, T[1]) +
          chunk_tab_elems(nz, S, T[2]) + 2 * (size_t)kSmallThreads) * sizeof(double);
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
