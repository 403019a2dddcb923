// Sweep kernels of the LOD diffusion-decay step for sm_103a.
//
// Every line solve is the Thomas algorithm of the paper (Sect. 2.1,
// Algorithm 1) on the constant-coefficient system of Appendix A, written with
// the precomputed constants inv_i = 1/denom_i and mul_i = r/denom_i:
//     forward   g_i = d_i*inv_i + mul_i*g_{i-1}        (g_{-1} = 0)
//     backward  x_i = g_i + mul_i*x_{i+1}              (x_n = 0)
// Both recurrences are affine in their carry, so a line can be cut into T
// chunks solved by T threads at once (partitioned / divide-and-conquer
// Thomas, the single-system parallelisation the paper cites in Sect. 2):
// each thread runs the recurrence over its chunk from a zero carry, the true
// carry entering each chunk is the composition of the earlier chunks' affine
// maps (a scan), and a chunk's values are corrected by the carry times the
// precomputed product of multipliers (pf, pb).  The result is Thomas's, in
// a different rounding order.  Each thread keeps its chunk in registers, so
// the field is read once and written once per sweep.
//
// x-sweep (lines along the contiguous axis, element stride S): a CTA stages
// rows_per_cta consecutive rows -- one contiguous block of memory -- into
// shared memory with one cp.async.bulk (TMA bulk copy, completion on an
// mbarrier), applies the source update and the first Dirichlet application
// there, solves with lanes (segment t, substrate s) of a warp and a
// shuffle-based scan across segments, applies the second Dirichlet
// application, and writes the block back with one bulk store.
//
// y- and z-sweeps (lines across planes): consecutive threads own consecutive
// columns, so every load and store of the recurrence is one coalesced
// 128-byte (FP32) or 256-byte (FP64) row segment per warp; the T warps of a
// CTA own the T chunks of the same 32 columns and exchange chunk carries
// through shared memory.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace bfv {

// ----------------------------------------------------------------------------
// PTX helpers (mbarrier, bulk async copies).
// ----------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ void bulk_s2g(void *dst, const void *src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
               "r"(smem_addr(src)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// Bounded wait on an mbarrier phase: gives up after ~2^31 cycles (about one
// second at GB300 clocks), records kStatusTimeout and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int *status) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > (1ll << 31)) {
      atomicExch(status, kStatusTimeout);
      return false;
    }
  }
  return true;
}

template <typename E>
__device__ __forceinline__ E ldg(const void *p, long long i) {
  return __ldg(static_cast<const E *>(p) + i);
}

// Value a Dirichlet application writes: the substrate's value, or 0 for the
// adjoint mask.
template <typename E>
__device__ __forceinline__ E dir_value(int flags, const void *dir_val, int s) {
  return (flags & kMaskZero) ? E(0) : ldg<E>(dir_val, s);
}

// FP32 kernels solve in defect-correction form (see AxisTab); FP64 solves
// the plain system.
template <typename E>
constexpr bool kDefect = sizeof(E) == 4;

// (L_N d)_j on an axis of n voxels with zero-flux ends: the FVM flux balance
// (d_j - d_{j-1}) + (d_j - d_{j+1}), one-sided at the two ends, 0 when n = 1.
template <typename E>
__device__ __forceinline__ E second_difference(E cur, E prev, E next, int j, int n) {
  if (n == 1) return E(0);
  if (j == 0) return cur - next;
  if (j == n - 1) return cur - prev;
  return (cur - prev) + (cur - next);
}

// ----------------------------------------------------------------------------
// x-sweep with the source update and two Dirichlet applications fused.
// ----------------------------------------------------------------------------
template <typename E, int MAXM>
__global__ void __launch_bounds__(256) x_sweep_kernel(const XLaunch a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int S = a.S, nx = a.nx;
  const int rowlen = nx * S;
  const int T = a.tab.T, m = a.tab.m;
  const long long nrows_total = (long long)a.ny * a.nz;
  const long long row0 = (long long)blockIdx.x * a.rows_per_cta;
  const int nrows = (int)min((long long)a.rows_per_cta, nrows_total - row0);
  const int tid = threadIdx.x, nthr = blockDim.x;

  E *tile = reinterpret_cast<E *>(smem_raw);
  E *t_inv = tile + (size_t)a.rows_per_cta * rowlen;
  E *t_mul = t_inv + rowlen;
  E *t_pf = t_mul + rowlen;
  E *t_pb = t_pf + rowlen;
  E *t_pc = t_pb + rowlen;
  uint64_t *bar = reinterpret_cast<uint64_t *>(
      (reinterpret_cast<uintptr_t>(t_pc + T * S) + 15) & ~uintptr_t(15));

  E *g_tile = static_cast<E *>(a.rho) + row0 * rowlen;
  const uint32_t bytes = (uint32_t)((size_t)nrows * rowlen * sizeof(E));

  // 1. stage the rows: one bulk copy when rows are 16-byte multiples
  if (a.use_bulk) {
    if (tid == 0) {
      mbar_init(bar, 1);
      fence_mbar_init();
      fence_proxy_async_smem();
    }
    __syncthreads();
    if (tid == 0) {
      mbar_arrive_expect_tx(bar, bytes);
      bulk_g2s(tile, g_tile, bytes, bar);
    }
  } else {
    for (int i = tid; i < nrows * rowlen; i += nthr) tile[i] = g_tile[i];
  }
  // 2. the axis constants (overlaps the bulk copy)
  if (a.flags & kSolve) {
    for (int i = tid; i < rowlen; i += nthr) {
      t_inv[i] = ldg<E>(a.tab.inv, i);
      t_mul[i] = ldg<E>(a.tab.mul, i);
      t_pf[i] = ldg<E>(a.tab.pf, i);
      t_pb[i] = ldg<E>(a.tab.pb, i);
    }
    for (int i = tid; i < T * S; i += nthr) t_pc[i] = ldg<E>(a.tab.pc, i);
  }
  bool ok = true;
  if (a.use_bulk) ok = mbar_wait_bounded(bar, 0, a.status);
  ok = __syncthreads_and(ok);
  if (!ok) {  // copy never completed: wait once more (bounded), write nothing
    if (a.use_bulk) mbar_wait_bounded(bar, 0, a.status);
    return;
  }

  // 3. Src: rho <- (rho + alpha) * 1/(1 + beta) on this block's entries
  if ((a.flags & kSrc) && a.has_src) {
    const long long e0 = a.src_row_off[row0], e1 = a.src_row_off[row0 + nrows];
    const long long base = row0 * rowlen;
    for (long long e = e0 + tid; e < e1; e += nthr) {
      const int off = (int)(a.src_elem[e] - base);
      tile[off] = (tile[off] + ldg<E>(a.src_alpha, e)) * ldg<E>(a.src_scale, e);
    }
    __syncthreads();
  }
  const int warp = tid >> 5, lane = tid & 31, nwarps = nthr >> 5;
  // 4. B before the solve (rows on a y/z face: whole row; others: x = 0, nx-1)
  if (a.flags & kDirBefore) {
    for (int r = warp; r < nrows; r += nwarps) {
      const long long row = row0 + r;
      const int y = (int)(row % a.ny), z = (int)(row / a.ny);
      const bool face = (y == 0 || y == a.ny - 1 || z == 0 || z == a.nz - 1);
      E *tr = tile + (size_t)r * rowlen;
      if (face) {
        for (int k = lane; k < rowlen; k += 32) {
          const int s = k % S;
          if (a.dir_on[s]) tr[k] = dir_value<E>(a.flags, a.dir_val, s);
        }
      } else {
        for (int k = lane; k < 2 * S; k += 32) {
          const int s = k % S;
          const int idx = (k < S) ? s : (nx - 1) * S + s;
          if (a.dir_on[s]) tr[idx] = dir_value<E>(a.flags, a.dir_val, s);
        }
      }
    }
    __syncthreads();
  }

  // 5. Thomas along x: lanes (row lr, segment t, substrate s), s fastest
  if (a.flags & kSolve) {
    const int G = T * S;
    const int lr = lane / G, q = lane - lr * G;
    const int t = q / S, s = q - t * S;
    const int r = warp * a.rows_per_warp + lr;
    const bool active = (lr < a.rows_per_warp) && (r < nrows);
    const int lo = t * m;
    const int len = active ? min(m, nx - lo) : 0;
    E *line = tile + (size_t)(active ? r : 0) * rowlen + s;
    E v[MAXM];
#pragma unroll
    for (int i = 0; i < MAXM; i++)
      if (i < len) v[i] = line[(lo + i) * S];
    if constexpr (kDefect<E>) {
      // right-hand side of the correction: e = L_N d (zero-flux second
      // difference), in place; the halo comes from the staged row
      E prev = (len > 0 && lo > 0) ? line[(lo - 1) * S] : E(0);
      const E after = (len > 0 && lo + len < nx) ? line[(lo + len) * S] : E(0);
#pragma unroll
      for (int i = 0; i < MAXM; i++)
        if (i < len) {
          const int j = lo + i;
          const E cur = v[i];
          const E nxt = (i + 1 < MAXM && i + 1 < len) ? v[i + 1] : after;
          v[i] = second_difference(cur, prev, nxt, j, nx);
          prev = cur;
        }
    }
    // forward elimination over the chunk from a zero carry
    E g = E(0);
#pragma unroll
    for (int i = 0; i < MAXM; i++)
      if (i < len) {
        const int k = (lo + i) * S + s;
        g = fma(t_mul[k], g, v[i] * t_inv[k]);
        v[i] = g;
      }
    // inclusive scan of the chunks' affine maps g -> pc*g + g_end
    const unsigned FULL = 0xffffffffu;
    E A = (len > 0) ? t_pc[t * S + s] : E(1), B = g;
    for (int d = 1; d < T; d <<= 1) {
      const E A2 = __shfl_up_sync(FULL, A, d * S);
      const E B2 = __shfl_up_sync(FULL, B, d * S);
      if (t >= d) {
        B = fma(A, B2, B);
        A = A * A2;
      }
    }
    E carry = __shfl_up_sync(FULL, B, S);
    if (t == 0) carry = E(0);
    // forward correction, then back substitution from a zero carry
#pragma unroll
    for (int i = 0; i < MAXM; i++)
      if (i < len) v[i] = fma(t_pf[(lo + i) * S + s], carry, v[i]);
    E x = E(0);
#pragma unroll
    for (int i = MAXM - 1; i >= 0; i--)
      if (i < len) {
        x = fma(t_mul[(lo + i) * S + s], x, v[i]);
        v[i] = x;
      }
    A = (len > 0) ? t_pc[t * S + s] : E(1);
    B = x;
    for (int d = 1; d < T; d <<= 1) {
      const E A2 = __shfl_down_sync(FULL, A, d * S);
      const E B2 = __shfl_down_sync(FULL, B, d * S);
      if (t + d < T) {
        B = fma(A, B2, B);
        A = A * A2;
      }
    }
    carry = __shfl_down_sync(FULL, B, S);
    if (t == T - 1) carry = E(0);
#pragma unroll
    for (int i = 0; i < MAXM; i++)
      if (i < len) v[i] = fma(t_pb[(lo + i) * S + s], carry, v[i]);
    if constexpr (kDefect<E>) {  // x = c_hi d + (c_lo d + y), one final rounding
      const E chi = ldg<E>(a.tab.cfix, s), clo = ldg<E>(a.tab.cfix, S + s);
#pragma unroll
      for (int i = 0; i < MAXM; i++)
        if (i < len) {
          const E d = line[(lo + i) * S];
          v[i] = fma(chi, d, fma(clo, d, v[i]));
        }
    }
    __syncwarp();  // every lane of the row has read its halo before any write-back
    // B after the solve, in registers
    if ((a.flags & kDirAfter) && active && a.dir_on[s]) {
      const long long row = row0 + r;
      const int y = (int)(row % a.ny), z = (int)(row / a.ny);
      const E val = dir_value<E>(a.flags, a.dir_val, s);
      if (y == 0 || y == a.ny - 1 || z == 0 || z == a.nz - 1) {
#pragma unroll
        for (int i = 0; i < MAXM; i++)
          if (i < len) v[i] = val;
      } else {
        if (lo == 0) v[0] = val;
#pragma unroll
        for (int i = 0; i < MAXM; i++)
          if (i < len && lo + i == nx - 1) v[i] = val;
      }
    }
#pragma unroll
    for (int i = 0; i < MAXM; i++)
      if (i < len) line[(lo + i) * S] = v[i];
  } else if (a.flags & kDirAfter) {
    // B alone (no solve): same rule as before the solve
    for (int r = warp; r < nrows; r += nwarps) {
      const long long row = row0 + r;
      const int y = (int)(row % a.ny), z = (int)(row / a.ny);
      const bool face = (y == 0 || y == a.ny - 1 || z == 0 || z == a.nz - 1);
      E *tr = tile + (size_t)r * rowlen;
      for (int k = lane; k < rowlen; k += 32) {
        const int s = k % S, x = k / S;
        if (a.dir_on[s] && (face || x == 0 || x == nx - 1)) tr[k] = dir_value<E>(a.flags, a.dir_val, s);
      }
    }
  }
  __syncthreads();

  // 6. write the rows back
  if (a.use_bulk) {
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      bulk_s2g(g_tile, tile, bytes);
      bulk_commit();
      bulk_wait_all();
    }
  } else {
    for (int i = tid; i < nrows * rowlen; i += nthr) g_tile[i] = tile[i];
  }
}

// ----------------------------------------------------------------------------
// y- / z-sweep: columns of a plane, T warps = T chunks of the same 32 columns.
// ----------------------------------------------------------------------------
// Largest CTA (threads) a column sweep with chunk capacity MAXM may use: the
// chunk takes MAXM*sizeof(E)/4 registers, about 40 more go to addressing.
template <typename E, int MAXM>
struct ColBound {
  static constexpr int regs = MAXM * (int)sizeof(E) / 4 + 64;
  static constexpr int raw = 65536 / regs;
  static constexpr int threads = (raw >= 1024 ? 1024 : raw) / 32 * 32;
};

template <typename E, int MAXM>
__global__ void __launch_bounds__(ColBound<E, MAXM>::threads) col_sweep_kernel(const ColLaunch a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  E *s_end = reinterpret_cast<E *>(smem_raw);  // [T][32] forward chunk ends
  E *s_beg = s_end + a.tab.T * 32;             // [T][32] backward chunk starts
  const int lane = threadIdx.x, t = threadIdx.y;
  const int T = a.tab.T, m = a.tab.m, n = a.n, S = a.S;
  const long long c = (long long)blockIdx.x * 32 + lane;
  const bool active = c < a.C;
  const int s = (int)(c % S);
  const int lo = t * m;
  const int len = active ? min(m, n - lo) : 0;
  E *col = static_cast<E *>(a.rho) + (long long)blockIdx.y * a.plane_stride + (active ? c : 0);
  const long long C = a.C;

  E v[MAXM];
#pragma unroll
  for (int i = 0; i < MAXM; i++)
    if (i < len) v[i] = col[(long long)(lo + i) * C];
  if constexpr (kDefect<E>) {
    // e = L_N d in place; halo values are read from the neighbouring chunks'
    // rows (not yet overwritten: every thread writes its own rows last)
    E prev = (len > 0 && lo > 0) ? col[(long long)(lo - 1) * C] : E(0);
    const E after = (len > 0 && lo + len < n) ? col[(long long)(lo + len) * C] : E(0);
#pragma unroll
    for (int i = 0; i < MAXM; i++)
      if (i < len) {
        const E cur = v[i];
        const E nxt = (i + 1 < MAXM && i + 1 < len) ? v[i + 1] : after;
        v[i] = second_difference(cur, prev, nxt, lo + i, n);
        prev = cur;
      }
  }
  E g = E(0);
#pragma unroll
  for (int i = 0; i < MAXM; i++)
    if (i < len) {
      const int k = (lo + i) * S + s;
      g = fma(ldg<E>(a.tab.mul, k), g, v[i] * ldg<E>(a.tab.inv, k));
      v[i] = g;
    }
  s_end[t * 32 + lane] = g;
  __syncthreads();
  // carry into chunk t: sum_{u<t} cw[u][t] * end_u
  E carry = E(0);
  for (int u = t - 1; u >= 0; u--)
    carry = fma(ldg<E>(a.tab.cw, (u * T + t) * S + s), s_end[u * 32 + lane], carry);
#pragma unroll
  for (int i = 0; i < MAXM; i++)
    if (i < len) v[i] = fma(ldg<E>(a.tab.pf, (lo + i) * S + s), carry, v[i]);
  E x = E(0);
#pragma unroll
  for (int i = MAXM - 1; i >= 0; i--)
    if (i < len) {
      x = fma(ldg<E>(a.tab.mul, (lo + i) * S + s), x, v[i]);
      v[i] = x;
    }
  s_beg[t * 32 + lane] = x;
  __syncthreads();
  carry = E(0);
  for (int u = t + 1; u < T; u++)
    carry = fma(ldg<E>(a.tab.cw, (u * T + t) * S + s), s_beg[u * 32 + lane], carry);
#pragma unroll
  for (int i = 0; i < MAXM; i++)
    if (i < len) v[i] = fma(ldg<E>(a.tab.pb, (lo + i) * S + s), carry, v[i]);
  if constexpr (kDefect<E>) {  // x = c_hi d + (c_lo d + y), one final rounding
    const E chi = ldg<E>(a.tab.cfix, s), clo = ldg<E>(a.tab.cfix, S + s);
#pragma unroll
    for (int i = 0; i < MAXM; i++)
      if (i < len) {
        const E d = col[(long long)(lo + i) * C];  // the right-hand side (L2-resident)
        v[i] = fma(chi, d, fma(clo, d, v[i]));
      }
  }

  if ((a.flags & kDirAfter) && len > 0 && a.dir_on[s]) {
    bool face;
    if (a.mode == 1) {
      const int x0 = (int)(c / S), z = blockIdx.y;
      face = (x0 == 0 || x0 == a.nx - 1 || z == 0 || z == a.nz - 1);
    } else {
      const long long vox = c / S;
      const int x0 = (int)(vox % a.nx), y = (int)(vox / a.nx);
      face = (x0 == 0 || x0 == a.nx - 1 || y == 0 || y == a.ny - 1);
    }
    const E val = dir_value<E>(a.flags, a.dir_val, s);
#pragma unroll
    for (int i = 0; i < MAXM; i++)
      if (i < len && (face || lo + i == 0 || lo + i == n - 1)) v[i] = val;
  }
#pragma unroll
  for (int i = 0; i < MAXM; i++)
    if (i < len) col[(long long)(lo + i) * C] = v[i];
}

// ----------------------------------------------------------------------------
// Dirichlet nodes (the listed part of every Dirichlet application): one thread
// per node, grid-strided.  The elements are unique, so the writes never meet.
// ----------------------------------------------------------------------------
template <typename E>
__global__ void __launch_bounds__(256) dirichlet_nodes_kernel(const NodeLaunch a) {
  E *rho = static_cast<E *>(a.rho);
  const E *val = static_cast<const E *>(a.val), *scale = static_cast<const E *>(a.scale);
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < a.n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = __ldg(a.elem + k);
    rho[e] = a.zero ? E(0) : scale ? __ldg(val + k) * __ldg(scale + e % a.S) : __ldg(val + k);
  }
}

template <typename E>
cudaError_t launch_nodes_one(const NodeLaunch &a, cudaStream_t st) {
  if (a.n <= 0) return cudaSuccess;
  dirichlet_nodes_kernel<E><<<a.grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Dispatch on the register-chunk capacity.
// ----------------------------------------------------------------------------
template <typename E, int MAXM>
cudaError_t allow_x_smem(size_t bytes) {
  return cudaFuncSetAttribute(x_sweep_kernel<E, MAXM>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename E, int MAXM>
cudaError_t launch_x_one(const XLaunch &a, cudaStream_t st) {
  auto k = x_sweep_kernel<E, MAXM>;
  const long long rows = (long long)a.ny * a.nz;
  const unsigned grid = (unsigned)((rows + a.rows_per_cta - 1) / a.rows_per_cta);
  k<<<grid, a.warps * 32, a.smem_bytes, st>>>(a);
  return cudaGetLastError();
}

template <typename E, int MAXM>
cudaError_t launch_col_one(const ColLaunch &a, cudaStream_t st) {
  auto k = col_sweep_kernel<E, MAXM>;
  if (a.tab.T * 32 > ColBound<E, MAXM>::threads) return cudaErrorInvalidConfiguration;
  const size_t smem = 2 * (size_t)a.tab.T * 32 * sizeof(E);
  dim3 grid((unsigned)((a.C + 31) / 32), (unsigned)a.nplanes);
  dim3 block(32, (unsigned)a.tab.T);
  k<<<grid, block, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace bfv
