// Batched LOD steps: many independent microenvironments of uneven size and
// substrate count advanced by ONE persistent launch (all environments, all
// steps).
//
// Work items are tiles of 32 independent lines of one sweep of one
// environment, in the order (step, phase x/y/z, environment, tile).  CTA b
// takes items b, b + G, b + 2G, ... (G = gridDim.x, every CTA resident).
// Before an item, its dependency on the previous phase of the same
// environment is checked on a per-(phase, environment) completion counter:
//     x of step k   needs all z tiles of step k-1 (k > 0)
//     y of step k   needs all x tiles of step k
//     z of step k   needs all y tiles of step k
// An item only ever waits on items earlier in the order, and the earliest
// unfinished item never waits, so the persistent grid cannot deadlock.  Every
// wait is bounded (about two seconds); on a timeout the status word is set
// and an abort flag makes every CTA stop at its next item.
//
// Tiles read and write the field directly (lines in registers, chunk carries
// through shared memory), with the arithmetic of the single-grid kernels:
// partitioned Thomas on the App. A system, FP32 in defect-correction form,
// the source update applied to an x tile's rows before its solve.  Zero-flux
// boundaries (the batched microenvironments have no Dirichlet faces).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "batch_args.h"
#include "sweeps.cuh"

namespace bfv {

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_relaxed_int(const int *p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

template <typename E, int MAXM>
__global__ void __launch_bounds__(kBatchWarps * 32) batch_kernel(const BatchArgs a) {
  __shared__ E s_end[kBatchWarps * 32], s_beg[kBatchWarps * 32];
  __shared__ int s_go;
  const int lane = threadIdx.x & 31, t = threadIdx.x >> 5;
  const int64_t total = a.per_step * a.n_steps;
  int last_env = -1, last_phase = -1, last_step = -1;  // last dependency known satisfied
  for (int64_t g = blockIdx.x; g < total; g += gridDim.x) {
    const int step = (int)(g / a.per_step);
    int64_t r = g - (int64_t)step * a.per_step;
    int phase = 0;
    while (phase < 2 && r >= a.tile_off[phase * (a.n_env + 1) + a.n_env]) {
      r -= a.tile_off[phase * (a.n_env + 1) + a.n_env];
      phase++;
    }
    const int64_t *off = a.tile_off + phase * (a.n_env + 1);
    int lo_e = 0, hi_e = a.n_env - 1;  // environment: last e with off[e] <= r
    while (lo_e < hi_e) {
      const int mid = (lo_e + hi_e + 1) >> 1;
      if (off[mid] <= r) lo_e = mid; else hi_e = mid - 1;
    }
    const int ei = lo_e;
    const int64_t tile = r - off[ei];
    const BatchEnv &E_ = a.env[ei];

    // ---- dependency on the previous phase of this environment ----
    if (threadIdx.x == 0) {
      int go = 1;
      if (ld_relaxed_int(a.abort_flag)) go = 0;
      const bool need = !(ei == last_env && phase == last_phase && step == last_step) &&
                        !(phase == 0 && step == 0);
      if (go && need) {
        const int dep_phase = phase == 0 ? 2 : phase - 1;
        unsigned want = (unsigned)(E_.tiles[dep_phase] * (phase == 0 ? step : step + 1));
        if (a.stall_test && phase == 1 && step == 0 && ei == 0 && tile == 0) want = 0xffffffffu;
        const unsigned *ctr = a.done + dep_phase * a.n_env + ei;
        const long long t0 = clock64();
        while (ld_acquire(ctr) < want) {
          if (ld_relaxed_int(a.abort_flag)) {
            go = 0;
            break;
          }
          if (clock64() - t0 > (1ll << 32)) {
            atomicExch(a.status, kStatusTimeout);
            atomicExch(a.abort_flag, 1);
            go = 0;
            break;
          }
          __nanosleep(64);
        }
      }
      s_go = go;
    }
    __syncthreads();
    if (!s_go) return;
    last_env = ei;
    last_phase = phase;
    last_step = step;

    // ---- geometry of the 32 lines of this tile ----
    const int S = E_.S, nx = E_.nx, ny = E_.ny;
    const int n = phase == 0 ? nx : phase == 1 ? ny : E_.nz;
    const int T = E_.T[phase], m = E_.m[phase];
    E *const field = static_cast<E *>(E_.field);
    const int64_t rowlen = (int64_t)nx * S;
    long long base = 0, pstride;
    bool active;
    int s;
    if (phase == 0) {
      const int64_t r0 = tile * E_.rows_per_tile;
      const int64_t nrows = (int64_t)ny * E_.nz;
      const int rows = (int)min((int64_t)E_.rows_per_tile, nrows - r0);
      // Src on this tile's rows (only this CTA touches them in this phase)
      if (E_.has_src) {
        const int64_t e0 = E_.src_row_off[r0], e1 = E_.src_row_off[r0 + rows];
        for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
          const int64_t el = E_.src_elem[e];
          field[el] = (field[el] + ldg<E>(E_.src_alpha, e)) * ldg<E>(E_.src_scale, e);
        }
        __syncthreads();
      }
      s = lane % S;
      active = lane < E_.rows_per_tile * S && lane / S < rows;
      base = (r0 + lane / S) * rowlen + s;
      pstride = S;
    } else {
      const int64_t C = phase == 1 ? rowlen : rowlen * ny;
      const int64_t tpp = (C + 31) / 32;
      const int64_t plane = tile / tpp;
      const int64_t c = (tile - plane * tpp) * 32 + lane;
      active = c < C;
      s = (int)(c % S);
      base = plane * C * n + c;
      pstride = C;
    }
    const int lo = t * m;
    const int len = (active && t < T) ? min(m, n - lo) : 0;
    E *col = field + (active ? base : 0);
    const E *tb = static_cast<const E *>(E_.tab[phase]);
    const E *T_inv = tb, *T_mul = tb + n * S, *T_pf = T_mul + n * S, *T_pb = T_pf + n * S;
    const E *T_pc = T_pb + n * S, *T_cfix = T_pc + T * S;

    E v[MAXM];
#pragma unroll
    for (int i = 0; i < MAXM; i++)
      if (i < len) v[i] = col[(lo + i) * pstride];
    if constexpr (kDefect<E>) {
      E prev = (len > 0 && lo > 0) ? col[(lo - 1) * pstride] : E(0);
      const E after = (len > 0 && lo + len < n) ? col[(lo + len) * pstride] : E(0);
#pragma unroll
      for (int i = 0; i < MAXM; i++)
        if (i < len) {
          const E cur = v[i];
          const E nxt = (i + 1 < MAXM && i + 1 < len) ? v[i + 1] : after;
          v[i] = second_difference(cur, prev, nxt, lo + i, n);
          prev = cur;
        }
    }
    E gcar = E(0);
#pragma unroll
    for (int i = 0; i < MAXM; i++)
      if (i < len) {
        const int q = (lo + i) * S + s;
        gcar = fma(__ldg(T_mul + q), gcar, v[i] * __ldg(T_inv + q));
        v[i] = gcar;
      }
    s_end[t * 32 + lane] = gcar;
    __syncthreads();
    const E *T_cw = T_cfix + 2 * S;  // [T][T][S]
    E carry = E(0);
    if (t < T)
      for (int u = t - 1; u >= 0; u--)
        carry = fma(__ldg(T_cw + (u * T + t) * S + s), s_end[u * 32 + lane], carry);
#pragma unroll
    for (int i = 0; i < MAXM; i++)
      if (i < len) v[i] = fma(__ldg(T_pf + (lo + i) * S + s), carry, v[i]);
    E xcar = E(0);
#pragma unroll
    for (int i = MAXM - 1; i >= 0; i--)
      if (i < len) {
        xcar = fma(__ldg(T_mul + (lo + i) * S + s), xcar, v[i]);
        v[i] = xcar;
      }
    s_beg[t * 32 + lane] = xcar;
    __syncthreads();
    carry = E(0);
    if (t < T)
      for (int u = t + 1; u < T; u++)
        carry = fma(__ldg(T_cw + (u * T + t) * S + s), s_beg[u * 32 + lane], carry);
#pragma unroll
    for (int i = 0; i < MAXM; i++)
      if (i < len) v[i] = fma(__ldg(T_pb + (lo + i) * S + s), carry, v[i]);
    if constexpr (kDefect<E>) {
      const E chi = __ldg(T_cfix + s), clo = __ldg(T_cfix + S + s);
#pragma unroll
      for (int i = 0; i < MAXM; i++)
        if (i < len) {
          const E d = col[(lo + i) * pstride];
          v[i] = fma(chi, d, fma(clo, d, v[i]));
        }
    }
    __syncthreads();  // every halo read of the tile precedes every write
#pragma unroll
    for (int i = 0; i < MAXM; i++)
      if (i < len) col[(lo + i) * pstride] = v[i];
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(a.done + phase * a.n_env + ei, 1u);
    }
  }
}

template <typename E, int MAXM>
cudaError_t launch_batch_one(const BatchArgs &a, int grid, cudaStream_t st) {
  batch_kernel<E, MAXM><<<grid, kBatchWarps * 32, 0, st>>>(a);
  return cudaGetLastError();
}

template <typename E, int MAXM>
cudaError_t batch_blocks_per_sm(int *out) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, batch_kernel<E, MAXM>, kBatchWarps * 32, 0);
}

}  // namespace bfv
