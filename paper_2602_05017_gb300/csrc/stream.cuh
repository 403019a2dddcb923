// Streaming line sweep: one lane owns one whole grid line.
//
// The FP64 pipe of a GB300 SM retires two FMAs per clock, so the FP64 step is
// bound by its FP64 operations, not by HBM.  Cutting a line into chunks (the
// partitioned solve of the other kernels) costs carry corrections on top of
// the three operations per element that the Thomas algorithm (App. A) needs;
// this kernel does not cut lines at all.  Written in the scaled form
//
//   forward   h_0 = d_0,  h_i = d_i + mul_{i-1} h_{i-1}    (h_i = d'_i / inv_i)
//   backward  x_{n-1} = inv_{n-1} h_{n-1},  x_i = inv_i h_i + mul_i x_{i+1}
//
// (mul_i = r inv_i = -c'_i), each recurrence carries one FMA per element
// along its dependency chain; the product inv_i h_i is off the chain.
//
// Scaled output (OUT 1, 2; the three sweeps of a whole step).  Away from the
// first few positions inv_i equals its interior limit sigma to the last bit,
// so the solve is run for y = x / sigma:
//   y_{n-1} = q_{n-1} h_{n-1},  y_i = q_i h_i + mul_i y_{i+1},  q_i = inv_i / sigma,
// with q_i = 1 (no multiply) from position k0 on.  The next sweep is linear,
// so the factor passes through it untouched; the x- and y-sweeps store y
// (OUT 1) and the z-sweep stores omega y with omega = sigma_x sigma_y sigma_z
// (OUT 2), the true field.  A step then costs about 7 FP64 operations per
// element instead of 9.  Dirichlet values are passed in the same units.
//
// Interior constants.  On [k0, n-1) the tables hold exactly inv = sigma and
// mul = r sigma (q = 1), so a group of positions inside that range runs on
// two per-substrate registers and loads no table entry.
//
// Memory.  The forward pass writes h back in place; the backward pass follows
// at once and reads it in reverse order, so h mostly stays in L2 between the
// two passes.  Two ways of keeping loads in flight (PF):
//   PF = G > 1  each lane prefetches its own line through a private ring of G
//         groups of 8 positions in shared memory (cp.async, 8 bytes per lane
//         and position): few registers, 8 (G-1) positions in flight per lane;
//   PF = 1  two register blocks of 16 positions (the next block loads while
//         the current one is solved): 16 to 32 positions in flight, many
//         registers.
//
// Lanes:  x-sweep  lane = (row, substrate), rows of nx*S elements, 32/S rows
//                  per warp; the warp owns whole rows, so it also applies the
//                  source update of those rows before its solve;
//         y/z      lane = one of 32 consecutive columns of a plane (a row of a
//                  warp is one 32-element coalesced access).
// Tables: inv, mul, q position-major [3][n][S], read through L1 (the S values
// a warp reads at one position share a cache line).
#pragma once
#include "sweeps.cuh"

namespace bfv {

constexpr int kStreamThreads = 128;
// PF 0 (cp.async ring of PF groups of 8 positions) or 1 (register blocks)
template <int PF>
struct StreamCfg {
  static constexpr int R = PF == 1 ? 16 : 8;   // positions per group
  static constexpr int G = PF == 1 ? 1 : PF;   // ring groups
  static constexpr int ctas = PF == 1 ? 3 : 8; // CTAs per SM the registers must allow
};

__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(smem)), "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <typename E, int PF, int OUT>
__global__ void __launch_bounds__(kStreamThreads, StreamCfg<PF>::ctas)
    stream_sweep_kernel(const StreamArgs a) {
  constexpr int R = StreamCfg<PF>::R, G = StreamCfg<PF>::G;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int S = a.S, n = a.n, flags = a.flags, k0 = a.k0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // PF 0: this lane's ring, [G][R] slots 32 elements apart (conflict-free)
  E *ring = reinterpret_cast<E *>(smem_raw) + (size_t)warp * G * R * 32 + lane;
  const E *tinv = static_cast<const E *>(a.tab);
  const E *tmul = tinv + (size_t)n * S, *tq = tmul + (size_t)n * S;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long nrows = (long long)a.ny * a.nz;
  E *const rho = static_cast<E *>(a.rho);
  const long long st = a.stride;
  const int ngrp = (n + R - 1) / R;

  for (long long grp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; grp < a.ngroups;
       grp += nwarps) {
    bool active, face;
    int s;
    long long base;
    if (a.mode == 0) {
      const int RW = a.rows_per_warp;
      const int lr = lane / S;
      s = lane - lr * S;
      const long long row = grp * RW + lr;
      active = lr < RW && row < nrows;
      const int y = (int)(row % a.ny), z = (int)(row / a.ny);
      face = y == 0 || y == a.ny - 1 || z == 0 || z == a.nz - 1;
      base = row * a.C + s;
      if ((flags & kSrc) && a.has_src) {  // Src on this warp's rows, then visible to the warp
        const long long r0 = grp * RW, r1 = min(r0 + RW, nrows);
        const long long e0 = a.src_row_off[r0], e1 = a.src_row_off[r1];
        for (long long e = e0 + lane; e < e1; e += 32) {
          const long long k = a.src_elem[e];
          rho[k] = (rho[k] + ldg<E>(a.src_alpha, e)) * ldg<E>(a.src_scale, e);
        }
        __syncwarp();
      }
    } else {
      const long long p = grp / a.colgroups;
      const long long c = (grp - p * a.colgroups) * 32 + lane;
      active = c < a.C;
      s = (int)(c % S);
      const long long xy = c / S;
      if (a.mode == 1) {  // column -> x, plane -> z
        face = xy == 0 || xy == a.nx - 1 || p == 0 || p == a.nz - 1;
      } else {            // column -> (x, y)
        const int x = (int)(xy % a.nx), y = (int)(xy / a.nx);
        face = x == 0 || x == a.nx - 1 || y == 0 || y == a.ny - 1;
      }
      base = p * a.plane_stride + c;
    }
    if (!(flags & kSolve)) continue;
    const bool dirl = active && (flags & (kDirBefore | kDirAfter)) && a.dir_on[s];
    const bool dB = dirl && (flags & kDirBefore), dA = dirl && (flags & kDirAfter);
    const bool dBf = dB && face, dAf = dA && face;
    const E dval = dirl ? dir_value<E>(flags, a.dir_val, s) : E(0);
    const E dval_in = dirl ? dir_value<E>(flags, a.dir_val_in, s) : E(0);
    E *line = rho + (active ? base : 0);
    const E om = (OUT == 2 && active) ? ldg<E>(a.omega, s) : E(1);
    const E sig = active ? ldg<E>(a.interior, s) : E(0);
    const E minf = active ? ldg<E>(a.interior, S + s) : E(0);

    // ---------------------------------------------------------------- forward
    E h = E(0), mp = E(0);
    auto fwd_group = [&](int g, auto get) {
      if (!active) return;
      const int i0 = g * R;
      E *q = line + (long long)i0 * st;
      if (i0 - 1 >= k0 && i0 + R < n) {  // interior: mul_{i-1} = r sigma (warp-uniform)
#pragma unroll
        for (int k = 0; k < R; k++) {
          const E d = dBf ? dval_in : get(k);
          h = fma(minf, h, d);
          *q = h;
          q += st;
        }
        mp = minf;
      } else {
#pragma unroll
        for (int k = 0; k < R; k++) {
          const int i = i0 + k;
          if (i < n) {
            E d = get(k);
            if (dB && (face || i == 0 || i == n - 1)) d = dval_in;
            h = fma(mp, h, d);
            *q = (OUT != 0 && i == n - 1) ? __ldg(tq + (size_t)i * S + s) * h : h;
            mp = __ldg(tmul + (size_t)i * S + s);
          }
          q += st;
        }
      }
    };
    // ---------------------------------------------------------------- backward
    // group g holds positions n-1-g*R down to n-R-g*R
    E x = E(0);
    auto bwd_group = [&](int g, auto get) {
      if (!active) return;
      const int i1 = n - 1 - g * R;
      E *q = line + (long long)i1 * st;
      // interior: inv = sigma, mul = r sigma, q = 1; with scaled output the
      // first position n-1 also qualifies (y_{n-1} was stored pre-scaled and
      // mul_{n-1} multiplies zero); position 0 never does (its Dirichlet end)
      if (i1 - R + 1 >= max(k0, 1) && (OUT != 0 || i1 < n - 1)) {
#pragma unroll
        for (int k = 0; k < R; k++) {
          const E hv = get(k);
          x = fma(minf, x, OUT == 0 ? sig * hv : hv);
          *q = dAf ? dval : (OUT == 2 ? om * x : x);
          q -= st;
        }
        if (dA && i1 == n - 1) line[(long long)(n - 1) * st] = dval;
      } else {
#pragma unroll
        for (int k = 0; k < R; k++) {
          const int i = i1 - k;
          if (i >= 0) {
            const E hv = get(k);
            const E t = OUT == 0 ? __ldg(tinv + (size_t)i * S + s) * hv
                                 : (i == n - 1 ? hv : __ldg(tq + (size_t)i * S + s) * hv);
            x = fma(__ldg(tmul + (size_t)i * S + s), x, t);
            *q = (dA && (face || i == 0 || i == n - 1)) ? dval : (OUT == 2 ? om * x : x);
          }
          q -= st;
        }
      }
    };

    if constexpr (PF != 1) {
      auto issue = [&](int g, bool fwd) {
        E *slot = ring + (g % G) * R * 32;
        const int i0 = fwd ? g * R : n - 1 - g * R;
        const E *q = line + (long long)i0 * st;
        const long long step = fwd ? st : -st;
#pragma unroll
        for (int k = 0; k < R; k++) {
          const int i = fwd ? i0 + k : i0 - k;
          if (active && i >= 0 && i < n) cp_async8(slot + k * 32, q);
          q += step;
        }
        cp_async_commit();  // possibly empty: keeps the group count uniform
      };
      for (int pass = 0; pass < 2; pass++) {
        const bool fwd = pass == 0;
#pragma unroll
        for (int g = 0; g < G - 1; g++) issue(g, fwd);
        for (int g = 0; g < ngrp; g++) {
          issue(g + G - 1, fwd);
          cp_async_wait<G - 1>();
          const E *slot = ring + (g % G) * R * 32;
          auto get = [&](int k) { return slot[k * 32]; };
          if (fwd)
            fwd_group(g, get);
          else
            bwd_group(g, get);
        }
        cp_async_wait<0>();
      }
    } else {
      E A[R], B[R];
      auto load = [&](E(&buf)[R], int g, bool fwd) {
        const int i0 = fwd ? g * R : n - 1 - g * R;
        const E *q = line + (long long)i0 * st;
        const long long step = fwd ? st : -st;
#pragma unroll
        for (int k = 0; k < R; k++) {
          const int i = fwd ? i0 + k : i0 - k;
          buf[k] = (active && i >= 0 && i < n) ? *q : E(0);
          q += step;
        }
      };
      for (int pass = 0; pass < 2; pass++) {
        const bool fwd = pass == 0;
        load(A, 0, fwd);
        for (int g = 0; g < ngrp; g += 2) {
          load(B, g + 1, fwd);
          if (fwd)
            fwd_group(g, [&](int k) { return A[k]; });
          else
            bwd_group(g, [&](int k) { return A[k]; });
          load(A, g + 2, fwd);
          if (g + 1 < ngrp) {
            if (fwd)
              fwd_group(g + 1, [&](int k) { return B[k]; });
            else
              bwd_group(g + 1, [&](int k) { return B[k]; });
          }
        }
      }
    }
  }
}

// Dynamic shared memory of one CTA: the warps' rings (PF != 1).
template <typename E, int PF>
constexpr size_t stream_smem_bytes() {
  return PF != 1 ? (size_t)(kStreamThreads / 32) * StreamCfg<PF>::G * StreamCfg<PF>::R * 32 *
                       sizeof(E)
                 : 0;
}

template <typename E, int PF>
cudaError_t allow_stream_smem() {
  cudaError_t e = cudaSuccess;
  for (auto f : {stream_sweep_kernel<E, PF, 0>, stream_sweep_kernel<E, PF, 1>,
                 stream_sweep_kernel<E, PF, 2>})
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)stream_smem_bytes<E, PF>());
  return e;
}

template <typename E, int PF>
cudaError_t launch_stream_one(const StreamArgs &a, int grid, cudaStream_t st) {
  const size_t smem = stream_smem_bytes<E, PF>();
  if (a.out == 1)
    stream_sweep_kernel<E, PF, 1><<<grid, kStreamThreads, smem, st>>>(a);
  else if (a.out == 2)
    stream_sweep_kernel<E, PF, 2><<<grid, kStreamThreads, smem, st>>>(a);
  else
    stream_sweep_kernel<E, PF, 0><<<grid, kStreamThreads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace bfv
