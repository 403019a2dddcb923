// Batched LOD steps: many independent microenvironments of uneven size and
// substrate count advanced by ONE persistent launch (all environments, all
// steps).
//
// Work items are groups of tiles (32 independent lines each) of one sweep of
// one environment, in the order (step, phase x/y/z, environment, item): a
// line cut into T chunks takes T warps, so the 8 warps of a CTA solve
// floor(8/T) tiles at once.  CTA b takes items b, b + G, b + 2G, ...
// (G = gridDim.x, every CTA resident), or, with a claim counter, the next
// unclaimed item each time it is free (items are claimed in order, so the
// argument below holds for both).
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
// A tile is solved either cut into chunks (chunk lengths m < n: chunks in
// shared memory, carries across the CTA's warps) or whole (m >= n: each
// warp streams its 32 lines as the single-grid streaming kernels do, no
// carries; an item is then 8 tiles, one per warp), with the arithmetic of the
// single-grid kernels: App. A system, FP32 in defect-correction form (the
// forward intermediate of whole lines in a scratch tile per warp, discarded
// from L2 once read back), the source update applied to an x item's rows
// before its solve.  Zero-flux boundaries (the batched microenvironments have
// no Dirichlet faces).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "batch_args.h"
#include "stream.cuh"
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

// Chunks live in shared memory ([warp][position][lane], lane fastest: every
// access of a warp is one conflict-free row) and every loop runs exactly the
// chunk's length: one launch serves environments whose chunk lengths differ,
// so a register array unrolled for the longest chunk would waste the issue
// slots of every shorter one.  A chunk and its two halo values arrive by
// cp.async (every element of the chunk in flight at once, no register round
// trip); FP32 keeps d beside the working array for the final x = c d + y.
__device__ __forceinline__ void cp_async_elem(void *smem, const void *gmem, int bytes) {
  if (bytes == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(smem)), "l"(gmem)
                 : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(smem)), "l"(gmem)
                 : "memory");
}

// FP32 whole-line tiles keep the first kBatchKS positions of g and d in shared
// memory (48 KB per CTA), streaming the rest in register blocks of kBatchRF
// positions (forward pass: one array per block) and kBatchR positions
// (backward pass: g and d), double-buffered, at 64 registers without spills;
// forward blocks of 8 measured 4% faster than blocks of 4.
constexpr int kBatchKS = 24;
constexpr int kBatchR = 4;
constexpr int kBatchRF = 8;
constexpr int kBatchWarpFloats = 2 * kBatchKS * 32;  // a warp's share of the line slabs

// Drops one 128-byte line (128-byte aligned) from L2 without writing it back;
// its contents become undefined.
__device__ __forceinline__ void discard_l2(const void *p) {
  asm volatile("discard.global.L2 [%0], 128;" ::"l"(p) : "memory");
}
// Hinted store at a compile-time byte offset from p (no address arithmetic).
template <int OFF>
__device__ __forceinline__ void st_hint_at(float *p, float v, unsigned long long pol) {
  asm volatile("st.global.L2::cache_hint.f32 [%0+%3], %1, %2;" ::"l"(p), "f"(v), "l"(pol),
               "n"(OFF));
}
template <int K, int N, typename F>
__device__ __forceinline__ void static_for(F &&f) {
  if constexpr (K < N) {
    f(std::integral_constant<int, K>{});
    static_for<K + 1, N>(f);
  }
}

// FP32 whole lines of the batched kernel: the arithmetic of solve_lines_f32
// (defect form, e = L_N d one position behind the loads with mirrored ends,
// g_i = mul_i g_{i-1} + inv'_i e_i, y_i = g_i + mul_i y_{i+1},
// x_i = c_hi d_i + (c_lo d_i + y_i)), for lines without Dirichlet faces.
//   * The forward intermediate goes to the warp's own scratch tile
//     [position][32 lanes] (sline: this lane's column), so every position of
//     the warp is one 128-byte line; the backward pass discards each line from
//     L2 once all lanes have read it, and the dead intermediate is never
//     written back to DRAM.
//   * Positions below KS keep g and d in shared-memory slabs (gsm, dsm).
//   * The kernel is issue-bound on these tiles, so a block of R positions
//     that lies inside the line past k0 (interior constants), wholly in the
//     slabs or wholly past them, takes a path with no per-position test,
//     table load or address increment of the scratch; other blocks (the
//     first, the one across KS, the last) take the general path.
//     Lanes without a line (active false) run the plain blocks too, on valid
//     addresses of their own (line = the field's start, their own scratch
//     column), and store nothing to the field.
template <int RF, int RB, int KS>
__device__ __forceinline__ void batch_lines_f32(float *line, float *sline, int n, long long st,
                                                bool active, const LineCoef<float> &cf,
                                                float *gsm, float *dsm) {
  const int S = cf.S;
  const int plain_lo = max(KS, cf.k0);  // plain blocks emit or read positions >= plain_lo
  const L2Pol pol = make_l2pol();
  float g = 0.f, dm1 = 0.f, dm2 = 0.f;
  // ---- forward, blocks of R = RF positions (its own scope: R is redefined below)
  {
    constexpr int R = RF;
    const int ngrp = (n + R - 1) / R;
    auto load_f = [&](float(&buf)[R], int gi) {
      const int i0 = gi * R;
      if (i0 + R <= n) {
        const float *q = line + (long long)i0 * st;
#pragma unroll
        for (int k = 0; k < R; k++) {
          buf[k] = *q;
          q += st;
        }
      } else {
        load_block<float, R>(buf, line, st, i0, true, n, active);
      }
    };
    auto emit = [&](int p, float e) {  // general: g of position p from its defect e
      const bool in = p >= cf.k0 && p < n - 1;
      const float iv = in ? cf.c0 : __ldg(cf.inv + (size_t)p * S);
      const float mu = in ? cf.c1 : __ldg(cf.mul + (size_t)p * S);
      g = fmaf(mu, g, e * iv);
      if (p < KS) gsm[p * 32] = g; else st_hint(sline + (long long)p * 32, g, pol.keep);
    };
    auto fwd = [&](int gi, const float(&buf)[R]) {
      const int i0 = gi * R;
      if (i0 - 1 >= plain_lo && i0 + R - 1 < n) {  // emits positions i0-1 .. i0+R-2
        float *sq = sline + (long long)(i0 - 1) * 32;
        static_for<0, R>([&](auto kc) {
          constexpr int k = decltype(kc)::value;
          const float d = buf[k];
          g = fmaf(cf.c1, g, ((dm1 - dm2) + (dm1 - d)) * cf.c0);
          st_hint_at<k * 128>(sq, g, pol.keep);
          dm2 = dm1;
          dm1 = d;
        });
        return;
      }
      if (i0 >= 1 && i0 - 1 >= cf.k0 && i0 + R <= KS && i0 + R - 1 < n) {  // inside the slabs
        float *gq = gsm + (i0 - 1) * 32, *dq = dsm + i0 * 32;
#pragma unroll
        for (int k = 0; k < R; k++) {
          const float d = buf[k];
          dq[k * 32] = d;
          g = fmaf(cf.c1, g, ((dm1 - dm2) + (dm1 - d)) * cf.c0);
          gq[k * 32] = g;
          dm2 = dm1;
          dm1 = d;
        }
        return;
      }
      if (!active) return;
#pragma unroll
      for (int k = 0; k < R; k++) {
        const int i = i0 + k;
        if (i < n) {
          const float d = buf[k];
          if (i < KS) dsm[i * 32] = d;
          if (i == 0) {
            dm1 = d;
            dm2 = d;  // mirrored start: d_{-1} = d_0
          } else {
            emit(i - 1, (dm1 - dm2) + (dm1 - d));
            dm2 = dm1;
            dm1 = d;
          }
        }
      }
    };
    {
      float A[R], B[R];
      load_f(A, 0);
      for (int gi = 0; gi < ngrp; gi += 2) {
        load_f(B, gi + 1);
        fwd(gi, A);
        load_f(A, gi + 2);
        if (gi + 1 < ngrp) fwd(gi + 1, B);
      }
      if (active && n > 0) emit(n - 1, dm1 - dm2);
    }
  }
  pass_barrier();
  // ---- backward, blocks of R = RB positions
  constexpr int R = RB;
  const int ngrp = (n + R - 1) / R;
  float y = 0.f;
  auto load_b = [&](float(&gb)[R], float(&db)[R], int gi) {
    const int i1 = n - 1 - gi * R;
    if (i1 - R + 1 >= KS && i1 - R + 1 >= 0) {  // the whole block in global memory
      const float *qs = sline + (long long)i1 * 32, *qd = line + (long long)i1 * st;
#pragma unroll
      for (int k = 0; k < R; k++) {
        gb[k] = qs[-k * 32];
        db[k] = *qd;
        qd -= st;
      }
    } else if (i1 < KS && i1 - R + 1 >= 0) {  // the whole block in the slabs
#pragma unroll
      for (int k = 0; k < R; k++) {
        gb[k] = gsm[(i1 - k) * 32];
        db[k] = dsm[(i1 - k) * 32];
      }
    } else {
      const float *qs = sline + (long long)i1 * 32, *qd = line + (long long)i1 * st;
#pragma unroll
      for (int k = 0; k < R; k++) {
        const int i = i1 - k;
        const bool ok = active && i >= 0 && i < n;
        gb[k] = !ok ? 0.f : (i < KS ? gsm[i * 32] : *qs);
        db[k] = !ok ? 0.f : (i < KS ? dsm[i * 32] : *qd);
        qs -= 32;
        qd -= st;
      }
    }
  };
  auto bwd = [&](int gi, const float(&gb)[R], const float(&db)[R]) {
    const int i1 = n - 1 - gi * R;
    float *q = line + (long long)i1 * st;
    if (gi >= 1 && i1 - R + 1 >= max(cf.k0, 0)) {  // interior positions i1 .. i1-R+1
#pragma unroll
      for (int k = 0; k < R; k++) {
        y = fmaf(cf.c1, y, gb[k]);
        const float xv = fmaf(cf.om, db[k], fmaf(cf.clo, db[k], y));
        if (active) st_hint(q, xv, pol.drop);
        q -= st;
      }
    } else if (active) {
#pragma unroll
      for (int k = 0; k < R; k++) {
        const int i = i1 - k;
        if (i >= 0) {
          const bool in = i >= cf.k0 && i < n - 1;
          const float mu = in ? cf.c1 : __ldg(cf.mul + (size_t)i * S);
          y = fmaf(mu, y, gb[k]);
          st_hint(q, fmaf(cf.om, db[k], fmaf(cf.clo, db[k], y)), pol.drop);
        }
        q -= st;
      }
    }
    // every lane has read block gi's scratch line: lane k discards position i1 - k's
    __syncwarp();
    const int lane = threadIdx.x & 31;
    if (lane < R && i1 - lane >= KS && i1 - lane >= 0)
      discard_l2(sline + ((long long)i1 * 32 - 33 * lane));
  };
  {
    float GA[R], DA[R], GB[R], DB[R];
    load_b(GA, DA, 0);
    for (int gi = 0; gi < ngrp; gi += 2) {
      load_b(GB, DB, gi + 1);
      bwd(gi, GA, DA);
      load_b(GA, DA, gi + 2);
      if (gi + 1 < ngrp) bwd(gi + 1, GB, DB);
    }
  }
}

// 256-thread CTAs, FP32 held to 64 registers (three or four per SM, as the
// chunk rows' shared memory allows), FP64 to 80: the kernel is latency-bound,
// so resident warps matter more than registers; FP32 with blocks of 4
// positions measured 3% faster than blocks of 8 at 80 registers.
template <typename E>
__global__ void __launch_bounds__(kBatchWarps * 32, sizeof(E) == 4 ? 4 : 3)
    batch_kernel(const BatchArgs a) {
  extern __shared__ __align__(16) unsigned char batch_smem[];
  constexpr int NB = kDefect<E> ? 2 : 1;                         // d (+ working array)
  E *const s_chunk = reinterpret_cast<E *>(batch_smem);          // [NB][8][maxm][32]
  E *const s_halo = s_chunk + NB * kBatchWarps * a.maxm * 32;    // [8][2][32]
  E *const s_end = s_halo + kBatchWarps * 64;                    // [8][32]
  E *const s_beg = s_end + kBatchWarps * 32;                     // [8][32]
  __shared__ int s_go;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int64_t total = a.per_step * a.n_steps;
  // (step, phase, environment) whose dependency thread 0 last saw satisfied
  // (shared memory: only thread 0 uses it, so it takes no register of the others)
  __shared__ long long s_last;
  if (threadIdx.x == 0) s_last = -1;
  __shared__ long long s_claim;
  for (int64_t g = blockIdx.x;; g += gridDim.x) {
    if (a.next) {  // claimed in order from the shared counter instead of every G-th item
      if (threadIdx.x == 0) s_claim = (long long)atomicAdd(a.next, 1ull);
      __syncthreads();
      g = s_claim;  // read by every thread before the dependency barrier below
    }
    if (g >= total) break;
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
    const int64_t item = r - off[ei];
    const BatchEnv &E_ = a.env[ei];

    // ---- dependency on the previous phase of this environment ----
    if (threadIdx.x == 0) {
      int go = 1;
      if (ld_relaxed_int(a.abort_flag)) go = 0;
      const long long key = ((long long)step * 3 + phase) * a.n_env + ei;
      const bool need = key != s_last && !(phase == 0 && step == 0);
      s_last = key;
      if (go && need) {
        const int dep_phase = phase == 0 ? 2 : phase - 1;
        unsigned want = (unsigned)(E_.items[dep_phase] * (phase == 0 ? step : step + 1));
        if (a.stall_test && phase == 1 && step == 0 && ei == 0 && item == 0) want = 0xffffffffu;
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

    const int S = E_.S, nx = E_.nx, ny = E_.ny;
    const int n = phase == 0 ? nx : phase == 1 ? ny : E_.nz;
    E *const field = static_cast<E *>(E_.field);
    const int64_t rowlen = (int64_t)nx * S;
    // Src on this item's rows (only this CTA touches them in this phase)
    if (phase == 0 && E_.has_src) {
      const int64_t nrows = (int64_t)ny * E_.nz;
      const int64_t ra = item * E_.group[0] * E_.rows_per_tile;
      const int64_t rb = min(nrows, ra + (int64_t)E_.group[0] * E_.rows_per_tile);
      const int64_t e0 = E_.src_row_off[ra], e1 = E_.src_row_off[rb];
      for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const int64_t el = E_.src_elem[e];
        field[el] = (field[el] + ldg<E>(E_.src_alpha, e)) * ldg<E>(E_.src_scale, e);
      }
      __syncthreads();
    }
    if (E_.whole[phase]) {  // ---- whole lines: warp w streams tile item*8 + w ----
      const int64_t tile = item * kBatchWarps + wp;
      if (tile < E_.tiles[phase]) {
        const LaneLine L = lane_line(phase, tile, lane, S, nx, ny, E_.nz, rowlen, E_.rows_per_tile);
        const long long st = phase == 0 ? S : phase == 1 ? rowlen : rowlen * ny;
        const E *tb = static_cast<const E *>(E_.stab[phase]);
        LineCoef<E> cf;
        cf.S = S;
        cf.k0 = E_.k0[phase];
        cf.inv = tb + L.s;
        cf.mul = tb + (size_t)n * S + L.s;
        cf.q = tb + 2 * (size_t)n * S + L.s;
        cf.c0 = ldg<E>(E_.sint[phase], L.s);
        cf.c1 = ldg<E>(E_.sint[phase], S + L.s);
        LineDir dr;
        dr.before = dr.after = false;
        dr.face = L.face;
        E *line = field + (L.active ? L.base : 0);
        if constexpr (sizeof(E) == 8) {
          cf.om = E(1);
          cf.clo = E(0);
          solve_lines_f64<0, 8>(line, n, st, L.active, cf, dr, E(0), E(0));
        } else {
          cf.om = ldg<E>(E_.cfix[phase], L.s);
          cf.clo = ldg<E>(E_.cfix[phase], S + L.s);
          // the warp's scratch tile: [position][lane], tiles in tile order
          E *sline = static_cast<E *>(E_.scratch) + tile * n * 32 + lane;
          float *wsm = reinterpret_cast<float *>(batch_smem) + (size_t)wp * kBatchWarpFloats + lane;
          batch_lines_f32<kBatchRF, kBatchR, kBatchKS>(line, sline, n, st, L.active, cf, wsm,
                                             wsm + kBatchKS * 32);
        }
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(a.done + phase * a.n_env + ei, 1u);
      }
      continue;
    }

    // ---- chunks: warp w solves chunk w % T of tile (item*group + w / T) ----
    const int T = E_.T[phase], m = E_.m[phase];
    const int grp = wp / T, t = wp - grp * T;  // warp group (tile) and chunk
    const int64_t tile = item * E_.group[phase] + grp;
    const bool tile_ok = grp < E_.group[phase] && tile < E_.tiles[phase];
    long long base = 0, pstride;
    bool active;
    int s;
    if (phase == 0) {
      const int64_t nrows = (int64_t)ny * E_.nz;
      const int64_t r0 = tile * E_.rows_per_tile;
      const int rows = tile_ok ? (int)min((int64_t)E_.rows_per_tile, nrows - r0) : 0;
      s = lane % S;
      active = tile_ok && lane < E_.rows_per_tile * S && lane / S < rows;
      base = (r0 + lane / S) * rowlen + s;
      pstride = S;
    } else {
      const int64_t C = phase == 1 ? rowlen : rowlen * ny;
      const int64_t tpp = (C + 31) / 32;
      const int64_t plane = tile / tpp;
      const int64_t c = (tile - plane * tpp) * 32 + lane;
      active = tile_ok && c < C;
      s = (int)(c % S);
      base = plane * C * n + c;
      pstride = C;
    }
    const int lo = t * m;
    const int len = active ? min(m, n - lo) : 0;
    E *col = field + (active ? base : 0) + (long long)lo * pstride;
    E *vd = s_chunk + (wp * a.maxm) * 32 + lane;  // d at position i: vd[i * 32]
    E *vs = kDefect<E> ? vd + kBatchWarps * a.maxm * 32 : vd;  // working array
    E *hl = s_halo + wp * 64 + lane;              // halos d_{lo-1}, d_{lo+len}
    const E *tb = static_cast<const E *>(E_.tab[phase]);
    const E *T_inv = tb, *T_mul = tb + n * S, *T_pf = T_mul + n * S, *T_pb = T_pf + n * S;
    const E *T_pc = T_pb + n * S, *T_cfix = T_pc + T * S;
    const E *T_cw = T_cfix + 2 * S;  // [T][T][S]
    const int q0 = lo * S + s;       // table index of position 0 of the chunk

    {
      const E *src = col;
      for (int i = 0; i < len; i++) {
        cp_async_elem(vd + i * 32, src, (int)sizeof(E));
        src += pstride;
      }
      if (kDefect<E> && len > 0) {
        if (lo > 0) cp_async_elem(hl, col - pstride, (int)sizeof(E));
        if (lo + len < n) cp_async_elem(hl + 32, col + (long long)len * pstride, (int)sizeof(E));
      }
      asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
    }
    if constexpr (kDefect<E>) {
      // e = L_N d; the zero-flux ends use mirrored halos (d_{-1} = d_0, d_n = d_{n-1})
      if (len > 0) {
        E prev = lo > 0 ? hl[0] : vd[0];
        const E after = lo + len < n ? hl[32] : vd[(len - 1) * 32];
        for (int i = 0; i < len; i++) {
          const E cur = vd[i * 32];
          const E nxt = i + 1 < len ? vd[(i + 1) * 32] : after;
          vs[i * 32] = (cur - prev) + (cur - nxt);
          prev = cur;
        }
      }
    }
    E gcar = E(0);
#pragma unroll 4
    for (int i = 0; i < len; i++) {
      const int q = q0 + i * S;
      gcar = fma(__ldg(T_mul + q), gcar, vs[i * 32] * __ldg(T_inv + q));
      vs[i * 32] = gcar;
    }
    s_end[wp * 32 + lane] = gcar;
    __syncthreads();
    if (grp < E_.group[phase] && t > 0) {  // chunk 0 enters with a zero carry
      E carry = E(0);
      for (int u = t - 1; u >= 0; u--)
        carry = fma(__ldg(T_cw + (u * T + t) * S + s), s_end[(grp * T + u) * 32 + lane], carry);
#pragma unroll 4
      for (int i = 0; i < len; i++) vs[i * 32] = fma(__ldg(T_pf + q0 + i * S), carry, vs[i * 32]);
    }
    E xcar = E(0);
#pragma unroll 4
    for (int i = len - 1; i >= 0; i--) {
      xcar = fma(__ldg(T_mul + q0 + i * S), xcar, vs[i * 32]);
      vs[i * 32] = xcar;
    }
    s_beg[wp * 32 + lane] = xcar;
    __syncthreads();
    if (grp < E_.group[phase] && t + 1 < T) {  // the last chunk enters with a zero carry
      E carry = E(0);
      for (int u = t + 1; u < T; u++)
        carry = fma(__ldg(T_cw + (u * T + t) * S + s), s_beg[(grp * T + u) * 32 + lane], carry);
#pragma unroll 4
      for (int i = 0; i < len; i++) vs[i * 32] = fma(__ldg(T_pb + q0 + i * S), carry, vs[i * 32]);
    }
    // every halo of the item arrived before the carry barriers above, so the
    // chunks can be written back now
    if constexpr (kDefect<E>) {  // x = c_hi d + (c_lo d + y), one final rounding
      const E chi = __ldg(T_cfix + s), clo = __ldg(T_cfix + S + s);
#pragma unroll 4
      for (int i = 0; i < len; i++) {
        const E d = vd[i * 32];
        col[(long long)i * pstride] = fma(chi, d, fma(clo, d, vs[i * 32]));
      }
    } else {
#pragma unroll 4
      for (int i = 0; i < len; i++) col[(long long)i * pstride] = vs[i * 32];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(a.done + phase * a.n_env + ei, 1u);
    }
  }
}

inline size_t batch_smem_bytes(int maxm, size_t esz) {
  const size_t nb = esz == 4 ? 2 : 1;  // FP32 keeps d beside the working array
  const size_t chunks = (nb * kBatchWarps * maxm * 32 + 4 * (size_t)kBatchWarps * 32) * esz;
  // FP32 whole-line tiles: g and d of the first kBatchKS positions per warp
  const size_t lines = esz == 4 ? (size_t)kBatchWarps * 2 * kBatchKS * 32 * 4 : 0;
  return chunks > lines ? chunks : lines;
}

template <typename E>
cudaError_t launch_batch_one(const BatchArgs &a, int grid, cudaStream_t st) {
  batch_kernel<E><<<grid, kBatchWarps * 32, batch_smem_bytes(a.maxm, sizeof(E)), st>>>(a);
  return cudaGetLastError();
}

template <typename E>
cudaError_t batch_blocks_per_sm(int maxm, int *out) {
  const size_t smem = batch_smem_bytes(maxm, sizeof(E));
  cudaError_t e = cudaFuncSetAttribute(batch_kernel<E>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, batch_kernel<E>, kBatchWarps * 32,
                                                       smem);
}

}  // namespace bfv
