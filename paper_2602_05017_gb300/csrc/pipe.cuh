// Persistent, TMA-pipelined sweep kernel for sm_103a (x, y and z sweeps).
//
// Same arithmetic as the plain kernels of sweeps.cuh -- partitioned Thomas of
// Algorithm 1 on the App. A system, FP32 in defect-correction form -- but
// every tile of CW independent lines ("columns") x n positions moves through
// a ring of shared-memory stages.  CW = 32 normally; for lines so long that two
// stages of 32 columns do not fit in shared memory, tiles of CW = 16 columns,
// and each consumer warp then solves two chunks, one per half-warp:
//
//   warp 0 (producer): TMA loads of tile k+NS-1 (cp.async.bulk.tensor boxes
//     for y/z tiles, issued by lane 0; one cp.async.bulk per row for x tiles,
//     the rows spread over the 32 lanes) completing on mbarrier `full`; once
//     the consumers have written tile k back into its stage (mbarrier `done`),
//     the bulk store of that tile; the stage is reloaded after the store has
//     finished reading it;
//   warp 1 (preparer, x tiles with a source update or a Dirichlet application
//     before the solve): applies them in shared memory to each tile once it
//     has landed -- running ahead of the consumers, who solve earlier tiles --
//     and arrives on mbarrier `ready`, which the consumers then wait for
//     instead of `full`;
//   the next ceil(T*CW/32) warps (consumers): chunk t of every column of the staged
//     tile, in registers (thread (warp w, lane l): chunk (w-1)*32/CW + l/CW of
//     column l % CW).  Halos and chunk carries cross warps through shared memory
//     between two named barriers per tile that only consumers join.
//
// The grid is persistent (tiles strided by gridDim.x), so loads of later
// tiles overlap the solve and the store of earlier ones.  The axis constants
// and the carry weights are staged once per CTA.
//
// Every mbarrier wait is bounded (mbar_wait_bounded): on a timeout the status
// word is set, the consumers agree to stop at the first carry barrier, which
// ANDs every consumer's wait outcome (no named barrier is left waiting), and
// the producer drains (bounded) the loads still in flight before the CTA exits.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "pipe_args.h"
#include "sweeps.cuh"

namespace bfv {

// Field storage H and arithmetic E: the same type, or 16-bit storage (bf16,
// fp16) with FP32 arithmetic -- values are widened on their way from the
// staged tile into registers and rounded to nearest on their way back.
template <typename E, typename H>
__device__ __forceinline__ E widen(H v) {
  if constexpr (std::is_same<H, __nv_bfloat16>::value) return __bfloat162float(v);
  else if constexpr (std::is_same<H, __half>::value) return __half2float(v);
  else return v;
}
template <typename H, typename E>
__device__ __forceinline__ H narrow(E v) {
  if constexpr (std::is_same<H, __nv_bfloat16>::value) return __float2bfloat16_rn(v);
  else if constexpr (std::is_same<H, __half>::value) return __float2half_rn(v);
  else return v;
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int c0, int c1,
                                            int c2, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
      "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ void tma_store_3d(const CUtensorMap *map, int c0, int c1, int c2,
                                             const void *src) {
  asm volatile(
      "cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
          map),
      "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(src))
      : "memory");
}
__device__ __forceinline__ void bulk_wait_read_all() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
// Barrier 1 over the consumer warps only.  The non-.aligned form, after a
// __syncwarp: lanes may reach it from divergent code (ragged tiles), and the
// compiler does not treat an asm barrier as a reconvergence point.
__device__ __forceinline__ void consumers_sync(int nthreads) {
  __syncwarp();
  asm volatile("barrier.cta.sync 1, %0;" ::"r"(nthreads) : "memory");
}
// Barrier 1 over the consumers with an AND of `ok` (uniform result).
__device__ __forceinline__ bool consumers_all(bool ok, int nthreads) {
  uint32_t r;
  __syncwarp();
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "barrier.cta.red.and.pred q, 1, %2, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)ok), "r"(nthreads)
      : "memory");
  return r != 0;
}

template <typename E, int MAXM>
struct PipeBound {  // chunk registers + about 96 for addressing, carries, constants
  static constexpr int regs = MAXM * (int)sizeof(E) / 4 + 96;
  static constexpr int raw = 65536 / regs;
  static constexpr int threads = (raw >= 1024 ? 1024 : raw) / 32 * 32;
};

// Constants of the pipelined kernel: inv, mul, pf, pb substrate-major
// [S][n_pad] (n_pad = 1 mod 32, so lanes of different substrates read
// different banks and each thread walks its own row with compile-time
// offsets) -- AxisTab::tabT, copied into shared memory (the planner only
// takes this kernel when they fit).
__host__ __device__ inline int pipe_npad(int n) { return (n + 31) / 32 * 32 + 1; }

// One chunk of one column: e = L_N d (FP32), forward elimination, carry in,
// back substitution, carry in, c d + y (FP32), Dirichlet, write-back.
// FULL: the chunk has exactly MAXM positions (no per-position guards).
// PS > 0: compile-time stride between positions in the staged tile.
template <typename E, int MAXM, bool FULL, int PS, int CW, typename H>
__device__ __forceinline__ bool pipe_chunk(H *p, const int ps_rt, const int len, const int lo,
                                           const int n, const int t, const int T, const int c,
                                           const E *Ti, const E *Tm, const E *Tf, const E *Tb,
                                           const E *Tcw, const int S, const int s, const E chi,
                                           const E clo, E *s_end, E *s_beg, const int ncons,
                                           const bool dir, const bool face, const E dval,
                                           const bool ok) {
  const int ps = PS > 0 ? PS : ps_rt;
  E v[MAXM];
#pragma unroll
  for (int i = 0; i < MAXM; i++)
    if (FULL || i < len) v[i] = widen<E>(p[i * ps]);
  if constexpr (kDefect<E>) {
    // e = L_N d.  At the two ends of the line the zero-flux rows equal the
    // interior formula with a mirrored ghost value (d_{-1} = d_0,
    // d_n = d_{n-1}), so no position needs a branch.
    E prev = E(0), after = E(0);
    if (len > 0) {
      prev = lo > 0 ? widen<E>(p[-ps]) : v[0];
      // (the last value is re-read from the tile: selecting v[len-1] would
      // index the register array dynamically)
      const E last = FULL ? v[MAXM - 1] : widen<E>(p[(len - 1) * ps]);
      after = lo + len < n ? widen<E>(p[(FULL ? MAXM : len) * ps]) : last;
    }
#pragma unroll
    for (int i = 0; i < MAXM; i++)
      if (FULL || i < len) {
        const E cur = v[i];
        const E nxt = (i + 1 < MAXM && (FULL || i + 1 < len)) ? v[i + 1] : after;
        v[i] = (cur - prev) + (cur - nxt);
        prev = cur;
      }
  }
  E g = E(0);
#pragma unroll
  for (int i = 0; i < MAXM; i++)
    if (FULL || i < len) {
      g = fma(Tm[i], g, v[i] * Ti[i]);
      v[i] = g;
    }
  s_end[t * CW + c] = g;
  // The first carry barrier also ANDs the outcome of every consumer's wait
  // for the tile: on a timeout all consumers leave together, before any
  // write-back (what they computed from the unfinished stage stays local).
  if (!consumers_all(ok, ncons)) return false;
  // carry weights Tcw[(u*T + t)*S + s] walked with pointer steps (no index
  // arithmetic per term), in the same order as the closed form's sum; not
  // unrolled (unrolling by 4 measured 5% slower on the y/z tiles)
  const int dw = T * S;
  if (t > 0 && t < T) {  // chunk 0 enters with a zero carry (t == T: a half-warp with no chunk)
    E carry = E(0);
    const E *w = Tcw + ((t - 1) * T + t) * S + s;
    const E *q = s_end + (t - 1) * CW + c;
#pragma unroll 1
    for (int u = t - 1; u >= 0; u--, w -= dw, q -= CW) carry = fma(*w, *q, carry);
#pragma unroll
    for (int i = 0; i < MAXM; i++)
      if (FULL || i < len) v[i] = fma(Tf[i], carry, v[i]);
  }
  E x = E(0);
#pragma unroll
  for (int i = MAXM - 1; i >= 0; i--)
    if (FULL || i < len) {
      x = fma(Tm[i], x, v[i]);
      v[i] = x;
    }
  s_beg[t * CW + c] = x;
  consumers_sync(ncons);
  if (t + 1 < T) {  // the last chunk enters with a zero carry
    E carry = E(0);
    const E *w = Tcw + ((t + 1) * T + t) * S + s;
    const E *q = s_beg + (t + 1) * CW + c;
#pragma unroll 1
    for (int u = t + 1; u < T; u++, w += dw, q += CW) carry = fma(*w, *q, carry);
#pragma unroll
    for (int i = 0; i < MAXM; i++)
      if (FULL || i < len) v[i] = fma(Tb[i], carry, v[i]);
  }
  if constexpr (kDefect<E>) {  // x = c_hi d + (c_lo d + y), d from the staged tile
#pragma unroll
    for (int i = 0; i < MAXM; i++)
      if (FULL || i < len) {
        const E d = widen<E>(p[i * ps]);
        v[i] = fma(chi, d, fma(clo, d, v[i]));
      }
  }
  if (dir && len > 0) {
#pragma unroll
    for (int i = 0; i < MAXM; i++)
      if ((FULL || i < len) && (face || lo + i == 0 || lo + i == n - 1)) v[i] = dval;
  }
  // No barrier before the write-back: the only reads of other chunks' positions
  // (the halos of e = L_N d) happen before the first barrier above, and the
  // carry arrays are rewritten only after barriers every warp has passed.
#pragma unroll
  for (int i = 0; i < MAXM; i++)
    if (FULL || i < len) p[i * ps] = narrow<H>(v[i]);
  return true;
}

// MODE 0: x tiles (per-row bulk copies, Src and B before the solve);
// MODE 1: y/z tiles (tensor boxes).  PSX > 0 (x tiles only): the substrate
// count S, known at compile time, so the staged positions (S apart) need no
// per-access address arithmetic; 0: S read at run time.  CW: columns per tile
// (32, or 16 for long lines).  H: the field's storage type (E, or bf16 / fp16
// with E = float): stages and TMA copies hold H, registers and constants E.
template <typename E, int MAXM, int MODE, int PSX = 0, int CW = 32, typename H = E>
__global__ void __launch_bounds__(PipeBound<E, MAXM>::threads)
    sweep_pipe_kernel(const __grid_constant__ CUtensorMap map, const PipeArgs a) {
  static_assert(CW == 32 || CW == 16, "tiles of 32 or 16 columns");
  constexpr int CPW = 32 / CW;  // chunks per consumer warp
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const int T = a.tab.T, m = a.tab.m, n = a.n, S = a.S, NS = a.stages;
  const int64_t stage_elems = a.stage_elems;
  const int npad = pipe_npad(n);
  H *stage0 = reinterpret_cast<H *>(smem_raw);
  // [4][S][npad], 16-byte aligned after the stages: offset arithmetic on the shared array itself
  // (a pointer rounded through an integer would hide from the compiler that the constants and
  // carry arrays derived from it live in shared memory, turning their loads into generic ones)
  E *tab = reinterpret_cast<E *>(smem_raw + ((size_t)NS * stage_elems * sizeof(H) + 15) / 16 * 16);
  const int W = (T + CPW - 1) / CPW;  // consumer warps
  E *s_end = tab + 4 * S * npad;      // [W*32]: chunk t, column c at t*CW + c
  E *s_beg = s_end + W * 32;
  E *s_cw = s_beg + W * 32;  // [T][T][S] carry weights
  uint64_t *full = reinterpret_cast<uint64_t *>(
      (reinterpret_cast<uintptr_t>(s_cw + T * T * S) + 15) & ~uintptr_t(15));
  uint64_t *done = full + NS;
  uint64_t *ready = done + NS;  // x tiles with a preparation: the stage is prepared

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long first = blockIdx.x;
  const long long count = (a.ntiles - first + gridDim.x - 1) / gridDim.x;
  const int ncons = W * 32;
  H *field = static_cast<H *>(a.field);

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; s++) {
      mbar_init(&full[s], 1);
      mbar_init(&done[s], ncons);
      mbar_init(&ready[s], 1);
    }
    fence_mbar_init();
    fence_proxy_async_smem();
  }
  {
    const E *gT = static_cast<const E *>(a.tab.tabT);
    for (int q = threadIdx.x; q < 4 * S * npad; q += blockDim.x) tab[q] = __ldg(gT + q);
    const E *gW = static_cast<const E *>(a.tab.cw);
    for (int q = threadIdx.x; q < T * T * S; q += blockDim.x) s_cw[q] = __ldg(gW + q);
  }
  __syncthreads();
  const E *s_inv = tab, *s_mul = tab + S * npad, *s_pf = s_mul + S * npad, *s_pb = s_pf + S * npad;
  const E *g_cfix = static_cast<const E *>(a.tab.cfix);

  // x tiles: Src and B before the solve, applied by warp 1 (the preparer) when
  // the launch has one (a.prep_warp: the host sets it exactly when there is a
  // source update or a Dirichlet application before the solve)
  const bool prep = MODE == 0 && a.prep_warp != 0;
  const bool srcs = prep && (a.flags & kSrc) && a.has_src;
  const bool dirb = prep && (a.flags & kDirBefore);
  const int cons0 = prep ? 2 : 1;  // first consumer warp
  // A tile with more source entries than the preparer holds prefetched (32 * kPF: dense agents)
  // gets its Src and B from all the consumers instead, before its solve.  Preparer and
  // consumers decide from the tile's entry count in the row offsets (read-only global data),
  // so they always agree, whatever the outcome of any wait.
  constexpr int kPF = 8;
  auto tile_range = [&](long long kk, long long &e0, long long &e1) {
    e0 = e1 = 0;
    if (!srcs || kk >= count) return;
    const long long r0 = (first + kk * gridDim.x) * a.rows_per_tile;
    e0 = __ldg(a.src_row_off + r0);
    e1 = __ldg(a.src_row_off + min(r0 + (long long)a.rows_per_tile, (long long)a.nrows));
  };
  auto is_dense = [&](long long e0, long long e1) { return e1 - e0 > 32 * kPF; };
  // B before the solve on a tile's staged rows: warp w of nw takes rows w, w + nw, ...; the
  // lanes walk a face row (a lane's substrate is fixed when S divides 32: flag and value once)
  auto dir_rows = [&](H *sg, long long r0, int rows, int w, int nw) {
    const bool lane_s = 32 % S == 0;
    const bool on_l = lane_s && a.dir_on[lane % S];
    const H val_l = on_l ? narrow<H>(dir_value<E>(a.flags, a.dir_val, lane % S)) : H(0);
    for (int rr = w; rr < rows; rr += nw) {
      const uint32_t row = (uint32_t)r0 + (uint32_t)rr;
      const int z = (int)(row / (uint32_t)a.ny), y = (int)row - z * a.ny;
      H *trow = sg + (size_t)rr * a.pitch;
      if (y == 0 || y == a.ny - 1 || z == 0 || z == a.nz - 1) {
        if (lane_s) {
          if (on_l)
            for (int q = lane; q < a.rowlen; q += 32) trow[q] = val_l;
        } else {
          for (int q = lane; q < a.rowlen; q += 32) {
            const int ss = q % S;
            if (a.dir_on[ss]) trow[q] = narrow<H>(dir_value<E>(a.flags, a.dir_val, ss));
          }
        }
      } else {
        for (int q = lane; q < 2 * S; q += 32) {
          const int ss = q % S;
          if (a.dir_on[ss])
            trow[q < S ? ss : (a.nx - 1) * S + ss] = narrow<H>(dir_value<E>(a.flags, a.dir_val, ss));
        }
      }
    }
  };

  if (warp == 0) {  // ------------------------------------------------ producer
    // x tiles: up to 32 rows per tile, one bulk copy each, issued by the lanes
    // in parallel (one thread issuing them in turn bounds the short-row tiles);
    // y/z tiles: one or two tensor boxes, lane 0 alone.  Each lane waits for
    // the stage itself (its own acquire of the consumers' writes) and for its
    // own stores; the lanes agree on the outcome of every bounded wait.
    constexpr unsigned pmask = MODE == 0 ? 0xffffffffu : 1u;
    if (MODE != 0 && lane != 0) return;
    auto rows_of = [&](long long tile) {
      const long long r0 = tile * a.rows_per_tile;
      return (int)min((long long)a.rows_per_tile, a.nrows - r0);
    };
    auto issue_load = [&](long long k, int s) {
      const long long tile = first + k * gridDim.x;
      H *dst = stage0 + s * stage_elems;
      if constexpr (MODE == 0) {
        const int rows = rows_of(tile);
        const uint32_t rb = (uint32_t)(a.gpitch * sizeof(H));
        // the expected bytes before any copy is issued: the phase cannot
        // complete while the producer's own arrival is pending
        if (lane == 0) mbar_arrive_expect_tx(&full[s], rb * rows);
        __syncwarp();
        for (int r = lane; r < rows; r += 32)
          bulk_g2s(dst + (size_t)r * a.pitch, field + (tile * a.rows_per_tile + r) * a.gpitch, rb,
                   &full[s]);
      } else {
        const int plane = (int)((uint32_t)tile / (uint32_t)a.tiles_per_plane);
        const int c0 = (int)((uint32_t)tile % (uint32_t)a.tiles_per_plane) * CW;
        mbar_arrive_expect_tx(&full[s], (uint32_t)(stage_elems * sizeof(H)));
        for (int b = 0; b < a.nbox; b++)
          tma_load_3d(dst + (size_t)b * a.box_rows * CW, &map, c0, b * a.box_rows, plane, &full[s]);
      }
    };
    auto issue_store = [&](long long k, int s) {
      const long long tile = first + k * gridDim.x;
      const H *src = stage0 + s * stage_elems;
      if constexpr (MODE == 0) {
        const int rows = rows_of(tile);
        const uint32_t rb = (uint32_t)(a.gpitch * sizeof(H));
        for (int r = lane; r < rows; r += 32)
          bulk_s2g(field + (tile * a.rows_per_tile + r) * a.gpitch, src + (size_t)r * a.pitch, rb);
      } else {
        const int plane = (int)((uint32_t)tile / (uint32_t)a.tiles_per_plane);
        const int c0 = (int)((uint32_t)tile % (uint32_t)a.tiles_per_plane) * CW;
        for (int b = 0; b < a.nbox; b++)
          tma_store_3d(&map, c0, b * a.box_rows, plane, src + (size_t)b * a.box_rows * CW);
      }
      bulk_commit();
    };
    const long long pre = count < NS ? count : NS;
    for (long long k = 0; k < pre; k++) issue_load(k, (int)k);
    long long k = 0;
    bool ok = true;
    for (; k < count; k++) {
      const int s = (int)(k % NS);
      ok = mbar_wait_bounded(&done[s], (uint32_t)((k / NS) & 1), a.status);
      if (!__all_sync(pmask, ok)) {
        ok = false;
        break;
      }
      issue_store(k, s);
      if (k + NS < count) {
        bulk_wait_read_all();  // the stage is free once every lane's store has read it
        __syncwarp(pmask);
        issue_load(k + NS, s);
      }
    }
    if (!ok && lane == 0) {  // drain the loads still in flight (bounded) before exiting
      for (long long j = k; j < count && j < k + NS; j++)
        mbar_wait_bounded(&full[j % NS], (uint32_t)((j / NS) & 1), a.status);
    }
    bulk_wait_all();
    return;
  }

  if (prep && warp == 1) {  // ---------------------------------------- preparer
    constexpr unsigned pmask = 0xffffffffu;
    // Src then B on tile kk's stage once it has landed (x tiles), then `ready`.
    // The source entries are unique elements (aggregated on the host or the
    // device), so the lanes update them independently.  They flow ahead of the
    // tiles: the entry range of a tile is loaded two preparations before its
    // own, its first 32*PF entries (PF per lane) one preparation before, so a
    // preparation waits on global memory only for a tile with more entries.
    // The Dirichlet rows follow the sources (a source can sit on a face).
    constexpr int PF = kPF;
    int2 prc[PF];
    E pal[PF], psc[PF];
    long long pe0 = 0, pe1 = 0, qe0 = 0, qe1 = 0;  // entry ranges: the next tile, the one after
    auto fetch_entries = [&]() {
#pragma unroll
      for (int j = 0; j < PF; j++) {
        const long long e = pe0 + lane + 32 * j;
        const bool v = e < pe1 && !is_dense(pe0, pe1);
        prc[j] = v ? __ldg(a.src_rowcol + e) : make_int2(-1, 0);
        pal[j] = v ? ldg<E>(a.src_alpha, e) : E(0);
        psc[j] = v ? ldg<E>(a.src_scale, e) : E(0);
      }
    };
    if (srcs) {
      tile_range(0, pe0, pe1);
      fetch_entries();
      tile_range(1, qe0, qe1);
    }
    auto prepare = [&](long long kk) -> bool {
      const int s = (int)(kk % NS);
      bool okw = mbar_wait_bounded(&full[s], (uint32_t)((kk / NS) & 1), a.status);
      if (!__all_sync(pmask, okw)) return false;
      H *const sg = stage0 + s * stage_elems;
      const long long r0 = (first + kk * gridDim.x) * a.rows_per_tile;
      const int rows = (int)min((long long)a.rows_per_tile, a.nrows - r0);
      const bool dense = srcs && is_dense(pe0, pe1);  // then the consumers prepare the tile
      if (srcs) {
        if (!dense) {
#pragma unroll
          for (int j = 0; j < PF; j++)
            if (prc[j].x >= 0) {
              H *q = sg + (prc[j].x - r0) * a.pitch + prc[j].y;
              *q = narrow<H>((widen<E>(*q) + pal[j]) * psc[j]);
            }
          __syncwarp();
        }
        pe0 = qe0;  // the next tile's entries, the range of the one after it
        pe1 = qe1;
        fetch_entries();
        tile_range(kk + 2, qe0, qe1);
      }
      if (dirb && !dense) {
        dir_rows(sg, r0, rows, 0, 1);
        __syncwarp();
      }
      if (lane == 0) mbar_arrive(&ready[s]);  // release: the warp's writes, ordered by __syncwarp
      return true;
    };
    for (long long k = 0; k < count; k++)
      if (!prepare(k)) break;  // (a timeout: the consumers' bounded wait on `ready` ends too)
    return;
  }

  // ---------------------------------------------------------------- consumers
  const int wc = warp - cons0;                     // consumer warp
  const int c = CW == 32 ? lane : (lane & (CW - 1));  // column of the tile
  const int t = wc * CPW + lane / CW;              // chunk (t == T: no chunk)
  const int lo = t * m;
  const int len_full = t < T ? min(m, n - lo) : 0;
  const int colbase = MODE == 0 ? (c / S) * a.pitch + c % S : c;
  const int ps_rt = MODE == 0 ? S : CW;
  const E *Tcw = s_cw;  // [T][T][S], staged beside the other constants
  const bool dir_after = (a.flags & kDirAfter) != 0;
  const int ctid = threadIdx.x - 32 * cons0;  // consumer thread
  long long cn0 = 0, cn1 = 0;                 // entry range of the next tile (dense check)
  if (srcs) tile_range(0, cn0, cn1);
  // A thread's substrate is the same in every tile when S divides the tile width (and, for
  // z tiles, the row pitch): its per-substrate constants are then loaded once, not per tile.
  const bool s_fixed = MODE == 0 || (CW % S == 0 && (a.mode == 1 || a.gpitch % S == 0));
  const int sf = c % S;
  const E chi_f = s_fixed ? __ldg(g_cfix + sf) : E(0), clo_f = s_fixed ? __ldg(g_cfix + S + sf) : E(0);
  const bool dir_f = s_fixed && dir_after && a.dir_on[sf];
  const E dval_f = dir_f ? dir_value<E>(a.flags, a.dir_val, sf) : E(0);
  // The planner keeps tile, row and column counts below 2^31, so the per-tile
  // index arithmetic below runs in 32 bits (a 64-bit division is a long
  // software sequence, and every consumer thread repeats it per tile).
  for (long long k = 0; k < count; k++) {
    const int st = (int)(k % NS);
    // (a timed-out wait is acted on at the first carry barrier of the chunk
    // solve; the steps before it only touch this stage and registers)
    // (x tiles with a preparation: the preparer's `ready`, after its own wait for the data)
    const bool ok = mbar_wait_bounded(prep ? &ready[st] : &full[st], (uint32_t)((k / NS) & 1),
                                      a.status);
    const long long tile = first + k * gridDim.x;
    H *const stg = stage0 + st * stage_elems;
    if (srcs) {
      const long long c0 = cn0, c1 = cn1;
      tile_range(k + 1, cn0, cn1);  // the next tile's range, used one tile later
      if (is_dense(c0, c1)) {       // every consumer agrees (global data); done whatever `ok`
        const long long r0 = tile * a.rows_per_tile;
        const int rows = (int)min((long long)a.rows_per_tile, a.nrows - r0);
        constexpr int U = 4;
        for (long long eb = c0 + ctid; eb < c1; eb += (long long)ncons * U) {
          int2 rc[U];
          E al[U], sc[U];
#pragma unroll
          for (int j = 0; j < U; j++) {
            const long long e = eb + (long long)ncons * j;
            const bool v = e < c1;
            rc[j] = v ? __ldg(a.src_rowcol + e) : make_int2(-1, 0);
            al[j] = v ? ldg<E>(a.src_alpha, e) : E(0);
            sc[j] = v ? ldg<E>(a.src_scale, e) : E(0);
          }
#pragma unroll
          for (int j = 0; j < U; j++)
            if (rc[j].x >= 0) {
              H *q = stg + (rc[j].x - r0) * a.pitch + rc[j].y;
              *q = narrow<H>((widen<E>(*q) + al[j]) * sc[j]);
            }
        }
        consumers_sync(ncons);
        if (dirb) {
          dir_rows(stg, r0, rows, wc, W);
          consumers_sync(ncons);
        }
      }
    }
    int s;
    bool active, face = false;
    if constexpr (MODE == 0) {
      const long long r0 = tile * a.rows_per_tile;
      const int rows = (int)min((long long)a.rows_per_tile, a.nrows - r0);
      s = c % S;
      active = c < a.rows_per_tile * S && c / S < rows;
      if (dir_after) {  // (only the Dirichlet application after the solve needs the face)
        const uint32_t row = (uint32_t)r0 + (uint32_t)(c / S);
        const int z = (int)(row / (uint32_t)a.ny), y = (int)row - z * a.ny;
        face = y == 0 || y == a.ny - 1 || z == 0 || z == a.nz - 1;
      }
    } else {
      const int plane = (int)((uint32_t)tile / (uint32_t)a.tiles_per_plane);
      const uint32_t cg = ((uint32_t)tile - (uint32_t)plane * (uint32_t)a.tiles_per_plane) *
                              (uint32_t)CW + (uint32_t)c;
      if (a.mode == 1) {
        active = cg < (uint32_t)a.C;
        s = (int)(cg % (uint32_t)S);
        if (dir_after) {
          const int x0 = (int)(cg / (uint32_t)S);
          face = (x0 == 0 || x0 == a.nx - 1 || plane == 0 || plane == a.nz - 1);
        }
      } else {  // a plane of ny rows gpitch apart: padding columns are not lines
        const uint32_t y = cg / (uint32_t)a.gpitch, xs = cg - y * (uint32_t)a.gpitch;
        active = cg < (uint32_t)a.C && xs < (uint32_t)a.rowlen;
        s = (int)(xs % (uint32_t)S);
        if (dir_after) {
          const int x0 = (int)(xs / (uint32_t)S);
          face = (x0 == 0 || x0 == a.nx - 1 || y == 0 || (int)y == a.ny - 1);
        }
      }
    }
    const int len = active ? len_full : 0;
    H *p = stg + colbase + lo * ps_rt;
    const int rowoff = s * npad + lo;
    const bool dir = s_fixed ? dir_f : dir_after && a.dir_on[s];
    const E dval = s_fixed ? dval_f : dir ? dir_value<E>(a.flags, a.dir_val, s) : E(0);
    const E chi = s_fixed ? chi_f : __ldg(g_cfix + s), clo = s_fixed ? clo_f : __ldg(g_cfix + S + s);
    // the unguarded path only when every lane of the warp has a full chunk:
    // the choice is warp-uniform, so a warp never splits across the paths
    constexpr int PS = MODE == 0 ? PSX : CW;
    bool solved;
    if (__all_sync(0xffffffffu, len == MAXM))
      solved = pipe_chunk<E, MAXM, true, PS, CW>(p, ps_rt, len, lo, n, t, T, c, s_inv + rowoff,
                                             s_mul + rowoff, s_pf + rowoff, s_pb + rowoff, Tcw, S,
                                             s, chi, clo, s_end, s_beg, ncons, dir, face, dval, ok);
    else
      solved = pipe_chunk<E, MAXM, false, PS, CW>(p, ps_rt, len, lo, n, t, T, c, s_inv + rowoff,
                                              s_mul + rowoff, s_pf + rowoff, s_pb + rowoff, Tcw, S,
                                              s, chi, clo, s_end, s_beg, ncons, dir, face, dval, ok);
    if (!solved) break;
    fence_proxy_async_smem();  // generic-proxy writes -> visible to the bulk store
    mbar_arrive(&done[st]);
  }
}

// x tiles with a compile-time substrate count: the default chunk length only
// (each specialisation is a full copy of the kernel).
template <int MAXM>
constexpr bool pipe_x_specialised() {
  return MAXM == 32;
}
// Tiles of 16 columns (long lines): the chunk capacities the planner offers them.
template <int MAXM>
constexpr bool pipe_half_tiles() {
  return MAXM == 32 || MAXM == 64;
}

template <typename E, int MAXM, typename H = E>
cudaError_t allow_pipe_smem(size_t bytes) {
  cudaError_t e = cudaSuccess;
  auto set = [&](const void *f) {
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  };
  set((const void *)sweep_pipe_kernel<E, MAXM, 0, 0, 32, H>);
  set((const void *)sweep_pipe_kernel<E, MAXM, 1, 0, 32, H>);
  if constexpr (pipe_half_tiles<MAXM>()) {
    set((const void *)sweep_pipe_kernel<E, MAXM, 0, 0, 16, H>);
    set((const void *)sweep_pipe_kernel<E, MAXM, 1, 0, 16, H>);
  }
  if constexpr (pipe_x_specialised<MAXM>()) {
    set((const void *)sweep_pipe_kernel<E, MAXM, 0, 1, 32, H>);
    set((const void *)sweep_pipe_kernel<E, MAXM, 0, 2, 32, H>);
    set((const void *)sweep_pipe_kernel<E, MAXM, 0, 4, 32, H>);
    set((const void *)sweep_pipe_kernel<E, MAXM, 0, 8, 32, H>);
  }
  if constexpr (std::is_same<H, E>::value && pipe_half_tiles<MAXM>()) {
    set((const void *)sweep_pipe_kernel<E, MAXM, 0, 1, 16>);
    set((const void *)sweep_pipe_kernel<E, MAXM, 0, 2, 16>);
    set((const void *)sweep_pipe_kernel<E, MAXM, 0, 4, 16>);
    set((const void *)sweep_pipe_kernel<E, MAXM, 0, 8, 16>);
  }
  return e;
}

template <typename E, int MAXM, typename H = E>
cudaError_t launch_pipe_one(const CUtensorMap &map, const PipeArgs &a, int grid, size_t smem,
                            cudaStream_t st) {
  const int cpw = a.cw == 16 ? 2 : 1;
  const int threads = ((a.tab.T + cpw - 1) / cpw + 1 + a.prep_warp) * 32;
  if (threads > PipeBound<E, MAXM>::threads) return cudaErrorInvalidConfiguration;
  if (a.cw == 16) {
    if constexpr (pipe_half_tiles<MAXM>()) {
      if (a.mode != 0) {
        sweep_pipe_kernel<E, MAXM, 1, 0, 16, H><<<grid, threads, smem, st>>>(map, a);
        return cudaGetLastError();
      }
      if constexpr (std::is_same<H, E>::value) {  // x tiles: S at compile time where it can be
        switch (a.S) {
          case 1: sweep_pipe_kernel<E, MAXM, 0, 1, 16><<<grid, threads, smem, st>>>(map, a); return cudaGetLastError();
          case 2: sweep_pipe_kernel<E, MAXM, 0, 2, 16><<<grid, threads, smem, st>>>(map, a); return cudaGetLastError();
          case 4: sweep_pipe_kernel<E, MAXM, 0, 4, 16><<<grid, threads, smem, st>>>(map, a); return cudaGetLastError();
          case 8: sweep_pipe_kernel<E, MAXM, 0, 8, 16><<<grid, threads, smem, st>>>(map, a); return cudaGetLastError();
          default: break;
        }
      }
      sweep_pipe_kernel<E, MAXM, 0, 0, 16, H><<<grid, threads, smem, st>>>(map, a);
      return cudaGetLastError();
    }
    return cudaErrorInvalidConfiguration;
  }
  if (a.cw != 32) return cudaErrorInvalidConfiguration;
  if (a.mode != 0) {
    sweep_pipe_kernel<E, MAXM, 1, 0, 32, H><<<grid, threads, smem, st>>>(map, a);
    return cudaGetLastError();
  }
  if constexpr (pipe_x_specialised<MAXM>()) {
    switch (a.S) {
      case 1: sweep_pipe_kernel<E, MAXM, 0, 1, 32, H><<<grid, threads, smem, st>>>(map, a); return cudaGetLastError();
      case 2: sweep_pipe_kernel<E, MAXM, 0, 2, 32, H><<<grid, threads, smem, st>>>(map, a); return cudaGetLastError();
      case 4: sweep_pipe_kernel<E, MAXM, 0, 4, 32, H><<<grid, threads, smem, st>>>(map, a); return cudaGetLastError();
      case 8: sweep_pipe_kernel<E, MAXM, 0, 8, 32, H><<<grid, threads, smem, st>>>(map, a); return cudaGetLastError();
      default: break;
    }
  }
  sweep_pipe_kernel<E, MAXM, 0, 0, 32, H><<<grid, threads, smem, st>>>(map, a);
  return cudaGetLastError();
}

}  // namespace bfv
