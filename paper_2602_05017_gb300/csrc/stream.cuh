// Streaming line sweeps: one lane owns one whole grid line.
//
// A warp owns 32 lines and runs the Thomas recurrences (App. A) along them
// without cutting them into chunks, so no carry corrections and no barriers
// are needed.  The forward pass writes its intermediate back to memory; the
// backward pass follows at once and reads it in reverse order, so it is
// mostly still in L2.  Loads run one register block of R positions ahead.
//
// FP64 (solve_lines_f64).  The FP64 pipe of a GB300 SM retires two FMAs per
// clock, so the FP64 step is bound by its FP64 operations, not by HBM.
// Scaled form:
//   forward   h_0 = d_0,  h_i = d_i + mul_{i-1} h_{i-1}    (h_i = d'_i / inv_i)
//   backward  x_{n-1} = inv_{n-1} h_{n-1},  x_i = inv_i h_i + mul_i x_{i+1}
// (mul_i = r inv_i = -c'_i): one FMA per element along each dependency
// chain, the product inv_i h_i off the chain; h is written back in place.
// Scaled output (OUT 1, 2; the three sweeps of a whole step): from position
// k0 on, inv_i equals its interior limit sigma to the last bit, so the
// solve is run for y = x / sigma:
//   y_{n-1} = q_{n-1} h_{n-1},  y_i = q_i h_i + mul_i y_{i+1},  q_i = inv_i / sigma,
// with q_i = 1 (no multiply) past k0.  The next sweep is linear, so the
// factor passes through it; the x- and y-sweeps store y (OUT 1), the z-sweep
// stores omega y with omega = sigma_x sigma_y sigma_z (OUT 2), the true
// field.  A step then costs about 7 FP64 operations per element instead of
// 9.  Dirichlet values come in the same units.
//
// FP32 (solve_lines_f32), defect-correction form: x = c d + y with
// y = (-c r) A^-1 (L_N d); e = L_N d is formed on the fly (one position
// behind the loads, mirrored ends), the forward intermediate g goes to a
// scratch field (d stays in place for the final c d), and the backward
// pass reads g and d and writes x = c_hi d + (c_lo d + y).
//
// Interior constants.  On [k0, n-1) the coefficient tables hold one value
// per substrate (FP64: the tables are set to exactly sigma and r sigma; FP32:
// the float-rounded entries already equal the float-rounded limits), so a
// group of positions inside that range runs on two per-substrate registers
// and loads no table entry.
//
// Lanes:  x-sweep  lane = (row, substrate), rows of nx*S elements, 32/S rows
//                  per warp; the warp owns whole rows, so it also applies the
//                  source update of those rows before its solve;
//         y/z      lane = one of 32 consecutive columns of a plane (a row of a
//                  warp is one coalesced access).
// Tables: inv, mul (and q) position-major [n][S], read through L1.
#pragma once
#include "sweeps.cuh"

namespace bfv {

constexpr int kStreamThreads = 128;
constexpr int kStreamR = 16;  // positions per register block
// FP64: 16-position blocks at three CTAs per SM (168 registers), or 8-position
// blocks at four (128 registers), for grids whose lines fill few rounds of warps
template <int R>
constexpr int stream_min_blocks() {
  return R == 8 ? 4 : 3;
}

// One lane's line within the warp's group of 32 lines.
struct LaneLine {
  long long base;  // element offset of position 0
  int s;           // substrate
  bool active;     // the lane has a line
  bool face;       // the line lies on a face of the two other axes
};

// mode 0: x (grp = group of rows_per_warp rows); 1: y (grp = plane z x column
// group); 2: z (grp = column group of the whole xy plane).
__device__ __forceinline__ LaneLine lane_line(int mode, long long grp, int lane, int S, int nx,
                                              int ny, int nz, long long rowlen, int rows_per_warp) {
  LaneLine L;
  if (mode == 0) {
    const int lr = lane / S;
    L.s = lane - lr * S;
    const long long row = grp * rows_per_warp + lr;
    L.active = lr < rows_per_warp && row < (long long)ny * nz;
    const int y = (int)(row % ny), z = (int)(row / ny);
    L.face = y == 0 || y == ny - 1 || z == 0 || z == nz - 1;
    L.base = row * rowlen + L.s;
  } else {
    const long long C = mode == 1 ? rowlen : rowlen * ny;
    const long long colgroups = (C + 31) / 32;
    const long long p = grp / colgroups;
    const long long c = (grp - p * colgroups) * 32 + lane;
    L.active = c < C;
    L.s = (int)(c % S);
    const long long xy = c / S;
    if (mode == 1) {
      L.face = xy == 0 || xy == nx - 1 || p == 0 || p == nz - 1;
      L.base = p * rowlen * ny + c;
    } else {
      const int x = (int)(xy % nx), y = (int)(xy / nx);
      L.face = x == 0 || x == nx - 1 || y == 0 || y == ny - 1;
      L.base = c;
    }
  }
  return L;
}

// Coefficients of one lane's line.
template <typename E>
struct LineCoef {
  const E *inv, *mul, *q;  // this substrate's entries: position i at [i * S]
  int S, k0;
  E c0, c1;                // interior constants (FP64: sigma, r sigma; FP32: inv', mul)
  E om;                    // FP64 OUT 2: omega; FP32: c_hi
  E clo;                   // FP32: c_lo
};

struct LineDir {
  bool before, after;  // Dirichlet applications on this line
  bool face;
};

// L2 eviction priorities.  The forward intermediate must survive in L2 until
// the backward pass reads it back (stored evict_last); the final values are
// not read again by this kernel (stored evict_first), so they leave L2 first.
struct L2Pol {
  unsigned long long keep, drop;
};
__device__ __forceinline__ L2Pol make_l2pol() {
  L2Pol p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p.keep));
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p.drop));
  return p;
}
__device__ __forceinline__ void st_hint(double *p, double v, unsigned long long pol) {
  asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(p), "d"(v), "l"(pol));
}
__device__ __forceinline__ void st_hint(float *p, float v, unsigned long long pol) {
  asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(v), "l"(pol));
}
// Compiler barrier between the passes: the hinted stores are asm statements,
// so the backward pass's ordinary loads must not move above them.
__device__ __forceinline__ void pass_barrier() { asm volatile("" ::: "memory"); }

// Load R positions starting at i0 and walking by +st (fwd) or -st.
template <typename E, int R>
__device__ __forceinline__ void load_block(E (&buf)[R], const E *line, long long st, int i0,
                                           bool fwd, int n, bool active) {
  const E *q = line + (long long)i0 * st;
  const long long step = fwd ? st : -st;
#pragma unroll
  for (int k = 0; k < R; k++) {
    const int i = fwd ? i0 + k : i0 - k;
    buf[k] = (active && i >= 0 && i < n) ? *q : E(0);
    q += step;
  }
}

// FP64 solve of a warp's lines (see the header).  OUT 0: x itself; 1: x/sigma;
// 2: omega x/sigma.  KS > 0: the intermediate of positions below KS (a
// multiple of R, warp-uniform) stays in shared memory (hsm: this lane's slab, position i at
// hsm[i * 32]) -- the first positions of a line live longest between the two
// passes, so they weigh most on the L2 footprint.
template <int OUT, int R = kStreamR>
__device__ __forceinline__ void solve_lines_f64(double *line, int n, long long st, bool active,
                                                const LineCoef<double> &cf, const LineDir &dr,
                                                double dval_in, double dval,
                                                double *hsm = nullptr, int KS = 0) {
  const int S = cf.S, k0 = cf.k0, ngrp = (n + R - 1) / R;
  const L2Pol pol = make_l2pol();
  // forward groups start at multiples of R, so a group is wholly below KS or not
  auto put_h = [&](double *q, int i, double v) {
    if (KS > 0 && i < KS) hsm[i * 32] = v; else st_hint(q, v, pol.keep);
  };
  const bool dBf = dr.before && dr.face, dAf = dr.after && dr.face;
  double h = 0.0, mp = 0.0;
  auto fwd_group = [&](int g, const double(&buf)[R]) {
    if (!active) return;
    const int i0 = g * R;
    double *q = line + (long long)i0 * st;
    if (i0 - 1 >= k0 && i0 + R < n) {  // interior: mul_{i-1} = r sigma (warp-uniform)
#pragma unroll
      for (int k = 0; k < R; k++) {
        h = fma(cf.c1, h, dBf ? dval_in : buf[k]);
        put_h(q, i0 + k, h);
        q += st;
      }
      mp = cf.c1;
    } else {
#pragma unroll
      for (int k = 0; k < R; k++) {
        const int i = i0 + k;
        if (i < n) {
          double d = buf[k];
          if (dr.before && (dr.face || i == 0 || i == n - 1)) d = dval_in;
          h = fma(mp, h, d);
          put_h(q, i, (OUT != 0 && i == n - 1) ? __ldg(cf.q + (size_t)i * S) * h : h);
          mp = __ldg(cf.mul + (size_t)i * S);
        }
        q += st;
      }
    }
  };
  double x = 0.0;
  auto bwd_group = [&](int g, const double(&buf)[R]) {
    if (!active) return;
    const int i1 = n - 1 - g * R;
    double *q = line + (long long)i1 * st;
    // interior: inv = sigma, mul = r sigma, q = 1; with scaled output the first
    // position n-1 also qualifies (y_{n-1} was stored pre-scaled and mul_{n-1}
    // multiplies zero); position 0 never does (its Dirichlet end)
    if (i1 - R + 1 >= max(k0, 1) && (OUT != 0 || i1 < n - 1)) {
#pragma unroll
      for (int k = 0; k < R; k++) {
        x = fma(cf.c1, x, OUT == 0 ? cf.c0 * buf[k] : buf[k]);
        st_hint(q, dAf ? dval : (OUT == 2 ? cf.om * x : x), pol.drop);
        q -= st;
      }
      if (dr.after && i1 == n - 1) st_hint(line + (long long)(n - 1) * st, dval, pol.drop);
    } else {
#pragma unroll
      for (int k = 0; k < R; k++) {
        const int i = i1 - k;
        if (i >= 0) {
          const double hv = buf[k];
          const double t = OUT == 0 ? __ldg(cf.inv + (size_t)i * S) * hv
                                    : (i == n - 1 ? hv : __ldg(cf.q + (size_t)i * S) * hv);
          x = fma(__ldg(cf.mul + (size_t)i * S), x, t);
          st_hint(q, (dr.after && (dr.face || i == 0 || i == n - 1)) ? dval
                                                                     : (OUT == 2 ? cf.om * x : x),
                  pol.drop);
        }
        q -= st;
      }
    }
  };
  double A[R], B[R];
  // backward blocks come from shared memory below KS, from the field above
  auto load = [&](double(&buf)[R], int i0, bool fwd) {
    if (KS == 0 || fwd || i0 - R + 1 >= KS) {
      load_block<double, R>(buf, line, st, i0, fwd, n, active);
    } else {
      const double *q = line + (long long)i0 * st;
#pragma unroll
      for (int k = 0; k < R; k++) {
        const int i = i0 - k;
        buf[k] = !(active && i >= 0 && i < n) ? 0.0 : (i < KS ? hsm[i * 32] : *q);
        q -= st;
      }
    }
  };
  for (int pass = 0; pass < 2; pass++) {
    const bool fwd = pass == 0;
    pass_barrier();
    auto first = [&](int g) { return fwd ? g * R : n - 1 - g * R; };
    load(A, first(0), fwd);
    for (int g = 0; g < ngrp; g += 2) {
      load(B, first(g + 1), fwd);
      if (fwd) fwd_group(g, A); else bwd_group(g, A);
      load(A, first(g + 2), fwd);
      if (g + 1 < ngrp) {
        if (fwd) fwd_group(g + 1, B); else bwd_group(g + 1, B);
      }
    }
  }
}

// x-sweep at a substrate count XS of 1, 2 or 4 (compile time), FP64: the same
// solve as solve_lines_f64 (lane = (row, substrate), 32/XS rows per warp), but
// the warp's global loads and stores are contiguous row segments.  Lanes owning
// rows would make every load instruction touch 32/XS rows (32 cache lines at
// XS = 1); here a block of R positions of the warp's rows is read as R*XS
// consecutive elements per row ("flat": element j*32 + lane of the block is
// row f / (R*XS), offset f % (R*XS)) and transposed through the warp's buffer
// tb ([32][R+1] doubles: lane, block index) to one line per lane, and the
// results go the opposite way.  The intermediate of positions below KS stays in
// the lane's shared-memory slab hsm as in solve_lines_f64.
//   wbase: the warp's first row (position 0); nrows_w: its rows in the grid.
template <int OUT, int XS, int R = kStreamR>
__device__ __forceinline__ void solve_rows_f64(double *wbase, long long rowlen, int nrows_w,
                                               int n, bool active, const LineCoef<double> &cf,
                                               const LineDir &dr, double dval_in, double dval,
                                               double *hsm, int KS, double *tb, int lane) {
  static_assert(XS == 1 || XS == 2 || XS == 4, "rows of 1, 2 or 4 substrates");
  constexpr int B = R * XS;  // elements of one row in a block
  constexpr int P = R + 1;   // tb pitch: lanes reading their rows hit distinct bank pairs
  const int k0 = cf.k0, ngrp = (n + R - 1) / R;
  const L2Pol pol = make_l2pol();
  const bool dBf = dr.before && dr.face, dAf = dr.after && dr.face;
  // flat element j of the block: (row, offset w in the row's segment)
  auto flat = [&](int j, int &row, int &w) {
    const int f = j * 32 + lane;
    row = f / B;
    w = f % B;
  };
  // global -> registers (flat) for positions p0 .. p0+R-1
  auto gload = [&](double(&buf)[R], int p0) {
#pragma unroll
    for (int j = 0; j < R; j++) {
      int row, w;
      flat(j, row, w);
      const int pos = p0 + w / XS;
      buf[j] = (row < nrows_w && pos >= 0 && pos < n)
                   ? wbase[row * rowlen + (long long)p0 * XS + w]
                   : 0.0;
    }
  };
  // flat registers -> this lane's line: buf[k] = position p0 + k (rev: p0 + R-1-k)
  auto to_lanes = [&](double(&buf)[R], bool rev) {
#pragma unroll
    for (int j = 0; j < R; j++) {
      int row, w;
      flat(j, row, w);
      const int k = w / XS, dl = row * XS + w % XS;
      tb[dl * P + (rev ? R - 1 - k : k)] = buf[j];
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < R; k++) buf[k] = tb[lane * P + k];
    __syncwarp();
  };
  auto out_lane = [&](int k, double v) { tb[lane * P + k] = v; };
  // this block's results (out_lane) -> global, positions p0 .. p0+R-1
  auto flush = [&](int p0, bool rev, unsigned long long policy) {
    __syncwarp();
#pragma unroll
    for (int j = 0; j < R; j++) {
      int row, w;
      flat(j, row, w);
      const int k = w / XS, dl = row * XS + w % XS, pos = p0 + k;
      if (row < nrows_w && pos >= 0 && pos < n)
        st_hint(wbase + row * rowlen + (long long)p0 * XS + w, tb[dl * P + (rev ? R - 1 - k : k)],
                policy);
    }
    __syncwarp();
  };
  double h = 0.0, mp = 0.0;
  auto fwd_group = [&](int g, double(&buf)[R]) {
    const int i0 = g * R;
    to_lanes(buf, false);
    const bool sm = KS > 0 && i0 < KS;  // the whole group (KS is a multiple of R)
    if (active) {
      if (i0 - 1 >= k0 && i0 + R < n) {  // interior: mul_{i-1} = r sigma (warp-uniform)
#pragma unroll
        for (int k = 0; k < R; k++) {
          h = fma(cf.c1, h, dBf ? dval_in : buf[k]);
          if (sm) hsm[(i0 + k) * 32] = h; else out_lane(k, h);
        }
        mp = cf.c1;
      } else {
#pragma unroll
        for (int k = 0; k < R; k++) {
          const int i = i0 + k;
          if (i < n) {
            double d = buf[k];
            if (dr.before && (dr.face || i == 0 || i == n - 1)) d = dval_in;
            h = fma(mp, h, d);
            const double hv = (OUT != 0 && i == n - 1) ? __ldg(cf.q + (size_t)i * XS) * h : h;
            if (sm) hsm[i * 32] = hv; else out_lane(k, hv);
            mp = __ldg(cf.mul + (size_t)i * XS);
          }
        }
      }
    }
    if (!sm) flush(i0, false, pol.keep);
  };
  double x = 0.0;
  // backward blocks run down from n-1, so one can straddle KS: positions below
  // KS come from the lane's slab, the others from the field
  auto in_slab = [&](int i1) { return KS > 0 && i1 < KS; };
  auto bwd_group = [&](int g, double(&buf)[R]) {
    const int i1 = n - 1 - g * R;
    if (!in_slab(i1)) {
      to_lanes(buf, true);
      if (KS > 0 && i1 - R + 1 < KS) {
#pragma unroll
        for (int k = 0; k < R; k++) {
          const int i = i1 - k;
          if (active && i >= 0 && i < KS) buf[k] = hsm[i * 32];
        }
      }
    }
    if (active) {
      if (i1 - R + 1 >= max(k0, 1) && (OUT != 0 || i1 < n - 1)) {
#pragma unroll
        for (int k = 0; k < R; k++) {
          x = fma(cf.c1, x, OUT == 0 ? cf.c0 * buf[k] : buf[k]);
          out_lane(k, dAf ? dval : (OUT == 2 ? cf.om * x : x));
        }
        if (dr.after && i1 == n - 1) out_lane(0, dval);
      } else {
#pragma unroll
        for (int k = 0; k < R; k++) {
          const int i = i1 - k;
          if (i >= 0) {
            const double hv = buf[k];
            const double t = OUT == 0 ? __ldg(cf.inv + (size_t)i * XS) * hv
                                      : (i == n - 1 ? hv : __ldg(cf.q + (size_t)i * XS) * hv);
            x = fma(__ldg(cf.mul + (size_t)i * XS), x, t);
            out_lane(k, (dr.after && (dr.face || i == 0 || i == n - 1)) ? dval
                                                                        : (OUT == 2 ? cf.om * x : x));
          }
        }
      }
    }
    flush(i1 - R + 1, true, pol.drop);
  };
  double A[R], Bf[R];
  // backward blocks wholly below KS from the slab; the others from the field
  // (loaded flat, transposed at use)
  auto bload = [&](double(&buf)[R], int i1) {
    if (in_slab(i1)) {
#pragma unroll
      for (int k = 0; k < R; k++) {
        const int i = i1 - k;
        buf[k] = (active && i >= 0 && i < n) ? hsm[i * 32] : 0.0;
      }
    } else {
      gload(buf, i1 - R + 1);
    }
  };
  pass_barrier();
  gload(A, 0);
  for (int g = 0; g < ngrp; g += 2) {
    gload(Bf, (g + 1) * R);
    fwd_group(g, A);
    gload(A, (g + 2) * R);
    if (g + 1 < ngrp) fwd_group(g + 1, Bf);
  }
  pass_barrier();
  bload(A, n - 1);
  for (int g = 0; g < ngrp; g += 2) {
    bload(Bf, n - 1 - (g + 1) * R);
    bwd_group(g, A);
    bload(A, n - 1 - (g + 2) * R);
    if (g + 1 < ngrp) bwd_group(g + 1, Bf);
  }
}

// FP32 defect-correction solve of a warp's lines (see the header); sline is
// the scratch field at the same offset as line.  KS > 0: for positions below
// KS (a multiple of R) both g and d stay in shared memory (gsm, dsm: this
// lane's slabs, position i at [i * 32]), since they live longest between the
// two passes.
template <int R = kStreamR, int KS = 0>
__device__ __forceinline__ void solve_lines_f32(float *line, float *sline, int n, long long st,
                                                bool active, const LineCoef<float> &cf,
                                                const LineDir &dr, float dval_in, float dval,
                                                float *gsm = nullptr, float *dsm = nullptr) {
  const int S = cf.S, k0 = cf.k0, ngrp = (n + R - 1) / R;
  const L2Pol pol = make_l2pol();
  auto dmod = [&](float v, int i) {
    return (dr.before && (dr.face || i == 0 || i == n - 1)) ? dval_in : v;
  };
  // ---- forward: d_i arrives, position p = i - 1 is eliminated
  float g = 0.f, dm1 = 0.f, dm2 = 0.f;
  auto emit = [&](int p, float e, bool interior, float *sq) {
    const float iv = interior ? cf.c0 : __ldg(cf.inv + (size_t)p * S);
    const float mu = interior ? cf.c1 : __ldg(cf.mul + (size_t)p * S);
    g = fmaf(mu, g, e * iv);
    if (KS > 0 && p < KS) gsm[p * 32] = g; else st_hint(sq, g, pol.keep);
  };
  auto fwd_group = [&](int gi, const float(&buf)[R]) {
    if (!active) return;
    const int i0 = gi * R;
    const bool interior = i0 - 1 >= k0 && i0 + R - 2 < n - 1;
    float *sq = sline + (long long)(i0 - 1) * st;  // position i - 1
#pragma unroll
    for (int k = 0; k < R; k++) {
      const int i = i0 + k;
      if (i < n) {
        if (KS > 0 && i < KS) dsm[i * 32] = buf[k];
        const float d = dmod(buf[k], i);
        if (i == 0) {
          dm1 = d;
          dm2 = d;  // mirrored start: d_{-1} = d_0
        } else {
          emit(i - 1, (dm1 - dm2) + (dm1 - d), interior, sq);
          dm2 = dm1;
          dm1 = d;
        }
      }
      sq += st;
    }
  };
  // ---- backward: y_i = g_i + mul_i y_{i+1}, x_i = c_hi d_i + (c_lo d_i + y_i)
  float y = 0.f;
  auto bwd_group = [&](int gi, const float(&gb)[R], const float(&db)[R]) {
    if (!active) return;
    const int i1 = n - 1 - gi * R;
    const bool interior = i1 < n - 1 && i1 - R + 1 >= k0;
    float *q = line + (long long)i1 * st;
#pragma unroll
    for (int k = 0; k < R; k++) {
      const int i = i1 - k;
      if (i >= 0) {
        const float mu = interior ? cf.c1 : __ldg(cf.mul + (size_t)i * S);
        y = fmaf(mu, y, gb[k]);
        const float d = dmod(db[k], i);
        const float xv = fmaf(cf.om, d, fmaf(cf.clo, d, y));
        st_hint(q, (dr.after && (dr.face || i == 0 || i == n - 1)) ? dval : xv, pol.drop);
      }
      q -= st;
    }
  };
  {
    float A[R], B[R];
    load_block<float, R>(A, line, st, 0, true, n, active);
    for (int gi = 0; gi < ngrp; gi += 2) {
      load_block<float, R>(B, line, st, (gi + 1) * R, true, n, active);
      fwd_group(gi, A);
      load_block<float, R>(A, line, st, (gi + 2) * R, true, n, active);
      if (gi + 1 < ngrp) fwd_group(gi + 1, B);
    }
    if (active && n > 0) emit(n - 1, dm1 - dm2, false, sline + (long long)(n - 1) * st);
  }
  pass_barrier();
  {
    // backward blocks: shared memory below KS, global above
    auto load2 = [&](float(&gb)[R], float(&db)[R], int i1) {
      if (KS == 0 || i1 - R + 1 >= KS) {
        load_block<float, R>(gb, sline, st, i1, false, n, active);
        load_block<float, R>(db, line, st, i1, false, n, active);
      } else {
        const float *qs = sline + (long long)i1 * st, *qd = line + (long long)i1 * st;
#pragma unroll
        for (int k = 0; k < R; k++) {
          const int i = i1 - k;
          const bool ok = active && i >= 0 && i < n;
          gb[k] = !ok ? 0.f : (i < KS ? gsm[i * 32] : *qs);
          db[k] = !ok ? 0.f : (i < KS ? dsm[i * 32] : *qd);
          qs -= st;
          qd -= st;
        }
      }
    };
    float GA[R], DA[R], GB[R], DB[R];
    load2(GA, DA, n - 1);
    for (int gi = 0; gi < ngrp; gi += 2) {
      load2(GB, DB, n - 1 - (gi + 1) * R);
      bwd_group(gi, GA, DA);
      load2(GA, DA, n - 1 - (gi + 2) * R);
      if (gi + 1 < ngrp) bwd_group(gi + 1, GB, DB);
    }
  }
}

// Source update of a warp's rows (x-sweep), then visible to the whole warp.
// fac (or NULL): per-substrate factor on alpha when the field is stored scaled.
// The entries are unique elements (aggregated and sorted on the host), so a
// lane issues the loads of U entries before any of their read-modify-writes:
// two rounds of memory latency per U entries instead of two per entry.
template <typename E>
__device__ __forceinline__ void warp_rows_src(E *rho, long long r0, long long r1,
                                              const int64_t *row_off, const int64_t *elem,
                                              const void *alpha, const void *scale, int lane,
                                              const void *fac = nullptr, int S = 1) {
  constexpr int U = 4;
  const long long e0 = row_off[r0], e1 = row_off[r1];
  for (long long eb = e0 + lane; eb < e1; eb += 32 * U) {
    long long k[U];
    E al[U], sc[U], v[U];
#pragma unroll
    for (int j = 0; j < U; j++) {
      const long long e = eb + 32 * j;
      k[j] = e < e1 ? __ldg(elem + e) : -1;
      al[j] = e < e1 ? ldg<E>(alpha, e) : E(0);
      sc[j] = e < e1 ? ldg<E>(scale, e) : E(0);
    }
#pragma unroll
    for (int j = 0; j < U; j++) {
      v[j] = k[j] >= 0 ? rho[k[j]] : E(0);
      if (fac && k[j] >= 0) al[j] *= ldg<E>(fac, (int)(k[j] % S));
    }
#pragma unroll
    for (int j = 0; j < U; j++)
      if (k[j] >= 0) rho[k[j]] = (v[j] + al[j]) * sc[j];
  }
  __syncwarp();
}

// Single-grid streaming sweep, persistent grid of 128-thread CTAs; E = double
// (OUT as above) or float (defect form, OUT 0, scratch field a.scratch).
// XS > 0 (FP64 x-sweep at S = XS = 1, 2 or 4): coalesced rows (solve_rows_f64),
// each warp's transpose buffer after the CTA's slabs.  R: positions per
// register block (FP64: 16, or 8 at four CTAs per SM).

template <typename E, int OUT, int XS = 0, int R = kStreamR>
__global__ void __launch_bounds__(kStreamThreads, sizeof(E) == 8 ? stream_min_blocks<R>() : 4)
    stream_sweep_kernel(const StreamArgs a) {
  extern __shared__ __align__(16) unsigned char stream_smem[];
  const int S = a.S, n = a.n, flags = a.flags;
  const int lane = threadIdx.x & 31;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long nrows = (long long)a.ny * a.nz;
  E *const rho = static_cast<E *>(a.rho);
  const long long rowlen = (long long)a.nx * S;
  const E *tinv = static_cast<const E *>(a.tab);
  for (long long grp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; grp < a.ngroups;
       grp += nwarps) {
    const LaneLine L = lane_line(a.mode, grp, lane, S, a.nx, a.ny, a.nz, rowlen, a.rows_per_warp);
    if (a.mode == 0 && (flags & kSrc) && a.has_src) {
      const long long r0 = grp * a.rows_per_warp;
      warp_rows_src<E>(rho, r0, min(r0 + a.rows_per_warp, nrows), a.src_row_off, a.src_elem,
                       a.src_alpha, a.src_scale, lane, a.src_fac, S);
    }
    if (!(flags & kSolve)) continue;
    const bool dirl = L.active && (flags & (kDirBefore | kDirAfter)) && a.dir_on[L.s];
    LineDir dr;
    dr.before = dirl && (flags & kDirBefore);
    dr.after = dirl && (flags & kDirAfter);
    dr.face = L.face;
    const E dval = dirl ? dir_value<E>(flags, a.dir_val, L.s) : E(0);
    const E dval_in = dirl ? dir_value<E>(flags, a.dir_val_in, L.s) : E(0);
    LineCoef<E> cf;
    cf.S = S;
    cf.k0 = a.k0;
    cf.inv = tinv + L.s;
    cf.mul = tinv + (size_t)n * S + L.s;
    cf.q = tinv + 2 * (size_t)n * S + L.s;
    cf.c0 = L.active ? ldg<E>(a.interior, L.s) : E(0);
    cf.c1 = L.active ? ldg<E>(a.interior, S + L.s) : E(0);
    cf.clo = E(0);
    E *line = rho + (L.active ? L.base : 0);
    if constexpr (sizeof(E) == 8) {
      cf.om = (OUT == 2 && L.active) ? ldg<E>(a.omega, L.s) : E(1);
      double *hsm = reinterpret_cast<double *>(stream_smem) +
                    (size_t)(threadIdx.x >> 5) * a.ks * 32 + lane;
      if constexpr (XS > 0) {  // x-sweep, S = XS
        const long long r0 = grp * a.rows_per_warp;
        double *tb = reinterpret_cast<double *>(stream_smem) +
                     (size_t)(kStreamThreads / 32) * a.ks * 32 +
                     (size_t)(threadIdx.x >> 5) * 32 * (R + 1);
        solve_rows_f64<OUT, XS, R>(rho + r0 * rowlen, rowlen,
                                          (int)min((long long)a.rows_per_warp, nrows - r0), n,
                                          L.active, cf, dr, dval_in, dval, hsm, a.ks, tb, lane);
      } else {
        solve_lines_f64<OUT, R>(line, n, a.stride, L.active, cf, dr, dval_in, dval, hsm, a.ks);
      }
    } else {
      cf.om = L.active ? ldg<E>(a.cfix, L.s) : E(0);
      cf.clo = L.active ? ldg<E>(a.cfix, S + L.s) : E(0);
      E *sline = static_cast<E *>(a.scratch) + (L.active ? L.base : 0);
      solve_lines_f32(line, sline, n, a.stride, L.active, cf, dr, dval_in, dval);
    }
  }
}

// Shared memory of one CTA: the warps' slabs of ks positions (FP64), and with
// xs > 0 their transpose buffers of blocks of r positions.
inline size_t stream_smem_bytes(int ks, size_t esz, int xs = 0, int r = kStreamR) {
  if (esz != 8) return 0;
  return (size_t)(kStreamThreads / 32) *
         ((size_t)ks * 32 + (xs > 0 ? (size_t)32 * (r + 1) : 0)) * sizeof(double);
}

// Raise the dynamic shared-memory limit of the FP64 instantiations (once per
// handle, outside any graph capture).
template <typename E>
cudaError_t allow_stream_smem() {
  cudaError_t e = cudaSuccess;
  auto set = [&](const void *f) {
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kMaxDynamicSmem);
  };
  set((const void *)stream_sweep_kernel<E, 0>);
  set((const void *)stream_sweep_kernel<E, 1>);
  set((const void *)stream_sweep_kernel<E, 2>);
  if constexpr (sizeof(E) == 8) {
    set((const void *)stream_sweep_kernel<E, 0, 1>);
    set((const void *)stream_sweep_kernel<E, 1, 1>);
    set((const void *)stream_sweep_kernel<E, 0, 2>);
    set((const void *)stream_sweep_kernel<E, 1, 2>);
    set((const void *)stream_sweep_kernel<E, 0, 4>);
    set((const void *)stream_sweep_kernel<E, 1, 4>);
    set((const void *)stream_sweep_kernel<E, 0, 0, 8>);
    set((const void *)stream_sweep_kernel<E, 1, 0, 8>);
    set((const void *)stream_sweep_kernel<E, 2, 0, 8>);
    set((const void *)stream_sweep_kernel<E, 0, 1, 8>);
    set((const void *)stream_sweep_kernel<E, 1, 1, 8>);
    set((const void *)stream_sweep_kernel<E, 0, 2, 8>);
    set((const void *)stream_sweep_kernel<E, 1, 2, 8>);
  }
  return e;
}

// a.xt (FP64 x-sweep): 1, 2 or 4 for the coalesced-row form, else 0.  The
// x-sweep never renormalises (OUT 2), so only OUT 0 and 1 have that form.
// a.r8 (FP64): 8-position blocks at four CTAs per SM (XS 0, 1, 2 only).
template <typename E, int OUT>
cudaError_t launch_stream_one(const StreamArgs &a, int grid, cudaStream_t st) {
  if constexpr (sizeof(E) == 8) {
    if (a.r8) {
      const size_t sm = stream_smem_bytes(a.ks, sizeof(E), a.xt, 8);
      if constexpr (OUT != 2) {
        switch (a.xt) {
          case 1: stream_sweep_kernel<E, OUT, 1, 8><<<grid, kStreamThreads, sm, st>>>(a); return cudaGetLastError();
          case 2: stream_sweep_kernel<E, OUT, 2, 8><<<grid, kStreamThreads, sm, st>>>(a); return cudaGetLastError();
          default: break;
        }
      }
      if (a.xt != 0) return cudaErrorInvalidValue;
      stream_sweep_kernel<E, OUT, 0, 8><<<grid, kStreamThreads, sm, st>>>(a);
      return cudaGetLastError();
    }
  }
  if constexpr (sizeof(E) == 8 && OUT != 2) {
    const size_t sm = stream_smem_bytes(a.ks, sizeof(E), a.xt);
    switch (a.xt) {
      case 1: stream_sweep_kernel<E, OUT, 1><<<grid, kStreamThreads, sm, st>>>(a); return cudaGetLastError();
      case 2: stream_sweep_kernel<E, OUT, 2><<<grid, kStreamThreads, sm, st>>>(a); return cudaGetLastError();
      case 4: stream_sweep_kernel<E, OUT, 4><<<grid, kStreamThreads, sm, st>>>(a); return cudaGetLastError();
      default: break;
    }
  }
  if (a.xt != 0 || a.r8) return cudaErrorInvalidValue;
  stream_sweep_kernel<E, OUT><<<grid, kStreamThreads, stream_smem_bytes(a.ks, sizeof(E)), st>>>(a);
  return cudaGetLastError();
}

}  // namespace bfv
