// Host half of libbiofvm: the C ABI of include/biofvm.h.
//
// Owns the handle, validates arguments, computes the Thomas constants of
// Appendix A in double (computed once and kept, as the paper's solver keeps
// them after its first iteration), chooses the launch plan of each sweep
// (FP64: streaming whole lines; FP32: the TMA pipeline; plain kernels as the
// fallback), aggregates agents into per-element source terms, captures blocks
// of steps into CUDA graphs, and maps CUDA failures to status codes.  All
// compute runs in the kernels of sweeps_fp64.cu / sweeps_fp32.cu / noalloc.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/biofvm.h"
#include "agents.h"
#include "batch_args.h"
#include "pipe_args.h"
#include "internal.h"

using namespace bfv;

namespace {

thread_local std::string g_last_error;

biofvm_status fail(biofvm_status st, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}

#define CK(call)                                                                   \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess)                                                         \
      return fail(BIOFVM_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// Device buffer owned by a handle.
struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
};

cudaError_t dev_alloc(DevBuf &b, size_t bytes) {
  b.release();
  if (bytes == 0) return cudaSuccess;
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e == cudaSuccess) b.bytes = bytes;
  return e;
}

struct ColPlan {
  int T = 1, m = 1, maxm = 8;
  int nosolve = 0;  // lines too long for register chunks: streaming or pipelined solve only
};
// Persistent TMA pipeline of one FP32 sweep (used when rows are 16-byte aligned
// and a ring of >= 2 stages with the constants fits in shared memory; otherwise
// the plain kernels).
struct PipePlan {
  int use = 0, T = 1, m = 1, maxm = 8;
  int cw = 32, W = 1;  // columns per tile (32, or 16 for long lines); consumer warps
  int box_rows = 0, nbox = 0, rows_per_tile = 0, pitch = 0;
  int stages = 0, grid = 0;
  int64_t stage_elems = 0, ntiles = 0;
  size_t smem = 0;
  CUtensorMap map[2]{};  // y/z: [0] the field, [1] the adjoint field
  int have_map[2]{};
};
constexpr int kMaxRenorm = 16;  // steps between renormalisations of the scaled FP64 field
constexpr int kRenormRows = 9;  // per-step constant rows of the scaled FP64 step

struct StreamPlan {
  int use = 0, grid = 0;
  int r8 = 0;  // FP64: 8-position register blocks at four CTAs per SM (else 16 at three)
};
struct XPlan {
  int T = 1, m = 1, maxm = 8, rows_per_warp = 1, warps = 1, rows_per_cta = 1, use_bulk = 0;
  int nosolve = 0;  // rows too long to cut into register chunks: only non-solve stages
  size_t smem = 0;
};

}  // namespace

struct biofvm {
  biofvm_grid g{};
  double dx = 0, dt = 0;
  double h3[3] = {0, 0, 0};  // voxel spacing along x, y, z (all dx unless set apart)
  std::vector<double> D, lam;
  std::vector<uint8_t> dir_on;
  std::vector<double> dir_val;
  bool any_dir = false;
  biofvm_precision prec = BIOFVM_FP64;
  size_t esz = 8;  // field element (storage): 8, 4, or 2 for bf16 / fp16
  size_t csz = 8;  // arithmetic and constants: 8 for FP64, else 4
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  size_t nel = 0;
  DevBuf rho, tab[3], tabT[3], dir_on_d, dir_val_d, status;
  // streaming sweep (FP64): [3][n][S] inv, mul, q per axis; Dirichlet values
  // in the units of each sweep's scaled output [3][S]; omega [S]; k0 per axis
  DevBuf tabS[3], stream_const_d;
  int stream_k0[3] = {0, 0, 0};
  XPlan xp;
  ColPlan cp[3];  // [1] = y, [2] = z
  PipePlan pp[3];
  // FP32 fields whose rows (nx*S elements) are not 16-byte multiples, which the TMA copies
  // need: biofvm_step runs the pipelined sweeps on a row-padded working copy (rows gpitch
  // elements apart, the padding zero), copied in at the start of the call and back at its
  // end.  ppx: the plans over that copy; tabP / tabTP: their axis tables when a plan's chunk
  // partition differs from the one the handle's own tables follow (tabP_own)
  int pitched = 0, gpitch = 0, pitched_enabled = 1;
  DevBuf prow, tabP[3], tabTP[3];
  int tabP_own[3] = {0, 0, 0};
  PipePlan ppx[3];
  StreamPlan sp[3];
  int num_sms = 0;
  int pipe_enabled = 1;
  int stream_enabled = 1;
  int stream_ctas_per_sm = 3;
  int stream_ks = 64;        // FP64: positions of each line's intermediate kept in shared memory
  // FP64 x-sweep at S = 1, 2 (BIOFVM_STREAM_XT=4: also 4): coalesced rows through per-warp
  // transpose buffers, with slabs of stream_ks_xt positions
  int stream_xt = 2, stream_ks_xt = 32;
  // FP64: 8-position register blocks at four CTAs per SM instead of 16 at three (per axis,
  // StreamPlan::r8; -1: chosen by the planner, 0 / 1 forced)
  int stream_r8_mode = -1;
  int stream32_enabled = 0;  // FP32 streaming sweeps instead of the pipelined ones
  // small FP64 grids: whole biofvm_step calls in one cooperative launch (small.cu)
  int small_enabled = 1, small_use = 0, small_grid = 0;
  size_t small_smem = 0;
  DevBuf small_bar;
  int small_T[3] = {1, 1, 1}, small_m[3] = {1, 1, 1};  // chunks per axis of the small step
  DevBuf small_tab[3];                                   // their axis tables
  int pipe_chunk = 0;        // FP32 pipelined sweeps: chunk length (0: the planner's)
  int pipe_cw = 0;           // FP32 pipelined sweeps: lines per tile, 32 or 16 (0: the planner's)
  int pipe_ns = 4;           // FP32 pipelined sweeps: most ring stages per CTA
  DevBuf scratch;            // FP32 streaming: forward intermediate, field-sized
  int forced = 0;  // chunk lengths fixed by the caller (batched environments)
  unsigned generation = 0;  // bumped when kernel arguments change (sources, constants)
  // sources
  int64_t n_entries = 0;
  DevBuf src_row_off, src_elem, src_rowcol, src_alpha, src_scale;
  // source lists rebuilt on the device from device agent arrays (biofvm_set_sources_device):
  // buffers reserved for up to agents_max agents, used instead of the host-built lists while
  // sources_device is set (their length lives on the device: dsrc_count)
  int64_t agents_max = 0;
  bool sources_device = false;
  DevBuf dsrc_row_off, dsrc_elem, dsrc_rowcol, dsrc_alpha, dsrc_scale, dsrc_count;
  DevBuf ag_key[2], ag_idx[2], ag_ea, ag_eb, ag_head, ag_pos, ag_hist, ag_part, ag_count32;
  // step graphs: [0] a block of renorm_k steps, [r] a tail of r < renorm_k steps
  cudaGraph_t graph[kMaxRenorm + 1] = {};
  cudaGraphExec_t gexec[kMaxRenorm + 1] = {};
  // FP64 streaming step: the field stays scaled by omega^-m for m < renorm_k
  // steps (no multiply by omega in the z-sweep) and is brought back every
  // renorm_k steps and at the end of every biofvm_step call; renorm_d holds the
  // per-step constants [renorm_k][kRenormRows][S] (see upload_constants)
  int renorm_k = 1;
  DevBuf renorm_d;
  // adjoint: the adjoint field, reduction partials, agents on the device
  DevBuf adj, partial, ag_elem, ag_entry, ag_weight, ag_target;
  int reduce_blocks = 0;
  bool agents_on_device = false;
  std::vector<int64_t> h_voxel, h_src_elem;
  std::vector<double> h_weight, h_target;
  // the agents as last given (the source list is rebuilt when the nodes change)
  std::vector<double> h_secretion, h_uptake;
  // Dirichlet nodes (biofvm_set_dirichlet_nodes): the caller's list, sorted by
  // element with the last value of a repeated element, and the list the
  // kernels apply: those nodes plus, for a substrate whose flagged faces hold a
  // node, its face voxels (the fused face application then skips that
  // substrate: dir_on_k), so that nodes always win over faces
  std::vector<int64_t> h_dn_elem, h_dn_kelem;
  std::vector<double> h_dn_val;
  std::vector<uint8_t> dir_on_k;  // face flags the kernels apply
  int64_t n_dnode = 0;            // nodes the kernels apply
  DevBuf dn_elem, dn_val;
};

namespace {

int axis_len(const biofvm *h, int axis) {
  return axis == 0 ? h->g.nx : axis == 1 ? h->g.ny : h->g.nz;
}

void drop_graphs(biofvm *h) {
  for (int r = 0; r <= kMaxRenorm; r++) {
    if (h->gexec[r]) cudaGraphExecDestroy(h->gexec[r]);
    if (h->graph[r]) cudaGraphDestroy(h->graph[r]);
    h->gexec[r] = nullptr;
    h->graph[r] = nullptr;
  }
}

// ---------------------------------------------------------------------------
// Appendix A constants (double) and chunk products for one axis.
// ---------------------------------------------------------------------------
void axis_constants(int n, double r, double lam3, double *inv, double *mul) {
  // a_i = c_i = -r; b = 1 + 2r + lam3 inside, 1 + r + lam3 at the ends,
  // 1 + lam3 when the axis has a single voxel (no neighbour to exchange with).
  auto b = [&](int i) {
    if (n == 1) return 1.0 + lam3;
    return (i == 0 || i == n - 1) ? 1.0 + r + lam3 : 1.0 + 2.0 * r + lam3;
  };
  double denom = b(0);
  for (int i = 0; i < n; i++) {
    if (i > 0) denom = b(i) - r * (r / denom);  // b_i - a_i c'_{i-1}, c'_{i-1} = -r/denom_{i-1}
    inv[i] = 1.0 / denom;
    mul[i] = r / denom;
  }
}

// Host tables of one axis in double, layout [i][S], [t][S] and [2][S].  With
// `defect` (FP32 path) inv is scaled by -c r and cfix holds c = 1/(1+lam3) as
// a (hi, lo) pair of floats.
void axis_tables(const biofvm *h, int axis, int T, int m, bool defect, std::vector<double> &out) {
  const int n = axis_len(h, axis), S = h->g.n_sub;
  out.assign((size_t)4 * n * S + (size_t)T * S + 2 * (size_t)S + (size_t)T * T * S, 0.0);
  double *inv = out.data(), *mul = inv + (size_t)n * S, *pf = mul + (size_t)n * S,
         *pb = pf + (size_t)n * S, *pc = pb + (size_t)n * S, *cfix = pc + (size_t)T * S,
         *cw = cfix + 2 * (size_t)S;
  std::vector<double> ci(n), cm(n);
  for (int s = 0; s < S; s++) {
    const double r = h->D[s] * h->dt / (h->h3[axis] * h->h3[axis]);
    const double lam3 = h->lam[s] * h->dt / 3.0;
    const double c = 1.0 / (1.0 + lam3);
    const double scale = defect ? -c * r : 1.0;
    const float c_hi = (float)c;
    cfix[s] = c_hi;
    cfix[S + s] = (float)(c - (double)c_hi);
    axis_constants(n, r, lam3, ci.data(), cm.data());
    for (int i = 0; i < n; i++) {
      inv[(size_t)i * S + s] = scale * ci[i];
      mul[(size_t)i * S + s] = cm[i];
    }
    for (int t = 0; t < T; t++) {
      const int lo = t * m, hi = std::min(n, lo + m) - 1;
      double p = 1.0;
      for (int i = lo; i <= hi; i++) {
        p *= cm[i];
        pf[(size_t)i * S + s] = p;
      }
      pc[(size_t)t * S + s] = p;
      p = 1.0;
      for (int i = hi; i >= lo; i--) {
        p *= cm[i];
        pb[(size_t)i * S + s] = p;
      }
    }
    // carry weight between chunks u and t: the product of pc over the chunks
    // strictly between them (the same in both directions)
    for (int u = 0; u < T; u++)
      for (int t = 0; t < T; t++) {
        double w = 1.0;
        for (int v = std::min(u, t) + 1; v < std::max(u, t); v++) w *= pc[(size_t)v * S + s];
        cw[((size_t)u * T + t) * S + s] = w;
      }
  }
}

// ---------------------------------------------------------------------------
// Launch plans.
// ---------------------------------------------------------------------------
int pick_maxm(int m, bool fp64) {
  if (fp64) {
    for (int c : kMaxmF64)
      if (c >= m) return c;
  } else {
    for (int c : kMaxmF32)
      if (c >= m) return c;
  }
  return 0;
}

// Threads a column-sweep CTA may use for a chunk capacity (mirrors ColBound).
int col_bound_threads(int maxm, size_t esz) {
  const int regs = maxm * (int)esz / 4 + 64;
  const int raw = 65536 / regs;
  return std::min(1024, raw) / 32 * 32;
}

bool plan_col(int n, bool fp64, ColPlan &p, int forced_m = 0) {
  const size_t esz = fp64 ? 8 : 4;
  if (forced_m > 0) {
    const int m = std::min(forced_m, n);
    const int T = (n + m - 1) / m;
    const int maxm = pick_maxm(m, fp64);
    if (maxm == 0 || T * 32 > col_bound_threads(maxm, esz)) return false;
    p.T = T;
    p.m = m;
    p.maxm = maxm;
    return true;
  }
  for (int target = 32; target <= 128; target *= 2) {
    // chunks of exactly `target` positions (the last one shorter): every full
    // chunk then matches its compiled capacity and takes the unguarded path
    int T = (n + target - 1) / target;
    if (T < 1) T = 1;
    const int m = T == 1 ? n : target;
    const int maxm = pick_maxm(m, fp64);
    if (maxm == 0) return false;
    if (T * 32 <= col_bound_threads(maxm, esz)) {
      p.T = T;
      p.m = m;
      p.maxm = maxm;
      return true;
    }
  }
  return false;
}

// Plan of the plain x-sweep.  When the rows cannot be cut into register
// chunks (more than 32/S chunks of the largest capacity) and `allow_nosolve`,
// the plan still stages rows for the stages that do not solve (the source
// update alone, a Dirichlet application alone); the solve then has to come
// from the streaming or pipelined x-sweep.
bool plan_x(int nx, int S, bool fp64, XPlan &p, int forced_m = 0, bool allow_nosolve = false) {
  const size_t esz = fp64 ? 8 : 4;
  const int Tmax = 32 / S;
  if (Tmax < 1) return false;
  const int largest = fp64 ? 64 : 128;
  const int target = fp64 ? 48 : 64;
  int T = std::min(Tmax, (nx + target - 1) / target);
  if (T < 1) T = 1;
  int m = (nx + T - 1) / T;
  if (m > largest) {
    T = std::min(Tmax, (nx + largest - 1) / largest);
    m = (nx + T - 1) / T;
  }
  if (forced_m > 0) m = std::min(forced_m, nx);
  T = (nx + m - 1) / m;
  p.nosolve = 0;
  if (m > largest || T > Tmax) {
    if (!allow_nosolve || forced_m > 0) return false;
    T = 1;
    m = nx;
    p.nosolve = 1;
  }
  p.T = T;
  p.m = m;
  p.maxm = p.nosolve ? (fp64 ? kMaxmF64[0] : kMaxmF32[0]) : pick_maxm(m, fp64);
  p.rows_per_warp = p.nosolve ? 1 : 32 / (T * S);  // lanes per row matter to the solve only
  const size_t rowbytes = (size_t)nx * S * esz;
  const size_t tabbytes = (4 * (size_t)nx * S + (size_t)T * S + 2 * (size_t)S) * esz + 32;
  p.use_bulk = (rowbytes % 16 == 0) ? 1 : 0;
  for (size_t budget : {(size_t)100 * 1024, (size_t)220 * 1024}) {
    for (int w = 8; w >= 1; w--) {
      const size_t rows = (size_t)w * p.rows_per_warp;
      const size_t smem = rows * rowbytes + tabbytes;
      if (smem <= budget) {
        p.warps = w;
        p.rows_per_cta = (int)rows;
        p.smem = (smem + 127) / 128 * 128;
        return true;
      }
    }
  }
  return false;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// Tensor map of axis 1/2 over `field` with rows gp elements apart ([nplanes][n]
// lines of C columns: y: C = nx*S columns of a row, rows gp apart; z: C = ny*gp
// columns of a plane) into p.map[buf]; box cw x box_rows.
bool encode_pipe_map(biofvm *h, PipePlan &p, int axis, int buf, void *field, int64_t gp) {
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return false;
  const int64_t nx = h->g.nx, ny = h->g.ny, nz = h->g.nz, S = h->g.n_sub;
  const int64_t C = axis == 1 ? nx * S : ny * gp;
  const int64_t n = axis == 1 ? ny : nz, nplanes = axis == 1 ? nz : 1;
  const int64_t lstride = axis == 1 ? gp : ny * gp;  // elements between positions of a line
  const size_t esz = h->esz;
  cuuint64_t dims[3] = {(cuuint64_t)C, (cuuint64_t)n, (cuuint64_t)nplanes};
  cuuint64_t strides[2] = {(cuuint64_t)(lstride * esz), (cuuint64_t)(lstride * esz * n)};
  cuuint32_t box[3] = {(cuuint32_t)p.cw, (cuuint32_t)p.box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  const CUtensorMapDataType dtype =
      h->prec == BIOFVM_FP64   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
      : h->prec == BIOFVM_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
      : h->prec == BIOFVM_FP16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                               : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  CUresult r = enc(&p.map[buf], dtype, 3,
                   field, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  p.have_map[buf] = r == CUDA_SUCCESS;
  return p.have_map[buf] != 0;
}

// Bank-conflict degree of 32 lanes reading column c at (c/S)*pitch + c%S
// (x tiles, pitch in elements): the largest number of distinct 4-byte words a
// bank serves (lanes on one word share it: 16-bit elements pair up), or for
// FP64 the largest number of lanes sharing a bank pair within a half warp.
// half_off >= 0 (tiles of 16 columns): lanes 16..31 read columns 0..15 of the
// next chunk, half_off elements further on.
int x_tile_conflicts(int64_t pitch, int S, int lanes, size_t esz, int64_t half_off = -1) {
  int worst = 0;
  if (esz == 8) {
    for (int half = 0; half < 2; half++) {
      int cnt[16] = {0};
      for (int c = half * 16; c < std::min(lanes, half * 16 + 16); c++)
        worst = std::max(worst, ++cnt[(int)(((c / S) * pitch + c % S) & 15)]);
    }
    return worst;
  }
  std::vector<int64_t> words[32];
  for (int l = 0; l < 32; l++) {
    const int c = half_off >= 0 ? (l & 15) : l;
    if (c >= lanes) continue;
    const int64_t e = (c / S) * pitch + c % S + (half_off >= 0 && l >= 16 ? half_off : 0);
    const int64_t word = e * (int64_t)esz / 4;
    std::vector<int64_t> &w = words[word & 31];
    if (std::find(w.begin(), w.end(), word) == w.end()) w.push_back(word);
    worst = std::max(worst, (int)w.size());
  }
  return worst;
}

// Plan the pipelined sweep of axis 0 (x), 1 (y) or 2 (z) over `field`, whose
// rows (nx*S elements) start gp elements apart; leaves p.use = 0 when the plain
// kernels have to be used instead.  Tiles of 32 columns when a ring of >= 2
// stages of them fits in shared memory with the constants, else tiles of 16
// columns (long lines; two chunks per consumer warp).
void plan_pipe(biofvm *h, int axis, PipePlan &p, int64_t gp, void *field) {
  p = PipePlan{};
  const int64_t nx = h->g.nx, ny = h->g.ny, nz = h->g.nz, S = h->g.n_sub;
  const size_t esz = h->esz, csz = h->csz;
  const int n = axis_len(h, axis);
  if (h->prec == BIOFVM_FP64) return;  // FP64 streams whole lines instead
  const bool h16 = esz == 2;  // 16-bit storage: chunk capacities 32 and 64 compiled
  for (int cw : {32, 16}) {
    if (h->pipe_cw && cw != h->pipe_cw) continue;
    PipePlan q{};
    q.cw = cw;
    const int cpw = 32 / cw;
    const int extra = axis == 0 ? 2 : 1;  // warps besides the consumers: producer (+ preparer)
    ColPlan cp;
    if (h->pipe_chunk > 0) {  // chunk length chosen by the caller (tuning)
      if (!plan_col(n, false, cp, std::min(h->pipe_chunk, n))) continue;
    } else if (cw == 32) {
      // a field that stays in L2 makes the sweep latency-bound: there the shortest chunk, 16
      // then 24 positions, whose CTA fits (more consumer warps per SM; measured: 250^3 x 1
      // z-sweep 0.036 against 0.050 ms); in the HBM-bound regime chunks of 32 (at 256^3 x 4
      // chunks of 16 took the x-sweep from 0.139 to 0.211 ms)
      const bool l2_resident = (double)h->nel * (double)esz <= 96.0e6;
      bool shortc = false;
      for (int target : {16, 24}) {
        const int T = (n + target - 1) / target;
        if (!l2_resident || h16 || T < 2 || (T + extra) * 32 > pipe_max_threads_f32(target))
          continue;
        cp.T = T;
        cp.m = target;
        cp.maxm = target;
        shortc = true;
        break;
      }
      if (!shortc && !plan_col(n, false, cp)) continue;
    } else {  // 16 columns: chunks of 32 or 64 (the capacities compiled for them)
      bool found = false;
      for (int target : {32, 64}) {
        const int T = std::max(1, (n + target - 1) / target);
        const int m = T == 1 ? n : target;
        const int maxm = pick_maxm(m, false);
        if (maxm != 32 && maxm != 64) continue;
        if (((T + 1) / 2 + extra) * 32 > pipe_max_threads_f32(maxm)) continue;
        cp.T = T;
        cp.m = m;
        cp.maxm = maxm;
        found = true;
        break;
      }
      if (!found) continue;
    }
    if (h16 && cp.maxm < 32) cp.maxm = 32;  // short chunks run on the guarded path
    if (h16 && cp.maxm > 64) continue;
    if (cw == 16 && cp.maxm != 32 && cp.maxm != 64) continue;
    // chunks above 64 registers spill (measured with -Xptxas -v): 16-column tiles instead
    if (cw == 32 && cp.maxm > 64 && h->pipe_chunk <= 0) continue;
    const int W = (cp.T + cpw - 1) / cpw;  // consumer warps
    if ((W + extra) * 32 > pipe_max_threads_f32(cp.maxm)) continue;
    q.T = cp.T;
    q.m = cp.m;
    q.maxm = cp.maxm;
    if (axis == 0) {
      if ((gp * (int64_t)esz) % 16 != 0 || S > cw) continue;
      q.rows_per_tile = (int)(cw / S);
      // the staged rows: gp elements each (a 16-byte multiple), at a shared-memory pitch in
      // elements that keeps every row 16-byte aligned
      const int align = (int)(16 / esz);
      int best = 1 << 30;
      for (int64_t pitch = gp; pitch <= gp + 64; pitch += align) {
        const int d = cw == 16 ? x_tile_conflicts(pitch, (int)S, q.rows_per_tile * (int)S, esz,
                                                  (int64_t)q.m * S)
                               : x_tile_conflicts(pitch, (int)S, q.rows_per_tile * (int)S, esz);
        if (d < best) {
          best = d;
          q.pitch = (int)pitch;
        }
      }
      q.stage_elems = (int64_t)q.rows_per_tile * q.pitch;
      if (ny * nz > (int64_t)0x7fffffff) return;  // the kernel tracks rows in 32 bits
      q.ntiles = (ny * nz + q.rows_per_tile - 1) / q.rows_per_tile;
    } else {
      const int64_t C = axis == 1 ? nx * S : ny * gp;
      const int nplanes = axis == 1 ? (int)nz : 1;
      // the map's stride between a line's positions must be a 16-byte multiple: y: the row
      // pitch gp; z: the plane, C = ny * gp (the inner extent C of a y map need not be)
      const int64_t lstride = axis == 1 ? gp : C;
      if ((lstride * (int64_t)esz) % 16 != 0 || C > (int64_t)0x7fffffff || nplanes > 65535)
        return;
      // boxes of at most 256 rows; a tensor copy's shared-memory destination must be
      // 128-byte aligned, so box_rows * cw * esz is rounded up to a 128-byte multiple (rows
      // past the line's end are filled with zeros on load and skipped on store)
      q.nbox = (n + 255) / 256;
      const int rgran = std::max(1, (int)(128 / ((size_t)cw * esz)));
      q.box_rows = ((n + q.nbox - 1) / q.nbox + rgran - 1) / rgran * rgran;
      if (((size_t)q.box_rows * cw * esz) % 128 != 0 || q.box_rows > 256) continue;
      q.stage_elems = (int64_t)q.nbox * q.box_rows * cw;
      q.ntiles = (int64_t)nplanes * ((C + cw - 1) / cw);
      if (q.ntiles > (int64_t)0x7fffffff) return;  // tiles are indexed in 32 bits
    }
    const size_t stage = (size_t)q.stage_elems * esz;
    const size_t tab = (size_t)pipe_tab_elems_host(n, (int)S) * csz + 16;  // + alignment
    // carry exchange [2][W*32], carry weights [T][T][S], alignment, mbarriers
    // (mbarriers: full, done, ready per stage, at most 8 stages)
    const size_t scratch = (2 * (size_t)W * 32 + (size_t)q.T * q.T * S) * csz + 16 + 3 * 8 * 8;
    for (int ns = std::max(2, std::min(h->pipe_ns, 8)); ns >= 2 && !q.stages; ns--)  // the constants always staged
      if (ns * stage + tab + scratch <= kMaxDynamicSmem) q.stages = ns;
    if (!q.stages) continue;
    q.smem = q.stages * stage + tab + scratch;
    q.W = W;
    p = q;
    break;
  }
  if (!p.stages) {
    p = PipePlan{};
    return;
  }
  if (axis != 0 && !encode_pipe_map(h, p, axis, 0, field, gp)) {
    p.use = 0;
    return;
  }
  // the attribute is per kernel, shared by every handle: always the opt-in maximum
  const cudaError_t e = h->prec == BIOFVM_BF16   ? allow_pipe_smem_bf16(p.maxm, kMaxDynamicSmem)
                        : h->prec == BIOFVM_FP16 ? allow_pipe_smem_fp16(p.maxm, kMaxDynamicSmem)
                                                 : allow_pipe_smem_f32(p.maxm, kMaxDynamicSmem);
  if (e != cudaSuccess) {
    cudaGetLastError();
    p.use = 0;
    return;
  }
  const int threads = (p.W + (axis == 0 ? 2 : 1)) * 32;
  const int regs = p.maxm + 96;
  int per_sm = (int)std::min<size_t>({kMaxDynamicSmem / p.smem, (size_t)(2048 / threads),
                                      (size_t)(65536 / (threads * regs))});
  per_sm = std::max(per_sm, 1);
  p.grid = (int)std::min<int64_t>(p.ntiles, (int64_t)h->num_sms * per_sm);
  p.use = 1;
}

// Plan the streaming sweep of an axis: a persistent grid of
// stream_ctas_per_sm 128-thread CTAs per SM.  Each warp keeps its 32 lines'
// intermediates (32 n elements; FP32: and the field values the backward pass
// re-reads) in L2 between the two passes, so the warps in flight bound the L2
// footprint (12 warps per SM at n = 400: about 93 MB on average).  FP64 always
// (the FP64 step is bound by FP64 operations); FP32 when stream32_enabled, or
// for an axis the pipelined sweep cannot take whose plain kernel would hold
// chunks of more than 64 positions in registers (or cannot hold the lines at
// all), with a field-sized scratch buffer.
void plan_stream(biofvm *h, int axis) {
  StreamPlan &p = h->sp[axis];
  p = StreamPlan{};
  if (!h->stream_enabled || h->esz == 2) return;  // 16-bit fields: the pipelined sweep only
  if (h->prec == BIOFVM_FP32) {
    const bool plain_slow = axis == 0 ? (h->xp.nosolve || h->xp.maxm > 64)
                                      : (h->cp[axis].nosolve || h->cp[axis].maxm > 64);
    if (!h->stream32_enabled && (h->pp[axis].use || !plain_slow)) return;
    if (!h->scratch.p && dev_alloc(h->scratch, h->nel * h->esz) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
  }
  const int S = h->g.n_sub;
  if (axis == 0 && S > 32) return;
  if (h->prec == BIOFVM_FP64 && allow_stream_smem_f64() != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  // FP64: a warp takes one group of 32 lines at a time.  When the groups just overflow the
  // warps of three 4-warp CTAs per SM but fit those of four, the second round would hold a
  // few groups run at a single group's latency: there the 8-position blocks at four CTAs per
  // SM take every group in one round (250^3 x 1: 1953 groups per axis, step 0.41 -> 0.30 ms).
  // Otherwise the 16-position blocks (measured 4-5% faster at 200^3 x 4 and 400^3 x 4).
  p.r8 = 0;
  if (h->prec == BIOFVM_FP64) {
    const int64_t nx = h->g.nx, ny = h->g.ny, nz = h->g.nz;
    const int64_t rpw = 32 / S;
    const int64_t C = axis == 1 ? nx * S : nx * ny * S;  // as launch_stream counts them
    const int64_t groups = axis == 0 ? (ny * nz + rpw - 1) / rpw : (C + 31) / 32 * (axis == 1 ? nz : 1);
    const int64_t warps3 = (int64_t)h->num_sms * 3 * 4, warps4 = (int64_t)h->num_sms * 4 * 4;
    p.r8 = h->stream_r8_mode >= 0 ? h->stream_r8_mode : (groups > warps3 && groups <= warps4);
  }
  p.grid = h->num_sms * (p.r8 ? 4 : std::max(1, h->stream_ctas_per_sm));
  p.use = 1;
}

// Small FP64 grids (a field of at most 32 MB whose z-planes fit in shared
// memory): biofvm_step runs all its steps in one cooperative launch.  The grid covers the z-planes and at least one CTA
// per SM, within what can be co-resident.
void plan_small(biofvm *h) {
  h->small_use = 0;
  if (!h->small_enabled || h->prec != BIOFVM_FP64 || h->forced) return;
  const int nx = h->g.nx, ny = h->g.ny, nz = h->g.nz, S = h->g.n_sub;
  if ((double)h->nel * 8.0 > 32.0e6 || !h->sp[2].use) return;
  // chunks: x-lines ny*S per plane, y-lines nx*S, z-lines in groups of 32
  const int n3[3] = {nx, ny, nz}, L3[3] = {ny * S, nx * S, 32};
  int T[3];
  for (int a = 0; a < 3; a++) {
    T[a] = small_chunks(n3[a], L3[a]);
    h->small_T[a] = T[a];
    h->small_m[a] = (n3[a] + T[a] - 1) / T[a];
  }
  const size_t smem = small_smem_bytes(nx, ny, nz, S, T);
  if (smem > 200 * 1024) return;
  int per_sm = 0;
  if (small_max_blocks(&per_sm, smem) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    return;
  }
  if (dev_alloc(h->small_bar, 16) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  h->small_smem = smem;
  // one CTA per plane (phase 1) or per group of 32 z-lines (phase 2), whichever is more: a grid
  // barrier's cost grows with its CTAs
  const int groups = (int)(((int64_t)nx * ny * S + 31) / 32);
  h->small_grid = std::max(1, std::min(h->num_sms * per_sm, std::max(nz, groups)));
  h->small_use = 1;
}

// FP32 fields whose rows are not 16-byte multiples (the TMA copies' unit): a
// row-padded working copy for biofvm_step (biofvm::pitched), when the three
// pipelined sweeps can all run on it.
void plan_pitched(biofvm *h) {
  h->pitched = 0;
  const int64_t rowlen = (int64_t)h->g.nx * h->g.n_sub;
  if (h->prec != BIOFVM_FP32 || h->forced || !h->pipe_enabled || !h->pitched_enabled ||
      h->stream32_enabled || (rowlen * (int64_t)h->esz) % 16 == 0)
    return;
  const int64_t align = 16 / (int64_t)h->esz;
  const int64_t gp = (rowlen + align - 1) / align * align;
  const size_t bytes = (size_t)h->g.ny * h->g.nz * gp * h->esz;
  if (dev_alloc(h->prow, bytes) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  h->gpitch = (int)gp;
  bool all = true;
  for (int axis = 0; axis < 3; axis++) {
    plan_pipe(h, axis, h->ppx[axis], gp, h->prow.p);
    all = all && h->ppx[axis].use;
  }
  if (!all || cudaMemsetAsync(h->prow.p, 0, bytes, h->stream) != cudaSuccess) {
    cudaGetLastError();
    h->prow.release();
    for (int axis = 0; axis < 3; axis++) h->ppx[axis] = PipePlan{};
    return;
  }
  h->pitched = 1;
}

// ---------------------------------------------------------------------------
// Upload of constants and Dirichlet data.
// ---------------------------------------------------------------------------
template <typename E>
std::vector<E> cast_vec(const std::vector<double> &v) {
  std::vector<E> out(v.size());
  for (size_t i = 0; i < v.size(); i++) out[i] = (E)v[i];
  return out;
}

biofvm_status upload_doubles(biofvm *h, DevBuf &b, const std::vector<double> &v) {
  if (dev_alloc(b, v.size() * h->csz) != cudaSuccess)
    return fail(BIOFVM_ERR_OOM, "device allocation of %zu bytes failed", v.size() * h->csz);
  if (h->prec == BIOFVM_FP64) {
    CK(cudaMemcpyAsync(b.p, v.data(), v.size() * 8, cudaMemcpyHostToDevice, h->stream));
  } else {
    auto f = cast_vec<float>(v);
    CK(cudaMemcpyAsync(b.p, f.data(), f.size() * 4, cudaMemcpyHostToDevice, h->stream));
  }
  CK(cudaStreamSynchronize(h->stream));
  return BIOFVM_OK;
}

// The chunk partition of an axis, shared by its tables and every kernel that
// solves along it: the pipelined plan's when the pipeline runs that axis.
void axis_partition(const biofvm *h, int axis, int &T, int &m) {
  if (h->pp[axis].use) {
    T = h->pp[axis].T;
    m = h->pp[axis].m;
  } else if (axis == 0) {
    T = h->xp.T;
    m = h->xp.m;
  } else {
    T = h->cp[axis].T;
    m = h->cp[axis].m;
  }
}

// Tables of the streaming sweep of one axis, position-major [3][n][S]:
// inv_i, mul_i (App. A) and q_i = inv_i / sigma, sigma being the interior limit
// of inv_i: 1/denom_inf with denom_inf = (b + sqrt(b^2 - 4 r^2)) / 2 the fixed
// point of denom = b - r^2 / denom, b = 1 + 2r + lam3 (inv_0 when n < 3).
// k0 = 1 + the last position below n-1 where some substrate's inv_i differs
// from sigma, or mul_i from r sigma, by more than 4e-16 relative; on
// [k0, n-1) the tables hold exactly inv = sigma, mul = r sigma, q = 1 (a
// rounding-level change of single terms), so the kernels use per-substrate
// constants there instead of loading them.  mulinf[S] = r sigma.
void stream_tables(const biofvm *h, int axis, std::vector<double> &tt, double *sigma,
                   double *mulinf, int &k0) {
  const int n = axis_len(h, axis), S = h->g.n_sub;
  tt.assign((size_t)3 * n * S, 0.0);
  std::vector<double> inv(n), mul(n);
  std::vector<double> rr(S);
  k0 = 0;
  for (int s = 0; s < S; s++) {
    const double r = h->D[s] * h->dt / (h->h3[axis] * h->h3[axis]);
    const double lam3 = h->lam[s] * h->dt / 3.0;
    axis_constants(n, r, lam3, inv.data(), mul.data());
    double sg = inv[0];
    if (n >= 3) {
      const double b = 1.0 + 2.0 * r + lam3;
      sg = 2.0 / (b + std::sqrt((1.0 + lam3) * (1.0 + 4.0 * r + lam3)));
    }
    sigma[s] = sg;
    mulinf[s] = r * sg;
    rr[s] = r;
    for (int i = 0; i < n; i++) {
      tt[(size_t)i * S + s] = inv[i];
      tt[((size_t)n + i) * S + s] = mul[i];
      tt[((size_t)2 * n + i) * S + s] = inv[i] / sg;
      const bool same = std::fabs(inv[i] / sg - 1.0) <= 4e-16 &&
                        (mulinf[s] == 0.0 || std::fabs(mul[i] / mulinf[s] - 1.0) <= 4e-16);
      if (!same && i < n - 1) k0 = std::max(k0, i + 1);
    }
  }
  for (int i = k0; i < n - 1; i++)
    for (int s = 0; s < S; s++) {
      tt[(size_t)i * S + s] = sigma[s];
      tt[((size_t)n + i) * S + s] = mulinf[s];
      tt[((size_t)2 * n + i) * S + s] = 1.0;
    }
}

// FP32 streaming constants of one axis from its (defect-form) tables t:
// the float-rounded interior limits inv'_inf = (-c r) sigma and mul_inf =
// r sigma into c[0][S], c[1][S], and k0 = 1 + the last position below n-1
// whose float-rounded entry differs from them (the entries from k0 to n-2
// then equal the constants bit for bit; n < 3 has no interior: k0 = n).
void stream_consts_f32(const biofvm *h, int axis, const std::vector<double> &t, double *c,
                       int &k0) {
  const int n = axis_len(h, axis), S = h->g.n_sub;
  k0 = n < 3 ? n : 0;
  for (int s = 0; s < S; s++) {
    const double r = h->D[s] * h->dt / (h->h3[axis] * h->h3[axis]);
    const double lam3 = h->lam[s] * h->dt / 3.0;
    const double b = 1.0 + 2.0 * r + lam3;
    const double den = 0.5 * (b + std::sqrt((1.0 + lam3) * (1.0 + 4.0 * r + lam3)));
    const double cc = 1.0 / (1.0 + lam3), scale = -cc * r;  // as the tables form them
    const float iv = (float)(scale * (1.0 / den)), mu = (float)(r / den);
    c[s] = iv;
    c[S + s] = mu;
    if (n < 3) continue;
    for (int i = 0; i < n - 1; i++)
      if ((float)t[(size_t)i * S + s] != iv || (float)t[((size_t)n + i) * S + s] != mu)
        k0 = std::max(k0, i + 1);
  }
}

biofvm_status upload_constants(biofvm *h) {
  std::vector<double> t;
  std::vector<double> c32((size_t)6 * h->g.n_sub);
  for (int axis = 0; axis < 3; axis++) {
    int T, m;
    axis_partition(h, axis, T, m);
    const bool f32 = h->prec != BIOFVM_FP64;  // float arithmetic: FP32 and 16-bit storage
    axis_tables(h, axis, T, m, f32, t);
    biofvm_status st = upload_doubles(h, h->tab[axis], t);
    if (st) return st;
    if (f32)
      stream_consts_f32(h, axis, t, &c32[(size_t)axis * 2 * h->g.n_sub], h->stream_k0[axis]);
    // the same inv, mul, pf, pb substrate-major [4][S][npad] for the pipelined kernel
    auto upload_T = [&](DevBuf &dst) {
      const int n = axis_len(h, axis), S = h->g.n_sub, npad = pipe_npad_host(n);
      std::vector<double> tt((size_t)4 * S * npad, 0.0);
      for (int w = 0; w < 4; w++)
        for (int i = 0; i < n; i++)
          for (int s = 0; s < S; s++)
            tt[((size_t)w * S + s) * npad + i] = t[(size_t)w * n * S + (size_t)i * S + s];
      return upload_doubles(h, dst, tt);
    };
    if ((st = upload_T(h->tabT[axis])) != BIOFVM_OK) return st;
    if (h->small_use) {  // the small step's own chunk partition
      std::vector<double> ts;
      axis_tables(h, axis, h->small_T[axis], h->small_m[axis], false, ts);
      if ((st = upload_doubles(h, h->small_tab[axis], ts)) != BIOFVM_OK) return st;
    }
    // the row-padded working copy's plans: tables of their own partition where it differs
    const PipePlan &q = h->ppx[axis];
    h->tabP_own[axis] = h->pitched && (q.T != T || q.m != m);
    if (h->tabP_own[axis]) {
      axis_tables(h, axis, q.T, q.m, f32, t);
      if ((st = upload_doubles(h, h->tabP[axis], t)) != BIOFVM_OK ||
          (st = upload_T(h->tabTP[axis])) != BIOFVM_OK)
        return st;
    }
  }
  if (h->prec != BIOFVM_FP64) {
    biofvm_status st = upload_doubles(h, h->stream_const_d, c32);
    if (st) return st;
  }
  if (h->prec == BIOFVM_FP64) {
    const int S = h->g.n_sub;
    std::vector<double> sigma((size_t)3 * S), minf((size_t)3 * S), tt;
    for (int axis = 0; axis < 3; axis++) {
      stream_tables(h, axis, tt, &sigma[(size_t)axis * S], &minf[(size_t)axis * S],
                    h->stream_k0[axis]);
      biofvm_status st = upload_doubles(h, h->tabS[axis], tt);
      if (st) return st;
    }
    {
      // per-axis constants [3][2][S]: sigma, r sigma (the interior inv and mul)
      std::vector<double> c((size_t)6 * S);
      for (int axis = 0; axis < 3; axis++)
        for (int s = 0; s < S; s++) {
          c[((size_t)axis * 2) * S + s] = sigma[(size_t)axis * S + s];
          c[((size_t)axis * 2 + 1) * S + s] = minf[(size_t)axis * S + s];
        }
      biofvm_status st = upload_doubles(h, h->stream_const_d, c);
      if (st) return st;
    }
    // Per-step constants of the scaled step.  Step m of a block reads a field
    // stored as true / omega^m (omega = sigma_x sigma_y sigma_z); its rows:
    //   [0] omega^-m                  source alpha factor (and Dirichlet-node factor before x)
    //   [1] dval omega^-m             Dirichlet before the x-solve
    //   [2] dval / (omega^m sigma_x)  after x      [3] ... / (sigma_x sigma_y)  after y
    //   [4] dval / omega^(m+1)        after z, field left scaled
    //   [5] omega^(m+1)               z multiplier of the renormalising step (then dval after z)
    //   [6] [7] [8]                   rows 2, 3, 4 as factors (dval = 1): Dirichlet nodes
    // renorm_k: the longest block (<= kMaxRenorm) whose omega^k stays above 1e-150.
    std::vector<double> om(S);
    double om_min = 1.0;
    for (int s = 0; s < S; s++) {
      om[s] = sigma[s] * sigma[S + s] * sigma[2 * S + s];
      om_min = std::min(om_min, om[s]);
    }
    int K = 1;
    while (K < kMaxRenorm && std::pow(om_min, K + 1) >= 1e-150) K++;
    h->renorm_k = K;
    std::vector<double> tb((size_t)K * kRenormRows * S);
    for (int m = 0; m < K; m++)
      for (int s = 0; s < S; s++) {
        const double dv = h->dir_val[s], wm = std::pow(om[s], m);
        double *r = &tb[(size_t)m * kRenormRows * S];
        r[s] = 1.0 / wm;
        r[S + s] = dv / wm;
        r[2 * S + s] = dv / (wm * sigma[s]);
        r[3 * S + s] = dv / (wm * sigma[s] * sigma[S + s]);
        r[4 * S + s] = dv / (wm * om[s]);
        r[5 * S + s] = wm * om[s];
        r[6 * S + s] = 1.0 / (wm * sigma[s]);
        r[7 * S + s] = 1.0 / (wm * sigma[s] * sigma[S + s]);
        r[8 * S + s] = 1.0 / (wm * om[s]);
      }
    biofvm_status st = upload_doubles(h, h->renorm_d, tb);
    if (st) return st;
  }
  drop_graphs(h);
  h->generation++;
  return BIOFVM_OK;
}

// The source lists the kernels read: host-built (biofvm_set_sources) or rebuilt on the device
// (biofvm_set_sources_device; their length is only known on the device, so `has` is set and
// the kernels take the range from the row offsets).
struct SrcLists {
  const int64_t *row_off, *elem;
  const int2 *rowcol;
  const void *alpha, *scale;
  int has;
};
SrcLists src_lists(const biofvm *h) {
  SrcLists l;
  if (h->sources_device) {
    l.row_off = static_cast<const int64_t *>(h->dsrc_row_off.p);
    l.elem = static_cast<const int64_t *>(h->dsrc_elem.p);
    l.rowcol = static_cast<const int2 *>(h->dsrc_rowcol.p);
    l.alpha = h->dsrc_alpha.p;
    l.scale = h->dsrc_scale.p;
    l.has = 1;
  } else {
    l.row_off = static_cast<const int64_t *>(h->src_row_off.p);
    l.elem = static_cast<const int64_t *>(h->src_elem.p);
    l.rowcol = static_cast<const int2 *>(h->src_rowcol.p);
    l.alpha = h->src_alpha.p;
    l.scale = h->src_scale.p;
    l.has = h->n_entries > 0;
  }
  return l;
}

// The tables of an axis (layout of axis_tables, chunk partition T x m) as kernel arguments.
AxisTab axis_tab_of(const biofvm *h, int axis, const DevBuf &tab, const DevBuf &tabT, int T,
                    int m) {
  const int n = axis_len(h, axis), S = h->g.n_sub;
  const char *base = static_cast<const char *>(tab.p);
  const size_t blk = (size_t)n * S * h->csz;
  AxisTab t;
  t.inv = base;
  t.mul = base + blk;
  t.pf = base + 2 * blk;
  t.pb = base + 3 * blk;
  t.pc = base + 4 * blk;
  t.cfix = base + 4 * blk + (size_t)T * S * h->csz;
  t.cw = base + 4 * blk + ((size_t)T * S + 2 * (size_t)S) * h->csz;
  t.tabT = tabT.p;
  t.n = n;
  t.T = T;
  t.m = m;
  return t;
}

AxisTab axis_tab(const biofvm *h, int axis) {
  int T, m;
  axis_partition(h, axis, T, m);
  return axis_tab_of(h, axis, h->tab[axis], h->tabT[axis], T, m);
}

// ---------------------------------------------------------------------------
// Kernel launches.
// ---------------------------------------------------------------------------
// Launch the pipelined sweep of `axis` on `field` (buf selects the y/z tensor map).  The
// row-padded working copy (`pitched`): the plans ppx over it, rows gpitch elements apart.
cudaError_t launch_pipe(const biofvm *h, int axis, int flags, cudaStream_t st, void *field,
                        int buf, bool pitched = false) {
  const PipePlan &p = pitched ? h->ppx[axis] : h->pp[axis];
  const int gp = pitched ? h->gpitch : h->g.nx * h->g.n_sub;
  PipeArgs b{};
  b.mode = axis;
  b.n = axis_len(h, axis);
  b.S = h->g.n_sub;
  b.nx = h->g.nx;
  b.ny = h->g.ny;
  b.nz = h->g.nz;
  b.ntiles = p.ntiles;
  b.C = axis == 1 ? (int64_t)h->g.nx * h->g.n_sub : (int64_t)h->g.ny * gp;
  b.cw = p.cw;
  b.tiles_per_plane = (int)((b.C + p.cw - 1) / p.cw);
  b.nplanes = axis == 1 ? h->g.nz : 1;
  b.box_rows = p.box_rows;
  b.nbox = p.nbox;
  b.rows_per_tile = p.rows_per_tile;
  b.rowlen = h->g.nx * h->g.n_sub;
  b.pitch = p.pitch;
  b.gpitch = gp;
  b.nrows = (int64_t)h->g.ny * h->g.nz;
  b.field = field;
  b.stages = p.stages;
  b.stage_elems = p.stage_elems;
  b.tab = pitched && h->tabP_own[axis]
              ? axis_tab_of(h, axis, h->tabP[axis], h->tabTP[axis], p.T, p.m)
              : axis_tab(h, axis);
  b.tab.T = p.T;
  b.tab.m = p.m;
  b.flags = flags;
  if (!h->any_dir) b.flags &= ~(kDirBefore | kDirAfter);
  const SrcLists sl = src_lists(h);
  b.src_row_off = sl.row_off;
  b.src_elem = sl.elem;
  b.src_rowcol = sl.rowcol;
  b.src_alpha = sl.alpha;
  b.src_scale = sl.scale;
  b.has_src = sl.has;
  b.prep_warp = axis == 0 && (((b.flags & kSrc) && b.has_src) || (b.flags & kDirBefore)) ? 1 : 0;
  b.dir_on = static_cast<const uint8_t *>(h->dir_on_d.p);
  b.dir_val = h->dir_val_d.p;
  b.status = static_cast<int *>(h->status.p);
  const CUtensorMap &map = p.map[axis == 0 ? 0 : buf];
  if (h->prec == BIOFVM_BF16) return launch_pipe_bf16(map, b, p.maxm, p.grid, p.smem, st);
  if (h->prec == BIOFVM_FP16) return launch_pipe_fp16(map, b, p.maxm, p.grid, p.smem, st);
  return launch_pipe_f32(map, b, p.maxm, p.grid, p.smem, st);
}

bool stream_ok(const biofvm *h, int axis, int flags) {
  return h->sp[axis].use && (flags & kSolve);
}

cudaError_t launch_stream(const biofvm *h, int axis, int flags, cudaStream_t st, void *field) {
  const StreamPlan &p = h->sp[axis];
  const int64_t nx = h->g.nx, ny = h->g.ny, nz = h->g.nz, S = h->g.n_sub;
  StreamArgs a{};
  a.rho = field;
  a.n = axis_len(h, axis);
  a.S = (int)S;
  a.mode = axis;
  a.nx = (int)nx;
  a.ny = (int)ny;
  a.nz = (int)nz;
  if (axis == 0) {
    a.stride = S;
    a.rows_per_warp = (int)(32 / S);
    a.ngroups = (ny * nz + a.rows_per_warp - 1) / a.rows_per_warp;
  } else {
    const int64_t C = axis == 1 ? nx * S : nx * ny * S;
    a.stride = C;
    a.ngroups = (C + 31) / 32 * (axis == 1 ? nz : 1);
  }
  const bool fp64 = h->prec == BIOFVM_FP64;
  a.tab = fp64 ? h->tabS[axis].p : h->tab[axis].p;  // FP32: inv, mul lead the axis table
  a.cfix = fp64 ? nullptr : axis_tab(h, axis).cfix;
  a.scratch = h->scratch.p;
  a.ks = std::max(0, std::min(h->stream_ks, 208));  // 4 warps x ks x 256 B <= 208 KB
  a.r8 = fp64 && p.r8 ? 1 : 0;
  // (8-position blocks: XS 1 and 2 only; slabs of at most 48 positions keep four CTAs per SM)
  a.xt = (fp64 && axis == 0 && (S == 1 || S == 2 || (S == 4 && !a.r8)) && S <= h->stream_xt)
             ? (int)S : 0;
  if (a.r8) a.ks = std::min(a.ks, 48);
  if (a.xt) a.ks = std::max(0, std::min(h->stream_ks_xt, a.r8 ? 32 : 192));  // + 4 transpose buffers
  a.flags = flags;
  if (!h->any_dir) a.flags &= ~(kDirBefore | kDirAfter);
  const bool scaled = fp64 && (flags & kScaled);
  a.out = !scaled ? 0 : (axis == 2 && !(flags & kKeepScale)) ? 2 : 1;
  a.k0 = h->stream_k0[axis];
  a.interior = static_cast<const char *>(h->stream_const_d.p) + (size_t)axis * 2 * S * h->csz;
  const SrcLists sl = src_lists(h);
  a.src_row_off = sl.row_off;
  a.src_elem = sl.elem;
  a.src_alpha = sl.alpha;
  a.src_scale = sl.scale;
  a.has_src = sl.has;
  a.dir_on = static_cast<const uint8_t *>(h->dir_on_d.p);
  a.dir_val = a.dir_val_in = h->dir_val_d.p;
  if (scaled) {  // the step's row of the renormalisation table (upload_constants)
    const int m = (flags >> 8) & 0xff;
    const char *row = static_cast<const char *>(h->renorm_d.p) + (size_t)m * kRenormRows * S * h->csz;
    auto at = [&](int k) { return static_cast<const void *>(row + (size_t)k * S * h->csz); };
    if (axis == 0) {
      a.src_fac = m > 0 ? at(0) : nullptr;
      a.dir_val_in = at(1);
      a.dir_val = at(2);
    } else if (axis == 1) {
      a.dir_val = at(3);
    } else if (flags & kKeepScale) {
      a.dir_val = at(4);
    } else {
      a.omega = at(5);  // renormalising: omega^(m+1), the true field, dval itself
    }
  }
  const int grid = (int)std::min<int64_t>(p.grid, (a.ngroups + 3) / 4);
  return fp64 ? launch_stream_f64(a, grid, st) : launch_stream_f32(a, grid, st);
}

bool pipe_ok(const biofvm *h, int axis, int flags, int buf) {
  const PipePlan &p = h->pp[axis];
  return p.use && (flags & kSolve) && (axis == 0 || p.have_map[buf]);
}

cudaError_t launch_x(const biofvm *h, int flags, cudaStream_t st, void *field = nullptr) {
  if (stream_ok(h, 0, flags)) return launch_stream(h, 0, flags, st, field ? field : h->rho.p);
  if (pipe_ok(h, 0, flags, 0)) return launch_pipe(h, 0, flags, st, field ? field : h->rho.p, 0);
  if ((flags & kSolve) && h->xp.nosolve) return cudaErrorInvalidConfiguration;
  XLaunch a{};
  a.rho = field ? field : h->rho.p;
  a.nx = h->g.nx;
  a.ny = h->g.ny;
  a.nz = h->g.nz;
  a.S = h->g.n_sub;
  a.tab = axis_tab(h, 0);
  a.rows_per_cta = h->xp.rows_per_cta;
  a.rows_per_warp = h->xp.rows_per_warp;
  a.warps = h->xp.warps;
  a.maxm = h->xp.maxm;
  a.use_bulk = h->xp.use_bulk;
  a.smem_bytes = h->xp.smem;
  a.flags = flags;
  if (!h->any_dir) a.flags &= ~(kDirBefore | kDirAfter);
  const SrcLists sl = src_lists(h);
  a.has_src = sl.has;
  a.src_row_off = sl.row_off;
  a.src_elem = sl.elem;
  a.src_alpha = sl.alpha;
  a.src_scale = sl.scale;
  a.dir_on = static_cast<const uint8_t *>(h->dir_on_d.p);
  a.dir_val = h->dir_val_d.p;
  a.status = static_cast<int *>(h->status.p);
  return h->prec == BIOFVM_FP64 ? launch_x_f64(a, st) : launch_x_f32(a, st);
}

cudaError_t launch_col(const biofvm *h, int axis, int flags, cudaStream_t st, int buf = 0) {
  ColLaunch a{};
  a.rho = buf ? h->adj.p : h->rho.p;
  const int64_t nx = h->g.nx, ny = h->g.ny, nz = h->g.nz, S = h->g.n_sub;
  if (axis == 1) {
    a.C = nx * S;
    a.plane_stride = nx * ny * S;
    a.nplanes = (int)nz;
    a.n = (int)ny;
    a.mode = 1;
  } else {
    a.C = nx * ny * S;
    a.plane_stride = 0;
    a.nplanes = 1;
    a.n = (int)nz;
    a.mode = 2;
  }
  a.S = (int)S;
  a.nx = (int)nx;
  a.ny = (int)ny;
  a.nz = (int)nz;
  a.tab = axis_tab(h, axis);
  a.maxm = h->cp[axis].maxm;
  a.flags = flags;
  if (!h->any_dir) a.flags &= ~kDirAfter;
  a.dir_on = static_cast<const uint8_t *>(h->dir_on_d.p);
  a.dir_val = h->dir_val_d.p;
  if (stream_ok(h, axis, flags)) return launch_stream(h, axis, flags, st, a.rho);
  if (pipe_ok(h, axis, flags, buf)) return launch_pipe(h, axis, flags, st, a.rho, buf);
  if (h->cp[axis].nosolve) return cudaErrorInvalidConfiguration;
  return h->prec == BIOFVM_FP64 ? launch_col_f64(a, st) : launch_col_f32(a, st);
}

// Scaled intermediates (FP64, stream.cuh) only when all three sweeps of a step stream.
int step_scaled(const biofvm *h) {
  return (h->prec == BIOFVM_FP64 && h->sp[0].use && h->sp[1].use && h->sp[2].use) ? kScaled : 0;
}

// The Dirichlet nodes of one application on `field` (the handle's field when
// NULL): their values times row `row` of step m of the renormalisation table
// (row < 0: the values themselves), or zeros (the adjoint's mask).
cudaError_t launch_nodes(const biofvm *h, cudaStream_t st, int m, int row, bool zero = false,
                         void *field = nullptr) {
  if (h->n_dnode <= 0) return cudaSuccess;
  NodeLaunch a{};
  a.rho = field ? field : h->rho.p;
  a.elem = static_cast<const int64_t *>(h->dn_elem.p);
  a.val = h->dn_val.p;
  a.scale = row < 0 ? nullptr
                    : static_cast<const char *>(h->renorm_d.p) +
                          ((size_t)m * kRenormRows + row) * h->g.n_sub * h->csz;
  a.n = h->n_dnode;
  a.S = h->g.n_sub;
  a.zero = zero ? 1 : 0;
  a.grid = (int)std::max<int64_t>(1, std::min<int64_t>((a.n + 255) / 256, 4 * (int64_t)h->num_sms));
  return h->prec == BIOFVM_FP64 ? launch_nodes_f64(a, st) : launch_nodes_f32(a, st);
}

// One step.  Scaled (FP64 streaming): step m of a renormalisation block reads a
// field stored as true / omega^m and, unless `renorm`, leaves it as
// true / omega^(m+1); a renormalising step stores the true field.  Dirichlet
// nodes, when set, take one launch around each sweep: the one before the
// x-sweep stands for the node part of the application between Src and X^-1
// (the source list holds no node element, and the fused face application
// skips every substrate with a node on its faces, so the order holds).
// The field into its row-padded working copy (in) or back (out).
cudaError_t pitch_copy(const biofvm *h, bool in, cudaStream_t st) {
  const int64_t rows = (int64_t)h->g.ny * h->g.nz;
  const int rowlen = h->g.nx * h->g.n_sub;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((rows + 7) / 8, 8 * h->num_sms));
  return in ? launch_pitch_rows(h->rho.p, h->prow.p, rows, rowlen, rowlen, h->gpitch, h->esz,
                                grid, st)
            : launch_pitch_rows(h->prow.p, h->rho.p, rows, rowlen, h->gpitch, rowlen, h->esz,
                                grid, st);
}

// `pitched`: the three pipelined sweeps on the row-padded working copy (no
// Dirichlet nodes then).
biofvm_status launch_step(const biofvm *h, cudaStream_t st, int m = 0, bool renorm = true,
                          bool pitched = false) {
  if (pitched) {
    CK(launch_pipe(h, 0, kSrc | kDirBefore | kSolve | kDirAfter, st, h->prow.p, 0, true));
    CK(launch_pipe(h, 1, kSolve | kDirAfter, st, h->prow.p, 0, true));
    CK(launch_pipe(h, 2, kSolve | kDirAfter, st, h->prow.p, 0, true));
    return BIOFVM_OK;
  }
  const int sc = step_scaled(h);
  const int mf = sc ? (m << 8) : 0;
  CK(launch_nodes(h, st, m, sc ? 0 : -1));
  CK(launch_x(h, kSrc | kDirBefore | kSolve | kDirAfter | sc | mf, st));
  CK(launch_nodes(h, st, m, sc ? 6 : -1));
  CK(launch_col(h, 1, kSolve | kDirAfter | sc | mf, st));
  CK(launch_nodes(h, st, m, sc ? 7 : -1));
  CK(launch_col(h, 2, kSolve | kDirAfter | sc | mf | (sc && !renorm ? kKeepScale : 0), st));
  CK(launch_nodes(h, st, m, sc && !renorm ? 8 : -1));
  return BIOFVM_OK;
}

// The device source lists from the agents as last given: (element, alpha,
// beta) per agent and substrate, sorted by element and summed, without the
// elements of Dirichlet nodes (a node's application overwrites whatever the
// source update left there, so its entry would have no effect).
biofvm_status build_sources(biofvm *h) {
  const int S = h->g.n_sub;
  const int64_t n = (int64_t)h->h_voxel.size();
  struct Ent {
    int64_t e;
    double alpha, beta;
  };
  std::vector<Ent> ent;
  ent.reserve((size_t)n * S);
  for (int64_t k = 0; k < n; k++) {
    const double w = h->h_weight.empty() ? 1.0 : h->h_weight[k];
    for (int s = 0; s < S; s++) {
      const double sv = h->h_secretion[k * S + s], uv = h->h_uptake[k * S + s];
      const double tv = h->h_target[k * S + s];
      const double alpha = h->dt * w * sv * tv, beta = h->dt * w * (sv + uv);
      const int64_t e = h->h_voxel[k] * S + s;
      if ((alpha != 0.0 || beta != 0.0) &&
          !std::binary_search(h->h_dn_kelem.begin(), h->h_dn_kelem.end(), e))
        ent.push_back({e, alpha, beta});
    }
  }
  std::stable_sort(ent.begin(), ent.end(), [](const Ent &a, const Ent &b) { return a.e < b.e; });
  size_t u = 0;
  for (size_t i = 0; i < ent.size(); i++) {
    if (u > 0 && ent[u - 1].e == ent[i].e) {
      ent[u - 1].alpha += ent[i].alpha;
      ent[u - 1].beta += ent[i].beta;
    } else {
      ent[u++] = ent[i];
    }
  }
  ent.resize(u);
  const int64_t rowlen = (int64_t)h->g.nx * S;
  const int64_t nrows = (int64_t)h->g.ny * h->g.nz;
  std::vector<int64_t> off(nrows + 1, 0), elem(u);
  std::vector<int32_t> rowcol(2 * u);  // (row, position in the row) of each entry
  std::vector<double> alpha(u), scale(u);
  for (size_t i = 0; i < u; i++) {
    off[ent[i].e / rowlen + 1]++;
    elem[i] = ent[i].e;
    rowcol[2 * i] = (int32_t)(ent[i].e / rowlen);
    rowcol[2 * i + 1] = (int32_t)(ent[i].e % rowlen);
    alpha[i] = ent[i].alpha;
    scale[i] = 1.0 / (1.0 + ent[i].beta);
  }
  for (int64_t r = 0; r < nrows; r++) off[r + 1] += off[r];
  CK(cudaStreamSynchronize(h->stream));  // the kernels may still read the old lists
  h->n_entries = 0;
  if (dev_alloc(h->src_row_off, off.size() * 8) != cudaSuccess)
    return fail(BIOFVM_ERR_OOM, "device allocation for the source offsets failed");
  CK(cudaMemcpy(h->src_row_off.p, off.data(), off.size() * 8, cudaMemcpyHostToDevice));
  if (u > 0) {
    if (dev_alloc(h->src_elem, u * 8) != cudaSuccess)
      return fail(BIOFVM_ERR_OOM, "device allocation for %zu source entries failed", u);
    CK(cudaMemcpy(h->src_elem.p, elem.data(), u * 8, cudaMemcpyHostToDevice));
    if (dev_alloc(h->src_rowcol, u * 8) != cudaSuccess)
      return fail(BIOFVM_ERR_OOM, "device allocation for %zu source entries failed", u);
    CK(cudaMemcpy(h->src_rowcol.p, rowcol.data(), u * 8, cudaMemcpyHostToDevice));
    biofvm_status st = upload_doubles(h, h->src_alpha, alpha);
    if (st) return st;
    st = upload_doubles(h, h->src_scale, scale);
    if (st) return st;
  }
  h->n_entries = (int64_t)u;
  h->h_src_elem = elem;
  h->sources_device = false;
  h->agents_on_device = false;  // the adjoint's agent-to-entry map follows the list
  h->generation++;
  drop_graphs(h);  // kernel arguments changed
  return BIOFVM_OK;
}

biofvm_status check_status(biofvm *h) {
  int st = 0;
  CK(cudaMemcpy(&st, h->status.p, sizeof(int), cudaMemcpyDeviceToHost));
  if (st != kStatusOk) {
    CK(cudaMemset(h->status.p, 0, sizeof(int)));
    if (st == kStatusBadInput)
      return fail(BIOFVM_ERR_ARG, "a device agent array held an invalid agent (voxel out of "
                                  "range, or a negative or non-finite rate or weight); it was "
                                  "left out of the source lists");
    return fail(BIOFVM_ERR_TIMEOUT, "a bounded device-side wait timed out (status %d)", st);
  }
  return BIOFVM_OK;
}

bool valid_params(int S, const double *D, const double *lam) {
  if (!D || !lam) return false;
  for (int s = 0; s < S; s++)
    if (!(D[s] >= 0.0) || !(lam[s] >= 0.0) || !std::isfinite(D[s]) || !std::isfinite(lam[s]))
      return false;
  return true;
}

void destroy_impl(biofvm *h) {
  if (!h) return;
  cudaSetDevice(h->device);
  if (h->stream || h->rho.p) cudaStreamSynchronize(h->stream);
  drop_graphs(h);
  for (DevBuf *b : {&h->rho, &h->tab[0], &h->tab[1], &h->tab[2], &h->tabT[0], &h->tabT[1],
                    &h->tabT[2], &h->tabS[0], &h->tabS[1], &h->tabS[2], &h->renorm_d,
                    &h->stream_const_d, &h->scratch, &h->dir_on_d, &h->dir_val_d,
                    &h->status, &h->src_row_off, &h->src_elem, &h->src_rowcol, &h->src_alpha, &h->src_scale,
                    &h->adj, &h->partial, &h->ag_elem, &h->ag_entry, &h->ag_weight,
                    &h->ag_target, &h->dn_elem, &h->dn_val, &h->dsrc_row_off, &h->dsrc_elem,
                    &h->dsrc_rowcol, &h->dsrc_alpha, &h->dsrc_scale, &h->dsrc_count,
                    &h->ag_key[0], &h->ag_key[1], &h->ag_idx[0], &h->ag_idx[1], &h->ag_ea,
                    &h->ag_eb, &h->ag_head, &h->ag_pos, &h->ag_hist, &h->ag_part,
                    &h->ag_count32, &h->small_bar, &h->small_tab[0], &h->small_tab[1],
                    &h->small_tab[2], &h->prow, &h->tabP[0], &h->tabP[1],
                    &h->tabP[2], &h->tabTP[0], &h->tabTP[1], &h->tabTP[2]})
    b->release();
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  delete h;
}

biofvm_status create_impl(const biofvm_grid *grid, double dx, double dt, const double *D,
                          const double *lambda, const biofvm_boundary *bc, biofvm_precision prec,
                          uintptr_t cuda_stream, const int *force_m, biofvm_t **out);
}  // namespace

namespace bfv {
void set_error_message(const char *msg) { g_last_error = msg ? msg : ""; }
}  // namespace bfv

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char *biofvm_last_error(void) { return g_last_error.c_str(); }

biofvm_status biofvm_create(const biofvm_grid *grid, double dx, double dt, const double *D,
                            const double *lambda, const biofvm_boundary *bc,
                            biofvm_precision prec, uintptr_t cuda_stream, biofvm_t **out) {
  return create_impl(grid, dx, dt, D, lambda, bc, prec, cuda_stream, nullptr, out);
}

}  // extern "C"

namespace {
// biofvm_create with optional chunk lengths force_m[3] (x, y, z): the batched
// kernel needs every environment's partition to fit its CTA; no pipelines then.
biofvm_status create_impl(const biofvm_grid *grid, double dx, double dt, const double *D,
                          const double *lambda, const biofvm_boundary *bc, biofvm_precision prec,
                          uintptr_t cuda_stream, const int *force_m, biofvm_t **out) {
  g_last_error.clear();
  if (!out) return fail(BIOFVM_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!grid) return fail(BIOFVM_ERR_ARG, "grid is NULL");
  const biofvm_grid g = *grid;
  if (g.nx < 1 || g.ny < 1 || g.nz < 1)
    return fail(BIOFVM_ERR_ARG, "grid sizes must be >= 1 (got %d x %d x %d)", g.nx, g.ny, g.nz);
  if (g.n_sub < 1 || g.n_sub > 32)
    return fail(BIOFVM_ERR_ARG, "n_sub must be in [1, 32] (got %d)", g.n_sub);
  if (!(dx > 0.0) || !std::isfinite(dx)) return fail(BIOFVM_ERR_ARG, "dx must be > 0");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(BIOFVM_ERR_ARG, "dt must be > 0");
  if (!valid_params(g.n_sub, D, lambda))
    return fail(BIOFVM_ERR_ARG, "D and lambda must be finite, >= 0 and non-NULL");
  if (prec != BIOFVM_FP64 && prec != BIOFVM_FP32 && prec != BIOFVM_BF16 && prec != BIOFVM_FP16)
    return fail(BIOFVM_ERR_ARG, "unknown precision %d", (int)prec);
  if (force_m && (prec == BIOFVM_BF16 || prec == BIOFVM_FP16))
    return fail(BIOFVM_ERR_ARG, "batched environments are FP64 or FP32");
  const bool fp64 = prec == BIOFVM_FP64;
  const double nel_d = (double)g.nx * g.ny * g.nz * g.n_sub;
  if (nel_d > 9.0e18 / 8) return fail(BIOFVM_ERR_ARG, "grid too large");
  if ((double)g.nx * g.n_sub * (fp64 ? 8 : 4) >= 4.0e9 || (double)g.ny * g.nz >= 4.0e9)
    return fail(BIOFVM_ERR_ARG, "grid too large for 32-bit row offsets");

  biofvm *h = new (std::nothrow) biofvm();
  if (!h) return fail(BIOFVM_ERR_OOM, "host allocation failed");
  h->g = g;
  h->dx = dx;
  h->h3[0] = h->h3[1] = h->h3[2] = dx;
  h->dt = dt;
  h->D.assign(D, D + g.n_sub);
  h->lam.assign(lambda, lambda + g.n_sub);
  h->dir_on.assign(g.n_sub, 0);
  h->dir_val.assign(g.n_sub, 0.0);
  if (bc && bc->dirichlet_on) {
    if (!bc->dirichlet_value) {
      delete h;
      return fail(BIOFVM_ERR_ARG, "dirichlet_value is NULL while dirichlet_on is set");
    }
    for (int s = 0; s < g.n_sub; s++) {
      h->dir_on[s] = bc->dirichlet_on[s] ? 1 : 0;
      h->dir_val[s] = bc->dirichlet_value[s];
      if (h->dir_on[s]) {
        if (!std::isfinite(h->dir_val[s])) {
          delete h;
          return fail(BIOFVM_ERR_ARG, "Dirichlet value of substrate %d is not finite", s);
        }
        h->any_dir = true;
      }
    }
  }
  h->dir_on_k = h->dir_on;
  h->prec = prec;
  h->esz = fp64 ? 8 : (prec == BIOFVM_FP32 ? 4 : 2);
  h->csz = fp64 ? 8 : 4;
  h->nel = (size_t)g.nx * g.ny * g.nz * g.n_sub;
  h->forced = force_m != nullptr;
  if (!plan_x(g.nx, g.n_sub, fp64, h->xp, force_m ? force_m[0] : 0, !force_m)) {
    delete h;
    return fail(BIOFVM_ERR_ARG, "x lines too long for the x-sweep tile (nx*n_sub = %d)",
                g.nx * g.n_sub);
  }
  for (int axis = 1; axis <= 2; axis++) {
    const int n = axis == 1 ? g.ny : g.nz;
    if (plan_col(n, fp64, h->cp[axis], force_m ? force_m[axis] : 0)) continue;
    if (force_m) {
      delete h;
      return fail(BIOFVM_ERR_ARG, "y or z lines too long for the column sweep (ny=%d nz=%d)",
                  g.ny, g.nz);
    }
    // the plain column kernel cannot hold these lines; the streaming or pipelined sweep must
    // (checked once they are planned)
    h->cp[axis] = ColPlan{};
    h->cp[axis].T = 1;
    h->cp[axis].m = n;
    h->cp[axis].nosolve = 1;
  }
  h->stream = reinterpret_cast<cudaStream_t>(cuda_stream);

  // --- device work starts here ---
  biofvm_status st = BIOFVM_OK;
  cudaError_t e = cudaGetDevice(&h->device);
  cudaDeviceProp prop{};
  if (e == cudaSuccess) e = cudaGetDeviceProperties(&prop, h->device);
  if (e != cudaSuccess) {
    destroy_impl(h);
    return fail(BIOFVM_ERR_CUDA, "no usable CUDA device: %s", cudaGetErrorString(e));
  }
  if (!(prop.major == 10 && prop.minor == 3)) {
    destroy_impl(h);
    return fail(BIOFVM_ERR_CUDA, "device %d is sm_%d%d; this library is built for sm_103a",
                h->device, prop.major, prop.minor);
  }
  if ((e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking)) != cudaSuccess) {
    destroy_impl(h);
    return fail(BIOFVM_ERR_CUDA, "cudaStreamCreate failed: %s", cudaGetErrorString(e));
  }
  if (dev_alloc(h->rho, h->nel * h->esz) != cudaSuccess ||
      dev_alloc(h->status, sizeof(int)) != cudaSuccess ||
      dev_alloc(h->dir_on_d, (size_t)g.n_sub) != cudaSuccess) {
    destroy_impl(h);
    return fail(BIOFVM_ERR_OOM, "device allocation of the field (%zu bytes) failed",
                h->nel * h->esz);
  }
  if ((e = cudaMemsetAsync(h->rho.p, 0, h->nel * h->esz, h->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(h->status.p, 0, sizeof(int), h->stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(h->dir_on_d.p, h->dir_on_k.data(), g.n_sub, cudaMemcpyHostToDevice,
                           h->stream)) != cudaSuccess) {
    destroy_impl(h);
    return fail(BIOFVM_ERR_CUDA, "initialising device memory failed: %s", cudaGetErrorString(e));
  }
  // the attribute is per kernel, shared by every handle: always the opt-in maximum
  e = fp64 ? allow_x_smem_f64(h->xp.maxm, kMaxDynamicSmem)
           : allow_x_smem_f32(h->xp.maxm, kMaxDynamicSmem);
  if (e != cudaSuccess) {
    destroy_impl(h);
    return fail(BIOFVM_ERR_CUDA, "x-sweep shared memory of %zu bytes refused: %s", h->xp.smem,
                cudaGetErrorString(e));
  }
  h->num_sms = prop.multiProcessorCount;
  // sweep selection and tuning knobs (environment, read once per handle)
  if (const char *env = getenv("BIOFVM_PIPELINE")) h->pipe_enabled = atoi(env) != 0;
  if (const char *env = getenv("BIOFVM_PIPE_CHUNK")) h->pipe_chunk = atoi(env);
  if (const char *env = getenv("BIOFVM_PIPE_CW")) h->pipe_cw = atoi(env);
  if (const char *env = getenv("BIOFVM_PIPE_NS")) h->pipe_ns = atoi(env);
  if (const char *env = getenv("BIOFVM_STREAM")) h->stream_enabled = atoi(env) != 0;
  if (const char *env = getenv("BIOFVM_STREAM_CTAS")) h->stream_ctas_per_sm = atoi(env);
  if (const char *env = getenv("BIOFVM_STREAM32")) h->stream32_enabled = atoi(env) != 0;
  if (const char *env = getenv("BIOFVM_STREAM_KS")) h->stream_ks = atoi(env) / 16 * 16;
  if (const char *env = getenv("BIOFVM_STREAM_XT")) h->stream_xt = atoi(env);
  if (const char *env = getenv("BIOFVM_STREAM_KS_XT")) h->stream_ks_xt = atoi(env) / 16 * 16;
  if (const char *env = getenv("BIOFVM_STREAM_R")) h->stream_r8_mode = atoi(env) == 8 ? 1 : 0;
  if (h->pipe_enabled && !h->forced)
    for (int axis = 0; axis < 3; axis++)
      plan_pipe(h, axis, h->pp[axis], (int64_t)g.nx * g.n_sub, h->rho.p);
  if (!h->forced)
    for (int axis = 0; axis < 3; axis++) plan_stream(h, axis);
  if (h->xp.nosolve && !h->sp[0].use && !h->pp[0].use) {
    destroy_impl(h);
    return fail(BIOFVM_ERR_ARG, "x lines too long for the x-sweep tile (nx*n_sub = %d)",
                g.nx * g.n_sub);
  }
  for (int axis = 1; axis <= 2; axis++)
    if (h->cp[axis].nosolve && !h->sp[axis].use && !h->pp[axis].use) {
      destroy_impl(h);
      return fail(BIOFVM_ERR_ARG, "y or z lines too long for the column sweep (ny=%d nz=%d)",
                  g.ny, g.nz);
    }
  if (h->esz == 2 && !(h->pp[0].use && h->pp[1].use && h->pp[2].use)) {
    destroy_impl(h);
    return fail(BIOFVM_ERR_ARG,
                "16-bit storage runs on the pipelined sweep only: nx*n_sub and nx*n_sub*ny "
                "must be multiples of 8 elements and the lines short enough for its tiles");
  }
  if (const char *env = getenv("BIOFVM_SMALL")) h->small_enabled = atoi(env) != 0;
  plan_small(h);
  if (const char *env = getenv("BIOFVM_PITCHED")) h->pitched_enabled = atoi(env) != 0;
  plan_pitched(h);
  if ((st = upload_doubles(h, h->dir_val_d, h->dir_val)) != BIOFVM_OK ||
      (st = upload_constants(h)) != BIOFVM_OK) {
    std::string msg = g_last_error;
    destroy_impl(h);
    g_last_error = msg;
    return st;
  }
  *out = h;
  return BIOFVM_OK;
}
}  // namespace

extern "C" {

biofvm_status biofvm_set_density(biofvm_t *h, const void *src, int src_on_device) {
  if (!h || !src) return fail(BIOFVM_ERR_ARG, "NULL handle or source");
  CK(cudaSetDevice(h->device));
  CK(cudaMemcpyAsync(h->rho.p, src, h->nel * h->esz,
                     src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                     h->stream));
  if (!src_on_device) CK(cudaStreamSynchronize(h->stream));
  return BIOFVM_OK;
}

biofvm_status biofvm_density(biofvm_t *h, void *dst, int dst_on_device) {
  if (!h || !dst) return fail(BIOFVM_ERR_ARG, "NULL handle or destination");
  CK(cudaSetDevice(h->device));
  CK(cudaMemcpyAsync(dst, h->rho.p, h->nel * h->esz,
                     dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return check_status(h);
}

biofvm_status biofvm_sync(biofvm_t *h) {
  if (!h) return fail(BIOFVM_ERR_ARG, "NULL handle");
  CK(cudaSetDevice(h->device));
  CK(cudaStreamSynchronize(h->stream));
  return check_status(h);
}

biofvm_status biofvm_density_ptr(biofvm_t *h, void **dev_ptr) {
  if (!h || !dev_ptr) return fail(BIOFVM_ERR_ARG, "NULL handle or output");
  *dev_ptr = h->rho.p;
  return BIOFVM_OK;
}

int biofvm_launches_per_step(const biofvm_t *h) {
  if (!h) return 0;
  if (h->small_use && h->n_dnode == 0) return 1;  // one launch runs every step of a call
  return 3 + (h->n_dnode > 0 ? 4 : 0);             // the sweeps (+ the Dirichlet nodes)
}

biofvm_status biofvm_describe(const biofvm_t *h, char *out, size_t len) {
  if (!h || !out) return fail(BIOFVM_ERR_ARG, "NULL handle or buffer");
  std::string d;
  if (h->small_use && h->n_dnode == 0) {
    d = "cooperative";
  } else {
    const bool pitched = h->pitched && h->n_dnode == 0;
    const char *names[3] = {"x=", " y=", " z="};
    for (int axis = 0; axis < 3; axis++) {
      d += names[axis];
      const bool stream = !pitched && h->sp[axis].use;
      const PipePlan &p = pitched ? h->ppx[axis] : h->pp[axis];
      if (stream) {
        d += "stream";
      } else if (p.use) {
        char b[48];
        snprintf(b, sizeof b, "pipe/cw%d/m%d", p.cw, p.m);
        d += b;
      } else {
        d += "plain";
      }
    }
    if (step_scaled(h)) d += " scaled";
    if (pitched) d += " pitched";
    if (h->n_dnode > 0) d += " nodes";
  }
  if (len > 0) snprintf(out, len, "%s", d.c_str());
  if (d.size() + 1 > len) return fail(BIOFVM_ERR_ARG, "buffer of %zu bytes too small", len);
  return BIOFVM_OK;
}

biofvm_status biofvm_set_params(biofvm_t *h, const double *D, const double *lambda) {
  if (!h) return fail(BIOFVM_ERR_ARG, "NULL handle");
  if (!valid_params(h->g.n_sub, D, lambda))
    return fail(BIOFVM_ERR_ARG, "D and lambda must be finite, >= 0 and non-NULL");
  CK(cudaSetDevice(h->device));
  h->D.assign(D, D + h->g.n_sub);
  h->lam.assign(lambda, lambda + h->g.n_sub);
  return upload_constants(h);
}

biofvm_status biofvm_set_spacing(biofvm_t *h, double dx, double dy, double dz) {
  if (!h) return fail(BIOFVM_ERR_ARG, "NULL handle");
  if (!(dx > 0 && dy > 0 && dz > 0 && std::isfinite(dx) && std::isfinite(dy) && std::isfinite(dz)))
    return fail(BIOFVM_ERR_ARG, "spacings must be finite and > 0");
  CK(cudaSetDevice(h->device));
  h->h3[0] = dx;
  h->h3[1] = dy;
  h->h3[2] = dz;
  return upload_constants(h);
}

biofvm_status biofvm_set_dirichlet_nodes(biofvm_t *h, int64_t n, const int64_t *voxel,
                                         const int32_t *substrate, const double *value) {
  if (!h) return fail(BIOFVM_ERR_ARG, "NULL handle");
  if (h->esz == 2) return fail(BIOFVM_ERR_STATE, "16-bit fields take no Dirichlet nodes");
  if (n < 0) return fail(BIOFVM_ERR_ARG, "negative node count");
  if (n > 0 && (!voxel || !substrate || !value))
    return fail(BIOFVM_ERR_ARG, "voxel, substrate or value is NULL");
  const int S = h->g.n_sub, nx = h->g.nx, ny = h->g.ny, nz = h->g.nz;
  const int64_t nvox = (int64_t)nx * ny * nz;
  for (int64_t k = 0; k < n; k++) {
    if (voxel[k] < 0 || voxel[k] >= nvox)
      return fail(BIOFVM_ERR_ARG, "node %lld: voxel %lld out of range [0, %lld)", (long long)k,
                  (long long)voxel[k], (long long)nvox);
    if (substrate[k] < 0 || substrate[k] >= S)
      return fail(BIOFVM_ERR_ARG, "node %lld: substrate %d out of range [0, %d)", (long long)k,
                  (int)substrate[k], S);
    if (!std::isfinite(value[k]))
      return fail(BIOFVM_ERR_ARG, "node %lld: value is not finite", (long long)k);
  }
  CK(cudaSetDevice(h->device));
  // the caller's list: sorted by element, a repeated element keeps its last value
  std::vector<std::pair<int64_t, double>> user((size_t)n);
  for (int64_t k = 0; k < n; k++) user[k] = {voxel[k] * S + substrate[k], value[k]};
  std::stable_sort(user.begin(), user.end(),
                   [](const std::pair<int64_t, double> &a, const std::pair<int64_t, double> &b) {
                     return a.first < b.first;
                   });
  size_t u = 0;
  for (size_t i = 0; i < user.size(); i++) {
    if (u > 0 && user[u - 1].first == user[i].first) user[u - 1] = user[i];
    else user[u++] = user[i];
  }
  user.resize(u);
  auto on_face = [&](int64_t v) {
    const int x = (int)(v % nx), y = (int)((v / nx) % ny), z = (int)(v / ((int64_t)nx * ny));
    return x == 0 || x == nx - 1 || y == 0 || y == ny - 1 || z == 0 || z == nz - 1;
  };
  // a substrate whose flagged faces hold a node has its faces applied as nodes
  // too (the node values win there), the fused face application skipping it
  std::vector<uint8_t> conv(S, 0);
  for (const auto &p : user) {
    const int s = (int)(p.first % S);
    if (h->dir_on[s] && on_face(p.first / S)) conv[s] = 1;
  }
  std::vector<std::pair<int64_t, double>> kern = user;
  for (int s = 0; s < S; s++) {
    if (!conv[s]) continue;
    auto add = [&](int64_t v) {  // a face voxel, unless the caller listed it
      const int64_t e = v * S + s;
      auto it = std::lower_bound(
          user.begin(), user.end(), e,
          [](const std::pair<int64_t, double> &a, int64_t key) { return a.first < key; });
      if (it == user.end() || it->first != e) kern.push_back({e, h->dir_val[s]});
    };
    // the face voxels only (each once): whole z = 0 and z = nz-1 planes, then
    // the y = 0 and y = ny-1 rows of the planes between, then their x ends
    for (int z = 0; z < nz; z++) {
      const bool zf = z == 0 || z == nz - 1;
      for (int y = 0; y < ny; y++) {
        const int64_t row = ((int64_t)z * ny + y) * nx;
        if (zf || y == 0 || y == ny - 1) {
          for (int x = 0; x < nx; x++) add(row + x);
        } else {
          add(row);
          if (nx > 1) add(row + nx - 1);
        }
      }
    }
  }
  std::sort(kern.begin(), kern.end(),
            [](const std::pair<int64_t, double> &a, const std::pair<int64_t, double> &b) {
              return a.first < b.first;
            });
  std::vector<int64_t> kel(kern.size());
  std::vector<double> kval(kern.size());
  for (size_t i = 0; i < kern.size(); i++) {
    kel[i] = kern[i].first;
    kval[i] = kern[i].second;
  }
  CK(cudaStreamSynchronize(h->stream));  // launches in flight may read the old lists
  h->n_dnode = 0;
  if (!kel.empty()) {
    if (dev_alloc(h->dn_elem, kel.size() * 8) != cudaSuccess)
      return fail(BIOFVM_ERR_OOM, "device allocation for %zu Dirichlet nodes failed", kel.size());
    CK(cudaMemcpy(h->dn_elem.p, kel.data(), kel.size() * 8, cudaMemcpyHostToDevice));
    biofvm_status st = upload_doubles(h, h->dn_val, kval);
    if (st) return st;
  }
  h->n_dnode = (int64_t)kel.size();
  h->h_dn_elem.resize(u);
  h->h_dn_val.resize(u);
  for (size_t i = 0; i < u; i++) {
    h->h_dn_elem[i] = user[i].first;
    h->h_dn_val[i] = user[i].second;
  }
  h->h_dn_kelem = kel;
  h->any_dir = false;
  for (int s = 0; s < S; s++) {
    h->dir_on_k[s] = h->dir_on[s] && !conv[s];
    h->any_dir = h->any_dir || h->dir_on_k[s];
  }
  CK(cudaMemcpy(h->dir_on_d.p, h->dir_on_k.data(), (size_t)S, cudaMemcpyHostToDevice));
  if (h->sources_device) {  // device-built lists: the next biofvm_set_sources_device drops nodes
    h->generation++;
    drop_graphs(h);
    return BIOFVM_OK;
  }
  return build_sources(h);  // no source entry on a node element; new graphs
}

biofvm_status biofvm_set_sources(biofvm_t *h, int64_t n, const int64_t *voxel,
                                 const double *secretion, const double *target,
                                 const double *uptake, const double *weight) {
  if (!h) return fail(BIOFVM_ERR_ARG, "NULL handle");
  if (n < 0) return fail(BIOFVM_ERR_ARG, "negative agent count");
  if (n > 0 && !voxel) return fail(BIOFVM_ERR_ARG, "voxel is NULL");
  const int S = h->g.n_sub;
  const int64_t nvox = (int64_t)h->g.nx * h->g.ny * h->g.nz;
  for (int64_t k = 0; k < n; k++) {
    if (voxel[k] < 0 || voxel[k] >= nvox)
      return fail(BIOFVM_ERR_ARG, "agent %lld: voxel %lld out of range [0, %lld)", (long long)k,
                  (long long)voxel[k], (long long)nvox);
    if (weight && !(weight[k] >= 0.0 && std::isfinite(weight[k])))
      return fail(BIOFVM_ERR_ARG, "agent %lld: weight must be finite and >= 0", (long long)k);
    for (int s = 0; s < S; s++) {
      const double sv = secretion ? secretion[k * S + s] : 0.0;
      const double uv = uptake ? uptake[k * S + s] : 0.0;
      const double tv = target ? target[k * S + s] : 0.0;
      if (!(sv >= 0.0) || !(uv >= 0.0) || !std::isfinite(sv) || !std::isfinite(uv) ||
          !std::isfinite(tv))
        return fail(BIOFVM_ERR_ARG, "agent %lld: rates must be finite and >= 0", (long long)k);
    }
  }
  CK(cudaSetDevice(h->device));
  h->h_voxel.assign(voxel, voxel + n);
  h->h_weight.clear();
  if (weight) h->h_weight.assign(weight, weight + n);
  h->h_target.assign((size_t)n * S, 0.0);
  h->h_secretion.assign((size_t)n * S, 0.0);
  h->h_uptake.assign((size_t)n * S, 0.0);
  if (target) std::copy(target, target + (size_t)n * S, h->h_target.begin());
  if (secretion) std::copy(secretion, secretion + (size_t)n * S, h->h_secretion.begin());
  if (uptake) std::copy(uptake, uptake + (size_t)n * S, h->h_uptake.begin());
  return build_sources(h);
}

biofvm_status biofvm_reserve_agents(biofvm_t *h, int64_t n_max) {
  if (!h) return fail(BIOFVM_ERR_ARG, "NULL handle");
  if (h->forced) return fail(BIOFVM_ERR_STATE, "batched environments take host agent arrays");
  const int S = h->g.n_sub;
  if (n_max < 0 || n_max * (int64_t)S >= (int64_t)0xffffffffLL)
    return fail(BIOFVM_ERR_ARG, "n_max must be in [0, 2^32 / n_sub)");
  CK(cudaSetDevice(h->device));
  CK(cudaStreamSynchronize(h->stream));  // launches in flight may read the old buffers
  const int64_t N = std::max<int64_t>(1, n_max * S);
  const int64_t nrows = (int64_t)h->g.ny * h->g.nz;
  const long long nb = agent_sort_blocks(N);
  const long long parts = std::max(agent_scan_blocks(N), agent_scan_blocks(256 * nb));
  struct {
    DevBuf *b;
    size_t bytes;
  } want[] = {{&h->dsrc_row_off, (size_t)(nrows + 1) * 8}, {&h->dsrc_elem, (size_t)N * 8},
              {&h->dsrc_rowcol, (size_t)N * 8},          {&h->dsrc_alpha, (size_t)N * h->csz},
              {&h->dsrc_scale, (size_t)N * h->csz},      {&h->dsrc_count, 8},
              {&h->ag_key[0], (size_t)N * 8},            {&h->ag_key[1], (size_t)N * 8},
              {&h->ag_idx[0], (size_t)N * 4},            {&h->ag_idx[1], (size_t)N * 4},
              {&h->ag_ea, (size_t)N * 8},                {&h->ag_eb, (size_t)N * 8},
              {&h->ag_head, (size_t)N * 4},              {&h->ag_pos, (size_t)N * 4},
              {&h->ag_hist, (size_t)256 * nb * 4},       {&h->ag_part, (size_t)parts * 4},
              {&h->ag_count32, 4}};
  if (h->sources_device) {  // the kernels read the reserved lists: switch to empty host lists
    h->sources_device = false;
    h->h_voxel.clear();
    h->h_weight.clear();
    h->h_target.clear();
    h->h_secretion.clear();
    h->h_uptake.clear();
    biofvm_status st = build_sources(h);
    if (st) return st;
  }
  for (auto &w : want)
    if (dev_alloc(*w.b, w.bytes) != cudaSuccess) {
      for (auto &v : want) v.b->release();
      h->agents_max = 0;
      return fail(BIOFVM_ERR_OOM, "device allocation for %lld agents failed", (long long)n_max);
    }
  h->agents_max = n_max;
  return BIOFVM_OK;
}

biofvm_status biofvm_set_sources_device(biofvm_t *h, int64_t n, const int64_t *voxel,
                                        const double *secretion, const double *target,
                                        const double *uptake, const double *weight) {
  if (!h) return fail(BIOFVM_ERR_ARG, "NULL handle");
  if (h->forced) return fail(BIOFVM_ERR_STATE, "batched environments take host agent arrays");
  if (n < 0 || n > h->agents_max)
    return fail(BIOFVM_ERR_ARG, "n = %lld agents: reserve them first (biofvm_reserve_agents: %lld)",
                (long long)n, (long long)h->agents_max);
  if (n > 0 && !voxel) return fail(BIOFVM_ERR_ARG, "voxel is NULL");
  if (h->agents_max == 0) return fail(BIOFVM_ERR_STATE, "no agent buffers reserved");
  CK(cudaSetDevice(h->device));
  const int S = h->g.n_sub;
  AgentBuild b{};
  b.voxel = voxel;
  b.secretion = secretion;
  b.target = target;
  b.uptake = uptake;
  b.weight = weight;
  b.n_entries_max = (long long)n * S;
  b.S = S;
  b.nvox = (int64_t)h->g.nx * h->g.ny * h->g.nz;
  b.rowlen = (int64_t)h->g.nx * S;
  b.nrows = (int64_t)h->g.ny * h->g.nz;
  b.dt = h->dt;
  b.sentinel = (uint64_t)h->nel;
  b.node_elem = static_cast<const int64_t *>(h->dn_elem.p);
  b.n_nodes = h->n_dnode;
  for (int i = 0; i < 2; i++) {
    b.key[i] = static_cast<uint64_t *>(h->ag_key[i].p);
    b.idx[i] = static_cast<uint32_t *>(h->ag_idx[i].p);
  }
  b.ea = static_cast<double *>(h->ag_ea.p);
  b.eb = static_cast<double *>(h->ag_eb.p);
  b.head = static_cast<uint32_t *>(h->ag_head.p);
  b.pos = static_cast<uint32_t *>(h->ag_pos.p);
  b.hist = static_cast<uint32_t *>(h->ag_hist.p);
  b.part = static_cast<uint32_t *>(h->ag_part.p);
  b.count32 = static_cast<uint32_t *>(h->ag_count32.p);
  b.src_elem = static_cast<int64_t *>(h->dsrc_elem.p);
  b.src_alpha = h->dsrc_alpha.p;
  b.src_scale = h->dsrc_scale.p;
  b.src_rowcol = static_cast<int2 *>(h->dsrc_rowcol.p);
  b.src_row_off = static_cast<int64_t *>(h->dsrc_row_off.p);
  b.count = static_cast<int64_t *>(h->dsrc_count.p);
  b.status = static_cast<int *>(h->status.p);
  CK(build_sources_device(b, h->prec == BIOFVM_FP64, h->stream));
  if (!h->sources_device) {  // the kernels' source pointers change once: new graphs
    h->sources_device = true;
    h->n_entries = 0;
    h->agents_on_device = false;
    h->generation++;
    drop_graphs(h);
  }
  return BIOFVM_OK;
}

biofvm_status biofvm_step(biofvm_t *h, int n_steps) {
  if (!h) return fail(BIOFVM_ERR_ARG, "NULL handle");
  if (n_steps < 0) return fail(BIOFVM_ERR_ARG, "n_steps must be >= 0");
  if (n_steps == 0) return BIOFVM_OK;
  CK(cudaSetDevice(h->device));
  if (h->small_use && h->n_dnode == 0) {  // one cooperative launch for all the steps
    SmallArgs a{};
    a.rho = static_cast<double *>(h->rho.p);
    a.nx = h->g.nx;
    a.ny = h->g.ny;
    a.nz = h->g.nz;
    a.S = h->g.n_sub;
    for (int axis = 0; axis < 3; axis++) {
      a.tab[axis] = static_cast<const double *>(h->small_tab[axis].p);
      a.T[axis] = h->small_T[axis];
      a.m[axis] = h->small_m[axis];
    }
    const SrcLists sl = src_lists(h);
    a.src_row_off = sl.row_off;
    a.src_elem = sl.elem;
    a.src_alpha = static_cast<const double *>(sl.alpha);
    a.src_scale = static_cast<const double *>(sl.scale);
    a.has_src = sl.has;
    a.dir_on = static_cast<const uint8_t *>(h->dir_on_d.p);
    a.dir_val = static_cast<const double *>(h->dir_val_d.p);
    a.any_dir = h->any_dir ? 1 : 0;
    a.n_steps = n_steps;
    a.bar = static_cast<unsigned *>(h->small_bar.p);
    a.status = static_cast<int *>(h->status.p);
    CK(cudaMemsetAsync(h->small_bar.p, 0, 16, h->stream));
    CK(launch_small_f64(a, h->small_grid, h->small_smem, h->stream));
    return BIOFVM_OK;
  }
  // graphs of K steps (a renormalisation block) and of a shorter tail, each
  // ending with the true field; K = 1 unless the FP64 streaming step applies.
  // A field with unaligned rows: the steps run on the row-padded copy (the
  // graphs are dropped whenever nodes are set, so they never mix the two forms)
  const int K = step_scaled(h) ? h->renorm_k : 1;
  const bool pitched = h->pitched && h->n_dnode == 0;
  auto ensure = [&](int r) -> biofvm_status {  // graph slot 0: K steps; slot r: r < K steps
    const int slot = r == K ? 0 : r;
    if (h->gexec[slot]) return BIOFVM_OK;
    CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    biofvm_status st = BIOFVM_OK;
    for (int m = 0; m < r && st == BIOFVM_OK; m++)
      st = launch_step(h, h->cap_stream, m, m == r - 1, pitched);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->cap_stream, &graph);
    if (st != BIOFVM_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (e != cudaSuccess)
      return fail(BIOFVM_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&h->gexec[slot], graph, 0);
    if (e != cudaSuccess) {
      cudaGraphDestroy(graph);
      return fail(BIOFVM_ERR_CUDA, "cudaGraphInstantiate failed: %s", cudaGetErrorString(e));
    }
    h->graph[slot] = graph;
    return BIOFVM_OK;
  };
  const int blocks = n_steps / K, tail = n_steps % K;
  biofvm_status st;
  if (blocks > 0 && (st = ensure(K)) != BIOFVM_OK) return st;
  if (tail > 0 && (st = ensure(tail)) != BIOFVM_OK) return st;
  if (pitched) CK(pitch_copy(h, true, h->stream));
  for (int b = 0; b < blocks; b++) CK(cudaGraphLaunch(h->gexec[0], h->stream));
  if (tail > 0) CK(cudaGraphLaunch(h->gexec[tail], h->stream));
  if (pitched) CK(pitch_copy(h, false, h->stream));
  return BIOFVM_OK;
}

biofvm_status biofvm_run_stage(biofvm_t *h, int stage) {
  if (!h) return fail(BIOFVM_ERR_ARG, "NULL handle");
  CK(cudaSetDevice(h->device));
  if (stage < 0 || stage > 12) return fail(BIOFVM_ERR_ARG, "stage must be in [0, 12] (got %d)", stage);
  if (h->esz == 2 && (stage == 0 || stage == 4))
    return fail(BIOFVM_ERR_STATE, "16-bit fields run only the stages that solve");
  cudaStream_t st = h->stream;
  const int sc = step_scaled(h);
  // Dirichlet nodes: after Src (stage 0), after each solve followed by B, and
  // around the fused first kernel of a step (as launch_step does, step m = 0)
  switch (stage) {
    case 0: CK(launch_x(h, kSrc | kDirBefore, st)); CK(launch_nodes(h, st, 0, -1)); break;
    case 1: CK(launch_x(h, kSolve | kDirAfter, st)); CK(launch_nodes(h, st, 0, -1)); break;
    case 2: CK(launch_col(h, 1, kSolve | kDirAfter, st)); CK(launch_nodes(h, st, 0, -1)); break;
    case 3: CK(launch_col(h, 2, kSolve | kDirAfter, st)); CK(launch_nodes(h, st, 0, -1)); break;
    case 4: CK(launch_x(h, kSrc, st)); break;
    case 5: CK(launch_x(h, kSolve, st)); break;
    case 6: CK(launch_col(h, 1, kSolve, st)); break;
    case 7: CK(launch_col(h, 2, kSolve, st)); break;
    case 8:
      CK(launch_nodes(h, st, 0, -1));
      CK(launch_x(h, kSrc | kDirBefore | kSolve | kDirAfter, st));
      CK(launch_nodes(h, st, 0, -1));
      break;
    case 9:
      CK(launch_nodes(h, st, 0, sc ? 0 : -1));
      CK(launch_x(h, kSrc | kDirBefore | kSolve | kDirAfter | sc, st));
      CK(launch_nodes(h, st, 0, sc ? 6 : -1));
      break;
    case 10:
      CK(launch_col(h, 1, kSolve | kDirAfter | sc, st));
      CK(launch_nodes(h, st, 0, sc ? 7 : -1));
      break;
    case 11:
      CK(launch_col(h, 2, kSolve | kDirAfter | sc, st));
      CK(launch_nodes(h, st, 0, -1));
      break;
    case 12:
      CK(launch_col(h, 2, kSolve | kDirAfter | sc | (sc ? kKeepScale : 0), st));
      CK(launch_nodes(h, st, 0, sc ? 8 : -1));
      break;
  }
  return BIOFVM_OK;
}

biofvm_status biofvm_step_save(biofvm_t *h, void *saved) {
  if (!h || !saved) return fail(BIOFVM_ERR_ARG, "NULL handle or saved buffer");
  if (h->esz == 2) return fail(BIOFVM_ERR_STATE, "the adjoint takes FP64 or FP32 fields");
  CK(cudaSetDevice(h->device));
  const size_t bytes = h->nel * h->esz;
  char *sv = static_cast<char *>(saved);
  cudaStream_t st = h->stream;
  auto B = [&]() -> cudaError_t {  // faces, then nodes
    if (h->any_dir) {
      const cudaError_t e = launch_x(h, kDirAfter, st);
      if (e != cudaSuccess) return e;
    }
    return launch_nodes(h, st, 0, -1);
  };
  CK(launch_x(h, kSrc, st));
  CK(cudaMemcpyAsync(sv, h->rho.p, bytes, cudaMemcpyDeviceToDevice, st));
  CK(B());
  CK(launch_x(h, kSolve, st));
  CK(cudaMemcpyAsync(sv + bytes, h->rho.p, bytes, cudaMemcpyDeviceToDevice, st));
  CK(B());
  CK(launch_col(h, 1, kSolve, st));
  CK(cudaMemcpyAsync(sv + 2 * bytes, h->rho.p, bytes, cudaMemcpyDeviceToDevice, st));
  CK(B());
  CK(launch_col(h, 2, kSolve, st));
  CK(cudaMemcpyAsync(sv + 3 * bytes, h->rho.p, bytes, cudaMemcpyDeviceToDevice, st));
  CK(B());
  return BIOFVM_OK;
}

biofvm_status biofvm_adjoint_step(biofvm_t *h, const void *grad_out, void *grad_in, double *dD,
                                  double *dlambda, double *dsecretion, const void *saved) {
  return biofvm_adjoint_step_rates(h, grad_out, grad_in, dD, dlambda, dsecretion, nullptr, saved);
}

biofvm_status biofvm_adjoint_step_rates(biofvm_t *h, const void *grad_out, void *grad_in,
                                        double *dD, double *dlambda, double *dsecretion,
                                        double *duptake, const void *saved) {
  if (!h || !grad_out || !grad_in || !dD || !dlambda || !saved)
    return fail(BIOFVM_ERR_ARG, "NULL handle, gradient or saved-state pointer");
  if (h->esz == 2) return fail(BIOFVM_ERR_STATE, "the adjoint takes FP64 or FP32 fields");
  if (h->sources_device)
    return fail(BIOFVM_ERR_STATE, "the adjoint needs the agents given through "
                                  "biofvm_set_sources (the device-built lists have no host copy)");
  CK(cudaSetDevice(h->device));
  cudaStream_t st = h->stream;
  const size_t bytes = h->nel * h->esz;
  const int S = h->g.n_sub;
  // lazily: adjoint field (+ its tensor maps), reduction scratch, device agents
  if (!h->adj.p) {
    if (dev_alloc(h->adj, bytes) != cudaSuccess)
      return fail(BIOFVM_ERR_OOM, "device allocation of the adjoint field failed");
    for (int axis = 1; axis <= 2; axis++)
      if (h->pp[axis].use)  // x tiles need no map
        encode_pipe_map(h, h->pp[axis], axis, 1, h->adj.p, (int64_t)h->g.nx * h->g.n_sub);
  }
  if (!h->partial.p) {
    h->reduce_blocks = 4 * h->num_sms;
    if (dev_alloc(h->partial, (size_t)h->reduce_blocks * 2 * S * sizeof(double)) != cudaSuccess)
      return fail(BIOFVM_ERR_OOM, "device allocation of the reduction scratch failed");
  }
  const int64_t na = (int64_t)h->h_voxel.size();
  if (!h->agents_on_device && na > 0) {
    std::vector<int64_t> el((size_t)na * S), en((size_t)na * S);
    for (int64_t k = 0; k < na; k++)
      for (int s = 0; s < S; s++) {
        const int64_t e = h->h_voxel[k] * S + s;
        auto it = std::lower_bound(h->h_src_elem.begin(), h->h_src_elem.end(), e);
        el[k * S + s] = e;
        en[k * S + s] = (it != h->h_src_elem.end() && *it == e) ? (it - h->h_src_elem.begin()) : -1;
      }
    if (dev_alloc(h->ag_elem, el.size() * 8) != cudaSuccess ||
        dev_alloc(h->ag_entry, en.size() * 8) != cudaSuccess ||
        dev_alloc(h->ag_target, h->h_target.size() * 8) != cudaSuccess ||
        dev_alloc(h->ag_weight, h->h_weight.size() * 8) != cudaSuccess)
      return fail(BIOFVM_ERR_OOM, "device allocation of the agent arrays failed");
    CK(cudaMemcpy(h->ag_elem.p, el.data(), el.size() * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->ag_entry.p, en.data(), en.size() * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->ag_target.p, h->h_target.data(), h->h_target.size() * 8,
                  cudaMemcpyHostToDevice));
    if (!h->h_weight.empty())
      CK(cudaMemcpy(h->ag_weight.p, h->h_weight.data(), h->h_weight.size() * 8,
                    cudaMemcpyHostToDevice));
    h->agents_on_device = true;
  }
  const char *sv = static_cast<const char *>(saved);
  const int mask = kDirAfter | kMaskZero;
  auto reduce = [&](int axis, const void *u) -> cudaError_t {
    ReduceLaunch r{};
    r.mu = h->adj.p;
    r.u = u;
    r.nel = (long long)h->nel;
    r.S = S;
    r.stride = axis == 0 ? S : axis == 1 ? (long long)h->g.nx * S : (long long)h->g.nx * h->g.ny * S;
    r.n_axis = axis_len(h, axis);
    r.nblocks = h->reduce_blocks;
    r.used = (long long)r.nblocks * kReduceThreads / S * S;
    r.partial = static_cast<double *>(h->partial.p);
    r.scale_lambda = -h->dt / 3.0;
    r.scale_D = -h->dt / (h->h3[axis] * h->h3[axis]);
    r.dlambda = dlambda;
    r.dD = dD;
    return h->prec == BIOFVM_FP64 ? launch_adj_reduce_f64(r, st) : launch_adj_reduce_f32(r, st);
  };
  auto Bt = [&]() -> cudaError_t {  // adjoint of B: zero at the faces and the nodes
    if (h->any_dir) {
      const cudaError_t e = launch_x(h, mask, st, h->adj.p);
      if (e != cudaSuccess) return e;
    }
    return launch_nodes(h, st, 0, -1, true, h->adj.p);
  };
  CK(cudaMemcpyAsync(h->adj.p, grad_out, bytes, cudaMemcpyDeviceToDevice, st));
  CK(Bt());
  CK(launch_col(h, 2, kSolve, st, 1));
  CK(reduce(2, sv + 3 * bytes));
  CK(Bt());
  CK(launch_col(h, 1, kSolve, st, 1));
  CK(reduce(1, sv + 2 * bytes));
  CK(Bt());
  CK(launch_x(h, kSolve, st, h->adj.p));
  CK(reduce(0, sv + bytes));
  CK(Bt());
  SrcAdjLaunch a{};
  a.gbar = h->adj.p;
  a.u1 = sv;
  a.elem = static_cast<const int64_t *>(h->ag_elem.p);
  a.entry = static_cast<const int64_t *>(h->ag_entry.p);
  a.weight = h->h_weight.empty() ? nullptr : static_cast<const double *>(h->ag_weight.p);
  a.target = static_cast<const double *>(h->ag_target.p);
  a.n = na * S;
  a.src_elem = static_cast<const int64_t *>(h->src_elem.p);
  a.src_scale = h->src_scale.p;
  a.n_entries = h->n_entries;
  a.dt = h->dt;
  a.S = S;
  a.dsec = dsecretion;
  a.dupt = duptake;
  CK(h->prec == BIOFVM_FP64 ? launch_src_adjoint_f64(a, st) : launch_src_adjoint_f32(a, st));
  CK(cudaMemcpyAsync(grad_in, h->adj.p, bytes, cudaMemcpyDeviceToDevice, st));
  return BIOFVM_OK;
}

void biofvm_destroy(biofvm_t *h) { destroy_impl(h); }

}  // extern "C"

// ===========================================================================
// Batched environments: one persistent launch advances all of them.
// ===========================================================================
struct biofvm_batch {
  std::vector<biofvm *> env;
  std::vector<unsigned> env_gen;
  std::vector<std::array<int, 3>> whole;  // per environment and axis: whole-line tiles
  biofvm_precision prec = BIOFVM_FP32;
  cudaStream_t stream = nullptr, cap_stream = nullptr;
  int device = 0, maxm = 8, grid = 0;
  int64_t per_step = 0;
  DevBuf envs_d, tile_off_d, done_d, flags_d;  // flags: [0] abort, [1] status, [2..3] claims
  int dynamic = 1;  // work items claimed from a counter (else static round robin)
  int ctas_cap = 0;  // CTAs per SM of the persistent launch at most (0: as many as fit)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int graph_steps = -1;
  int stall_test = 0;
  // Per-environment mode (graph_mode): each environment is an ordinary handle with the
  // single-grid plans (pipelined or streaming sweeps), and a batch step is one CUDA graph of
  // every environment's three sweep launches, environments on parallel branches (forked
  // over kForks capture streams); the persistent kernel is not used.
  int graph_mode = 0;
  std::vector<cudaStream_t> fork;
  std::vector<cudaEvent_t> fork_ev;  // [0] fork, [1 + f] join of branch f
  std::vector<int> fork_of;          // environment -> branch (largest first to the least loaded)
  // graphs of K = 1..kGraphSteps steps of every environment (slot K)
  cudaGraph_t ggraph[9] = {};
  cudaGraphExec_t gg[9] = {};
};

namespace {

// Tile shape of one batched axis of n voxels.  want >= n: whole lines
// (streaming solve, chunk_m = 0 lets the environment's own handle plan its
// chunks); otherwise chunks of want positions -- at most kBatchWarps chunks of
// at most 48 positions, and along x a row's S lines in one warp (T*S <= 32);
// want <= 0 picks a default.  Returns false (message set) if not allowed.
bool batch_axis_shape(int e, int axis, int n, int S, int want, int &chunk_m, int &whole) {
  whole = 0;
  chunk_m = 0;
  // default: whole lines, except along x with one or two substrates (a warp
  // would then read 16 or 32 rows at once), where chunks measured faster
  if (want <= 0 && (axis > 0 || S >= 3)) want = n;
  if (want >= n && n >= 1) {
    whole = 1;
    return true;
  }
  if (want <= 0) want = std::max(8, (n + kBatchWarps - 1) / kBatchWarps);
  if (axis == 0 && S >= 1 && S <= 32)
    want = std::max(want, (n + 32 / S - 1) / (32 / S));
  const int m = std::min(want, std::max(n, 1));
  if (m >= n) {  // the default reached the whole line
    whole = 1;
    return true;
  }
  if ((n + m - 1) / m > kBatchWarps || m > 48) {
    fail(BIOFVM_ERR_ARG,
         "environment %d axis %d: chunk length %d gives more than %d chunks or exceeds 48 "
         "(use >= %d for whole lines)", e, axis, m, kBatchWarps, n);
    return false;
  }
  chunk_m = m;
  return true;
}

void batch_drop_graph(biofvm_batch *b) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->gexec = nullptr;
  b->graph = nullptr;
  b->graph_steps = -1;
}

void batch_drop_graph_mode(biofvm_batch *b);

void batch_destroy_impl(biofvm_batch *b) {
  if (!b) return;
  cudaSetDevice(b->device);
  cudaStreamSynchronize(b->stream);
  batch_drop_graph(b);
  batch_drop_graph_mode(b);
  for (biofvm *h : b->env) destroy_impl(h);
  for (DevBuf *d : {&b->envs_d, &b->tile_off_d, &b->done_d, &b->flags_d}) d->release();
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  for (cudaStream_t s : b->fork) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->fork_ev) cudaEventDestroy(e);
  delete b;
}

constexpr int kForks = 32;       // parallel capture streams of the per-environment mode
constexpr int kGraphSteps = 8;   // steps of every environment in one graph

void batch_drop_graph_mode(biofvm_batch *b) {
  for (int k = 0; k <= kGraphSteps; k++) {
    if (b->gg[k]) cudaGraphExecDestroy(b->gg[k]);
    if (b->ggraph[k]) cudaGraphDestroy(b->ggraph[k]);
    b->gg[k] = nullptr;
    b->ggraph[k] = nullptr;
  }
}

// K steps of every environment as one CUDA graph (per-environment mode): environment e's K
// steps (x-, y-, z-sweep launches each) on capture stream fork_of[e], forked from and joined
// back to the batch's capture stream, so environments run through their K steps without
// waiting for one another.  A field with unaligned rows steps on its row-padded copy (copied
// in and out by biofvm_batch_step around all the steps of the call).
biofvm_status batch_capture_graph_mode(biofvm_batch *b, int K) {
  const int ne = (int)b->env.size(), nf = (int)b->fork.size();
  CK(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
  biofvm_status st = BIOFVM_OK;
  cudaError_t e = cudaEventRecord(b->fork_ev[0], b->cap_stream);
  for (int f = 0; f < nf && e == cudaSuccess; f++) e = cudaStreamWaitEvent(b->fork[f], b->fork_ev[0], 0);
  for (int i = 0; i < ne && e == cudaSuccess && st == BIOFVM_OK; i++) {
    const biofvm *h = b->env[i];
    for (int k = 0; k < K && st == BIOFVM_OK; k++)
      st = launch_step(h, b->fork[b->fork_of[i]], 0, true, h->pitched != 0);
  }
  for (int f = 0; f < nf && e == cudaSuccess; f++) {
    e = cudaEventRecord(b->fork_ev[1 + f], b->fork[f]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->cap_stream, b->fork_ev[1 + f], 0);
  }
  cudaGraph_t graph = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(b->cap_stream, &graph);
  if (st != BIOFVM_OK || e != cudaSuccess || e2 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    if (st != BIOFVM_OK) return st;
    return fail(BIOFVM_ERR_CUDA, "batch graph capture failed: %s",
                cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  const cudaError_t e3 = cudaGraphInstantiate(&b->gg[K], graph, 0);
  if (e3 != cudaSuccess) {
    cudaGraphDestroy(graph);
    return fail(BIOFVM_ERR_CUDA, "cudaGraphInstantiate failed: %s", cudaGetErrorString(e3));
  }
  b->ggraph[K] = graph;
  return BIOFVM_OK;
}

// Tiles of 32 lines per sweep of a batched environment: x tiles hold
// floor(32/S) rows of S lines, y and z tiles 32 consecutive columns.
void batch_tiles(const biofvm *h, int64_t tiles[3]) {
  const int S = h->g.n_sub, rpt = 32 / S;
  const int64_t nrows = (int64_t)h->g.ny * h->g.nz, rowlen = (int64_t)h->g.nx * S;
  tiles[0] = (nrows + rpt - 1) / rpt;
  tiles[1] = (int64_t)h->g.nz * ((rowlen + 31) / 32);
  tiles[2] = (rowlen * h->g.ny + 31) / 32;
}

// Scratch bytes of an FP32 environment with whole-line axes: one [n][32]
// tile per tile of the largest sweep (the single-grid streaming sweep's
// field-sized scratch is never larger).
size_t batch_scratch_bytes(const biofvm *h) {
  int64_t tiles[3];
  batch_tiles(h, tiles);
  const int64_t ns[3] = {h->g.nx, h->g.ny, h->g.nz};
  int64_t el = (int64_t)h->nel;
  for (int a = 0; a < 3; a++) el = std::max(el, tiles[a] * ns[a] * 32);
  return (size_t)el * h->esz;
}

// Environment descriptors (device pointers of every environment's field,
// constants and sources) and the tile prefix sums.
biofvm_status batch_upload(biofvm_batch *b) {
  const int ne = (int)b->env.size();
  std::vector<BatchEnv> d(ne);
  std::vector<int64_t> off(3 * (size_t)(ne + 1), 0);
  for (int e = 0; e < ne; e++) {
    const biofvm *h = b->env[e];
    if (h->n_dnode > 0)
      return fail(BIOFVM_ERR_ARG, "environment %d: Dirichlet nodes are not supported in a batch", e);
    BatchEnv &x = d[e];
    x.field = h->rho.p;
    x.nx = h->g.nx;
    x.ny = h->g.ny;
    x.nz = h->g.nz;
    x.S = h->g.n_sub;
    for (int axis = 0; axis < 3; axis++) {
      const AxisTab t = axis_tab(h, axis);
      x.tab[axis] = t.inv;
      x.T[axis] = t.T;
      x.m[axis] = t.m;
    }
    x.rows_per_tile = 32 / x.S;
    batch_tiles(h, x.tiles);
    const bool fp64 = h->prec == BIOFVM_FP64;
    for (int ph = 0; ph < 3; ph++) {
      x.whole[ph] = b->whole[e][ph];
      x.group[ph] = x.whole[ph] ? kBatchWarps : std::max(1, kBatchWarps / x.T[ph]);
      x.items[ph] = (x.tiles[ph] + x.group[ph] - 1) / x.group[ph];
      x.stab[ph] = fp64 ? h->tabS[ph].p : h->tab[ph].p;
      x.sint[ph] = static_cast<const char *>(h->stream_const_d.p) + (size_t)ph * 2 * x.S * h->csz;
      x.cfix[ph] = axis_tab(h, ph).cfix;
      x.k0[ph] = h->stream_k0[ph];
    }
    x.scratch = h->scratch.p;
    x.src_row_off = static_cast<const int64_t *>(h->src_row_off.p);
    x.src_elem = static_cast<const int64_t *>(h->src_elem.p);
    x.src_alpha = h->src_alpha.p;
    x.src_scale = h->src_scale.p;
    x.has_src = h->n_entries > 0;
    for (int ph = 0; ph < 3; ph++) off[ph * (ne + 1) + e + 1] = off[ph * (ne + 1) + e] + x.items[ph];
    b->env_gen[e] = h->generation;
  }
  b->per_step = off[0 * (ne + 1) + ne] + off[1 * (ne + 1) + ne] + off[2 * (ne + 1) + ne];
  CK(cudaMemcpy(b->envs_d.p, d.data(), d.size() * sizeof(BatchEnv), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(b->tile_off_d.p, off.data(), off.size() * 8, cudaMemcpyHostToDevice));
  batch_drop_graph(b);
  return BIOFVM_OK;
}

}  // namespace

extern "C" {

biofvm_status biofvm_batch_create(int n_env, const biofvm_grid *grids, const double *dx,
                                  const double *dt, const double *D_flat,
                                  const double *lambda_flat, biofvm_precision prec,
                                  uintptr_t cuda_stream, const int *tile_m,
                                  biofvm_batch_t **out) {
  g_last_error.clear();
  if (!out) return fail(BIOFVM_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (n_env < 1 || !grids || !dx || !dt || !D_flat || !lambda_flat)
    return fail(BIOFVM_ERR_ARG, "n_env must be >= 1 and every array non-NULL");
  biofvm_batch *b = new (std::nothrow) biofvm_batch();
  if (!b) return fail(BIOFVM_ERR_OOM, "host allocation failed");
  b->prec = prec;
  b->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  // mode: BIOFVM_BATCH_MODE=graph / persistent, else per-environment graphs when the mean
  // environment holds >= 2^20 voxel-substrates (enough for the single-grid sweeps to fill the
  // GPU in a few concurrent launches), the persistent kernel for smaller ones
  {
    const char *env = getenv("BIOFVM_BATCH_MODE");
    if (env && (!strcmp(env, "graph") || !strcmp(env, "persistent"))) {
      b->graph_mode = !strcmp(env, "graph");
    } else {
      double total = 0.0;
      for (int e = 0; e < n_env; e++)
        total += (double)grids[e].nx * grids[e].ny * grids[e].nz * grids[e].n_sub;
      b->graph_mode = total / n_env >= 1048576.0;
    }
  }
  if (const char *env = getenv("BIOFVM_BATCH_DYNAMIC")) b->dynamic = atoi(env) != 0;
  if (const char *env = getenv("BIOFVM_BATCH_CTAS")) b->ctas_cap = std::max(0, atoi(env));
  int64_t off = 0;
  for (int e = 0; e < n_env; e++) {
    const biofvm_grid &g = grids[e];
    int m[3] = {0, 0, 0}, whole[3] = {0, 0, 0};
    const int ns[3] = {g.nx, g.ny, g.nz};
    if (g.n_sub < 1 || g.n_sub > 32) {
      batch_destroy_impl(b);
      return fail(BIOFVM_ERR_ARG, "environment %d: n_sub must be in [1, 32]", e);
    }
    for (int a = 0; a < 3 && !b->graph_mode; a++)
      if (!batch_axis_shape(e, a, ns[a], g.n_sub, tile_m ? tile_m[3 * e + a] : 0, m[a],
                            whole[a])) {
        const biofvm_status st = BIOFVM_ERR_ARG;
        batch_destroy_impl(b);
        return st;
      }
    biofvm *h = nullptr;
    biofvm_status st = create_impl(&g, dx[e], dt[e], D_flat + off, lambda_flat + off, nullptr,
                                   prec, cuda_stream, b->graph_mode ? nullptr : m, &h);
    if (st != BIOFVM_OK) {
      std::string msg = g_last_error;
      batch_destroy_impl(b);
      return fail(st, "environment %d: %s", e, msg.c_str());
    }
    b->env.push_back(h);
    b->env_gen.push_back(0);
    b->whole.push_back({whole[0], whole[1], whole[2]});
    for (int a = 0; a < 3; a++) b->maxm = std::max(b->maxm, m[a]);
    if ((whole[0] || whole[1] || whole[2]) && prec == BIOFVM_FP32 &&
        h->scratch.bytes < batch_scratch_bytes(h) &&
        dev_alloc(h->scratch, batch_scratch_bytes(h)) != cudaSuccess) {
      batch_destroy_impl(b);
      return fail(BIOFVM_ERR_OOM, "environment %d: scratch field allocation failed", e);
    }
    off += g.n_sub;
  }
  b->device = b->env[0]->device;
  if (b->graph_mode) {  // capture streams and fork / join events; no persistent-kernel state
    const int nf = std::min(n_env, kForks);
    cudaError_t e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    for (int f = 0; f < nf && e == cudaSuccess; f++) {
      cudaStream_t s = nullptr;
      e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
      if (e == cudaSuccess) b->fork.push_back(s);
    }
    for (int f = 0; f <= nf && e == cudaSuccess; f++) {
      cudaEvent_t ev = nullptr;
      e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      if (e == cudaSuccess) b->fork_ev.push_back(ev);
    }
    if (e != cudaSuccess) {
      batch_destroy_impl(b);
      return fail(BIOFVM_ERR_CUDA, "batch set-up failed: %s", cudaGetErrorString(e));
    }
    // branches balanced by voxel-substrates: largest environment first, to the least loaded
    std::vector<int> order(n_env);
    for (int i = 0; i < n_env; i++) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return b->env[x]->nel > b->env[y]->nel; });
    std::vector<double> load(nf, 0.0);
    b->fork_of.assign(n_env, 0);
    for (int i : order) {
      const int f = (int)(std::min_element(load.begin(), load.end()) - load.begin());
      b->fork_of[i] = f;
      load[f] += (double)b->env[i]->nel;
    }
    *out = b;
    return BIOFVM_OK;
  }
  for (int c : kBatchMaxm)
    if (c >= b->maxm) {
      b->maxm = c;
      break;
    }
  const bool fp64 = prec == BIOFVM_FP64;
  int per_sm = 0;
  cudaError_t e = fp64 ? batch_occupancy_f64(b->maxm, &per_sm) : batch_occupancy_f32(b->maxm, &per_sm);
  if (e != cudaSuccess || per_sm < 1) {
    batch_destroy_impl(b);
    return fail(BIOFVM_ERR_CUDA, "batched kernel occupancy query failed");
  }
  if (b->ctas_cap > 0) per_sm = std::min(per_sm, b->ctas_cap);
  b->grid = per_sm * b->env[0]->num_sms;  // every CTA resident (the schedule relies on it)
  if (dev_alloc(b->envs_d, (size_t)n_env * sizeof(BatchEnv)) != cudaSuccess ||
      dev_alloc(b->tile_off_d, 3 * (size_t)(n_env + 1) * 8) != cudaSuccess ||
      dev_alloc(b->done_d, 3 * (size_t)n_env * sizeof(unsigned)) != cudaSuccess ||
      dev_alloc(b->flags_d, 4 * sizeof(int)) != cudaSuccess) {
    batch_destroy_impl(b);
    return fail(BIOFVM_ERR_OOM, "device allocation of the batch descriptors failed");
  }
  if ((e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaMemset(b->flags_d.p, 0, 4 * sizeof(int))) != cudaSuccess) {
    batch_destroy_impl(b);
    return fail(BIOFVM_ERR_CUDA, "batch set-up failed: %s", cudaGetErrorString(e));
  }
  biofvm_status st = batch_upload(b);
  if (st != BIOFVM_OK) {
    std::string msg = g_last_error;
    batch_destroy_impl(b);
    g_last_error = msg;
    return st;
  }
  *out = b;
  return BIOFVM_OK;
}

biofvm_status biofvm_batch_env(biofvm_batch_t *b, int e, biofvm_t **env) {
  if (!b || !env || e < 0 || e >= (int)b->env.size())
    return fail(BIOFVM_ERR_ARG, "bad batch handle, environment index or output");
  *env = b->env[e];
  return BIOFVM_OK;
}

biofvm_status biofvm_batch_step(biofvm_batch_t *b, int n_steps) {
  if (!b) return fail(BIOFVM_ERR_ARG, "NULL batch handle");
  if (n_steps < 0) return fail(BIOFVM_ERR_ARG, "n_steps must be >= 0");
  if (n_steps == 0) return BIOFVM_OK;
  CK(cudaSetDevice(b->device));
  bool stale = false;
  for (size_t e = 0; e < b->env.size(); e++) stale |= b->env[e]->generation != b->env_gen[e];
  if (b->graph_mode) {  // one graph of one step for all environments, launched n_steps times
    for (size_t e = 0; e < b->env.size(); e++)
      if (b->env[e]->n_dnode > 0)
        return fail(BIOFVM_ERR_ARG, "environment %zu: Dirichlet nodes are not supported in "
                                    "batched environments", e);
    if (stale) {
      batch_drop_graph_mode(b);
      for (size_t e = 0; e < b->env.size(); e++) b->env_gen[e] = b->env[e]->generation;
    }
    const int K = std::min(n_steps, kGraphSteps), blocks = n_steps / K, tail = n_steps % K;
    for (int k : {K, tail})
      if (k > 0 && !b->gg[k]) {
        biofvm_status st = batch_capture_graph_mode(b, k);
        if (st) return st;
      }
    for (const biofvm *h : b->env)
      if (h->pitched) CK(pitch_copy(h, true, b->stream));
    for (int k = 0; k < blocks; k++) CK(cudaGraphLaunch(b->gg[K], b->stream));
    if (tail > 0) CK(cudaGraphLaunch(b->gg[tail], b->stream));
    for (const biofvm *h : b->env)
      if (h->pitched) CK(pitch_copy(h, false, b->stream));
    return BIOFVM_OK;
  }
  if (stale) {
    CK(cudaStreamSynchronize(b->stream));  // descriptors are read by launches in flight
    biofvm_status st = batch_upload(b);
    if (st) return st;
  }
  if (!b->gexec || b->graph_steps != n_steps) {
    batch_drop_graph(b);
    const int ne = (int)b->env.size();
    BatchArgs a{};
    a.env = static_cast<const BatchEnv *>(b->envs_d.p);
    a.n_env = ne;
    a.n_steps = n_steps;
    a.tile_off = static_cast<const int64_t *>(b->tile_off_d.p);
    a.per_step = b->per_step;
    a.done = static_cast<unsigned *>(b->done_d.p);
    a.abort_flag = static_cast<int *>(b->flags_d.p);
    a.status = static_cast<int *>(b->flags_d.p) + 1;
    a.stall_test = b->stall_test;
    a.next = b->dynamic ? reinterpret_cast<unsigned long long *>(
                              static_cast<int *>(b->flags_d.p) + 2)
                        : nullptr;
    a.maxm = b->maxm;
    const int grid = (int)std::min<int64_t>(b->grid, b->per_step * n_steps);
    CK(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e1 = cudaMemsetAsync(b->done_d.p, 0, 3 * (size_t)ne * sizeof(unsigned), b->cap_stream);
    cudaError_t e2 = cudaMemsetAsync(b->flags_d.p, 0, sizeof(int), b->cap_stream);  // abort flag
    if (e2 == cudaSuccess && a.next) e2 = cudaMemsetAsync(a.next, 0, 8, b->cap_stream);
    cudaError_t e3 = b->prec == BIOFVM_FP64 ? launch_batch_f64(a, b->maxm, grid, b->cap_stream)
                                            : launch_batch_f32(a, b->maxm, grid, b->cap_stream);
    cudaGraph_t graph = nullptr;
    cudaError_t e4 = cudaStreamEndCapture(b->cap_stream, &graph);
    for (cudaError_t ee : {e1, e2, e3, e4})
      if (ee != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return fail(BIOFVM_ERR_CUDA, "batch graph capture failed: %s", cudaGetErrorString(ee));
      }
    cudaError_t e5 = cudaGraphInstantiate(&b->gexec, graph, 0);
    if (e5 != cudaSuccess) {
      cudaGraphDestroy(graph);
      return fail(BIOFVM_ERR_CUDA, "cudaGraphInstantiate failed: %s", cudaGetErrorString(e5));
    }
    b->graph = graph;
    b->graph_steps = n_steps;
  }
  CK(cudaGraphLaunch(b->gexec, b->stream));
  return BIOFVM_OK;
}

biofvm_status biofvm_batch_sync(biofvm_batch_t *b) {
  if (!b) return fail(BIOFVM_ERR_ARG, "NULL batch handle");
  CK(cudaSetDevice(b->device));
  CK(cudaStreamSynchronize(b->stream));
  if (b->graph_mode) {  // every environment's own status word
    for (biofvm *h : b->env) {
      biofvm_status st = check_status(h);
      if (st) return st;
    }
    return BIOFVM_OK;
  }
  int st = 0;
  CK(cudaMemcpy(&st, static_cast<int *>(b->flags_d.p) + 1, sizeof(int), cudaMemcpyDeviceToHost));
  if (st != kStatusOk) {
    CK(cudaMemset(b->flags_d.p, 0, 2 * sizeof(int)));
    return fail(BIOFVM_ERR_TIMEOUT, "a bounded wait of the batched kernel timed out");
  }
  return BIOFVM_OK;
}

int biofvm_batch_grid(const biofvm_batch_t *b) { return b && !b->graph_mode ? b->grid : 0; }

int biofvm_batch_mode(const biofvm_batch_t *b) { return b ? b->graph_mode : -1; }

biofvm_status biofvm_batch_set_tiles(biofvm_batch_t *b, const int *tile_m) {
  if (!b || !tile_m) return fail(BIOFVM_ERR_ARG, "NULL batch handle or tile shapes");
  if (b->graph_mode)
    return fail(BIOFVM_ERR_STATE, "per-environment graph mode: the environments use the "
                                  "single-grid plans, there are no batched tiles to set");
  CK(cudaSetDevice(b->device));
  CK(cudaStreamSynchronize(b->stream));
  const bool fp64 = b->prec == BIOFVM_FP64;
  std::vector<XPlan> xp(b->env.size());
  std::vector<ColPlan> cy(b->env.size()), cz(b->env.size());
  int maxm = 8;
  std::vector<std::array<int, 3>> whole(b->env.size());
  for (size_t e = 0; e < b->env.size(); e++) {  // validate everything before changing anything
    const biofvm *h = b->env[e];
    const int ns[3] = {h->g.nx, h->g.ny, h->g.nz};
    int m[3];
    for (int a = 0; a < 3; a++) {
      if (!batch_axis_shape((int)e, a, ns[a], h->g.n_sub, tile_m[3 * e + a], m[a], whole[e][a]))
        return BIOFVM_ERR_ARG;
      maxm = std::max(maxm, m[a]);
    }
    if (!plan_x(h->g.nx, h->g.n_sub, fp64, xp[e], m[0]) || !plan_col(h->g.ny, fp64, cy[e], m[1]) ||
        !plan_col(h->g.nz, fp64, cz[e], m[2]))
      return fail(BIOFVM_ERR_ARG, "environment %zu: tile shapes do not fit the kernels", e);
  }
  for (size_t e = 0; e < b->env.size(); e++) {  // scratch fields for FP32 whole-line axes
    biofvm *h = b->env[e];
    if ((whole[e][0] || whole[e][1] || whole[e][2]) && !fp64 &&
        h->scratch.bytes < batch_scratch_bytes(h) &&
        dev_alloc(h->scratch, batch_scratch_bytes(h)) != cudaSuccess)
      return fail(BIOFVM_ERR_OOM, "environment %zu: scratch field allocation failed", e);
  }
  for (int c : kBatchMaxm)
    if (c >= maxm) {
      maxm = c;
      break;
    }
  int per_sm = 0;
  CK(fp64 ? batch_occupancy_f64(maxm, &per_sm) : batch_occupancy_f32(maxm, &per_sm));
  for (size_t e = 0; e < b->env.size(); e++) {
    biofvm *h = b->env[e];
    h->xp = xp[e];
    h->cp[1] = cy[e];
    h->cp[2] = cz[e];
    biofvm_status st = upload_constants(h);
    if (st) return st;
  }
  b->maxm = maxm;
  b->whole = whole;
  if (b->ctas_cap > 0) per_sm = std::min(per_sm, b->ctas_cap);
  b->grid = std::max(per_sm, 1) * b->env[0]->num_sms;
  return batch_upload(b);
}

biofvm_status biofvm_batch_test_stall(biofvm_batch_t *b, int on) {
  if (!b) return fail(BIOFVM_ERR_ARG, "NULL batch handle");
  if (b->graph_mode)
    return fail(BIOFVM_ERR_STATE, "the stall hook belongs to the persistent batched kernel");
  b->stall_test = on ? 1 : 0;
  batch_drop_graph(b);  // the hook is a kernel argument
  return BIOFVM_OK;
}

void biofvm_batch_destroy(biofvm_batch_t *b) { batch_destroy_impl(b); }

}  // extern "C"
