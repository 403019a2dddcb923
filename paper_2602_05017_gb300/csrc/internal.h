// Internal interface between the host half of libbiofvm (api.cpp) and the
// sweep kernels (sweeps_fp64.cu, sweeps_fp32.cu, pipe_fp32.cu).  Not installed; the public
// C ABI is include/biofvm.h.
#pragma once
#include <cuda.h>  // CUtensorMap (type only; the encoder is fetched at run time)
#include <cuda_runtime.h>
#include <stdint.h>

namespace bfv {

// Stage flags of the sweep kernels (the x-sweep also owns Src and the first
// two Dirichlet applications of a step).
enum : int {
  kSrc = 1,        // rho <- (rho + alpha) * scale on the listed elements
  kDirBefore = 2,  // Dirichlet application before the solve
  kSolve = 4,      // Thomas solve along the axis
  kDirAfter = 8,   // Dirichlet application after the solve
  kMaskZero = 16,  // Dirichlet applications write 0 (the adjoint of B: dB/du = mask)
  kScaled = 32,    // streaming sweeps of a whole step: scaled intermediate output
  kKeepScale = 64, // z-sweep of a scaled step that leaves the field scaled (no omega)
  // bits 8..15: the step's index m within its renormalisation block (host only)
};

// Status word values written by kernels (mirror biofvm_status).
enum : int { kStatusOk = 0, kStatusTimeout = 4 };

// Thomas constants of one axis, element type E, layout [i][S] (position-major,
// substrate fastest), computed in double on the host (App. A) and rounded:
//   inv[i]  = 1/denom_i           mul[i] = r/denom_i = -c'_i
//   pf[i]   = prod_{l=lo(i)}^{i} mul_l     (forward carry weight in a chunk)
//   pb[i]   = prod_{l=i}^{hi(i)} mul_l     (backward carry weight in a chunk)
//   pc[t]   = prod over chunk t of mul_l   (layout [t][S])
// where the axis is cut into T chunks of m positions (the last may be short).
//
// FP32 path (defect-correction form): the zero-flux rows of A = (1 + lam3) I
// + r L_N sum to 1 + lam3, so A^-1 d = c d - c r A^-1 (L_N d), c = 1/(1+lam3).
// The kernels solve for the small correction y = (-c r) A^-1 (L_N d) -- inv
// then holds (-c r)/denom_i -- and form x = c_hi d + (c_lo d + y) with one
// final rounding; cfix = [c_hi[S], c_lo[S]].  Plain FP32 Thomas accumulates a
// rounding bias along smooth lines (about 3e-5 after 300 sweeps); this form
// stays at the storage-rounding level (about 2e-7).
//
// cw [T][T][S]: the carry entering chunk t from chunk u is cw[u][t] times the
// end (forward) or start (backward) value of chunk u, cw[u][t] being the
// product of pc over the chunks strictly between u and t.
//
// tabT: inv, mul, pf, pb again, substrate-major [4][S][n_pad] with
// n_pad = 32*ceil(n/32) + 1 (the layout the pipelined kernel stages into
// shared memory; the planner takes that kernel only when they fit).
struct AxisTab {
  const void *inv, *mul, *pf, *pb, *pc, *cfix, *cw, *tabT;
  int n, T, m;
};

// x-sweep launch: rows (y, z) of nx*S contiguous elements, rows_per_cta rows
// staged per CTA; a row's S lines are cut into T segments, one lane each.
struct XLaunch {
  void *rho;
  int nx, ny, nz, S;
  AxisTab tab;
  int rows_per_cta, rows_per_warp, warps, maxm;
  int use_bulk;        // tile staged with cp.async.bulk (16-byte aligned rows)
  size_t smem_bytes;
  int flags;
  // sources: CSR over rows; element index (global); alpha; scale = 1/(1+beta)
  const int64_t *src_row_off;
  const int64_t *src_elem;
  const void *src_alpha, *src_scale;
  int has_src;
  const uint8_t *dir_on;
  const void *dir_val;
  int *status;
};

// y- or z-sweep launch: lines are columns of a plane, column c at
// plane*plane_stride + j*C + c for j = 0..n-1 (C = stride between positions).
struct ColLaunch {
  void *rho;
  int64_t C, plane_stride;
  int nplanes, n, S;
  int mode;  // 1 = y-sweep (plane = z, column -> x), 2 = z-sweep (column -> x, y)
  int nx, ny, nz;
  AxisTab tab;
  int maxm;
  int flags;  // kSolve | kDirAfter
  const uint8_t *dir_on;
  const void *dir_val;
};

// Streaming sweep (stream.cuh): one lane per whole line, persistent grid of
// 128-thread CTAs, warps striding over groups of 32 lines.
struct StreamArgs {
  void *rho;
  int n, S;
  int mode;               // 0 = x (lanes: rows x substrates), 1 = y, 2 = z (lanes: columns)
  int nx, ny, nz;
  long long stride;       // elements between consecutive positions of a line
  long long ngroups;      // 32-line groups in all
  int rows_per_warp;      // x: 32/S
  const void *tab;        // position-major [n][S] blocks: inv, mul (FP64: and q)
  int out;                // FP64: 0: x; 1: y = x / sigma; 2: omega y (stream.cuh)
  int k0;                 // interior (one value per substrate) from k0 to n-2
  const void *interior;   // [2][S] the interior inv and mul (FP64: sigma, r sigma)
  const void *omega;      // FP64 [S] z multiplier of a renormalising step (out 2)
  const void *src_fac;    // FP64 [S] factor on the source alpha (field stored scaled), or NULL
  const void *cfix;       // FP32 [2][S] c_hi, c_lo (defect form)
  void *scratch;          // FP32: field-sized scratch for the forward intermediate
  int ks;                 // FP64: positions whose intermediate stays in shared memory
  int xt;                 // FP64 x-sweep at S = 1, 2, 4: S (coalesced rows), else 0
  int r8;                 // FP64: 8-position register blocks, four CTAs per SM (else 16, three)
  int flags;
  const int64_t *src_row_off, *src_elem;
  const void *src_alpha, *src_scale;
  int has_src;
  const uint8_t *dir_on;
  const void *dir_val;     // Dirichlet value written after the solve (output units)
  const void *dir_val_in;  // ... and before it (input units)
};

// Persistent TMA-pipelined sweep (pipe.cuh): tiles of 32 lines x n positions
// through a ring of shared-memory stages.
struct PipeArgs;

// Opt-in dynamic shared memory per CTA on sm_100-class GPUs (227 KB).
constexpr size_t kMaxDynamicSmem = 232448;

// Threads per block of the adjoint reduction.
constexpr int kReduceThreads = 256;

// Adjoint parameter-gradient reduction of one sweep (adjoint.cuh).
// Dirichlet nodes: rho[elem[k]] = val[k] * scale[elem[k] % S] (scale NULL: 1),
// or 0 with `zero` (the adjoint's mask).  elem sorted and unique.
struct NodeLaunch {
  void *rho;
  const int64_t *elem;
  const void *val, *scale;
  int64_t n;
  int S, zero, grid;
};

struct ReduceLaunch {
  const void *mu, *u;           // adjoint after the sweep, forward sweep output
  long long nel, stride, used;  // elements; element stride along the axis; threads used
  int S, n_axis, nblocks;
  double *partial;              // [nblocks][2][S] scratch
  double scale_lambda, scale_D; // -dt/3, -dt/dx^2
  double *dlambda, *dD;         // [S] accumulated (device)
};
// Adjoint of the source update (adjoint.cuh).
struct SrcAdjLaunch {
  void *gbar;
  const void *u1;                      // forward source output
  const int64_t *elem, *entry;         // [n] per (agent, substrate)
  const double *weight, *target;       // [n/S] or NULL, [n]
  long long n;
  const int64_t *src_elem;             // aggregated entries
  const void *src_scale;               // 1/(1+beta) per entry
  long long n_entries;
  double dt;
  int S;
  double *dsec;                        // [n] accumulated (device) or NULL
  double *dupt;                        // [n] accumulated (device) or NULL
};

// Batched persistent step (batch.cuh).
struct BatchArgs;
constexpr int kBatchMaxm[] = {8, 16, 24, 32, 48};
constexpr int kBatchWarps = 8;  // chunks per line at most (256-thread CTAs)

// Register-chunk capacities compiled for each precision (ascending).
constexpr int kMaxmF64[] = {8, 16, 24, 32, 48, 64};
constexpr int kMaxmF32[] = {8, 16, 24, 32, 48, 64, 96, 128};

// Raise the dynamic shared-memory limit of the x-sweep instantiation for
// chunk capacity maxm (called once per handle, outside any graph capture).
cudaError_t allow_x_smem_f64(int maxm, size_t bytes);
cudaError_t allow_x_smem_f32(int maxm, size_t bytes);
cudaError_t launch_x_f64(const XLaunch &a, cudaStream_t st);
cudaError_t launch_x_f32(const XLaunch &a, cudaStream_t st);
cudaError_t launch_col_f64(const ColLaunch &a, cudaStream_t st);
cudaError_t launch_col_f32(const ColLaunch &a, cudaStream_t st);
// The pipelined sweep is FP32 only (FP64 streams whole lines, stream.cuh).
cudaError_t allow_pipe_smem_f32(int maxm, size_t bytes);
cudaError_t launch_pipe_f32(const CUtensorMap &map, const PipeArgs &a, int maxm, int grid,
                            size_t smem, cudaStream_t st);
// Streaming sweeps (stream.cuh).
cudaError_t allow_stream_smem_f64();
cudaError_t launch_stream_f64(const StreamArgs &a, int grid, cudaStream_t st);
cudaError_t launch_stream_f32(const StreamArgs &a, int grid, cudaStream_t st);
// Small FP64 grids: all steps of a call in one cooperative launch (small.cu).
// Planes of nx*ny*S elements in shared memory for the x and y solves, z-lines
// by the streaming line solver; bar: 3 words (arrivals, generation, abort) of
// the bounded grid barrier, zeroed before each launch.
struct SmallArgs {
  double *rho;
  int nx, ny, nz, S;
  // per axis: the host's chunked axis tables (inv, mul, pf, pb [n][S], pc [T][S],
  // [2][S], cw [T][T][S]) for T chunks of m positions
  const double *tab[3];
  int T[3], m[3];
  const int64_t *src_row_off, *src_elem;
  const double *src_alpha, *src_scale;
  int has_src;
  const uint8_t *dir_on;
  const double *dir_val;
  int any_dir;
  int n_steps;
  unsigned *bar;
  int *status;
};
int small_chunks(int n, int L);
size_t small_smem_bytes(int nx, int ny, int nz, int S, const int T[3]);
cudaError_t small_max_blocks(int *blocks_per_sm, size_t smem);
cudaError_t launch_small_f64(const SmallArgs &a, int grid, size_t smem, cudaStream_t st);
// Sets the thread-local message biofvm_last_error() returns.
void set_error_message(const char *msg);

cudaError_t launch_adj_reduce_f64(const ReduceLaunch &a, cudaStream_t st);
cudaError_t launch_nodes_f64(const NodeLaunch &a, cudaStream_t st);
cudaError_t launch_nodes_f32(const NodeLaunch &a, cudaStream_t st);
cudaError_t launch_adj_reduce_f32(const ReduceLaunch &a, cudaStream_t st);
cudaError_t launch_src_adjoint_f64(const SrcAdjLaunch &a, cudaStream_t st);
cudaError_t launch_src_adjoint_f32(const SrcAdjLaunch &a, cudaStream_t st);
cudaError_t launch_batch_f64(const BatchArgs &a, int maxm, int grid, cudaStream_t st);
cudaError_t launch_batch_f32(const BatchArgs &a, int maxm, int grid, cudaStream_t st);
cudaError_t batch_occupancy_f64(int maxm, int *out);
cudaError_t batch_occupancy_f32(int maxm, int *out);
// The same sweep for fields stored in 16 bits (bf16 / fp16), FP32 arithmetic;
// chunk capacities 32 and 64.
cudaError_t allow_pipe_smem_bf16(int maxm, size_t bytes);
cudaError_t allow_pipe_smem_fp16(int maxm, size_t bytes);
cudaError_t launch_pipe_bf16(const CUtensorMap &map, const PipeArgs &a, int maxm, int grid,
                             size_t smem, cudaStream_t st);
cudaError_t launch_pipe_fp16(const CUtensorMap &map, const PipeArgs &a, int maxm, int grid,
                             size_t smem, cudaStream_t st);
// Copy `rows` rows of `len` elements of esz (4 or 2) bytes from rows spitch
// elements apart into rows dpitch elements apart (the row-padded working copy
// of a field whose rows are not 16-byte multiples).
cudaError_t launch_pitch_rows(const void *src, void *dst, int64_t rows, int len, int spitch,
                              int dpitch, size_t esz, int grid, cudaStream_t st);
// Largest CTA the FP32 pipelined sweep with chunk capacity maxm may use.
int pipe_max_threads_f32(int maxm);
// Substrate-major constants of the pipelined sweep (elements): [4][S][npad].
inline int pipe_npad_host(int n) { return (n + 31) / 32 * 32 + 1; }
inline int pipe_tab_elems_host(int n, int S) { return 4 * S * pipe_npad_host(n); }

}  // namespace bfv
