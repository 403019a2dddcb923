/*
 * libbiofvm -- GB300 (sm_103a) LOD diffusion-decay step of BioFVM-B
 * (Estragues-Munoz et al., "A Novel Scalable High Performance diffusion
 * solver for multiscale cell simulations", arXiv 2602.05017).
 *
 * One time step advances every substrate of a 3D voxel grid (Sect. 2):
 *
 *   rho <- B . Z^-1 . B . Y^-1 . B . X^-1 . B . Src (rho)
 *
 *   Src   cell source/uptake update, rho <- (rho + alpha)/(1 + beta) per
 *         voxel with alpha = sum dt*w*S*rho_target and beta = sum dt*w*(S+U)
 *         over the agents in that voxel (the end-to-end run of Sect. 5.3;
 *         implicit form of the cited BioFVM);
 *   B     Dirichlet application: the voxels of the six faces take the
 *         substrate's Dirichlet value when its flag is on ("four
 *         applications of Dirichlet conditions", Sect. 2);
 *   X^-1  every x-line of every substrate solved with the Thomas algorithm
 *         (Algorithm 1; Sect. 2.1) on the system of Appendix A:
 *         a_i = c_i = -r, b = 1 + 2r + lambda*dt/3 inside, 1 + r + lambda*dt/3
 *         at the two ends (zero flux), 1 + lambda*dt/3 on a one-voxel axis,
 *         r = D*dt/dx^2;  Y^-1 and Z^-1 likewise along y and z.
 *
 * Field layout (Sect. 3.1, one contiguous 4D array): element (x, y, z, s) is
 * at index ((z*ny + y)*nx + x)*n_sub + s -- substrates interleaved per voxel,
 * x the fastest of the three axes.  The element type is double for
 * BIOFVM_FP64, float for BIOFVM_FP32, and a 16-bit bfloat16 / IEEE half for
 * BIOFVM_BF16 / BIOFVM_FP16 (Thomas constants are always computed in double on
 * the host, then rounded to the arithmetic type: double or float).
 *
 * Conventions of every call:
 *   - Errors are returned as a biofvm_status, never thrown; the thread-local
 *     message of the last failure is biofvm_last_error().
 *   - The library owns all device memory it allocates.  The caller owns and
 *     keeps every array it passes; the library copies what it needs (host
 *     arrays host->device, device arrays device->device) before returning.
 *   - All device work of a handle is ordered on the CUDA stream given at
 *     create (0 = the legacy default stream).  Calls marked "async" return
 *     before the GPU has finished; biofvm_density/biofvm_sync wait.
 *   - A handle is not thread-safe; distinct handles are independent.
 */
#ifndef BIOFVM_H
#define BIOFVM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct biofvm biofvm_t; /* opaque handle */

typedef enum {
  BIOFVM_OK = 0,
  BIOFVM_ERR_ARG = 1,     /* invalid argument (nothing was changed)        */
  BIOFVM_ERR_OOM = 2,     /* device or host allocation failed              */
  BIOFVM_ERR_CUDA = 3,    /* a CUDA call failed (message has its name)     */
  BIOFVM_ERR_TIMEOUT = 4, /* a bounded device-side wait gave up            */
  BIOFVM_ERR_STATE = 5    /* call not valid in the handle's current state  */
} biofvm_status;

/* BIOFVM_BF16 / BIOFVM_FP16: the field stored in 16 bits (bfloat16 / IEEE
 * half) with FP32 arithmetic and FP32 constants -- half the bytes of FP32, at
 * the storage rounding of 2^-8 (bf16) or 2^-11 (fp16) per stored value.  These
 * handles run whole steps (and the solve stages) on the pipelined sweep only:
 * create fails with ARG unless nx*n_sub and nx*ny*n_sub are multiples of 8
 * and the lines fit its tiles; Dirichlet nodes, the adjoint, stages 0 and 4
 * and batched environments are refused (STATE or ARG). */
typedef enum {
  BIOFVM_FP64 = 0,
  BIOFVM_FP32 = 1,
  BIOFVM_BF16 = 2,
  BIOFVM_FP16 = 3
} biofvm_precision;

typedef struct {
  int nx, ny, nz; /* voxels per axis, each >= 1                          */
  int n_sub;      /* substrates per voxel, 1 <= n_sub <= 32              */
} biofvm_grid;

/* Dirichlet condition per substrate (Sect. 2, the four applications).
 * dirichlet_on[s] != 0 switches it on for substrate s; dirichlet_value[s]
 * is the value written on the six faces.  A NULL biofvm_boundary pointer, or
 * NULL dirichlet_on, means zero-flux (Neumann) for every substrate. */
typedef struct {
  const uint8_t *dirichlet_on;    /* [n_sub] host */
  const double *dirichlet_value;  /* [n_sub] host */
} biofvm_boundary;

/* Create a microenvironment.  grid: sizes (host, read once).  dx: voxel edge
 * (> 0, same unit as sqrt(D*dt)).  dt: time step (> 0).  D[n_sub] >= 0 and
 * lambda[n_sub] >= 0: diffusion and decay per substrate (host).  bc: see
 * biofvm_boundary.  cuda_stream: a cudaStream_t cast to uintptr_t, kept for
 * the handle's life (the caller must keep it alive).  On success *out holds
 * the handle; the field is zero and there are no agents.
 * Computes the Thomas constants of App. A (denom, c') in double.
 * Errors: ARG (sizes, dx, dt, D, lambda, NULL), OOM, CUDA. */
biofvm_status biofvm_create(const biofvm_grid *grid, double dx, double dt,
                            const double *D, const double *lambda,
                            const biofvm_boundary *bc, biofvm_precision prec,
                            uintptr_t cuda_stream, biofvm_t **out);

/* Copy the whole field in.  src: nx*ny*nz*n_sub elements of the handle's
 * element type in the layout above; a host pointer (src_on_device = 0) or a
 * device pointer (1).  Async with respect to the host for device sources;
 * a host source is fully read before return.  Errors: ARG, CUDA. */
biofvm_status biofvm_set_density(biofvm_t *h, const void *src,
                                 int src_on_device);

/* Replace the agents (cell sources/sinks, Sect. 5.3).  n >= 0 agents; agent
 * k sits in voxel voxel[k] = (z*ny + y)*nx + x and has, per substrate s,
 * secretion rate secretion[k*n_sub+s] >= 0 toward target density
 * target[k*n_sub+s], uptake rate uptake[k*n_sub+s] >= 0, and volume weight
 * weight[k] >= 0 (cell volume / voxel volume; NULL means 1).  secretion,
 * target and uptake may each be NULL (= 0).  All arrays are host arrays.
 * Agents sharing a voxel are aggregated on the host into one (alpha, beta)
 * pair per (voxel, substrate), which makes the update independent of the
 * order of the agents.  Not timed as part of a step.
 * Errors: ARG (voxel out of range, negative rates or weights), OOM, CUDA. */
biofvm_status biofvm_set_sources(biofvm_t *h, int64_t n, const int64_t *voxel,
                                 const double *secretion, const double *target,
                                 const double *uptake, const double *weight);

/* Moving agents (the end-to-end run of Sect. 5.3 moves its cells between
 * steps): reserve device buffers for up to n_max >= 0 agents, so that
 * biofvm_set_sources_device can rebuild the source lists on the device without
 * allocating.  Waits for the stream.  If device-built lists were in use they
 * are replaced by an empty agent set.  Not for batched environments (STATE).
 * Errors: ARG (n_max * n_sub must stay below 2^32), OOM, CUDA, STATE. */
biofvm_status biofvm_reserve_agents(biofvm_t *h, int64_t n_max);

/* Replace the agents from DEVICE arrays, entirely on the handle's stream
 * (async: no host synchronisation, no allocation; a graph may capture it).
 * Same arrays and meaning as biofvm_set_sources (voxel[n] int64;
 * secretion, target, uptake [n*n_sub] double, each may be NULL = 0; weight[n]
 * double, NULL = 1), which must stay valid until the stream has run the call.
 * 0 <= n <= the reserved n_max.  The per-(voxel, substrate) entries are formed,
 * sorted by element (a stable radix sort) and summed in agent order on the
 * device: the same lists, to the bit, as biofvm_set_sources builds on the host.
 * Entries on Dirichlet nodes are left out (the nodes current at this call).
 * An invalid agent (voxel out of range, a negative or non-finite rate or
 * weight) is left out and makes the next synchronising call return ARG.
 * While device-built lists are in use biofvm_adjoint_step returns STATE.
 * Errors: ARG, CUDA, STATE (nothing reserved, or a batched environment). */
biofvm_status biofvm_set_sources_device(biofvm_t *h, int64_t n, const int64_t *voxel,
                                        const double *secretion, const double *target,
                                        const double *uptake, const double *weight);

/* Advance n_steps >= 0 time steps (async).  Steps run as CUDA graphs captured
 * on first use (after create or a parameter change): a block of K steps
 * (K = 1; with the FP64 streaming sweeps up to 16, the steps between which the
 * field may stay divided by a per-substrate constant) and shorter tails; the
 * field is the true one whenever the call's steps are done.  Errors: ARG,
 * CUDA, TIMEOUT (reported by the next synchronising call). */
biofvm_status biofvm_step(biofvm_t *h, int n_steps);

/* Copy the field out into dst (host pointer if dst_on_device = 0, device
 * pointer if 1), same layout and type as biofvm_set_density.  Waits for the
 * stream, then checks the device status word.  Errors: ARG, CUDA, TIMEOUT. */
biofvm_status biofvm_density(biofvm_t *h, void *dst, int dst_on_device);

/* Replace D[n_sub] and lambda[n_sub] (host) and recompute the App. A
 * constants (used by finite-difference checks).  Errors: ARG, CUDA. */
biofvm_status biofvm_set_params(biofvm_t *h, const double *D,
                                const double *lambda);

/* Anisotropic grid: set the voxel spacing along x, y and z (um) and recompute
 * the App. A constants, each axis taking r = D dt / h^2 with its own h.  The
 * paper's grids are isotropic (biofvm_create's dx on all three axes); this is
 * an extension.  The adjoint's D gradient follows (per-axis dt / h^2).
 * Errors: ARG (a spacing not finite and > 0; nothing changed), CUDA. */
biofvm_status biofvm_set_spacing(biofvm_t *h, double dx, double dy, double dz);

/* Dirichlet nodes: voxels anywhere in the grid held at a value, and faces
 * whose values differ (give the face voxels as nodes).  Each of the four
 * Dirichlet applications of a step (Sect. 2: before the x-solve and after each
 * solve) overwrites the flagged faces of biofvm_boundary and then every node
 * (voxel[k], substrate[k]) with value[k]; a (voxel, substrate) listed more
 * than once takes its last value, and a node wins over a flagged face.  n >= 0
 * nodes (0 removes them); voxel[k] in [0, nx*ny*nz), substrate[k] in
 * [0, n_sub), value[k] finite; host arrays, copied.  The agents' source
 * entries on node elements are dropped (the node overwrites them anyway), and
 * the adjoint zeroes its gradient at the nodes at each application.  Not
 * supported in batched environments (biofvm_batch_step then fails with ARG).
 * Errors: ARG (nothing changed), OOM, CUDA. */
biofvm_status biofvm_set_dirichlet_nodes(biofvm_t *h, int64_t n, const int64_t *voxel,
                                         const int32_t *substrate, const double *value);

/* Run exactly one stage of the step in place, for stage-by-stage checks:
 * stage 0 = Src then B, 1 = X^-1 then B, 2 = Y^-1 then B, 3 = Z^-1 then B,
 * 4 = the source update alone (no Dirichlet), 5 = X^-1 alone, 6 = Y^-1
 * alone, 7 = Z^-1 alone, 8 = Src, B, X^-1, B in one launch (the first kernel
 * of a step; with stages 2 and 3 it makes one whole step).  Stages 9, 10, 11
 * are the three kernels of biofvm_step itself, launched one by one (for
 * timing each): in FP64 the step's x- and y-sweeps leave the field divided
 * by a per-substrate constant that the z-sweep takes out again, so only the
 * sequence 9, 10, 11 as a whole is a step (equal to stages 8, 2, 3 up to
 * rounding).  Stage 12 is the z-sweep as it runs inside a block of FP64
 * steps: it leaves the field divided by that constant (biofvm_step brings
 * the field back every 16 steps or fewer, and always before it returns);
 * without the FP64 streaming sweeps it equals stage 11.  Async.  Errors: ARG,
 * CUDA. */
biofvm_status biofvm_run_stage(biofvm_t *h, int stage);

/* One time step, like biofvm_step(h, 1), that also writes the forward states
 * the adjoint of that step needs into `saved` (device, 4*nx*ny*nz*n_sub
 * elements of the handle's type, layout [4][field]): [0] the source output
 * (before its Dirichlet application), [1] the X^-1 output, [2] the Y^-1
 * output, [3] the Z^-1 output (each before the B that follows it).  Async.
 * Errors: ARG, CUDA. */
biofvm_status biofvm_step_save(biofvm_t *h, void *saved);

/* Reverse mode of one step (the stages of Sect. 2 transposed; each 1D matrix
 * of App. A is symmetric, so the adjoint sweeps are the forward sweeps run in
 * the order Z, Y, X).  grad_out: adjoint of the step's output; grad_in:
 * receives the adjoint of the step's input (may equal grad_out); saved: the
 * states biofvm_step_save wrote for this step.  All three are device arrays
 * in the field layout and type.  ACCUMULATES (+=) into device FP64 arrays:
 * dD[n_sub], dlambda[n_sub] (reduced in a fixed order: bit-reproducible), and,
 * if dsecretion is not NULL, dsecretion[n_agents*n_sub], the gradient with
 * respect to each agent's secretion rate (agents as last passed to
 * biofvm_set_sources).  The first call allocates the adjoint field and a
 * small reduction buffer.  Async.  Errors: ARG, OOM, CUDA. */
biofvm_status biofvm_adjoint_step(biofvm_t *h, const void *grad_out, void *grad_in, double *dD,
                                  double *dlambda, double *dsecretion, const void *saved);

/* biofvm_adjoint_step that also ACCUMULATES, if duptake is not NULL, the
 * gradient with respect to each agent's uptake rate into the device FP64 array
 * duptake[n_agents*n_sub] (Sect. 5.3 sinks; in the source update
 * rho <- (rho + alpha)/(1 + beta) an uptake rate U_k enters beta only, so
 * d rho'/d U_k = -dt w_k rho' / (1 + beta)).  biofvm_adjoint_step is this call
 * with duptake = NULL.  Errors: as biofvm_adjoint_step. */
biofvm_status biofvm_adjoint_step_rates(biofvm_t *h, const void *grad_out, void *grad_in,
                                        double *dD, double *dlambda, double *dsecretion,
                                        double *duptake, const void *saved);

/* Wait for the handle's stream and check the device status word.
 * Errors: CUDA, TIMEOUT. */
biofvm_status biofvm_sync(biofvm_t *h);

/* Device address of the handle's field (owned by the library, valid until
 * destroy), for zero-copy interop with a framework's device tensors.
 * Errors: ARG. */
biofvm_status biofvm_density_ptr(biofvm_t *h, void **dev_ptr);

/* Number of kernel launches one time step makes: 3 (x-, y-, z-sweep), plus 4
 * (one Dirichlet-node launch around each sweep) while Dirichlet nodes are set;
 * 1 for the cooperative small-grid step.  A call on a row-padded copy (see
 * biofvm_describe) adds two copy launches per call, not per step. */
int biofvm_launches_per_step(const biofvm_t *h);

/* Which kernels biofvm_step runs for this handle, as a NUL-terminated ASCII
 * line written to the host buffer out[len]: "cooperative" (small FP64 grids:
 * all steps of a call in one launch), or "x=K y=K z=K" with K one of stream
 * (whole-line streaming sweep), pipe (TMA-pipelined tiles, followed by
 * "/cwC/mM": C lines per tile, chunks of M positions) or plain (register-chunk
 * kernels), then " scaled" when the FP64 steps carry the renormalisation
 * factor, " pitched" when the steps run on a row-padded copy of the field (an
 * FP32 field whose rows of nx*n_sub elements are not 16-byte multiples,
 * copied in and back once per call), " nodes" while Dirichlet nodes are set.
 * Diagnostic only; the text may change between versions.  Errors: ARG (NULL
 * handle or buffer, or len too small for the line; out then holds a
 * truncated line if len > 0). */
biofvm_status biofvm_describe(const biofvm_t *h, char *out, size_t len);

/* Measure the FMA issue rate of the current device in FP64 (prec =
 * BIOFVM_FP64) or FP32 (BIOFVM_FP32): the arithmetic roof of the Thomas
 * recurrences (Sect. 2.1, Eq. 2: an axpy and a division forward, an axpy
 * backward per position; the sweeps issue them as FMAs).  Runs a kernel of
 * independent FMA chains over the whole device on cuda_stream for about
 * 0.1 s and writes the best of three CUDA-event timings, in FMA/s, to
 * *fma_per_second (host).  Waits for the stream.  Allocates no device
 * memory.  Errors: ARG, CUDA. */
biofvm_status biofvm_probe_fma_rate(biofvm_precision prec, uintptr_t cuda_stream,
                                    double *fma_per_second);

/* ------------------------------------------------------------------------
 * Batched microenvironments: many independent grids of uneven size and
 * substrate count, advanced together.  Two modes, fixed at create:
 *   persistent (mode 0): ONE persistent kernel launch per biofvm_batch_step
 *     call (all environments, all steps; captured in a CUDA graph), for many
 *     small environments;
 *   per-environment graph (mode 1): each environment runs the single-grid
 *     sweeps (pipelined or streaming, as biofvm_step would), and a batch step
 *     is ONE CUDA graph of every environment's three sweep launches on
 *     parallel branches, launched once per step -- for environments large
 *     enough to fill the GPU in a few concurrent launches.
 * The mode is taken from the environment variable BIOFVM_BATCH_MODE (graph or
 * persistent) if set, else mode 1 when the mean environment holds at least
 * 2^20 voxel-substrates.  The persistent kernel's CTAs claim work items in
 * order from a counter (BIOFVM_BATCH_DYNAMIC=0: a static stride instead) and
 * fill every SM with as many CTAs as fit (BIOFVM_BATCH_CTAS caps the CTAs per
 * SM); the results do not depend on either.  Each environment is an ordinary handle (zero-flux
 * boundaries) reachable through biofvm_batch_env, so biofvm_set_density,
 * biofvm_set_sources, biofvm_density (and even biofvm_step) work on it.
 * ---------------------------------------------------------------------- */
typedef struct biofvm_batch biofvm_batch_t;

/* Create n_env >= 1 environments: grids[e] (host), dx[e], dt[e], and
 * D_flat / lambda_flat holding the n_sub of environment 0, then of
 * environment 1, ... (host).  tile_m (persistent mode only; ignored in the
 * per-environment mode): NULL or [n_env][3] tile shapes along
 * x, y, z per environment -- the shapes an autotuner chooses: a value >= the
 * axis length solves whole lines (one warp streams 32 lines, no chunks; FP32
 * then allocates a scratch of one [n][32] tile per 32-line tile of the
 * largest sweep, about the field's size); a smaller value
 * is the chunk length of the partitioned solve (at most 8 chunks of at most
 * 48 positions); <= 0 picks a default (whole lines, except chunks along x
 * when n_sub <= 2).  All environments share `prec` and the stream.
 * Errors: ARG, OOM, CUDA (with the failing environment in the message). */
biofvm_status biofvm_batch_create(int n_env, const biofvm_grid *grids, const double *dx,
                                  const double *dt, const double *D_flat,
                                  const double *lambda_flat, biofvm_precision prec,
                                  uintptr_t cuda_stream, const int *tile_m,
                                  biofvm_batch_t **out);

/* The handle of environment e (owned by the batch; do not destroy it). */
biofvm_status biofvm_batch_env(biofvm_batch_t *b, int e, biofvm_t **env);

/* Advance every environment n_steps >= 0 steps (async).  Persistent mode:
 * one launch; work items (step, sweep, environment, tile of 32 lines) are
 * spread over a resident grid; each waits, with a bounded spin, for the
 * previous sweep of its own environment.  Per-environment mode: n_steps
 * launches of the one-step graph (captured at the first call and whenever an
 * environment's sources or constants change), plus, for environments whose
 * rows are no 16-byte multiple, one copy into and out of their row-padded
 * copies per call.  Errors: ARG (Dirichlet nodes set on an environment), CUDA;
 * a timed-out wait is reported by biofvm_batch_sync as TIMEOUT. */
biofvm_status biofvm_batch_step(biofvm_batch_t *b, int n_steps);

/* Wait for the batch's stream and check its status word (per-environment
 * mode: every environment's).  Errors: CUDA, TIMEOUT. */
biofvm_status biofvm_batch_sync(biofvm_batch_t *b);

/* Change the tile shapes (same rules as tile_m of biofvm_batch_create) of
 * every environment without touching the fields or agents: re-partitions the
 * App. A constants.  Used by the autotuner.  Waits for the stream.  Errors:
 * ARG (nothing changed), OOM (scratch), CUDA, STATE (per-environment mode). */
biofvm_status biofvm_batch_set_tiles(biofvm_batch_t *b, const int *tile_m);

/* CTAs of the persistent batched launch (resident at once); 0 in the
 * per-environment mode. */
int biofvm_batch_grid(const biofvm_batch_t *b);

/* The batch's mode: 0 persistent kernel, 1 per-environment graph; -1 for a
 * NULL handle. */
int biofvm_batch_mode(const biofvm_batch_t *b);

/* Failure-detection test hook (persistent mode; STATE in the per-environment
 * mode): with on != 0, every following batched launch
 * makes the first y-sweep tile of environment 0 wait for a completion count
 * that never comes.  Its bounded wait gives up after about two seconds, the
 * kernel sets the status word and every CTA stops at its next item (results
 * of that launch are undefined); biofvm_batch_sync then returns TIMEOUT and
 * the context stays usable.  on = 0 restores normal launches.  No GPU fault
 * or hang is involved.  Errors: ARG. */
biofvm_status biofvm_batch_test_stall(biofvm_batch_t *b, int on);

/* Free the batch and every environment (waits for the stream). */
void biofvm_batch_destroy(biofvm_batch_t *b);

/* ------------------------------------------------------------------------
 * Allocation-free variant of the adjoint's parameter-gradient reduction.
 * The paper has no counterpart: it serves callers that cannot call
 * cudaMalloc -- code inside a host framework that owns all device memory
 * through its own pool or arena, processes under a fixed device-memory
 * budget, or loops where allocating is not allowed.
 *
 * For one sweep with adjoint field mu and forward sweep output u (device
 * arrays, the field layout, double for BIOFVM_FP64 or float for BIOFVM_FP32)
 * along `axis` (0 = x, 1 = y, 2 = z) of an nx x ny x nz grid of n_sub
 * substrates, ACCUMULATES into device doubles
 *     dlambda[s] += -(dt/3)        * sum_elements(s) mu * u
 *     dD[s]      += -(dt/h_axis^2) * sum_lines(s) sum_i (mu_{i+1}-mu_i)(u_{i+1}-u_i)
 * where h_axis is the voxel spacing along `axis` (biofvm_create's dx on an
 * isotropic grid; the dx, dy or dz of biofvm_set_spacing on an anisotropic
 * one), on cuda_stream (async).  These are the sums biofvm_adjoint_step
 * forms for each of its three sweeps, but split over a different number of
 * blocks, so the two agree to rounding (summation order), not bit for bit.
 * It calls no allocator: its per-block partial sums live in one file-scope
 * device array of 256 KB (512 blocks x 2 sums x 32 substrates, FP64) that
 * every GPU loading the library holds until the process exits.  Every call
 * overwrites all the partials it reads, so nothing carries over from the
 * previous call; calls whose kernels overlap on the GPU (other streams, other
 * host threads) race on that array.  The first call on each device, and the
 * first in each new CUDA context of a device, looks the array's address up
 * (cudaGetSymbolAddress): make that first call before any stream capture.
 * Limits: 1 <= n_sub <= 32 (larger is rejected with BIOFVM_ERR_ARG).
 * Errors: ARG, CUDA. */
biofvm_status biofvm_param_grad_noalloc(const void *mu, const void *u, int nx, int ny, int nz,
                                        int n_sub, int axis, biofvm_precision prec, double dt,
                                        double h_axis, double *dD, double *dlambda,
                                        uintptr_t cuda_stream);

/* Free the handle and all device memory it owns (waits for its stream).
 * NULL is a no-op. */
void biofvm_destroy(biofvm_t *h);

/* Message of the last failed call on this thread ("" if none). */
const char *biofvm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* BIOFVM_H */
