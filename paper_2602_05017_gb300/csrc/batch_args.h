// Descriptors of the batched persistent step (batch.cuh), shared with the host.
#pragma once
#include <stdint.h>

#include "internal.h"

namespace bfv {

// One environment: its field, per-axis constants (the same blocks and chunk
// partition as its single-grid handle) and its aggregated sources.
struct BatchEnv {
  void *field;
  int nx, ny, nz, S;
  const void *tab[3];  // per axis: inv, mul, pf, pb [n][S]; pc [T][S]; cfix [2][S]
  int T[3], m[3];
  int rows_per_tile;    // x tiles: floor(32/S) rows of S lines each
  int64_t tiles[3];     // tiles per phase
  int group[3];         // tiles solved together by one work item: floor(8 / T) warp groups
  int64_t items[3];     // work items per phase = ceil(tiles / group)
  const int64_t *src_row_off, *src_elem;
  const void *src_alpha, *src_scale;
  int has_src;
  // whole-line axes (tile shape m >= n): streaming solve, one warp per tile
  // (stream.cuh), coefficients position-major [n][S] (FP64: inv, mul, q;
  // FP32: inv', mul of the defect form), interior constants [2][S] from
  // position k0 on, FP32 c_hi/c_lo and a scratch of one [n][32] tile per
  // whole-line tile (batch_scratch_elems)
  int whole[3];
  const void *stab[3], *sint[3], *cfix[3];
  int k0[3];
  void *scratch;
};

struct BatchArgs {
  const BatchEnv *env;
  int n_env, n_steps;
  int maxm;                 // longest chunk of any environment (shared-memory chunk rows)
  const int64_t *tile_off;  // [3][n_env + 1] prefix sums of work items per phase
  int64_t per_step;         // work items of one step
  unsigned int *done;       // [3][n_env] completed work items (cumulative over steps)
  int *abort_flag, *status;
  unsigned long long *next;  // claim counter (zero at launch), or NULL: static round robin
  int stall_test;           // test hook: the first y tile of environment 0 waits for a count
                            // that never comes, so its bounded wait expires
};

}  // namespace bfv
