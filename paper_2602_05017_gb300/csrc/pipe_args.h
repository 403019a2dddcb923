// Arguments of the persistent TMA-pipelined sweep kernel (pipe.cuh).
#pragma once
#include <stdint.h>

#include "internal.h"

namespace bfv {

// A tile is cw "columns" (independent lines) x n positions along the axis,
// cw = 32, or 16 for lines too long for two stages of 32 columns.
//
// The field's rows (fixed y, z: rowlen = nx*S elements) start gpitch elements
// apart in global memory: gpitch = rowlen, or rowlen rounded up to 16 bytes for
// a row-padded copy of a field whose rows are not 16-byte multiples (TMA copies
// need 16-byte aligned rows); the padding elements are carried along untouched.
//
//   mode 0 (x-sweep): a column is one (row, substrate) pair of
//     rows_per_tile = floor(cw/S) consecutive rows (y, z); the rows (gpitch
//     elements each) are staged with one cp.async.bulk each, issued by the
//     lanes of the producer warp, into shared memory at a padded `pitch`
//     (elements) chosen on the host so that the lanes of a warp hit different
//     banks; element (column c, position x) sits at (c/S)*pitch + x*S + c%S.
//   mode 1 / 2 (y- / z-sweep): a column is one of cw consecutive (x, s)
//     entries of a row (mode 1) or entries of a plane, C = ny*gpitch
//     including any padding (mode 2); the tile [n][cw] is staged with
//     cp.async.bulk.tensor boxes of box_rows x cw; element (c, j) sits at
//     j*cw + c.
//
// Tile k of a CTA is tile blockIdx.x + k*gridDim.x of ntiles.
struct PipeArgs {
  int mode, n, S, nx, ny, nz;
  int cw;  // columns per tile: 32 or 16
  int64_t ntiles;
  // mode 1 / 2
  int64_t C;
  int tiles_per_plane, nplanes, box_rows, nbox;
  // mode 0
  int rows_per_tile, rowlen, pitch;
  int gpitch;  // elements between consecutive rows of the field (rowlen, or padded)
  int64_t nrows;
  void *field;
  // ring of stages
  int stages;
  int64_t stage_elems;
  AxisTab tab;
  int flags;
  // mode 0: sources (CSR over rows) and the Dirichlet application before the solve
  const int64_t *src_row_off, *src_elem;
  const int2 *src_rowcol;  // (row, position in the row) of each entry
  const void *src_alpha, *src_scale;
  int has_src;
  int prep_warp;  // mode 0: a warp of its own applies Src and B before the solve (1) or none (0)
  const uint8_t *dir_on;
  const void *dir_val;
  int *status;
};

}  // namespace bfv
