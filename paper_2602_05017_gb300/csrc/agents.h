// Device-side rebuild of the source lists (agents.cu): the descriptor the host
// fills from a handle's reserved buffers, and the launcher.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace bfv {

// Status word value of a device agent array holding an invalid agent (voxel out
// of range, a negative or non-finite rate or weight); that agent is dropped.
constexpr int kStatusBadInput = 1;

struct AgentBuild {
  // inputs (device): voxel[n], secretion/target/uptake[n*S] (NULL: 0), weight[n] (NULL: 1)
  const int64_t *voxel;
  const double *secretion, *target, *uptake, *weight;
  long long n_entries_max;  // n * S
  int S;
  int64_t nvox, rowlen, nrows;
  double dt;
  uint64_t sentinel;  // key of a dropped entry: the element count (above every element)
  const int64_t *node_elem;  // sorted elements of the Dirichlet nodes the kernels apply
  int64_t n_nodes;
  // work buffers [n_entries_max] (two of key and idx: the sort ping-pongs)
  uint64_t *key[2];
  uint32_t *idx[2];
  double *ea, *eb;       // alpha, beta of each entry, by entry index
  uint32_t *head, *pos;  // run heads and their exclusive scan
  uint32_t *hist;        // [256][sort blocks]
  uint32_t *part;        // scan block sums
  uint32_t *count32;
  // outputs: the handle's source lists (capacity n_entries_max) and their length
  int64_t *src_elem;
  void *src_alpha, *src_scale;  // field type
  int2 *src_rowcol;
  int64_t *src_row_off;  // [nrows + 1]
  int64_t *count;
  int *status;
};

// Passes of 8 bits that cover every key up to `sentinel`.
int radix_passes(uint64_t sentinel);
// Tiles of the sort and of the scan for n entries (to size hist and part).
long long agent_sort_blocks(long long n);
long long agent_scan_blocks(long long n);
// Enqueue the rebuild on `st` (no synchronisation, no allocation).
cudaError_t build_sources_device(AgentBuild b, bool fp64, cudaStream_t st);

}  // namespace bfv
