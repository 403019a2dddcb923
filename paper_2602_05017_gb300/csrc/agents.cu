// Device-side rebuild of the source lists from agent arrays in device memory,
// for agents that move between steps (the end-to-end run of Sect. 5.3 moves
// its cells; the source/uptake update applies them before every step).
//
// The lists are the ones biofvm_set_sources builds on the host: one entry per
// (voxel, substrate) that some agent touches, holding
//   alpha = sum_k dt w_k S_k rho*_k   and   scale = 1 / (1 + sum_k dt w_k (S_k + U_k))
// over the agents k in that voxel, sorted by element, with CSR offsets per
// x-row and (row, position) pairs for the pipelined x tiles.  Elements of
// Dirichlet nodes and entries with alpha = beta = 0 are left out.
//
// Steps, all stream-ordered kernels (no host synchronisation, no allocation:
// every buffer is reserved beforehand, see AgentBuffers):
//   1. entries: per (agent, substrate) its element key, alpha and beta, or a
//      sentinel key (dropped: zero entry, node element, invalid agent -- an
//      invalid agent also sets the status word);
//   2. a stable LSD radix sort of (key, entry index) by key, 8 bits per pass
//      (histogram per 2048-entry tile, one exclusive scan of the digit-major
//      histograms, a scatter that ranks equal digits in entry order);
//   3. run heads, an exclusive scan of them, and one thread per run summing its
//      alpha and beta in entry order -- the host builder's order, so the two
//      give the same bits;
//   4. row offsets by a binary search per row.
// Up to kSmallBuild entries (n agents x S substrates) take one CTA instead --
// entries in shared memory, a bitonic sort of (element, entry index) pairs
// (unique, so the order is the radix sort's), block scans, the same sums --
// and one more launch for the row offsets: two launches instead of about
// thirty, which at a thousand agents are mostly launch time.
#include <cuda_runtime.h>
#include <stdint.h>

#include "agents.h"

namespace bfv {

namespace {

constexpr int kSortThreads = 256;  // one digit per thread in the per-digit loops
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;
constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------------------
// Exclusive scan of uint32 counts (totals stay below 2^32: entry counts).
// ---------------------------------------------------------------------------
// Block-wide exclusive scan of one value per thread (1024 threads); *total gets
// the block's sum.
__device__ __forceinline__ uint32_t block_scan_1024(uint32_t v, uint32_t *total) {
  __shared__ uint32_t warp_sum[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) warp_sum[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t s = warp_sum[lane];
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, s, d);
      if (lane >= d) s += y;
    }
    warp_sum[lane] = s;  // inclusive over warps
  }
  __syncthreads();
  const uint32_t before = warp == 0 ? 0u : warp_sum[warp - 1];
  *total = warp_sum[31];
  __syncthreads();  // warp_sum is reused by the next call
  return before + x - v;
}

__global__ void __launch_bounds__(kScanThreads)
    scan_reduce_kernel(const uint32_t *__restrict__ in, long long L, uint32_t *__restrict__ part) {
  const long long i0 = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; k++)
    if (i0 + k < L) s += in[i0 + k];
  uint32_t total;
  block_scan_1024(s, &total);
  if (threadIdx.x == 0) part[blockIdx.x] = total;
}

// One block: exclusive scan of the nb block sums in place; *total = their sum.
__global__ void __launch_bounds__(kScanThreads)
    scan_parts_kernel(uint32_t *__restrict__ part, int nb, uint32_t *__restrict__ total) {
  uint32_t carry = 0;
  for (int b0 = 0; b0 < nb; b0 += kScanThreads) {
    const int b = b0 + threadIdx.x;
    const uint32_t v = b < nb ? part[b] : 0u;
    uint32_t t;
    const uint32_t ex = block_scan_1024(v, &t);
    if (b < nb) part[b] = carry + ex;
    carry += t;
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void __launch_bounds__(kScanThreads)
    scan_apply_kernel(const uint32_t *__restrict__ in, long long L,
                      const uint32_t *__restrict__ part, uint32_t *__restrict__ out) {
  const long long i0 = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
  uint32_t v[kScanItems], s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; k++) {
    v[k] = i0 + k < L ? in[i0 + k] : 0u;
    s += v[k];
  }
  uint32_t total;
  uint32_t run = part[blockIdx.x] + block_scan_1024(s, &total);
#pragma unroll
  for (int k = 0; k < kScanItems; k++) {
    if (i0 + k < L) out[i0 + k] = run;
    run += v[k];
  }
}

cudaError_t exclusive_scan(const uint32_t *in, uint32_t *out, long long L, uint32_t *part,
                           uint32_t *total, cudaStream_t st) {
  const int nb = (int)((L + kScanTile - 1) / kScanTile);
  if (nb < 1) return cudaSuccess;
  scan_reduce_kernel<<<nb, kScanThreads, 0, st>>>(in, L, part);
  scan_parts_kernel<<<1, kScanThreads, 0, st>>>(part, nb, total);
  scan_apply_kernel<<<nb, kScanThreads, 0, st>>>(in, L, part, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// 1. Entries.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool sorted_contains(const int64_t *a, int64_t n, int64_t key) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (a[mid] < key) lo = mid + 1; else hi = mid;
  }
  return lo < n && a[lo] == key;
}

__global__ void agent_entries_kernel(AgentBuild b) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= b.n_entries_max) return;
  const long long k = i / b.S;
  const int s = (int)(i - k * b.S);
  uint64_t key = b.sentinel;
  double alpha = 0.0, beta = 0.0;
  const int64_t v = b.voxel[k];
  const double sv = b.secretion ? b.secretion[i] : 0.0;
  const double uv = b.uptake ? b.uptake[i] : 0.0;
  const double tv = b.target ? b.target[i] : 0.0;
  const double w = b.weight ? b.weight[k] : 1.0;
  const bool valid = v >= 0 && v < b.nvox && sv >= 0.0 && uv >= 0.0 && w >= 0.0 &&
                     isfinite(sv) && isfinite(uv) && isfinite(tv) && isfinite(w);
  if (!valid) {
    atomicCAS(b.status, 0, kStatusBadInput);
  } else {
    // the host builder's expressions, without contraction
    const double dtw = __dmul_rn(b.dt, w);
    alpha = __dmul_rn(__dmul_rn(dtw, sv), tv);
    beta = __dmul_rn(dtw, __dadd_rn(sv, uv));
    const int64_t e = v * b.S + s;
    if ((alpha != 0.0 || beta != 0.0) && !sorted_contains(b.node_elem, b.n_nodes, e))
      key = (uint64_t)e;
  }
  b.key[0][i] = key;
  b.idx[0][i] = (uint32_t)i;
  b.ea[i] = alpha;
  b.eb[i] = beta;
}

// ---------------------------------------------------------------------------
// 2. Stable LSD radix sort, 8 bits per pass.  A tile of 2048 entries is read
// striped (entry tile0 + j*256 + thread), so (slot, thread) order is entry
// order.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kSortThreads)
    radix_hist_kernel(const uint64_t *__restrict__ key, long long N, int shift,
                      uint32_t *__restrict__ hist, int nb) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const long long tile0 = (long long)blockIdx.x * kSortTile;
#pragma unroll
  for (int j = 0; j < kSortItems; j++) {
    const long long i = tile0 + (long long)j * kSortThreads + threadIdx.x;
    if (i < N) atomicAdd(&h[(uint32_t)(key[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[(long long)threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];  // digit-major
}

// offs: the exclusive scan of the digit-major histograms: the first output slot
// of digit d for this block.  Entries of equal digit keep their order: within a
// slot, lanes of lower warps and lower lanes come first (warp counts in shared
// memory, __match_any_sync inside a warp); slots go in order.
__global__ void __launch_bounds__(kSortThreads)
    radix_scatter_kernel(const uint64_t *__restrict__ key_in, const uint32_t *__restrict__ idx_in,
                         long long N, int shift, const uint32_t *__restrict__ offs, int nb,
                         uint64_t *__restrict__ key_out, uint32_t *__restrict__ idx_out) {
  constexpr int kWarps = kSortThreads / 32;
  __shared__ uint32_t base[256];          // next output slot of each digit
  __shared__ uint32_t wcnt[kWarps][256];  // this slot's digit counts per warp
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  base[tid] = offs[(long long)tid * nb + blockIdx.x];
#pragma unroll
  for (int w = 0; w < kWarps; w++) wcnt[w][tid] = 0;
  __syncthreads();
  const long long tile0 = (long long)blockIdx.x * kSortTile;
  for (int j = 0; j < kSortItems; j++) {
    const long long i = tile0 + (long long)j * kSortThreads + tid;
    const bool ok = i < N;
    const uint64_t k = ok ? key_in[i] : 0;
    const uint32_t v = ok ? idx_in[i] : 0;
    const uint32_t d = (uint32_t)(k >> shift) & 255u;
    const unsigned valid = __ballot_sync(kFull, ok);
    const unsigned peers = __match_any_sync(kFull, ok ? d : 0xffffffffu) & valid;
    if (ok && lane == __ffs(peers) - 1) wcnt[warp][d] = __popc(peers);
    __syncthreads();
    if (ok) {
      uint32_t r = base[d] + __popc(peers & ((1u << lane) - 1u));
      for (int w = 0; w < warp; w++) r += wcnt[w][d];
      key_out[r] = k;
      idx_out[r] = v;
    }
    __syncthreads();
    uint32_t sum = 0;
#pragma unroll
    for (int w = 0; w < kWarps; w++) {
      sum += wcnt[w][tid];
      wcnt[w][tid] = 0;
    }
    base[tid] += sum;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// 3. Runs of equal keys: heads, their scan, and the sums.
// ---------------------------------------------------------------------------
__global__ void run_heads_kernel(const uint64_t *__restrict__ key, long long N, uint64_t sentinel,
                                 uint32_t *__restrict__ head) {
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  const uint64_t k = key[j];
  head[j] = (k != sentinel && (j == 0 || key[j - 1] != k)) ? 1u : 0u;
}

template <typename E>
__global__ void run_sums_kernel(AgentBuild b, const uint64_t *__restrict__ key,
                                const uint32_t *__restrict__ idx, long long N) {
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N || !b.head[j]) return;
  const uint64_t e = key[j];
  double a = 0.0, be = 0.0;
  for (long long t = j; t < N && key[t] == e; t++) {  // entry order within the run
    const uint32_t q = idx[t];
    a = t == j ? b.ea[q] : __dadd_rn(a, b.ea[q]);
    be = t == j ? b.eb[q] : __dadd_rn(be, b.eb[q]);
  }
  const uint32_t o = b.pos[j];
  b.src_elem[o] = (int64_t)e;
  static_cast<E *>(b.src_alpha)[o] = (E)a;
  static_cast<E *>(b.src_scale)[o] = (E)__ddiv_rn(1.0, __dadd_rn(1.0, be));
  b.src_rowcol[o] = make_int2((int)((int64_t)e / b.rowlen), (int)((int64_t)e % b.rowlen));
}

// ---------------------------------------------------------------------------
// 4. Row offsets: row_off[r] = first entry with element >= r * rowlen.
// ---------------------------------------------------------------------------
__global__ void row_offsets_kernel(AgentBuild b) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r > b.nrows) return;
  const int64_t key = r * b.rowlen;
  int64_t lo = 0, hi = *b.count;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (b.src_elem[mid] < key) lo = mid + 1; else hi = mid;
  }
  b.src_row_off[r] = lo;
}

__global__ void count_to_i64_kernel(const uint32_t *__restrict__ c, int64_t *__restrict__ out) {
  *out = (int64_t)*c;
}

// ---------------------------------------------------------------------------
// One-CTA rebuild for up to kSmallBuild entries.
// ---------------------------------------------------------------------------
constexpr int kSmallBuild = 2048;  // entries: 32 KB of static shared memory
constexpr int kSmallBuildThreads = 1024;

// Entry of agent k, substrate s (i = k*S + s): its key, alpha, beta (the first
// step of the multi-CTA path, one entry).
__device__ __forceinline__ uint64_t entry_of(const AgentBuild &b, long long i, double &alpha,
                                             double &beta) {
  const long long k = i / b.S;
  const int s = (int)(i - k * b.S);
  alpha = beta = 0.0;
  const int64_t v = b.voxel[k];
  const double sv = b.secretion ? b.secretion[i] : 0.0;
  const double uv = b.uptake ? b.uptake[i] : 0.0;
  const double tv = b.target ? b.target[i] : 0.0;
  const double w = b.weight ? b.weight[k] : 1.0;
  const bool valid = v >= 0 && v < b.nvox && sv >= 0.0 && uv >= 0.0 && w >= 0.0 &&
                     isfinite(sv) && isfinite(uv) && isfinite(tv) && isfinite(w);
  if (!valid) {
    atomicCAS(b.status, 0, kStatusBadInput);
    return b.sentinel;
  }
  const double dtw = __dmul_rn(b.dt, w);
  alpha = __dmul_rn(__dmul_rn(dtw, sv), tv);
  beta = __dmul_rn(dtw, __dadd_rn(sv, uv));
  const int64_t e = v * b.S + s;
  if ((alpha != 0.0 || beta != 0.0) && !sorted_contains(b.node_elem, b.n_nodes, e))
    return (uint64_t)e;
  return b.sentinel;
}

template <typename E>
__global__ void __launch_bounds__(kSmallBuildThreads) small_build_kernel(AgentBuild b) {
  __shared__ uint64_t key[kSmallBuild];
  __shared__ uint32_t idx[kSmallBuild];
  __shared__ uint32_t pos[kSmallBuild];
  __shared__ uint32_t warp_tot[32];
  const int N = (int)b.n_entries_max;
  int P = 1;
  while (P < N) P <<= 1;
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    if (i < N) {
      double al, be;
      key[i] = entry_of(b, i, al, be);
      b.ea[i] = al;
      b.eb[i] = be;
    } else {
      key[i] = ~0ull;  // padding sorts last
    }
    idx[i] = (uint32_t)i;
  }
  __syncthreads();
  // bitonic sort of (key, idx) -- distinct pairs, so the result is unique
  for (int k = 2; k <= P; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int l = i ^ j;
        if (l > i) {
          const bool up = (i & k) == 0;
          const bool gt = key[i] > key[l] || (key[i] == key[l] && idx[i] > idx[l]);
          if (gt == up) {
            const uint64_t tk = key[i];
            key[i] = key[l];
            key[l] = tk;
            const uint32_t ti = idx[i];
            idx[i] = idx[l];
            idx[l] = ti;
          }
        }
      }
      __syncthreads();
    }
  // run heads and their exclusive scan (four entries per thread, in order)
  const int per = (P + blockDim.x - 1) / blockDim.x;
  const int i0 = threadIdx.x * per;
  uint32_t cnt = 0;
  for (int i = i0; i < i0 + per && i < N; i++)
    cnt += (key[i] != b.sentinel && (i == 0 || key[i - 1] != key[i])) ? 1u : 0u;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = cnt;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t t = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0u;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, t, d);
      if (lane >= d) t += y;
    }
    warp_tot[lane] = t;
  }
  __syncthreads();
  uint32_t run = (warp ? warp_tot[warp - 1] : 0u) + x - cnt;
  for (int i = i0; i < i0 + per && i < N; i++) {
    pos[i] = run;
    run += (key[i] != b.sentinel && (i == 0 || key[i - 1] != key[i])) ? 1u : 0u;
  }
  if (threadIdx.x == 0) *b.count = (int64_t)warp_tot[(blockDim.x >> 5) - 1];
  __syncthreads();
  // one thread per run: sums in entry order
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    const uint64_t e = key[j];
    if (e == b.sentinel || (j > 0 && key[j - 1] == e)) continue;
    double a = 0.0, be = 0.0;
    for (int t = j; t < N && key[t] == e; t++) {
      const uint32_t q = idx[t];
      a = t == j ? b.ea[q] : __dadd_rn(a, b.ea[q]);
      be = t == j ? b.eb[q] : __dadd_rn(be, b.eb[q]);
    }
    const uint32_t o = pos[j];
    b.src_elem[o] = (int64_t)e;
    static_cast<E *>(b.src_alpha)[o] = (E)a;
    static_cast<E *>(b.src_scale)[o] = (E)__ddiv_rn(1.0, __dadd_rn(1.0, be));
    b.src_rowcol[o] = make_int2((int)((int64_t)e / b.rowlen), (int)((int64_t)e % b.rowlen));
  }
}

}  // namespace

int radix_passes(uint64_t sentinel) {
  int bits = 0;
  while (bits < 64 && (sentinel >> bits) != 0) bits++;
  return bits == 0 ? 1 : (bits + 7) / 8;
}

long long agent_sort_blocks(long long n) { return (n + kSortTile - 1) / kSortTile; }
long long agent_scan_blocks(long long n) { return (n + kScanTile - 1) / kScanTile; }

cudaError_t build_sources_device(AgentBuild b, bool fp64, cudaStream_t st) {
  const long long N = b.n_entries_max;
  const unsigned g256 = (unsigned)((N + 255) / 256);
  if (N > 0 && N <= kSmallBuild) {  // one CTA, then the row offsets
    if (fp64)
      small_build_kernel<double><<<1, kSmallBuildThreads, 0, st>>>(b);
    else
      small_build_kernel<float><<<1, kSmallBuildThreads, 0, st>>>(b);
  } else if (N > 0) {
    agent_entries_kernel<<<g256, 256, 0, st>>>(b);
    const int nb = (int)agent_sort_blocks(N);
    const int passes = radix_passes(b.sentinel);
    int cur = 0;
    for (int p = 0; p < passes; p++) {
      const int shift = 8 * p;
      radix_hist_kernel<<<nb, kSortThreads, 0, st>>>(b.key[cur], N, shift, b.hist, nb);
      cudaError_t e = exclusive_scan(b.hist, b.hist, 256LL * nb, b.part, nullptr, st);
      if (e != cudaSuccess) return e;
      radix_scatter_kernel<<<nb, kSortThreads, 0, st>>>(b.key[cur], b.idx[cur], N, shift, b.hist,
                                                        nb, b.key[cur ^ 1], b.idx[cur ^ 1]);
      cur ^= 1;
    }
    run_heads_kernel<<<g256, 256, 0, st>>>(b.key[cur], N, b.sentinel, b.head);
    cudaError_t e = exclusive_scan(b.head, b.pos, N, b.part, b.count32, st);
    if (e != cudaSuccess) return e;
    count_to_i64_kernel<<<1, 1, 0, st>>>(b.count32, b.count);
    if (fp64)
      run_sums_kernel<double><<<g256, 256, 0, st>>>(b, b.key[cur], b.idx[cur], N);
    else
      run_sums_kernel<float><<<g256, 256, 0, st>>>(b, b.key[cur], b.idx[cur], N);
  } else {
    cudaError_t e = cudaMemsetAsync(b.count, 0, sizeof(int64_t), st);
    if (e != cudaSuccess) return e;
  }
  row_offsets_kernel<<<(unsigned)((b.nrows + 1 + 255) / 256), 256, 0, st>>>(b);
  return cudaGetLastError();
}

}  // namespace bfv
