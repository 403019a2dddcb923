// Host half of libbiofvm: the C ABI of include/biofvm.h.
//
// Owns the handle, validates arguments, computes the Thomas constants of
// Appendix A in double (the paper's "first solver iteration ... stores the
// constant coefficients"), chooses the launch plan of each sweep, aggregates
// agents into per-element source terms, captures one step into a CUDA graph,
// and maps CUDA failures to status codes.  All compute runs in the kernels of
// sweeps_fp64.cu / sweeps_fp32.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/biofvm.h"
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
};
struct XPlan {
  int T = 1, m = 1, maxm = 8, rows_per_warp = 1, warps = 1, rows_per_cta = 1, use_bulk = 0;
  size_t smem = 0;
};

}  // namespace

struct biofvm {
  biofvm_grid g{};
  double dx = 0, dt = 0;
  std::vector<double> D, lam;
  std::vector<uint8_t> dir_on;
  std::vector<double> dir_val;
  bool any_dir = false;
  biofvm_precision prec = BIOFVM_FP64;
  size_t esz = 8;
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  size_t nel = 0;
  DevBuf rho, tab[3], dir_on_d, dir_val_d, status;
  XPlan xp;
  ColPlan cp[3];  // [1] = y, [2] = z
  // sources
  int64_t n_entries = 0;
  DevBuf src_row_off, src_elem, src_alpha, src_scale;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
};

namespace {

int axis_len(const biofvm *h, int axis) {
  return axis == 0 ? h->g.nx : axis == 1 ? h->g.ny : h->g.nz;
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
  out.assign((size_t)4 * n * S + (size_t)T * S + 2 * (size_t)S, 0.0);
  double *inv = out.data(), *mul = inv + (size_t)n * S, *pf = mul + (size_t)n * S,
         *pb = pf + (size_t)n * S, *pc = pb + (size_t)n * S, *cfix = pc + (size_t)T * S;
  std::vector<double> ci(n), cm(n);
  for (int s = 0; s < S; s++) {
    const double r = h->D[s] * h->dt / (h->dx * h->dx);
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
int col_bound_threads(int maxm, size_t) {
  const int regs = 2 * maxm + 64;
  const int raw = 65536 / regs;
  return std::min(1024, raw) / 32 * 32;
}

bool plan_col(int n, bool fp64, ColPlan &p) {
  const size_t esz = fp64 ? 8 : 4;
  for (int target = 32; target <= 128; target *= 2) {
    int T = (n + target - 1) / target;
    if (T < 1) T = 1;
    int m = (n + T - 1) / T;
    T = (n + m - 1) / m;  // every chunk non-empty
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

bool plan_x(int nx, int S, bool fp64, XPlan &p) {
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
  T = (nx + m - 1) / m;
  if (m > largest) return false;
  p.T = T;
  p.m = m;
  p.maxm = pick_maxm(m, fp64);
  p.rows_per_warp = 32 / (T * S);
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
  if (dev_alloc(b, v.size() * h->esz) != cudaSuccess)
    return fail(BIOFVM_ERR_OOM, "device allocation of %zu bytes failed", v.size() * h->esz);
  if (h->prec == BIOFVM_FP64) {
    CK(cudaMemcpyAsync(b.p, v.data(), v.size() * 8, cudaMemcpyHostToDevice, h->stream));
  } else {
    auto f = cast_vec<float>(v);
    CK(cudaMemcpyAsync(b.p, f.data(), f.size() * 4, cudaMemcpyHostToDevice, h->stream));
  }
  CK(cudaStreamSynchronize(h->stream));
  return BIOFVM_OK;
}

biofvm_status upload_constants(biofvm *h) {
  std::vector<double> t;
  for (int axis = 0; axis < 3; axis++) {
    const int T = axis == 0 ? h->xp.T : h->cp[axis].T;
    const int m = axis == 0 ? h->xp.m : h->cp[axis].m;
    axis_tables(h, axis, T, m, h->prec == BIOFVM_FP32, t);
    biofvm_status st = upload_doubles(h, h->tab[axis], t);
    if (st) return st;
  }
  if (h->graph) {
    cudaGraphExecDestroy(h->gexec);
    cudaGraphDestroy(h->graph);
    h->graph = nullptr;
    h->gexec = nullptr;
  }
  return BIOFVM_OK;
}

AxisTab axis_tab(const biofvm *h, int axis) {
  const int n = axis_len(h, axis), S = h->g.n_sub;
  const char *base = static_cast<const char *>(h->tab[axis].p);
  const size_t blk = (size_t)n * S * h->esz;
  AxisTab t;
  t.inv = base;
  t.mul = base + blk;
  t.pf = base + 2 * blk;
  t.pb = base + 3 * blk;
  t.pc = base + 4 * blk;
  t.cfix = base + 4 * blk + (size_t)(axis == 0 ? h->xp.T : h->cp[axis].T) * S * h->esz;
  t.n = n;
  t.T = axis == 0 ? h->xp.T : h->cp[axis].T;
  t.m = axis == 0 ? h->xp.m : h->cp[axis].m;
  return t;
}

// ---------------------------------------------------------------------------
// Kernel launches.
// ---------------------------------------------------------------------------
cudaError_t launch_x(const biofvm *h, int flags, cudaStream_t st) {
  XLaunch a{};
  a.rho = h->rho.p;
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
  a.has_src = h->n_entries > 0;
  a.src_row_off = static_cast<const int64_t *>(h->src_row_off.p);
  a.src_elem = static_cast<const int64_t *>(h->src_elem.p);
  a.src_alpha = h->src_alpha.p;
  a.src_scale = h->src_scale.p;
  a.dir_on = static_cast<const uint8_t *>(h->dir_on_d.p);
  a.dir_val = h->dir_val_d.p;
  a.status = static_cast<int *>(h->status.p);
  return h->prec == BIOFVM_FP64 ? launch_x_f64(a, st) : launch_x_f32(a, st);
}

cudaError_t launch_col(const biofvm *h, int axis, int flags, cudaStream_t st) {
  ColLaunch a{};
  a.rho = h->rho.p;
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
  return h->prec == BIOFVM_FP64 ? launch_col_f64(a, st) : launch_col_f32(a, st);
}

biofvm_status launch_step(const biofvm *h, cudaStream_t st) {
  CK(launch_x(h, kSrc | kDirBefore | kSolve | kDirAfter, st));
  CK(launch_col(h, 1, kSolve | kDirAfter, st));
  CK(launch_col(h, 2, kSolve | kDirAfter, st));
  return BIOFVM_OK;
}

biofvm_status check_status(biofvm *h) {
  int st = 0;
  CK(cudaMemcpy(&st, h->status.p, sizeof(int), cudaMemcpyDeviceToHost));
  if (st != kStatusOk) {
    CK(cudaMemset(h->status.p, 0, sizeof(int)));
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
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->graph) cudaGraphDestroy(h->graph);
  for (DevBuf *b : {&h->rho, &h->tab[0], &h->tab[1], &h->tab[2], &h->dir_on_d, &h->dir_val_d,
                    &h->status, &h->src_row_off, &h->src_elem, &h->src_alpha, &h->src_scale})
    b->release();
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  delete h;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char *biofvm_last_error(void) { return g_last_error.c_str(); }

biofvm_status biofvm_create(const biofvm_grid *grid, double dx, double dt, const double *D,
                            const double *lambda, const biofvm_boundary *bc,
                            biofvm_precision prec, uintptr_t cuda_stream, biofvm_t **out) {
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
  if (prec != BIOFVM_FP64 && prec != BIOFVM_FP32)
    return fail(BIOFVM_ERR_ARG, "unknown precision %d", (int)prec);
  const bool fp64 = prec == BIOFVM_FP64;
  const double nel_d = (double)g.nx * g.ny * g.nz * g.n_sub;
  if (nel_d > 9.0e18 / 8) return fail(BIOFVM_ERR_ARG, "grid too large");
  if ((double)g.nx * g.n_sub * (fp64 ? 8 : 4) >= 4.0e9 || (double)g.ny * g.nz >= 4.0e9)
    return fail(BIOFVM_ERR_ARG, "grid too large for 32-bit row offsets");

  biofvm *h = new (std::nothrow) biofvm();
  if (!h) return fail(BIOFVM_ERR_OOM, "host allocation failed");
  h->g = g;
  h->dx = dx;
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
  h->prec = prec;
  h->esz = fp64 ? 8 : 4;
  h->nel = (size_t)g.nx * g.ny * g.nz * g.n_sub;
  if (!plan_x(g.nx, g.n_sub, fp64, h->xp)) {
    delete h;
    return fail(BIOFVM_ERR_ARG, "x lines too long for the x-sweep tile (nx*n_sub = %d)",
                g.nx * g.n_sub);
  }
  if (!plan_col(g.ny, fp64, h->cp[1]) || !plan_col(g.nz, fp64, h->cp[2])) {
    delete h;
    return fail(BIOFVM_ERR_ARG, "y or z lines too long for the column sweep (ny=%d nz=%d)", g.ny,
                g.nz);
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
      (e = cudaMemcpyAsync(h->dir_on_d.p, h->dir_on.data(), g.n_sub, cudaMemcpyHostToDevice,
                           h->stream)) != cudaSuccess) {
    destroy_impl(h);
    return fail(BIOFVM_ERR_CUDA, "initialising device memory failed: %s", cudaGetErrorString(e));
  }
  e = fp64 ? allow_x_smem_f64(h->xp.maxm, h->xp.smem) : allow_x_smem_f32(h->xp.maxm, h->xp.smem);
  if (e != cudaSuccess) {
    destroy_impl(h);
    return fail(BIOFVM_ERR_CUDA, "x-sweep shared memory of %zu bytes refused: %s", h->xp.smem,
                cudaGetErrorString(e));
  }
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

int biofvm_launches_per_step(const biofvm_t *h) { return h ? 3 : 0; }

biofvm_status biofvm_set_params(biofvm_t *h, const double *D, const double *lambda) {
  if (!h) return fail(BIOFVM_ERR_ARG, "NULL handle");
  if (!valid_params(h->g.n_sub, D, lambda))
    return fail(BIOFVM_ERR_ARG, "D and lambda must be finite, >= 0 and non-NULL");
  CK(cudaSetDevice(h->device));
  h->D.assign(D, D + h->g.n_sub);
  h->lam.assign(lambda, lambda + h->g.n_sub);
  return upload_constants(h);
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
  // (element, alpha, beta) per agent and substrate, sorted by element and summed
  struct Ent {
    int64_t e;
    double alpha, beta;
  };
  std::vector<Ent> ent;
  ent.reserve((size_t)n * S);
  for (int64_t k = 0; k < n; k++) {
    const double w = weight ? weight[k] : 1.0;
    for (int s = 0; s < S; s++) {
      const double sv = secretion ? secretion[k * S + s] : 0.0;
      const double uv = uptake ? uptake[k * S + s] : 0.0;
      const double tv = target ? target[k * S + s] : 0.0;
      const double alpha = h->dt * w * sv * tv, beta = h->dt * w * (sv + uv);
      if (alpha != 0.0 || beta != 0.0) ent.push_back({voxel[k] * S + s, alpha, beta});
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
  std::vector<double> alpha(u), scale(u);
  for (size_t i = 0; i < u; i++) {
    off[ent[i].e / rowlen + 1]++;
    elem[i] = ent[i].e;
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
    biofvm_status st = upload_doubles(h, h->src_alpha, alpha);
    if (st) return st;
    st = upload_doubles(h, h->src_scale, scale);
    if (st) return st;
  }
  h->n_entries = (int64_t)u;
  if (h->graph) {  // kernel arguments changed
    cudaGraphExecDestroy(h->gexec);
    cudaGraphDestroy(h->graph);
    h->graph = nullptr;
    h->gexec = nullptr;
  }
  return BIOFVM_OK;
}

biofvm_status biofvm_step(biofvm_t *h, int n_steps) {
  if (!h) return fail(BIOFVM_ERR_ARG, "NULL handle");
  if (n_steps < 0) return fail(BIOFVM_ERR_ARG, "n_steps must be >= 0");
  if (n_steps == 0) return BIOFVM_OK;
  CK(cudaSetDevice(h->device));
  if (!h->gexec) {
    CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    biofvm_status st = launch_step(h, h->cap_stream);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->cap_stream, &graph);
    if (st != BIOFVM_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (e != cudaSuccess)
      return fail(BIOFVM_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&h->gexec, graph, 0);
    if (e != cudaSuccess) {
      cudaGraphDestroy(graph);
      return fail(BIOFVM_ERR_CUDA, "cudaGraphInstantiate failed: %s", cudaGetErrorString(e));
    }
    h->graph = graph;
  }
  for (int k = 0; k < n_steps; k++) CK(cudaGraphLaunch(h->gexec, h->stream));
  return BIOFVM_OK;
}

biofvm_status biofvm_run_stage(biofvm_t *h, int stage) {
  if (!h) return fail(BIOFVM_ERR_ARG, "NULL handle");
  CK(cudaSetDevice(h->device));
  switch (stage) {
    case 0: CK(launch_x(h, kSrc | kDirBefore, h->stream)); break;
    case 1: CK(launch_x(h, kSolve | kDirAfter, h->stream)); break;
    case 2: CK(launch_col(h, 1, kSolve | kDirAfter, h->stream)); break;
    case 3: CK(launch_col(h, 2, kSolve | kDirAfter, h->stream)); break;
    case 4: CK(launch_x(h, kSrc, h->stream)); break;
    case 5: CK(launch_x(h, kSolve, h->stream)); break;
    case 6: CK(launch_col(h, 1, kSolve, h->stream)); break;
    case 7: CK(launch_col(h, 2, kSolve, h->stream)); break;
    case 8: CK(launch_x(h, kSrc | kDirBefore | kSolve | kDirAfter, h->stream)); break;
    default: return fail(BIOFVM_ERR_ARG, "stage must be in [0, 8] (got %d)", stage);
  }
  return BIOFVM_OK;
}

void biofvm_destroy(biofvm_t *h) { destroy_impl(h); }

}  // extern "C"
