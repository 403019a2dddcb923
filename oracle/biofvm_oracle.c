/*
 * FP64 CPU oracle for one BioFVM-B diffusion-decay time step.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, header, table or helper with
 * the CUDA library: it restates the method from the paper in the plainest
 * form, one line at a time, in double precision, single-threaded.
 *
 * What one step computes (paper Sect. 2: seven stages, four Dirichlet
 * applications around the three axis solves; preceded by the cell
 * source/uptake update of the end-to-end run, Sect. 5.3):
 *
 *     rho+ = B . Z^-1 . B . Y^-1 . B . X^-1 . B . Src (rho)
 *
 *   Src   implicit per-voxel source/uptake update of BioFVM (reading below);
 *   B     Dirichlet application: overwrite the boundary-face voxels of every
 *         substrate whose Dirichlet flag is on (identity otherwise);
 *   X^-1  for every x-line and substrate, solve the tridiagonal system of
 *         Appendix A with the Thomas algorithm (Algorithm 1; forward sweep
 *         divides by denom, backward sweep is a negated axpy, Sect. 2.1);
 *   Y^-1, Z^-1 the same along y and z.
 *
 * Readings of the paper taken here (each also listed in the design notes):
 *   - Appendix A prints a_i = +dt*D/dx^2 but c_i = -dt*D/dx^2; the finite
 *     volume operator that conserves mass (Sect. 2, FVM vs FDM) is symmetric,
 *     so a_i = c_i = -r with r = D*dt/dx^2.
 *   - On an axis of a single voxel there is no neighbour to exchange with:
 *     b = 1 + lambda*dt/3 there (the printed end-row value would add r).
 *   - Decay lambda*dt/3 sits on every diagonal, one third per sweep (App. A).
 *   - Stage order of the 7 stages: B, X^-1, B, Y^-1, B, Z^-1, B.
 *   - Dirichlet application overwrites the voxels of the six faces; the
 *     matrices keep their zero-flux end rows.
 *   - Dirichlet nodes (BioFVM's Dirichlet voxels anywhere in the grid, and
 *     face values that differ per face): a list of (element, value) pairs
 *     overwritten at each of the same four applications, after the faces;
 *     an element listed twice takes its last value.
 *   - Source/uptake (not printed in this paper; the implicit update of the
 *     cited BioFVM): rho <- (rho + alpha) / (1 + beta) with, summed over the
 *     agents in the voxel, alpha = sum dt*w*S*rho_target and
 *     beta = sum dt*w*(S + U).  Agents sharing a voxel are aggregated, which
 *     makes the update independent of agent order.
 *
 * Layout of every field: rho[((z*ny + y)*nx + x)*ns + s].
 *
 * Built plain (single-threaded: the parity oracle) and, as a separate
 * library, with -fopenmp: the "paper-style" CPU rate, the independent lines
 * of a sweep and the elements of the source update split over the host's
 * cores (the paper's own CPU parallelisation is over lines).  Every line and
 * element is computed by the same statements in both builds, so the two
 * agree bit for bit.
 * All entry points return 0 on success, -1 on bad arguments, -2 on OOM.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef long long i64;

/* ------------------------------------------------------------------------ */
/* Appendix A: the tridiagonal system of one axis and its Thomas constants.  */
/* ------------------------------------------------------------------------ */

/* Fill a, b, c (length n) of the system a_i x_{i-1} + b_i x_i + c_i x_{i+1}
 * = d_i for one axis of n voxels (App. A, Eqs. for a, b, c), and the
 * precomputed constants denom_i and constant_c_i = c'_i (App. A, Eqs. for
 * constant_c and denom).  r = D*dt/dx^2, lam3 = lambda*dt/3. */
int oracle_axis_coefficients(int n, double r, double lam3, double *a,
                             double *b, double *c, double *denom,
                             double *cprime) {
  if (n < 1 || !a || !b || !c || !denom || !cprime) return -1;
  for (int i = 0; i < n; i++) {
    a[i] = -r;
    c[i] = -r;
    if (n == 1)
      b[i] = 1.0 + lam3;
    else if (i == 0 || i == n - 1)
      b[i] = 1.0 + r + lam3;
    else
      b[i] = 1.0 + 2.0 * r + lam3;
  }
  denom[0] = b[0];
  cprime[0] = c[0] / b[0];
  for (int i = 1; i < n; i++) {
    denom[i] = b[i] - a[i] * cprime[i - 1];
    cprime[i] = c[i] / denom[i];
  }
  return 0;
}

/* Thomas algorithm on one system, in place on d (Sect. 2.1: the first
 * forward row divides by b_1, every other forward row does an axpy and a
 * division; the backward sweep does a negated axpy on all rows but the
 * last).  General coefficients so that tests can drive it directly. */
int oracle_thomas(int n, const double *a, const double *b, const double *c,
                  double *d) {
  if (n < 1 || !a || !b || !c || !d) return -1;
  double *cp = (double *)malloc(sizeof(double) * (size_t)n);
  if (!cp) return -2;
  double den = b[0];
  cp[0] = c[0] / den;
  d[0] = d[0] / den;
  for (int i = 1; i < n; i++) {
    den = b[i] - a[i] * cp[i - 1];
    cp[i] = c[i] / den;
    d[i] = (d[i] - a[i] * d[i - 1]) / den;
  }
  for (int i = n - 2; i >= 0; i--) d[i] = d[i] - cp[i] * d[i + 1];
  free(cp);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Line geometry.                                                            */
/* ------------------------------------------------------------------------ */

/* For axis 0/1/2 (x/y/z): the length of a line, the element stride along
 * it, and the number of lines per substrate. */
static void axis_shape(int axis, int nx, int ny, int nz, int ns, int *n,
                       i64 *stride, i64 *nlines) {
  if (axis == 0) {
    *n = nx;
    *stride = ns;
    *nlines = (i64)ny * nz;
  } else if (axis == 1) {
    *n = ny;
    *stride = (i64)nx * ns;
    *nlines = (i64)nx * nz;
  } else {
    *n = nz;
    *stride = (i64)nx * ny * ns;
    *nlines = (i64)nx * ny;
  }
}

/* Index of element 0 of line `l` (0 <= l < nlines) of substrate s. */
static i64 line_base(int axis, int nx, int ny, int ns, i64 l, int s) {
  if (axis == 0) { /* l = z*ny + y */
    return l * nx * ns + s;
  } else if (axis == 1) { /* l = z*nx + x */
    i64 z = l / nx, x = l % nx;
    return (z * ny * nx + x) * ns + s;
  } else { /* l = y*nx + x */
    return l * ns + s;
  }
}

static int check_grid(int nx, int ny, int nz, int ns) {
  return nx >= 1 && ny >= 1 && nz >= 1 && ns >= 1;
}

/* ------------------------------------------------------------------------ */
/* Stages.                                                                   */
/* ------------------------------------------------------------------------ */

/* X^-1, Y^-1 or Z^-1 (axis 0, 1, 2): Algorithm 1 for that dimension, every
 * substrate.  Coefficients from App. A are recomputed here per substrate. */
int oracle_sweep(int axis, int nx, int ny, int nz, int ns, double dx,
                 double dt, const double *D, const double *lambda,
                 double *rho) {
  if (axis < 0 || axis > 2 || !check_grid(nx, ny, nz, ns) || !(dx > 0) ||
      !(dt > 0) || !D || !lambda || !rho)
    return -1;
  int n;
  i64 stride, nlines;
  axis_shape(axis, nx, ny, nz, ns, &n, &stride, &nlines);
  int nthreads = 1; /* one line buffer per thread (the OpenMP build) */
#ifdef _OPENMP
  nthreads = omp_get_max_threads();
#endif
  double *a = (double *)malloc(sizeof(double) * (size_t)n * (5 + (size_t)nthreads));
  if (!a) return -2;
  double *b = a + n, *c = b + n, *den = c + n, *cp = den + n, *lines = cp + n;
  for (int s = 0; s < ns; s++) {
    double r = D[s] * dt / (dx * dx);
    double lam3 = lambda[s] * dt / 3.0;
    oracle_axis_coefficients(n, r, lam3, a, b, c, den, cp);
    /* the lines of one substrate are independent systems */
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (i64 l = 0; l < nlines; l++) {
      int tid = 0;
#ifdef _OPENMP
      tid = omp_get_thread_num();
#endif
      double *line = lines + (size_t)tid * n;
      i64 base = line_base(axis, nx, ny, ns, l, s);
      for (int i = 0; i < n; i++) line[i] = rho[base + i * stride];
      /* forward sweep: g_1 = d_1/denom_1, g_i = (d_i - a_i g_{i-1})/denom_i */
      line[0] = line[0] / den[0];
      for (int i = 1; i < n; i++)
        line[i] = (line[i] - a[i] * line[i - 1]) / den[i];
      /* backward sweep: x_n = g_n, x_i = g_i - c'_i x_{i+1} */
      for (int i = n - 2; i >= 0; i--) line[i] = line[i] - cp[i] * line[i + 1];
      for (int i = 0; i < n; i++) rho[base + i * stride] = line[i];
    }
  }
  free(a);
  return 0;
}

/* Is voxel (x, y, z) on one of the six faces of the box? */
static int on_face(int x, int y, int z, int nx, int ny, int nz) {
  return x == 0 || x == nx - 1 || y == 0 || y == ny - 1 || z == 0 ||
         z == nz - 1;
}

/* B: one Dirichlet application (Sect. 2, the 7 stages). */
int oracle_dirichlet(int nx, int ny, int nz, int ns, const unsigned char *on,
                     const double *value, double *rho) {
  if (!check_grid(nx, ny, nz, ns) || !rho) return -1;
  if (!on) return 0;
  if (!value) return -1;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (int z = 0; z < nz; z++)
    for (int y = 0; y < ny; y++)
      for (int x = 0; x < nx; x++) {
        if (!on_face(x, y, z, nx, ny, nz)) continue;
        i64 v = ((i64)z * ny + y) * nx + x;
        for (int s = 0; s < ns; s++)
          if (on[s]) rho[v * ns + s] = value[s];
      }
  return 0;
}

/* The node part of B: rho[elem[k]] = val[k] in list order. */
int oracle_dirichlet_nodes(int nx, int ny, int nz, int ns, i64 n_nodes,
                           const i64 *elem, const double *val, double *rho) {
  if (!check_grid(nx, ny, nz, ns) || !rho || n_nodes < 0) return -1;
  if (n_nodes == 0) return 0;
  if (!elem || !val) return -1;
  i64 nel = (i64)nx * ny * nz * ns;
  for (i64 k = 0; k < n_nodes; k++)
    if (elem[k] < 0 || elem[k] >= nel) return -1;
  for (i64 k = 0; k < n_nodes; k++) rho[elem[k]] = val[k];
  return 0;
}

/* One full Dirichlet application: the faces, then the nodes. */
static int apply_b(int nx, int ny, int nz, int ns, const unsigned char *on,
                   const double *value, i64 n_nodes, const i64 *node_elem,
                   const double *node_val, double *rho) {
  int rc = oracle_dirichlet(nx, ny, nz, ns, on, value, rho);
  if (rc) return rc;
  return oracle_dirichlet_nodes(nx, ny, nz, ns, n_nodes, node_elem, node_val,
                                rho);
}

/* Dense per-element alpha and beta aggregated from an agent list. */
static int aggregate_sources(i64 nvox, int ns, double dt, i64 n_agents,
                             const i64 *voxel, const double *sec,
                             const double *tgt, const double *upt,
                             const double *w, double **alpha_out,
                             double **beta_out) {
  double *alpha = (double *)calloc((size_t)(nvox * ns), sizeof(double));
  double *beta = (double *)calloc((size_t)(nvox * ns), sizeof(double));
  if (!alpha || !beta) {
    free(alpha);
    free(beta);
    return -2;
  }
  for (i64 k = 0; k < n_agents; k++) {
    i64 v = voxel[k];
    if (v < 0 || v >= nvox) {
      free(alpha);
      free(beta);
      return -1;
    }
    double wk = w ? w[k] : 1.0;
    for (int s = 0; s < ns; s++) {
      double S = sec ? sec[k * ns + s] : 0.0;
      double T = tgt ? tgt[k * ns + s] : 0.0;
      double U = upt ? upt[k * ns + s] : 0.0;
      alpha[v * ns + s] += dt * wk * S * T;
      beta[v * ns + s] += dt * wk * (S + U);
    }
  }
  *alpha_out = alpha;
  *beta_out = beta;
  return 0;
}

/* Src: the implicit source/uptake update (reading of cited BioFVM). */
int oracle_sources(int nx, int ny, int nz, int ns, double dt, i64 n_agents,
                   const i64 *voxel, const double *sec, const double *tgt,
                   const double *upt, const double *w, double *rho) {
  if (!check_grid(nx, ny, nz, ns) || !rho || n_agents < 0) return -1;
  if (n_agents == 0) return 0;
  if (!voxel) return -1;
  i64 nvox = (i64)nx * ny * nz;
  double *alpha, *beta;
  int rc = aggregate_sources(nvox, ns, dt, n_agents, voxel, sec, tgt, upt, w,
                             &alpha, &beta);
  if (rc) return rc;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (i64 e = 0; e < nvox * ns; e++)
    rho[e] = (rho[e] + alpha[e]) / (1.0 + beta[e]);
  free(alpha);
  free(beta);
  return 0;
}

/* n_steps full time steps, in place on rho.  h3: the voxel spacing along x, y
 * and z (the paper's grids are isotropic, h3[0] = h3[1] = h3[2]; each axis's
 * App. A system takes r = D dt / h^2 with its own h). */
int oracle_step(int nx, int ny, int nz, int ns, const double *h3, double dt,
                const double *D, const double *lambda, const unsigned char *on,
                const double *value, i64 n_nodes, const i64 *node_elem,
                const double *node_val, i64 n_agents, const i64 *voxel,
                const double *sec, const double *tgt, const double *upt,
                const double *w, int n_steps, double *rho) {
  if (n_steps < 0 || !h3) return -1;
  for (int k = 0; k < n_steps; k++) {
    int rc = oracle_sources(nx, ny, nz, ns, dt, n_agents, voxel, sec, tgt, upt,
                            w, rho);
    if (rc) return rc;
    for (int axis = 0; axis < 3; axis++) {
      rc = apply_b(nx, ny, nz, ns, on, value, n_nodes, node_elem, node_val, rho);
      if (rc) return rc;
      rc = oracle_sweep(axis, nx, ny, nz, ns, h3[axis], dt, D, lambda, rho);
      if (rc) return rc;
    }
    rc = apply_b(nx, ny, nz, ns, on, value, n_nodes, node_elem, node_val, rho);
    if (rc) return rc;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Adjoint of one step (reverse mode), derived from the stages above.        */
/* ------------------------------------------------------------------------ */

/* Zero the adjoint where B overwrote the forward value (dB/du = mask): the
 * flagged faces and the nodes. */
static void dirichlet_mask(int nx, int ny, int nz, int ns,
                           const unsigned char *on, i64 n_nodes,
                           const i64 *node_elem, double *g) {
  for (i64 k = 0; k < n_nodes; k++) g[node_elem[k]] = 0.0;
  if (!on) return;
  for (int z = 0; z < nz; z++)
    for (int y = 0; y < ny; y++)
      for (int x = 0; x < nx; x++) {
        if (!on_face(x, y, z, nx, ny, nz)) continue;
        i64 v = ((i64)z * ny + y) * nx + x;
        for (int s = 0; s < ns; s++)
          if (on[s]) g[v * ns + s] = 0.0;
      }
}

/* Parameter gradient of one sweep u = A^-1 d, with mu = A^-T ubar:
 * dL/dtheta = -mu^T (dA/dtheta) u.  A = (1 + lambda dt/3) I + r L_N, where
 * L_N = G^T G is the zero-flux second difference (G the first difference),
 * so mu^T L_N u = sum_i (mu_{i+1} - mu_i)(u_{i+1} - u_i). */
static void sweep_param_grad(int axis, int nx, int ny, int nz, int ns,
                             double dx, double dt, const double *mu,
                             const double *u, double *dD, double *dlambda) {
  int n;
  i64 stride, nlines;
  axis_shape(axis, nx, ny, nz, ns, &n, &stride, &nlines);
  for (int s = 0; s < ns; s++) {
    double sum_mu_u = 0.0, sum_grad = 0.0;
    for (i64 l = 0; l < nlines; l++) {
      i64 base = line_base(axis, nx, ny, ns, l, s);
      for (int i = 0; i < n; i++)
        sum_mu_u += mu[base + i * stride] * u[base + i * stride];
      for (int i = 0; i + 1 < n; i++) {
        double dmu = mu[base + (i + 1) * stride] - mu[base + i * stride];
        double du = u[base + (i + 1) * stride] - u[base + i * stride];
        sum_grad += dmu * du;
      }
    }
    dlambda[s] += -(dt / 3.0) * sum_mu_u;
    dD[s] += -(dt / (dx * dx)) * sum_grad;
  }
}

/* Given the step's input rho_in and the adjoint gbar_out of its output,
 * write the adjoint of rho_in to gbar_in and ACCUMULATE (+=) the gradients
 * w.r.t. D[ns], lambda[ns] and, per agent and substrate, the secretion and
 * uptake rates dsec[n_agents*ns], dupt[n_agents*ns] (either may be NULL).
 * Each 1D matrix is symmetric, so A^-T = A^-1 and the adjoint sweeps are the
 * forward sweeps run in reverse stage order. */
int oracle_adjoint_step(int nx, int ny, int nz, int ns, const double *h3, double dt,
                        const double *D, const double *lambda,
                        const unsigned char *on, const double *value,
                        i64 n_nodes, const i64 *node_elem,
                        const double *node_val, i64 n_agents, const i64 *voxel,
                        const double *sec, const double *tgt, const double *upt,
                        const double *w, const double *rho_in,
                        const double *gbar_out, double *gbar_in, double *dD,
                        double *dlambda, double *dsec, double *dupt) {
  if (!check_grid(nx, ny, nz, ns) || !h3 || !rho_in || !gbar_out || !gbar_in ||
      !dD || !dlambda || n_agents < 0 || n_nodes < 0 ||
      (n_nodes > 0 && (!node_elem || !node_val)))
    return -1;
  for (i64 k = 0; k < n_nodes; k++)
    if (node_elem[k] < 0 || node_elem[k] >= (i64)nx * ny * nz * ns) return -1;
  i64 nel = (i64)nx * ny * nz * ns;
  size_t bytes = sizeof(double) * (size_t)nel;
  /* forward intermediates: u1 = Src(rho), u3 = X^-1 B u1, u5, u7 */
  double *u1 = (double *)malloc(bytes), *u3 = (double *)malloc(bytes);
  double *u5 = (double *)malloc(bytes), *u7 = (double *)malloc(bytes);
  if (!u1 || !u3 || !u5 || !u7) {
    free(u1);
    free(u3);
    free(u5);
    free(u7);
    return -2;
  }
  int rc = 0;
  memcpy(u1, rho_in, bytes);
  rc |= oracle_sources(nx, ny, nz, ns, dt, n_agents, voxel, sec, tgt, upt, w,
                       u1);
  memcpy(u3, u1, bytes);
  rc |= apply_b(nx, ny, nz, ns, on, value, n_nodes, node_elem, node_val, u3);
  rc |= oracle_sweep(0, nx, ny, nz, ns, h3[0], dt, D, lambda, u3);
  memcpy(u5, u3, bytes);
  rc |= apply_b(nx, ny, nz, ns, on, value, n_nodes, node_elem, node_val, u5);
  rc |= oracle_sweep(1, nx, ny, nz, ns, h3[1], dt, D, lambda, u5);
  memcpy(u7, u5, bytes);
  rc |= apply_b(nx, ny, nz, ns, on, value, n_nodes, node_elem, node_val, u7);
  rc |= oracle_sweep(2, nx, ny, nz, ns, h3[2], dt, D, lambda, u7);
  if (rc) goto done;

  /* reverse: gbar_in walks back through B, Z^-1, B, Y^-1, B, X^-1, B, Src */
  memcpy(gbar_in, gbar_out, bytes);
  dirichlet_mask(nx, ny, nz, ns, on, n_nodes, node_elem, gbar_in);
  rc |= oracle_sweep(2, nx, ny, nz, ns, h3[2], dt, D, lambda, gbar_in);
  sweep_param_grad(2, nx, ny, nz, ns, h3[2], dt, gbar_in, u7, dD, dlambda);
  dirichlet_mask(nx, ny, nz, ns, on, n_nodes, node_elem, gbar_in);
  rc |= oracle_sweep(1, nx, ny, nz, ns, h3[1], dt, D, lambda, gbar_in);
  sweep_param_grad(1, nx, ny, nz, ns, h3[1], dt, gbar_in, u5, dD, dlambda);
  dirichlet_mask(nx, ny, nz, ns, on, n_nodes, node_elem, gbar_in);
  rc |= oracle_sweep(0, nx, ny, nz, ns, h3[0], dt, D, lambda, gbar_in);
  sweep_param_grad(0, nx, ny, nz, ns, h3[0], dt, gbar_in, u3, dD, dlambda);
  dirichlet_mask(nx, ny, nz, ns, on, n_nodes, node_elem, gbar_in);
  if (rc) goto done;

  /* Src: u1 = (u0 + alpha)/(1 + beta).  du1/du0 = 1/(1+beta);
   * du1/dS_k = dt w_k (target_k - u1)/(1+beta); du1/dU_k = -dt w_k u1/(1+beta) */
  if (n_agents > 0) {
    i64 nvox = (i64)nx * ny * nz;
    double *alpha, *beta;
    rc = aggregate_sources(nvox, ns, dt, n_agents, voxel, sec, tgt, upt, w,
                           &alpha, &beta);
    if (rc) goto done;
    for (i64 k = 0; k < n_agents; k++) {
      double wk = w ? w[k] : 1.0;
      for (int s = 0; s < ns; s++) {
        i64 e = voxel[k] * ns + s;
        double T = tgt ? tgt[k * ns + s] : 0.0;
        if (dsec) dsec[k * ns + s] += gbar_in[e] * dt * wk * (T - u1[e]) / (1.0 + beta[e]);
        if (dupt) dupt[k * ns + s] += gbar_in[e] * (-dt * wk * u1[e]) / (1.0 + beta[e]);
      }
    }
    for (i64 e = 0; e < nel; e++) gbar_in[e] = gbar_in[e] / (1.0 + beta[e]);
    free(alpha);
    free(beta);
  }
done:
  free(u1);
  free(u3);
  free(u5);
  free(u7);
  return rc;
}
