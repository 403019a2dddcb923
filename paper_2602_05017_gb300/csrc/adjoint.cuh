// Adjoint (reverse-mode) kernels of the LOD step, derived from the forward
// stages:  rho+ = B Z^-1 B Y^-1 B X^-1 B Src(rho).
//
// Each 1D matrix A = (1 + lambda dt/3) I + r L_N is symmetric, so A^-T = A^-1
// and the adjoint sweeps are the forward sweep kernels run on the adjoint
// field in reverse order (Z, Y, X); B's adjoint zeroes the Dirichlet faces
// (kMaskZero).  For a sweep u = A^-1 d with adjoint mu = A^-1 ubar,
//     dL/dlambda_s += -(dt/3)      * sum_{elements of s} mu * u
//     dL/dD_s      += -(dt/dx^2)   * sum_{lines of s} sum_i (mu_{i+1}-mu_i)(u_{i+1}-u_i)
// (L_N = G^T G with G the first difference).  These sums are reduced in FP64
// in a fixed order -- per-block partials, then one block over the partials --
// so repeated runs give bit-identical gradients.
//
// Src: u1 = (u0 + alpha) / (1 + beta) per element, alpha = sum_k dt w_k S_k
// rho*_k, beta = sum_k dt w_k (S_k + U_k).  Hence du1/du0 = 1/(1+beta) and,
// for agent k in that voxel, du1/dS_k = dt w_k (rho*_k - u1) / (1 + beta) and
// du1/dU_k = -dt w_k u1 / (1 + beta).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace bfv {

// Per-block partial sums of (sum mu*u, sum dmu*du along the axis) for every
// substrate.  Thread tid < used (a multiple of S) walks elements tid,
// tid + used, ... so its substrate tid % S never changes.  partial layout:
// [block][2][S].
template <typename E>
__global__ void __launch_bounds__(kReduceThreads)
    adj_reduce_kernel(const E *__restrict__ mu, const E *__restrict__ u, long long nel, int S,
                      long long stride, int n_axis, long long used, double *__restrict__ partial) {
  __shared__ double sh[2][kReduceThreads];
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double s1 = 0.0, s2 = 0.0;
  if (tid < used) {
    for (long long e = tid; e < nel; e += used) {
      const double m0 = (double)mu[e], u0 = (double)u[e];
      s1 = fma(m0, u0, s1);
      const long long pos = (e / stride) % n_axis;
      if (pos + 1 < n_axis) {
        const double dm = (double)mu[e + stride] - m0, du = (double)u[e + stride] - u0;
        s2 = fma(dm, du, s2);
      }
    }
  }
  sh[0][threadIdx.x] = s1;
  sh[1][threadIdx.x] = s2;
  __syncthreads();
  if ((int)threadIdx.x < S) {
    const int j0 = threadIdx.x;
    const int sub = (int)(((long long)blockIdx.x * blockDim.x + j0) % S);
    double a = 0.0, b = 0.0;
    for (int j = j0; j < (int)blockDim.x; j += S) {  // fixed order
      a += sh[0][j];
      b += sh[1][j];
    }
    partial[((long long)blockIdx.x * 2 + 0) * S + sub] = a;
    partial[((long long)blockIdx.x * 2 + 1) * S + sub] = b;
  }
}

// One block: sum the partials in block order and accumulate the gradients.
// (Templated on the field type only so that each precision's translation unit
// owns its instance.)
template <typename E>
__global__ void adj_reduce_final_kernel(const double *__restrict__ partial, int nblocks, int S,
                                        double scale_lambda, double scale_D, double *dlambda,
                                        double *dD) {
  const int s = threadIdx.x;
  if (s >= S) return;
  double a = 0.0, b = 0.0;
  for (int k = 0; k < nblocks; k++) {
    a += partial[((long long)k * 2 + 0) * S + s];
    b += partial[((long long)k * 2 + 1) * S + s];
  }
  dlambda[s] += scale_lambda * a;
  dD[s] += scale_D * b;
}

// Secretion and uptake gradients per (agent, substrate): one thread each, no
// reduction.  elem[k*S+s] = voxel_k*S + s; entry[k*S+s] = index of that
// element in the aggregated source list (its 1/(1+beta)), or -1 when the
// element has none.  dsec or dupt may be NULL.
template <typename E>
__global__ void src_adjoint_agents_kernel(const E *__restrict__ gbar, const E *__restrict__ u1,
                                          const int64_t *__restrict__ elem,
                                          const int64_t *__restrict__ entry,
                                          const E *__restrict__ src_scale,
                                          const double *__restrict__ weight,
                                          const double *__restrict__ target, long long n, double dt,
                                          int S, double *__restrict__ dsec,
                                          double *__restrict__ dupt) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const long long e = elem[i], ent = entry[i];
  const double scale = ent >= 0 ? (double)src_scale[ent] : 1.0;
  const double w = weight ? weight[i / S] : 1.0;
  const double gw = (double)gbar[e] * dt * w * scale, u = (double)u1[e];
  if (dsec) dsec[i] += gw * (target[i] - u);
  if (dupt) dupt[i] -= gw * u;
}

// gbar <- gbar / (1 + beta) on the elements that have a source entry.
template <typename E>
__global__ void src_adjoint_scale_kernel(E *__restrict__ gbar, const int64_t *__restrict__ src_elem,
                                         const E *__restrict__ src_scale, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) gbar[src_elem[i]] *= src_scale[i];
}

}  // namespace bfv
