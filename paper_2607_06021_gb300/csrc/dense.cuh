// Block-cooperative small dense routines (one CTA): one-sided Jacobi SVD,
// descending sort permutation, smallest singular value.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#include "common.cuh"

namespace lrp {

constexpr int kJacobiSweeps = 40;

// One-sided Jacobi SVD of the mr x nc matrix A (col-major, lda; mr >= nc is the
// intended use).  On exit the columns of A are U*Sigma (mutually orthogonal),
// sig[j] = ||A(:,j)|| and, if V != nullptr, A_in = A_out V^T with V orthogonal.
__device__ inline void blk_jacobi(double* A, int lda, int mr, int nc, double* V, int ldv, double* sig, int* flag) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  if (V) {
    for (int e = tid; e < nc * nc; e += blockDim.x) {
      const int i = e % nc, j = e / nc;
      V[(int64_t)j * ldv + i] = (i == j) ? 1.0 : 0.0;
    }
  }
  __syncthreads();
  const int ne = nc + (nc & 1);
  const double tol = 1e-15;
  for (int sweep = 0; sweep < kJacobiSweeps && ne >= 2; ++sweep) {
    if (tid == 0) *flag = 0;
    __syncthreads();
    for (int rnd = 0; rnd < ne - 1; ++rnd) {
      for (int k = warp; k < ne / 2; k += nwarps) {
        int a, b;
        if (k == 0) {
          a = rnd % (ne - 1);
          b = ne - 1;
        } else {
          a = (rnd + k) % (ne - 1);
          b = (rnd + ne - 1 - k) % (ne - 1);
        }
        if (a >= nc || b >= nc) continue;
        if (a > b) {
          const int t = a;
          a = b;
          b = t;
        }
        double* ca = A + (int64_t)a * lda;
        double* cb = A + (int64_t)b * lda;
        double alpha = 0.0, beta = 0.0, gamma = 0.0;
        for (int i = lane; i < mr; i += 32) {
          const double x = ca[i], y = cb[i];
          alpha = fma(x, x, alpha);
          beta = fma(y, y, beta);
          gamma = fma(x, y, gamma);
        }
        alpha = warp_sum(alpha);
        beta = warp_sum(beta);
        gamma = warp_sum(gamma);
        if (gamma == 0.0 || fabs(gamma) <= tol * sqrt(alpha * beta)) continue;
        const double zeta = (beta - alpha) / (2.0 * gamma);
        const double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / sqrt(1.0 + t * t);
        const double s = c * t;
        for (int i = lane; i < mr; i += 32) {
          const double x = ca[i], y = cb[i];
          ca[i] = c * x - s * y;
          cb[i] = s * x + c * y;
        }
        if (V) {
          double* va = V + (int64_t)a * ldv;
          double* vb = V + (int64_t)b * ldv;
          for (int i = lane; i < nc; i += 32) {
            const double x = va[i], y = vb[i];
            va[i] = c * x - s * y;
            vb[i] = s * x + c * y;
          }
        }
        if (lane == 0) *flag = 1;
      }
      __syncthreads();
    }
    const int rotated = *flag;
    __syncthreads();
    if (!rotated) break;
  }
  for (int j = warp; j < nc; j += nwarps) {
    const double* cj = A + (int64_t)j * lda;
    double s = 0.0;
    for (int i = lane; i < mr; i += 32) s = fma(cj[i], cj[i], s);
    s = warp_sum(s);
    if (lane == 0) sig[j] = sqrt(s);
  }
  __syncthreads();
}

// perm[t] = index of the t-th largest of v[0..n) (ties to the lower index).
__device__ inline void blk_sort_desc(const double* v, int n, int* perm) {
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    int rank = 0;
    const double x = v[j];
    for (int l = 0; l < n; ++l) {
      const double y = v[l];
      rank += (y > x) || (y == x && l < j);
    }
    perm[rank] = j;
  }
  __syncthreads();
}

// Smallest singular value of the mr x nc matrix (copied to work first).
__device__ inline double blk_smin(const double* src, int lds, int mr, int nc, double* work, int ldw, double* sig, int* flag) {
  if (nc == 0) return 0.0;
  if (mr < nc) return 0.0;
  for (int e = threadIdx.x; e < mr * nc; e += blockDim.x) {
    const int i = e % mr, j = e / mr;
    work[(int64_t)j * ldw + i] = src[(int64_t)j * lds + i];
  }
  __syncthreads();
  blk_jacobi(work, ldw, mr, nc, nullptr, 0, sig, flag);
  __shared__ double red[32];
  double mn = 1e308;
  for (int j = threadIdx.x; j < nc; j += blockDim.x) mn = fmin(mn, sig[j]);
  mn = -block_max(-mn, red);
  return mn;
}

}  // namespace lrp
