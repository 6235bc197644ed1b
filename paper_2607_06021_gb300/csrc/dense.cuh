// Block-cooperative small dense routines (one CTA): one-sided Jacobi SVD,
// descending sort permutation, smallest singular value.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#include "common.cuh"

namespace lrp {

constexpr int kJacobiSweeps = 40;

template <typename TC>
struct Eps;
template <>
struct Eps<double> {
  static constexpr double value = 2.220446049250313e-16;
};
template <>
struct Eps<float> {
  static constexpr double value = 1.1920928955078125e-07;
};

// One-sided Jacobi SVD of the mr x nc matrix A (col-major, lda; mr >= nc is the
// intended use) in arithmetic TC.  On exit the columns of A are U*Sigma
// (mutually orthogonal), sig[j] = ||A(:,j)|| and, if V != nullptr,
// A_in = A_out V^T with V orthogonal.
template <typename TC>
__device__ __forceinline__ TC half_warp_sum(TC v) {
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One-sided Jacobi SVD of the mr x nc matrix A (col-major, lda; mr >= nc is the
// intended use) in arithmetic TC, round-robin pair ordering.  Each half-warp
// rotates one column pair; a warp always takes two pairs of a round together so
// that its shuffles stay warp-uniform.  On exit the columns of A are U*Sigma
// (mutually orthogonal), sig[j] = ||A(:,j)|| and, if V != nullptr,
// A_in = A_out V^T with V orthogonal.
// A is scaled by a power of two to ||A||_F in [1/2, 1) for the sweeps (exact;
// undone on exit), so that squared column norms cannot underflow in FP32.  A
// pair is left alone once |a_i . a_j| <= mr eps ||a_i|| ||a_j|| (rounding noise)
// or one of its columns is below eps ||A||_F: such columns lie below every
// cutoff applied to the singular values (the pseudoinverse's
// max(|I|,|J|) eps sigma_1, the tail rules), and rotating them only chases
// rounding noise.
template <typename TC>
__device__ inline void blk_jacobi(TC* A, int lda, int mr, int nc, TC* V, int ldv, double* sig, int* flag) {
  const int tid = threadIdx.x, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int half = (tid >> 4) & 1, hl = tid & 15;
  if (V) {
    for (int e = tid; e < nc * nc; e += blockDim.x) {
      const int i = e % nc, j = e / nc;
      V[(int64_t)j * ldv + i] = (i == j) ? (TC)1 : (TC)0;
    }
  }
  __shared__ double jac_red[32];
  double f2 = 0.0;
  for (int e = tid; e < mr * nc; e += blockDim.x) {
    const double v = (double)A[(int64_t)(e / mr) * lda + (e % mr)];
    f2 = fma(v, v, f2);
  }
  f2 = warp_sum(f2);
  if ((tid & 31) == 0) jac_red[warp] = f2;
  __syncthreads();
  if (tid < 32) {
    double v = tid < nwarps ? jac_red[tid] : 0.0;
    v = warp_sum(v);
    if (tid == 0) jac_red[0] = v;
  }
  __syncthreads();
  const double fro2 = jac_red[0];
  int ex = 0;
  if (fro2 > 0.0) frexp(sqrt(fro2), &ex);
  const TC down = (TC)ldexp(1.0, -ex);
  if (ex != 0)
    for (int e = tid; e < mr * nc; e += blockDim.x) A[(int64_t)(e / mr) * lda + (e % mr)] *= down;
  __syncthreads();
  const int ne = nc + (nc & 1);
  const int npairs = ne / 2;
  const TC tol = (TC)((double)(mr > 1 ? mr : 1) * Eps<TC>::value);
  const TC nu = (TC)(Eps<TC>::value * Eps<TC>::value);
  // Squared column norms: computed at the start of every sweep, then carried
  // through its rotations (a rotation that zeroes a.b maps ||a||^2, ||b||^2 to
  // ||a||^2 - t (a.b), ||b||^2 + t (a.b)), so that a pair needs only its dot
  // product a.b.
  __shared__ TC jac_nrm[kMaxM];
  const int lane32 = tid & 31;
  for (int sweep = 0; sweep < kJacobiSweeps && ne >= 2; ++sweep) {
    for (int j = warp; j < nc; j += nwarps) {
      const TC* cj = A + (int64_t)j * lda;
      TC v = 0;
      for (int i = lane32; i < mr; i += 32) v = fma(cj[i], cj[i], v);
      v = warp_sum(v);
      if (lane32 == 0) jac_nrm[j] = v;
    }
    if (tid == 0) *flag = 0;
    __syncthreads();
    for (int rnd = 0; rnd < ne - 1; ++rnd) {
      for (int kw = warp; 2 * kw < npairs; kw += nwarps) {
        const int k = 2 * kw + half;
        int a = -1, b = -1;
        if (k < npairs) {
          if (k == 0) {
            a = rnd % (ne - 1);
            b = ne - 1;
          } else {
            a = (rnd + k) % (ne - 1);
            b = (rnd + ne - 1 - k) % (ne - 1);
          }
          if (a >= nc || b >= nc) a = b = -1;
          if (a > b) {
            const int t = a;
            a = b;
            b = t;
          }
        }
        const bool valid = a >= 0;
        TC* ca = A + (int64_t)(valid ? a : 0) * lda;
        TC* cb = A + (int64_t)(valid ? b : 0) * lda;
        TC gamma = 0;
        if (valid)
          for (int i = hl; i < mr; i += 16) gamma = fma(ca[i], cb[i], gamma);
        gamma = half_warp_sum(gamma);
        const TC alpha = valid ? jac_nrm[a] : (TC)0, beta = valid ? jac_nrm[b] : (TC)0;
        if (!valid || gamma == (TC)0 || fabs(gamma) <= tol * sqrt(alpha) * sqrt(beta) || fmin(alpha, beta) <= nu)
          continue;
        const TC zeta = (beta - alpha) / ((TC)2 * gamma);
        const TC t = copysign((TC)1, zeta) / (fabs(zeta) + sqrt((TC)1 + zeta * zeta));
        const TC c = (TC)1 / sqrt((TC)1 + t * t);
        const TC s = c * t;
        for (int i = hl; i < mr; i += 16) {
          const TC x = ca[i], y = cb[i];
          ca[i] = c * x - s * y;
          cb[i] = s * x + c * y;
        }
        if (V) {
          TC* va = V + (int64_t)a * ldv;
          TC* vb = V + (int64_t)b * ldv;
          for (int i = hl; i < nc; i += 16) {
            const TC x = va[i], y = vb[i];
            va[i] = c * x - s * y;
            vb[i] = s * x + c * y;
          }
        }
        if (hl == 0) {
          jac_nrm[a] = alpha - t * gamma;
          jac_nrm[b] = beta + t * gamma;
          *flag = 1;
        }
      }
      __syncthreads();
    }
    const int rotated = *flag;
    __syncthreads();
    if (!rotated) break;
  }
  if (ex != 0) {
    const TC up = (TC)ldexp(1.0, ex);
    for (int e = tid; e < mr * nc; e += blockDim.x) A[(int64_t)(e / mr) * lda + (e % mr)] *= up;
    __syncthreads();
  }
  const int lane = tid & 31;
  for (int j = warp; j < nc; j += nwarps) {
    const TC* cj = A + (int64_t)j * lda;
    TC s = 0;
    for (int i = lane; i < mr; i += 32) s = fma(cj[i], cj[i], s);
    s = warp_sum(s);
    if (lane == 0) sig[j] = sqrt((double)s);
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

// Smallest nonzero-rank singular value of the mr x nc matrix: sigma_min(A) for a
// tall A, and the smallest of the mr singular values of a wide A, so that
// 1/result = ||A^+||_2 for a full-rank A of either shape.
template <typename TC>
__device__ inline double blk_smin(const TC* src, int lds, int mr, int nc, TC* work, int ldw, double* sig, int* flag) {
  if (nc == 0 || mr == 0) return 0.0;
  const bool wide = mr < nc;
  const int rows = wide ? nc : mr, cols = wide ? mr : nc;
  for (int e = threadIdx.x; e < mr * nc; e += blockDim.x) {
    const int i = e % mr, j = e / mr;
    const TC v = src[(int64_t)j * lds + i];
    if (wide)
      work[(int64_t)i * ldw + j] = v;
    else
      work[(int64_t)j * ldw + i] = v;
  }
  __syncthreads();
  blk_jacobi<TC>(work, ldw, rows, cols, nullptr, 0, sig, flag);
  __shared__ double red[32];
  double mn = 1e308;
  for (int j = threadIdx.x; j < cols; j += blockDim.x) mn = fmin(mn, sig[j]);
  mn = -block_max(-mn, red);
  return mn;
}

// ||A^+||_2 for the mr x nc matrix A (1 / its smallest nonzero-rank singular
// value), from the Gram of the smaller side: G = A^T A (mr >= nc) or A A^T,
// Cholesky G = R^T R, G^{-1} = R^{-1} R^{-T}, and power iteration on G^{-1}
// (lambda_max(G^{-1}) = 1 / sigma_min^2).  Returns +inf when G is numerically
// singular.  G, Ri are k x k work areas (k = min(mr, nc)), vec holds 2k values.
template <typename TC>
__device__ inline double blk_inv_smin(const TC* A, int lda, int mr, int nc, TC* G, TC* Ri, int ldg, TC* vec,
                                      int* flag) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const bool tall = mr >= nc;
  const int k = tall ? nc : mr, len = tall ? mr : nc;
  __shared__ double red_i[32];
  if (k == 0) return INFINITY;
  for (int e = tid; e < k * k; e += nt) {
    const int i = e % k, j = e / k;
    if (i > j) continue;
    TC s = 0;
    for (int l = 0; l < len; ++l) {
      const TC x = tall ? A[(int64_t)i * lda + l] : A[(int64_t)l * lda + i];
      const TC y = tall ? A[(int64_t)j * lda + l] : A[(int64_t)l * lda + j];
      s = fma(x, y, s);
    }
    G[(int64_t)j * ldg + i] = s;
  }
  if (tid == 0) *flag = 0;
  __syncthreads();
  // Cholesky (upper R in the upper triangle of G).
  for (int j = 0; j < k; ++j) {
    const TC d = G[(int64_t)j * ldg + j];
    const bool bad = !(d > (TC)0);
    if (bad) {
      if (tid == 0) *flag = 1;
      break;
    }
    const TC rjj = sqrt(d);
    __syncthreads();
    for (int l = j + 1 + tid; l < k; l += nt) G[(int64_t)l * ldg + j] /= rjj;
    if (tid == 0) G[(int64_t)j * ldg + j] = rjj;
    __syncthreads();
    const int t = k - j - 1;
    for (int e = tid; e < t * t; e += nt) {
      const int a = e % t, b = e / t;
      if (a > b) continue;
      G[(int64_t)(j + 1 + b) * ldg + (j + 1 + a)] -= G[(int64_t)(j + 1 + a) * ldg + j] * G[(int64_t)(j + 1 + b) * ldg + j];
    }
    __syncthreads();
  }
  __syncthreads();
  if (*flag) return INFINITY;
  // Ri = R^{-1} (upper), column l by back substitution.
  for (int l = tid; l < k; l += nt) {
    for (int i = k - 1; i > l; --i) Ri[(int64_t)l * ldg + i] = (TC)0;
    for (int i = l; i >= 0; --i) {
      TC s = (i == l) ? (TC)1 : (TC)0;
      for (int c = i + 1; c <= l; ++c) s -= G[(int64_t)c * ldg + i] * Ri[(int64_t)l * ldg + c];
      Ri[(int64_t)l * ldg + i] = s / G[(int64_t)i * ldg + i];
    }
  }
  __syncthreads();
  // Power iteration on G^{-1} = Ri Ri^T: x <- Ri (Ri^T x).
  TC* x = vec;
  TC* y = vec + k;
  for (int i = tid; i < k; i += nt) x[i] = (TC)1 / sqrt((TC)k) * (TC)(1 + (i & 1));
  __syncthreads();
  double lam = 0.0;
  for (int it = 0; it < 30; ++it) {
    for (int i = tid; i < k; i += nt) {  // y = Ri^T x
      TC s = 0;
      for (int c = 0; c <= i; ++c) s = fma(Ri[(int64_t)i * ldg + c], x[c], s);
      y[i] = s;
    }
    __syncthreads();
    double nrm = 0.0;
    for (int i = tid; i < k; i += nt) {  // x_new = Ri y
      TC s = 0;
      for (int c = i; c < k; ++c) s = fma(Ri[(int64_t)c * ldg + i], y[c], s);
      nrm += (double)s * (double)s;
    }
    nrm = block_sum(nrm, red_i);
    const double prev = lam;
    double xx = 0.0;
    for (int i = tid; i < k; i += nt) xx += (double)x[i] * (double)x[i];
    xx = block_sum(xx, red_i);
    lam = sqrt(nrm / xx);  // ||G^{-1} x|| / ||x|| -> lambda_max(G^{-1})
    for (int i = tid; i < k; i += nt) {
      TC s = 0;
      for (int c = i; c < k; ++c) s = fma(Ri[(int64_t)c * ldg + i], y[c], s);
      x[i] = s / (TC)sqrt(nrm);
    }
    __syncthreads();
    if (it > 3 && fabs(lam - prev) <= 1e-3 * lam) break;
  }
  return sqrt(lam);
}

}  // namespace lrp
