// Small dense routines of the per-problem cores: one-sided Jacobi SVD and a
// descending sort permutation (block-cooperative), the Gram of a small matrix
// (block) and ||A^+||_2 from it (one warp).
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
// undone on exit), so that squared column norms cannot underflow in FP32.  In
// FP64 a round is split in three phases (the half-warps' dot products; one
// lane per pair of warp 0 computing every rotation; the rotations), because the
// FP64 pipe charges a warp instruction for all 32 lanes whatever its mask: one
// warp then issues the rotation arithmetic of the whole round.  A
// pair is left alone once |a_i . a_j| <= mr eps ||a_i|| ||a_j|| (rounding noise)
// or one of its columns is below eps ||A||_F: such columns lie below every
// cutoff applied to the singular values (the pseudoinverse's
// max(|I|,|J|) eps sigma_1, the tail rules), and rotating them only chases
// rounding noise.
// Pair k of round rnd of the cyclic schedule over ne (even) columns, a < b;
// a = b = -1 for a pair with the padding column.
__device__ __forceinline__ void jacobi_pair(int rnd, int k, int ne, int nc, int& a, int& b) {
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

// One round of blk_jacobi in three phases (FP64): dot products a.b by
// half-warps; warp 0 tests each pair (lane per pair) and computes its rotation
// (t from zeta = (||b||^2 - ||a||^2) / (2 a.b), c = 1/sqrt(1 + t^2) by reciprocal
// square roots) and the carried norms; the half-warps rotate.
template <typename TC>
__device__ inline void jacobi_round_split(TC* A, int lda, int mr, int nc, TC* V, int ldv, int rnd, int ne, TC tol, TC nu,
                                          TC* jac_nrm, int* flag) {
  const int tid = threadIdx.x, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int half = (tid >> 4) & 1, hl = tid & 15;
  const int npairs = ne / 2;
  __shared__ TC jac_g[kMaxM / 2];
  __shared__ TC jac_c[kMaxM / 2];
  __shared__ TC jac_s[kMaxM / 2];
  for (int kw = warp; 2 * kw < npairs; kw += nwarps) {
    const int k = 2 * kw + half;
    int a = -1, b = -1;
    if (k < npairs) jacobi_pair(rnd, k, ne, nc, a, b);
    const bool valid = a >= 0;
    const TC* ca = A + (int64_t)(valid ? a : 0) * lda;
    const TC* cb = A + (int64_t)(valid ? b : 0) * lda;
    TC gamma = 0;
    if (valid)
      for (int i = hl; i < mr; i += 16) gamma = fma(ca[i], cb[i], gamma);
    gamma = half_warp_sum(gamma);
    if (k < npairs && hl == 0) jac_g[k] = gamma;
  }
  __syncthreads();
  if (warp == 0) {
    const TC tol2 = tol * tol;
    for (int k = tid; k < npairs; k += 32) {
      int a = -1, b = -1;
      jacobi_pair(rnd, k, ne, nc, a, b);
      TC c = 1, s = 0;
      if (a >= 0) {
        const TC gamma = jac_g[k];
        const TC alpha = jac_nrm[a], beta = jac_nrm[b];
        if (!(gamma == (TC)0 || gamma * gamma <= tol2 * alpha * beta || fmin(alpha, beta) <= nu)) {
          const TC zeta = (beta - alpha) / ((TC)2 * gamma);
          TC t;
          if (fabs(zeta) > (TC)1e150) {
            t = (TC)0.5 / zeta;
          } else {
            const TC w = (TC)1 + zeta * zeta;
            t = copysign((TC)1, zeta) / (fabs(zeta) + w * rsqrt(w));
          }
          c = rsqrt((TC)1 + t * t);
          s = c * t;
          jac_nrm[a] = alpha - t * gamma;
          jac_nrm[b] = beta + t * gamma;
          *flag = 1;
        }
      }
      jac_c[k] = c;
      jac_s[k] = s;
    }
  }
  __syncthreads();
  for (int kw = warp; 2 * kw < npairs; kw += nwarps) {
    const int k = 2 * kw + half;
    if (k >= npairs) continue;
    const TC s = jac_s[k];
    if (s == (TC)0) continue;
    const TC c = jac_c[k];
    int a = -1, b = -1;
    jacobi_pair(rnd, k, ne, nc, a, b);
    TC* ca = A + (int64_t)a * lda;
    TC* cb = A + (int64_t)b * lda;
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
  }
  __syncthreads();
}

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
      if constexpr (sizeof(TC) == 8) {
        jacobi_round_split<TC>(A, lda, mr, nc, V, ldv, rnd, ne, tol, nu, jac_nrm, flag);
        continue;
      }
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

// Rotation (c, s) of the pair with squared norms a, b and dot product g (FP32):
// t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), zeta = (b - a) / (2 g), from
// hardware reciprocals and reciprocal square roots (t only sets how far the
// rotation reduces a.b), c = (1 + t^2)^{-1/2} refined by one Newton step so that
// c^2 + s^2 = 1 to working precision (the rotation stays orthogonal), s = c t.
__device__ __forceinline__ void rot_params_f32(float a, float b, float g, float& c, float& sn, float& t) {
  const float zeta = __fdividef(b - a, 2.f * g);
  if (fabsf(zeta) > 1e18f) {
    t = __fdividef(0.5f, zeta);
  } else {
    const float w = fmaf(zeta, zeta, 1.f);
    t = copysignf(__fdividef(1.f, fabsf(zeta) + w * rsqrtf(w)), zeta);
  }
  const float u = fmaf(t, t, 1.f);
  const float c0 = rsqrtf(u);
  c = c0 * fmaf(-0.5f * u * c0, c0, 1.5f);
  sn = c * t;
}

// One-sided Jacobi SVD in FP32 with the columns in registers: the same
// round-robin pair ordering, stopping test and Frobenius scaling as
// blk_jacobi, one column pair per half-warp (pair k on half-warp k, P = ne/2
// <= 2 nwarps).  A column is its mr rows of A followed by its nc rows of V (V
// starts as the identity), spread over the half-warp's 16 lanes, NV2 values
// per lane (mr + nc <= 16 NV2).  The ordering moves each pair's first column to
// pair k-1 (pair 0's to pair 1's second place) and each second column to pair
// k+1 (the last pair's into its own first place; pair 0's second column
// stays), which reproduces the cyclic schedule (a, b) = ((rnd + k) mod (ne-1),
// (rnd - k) mod (ne-1)), pair 0 = (rnd mod (ne-1), ne-1).  The moving columns
// and their carried squared norms pass through `buf` (2P columns of 16 NV2
// floats; twice that with `dbl`: alternate halves and one barrier per round,
// else two barriers per round).  After each sweep (ne-1 rounds, the schedule's
// period) the columns are back in their starting pairs.
template <int NV2>
__device__ inline void blk_jacobi_hreg(float* A, int lda, int mr, int nc, float* V, int ldv, double* sig, float* buf,
                                       bool dbl, double* jr_red, float* jr_nrm) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nwarps = blockDim.x >> 5;
  const int hl = lane & 15, k = tid >> 4;  // this half-warp's pair
  const int ne = nc + (nc & 1), P = ne >> 1, R = ne - 1, rows = mr + nc;
  constexpr int S = 16 * NV2;
  double f2 = 0.0;
  for (int e = tid; e < mr * nc; e += blockDim.x) {
    const double v = (double)A[(int64_t)(e / mr) * lda + (e % mr)];
    f2 = fma(v, v, f2);
  }
  f2 = warp_sum(f2);
  if (lane == 0) jr_red[warp] = f2;
  __syncthreads();
  if (tid < 32) {
    double v = tid < nwarps ? jr_red[tid] : 0.0;
    v = warp_sum(v);
    if (tid == 0) jr_red[0] = v;
  }
  __syncthreads();
  const double fro2 = jr_red[0];
  int ex = 0;
  if (fro2 > 0.0) frexp(sqrt(fro2), &ex);
  const float down = (float)ldexp(1.0, -ex), up = (float)ldexp(1.0, ex);
  const bool live = k < P;
  float x[NV2], y[NV2];
  {
    const int ia = k, ib = (k == 0) ? ne - 1 : ne - 1 - k;
#pragma unroll
    for (int v = 0; v < NV2; ++v) {
      const int e = hl + 16 * v;
      float xv = 0.f, yv = 0.f;
      if (live && e < rows) {
        if (e < mr) {
          if (ia < nc) xv = A[(int64_t)ia * lda + e] * down;
          if (ib < nc) yv = A[(int64_t)ib * lda + e] * down;
        } else {
          xv = (e - mr == ia) ? 1.f : 0.f;
          yv = (e - mr == ib) ? 1.f : 0.f;
        }
      }
      x[v] = xv;
      y[v] = yv;
    }
  }
  // exchange destinations of this pair's two columns (fixed for the solve)
  const int da = (k >= 1) ? 2 * (k - 1) : 3;
  const int db = (k == 0) ? -1 : ((k <= P - 2) ? 2 * (k + 1) + 1 : 2 * (P - 1));
  const float tol = (float)((double)(mr > 1 ? mr : 1) * Eps<float>::value);
  const float tol2 = tol * tol;
  const float nu = (float)(Eps<float>::value * Eps<float>::value);
  int par = 0;
  float al = 0.f, be = 0.f;
  for (int sweep = 0; sweep < kJacobiSweeps && ne >= 2; ++sweep) {
    {
      float sa = 0.f, sb = 0.f;
#pragma unroll
      for (int v = 0; v < NV2; ++v)
        if (hl + 16 * v < mr) {
          sa = fmaf(x[v], x[v], sa);
          sb = fmaf(y[v], y[v], sb);
        }
      al = half_warp_sum(sa);
      be = half_warp_sum(sb);
    }
    int rot = 0;
    for (int rnd = 0; rnd < R; ++rnd) {
      float g = 0.f;
#pragma unroll
      for (int v = 0; v < NV2; ++v)
        if (hl + 16 * v < mr) g = fmaf(x[v], y[v], g);
      g = half_warp_sum(g);
      if (live && !(g == 0.f || g * g <= tol2 * al * be || fminf(al, be) <= nu)) {
        float c, sn, t;
        rot_params_f32(al, be, g, c, sn, t);
#pragma unroll
        for (int v = 0; v < NV2; ++v) {
          const float xv = x[v], yv = y[v];
          x[v] = c * xv - sn * yv;
          y[v] = sn * xv + c * yv;
        }
        al = al - t * g;
        be = be + t * g;
        rot = 1;
      }
      if (P > 1) {
        float* bw = buf + (dbl ? par : 0) * (2 * P * S);
        float* nw = jr_nrm + (dbl ? par : 0) * (2 * P);
        if (live) {
#pragma unroll
          for (int v = 0; v < NV2; ++v) bw[da * S + hl + 16 * v] = x[v];
          if (hl == 0) nw[da] = al;
          if (db >= 0) {
#pragma unroll
            for (int v = 0; v < NV2; ++v) bw[db * S + hl + 16 * v] = y[v];
            if (hl == 0) nw[db] = be;
          }
        }
        __syncthreads();
        if (live) {
#pragma unroll
          for (int v = 0; v < NV2; ++v) x[v] = bw[2 * k * S + hl + 16 * v];
          al = nw[2 * k];
          if (k >= 1) {
#pragma unroll
            for (int v = 0; v < NV2; ++v) y[v] = bw[(2 * k + 1) * S + hl + 16 * v];
            be = nw[2 * k + 1];
          }
        }
        if (dbl)
          par ^= 1;
        else
          __syncthreads();
      }
    }
    if (!__syncthreads_or(rot)) break;
  }
  {
    // every lane takes part in the half-warp sums; only live pairs store
    const int ia = k, ib = (k == 0) ? ne - 1 : ne - 1 - k;
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const int col = side ? ib : ia;
      const bool st = live && col < nc;
      float s2 = 0.f;
#pragma unroll
      for (int v = 0; v < NV2; ++v) {
        const int e = hl + 16 * v;
        const float val = side ? y[v] : x[v];
        if (e < mr) {
          const float u = val * up;
          s2 = fmaf(u, u, s2);
          if (st) A[(int64_t)col * lda + e] = u;
        } else if (e < rows && st) {
          V[(int64_t)col * ldv + (e - mr)] = val;
        }
      }
      s2 = half_warp_sum(s2);
      if (hl == 0 && st) sig[col] = sqrt((double)s2);
    }
  }
  __syncthreads();
}

// FP32 one-sided Jacobi SVD (blk_jacobi's contract, V required): the register
// form when the sizes fit it (mr + nc <= 96, ne/2 <= 2 nwarps and <= 32,
// `buf_floats` covering one set of 2P columns), else blk_jacobi<float>.
__device__ inline void blk_jacobi_f32(float* A, int lda, int mr, int nc, float* V, int ldv, double* sig, int* flag,
                                      float* buf, int buf_floats) {
  const int ne = nc + (nc & 1), P = ne >> 1, rows = mr + nc;
  const int nv2 = (rows + 15) >> 4;
  const int need = 2 * P * 16 * nv2;
  const bool fits = nc >= 1 && P <= 2 * (int)(blockDim.x >> 5) && P <= 32 && nv2 <= 6 && need <= buf_floats;
  if (!fits) {
    blk_jacobi<float>(A, lda, mr, nc, V, ldv, sig, flag);
    return;
  }
  const bool dbl = 2 * need <= buf_floats;
  __shared__ double jr_red[32];     // block reduction of ||A||_F^2
  __shared__ float jr_nrm[2 * 64];  // carried squared norms of the moving columns
  switch (nv2) {
    case 1: blk_jacobi_hreg<1>(A, lda, mr, nc, V, ldv, sig, buf, dbl, jr_red, jr_nrm); break;
    case 2: blk_jacobi_hreg<2>(A, lda, mr, nc, V, ldv, sig, buf, dbl, jr_red, jr_nrm); break;
    case 3: blk_jacobi_hreg<3>(A, lda, mr, nc, V, ldv, sig, buf, dbl, jr_red, jr_nrm); break;
    case 4: blk_jacobi_hreg<4>(A, lda, mr, nc, V, ldv, sig, buf, dbl, jr_red, jr_nrm); break;
    case 5: blk_jacobi_hreg<5>(A, lda, mr, nc, V, ldv, sig, buf, dbl, jr_red, jr_nrm); break;
    default: blk_jacobi_hreg<6>(A, lda, mr, nc, V, ldv, sig, buf, dbl, jr_red, jr_nrm); break;
  }
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

// G = A^T A (mr >= nc) or A A^T (mr < nc), upper triangle, for the mr x nc
// matrix A (col-major, lda); k = min(mr, nc) is returned.  Block-cooperative:
// the caller synchronises before G is read.
template <typename TC>
__device__ inline int blk_gram_upper(const TC* A, int lda, int mr, int nc, TC* G, int ldg) {
  const bool tall = mr >= nc;
  const int k = tall ? nc : mr, len = tall ? mr : nc;
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
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
  return k;
}

// ||A^+||_2 = 1 / sigma_min(A) from the k x k Gram G of the smaller side (upper
// triangle filled by blk_gram_upper), by ONE warp (warp-synchronous; the other
// warps of the block are free): Cholesky G = R^T R in place, Ri = R^{-1} by back
// substitution, and power iteration on G^{-1} = Ri Ri^T, whose largest
// eigenvalue is 1 / sigma_min^2, to a relative change of 1e-3 (at least 5 and at
// most 30 steps).  Returns +inf when G is numerically singular (a pivot not > 0)
// and for k = 0.  vec holds 2k values.
template <typename TC>
__device__ inline double warp_inv_smin(TC* G, TC* Ri, int ldg, int k, TC* vec) {
  const int lane = threadIdx.x & 31;
  if (k == 0) return INFINITY;
  for (int j = 0; j < k; ++j) {
    const TC d = G[(int64_t)j * ldg + j];
    if (!(d > (TC)0)) return INFINITY;  // every lane reads the same pivot
    const TC rjj = sqrt(d);
    for (int l = j + 1 + lane; l < k; l += 32) G[(int64_t)l * ldg + j] /= rjj;
    __syncwarp();
    if (lane == 0) G[(int64_t)j * ldg + j] = rjj;
    const int t = k - j - 1;
    for (int e = lane; e < t * t; e += 32) {
      const int a = e % t, b = e / t;
      if (a > b) continue;
      G[(int64_t)(j + 1 + b) * ldg + (j + 1 + a)] -= G[(int64_t)(j + 1 + a) * ldg + j] * G[(int64_t)(j + 1 + b) * ldg + j];
    }
    __syncwarp();
  }
  for (int l = lane; l < k; l += 32) {
    for (int i = k - 1; i > l; --i) Ri[(int64_t)l * ldg + i] = (TC)0;
    for (int i = l; i >= 0; --i) {
      TC s = (i == l) ? (TC)1 : (TC)0;
      for (int c = i + 1; c <= l; ++c) s -= G[(int64_t)c * ldg + i] * Ri[(int64_t)l * ldg + c];
      Ri[(int64_t)l * ldg + i] = s / G[(int64_t)i * ldg + i];
    }
  }
  TC* x = vec;
  TC* y = vec + k;
  for (int i = lane; i < k; i += 32) x[i] = (TC)1 / sqrt((TC)k) * (TC)(1 + (i & 1));
  __syncwarp();
  double lam = 0.0;
  for (int it = 0; it < 30; ++it) {
    for (int i = lane; i < k; i += 32) {  // y = Ri^T x
      TC s = 0;
      for (int c = 0; c <= i; ++c) s = fma(Ri[(int64_t)i * ldg + c], x[c], s);
      y[i] = s;
    }
    __syncwarp();
    double nrm = 0.0, xx = 0.0;
    for (int i = lane; i < k; i += 32) {  // ||Ri y||^2 and ||x||^2
      TC s = 0;
      for (int c = i; c < k; ++c) s = fma(Ri[(int64_t)c * ldg + i], y[c], s);
      nrm += (double)s * (double)s;
      xx += (double)x[i] * (double)x[i];
    }
    nrm = warp_sum(nrm);
    xx = warp_sum(xx);
    const double prev = lam;
    lam = sqrt(nrm / xx);  // ||G^{-1} x|| / ||x|| -> lambda_max(G^{-1})
    for (int i = lane; i < k; i += 32) {  // x <- Ri y / ||Ri y||
      TC s = 0;
      for (int c = i; c < k; ++c) s = fma(Ri[(int64_t)c * ldg + i], y[c], s);
      x[i] = s / (TC)sqrt(nrm);
    }
    __syncwarp();
    if (it > 3 && fabs(lam - prev) <= 1e-3 * lam) break;
  }
  return sqrt(lam);
}

}  // namespace lrp
