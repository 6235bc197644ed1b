// Per-problem kernels of the Cross-DEIM iteration: one CTA per problem (or per
// problem and side), FP64 small dense linear algebra on m x m matrices
// (m = |I|, |J| <= m_cap) held in an L2-resident per-problem scratch area.
//
//  k_chol      one pass of shifted CholeskyQR: Cholesky of the reduced Gram
//              with pivot dropping, R^{-1}, and the accumulated R = R_k ... R_1
//              whose diagonal is Algorithm scross's r_C / r_R.
//  k_core      the small part of Algorithm scross: Q(I,:), the pseudoinverse
//              solve (branch |J| <= |I| or its mirror), the SVD of the core,
//              the in-loop truncation, the redundancy removal of Algorithm
//              Cross-DEIM and the DEIM constants eta_1, eta_2.
//  k_select    index enrichment of Algorithm Cross-DEIM: top-c leverage
//              candidates, ordered union with the previous set and the growth
//              safeguard (one index from the complement).
//  k_stop      rho = ||A_k - A_{k-1}||_F / ||S_k||_F from small Gram terms and
//              the stop test max(rho, min(eta1(1+eta2), eta2(1+eta1)) S_min) < eps.
//  k_finalize  final truncation sum_{l>r} S_l^2 < eps^2 ||S||^2, r = max(min(r*, r_max), 1).
//
// Singular value decompositions use one-sided (Hestenes) Jacobi with the
// round-robin pair ordering; each warp rotates one column pair at a time.
#include <cuda_runtime.h>
#include <math.h>

#include "common.cuh"
#include "core.cuh"
#include "dense.cuh"
#include "dst.cuh"
#include "f64cvt.cuh"

namespace lrp {

namespace {
constexpr int CT = 256;  // threads of the Cholesky and stop CTAs
// Threads of a k_core CTA: 16 warps = 32 half-warps, one Jacobi column pair
// each, so that a round of up to 64 columns takes one pass; two CTAs per SM.
constexpr int CTC = 512;
}  // namespace

// ------------------------------------------------------- work accounting

__device__ inline void acct_add(double* row, int cls, double flops, double bytes) {
  row[2 * cls] += flops;
  row[2 * cls + 1] += bytes;
}

// Algorithmic flops of one orthonormal DST-I column: a real FFT of length N
// (one complex FFT of length N/2, 2.5 N log2 N), the count of a transform that
// uses the odd symmetry (the pre- and post-processing add O(N)).
__device__ inline double dst_col_flops(int n) {
  const double N = (double)(n + 1);
  return 2.5 * N * log2(N);
}

// Three symmetric Gram passes, two triangular applies, on side sizes m0, m1.
// FP32 data (w == 4) run every pass on the FP32 pipe, pass 1 in double-float.
__device__ inline void acct_cholqr3(double* row, double n, double m0, double m1, int NB, double w) {
  for (double m : {m0, m1}) {
    const double gf = n * m * (m + 1.0), gb = n * m * w + NB * m * (m + 1.0) / 2.0 * 8.0;
    if (w == 4.0) {
      acct_add(row, LRP_K_GRAM_DF, gf, gb);
      acct_add(row, LRP_K_GRAM_F32, 2.0 * gf, 2.0 * gb);
    } else {
      acct_add(row, LRP_K_GRAM, 3.0 * gf, 3.0 * gb);
    }
    acct_add(row, LRP_K_REDUCE, 3.0 * NB * m * (m + 1.0) / 2.0, 3.0 * (NB + 1.0) * m * (m + 1.0) / 2.0 * 8.0);
    acct_add(row, w == 4.0 ? LRP_K_GEMM_F32 : LRP_K_GEMM, 2.0 * n * m * (m + 1.0), 2.0 * 2.0 * n * m * w);
  }
}

__device__ void acct_setup(double* row, int n_, int rf_, int NB, int w_) {
  const double n = n_, rf = rf_, w = w_;
  acct_add(row, LRP_K_DST, 2.0 * rf * dst_col_flops(n_), 2.0 * rf * n * (8.0 + w));
  acct_cholqr3(row, n, rf, rf, NB, w);
  acct_add(row, w_ == 4 ? LRP_K_GEMM_F32 : LRP_K_GEMM, 2.0 * n * rf * (rf + 1.0), 2.0 * 2.0 * n * rf * w);  // U_{-1}
  acct_add(row, LRP_K_LEVERAGE, 2.0 * 2.0 * n * rf, 2.0 * n * rf * w);
}

__device__ void acct_iteration(double* row, int n_, int p_, int q_, int r_, int rp_, int rf_, int NB, int w_) {
  const double n = n_, p = p_, q = q_, r = r_, rp = rp_, rf = rf_, w = w_;
  // side 0 columns: p = |J|; side 1 columns: q = |I|
  acct_add(row, LRP_K_CROSS, 2.0 * n * rf * (p + q), w * (2.0 * n * rf + n * (p + q) + n));
  acct_cholqr3(row, n, p, q, NB, w);
  const int mcls = (w_ == 4) ? LRP_K_GEMM_F32 : LRP_K_GEMM;
  acct_add(row, mcls, 2.0 * n * r * (p + q), w * n * (p + q + 2.0 * r));  // U_k = Q2 Bf
  acct_add(row, LRP_K_LEVERAGE, 2.0 * 2.0 * n * r, 2.0 * n * r * w);
  const int gcls = (w_ == 4) ? LRP_K_GRAM_F32 : LRP_K_GRAM;
  if (rp_ > 0) {
    acct_add(row, gcls, 2.0 * 2.0 * n * r * rp, 2.0 * (n * (r + rp) * w + NB * r * rp * 8.0));
    acct_add(row, LRP_K_REDUCE, 2.0 * NB * r * rp, 2.0 * (NB + 1.0) * r * rp * 8.0);
    acct_add(row, mcls, 2.0 * 2.0 * n * r * rp, 2.0 * n * (r + 2.0 * rp) * w);
    acct_add(row, gcls, 2.0 * n * rp * (rp + 1.0), 2.0 * (n * rp * w + NB * rp * (rp + 1.0) / 2.0 * 8.0));
    acct_add(row, LRP_K_REDUCE, 2.0 * NB * rp * (rp + 1.0) / 2.0, 2.0 * (NB + 1.0) * rp * (rp + 1.0) / 2.0 * 8.0);
  }
}

__device__ void acct_back(double* row, int n_, int r_out, int w_, bool df) {
  const double n = n_, w = w_;
  acct_add(row, df ? LRP_K_DST_DF : LRP_K_DST, 2.0 * r_out * dst_col_flops(n_), 2.0 * r_out * n * (8.0 + w));
}

// ------------------------------------------------------------------- kernels

// FP32 <-> FP64 conversions of the small matrices on the integer pipe
// (f64cvt.cuh: the same values as the hardware conversions, which GB300 runs
// on its FP64 pipe).
__device__ __forceinline__ double widen64(double x) { return x; }
__device__ __forceinline__ double widen64(float x) { return f32_to_f64(x); }
template <typename TC>
__device__ __forceinline__ TC narrow_to(double x) {
  if constexpr (sizeof(TC) == 4) {
    return f64_to_f32_rn(x);
  } else {
    return x;
  }
}

constexpr int kCholSmemDim = 64;
constexpr size_t kCholSmemBytes = kCholSmemDim * kCholSmemDim * sizeof(double);

// Column l of X = R^{-1} for each of the CTA's warps in turn (columns l = wid,
// wid + nw, ...): back substitution in axpy form, lanes owning rows
// i' = lane + 32 q of the running sums s(i') = -sum_{k > i'} R(i', k) x_k, so
// that each step is one shuffle and one update per lane.  Dropped pivots give
// zero rows; entries below the diagonal are zeroed.
template <typename TC, int Q>
__device__ void chol_inverse_cols(const TC* __restrict__ W, int Lc, TC* __restrict__ X, int ldx, int m,
                                  const TC* __restrict__ rinv, const int* __restrict__ dropped) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int l = wid; l < m; l += nw) {
    TC acc[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) acc[q] = TC(0);
    for (int i = l; i >= 0; --i) {
      TC si = TC(0);
#pragma unroll
      for (int q = 0; q < Q; ++q)
        if (q == (i >> 5)) si = acc[q];
      si = __shfl_sync(0xffffffffu, si, i & 31);
      const TC xi = dropped[i] ? TC(0) : ((i == l ? TC(1) : TC(0)) + si) * rinv[i];
      if (lane == (i & 31)) X[(int64_t)l * ldx + i] = xi;
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const int ip = lane + 32 * q;
        if (ip < i) acc[q] -= W[(int64_t)i * Lc + ip] * xi;
      }
    }
    for (int i = l + 1 + lane; i < m; i += 32) X[(int64_t)l * ldx + i] = TC(0);
  }
}

// Shifted/equilibrated Cholesky of one pass of CholeskyQR for every (problem,
// side): R with R^T R = G (+ shift), P = R^{-1} and the accumulated R.  TC is the
// arithmetic type: FP64 for the FP64 path and for the first (ill-conditioned)
// pass of the FP32 iterations, FP32 for their later passes, whose Grams are
// near the identity.
template <typename T, typename TC>
__global__ void __launch_bounds__(CT) k_chol(CoreParams p, CoreBufs<T> b, int sel, int pass) {
  extern __shared__ __align__(16) unsigned char chol_raw[];
  const int slot = slot_of(p.g, blockIdx.x >> 1), side = blockIdx.x & 1;
  if (slot < 0) return;
  SolveState* stp = p.st + slot;
  if (!stp->active) return;
  const int M = p.g.M;
  const int m = dim_of(*stp, side, sel);
  const double* G = b.G.at(slot, side);
  // Working triangle W: shared memory (leading dimension kCholSmemDim) when
  // m <= kCholSmemDim, else the slot's global scratch (leading dimension M).
  // The R^{-1} / product buffer Tm is in the slot's scratch (leading
  // dimension M, L2-resident): the inverse only writes it.
  const bool in_smem = m <= kCholSmemDim;
  const int Lc = in_smem ? kCholSmemDim : M;
  double* base = b.scratch + (int64_t)slot * b.scratch_stride;
  TC* W = in_smem ? reinterpret_cast<TC*>(chol_raw) : reinterpret_cast<TC*>(base + (int64_t)(8 + side) * M * M);
  TC* Tm = reinterpret_cast<TC*>(base + (int64_t)(10 + side) * M * M);
  double* P = b.P.at(slot, side);
  double* Racc = b.Racc.at(slot, side);
  __shared__ double red[32];
  __shared__ int dropped[kMaxM];
  __shared__ double dsc[kMaxM];
  __shared__ TC rinv[kMaxM];
  const int tid = threadIdx.x, nt = blockDim.x;

  // Pass 0 equilibrates: W = D G D with D = diag(G_jj^{-1/2}) (zero columns are
  // dropped), so R = R' D^{-1} and R^{-1} = D R'^{-1}; the relative diagonal test
  // on R is unchanged and the shift acts on unit-diagonal data.
  for (int j = tid; j < m; j += nt) {
    const double gjj = G[(int64_t)j * M + j];
    dsc[j] = (pass == 0) ? ((gjj > 0.0) ? 1.0 / sqrt(gjj) : 0.0) : 1.0;
  }
  __syncthreads();
  double tr = 0.0, mx = 0.0;
  for (int e = tid; e < m * m; e += nt) {
    const int i = e % m, j = e / m;
    const double v = G[(int64_t)j * M + i] * dsc[i] * dsc[j];
    W[(int64_t)j * Lc + i] = (i <= j) ? (TC)v : TC(0);
    if (i == j) {
      tr += v;
      mx = fmax(mx, v);
    }
  }
  tr = block_sum(tr, red);
  mx = block_max(mx, red);
  const double shift = (pass == 0) ? p.shift_rel * tr : 0.0;
  if (pass == 0 && tid == 0) stp->gram_trace[side] = tr;
  for (int j = tid; j < m; j += nt) W[(int64_t)j * Lc + j] += (dsc[j] > 0.0) ? (TC)shift : TC(0);
  const TC thr = (pass == 0) ? TC(0) : (TC)(p.drop_rel * mx);
  __syncthreads();

  // Right-looking factorisation.  The pivot's square root and reciprocal are
  // taken by one thread and shared (on GB300 an FP64 square root or division
  // by every thread of the CTA would occupy the FP64 pipe for thousands of
  // cycles per pivot); the trailing update gives warp w the columns
  // l = j+1+w, j+1+w+nw, ... and its lanes the rows k of column l.
  const int lane = tid & 31, wid = tid >> 5, nwarp = nt >> 5;
  for (int j = 0; j < m; ++j) {
    if (tid == 0) {
      const TC d = W[(int64_t)j * Lc + j];
      const bool drop = !(d > thr);
      const TC rjj = drop ? TC(0) : sqrt(d);
      W[(int64_t)j * Lc + j] = rjj;
      dropped[j] = drop ? 1 : 0;
      rinv[j] = drop ? TC(0) : TC(1) / rjj;
    }
    __syncthreads();
    const TC ri = rinv[j];
    for (int l = j + 1 + tid; l < m; l += nt) {
      TC* wl = W + (int64_t)l * Lc + j;
      *wl = *wl * ri;
    }
    __syncthreads();
    if (!dropped[j]) {
      for (int l = j + 1 + wid; l < m; l += nwarp) {
        const TC wlj = W[(int64_t)l * Lc + j];
        for (int k = j + 1 + lane; k <= l; k += 32) W[(int64_t)l * Lc + k] -= W[(int64_t)k * Lc + j] * wlj;
      }
    }
    __syncthreads();
  }

  // P = R^{-1} (dropped rows give zeros)
  if (m <= 64)
    chol_inverse_cols<TC, 2>(W, Lc, Tm, M, m, rinv, dropped);
  else
    chol_inverse_cols<TC, kMaxM / 32>(W, Lc, Tm, M, m, rinv, dropped);
  __syncthreads();
  // (warp w: columns j = w, w + nw, ...; lanes: rows i)
  for (int j = wid; j < m; j += nwarp)
    for (int i = lane; i < m; i += 32) P[(int64_t)j * M + i] = dsc[i] * widen64(Tm[(int64_t)j * M + i]);
  __syncthreads();
  // Racc <- R (pass 0, undoing the equilibration) or R * Racc.
  if (pass == 0) {
    for (int j = wid; j < m; j += nwarp)
      for (int i = lane; i < m; i += 32)
        Racc[(int64_t)j * M + i] = (i <= j && dsc[j] > 0.0) ? widen64(W[(int64_t)j * Lc + i]) / dsc[j] : 0.0;
  } else {
    for (int l = wid; l < m; l += nwarp) {
      for (int i = lane; i < m; i += 32) {
        TC s = TC(0);
        if (i <= l)
          for (int k = i; k <= l; ++k) s += W[(int64_t)k * Lc + i] * narrow_to<TC>(Racc[(int64_t)l * M + k]);
        Tm[(int64_t)l * M + i] = s;
      }
    }
    __syncthreads();
    for (int j = wid; j < m; j += nwarp)
      for (int i = lane; i < m; i += 32) Racc[(int64_t)j * M + i] = widen64(Tm[(int64_t)j * M + i]);
  }
}

// Small matrices of k_core live in six regions of L x L doubles: shared memory
// when |I|, |J| <= core_smem_dim (L = that), else the slot's global scratch
// (L = M).  Region use: R0 Q(I,:) -> compaction work; R1 Z(J,:) -> eta work;
// R2 pinv work -> V of the core SVD -> V_k(J,:); R3 V of the pinv SVD -> U~;
// R4 T1 -> V~; R5 core -> U_k(I,:).
// 64 in FP32 (96 KB, two CTAs per SM: index sets of the FP32 iterations reach
// 50-60 with leverage sampling), 48 in FP64 (110 KB).
template <typename TC>
__host__ __device__ constexpr int core_smem_dim() {
  return sizeof(TC) == 4 ? 64 : 48;
}
template <typename TC>
__host__ __device__ constexpr size_t core_smem_bytes() {
  return 6 * (size_t)core_smem_dim<TC>() * core_smem_dim<TC>() * sizeof(TC);
}

// Jacobi SVD of a core matrix: FP32 cores take the register form, whose column
// exchange uses two free tiles (`free2`, 2 L^2 values); FP64 the shared-memory form.
template <typename TC>
__device__ __forceinline__ void core_jacobi(TC* A, int lda, int mr, int nc, TC* V, int ldv, double* sig, int* flag,
                                            TC* free2, int64_t free_elems) {
  if constexpr (sizeof(TC) == 4)
    blk_jacobi_f32(A, lda, mr, nc, V, ldv, sig, flag, free2, (int)(free_elems < (1 << 30) ? free_elems : (1 << 30)));
  else
    blk_jacobi<TC>(A, lda, mr, nc, V, ldv, sig, flag);
}

// The small core computes in the precision of the iteration (TC = T): FP64 for
// the FP64 solve, FP32 for the inner solves of the mixed-precision path.
template <typename T>
__global__ void __launch_bounds__(CTC, 2) k_core(CoreParams p, CoreBufs<T> b, int parity) {
  using TC = T;
  extern __shared__ double core_smem_d[];
  TC* core_smem = reinterpret_cast<TC*>(core_smem_d);
  const int slot = slot_of(p.g, blockIdx.x);
  if (slot < 0) return;
  SolveState* stp = p.st + slot;
  if (!stp->active) return;
  const int M = p.g.M;
  const int q = stp->cnt[0];   // |I|
  const int pc = stp->cnt[1];  // |J|
  if (q < 1 || pc < 1) {
    if (threadIdx.x == 0) {
      stp->active = 0;
      stp->flags |= kFlagBadInput;
    }
    return;
  }
  constexpr int kDim = core_smem_dim<T>();
  const bool in_smem = (q <= kDim && pc <= kDim);
  const int L = in_smem ? kDim : M;
  const int64_t LL = (int64_t)L * L;
  TC* base = in_smem ? core_smem : reinterpret_cast<TC*>(b.scratch + (int64_t)slot * b.scratch_stride);
  TC* R0 = base + 0 * LL;
  TC* R1 = base + 1 * LL;
  TC* R2 = base + 2 * LL;
  TC* R3 = base + 3 * LL;
  TC* R4 = base + 4 * LL;
  TC* R5 = base + 5 * LL;
  TC* QI = R0;  // q x pc
  TC* ZJ = R1;  // pc x q
  const T* Q20 = b.Q2.at(slot, 0);
  const T* Q21 = b.Q2.at(slot, 1);
  const double* P0 = b.P.at(slot, 0);
  const double* P1 = b.P.at(slot, 1);
  const double* RC = b.Racc.at(slot, 0);
  const double* RR = b.Racc.at(slot, 1);
  int32_t* I = b.idx.at(slot, 0);
  int32_t* J = b.idx.at(slot, 1);
  const int64_t ld = p.g.ld;
  __shared__ double sig1[kMaxM];
  __shared__ double sig2[kMaxM];
  __shared__ int perm[kMaxM];
  __shared__ int keep[kMaxM];
  __shared__ int flag;
  __shared__ double red[32];
  const int tid = threadIdx.x, nt = blockDim.x;

  // Q(I,:) = Q2_0(I,:) P3_0 and Z(J,:) = Q2_1(J,:) P3_1 (P3 upper triangular).
  for (int e = tid; e < q * pc; e += nt) {
    const int a = e % q, c = e / q;
    const int64_t row = I[a];
    TC s = 0;
    for (int d = 0; d <= c; ++d) s += (TC)Q20[(int64_t)d * ld + row] * narrow_to<TC>(P0[(int64_t)c * M + d]);
    QI[(int64_t)c * L + a] = s;
  }
  for (int e = tid; e < pc * q; e += nt) {
    const int a = e % pc, c = e / pc;
    const int64_t row = J[a];
    TC s = 0;
    for (int d = 0; d <= c; ++d) s += (TC)Q21[(int64_t)d * ld + row] * narrow_to<TC>(P1[(int64_t)c * M + d]);
    ZJ[(int64_t)c * L + a] = s;
  }
  __syncthreads();
  const double eps_c = Eps<TC>::value;
  const int mx = max(pc, q);
  const int branch = (pc <= q) ? 0 : 1;
  // Pseudoinverse solve and the core M (pc x q), stored as Mt in R5 (tall orientation).
  TC* W1 = R2;
  TC* V1 = R3;
  TC* T1 = R4;
  TC* Mt = R5;
  TC* V2 = R2;  // reuses W1 once T1 is formed
  int nsv;
  if (branch == 0) {
    // Q(I,:) = U1 S1 V1^T (q x pc); M = V1 S1^+ U1^T R_R^T (pc x q); Mt = M^T (q x pc).
    for (int e = tid; e < q * pc; e += nt) {
      const int i = e % q, j = e / q;
      W1[(int64_t)j * L + i] = QI[(int64_t)j * L + i];
    }
    __syncthreads();
    core_jacobi(W1, L, q, pc, V1, L, sig1, &flag, R4, 2 * LL);  // R4, R5 free
    double smax = 0.0;
    for (int j = tid; j < pc; j += nt) smax = fmax(smax, sig1[j]);
    smax = block_max(smax, red);
    const double cut = mx * eps_c * smax;
    // T1(a, c) = sum_{d >= c} W1(d, a) R_R(c, d) / sig1[a]^2   (pc x q)
    for (int e = tid; e < pc * q; e += nt) {
      const int a = e % pc, c = e / pc;
      TC s = 0;
      if (sig1[a] > cut) {
        for (int d = c; d < q; ++d) s += W1[(int64_t)a * L + d] * narrow_to<TC>(RR[(int64_t)d * M + c]);
        s /= narrow_to<TC>(sig1[a] * sig1[a]);
      }
      T1[(int64_t)c * L + a] = s;
    }
    __syncthreads();
    for (int e = tid; e < q * pc; e += nt) {
      const int c = e % q, i = e / q;
      TC s = 0;
      for (int a = 0; a < pc; ++a) s += V1[(int64_t)a * L + i] * T1[(int64_t)c * L + a];
      Mt[(int64_t)i * L + c] = s;
    }
    __syncthreads();
    core_jacobi(Mt, L, q, pc, V2, L, sig2, &flag, R3, 2 * LL);  // R3 (V1), R4 (T1) free
    nsv = pc;
  } else {
    // Mirror: Z(J,:) = U2 S2 V2^T (pc x q); M = R_C U2 S2^+ V2^T (pc x q), tall.
    for (int e = tid; e < pc * q; e += nt) {
      const int i = e % pc, j = e / pc;
      W1[(int64_t)j * L + i] = ZJ[(int64_t)j * L + i];
    }
    __syncthreads();
    core_jacobi(W1, L, pc, q, V1, L, sig1, &flag, R4, 2 * LL);
    double smax = 0.0;
    for (int j = tid; j < q; j += nt) smax = fmax(smax, sig1[j]);
    smax = block_max(smax, red);
    const double cut = mx * eps_c * smax;
    // T1(i, a) = sum_{c >= i} R_C(i, c) W1(c, a) / sig1[a]^2  (pc x q)
    for (int e = tid; e < pc * q; e += nt) {
      const int i = e % pc, a = e / pc;
      TC s = 0;
      if (sig1[a] > cut) {
        for (int c = i; c < pc; ++c) s += narrow_to<TC>(RC[(int64_t)c * M + i]) * W1[(int64_t)a * L + c];
        s /= narrow_to<TC>(sig1[a] * sig1[a]);
      }
      T1[(int64_t)a * L + i] = s;
    }
    __syncthreads();
    for (int e = tid; e < pc * q; e += nt) {
      const int i = e % pc, bb = e / pc;
      TC s = 0;
      for (int a = 0; a < q; ++a) s += T1[(int64_t)a * L + i] * V1[(int64_t)a * L + bb];
      Mt[(int64_t)bb * L + i] = s;
    }
    __syncthreads();
    core_jacobi(Mt, L, pc, q, V2, L, sig2, &flag, R3, 2 * LL);
    nsv = q;
  }
  blk_sort_desc(sig2, nsv, perm);
  const double s1 = sig2[perm[0]];
  int r = 0;
  {
    const double cut = (double)mx * p.eps_data * s1;
    for (int t = 0; t < nsv; ++t) r += (sig2[perm[t]] >= cut && sig2[perm[t]] > 0.0) ? 1 : 0;
    if (r < 1) r = 1;
  }
  // U~ (pc x r) -> R3, V~ (q x r) -> R4.  Branch 0: U~ = V2, V~ = Mt/sig; branch 1: U~ = Mt/sig, V~ = V2.
  TC* Ut = R3;
  TC* Vt = R4;
  for (int e = tid; e < pc * r; e += nt) {
    const int i = e % pc, t = e / pc;
    const int j = perm[t];
    const TC sv = narrow_to<TC>(sig2[j]);
    Ut[(int64_t)t * L + i] = (branch == 0) ? V2[(int64_t)j * L + i] : (sv > 0 ? Mt[(int64_t)j * L + i] / sv : (TC)0);
  }
  for (int e = tid; e < q * r; e += nt) {
    const int i = e % q, t = e / q;
    const int j = perm[t];
    const TC sv = narrow_to<TC>(sig2[j]);
    Vt[(int64_t)t * L + i] = (branch == 0) ? (sv > 0 ? Mt[(int64_t)j * L + i] / sv : (TC)0) : V2[(int64_t)j * L + i];
  }
  double* sig_out = b.sig + (int64_t)slot * 2 * M + (int64_t)parity * M;
  for (int t = tid; t < r; t += nt) sig_out[t] = sig2[perm[t]];
  __syncthreads();
  // Bf0 = P3_0 U~ (pc x r), Bf1 = P3_1 V~ (q x r); U_k(I,:) = Q(I,:) U~ -> R5, V_k(J,:) = Z(J,:) V~ -> R2.
  double* B0 = b.Bf.at(slot, 0);
  double* B1 = b.Bf.at(slot, 1);
  TC* UI = R5;
  TC* VJ = R2;
  for (int e = tid; e < pc * r; e += nt) {
    const int i = e % pc, t = e / pc;
    TC s = 0;
    for (int d = i; d < pc; ++d) s += narrow_to<TC>(P0[(int64_t)d * M + i]) * Ut[(int64_t)t * L + d];
    B0[(int64_t)t * M + i] = widen64(s);
  }
  for (int e = tid; e < q * r; e += nt) {
    const int i = e % q, t = e / q;
    TC s = 0;
    for (int d = i; d < q; ++d) s += narrow_to<TC>(P1[(int64_t)d * M + i]) * Vt[(int64_t)t * L + d];
    B1[(int64_t)t * M + i] = widen64(s);
  }
  for (int e = tid; e < q * r; e += nt) {
    const int a = e % q, t = e / q;
    TC s = 0;
    for (int c = 0; c < pc; ++c) s += QI[(int64_t)c * L + a] * Ut[(int64_t)t * L + c];
    UI[(int64_t)t * L + a] = s;
  }
  for (int e = tid; e < pc * r; e += nt) {
    const int a = e % pc, t = e / pc;
    TC s = 0;
    for (int c = 0; c < q; ++c) s += ZJ[(int64_t)c * L + a] * Vt[(int64_t)t * L + c];
    VJ[(int64_t)t * L + a] = s;
  }
  __syncthreads();
  // Redundancy removal: keep I_l iff |R_R(l,l)| >= tau max|diag R_R|, J_l likewise with R_C.
  double mR = 0.0, mC = 0.0;
  for (int l = tid; l < q; l += nt) mR = fmax(mR, fabs(RR[(int64_t)l * M + l]));
  for (int l = tid; l < pc; l += nt) mC = fmax(mC, fabs(RC[(int64_t)l * M + l]));
  mR = block_max(mR, red);
  mC = block_max(mC, red);
  __shared__ int permJ[kMaxM];
  __shared__ int kept[2];
  for (int l = tid; l < q; l += nt) keep[l] = (mR > 0.0 && fabs(RR[(int64_t)l * M + l]) >= p.redundancy * mR) ? 1 : 0;
  for (int l = tid; l < pc; l += nt)
    permJ[l] = (mC > 0.0 && fabs(RC[(int64_t)l * M + l]) >= p.redundancy * mC) ? 1 : 0;
  __syncthreads();
  // Compaction of each set in its order (perm / permJ: source row of U_k(I,:) / V_k(J,:)).
  if (tid == 0) {
    int w = 0;
    for (int l = 0; l < q; ++l) {
      if (keep[l]) {
        I[w] = I[l];
        perm[w] = l;
        ++w;
      }
    }
    kept[0] = w;
  }
  if (tid == (nt > 32 ? 32 : 0)) {
    int w = 0;
    for (int l = 0; l < pc; ++l) {
      if (permJ[l]) {
        J[w] = J[l];
        permJ[w] = l;
        ++w;
      }
    }
    kept[1] = w;
  }
  __syncthreads();
  const int qn = kept[0], pn = kept[1];
  // U_k(I,:) and V_k(J,:) on the reduced sets -> R0, R1; their Grams -> R3, R4.
  TC* WI = R0;
  TC* WJ = R1;
  for (int e = tid; e < qn * r; e += nt) {
    const int a = e % qn, t = e / qn;
    WI[(int64_t)t * L + a] = UI[(int64_t)t * L + perm[a]];
  }
  for (int e = tid; e < pn * r; e += nt) {
    const int a = e % pn, t = e / pn;
    WJ[(int64_t)t * L + a] = VJ[(int64_t)t * L + permJ[a]];
  }
  __syncthreads();
  const int kI = blk_gram_upper(WI, L, qn, r, R3, L);
  const int kJ = blk_gram_upper(WJ, L, pn, r, R4, L);
  __syncthreads();
  // eta_1 = ||U_k(I,:)^+||_2 (warp 0) and eta_2 = ||V_k(J,:)^+||_2 (warp 1) at the
  // same time; R5 / R2 (the gathers' sources) become the inverse factors.
  __shared__ TC vec_w[2][2 * kMaxM];
  __shared__ double eta_w[2];
  const int warp = tid >> 5, nw = nt >> 5;
  if (warp == 0) {
    const double e = warp_inv_smin(R3, R5, L, kI, vec_w[0]);
    if ((tid & 31) == 0) eta_w[0] = e;
  }
  if (warp == (nw > 1 ? 1 : 0)) {
    const double e = warp_inv_smin(R4, R2, L, kJ, vec_w[1]);
    if ((tid & 31) == 0) eta_w[1] = e;
  }
  __syncthreads();
  const double e1 = eta_w[0], e2 = eta_w[1];
  double snorm2 = 0.0;
  for (int t = tid; t < r; t += nt) snorm2 += sig_out[t] * sig_out[t];
  snorm2 = block_sum(snorm2, red);
  if (tid == 0) {
    const double snorm = sqrt(snorm2);
    const double smin = snorm > 0.0 ? sig_out[r - 1] / snorm : 0.0;
    const double f = fmin(e1 * (1.0 + e2), e2 * (1.0 + e1));
    stp->eta_smin = snorm > 0.0 ? f * smin : 0.0;
    // Mixed-precision inner solves: singular values at the data's noise floor
    // cannot be resolved further, so the index set is as rich as the data allow.
    if (p.noise_floor_stop && sig_out[r - 1] <= 16.0 * (double)mx * p.eps_data * s1) stp->eta_smin = 0.0;
    stp->snorm = snorm;
    if (b.acct)
      acct_iteration(b.acct + (int64_t)slot * 2 * LRP_K_COUNT, p.g.n, pc, q, r, stp->r_prev, stp->rf, p.g.NB,
                     (int)sizeof(T));
    stp->r = r;
    stp->cnt_next[0] = qn;
    stp->cnt_next[1] = pn;
    stp->branch = branch;
  }
}

// Index enrichment (Algorithm Cross-DEIM): side s merges its leverage candidates.
template <typename T>
__global__ void k_select(CoreParams p, CoreBufs<T> b, int sel_c, int sort_len) {
  extern __shared__ unsigned char smem_raw[];
  double* key = reinterpret_cast<double*>(smem_raw);
  int* id = reinterpret_cast<int*>(key + sort_len);
  const int slot = slot_of(p.g, blockIdx.x >> 1), side = blockIdx.x & 1;
  if (slot < 0) return;
  SolveState* stp = p.st + slot;
  if (!stp->active) return;
  const int M = p.g.M;
  const int n = p.g.n;
  const int c = dim_of(*stp, side, sel_c);
  const int total = p.cand_blocks * p.cand_per_block;
  const int64_t base = (int64_t)(slot * 2 + side) * total;
  // Top-c merge of all candidates in chunks that fit the shared sort buffer: each
  // pass sorts the current best c entries together with the next chunk.  The
  // Bernoulli selector keeps every sampled candidate (up to kMaxM), best first.
  const bool take_all = p.selector == LRP_SEL_BERNOULLI;
  const int cc0 = take_all ? kMaxM : min(c, kMaxM);
  const int chunk = (total <= sort_len) ? sort_len : sort_len - kMaxM;
  int have = 0;  // best entries kept at key[0..have)
  for (int start = 0; start < total; start += chunk) {
    const int cnt = min(chunk, total - start);
    for (int t = threadIdx.x; t < sort_len; t += blockDim.x) {
      if (t < have) continue;  // keep the running best list in place
      const int src_i = t - have;
      double kv = -1.0;
      int iv = 0x7fffffff;
      if (src_i < cnt) {
        const int32_t ci = b.cand_idx[base + start + src_i];
        if (ci >= 0) {
          kv = b.cand_score[base + start + src_i];
          iv = ci;
        }
      }
      key[t] = kv;
      id[t] = iv;
    }
    __syncthreads();
    // bitonic sort (score desc, index asc)
    for (int size = 2; size <= sort_len; size <<= 1) {
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        for (int t = threadIdx.x; t < sort_len; t += blockDim.x) {
          const int pp = t ^ stride;
          if (pp > t) {
            const bool up = ((t & size) == 0);
            const bool tf = (key[t] > key[pp]) || (key[t] == key[pp] && id[t] < id[pp]);
            if (up != tf) {
              const double kk = key[t];
              key[t] = key[pp];
              key[pp] = kk;
              const int ii = id[t];
              id[t] = id[pp];
              id[pp] = ii;
            }
          }
        }
        __syncthreads();
      }
    }
    have = min(cc0, sort_len);
  }
  int32_t* set = b.idx.at(slot, side);
  __shared__ int isnew[kMaxM];
  const int cnt0 = stp->cnt[side];
  const int cc = min(take_all ? kMaxM : c, min(sort_len, kMaxM));
  for (int t = threadIdx.x; t < cc; t += blockDim.x) {
    int nw = (key[t] >= 0.0) ? 1 : 0;
    if (nw) {
      const int v = id[t];
      for (int l = 0; l < cnt0; ++l)
        if (set[l] == v) {
          nw = 0;
          break;
        }
    }
    isnew[t] = nw;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int cnt = cnt0;
    for (int t = 0; t < cc && cnt < M; ++t)
      if (isnew[t]) set[cnt++] = id[t];
    if ((cnt == cnt0 || stp->k == 0) && cnt < M && cnt < n) {
      // growth safeguard: SplitMix64 keyed by (seed, k, side), probed to the complement
      uint64_t g = splitmix64(p.seed + 2ull * (uint64_t)stp->k + (uint64_t)side) % (uint64_t)n;
      for (int probe = 0; probe < n; ++probe) {
        bool present = false;
        for (int l = 0; l < cnt; ++l)
          if (set[l] == (int32_t)g) {
            present = true;
            break;
          }
        if (!present) break;
        g = (g + 1) % (uint64_t)n;
      }
      set[cnt++] = (int32_t)g;
    }
    // both sides' CTAs may set the bit at once: an atomic OR loses neither
    if (cnt >= M) atomicOr(reinterpret_cast<unsigned int*>(&stp->flags), (unsigned int)kFlagCapacity);
    stp->cnt[side] = cnt;
  }
}

// Largest best change at which an FP32 solve may stop on a stall (see k_stop).
constexpr double kStallRhoMax = 1e-3;

template <typename T>
__global__ void k_stop(CoreParams p, CoreBufs<T> b, int parity) {
  const int slot = slot_of(p.g, blockIdx.x);
  if (slot < 0) return;
  SolveState* stp = p.st + slot;
  if (!stp->active) return;
  const int M = p.g.M;
  const int r = stp->r, rp = stp->r_prev;
  const double* sc = b.sig + (int64_t)slot * 2 * M + (int64_t)parity * M;
  const double* sp = b.sig + (int64_t)slot * 2 * M + (int64_t)(1 - parity) * M;
  __shared__ double red[32];
  double rho = 1.0;
  if (rp > 0) {
    const double* X0 = b.X.at(slot, 0);
    const double* X1 = b.X.at(slot, 1);
    const double* GU = b.GE.at(slot, 0);
    const double* GV = b.GE.at(slot, 1);
    double acc = 0.0;
    // ||S_k - X0 S' X1^T||^2
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
      const int a = e % r, bb = e / r;
      double v = (a == bb) ? sc[a] : 0.0;
      for (int cc = 0; cc < rp; ++cc) v -= X0[(int64_t)cc * M + a] * sp[cc] * X1[(int64_t)cc * M + bb];
      acc += v * v;
    }
    // tr(X0 S' GV S' X0^T) and tr(X1 S' GU S' X1^T)
    for (int e = threadIdx.x; e < r * rp; e += blockDim.x) {
      const int a = e % r, cc = e / r;
      double s0 = 0.0, s1 = 0.0;
      for (int d = 0; d < rp; ++d) {
        s0 += GV[(int64_t)d * M + cc] * sp[d] * X0[(int64_t)d * M + a];
        s1 += GU[(int64_t)d * M + cc] * sp[d] * X1[(int64_t)d * M + a];
      }
      acc += X0[(int64_t)cc * M + a] * sp[cc] * s0 + X1[(int64_t)cc * M + a] * sp[cc] * s1;
    }
    // tr(S' GU S' GV)
    for (int e = threadIdx.x; e < rp * rp; e += blockDim.x) {
      const int cc = e % rp, d = e / rp;
      acc += sp[cc] * GU[(int64_t)d * M + cc] * sp[d] * GV[(int64_t)cc * M + d];
    }
    acc = block_sum(acc, red);
    rho = stp->snorm > 0.0 ? sqrt(fmax(acc, 0.0)) / stp->snorm : 0.0;
  }
  if (stp->snorm == 0.0) rho = 0.0;  // zero right-hand side: W = 0 is exact
  if (threadIdx.x == 0) {
    if (p.trace && stp->total_iters < kTraceLen) {
      // {solve iteration, rho, eta1/eta2 S_min term, |I|, |J| (before redundancy
      //  removal), in-loop rank, ||S_k||_F, |I| after removal}
      double* e = p.trace + ((int64_t)slot * kTraceLen + stp->total_iters) * kTraceWidth;
      e[0] = stp->iters;
      e[1] = rho;
      e[2] = stp->eta_smin;
      e[3] = stp->cnt[0];
      e[4] = stp->cnt[1];
      e[5] = r;
      e[6] = stp->snorm;
      e[7] = stp->cnt_next[0];
    }
    const double rho_prev = stp->rho;
    stp->rho = rho;
    stp->iters += 1;
    stp->total_iters += 1;
    stp->k += 1;
    // A correction solve is done once its change is small against the solution
    // it corrects: tol_abs / ||S_k|| (clamped to [tol, 0.1]) relative to itself.
    double tol_eff = stp->tol;
    if (stp->tol_abs > 0.0 && stp->snorm > 0.0) tol_eff = fmax(tol_eff, fmin(0.1, stp->tol_abs / stp->snorm));
    const bool conv = fmax(rho, stp->eta_smin) < tol_eff;
    // FP32 solves: once the change has failed twice in a row to halve its best
    // value, with that best value within the FP32 noise region (<= 1e-3), the
    // iteration moves only within the data's rounding noise.  Above it the
    // iteration is still converging, slowly: it continues to max_iter.
    if (p.noise_floor_stop && stp->iters >= 2) {
      if (stp->rho_best > 0.0) stp->rho_jump = fmax(stp->rho_jump, rho / stp->rho_best);
      if (stp->rho_best == 0.0 || rho < 0.5 * stp->rho_best) {
        stp->rho_best = rho;
        stp->stall = 0;
      } else {
        stp->stall += 1;
      }
    }
    if (conv) {
      stp->flags |= kFlagConverged;
      stp->active = 0;
    } else if (p.noise_floor_stop && stp->stall >= 2 && stp->rho_best <= kStallRhoMax) {
      stp->flags |= kFlagStalled;
      stp->active = 0;
      // A last step that grew the change (an index update that FP32 noise
      // made worse) is undone: the previous iterate, still held in the other
      // half of the ping-pong buffers, is the result.
      if (stp->iters >= 2 && rho > rho_prev) {
        stp->k -= 1;
        stp->r = rp;
        stp->snorm = stp->snorm_prev;
        stp->rho = rho_prev;
        stp->flags |= kFlagRolledBack;
      }
    } else if (stp->k >= p.max_iter) {
      stp->active = 0;
    }
    stp->r_prev = stp->r;
    stp->snorm_prev = stp->snorm;
    stp->cnt[0] = stp->cnt_next[0];
    stp->cnt[1] = stp->cnt_next[1];
  }
}

template <typename T>
__global__ void k_finalize(CoreParams p, CoreBufs<T> b, DstBatch<T, double> back, T* const* ubufs,
                           int64_t ubuf_side_stride, int64_t ubuf_slot_stride) {
  const int slot = blockIdx.x;
  if (threadIdx.x != 0) return;
  SolveState* stp = p.st + slot;
  const ProblemDev& pr = b.prob[slot];
  T** in = const_cast<T**>(reinterpret_cast<const T* const*>(back.in));
  double** out = const_cast<double**>(back.out);
  int64_t* ldi = const_cast<int64_t*>(back.ld_in);
  int64_t* ldo = const_cast<int64_t*>(back.ld_out);
  if (pr.rf <= 0 || stp->iters == 0) {
    stp->r_out = 0;
    in[slot] = nullptr;
    in[back.nslots + slot] = nullptr;
    out[slot] = nullptr;
    out[back.nslots + slot] = nullptr;
    return;
  }
  const int M = p.g.M;
  const int parity = (stp->k - 1) & 1;
  const double* s = b.sig + (int64_t)slot * 2 * M + (int64_t)parity * M;
  const int r = stp->r;
  double tot = 0.0;
  for (int t = 0; t < r; ++t) tot += s[t] * s[t];
  int rstar = r;
  double tail = 0.0;  // sum_{l >= t} s_l^2, scanning from the end
  for (int t = r; t >= 0; --t) {
    if (t < r) tail += s[t] * s[t];
    if (tail < p.tol * p.tol * tot) rstar = t;
    else break;
  }
  if (rstar < 1) rstar = 1;
  int rout = rstar < p.r_max ? rstar : p.r_max;
  if (rout < 1) rout = 1;
  stp->r_star = rstar;
  stp->r_out = rout;
  if (b.acct) acct_back(b.acct + (int64_t)slot * 2 * LRP_K_COUNT, p.g.n, rout, (int)sizeof(T), p.dst_df != 0);
  if (rstar > p.r_max) stp->flags |= kFlagRankCapped;
  for (int t = 0; t < rout; ++t) pr.S[t] = s[t];
  T* ub = ubufs[parity];
  in[slot] = ub + (int64_t)slot * ubuf_slot_stride;
  in[back.nslots + slot] = ub + (int64_t)slot * ubuf_slot_stride + ubuf_side_stride;
  out[slot] = pr.U;
  out[back.nslots + slot] = pr.V;
  ldi[slot] = p.g.ld;
  ldi[back.nslots + slot] = p.g.ld;
  ldo[slot] = pr.ldu;
  ldo[back.nslots + slot] = pr.ldv;
  if (pr.info) {
    lrp_info inf;
    inf.rank = rout;
    inf.iterations = stp->iters;
    const bool conv = (stp->flags & kFlagConverged) != 0;
    inf.status = !conv ? LRP_NOT_CONVERGED : ((rstar > p.r_max) ? LRP_RANK_CAPPED : LRP_OK);
    inf.r_star = rstar;
    inf.size_I = stp->cnt[0];
    inf.size_J = stp->cnt[1];
    inf.total_iterations = stp->total_iters;
    inf.flags = stp->flags;
    inf.rho = stp->rho;
    inf.eta_smin = stp->eta_smin;
    inf.sigma_max = s[0];
    inf.reserved1 = 0.0;
    *pr.info = inf;
  }
}

template <typename T>
__global__ void k_setup(CoreParams p, const ProblemDev* prob, T* w, int wstride, int nactive, double* acct) {
  const int slot = blockIdx.x;
  SolveState* stp = p.st + slot;
  const bool act = slot < nactive && prob[slot].rf > 0;
  const int rf = act ? prob[slot].rf : 0;
  const double h = 1.0 / (double)(p.g.n + 1);
  if (prob[slot].s_f)  // weights of the Poisson right-hand side (unused for a matrix given by entries)
    for (int k = threadIdx.x; k < rf; k += blockDim.x) w[(int64_t)slot * wstride + k] = (T)(h * h * prob[slot].s_f[k]);
  if (threadIdx.x == 0) {
    SolveState st;
    memset(&st, 0, sizeof(st));
    st.active = act ? 1 : 0;
    st.valid = act ? 1 : 0;
    st.rf = rf;
    st.rf0 = rf;
    st.c0[0] = st.c0[1] = rf;
    st.warm_ok = (act && prob[slot].warm != nullptr) ? 1 : 0;
    st.tol = p.tol;
    *stp = st;
    if (act && acct) acct_setup(acct + (int64_t)slot * 2 * LRP_K_COUNT, p.g.n, rf, p.g.NB, (int)sizeof(T));
  }
}

template <typename T>
__global__ void k_warm_load(CoreParams p, CoreBufs<T> b, Strided<T> U1) {
  const int slot = blockIdx.y >> 1, side = blockIdx.y & 1;
  SolveState* stp = p.st + slot;
  if (!stp->active || !stp->warm_ok) return;
  const WarmDev* w = b.prob[slot].warm;
  if (!w || !w->valid) return;
  const int M = p.g.M;
  const int r = min(w->r, M);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < p.g.n) {
    const double* src = w->U + (int64_t)side * w->ld * M;
    T* dst = U1.at(slot, side);
    for (int c = 0; c < r; ++c) dst[(int64_t)c * p.g.ld + i] = (T)src[(int64_t)c * w->ld + i];
  }
  if (blockIdx.x == 0) {
    const int cnt = min(w->cnt[side], M);
    int32_t* set = b.idx.at(slot, side);
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) set[t] = w->idx[side * M + t];
    if (threadIdx.x == 0) {
      stp->cnt[side] = cnt;
      stp->c0[side] = r;
    }
  }
}

// Numerical range of the initial bases: after the CholeskyQR of the
// transformed right-hand side X = Q R, keep the columns l of Q = Q2 P with
// |R(l,l)| >= redundancy max|diag R| (the threshold of the redundancy removal),
// moved to the front of P in order, and c0 = their count, so that a
// numerically dependent factor column adds no noise direction to U_{-1}.
template <typename T>
__global__ void k_orth_keep(CoreParams p, CoreBufs<T> b) {
  const int slot = slot_of(p.g, blockIdx.x >> 1), side = blockIdx.x & 1;
  if (slot < 0) return;
  SolveState* stp = p.st + slot;
  if (!stp->active || threadIdx.x != 0) return;
  const int M = p.g.M;
  const int m = stp->rf;
  const double* R = b.Racc.at(slot, side);
  double* P = b.P.at(slot, side);
  double mx = 0.0;
  for (int l = 0; l < m; ++l) mx = fmax(mx, fabs(R[(int64_t)l * M + l]));
  int c = 0;
  for (int l = 0; l < m; ++l) {
    if (!(mx > 0.0) || fabs(R[(int64_t)l * M + l]) < p.redundancy * mx) continue;
    if (c != l)
      for (int i = 0; i < m; ++i) P[(int64_t)c * M + i] = P[(int64_t)l * M + i];
    ++c;
  }
  if (c == 0) c = 1;  // a zero right-hand side keeps one (zero) column
  stp->c0[side] = c;
}

template <typename T>
__global__ void k_warm_store(CoreParams p, CoreBufs<T> b, T* const* ubufs, int64_t side_stride, int64_t slot_stride) {
  const int slot = blockIdx.y >> 1, side = blockIdx.y & 1;
  const SolveState* stp = p.st + slot;
  if (!stp->valid || stp->iters == 0) return;
  WarmDev* w = b.prob[slot].warm;
  if (!w) return;
  const int M = p.g.M;
  const int r = stp->r;
  const T* src = ubufs[(stp->k - 1) & 1] + (int64_t)slot * slot_stride + (int64_t)side * side_stride;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < p.g.n) {
    double* dst = w->U + (int64_t)side * w->ld * M;
    for (int c = 0; c < r; ++c) dst[(int64_t)c * w->ld + i] = (double)src[(int64_t)c * p.g.ld + i];
  }
  if (blockIdx.x == 0) {
    const int cnt = stp->cnt[side];
    const int32_t* set = b.idx.at(slot, side);
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) w->idx[side * M + t] = set[t];
    if (threadIdx.x == 0) {
      w->cnt[side] = cnt;
      if (side == 0) {
        w->r = r;
        w->valid = 1;
      }
    }
  }
}

__global__ void k_eigenvalues(int n, double* lam64, float* lam32) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  // lambda_{k+1} = 4 sin^2(pi (k+1) / (2(n+1)))
  const double s = sinpi((double)(k + 1) / (2.0 * (double)(n + 1)));
  const double l = 4.0 * s * s;
  if (lam64) lam64[k] = l;
  if (lam32) lam32[k] = (float)l;
}

// Active slots: their count in out[0] and, when list is given, their indices in
// ascending order in list[0 .. count), then -1 up to nslots (the launch list
// of the next Cross-DEIM iteration).  One CTA; each thread scans a contiguous
// chunk of slots and the chunks' counts are prefix-summed across the block.
__global__ void k_count_active(const SolveState* st, int nslots, int32_t* out, int32_t* list) {
  __shared__ int wsum[32];
  __shared__ int total;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5;
  const int chunk = (nslots + nt - 1) / nt;
  const int b = min(nslots, tid * chunk), e = min(nslots, b + chunk);
  int local = 0;
  for (int s = b; s < e; ++s) local += st[s].active ? 1 : 0;
  int incl = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) wsum[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    const int v = lane < (nt >> 5) ? wsum[lane] : 0;
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += u;
    }
    if (lane < (nt >> 5)) wsum[lane] = inc - v;
    if (lane == (nt >> 5) - 1) total = inc;
  }
  __syncthreads();
  if (tid == 0) *out = total;
  if (!list) return;
  int pos = wsum[wid] + incl - local;
  for (int s = b; s < e; ++s)
    if (st[s].active) list[pos++] = s;
  for (int i = total + tid; i < nslots; i += nt) list[i] = -1;
}

// ------------------------------------------------------------------ launches

template <typename T>
cudaError_t launch_chol(const CoreParams& p, const CoreBufs<T>& b, int sel, int pass, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    if (pass > 0) {
      k_chol<T, float><<<p.g.nslots * 2, CT, kCholSmemDim * kCholSmemDim * sizeof(float), s>>>(p, b, sel, pass);
      return cudaGetLastError();
    }
  }
  k_chol<T, double><<<p.g.nslots * 2, CT, kCholSmemBytes, s>>>(p, b, sel, pass);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_core(const CoreParams& p, const CoreBufs<T>& b, int parity, cudaStream_t s) {
  auto kern = k_core<T>;
  kern<<<p.g.nslots, CTC, core_smem_bytes<T>(), s>>>(p, b, parity);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_select(const CoreParams& p, const CoreBufs<T>& b, int sel_c, cudaStream_t s) {
  const int total = p.cand_blocks * p.cand_per_block;
  int len = 1;
  while (len < total && len < 16384) len <<= 1;
  const size_t smem = (size_t)len * (sizeof(double) + sizeof(int));
  auto kern = k_select<T>;
  kern<<<p.g.nslots * 2, 512, smem, s>>>(p, b, sel_c, len);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_stop(const CoreParams& p, const CoreBufs<T>& b, int parity, cudaStream_t s) {
  k_stop<T><<<p.g.nslots, CT, 0, s>>>(p, b, parity);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_finalize_impl(const CoreParams& p, const CoreBufs<T>& b, const DstBatch<T, double>& back,
                                 T* const* ubufs, int64_t side_stride, int64_t slot_stride, cudaStream_t s) {
  k_finalize<T><<<p.g.nslots, 32, 0, s>>>(p, b, back, ubufs, side_stride, slot_stride);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_setup(const CoreParams& p, const ProblemDev* prob, T* w, int wstride, int nactive, double* acct,
                         cudaStream_t s) {
  k_setup<T><<<p.g.nslots, 64, 0, s>>>(p, prob, w, wstride, nactive, acct);
  return cudaGetLastError();
}

cudaError_t core_configure() {
  cudaError_t e = cudaSuccess;
  const int sel_bytes = 16384 * (int)(sizeof(double) + sizeof(int));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_core<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)core_smem_bytes<double>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_core<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)core_smem_bytes<float>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_chol<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCholSmemBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_chol<float, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCholSmemBytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_select<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, sel_bytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_select<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, sel_bytes);
  return e;
}

template <typename T>
cudaError_t launch_warm_load(const CoreParams& p, const CoreBufs<T>& b, Strided<T> U1, cudaStream_t s) {
  k_warm_load<T><<<dim3((p.g.n + 255) / 256, p.g.nslots * 2), 256, 0, s>>>(p, b, U1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_orth_keep(const CoreParams& p, const CoreBufs<T>& b, cudaStream_t s) {
  k_orth_keep<T><<<p.g.nslots * 2, 32, 0, s>>>(p, b);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_warm_store(const CoreParams& p, const CoreBufs<T>& b, T* const* ubufs, int64_t side_stride,
                              int64_t slot_stride, cudaStream_t s) {
  k_warm_store<T><<<dim3((p.g.n + 255) / 256, p.g.nslots * 2), 256, 0, s>>>(p, b, ubufs, side_stride, slot_stride);
  return cudaGetLastError();
}

cudaError_t launch_eigenvalues(int n, double* lam64, float* lam32, cudaStream_t s) {
  k_eigenvalues<<<(n + 255) / 256, 256, 0, s>>>(n, lam64, lam32);
  return cudaGetLastError();
}

cudaError_t launch_count_active(const SolveState* st, int nslots, int32_t* out, int32_t* list, cudaStream_t s) {
  k_count_active<<<1, 256, 0, s>>>(st, nslots, out, list);
  return cudaGetLastError();
}

// Device-side loop control of a conditional while-node: k_loop_begin runs
// before the node (the body runs only if a problem is still active), k_loop_next
// ends each trip of the body.  The trip bound keeps the loop finite whatever
// the per-problem state holds.
__global__ void k_loop_begin(const int32_t* active, int32_t* trips, cudaGraphConditionalHandle h) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    *trips = 0;
    cudaGraphSetConditional(h, *active > 0 ? 1u : 0u);
  }
}

__global__ void k_loop_next(const int32_t* active, int32_t* trips, int max_trips, cudaGraphConditionalHandle h) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const int t = *trips + 1;
    *trips = t;
    cudaGraphSetConditional(h, (*active > 0 && t < max_trips) ? 1u : 0u);
  }
}

// Condition of a conditional if-node: a positive device count.
__global__ void k_cond_positive(const int32_t* count, cudaGraphConditionalHandle h) {
  if (threadIdx.x == 0 && blockIdx.x == 0) cudaGraphSetConditional(h, *count > 0 ? 1u : 0u);
}

cudaError_t launch_cond_positive(const int32_t* count, cudaGraphConditionalHandle h, cudaStream_t s) {
  k_cond_positive<<<1, 32, 0, s>>>(count, h);
  return cudaGetLastError();
}

cudaError_t launch_loop_begin(const int32_t* active, int32_t* trips, cudaGraphConditionalHandle h, cudaStream_t s) {
  k_loop_begin<<<1, 32, 0, s>>>(active, trips, h);
  return cudaGetLastError();
}

cudaError_t launch_loop_next(const int32_t* active, int32_t* trips, int max_trips, cudaGraphConditionalHandle h,
                             cudaStream_t s) {
  k_loop_next<<<1, 32, 0, s>>>(active, trips, max_trips, h);
  return cudaGetLastError();
}

// dst[0 .. words) = src[0 .. words), 4-byte words; either side may be mapped
// pinned host memory (its device alias).
__global__ void k_stage(const uint32_t* __restrict__ src, uint32_t* __restrict__ dst, int64_t words) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < words; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

cudaError_t launch_stage(const void* src, void* dst, size_t bytes, cudaStream_t s) {
  if (bytes == 0) return cudaSuccess;
  if (!src || !dst || bytes % 4 != 0 || (reinterpret_cast<uintptr_t>(src) & 3) || (reinterpret_cast<uintptr_t>(dst) & 3))
    return cudaErrorInvalidValue;
  const int64_t words = (int64_t)(bytes / 4);
  const int64_t blocks = (words + 255) / 256;
  k_stage<<<(unsigned)(blocks < 64 ? blocks : 64), 256, 0, s>>>(static_cast<const uint32_t*>(src),
                                                               static_cast<uint32_t*>(dst), words);
  return cudaGetLastError();
}

#define LRP_INST(T)                                                                                          \
  template cudaError_t launch_chol<T>(const CoreParams&, const CoreBufs<T>&, int, int, cudaStream_t);       \
  template cudaError_t launch_core<T>(const CoreParams&, const CoreBufs<T>&, int, cudaStream_t);            \
  template cudaError_t launch_select<T>(const CoreParams&, const CoreBufs<T>&, int, cudaStream_t);          \
  template cudaError_t launch_stop<T>(const CoreParams&, const CoreBufs<T>&, int, cudaStream_t);            \
  template cudaError_t launch_finalize_impl<T>(const CoreParams&, const CoreBufs<T>&,                      \
                                               const DstBatch<T, double>&, T* const*, int64_t, int64_t,      \
                                               cudaStream_t);                                                 \
  template cudaError_t launch_setup<T>(const CoreParams&, const ProblemDev*, T*, int, int, double*, cudaStream_t); \
  template cudaError_t launch_warm_load<T>(const CoreParams&, const CoreBufs<T>&, Strided<T>, cudaStream_t);      \
  template cudaError_t launch_orth_keep<T>(const CoreParams&, const CoreBufs<T>&, cudaStream_t);                   \
  template cudaError_t launch_warm_store<T>(const CoreParams&, const CoreBufs<T>&, T* const*, int64_t, int64_t,    \
                                            cudaStream_t);
LRP_INST(double)
LRP_INST(float)
#undef LRP_INST

}  // namespace lrp
