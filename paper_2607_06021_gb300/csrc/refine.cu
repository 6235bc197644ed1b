// Mixed-precision refinement (an extension beyond the paper).
//
// The FP32 Cross-DEIM solve gives a trial solution What0 = Uh0 S0 Vh0^T in
// transformed variables.  Because T = Z Lambda Z (Sec. 3), the residual of
// T W + W T = h^2 F in the same variables is
//     Rhat = h^2 Fhat - (Lambda What0 + What0 Lambda)
//          = [Uh_f, Lambda Uh0, Uh0] diag(h^2 s_f, -S0, -S0) [Vh_f, Vh0, Lambda Vh0]^T,
// a rank r_f + 2 r0 product that is recompressed in FP64 (shifted CholeskyQR of
// both factor blocks and an SVD of the small core R_X diag(d) R_Y^T).  The
// correction dWhat(i,j) = Rhat(i,j)/(lambda_i + lambda_j) is then one more
// Cross-DEIM solve, and What1 = What0 + dWhat is recompressed in FP64 the same
// way before the back transform.
//
// Kernels here assemble the stacked factor blocks, form and factor the small
// cores and convert between the FP32 iteration workspace and the FP64 one.
#include <cuda_runtime.h>
#include <math.h>

#include "common.cuh"
#include "core.cuh"
#include "dense.cuh"
#include "dfloat.cuh"
#include "refine.cuh"

namespace lrp {

namespace {
constexpr int RT = 256;

__device__ inline void racct(const RefineArgs& a, int slot, int cls, double flops, double bytes) {
  if (!a.acct) return;
  double* row = a.acct + (int64_t)slot * 2 * LRP_K_COUNT;
  row[2 * cls] += flops;
  row[2 * cls + 1] += bytes;
}

// Gram passes (symmetric) and triangular applies of one shifted CholeskyQR on
// two n x m blocks: FP64 classes, or the double-float classes for the
// recompressions on the FP32 pipe (bytes per element w: 4 for FP32 data, 8 for
// FP64 data and for (hi, lo) planes).
__device__ inline void racct_cholqr(const RefineArgs& a, int slot, int passes, double m, bool df = false,
                                    double w_elem = 0.0) {
  const double n = a.n;
  const double w = w_elem > 0.0 ? w_elem : (df ? 4.0 : 8.0);
  racct(a, slot, df ? LRP_K_GRAM_DF : LRP_K_GRAM, 2.0 * passes * n * m * (m + 1.0),
        2.0 * passes * (n * m * w + a.NB * m * (m + 1.0) * 4.0));
  racct(a, slot, LRP_K_REDUCE, 2.0 * passes * a.NB * m * (m + 1.0) / 2.0,
        2.0 * passes * (a.NB + 1.0) * m * (m + 1.0) * 4.0);
  if (passes > 1)
    racct(a, slot, df ? LRP_K_GEMM_DF : LRP_K_GEMM, 2.0 * (passes - 1) * n * m * (m + 1.0),
          2.0 * (passes - 1) * n * m * (w + 8.0));
}
}  // namespace


// After the first FP32 solve: r0 = rank of the trial solution (capped so that
// r_f + 2 r0 <= M), d = [h^2 s_f, -S0, -S0], mx = r_f + 2 r0.
// Tail-rule rank of the descending values s[0..r): the smallest t >= 1 with
// sum_{l >= t} s_l^2 < tol^2 sum_l s_l^2 (the final truncation's rule).
__device__ int tail_rank_dev(const double* s, int r, double tol) {
  double tot = 0.0;
  for (int t = 0; t < r; ++t) tot += s[t] * s[t];
  int rs = r;
  double tail = 0.0;
  for (int t = r - 1; t >= 1; --t) {
    tail += s[t] * s[t];
    if (tail < tol * tol * tot) rs = t;
    else break;
  }
  return rs < 1 ? 1 : rs;
}

__global__ void k_prepare_refine(RefineArgs a) {
  const int slot = blockIdx.x;
  SolveState* st = a.st + slot;
  if (!st->valid) return;
  const int M = a.M;
  const int rf = st->rf0;
  const int par = (st->k - 1) & 1;
  const double* sig = a.sig32 + (int64_t)slot * 2 * M + (int64_t)par * M;
  // The trial solution enters at its tail-rule rank at the FP32 solve's own
  // tolerance; the part it drops is left to the correction.
  int r0 = tail_rank_dev(sig, st->r, st->tol);
  const int cap = (M - rf) / 2;
  if (r0 > cap) r0 = cap;
  if (r0 < 1) r0 = 1;
  double* d = a.dvec + (int64_t)slot * M;
  double* s0 = a.s0 + (int64_t)slot * M;
  const double h = 1.0 / (double)(a.n + 1);
  const ProblemDev& pr = a.prob[slot];
  for (int k = threadIdx.x; k < rf; k += blockDim.x) d[k] = h * h * pr.s_f[k];
  for (int t = threadIdx.x; t < r0; t += blockDim.x) {
    s0[t] = sig[t];
    d[rf + t] = -sig[t];
    d[rf + r0 + t] = -sig[t];
  }
  if (threadIdx.x == 0) {
    st->r0 = r0;
    st->mx[0] = st->mx[1] = rf + 2 * r0;
    st->active = 1;
    st->upar = par;
    const double m = rf + 2.0 * r0, n = a.n;
    // stacked blocks: read Uh_f (FP64) and Uh0 (FP32), write X and the FP64 stash
    racct(a, slot, LRP_K_REFINE, 2.0 * n * r0, 2.0 * n * (rf * 8.0 + r0 * 4.0 + m * 8.0 + r0 * 8.0));
    // the FP64 forward transform of the right-hand side (double-float), a real FFT of length N per column
    const double N = n + 1.0;
    racct(a, slot, LRP_K_DST_DF, 2.0 * rf * 2.5 * N * log2(N), 2.0 * rf * n * 16.0);
    if (a.X32lo.base) racct_cholqr(a, slot, 2, m, true, 8.0);
    else racct_cholqr(a, slot, 1, m);
  }
}

// Stacked blocks of the residual factors (ld = a.ld); side 0:
// [Uh_f | Lambda Uh0 | Uh0], side 1: [Vh_f | Vh0 | Lambda Vh0], in FP64, or as
// double-float (hi, lo) planes when a.X32lo is set.  Also stashes Uh0, Vh0 in
// FP64 for the final sum.
__global__ void k_assemble_residual(RefineArgs a) {
  const int slot = blockIdx.y >> 1, side = blockIdx.y & 1;
  const SolveState& st = a.st[slot];
  if (!st.valid) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const int rf = st.rf0, r0 = st.r0;
  const double lam = a.lam[i];
  const double* Fh = a.Fh64.at(slot, side);
  // the solution being refined: the FP32 trial, or (second step) the FP64 sum
  const float* U0 = a.U64.base ? nullptr : a.U32[st.upar].at(slot, side);
  const double* U0d = a.U64.base ? a.U64.at(slot, side) : nullptr;
  double* stash = a.stash.at(slot, side);
  if (a.X32lo.base) {
    float* Xh = a.X32.at(slot, side);
    float* Xl = a.X32lo.at(slot, side);
    auto put = [&](int j, double v) {
      const dfloat x(v);
      Xh[(int64_t)j * a.ld + i] = x.hi;
      Xl[(int64_t)j * a.ld + i] = x.lo;
    };
    for (int j = 0; j < rf; ++j) put(j, Fh[(int64_t)j * a.ld + i]);
    for (int t = 0; t < r0; ++t) {
      const double u = U0d ? U0d[(int64_t)t * a.ld + i] : f32_to_f64(U0[(int64_t)t * a.ld + i]);
      stash[(int64_t)t * a.ld + i] = u;
      put(rf + t, side == 0 ? lam * u : u);
      put(rf + r0 + t, side == 0 ? u : lam * u);
    }
    return;
  }
  double* X = a.X.at(slot, side);
  for (int j = 0; j < rf; ++j) X[(int64_t)j * a.ld + i] = Fh[(int64_t)j * a.ld + i];
  for (int t = 0; t < r0; ++t) {
    const double u = U0d ? U0d[(int64_t)t * a.ld + i] : f32_to_f64(U0[(int64_t)t * a.ld + i]);
    stash[(int64_t)t * a.ld + i] = u;
    const double first = (side == 0) ? lam * u : u;
    const double second = (side == 0) ? u : lam * u;
    X[(int64_t)(rf + t) * a.ld + i] = first;
    X[(int64_t)(rf + r0 + t) * a.ld + i] = second;
  }
}

// Small core K = R_0 diag(d) R_1^T (m = mx), its SVD by one-sided Jacobi, and the
// factors Bf_s = P3_s * (left / right singular vectors) so that the recompressed
// product is (Q2_0 Bf_0) diag(sigma) (Q2_1 Bf_1)^T.  mode 0 keeps the tail-rule
// rank at rel_tol (capped at rcap); mode 1 keeps every numerically nonzero value.
// K is always formed in FP64 (the cancellation between the stacked blocks happens
// there); its SVD runs in TC: FP32 suffices for the residual, whose correction is
// an FP32 solve, and FP64 keeps the final sum exact to working precision.
// FP32 <-> FP64 conversions on the integer pipe (f64cvt.cuh: the values of the
// hardware conversions, which GB300 runs on its FP64 pipe).
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

constexpr int kRecSmemDim = 64;
constexpr size_t kRecSmemBytes = 2 * kRecSmemDim * kRecSmemDim * sizeof(double);
constexpr int kRecThreads = 512;  // 16 warps (the register Jacobi's pairs for m <= 64), 64 registers: two CTAs per SM

template <typename TC>
__global__ void __launch_bounds__(kRecThreads, 2) k_recompress(RefineArgs a, int mode, double rel_tol, int rcap) {
  extern __shared__ double rec_smem[];
  const int slot = blockIdx.x;
  SolveState* st = a.st + slot;
  if (!st->valid) return;
  const int M = a.M;
  const int64_t MM = (int64_t)M * M;
  const int m = st->mx[0];
  const double* R0 = a.Racc.at(slot, 0);
  const double* R1 = a.Racc.at(slot, 1);
  const double* P0 = a.P.at(slot, 0);
  const double* P1 = a.P.at(slot, 1);
  const double* d = a.dvec + (int64_t)slot * M;
  // K and V in shared memory (leading dimension kRecSmemDim) when m is small,
  // else in the slot's global scratch (leading dimension M).
  const bool in_smem = m <= kRecSmemDim;
  const int L = in_smem ? kRecSmemDim : M;
  TC* base = in_smem ? reinterpret_cast<TC*>(rec_smem) : reinterpret_cast<TC*>(a.scratch + (int64_t)slot * a.scratch_stride);
  TC* K = base;                          // m x m
  TC* V = base + (int64_t)L * L;         // m x m
  (void)MM;
  double* B0 = a.Bf.at(slot, 0);
  double* B1 = a.Bf.at(slot, 1);
  double* sig_out = a.sig_out + (int64_t)slot * a.sig_out_stride;
  __shared__ double sig[kMaxM];
  __shared__ int perm[kMaxM];
  __shared__ int flag;
  const int tid = threadIdx.x, nt = blockDim.x;
  // K(i, j) = sum_{l >= max(i, j)} R0(i, l) d_l R1(j, l)   (warp: columns j; lanes: rows i)
  for (int j = threadIdx.x >> 5; j < m; j += blockDim.x >> 5) {
    for (int i = threadIdx.x & 31; i < m; i += 32) {
      double s = 0.0;
      for (int l = max(i, j); l < m; ++l) s += R0[(int64_t)l * M + i] * d[l] * R1[(int64_t)l * M + j];
      K[(int64_t)j * L + i] = narrow_to<TC>(s);
    }
  }
  __syncthreads();
  if constexpr (sizeof(TC) == 4) {
    // FP32: the register form; its column exchange takes the shared memory the
    // two FP32 tiles leave free (none in global scratch, where m > 64 falls back)
    blk_jacobi_f32(K, L, m, m, V, L, sig, &flag, V + (int64_t)L * L, in_smem ? 2 * L * L : 0);
  } else {
    blk_jacobi<TC>(K, L, m, m, V, L, sig, &flag);
  }
  blk_sort_desc(sig, m, perm);
  int r = 0;
  if (tid == 0) {
    double tot = 0.0;
    for (int t = 0; t < m; ++t) tot += sig[t] * sig[t];
    const double s1 = sig[perm[0]];
    if (mode == 0) {
      double tail = 0.0;
      r = m;
      for (int t = m; t >= 1; --t) {
        if (t < m) tail += sig[perm[t]] * sig[perm[t]];
        if (tail < rel_tol * rel_tol * tot) r = t;
        else break;
      }
    } else {
      r = 0;
      for (int t = 0; t < m; ++t) r += (sig[perm[t]] > (double)m * Eps<TC>::value * s1) ? 1 : 0;
    }
    if (r > rcap) r = rcap;
    if (r < 1) r = 1;
    flag = r;
  }
  __syncthreads();
  r = flag;
  // Left vectors: K(:, perm[t]) / sigma (K now holds U' Sigma); right: V(:, perm[t]).
  // Each quotient K(c, j) / sigma_j is formed once (an FP64 division occupies
  // GB300's FP64 pipe for dozens of instructions): in place for FP64 K, else
  // in the shared memory the Jacobi exchange left free (FP64, leading
  // dimension L).  K in global scratch (m > 64) divides inside the sums.
  const int lane = tid & 31, wid = tid >> 5, nwarp = nt >> 5;
  double* Kq = nullptr;
  if constexpr (sizeof(TC) == 8) {
    Kq = reinterpret_cast<double*>(K);
  } else {
    if (in_smem) Kq = reinterpret_cast<double*>(V + (int64_t)L * L);
  }
  if (Kq != nullptr) {
    for (int t = wid; t < r; t += nwarp) {
      const int j = perm[t];
      const double sv = sig[j];
      for (int c = lane; c < m; c += 32)
        Kq[(int64_t)j * L + c] = sv > 0.0 ? widen64(K[(int64_t)j * L + c]) / sv : 0.0;
    }
    __syncthreads();
  }
  for (int t = wid; t < r; t += nwarp) {
    const int j = perm[t];
    const double sv = sig[j];
    for (int i = lane; i < m; i += 32) {
      double s0 = 0.0, s1 = 0.0;
      for (int c = i; c < m; ++c) {
        const double kq = Kq != nullptr ? Kq[(int64_t)j * L + c]
                                        : (sv > 0.0 ? widen64(K[(int64_t)j * L + c]) / sv : 0.0);
        s0 += P0[(int64_t)c * M + i] * kq;
        s1 += P1[(int64_t)c * M + i] * widen64(V[(int64_t)j * L + c]);
      }
      B0[(int64_t)t * M + i] = s0;
      B1[(int64_t)t * M + i] = s1;
    }
  }
  for (int t = tid; t < r; t += nt) sig_out[t] = sig[perm[t]];
  if (tid == 0) {
    st->r = r;
    // the tall product (Q-basis block) * Bf that follows on both sides
    racct(a, slot, a.X32.base ? LRP_K_GEMM_DF : LRP_K_GEMM, 2.0 * 2.0 * a.n * m * r,
          2.0 * a.n * (m + r) * 8.0);
  }
}

// Prepare the FP32 correction solve: its right-hand side in transformed
// variables is the recompressed residual (factors already transformed) with
// weights sigma_R (no h^2: the residual already carries it).
__global__ void k_setup_correction(RefineArgs a) {
  const int slot = blockIdx.x;
  SolveState* st = a.st + slot;
  if (!st->valid) return;
  const int rR = st->r;
  const double* sR = a.sig_out + (int64_t)slot * a.sig_out_stride;
  for (int k = threadIdx.x; k < rR; k += blockDim.x) a.w32[(int64_t)slot * a.wstride + k] = (float)sR[k];
  // Thread 0 replaces the whole state below: every thread must have read the
  // rank first (a warp that read it after the replacement would see 0 and
  // leave its weights, k >= 32, stale).
  __syncthreads();
  if (threadIdx.x == 0) {
    const int total = st->total_iters;
    const int r0 = st->r0, rf0 = st->rf0;
    double s0n = 0.0;  // ||S0||_F = ||What0||_F of the trial solution
    for (int t = 0; t < r0; ++t) s0n += a.s0[(int64_t)slot * a.M + t] * a.s0[(int64_t)slot * a.M + t];
    SolveState z;
    memset(&z, 0, sizeof(z));
    z.active = 1;
    z.valid = 1;
    z.rf = rR;
    z.c0[0] = z.c0[1] = rR;
    z.warm_ok = 0;
    z.rf0 = rf0;
    z.r0 = r0;
    z.total_iters = total;
    z.flags = st->flags & ~kFlagConverged;
    // The first correction requires the FP32 trial to have finished, by its
    // stop test or at its noise floor (the correction compensates a stalled
    // trial).  A second correction corrects whatever the first step left, so
    // its own stop test alone decides.
    z.first_converged = (st->is_corr || (st->flags & (kFlagConverged | kFlagStalled))) ? 1 : 0;
    z.is_corr = 1;
    z.tol = a.corr_tol;
    z.tol_abs = a.final_tol * sqrt(s0n);
    *st = z;
  }
}

// dst[s](:, j) = (TD) src[s](:, j) for j < dim(sel).
template <typename TS, typename TD>
__global__ void k_convert(int n, int64_t ld, const SolveState* st_all, Strided<const TS> src, Strided<TD> dst,
                          int sel) {
  const int slot = blockIdx.y >> 1, side = blockIdx.y & 1;
  const SolveState& st = st_all[slot];
  if (!st.valid) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int c = dim_of(st, side, sel);
  const TS* s = src.at(slot, side);
  TD* d = dst.at(slot, side);
  for (int j = 0; j < c; ++j) {
    const TS v = s[(int64_t)j * ld + i];
    if constexpr (sizeof(TS) == 8 && sizeof(TD) == 4) {
      d[(int64_t)j * ld + i] = f64_to_f32_rn(v);  // the hardware rounding, on the integer pipe
    } else if constexpr (sizeof(TS) == 4 && sizeof(TD) == 8) {
      d[(int64_t)j * ld + i] = f32_to_f64(v);
    } else {
      d[(int64_t)j * ld + i] = (TD)v;
    }
  }
}

// After the correction solve: d = [S0, dS], mx = r0 + rd.
__global__ void k_prepare_sum(RefineArgs a) {
  const int slot = blockIdx.x;
  SolveState* st = a.st + slot;
  if (!st->valid) return;
  const int M = a.M;
  const int r0 = st->r0;
  const int par = (st->k - 1) & 1;
  const double* sig = a.sig32 + (int64_t)slot * 2 * M + (int64_t)par * M;
  // The correction enters at its tail-rule rank at the tolerance its stop test
  // used (relative to itself: tol ||S0|| / ||S_k||, within [tol_in, 0.1]).
  double tol_c = st->tol;
  if (st->tol_abs > 0.0 && st->snorm > 0.0) tol_c = fmax(tol_c, fmin(0.1, st->tol_abs / st->snorm));
  int rd = tail_rank_dev(sig, st->r, tol_c);
  if (rd > M - r0) rd = M - r0;
  double* d = a.dvec + (int64_t)slot * M;
  const double* s0 = a.s0 + (int64_t)slot * M;
  for (int t = threadIdx.x; t < r0; t += blockDim.x) d[t] = s0[t];
  for (int t = threadIdx.x; t < rd; t += blockDim.x) d[r0 + t] = sig[t];
  if (threadIdx.x == 0) {
    st->mx[0] = st->mx[1] = r0 + rd;
    st->upar = par;
    st->rd = rd;
    st->active = 1;
    const double n = a.n;
    racct(a, slot, LRP_K_REFINE, 0.0, 2.0 * n * (r0 * 8.0 + rd * 4.0 + (r0 + rd) * (a.X32.base ? 4.0 : 8.0)));
    racct_cholqr(a, slot, 2, r0 + rd, a.X32.base != nullptr);
  }
}

// Stacked [Uh0 | dUh] (side 0) and [Vh0 | dVh] (side 1) in FP64.
__global__ void k_assemble_sum(RefineArgs a) {
  const int slot = blockIdx.y >> 1, side = blockIdx.y & 1;
  const SolveState& st = a.st[slot];
  if (!st.valid) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const int r0 = st.r0, rd = st.rd;
  const double* stash = a.stash.at(slot, side);
  const float* dU = a.U32[st.upar].at(slot, side);
  if (a.X32.base && a.X32lo.base) {
    // second step: the solution being refined is FP64, stored as (hi, lo) planes
    float* Xh = a.X32.at(slot, side);
    float* Xl = a.X32lo.at(slot, side);
    for (int t = 0; t < r0; ++t) {
      const dfloat x(stash[(int64_t)t * a.ld + i]);
      Xh[(int64_t)t * a.ld + i] = x.hi;
      Xl[(int64_t)t * a.ld + i] = x.lo;
    }
    for (int t = 0; t < rd; ++t) {
      Xh[(int64_t)(r0 + t) * a.ld + i] = dU[(int64_t)t * a.ld + i];
      Xl[(int64_t)(r0 + t) * a.ld + i] = 0.f;
    }
    return;
  }
  if (a.X32.base) {
    // both blocks are FP32 values (the FP32 trial and the FP32 correction): exact
    float* X = a.X32.at(slot, side);
    for (int t = 0; t < r0; ++t) X[(int64_t)t * a.ld + i] = (float)stash[(int64_t)t * a.ld + i];
    for (int t = 0; t < rd; ++t) X[(int64_t)(r0 + t) * a.ld + i] = dU[(int64_t)t * a.ld + i];
    return;
  }
  double* X = a.X.at(slot, side);
  for (int t = 0; t < r0; ++t) X[(int64_t)t * a.ld + i] = stash[(int64_t)t * a.ld + i];
  for (int t = 0; t < rd; ++t) X[(int64_t)(r0 + t) * a.ld + i] = (double)dU[(int64_t)t * a.ld + i];
}

// The final recompressed iterate becomes "iteration 0" of the FP64 workspace so
// that the common finalize kernel truncates and transforms it back.
__global__ void k_final_state(RefineArgs a) {
  const int slot = blockIdx.x;
  SolveState* st = a.st + slot;
  if (!st->valid || threadIdx.x != 0) return;
  // The last correction must pass its own stop test: one that stalled (its
  // change stopped halving above the tolerance it was given) leaves an error
  // the method cannot bound, and the result is reported as not converged.
  const bool conv = st->first_converged && (st->flags & kFlagConverged);
  st->k = 1;
  st->iters = st->total_iters;
  st->flags = conv ? (st->flags | kFlagConverged) : (st->flags & ~kFlagConverged);
  st->active = 0;
}

// After the first refinement step: a problem goes through a second step when
// its first correction is unreliable, i.e. when
//   (a) the correction is large against the trial solution it corrects, so that
//       its FP32 accuracy (at best ~1e-5 of itself) leaves an error above
//       10 tol: ||dS|| / ||S0|| max(rho_c, 1e-5) > 10 tol, or
//   (b) the correction solve jumped (its change rose more than tenfold above
//       its best value, itself below 1e-2) and may have settled on a poor
//       index set, or
//   (c) (see below) a rollback or an unfinished correction.
// The others are held: valid = 0 until k_release_held, so that no kernel of
// the second step touches them.
__global__ void k_check_refine(RefineArgs a, int nslots, int32_t* count) {
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= nslots) return;
  SolveState* st = a.st + slot;
  if (!st->valid) return;
  double s0n = 0.0;
  for (int t = 0; t < st->r0; ++t) s0n += a.s0[(int64_t)slot * a.M + t] * a.s0[(int64_t)slot * a.M + t];
  s0n = sqrt(s0n);
  const double est = s0n > 0.0 ? st->snorm / s0n * fmax(st->rho, 1e-5) : 0.0;
  const bool jumped = st->rho_jump > 10.0 && st->rho_best > 0.0 && st->rho_best < 1e-2;
  // (c) a solve of the first step rolled back an FP32 update that grew its
  //     change, or the correction ended without passing its stop test: its
  //     iterate may sit on a poor index set whatever its last change says.
  const bool unclean = (st->flags & kFlagRolledBack) || !(st->flags & kFlagConverged);
  if (est > 10.0 * a.final_tol || jumped || unclean) {
    st->flags |= kFlagRefinedTwice;
    atomicAdd(count, 1);
  } else {
    st->valid = 0;
    st->active = 0;
    st->flags |= kFlagHeld;
  }
}

// Second step: the solution being refined is the FP64 sum of the first step
// (factors in a.U64, singular values in a.sig_out, rank st->r); it enters at
// its tail-rule rank at tol / 10, capped so that r_f + 2 r0 <= M.
__global__ void k_prepare_refine2(RefineArgs a) {
  const int slot = blockIdx.x;
  SolveState* st = a.st + slot;
  if (!st->valid) return;
  const int M = a.M;
  const int rf = st->rf0;
  const double* sig = a.sig_out + (int64_t)slot * a.sig_out_stride;
  int r0 = tail_rank_dev(sig, st->r, 0.1 * a.final_tol);
  const int cap = (M - rf) / 2;
  if (r0 > cap) r0 = cap;
  if (r0 < 1) r0 = 1;
  double* d = a.dvec + (int64_t)slot * M;
  double* s0 = a.s0 + (int64_t)slot * M;
  const double h = 1.0 / (double)(a.n + 1);
  const ProblemDev& pr = a.prob[slot];
  for (int k = threadIdx.x; k < rf; k += blockDim.x) d[k] = h * h * pr.s_f[k];
  for (int t = threadIdx.x; t < r0; t += blockDim.x) {
    s0[t] = sig[t];
    d[rf + t] = -sig[t];
    d[rf + r0 + t] = -sig[t];
  }
  if (threadIdx.x == 0) {
    st->r0 = r0;
    st->mx[0] = st->mx[1] = rf + 2 * r0;
    st->active = 1;
    const double m = rf + 2.0 * r0, n = a.n;
    racct(a, slot, LRP_K_REFINE, 2.0 * n * r0, 2.0 * n * (rf * 8.0 + r0 * 8.0 + m * 8.0 + r0 * 8.0));
    if (a.X32lo.base) racct_cholqr(a, slot, 2, m, true, 8.0);
    else racct_cholqr(a, slot, 1, m);
  }
}

// Held problems rejoin for the final state and transform.
__global__ void k_release_held(RefineArgs a, int nslots) {
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= nslots) return;
  SolveState* st = a.st + slot;
  if (st->flags & kFlagHeld) {
    st->flags &= ~kFlagHeld;
    st->valid = 1;
  }
}

// ------------------------------------------------------------------ launches

static inline int cdiv(int a, int b) { return (a + b - 1) / b; }

cudaError_t refine_configure() {
  cudaError_t e = cudaFuncSetAttribute(k_recompress<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kRecSmemBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_recompress<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRecSmemBytes);
  return e;
}

cudaError_t launch_prepare_refine(const RefineArgs& a, int nslots, cudaStream_t s) {
  k_prepare_refine<<<nslots, 128, 0, s>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_assemble_residual(const RefineArgs& a, int nslots, cudaStream_t s) {
  k_assemble_residual<<<dim3(cdiv(a.n, 256), 2 * nslots), 256, 0, s>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_recompress(const RefineArgs& a, int nslots, int mode, double rel_tol, int rcap, cudaStream_t s) {
  if (mode == 0)
    k_recompress<float><<<nslots, kRecThreads, kRecSmemBytes, s>>>(a, mode, rel_tol, rcap);
  else
    k_recompress<double><<<nslots, kRecThreads, kRecSmemBytes, s>>>(a, mode, rel_tol, rcap);
  return cudaGetLastError();
}
cudaError_t launch_setup_correction(const RefineArgs& a, int nslots, cudaStream_t s) {
  k_setup_correction<<<nslots, 128, 0, s>>>(a);
  return cudaGetLastError();
}
template <typename TS, typename TD>
cudaError_t launch_convert(int n, int64_t ld, int nslots, const SolveState* st, Strided<const TS> src,
                           Strided<TD> dst, int sel, cudaStream_t s) {
  k_convert<TS, TD><<<dim3(cdiv(n, 256), 2 * nslots), 256, 0, s>>>(n, ld, st, src, dst, sel);
  return cudaGetLastError();
}
template cudaError_t launch_convert<double, float>(int, int64_t, int, const SolveState*, Strided<const double>,
                                                   Strided<float>, int, cudaStream_t);
template cudaError_t launch_convert<float, double>(int, int64_t, int, const SolveState*, Strided<const float>,
                                                   Strided<double>, int, cudaStream_t);
cudaError_t launch_prepare_sum(const RefineArgs& a, int nslots, cudaStream_t s) {
  k_prepare_sum<<<nslots, 128, 0, s>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_assemble_sum(const RefineArgs& a, int nslots, cudaStream_t s) {
  k_assemble_sum<<<dim3(cdiv(a.n, 256), 2 * nslots), 256, 0, s>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_check_refine(const RefineArgs& a, int nslots, int32_t* count, cudaStream_t s) {
  k_check_refine<<<cdiv(nslots, 128), 128, 0, s>>>(a, nslots, count);
  return cudaGetLastError();
}

cudaError_t launch_prepare_refine2(const RefineArgs& a, int nslots, cudaStream_t s) {
  k_prepare_refine2<<<nslots, 64, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_release_held(const RefineArgs& a, int nslots, cudaStream_t s) {
  k_release_held<<<cdiv(nslots, 128), 128, 0, s>>>(a, nslots);
  return cudaGetLastError();
}

cudaError_t launch_final_state(const RefineArgs& a, int nslots, cudaStream_t s) {
  k_final_state<<<nslots, 32, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace lrp
