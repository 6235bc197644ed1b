// Tall-skinny kernels of the Cross-DEIM iteration, batched over problems and
// the two sides (blockIdx.z = slot * 2 + side).
//
//  k_cross     C = What(:,J) and R^T = What(I,:)^T from the transformed
//              right-hand side (Algorithm scross, "C = G(:,J), R = G(I,:)";
//              entries by Eq. g_for_p at O(r_f) each, Sec. 2.1 / Sec. 3.2).
//  k_gemm_narrow, k_gemm_nn
//              n x m times m x m' (the triangular applies of CholeskyQR, the
//              factor update U_k = Q U~ of Algorithm scross, and E = U' - U X):
//              thread per row for narrow products, register tiles otherwise.
//  k_gram_*    per-row-block partial products X^T Y (Gram matrices of
//              CholeskyQR, cross-Grams of consecutive iterates): FP64, FP32 or
//              double-float accumulation.
//  k_reduce    deterministic sum of the partials.
//  k_leverage  leverage scores pi_i = sum_c U(i,c)^2 / c (Algorithm
//              LeverageScores) and per-block top-c candidates.
//
// All kernels read their data-dependent sizes (|I|, |J|, ranks) from the
// per-slot SolveState and return early for finished slots; 256 threads per CTA.
#include <cuda_runtime.h>

#include "common.cuh"
#include "dfloat.cuh"
#include "f64cvt.cuh"
#include "tall.cuh"

namespace lrp {

namespace {
constexpr int TM = 64;
constexpr int TN = 64;
constexpr int TK = 16;
constexpr int TKG = 32;
constexpr int NT = 256;
}  // namespace

constexpr int kSmallGram = 64;
constexpr int kSmallRows = 32;

template <typename T>
__device__ __forceinline__ void ld4(const T* p, T (&v)[4]) {
  if constexpr (sizeof(T) == 4) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
  } else {
    const double2 a = *reinterpret_cast<const double2*>(p);
    const double2 b = *reinterpret_cast<const double2*>(p + 2);
    v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
  }
}

template <typename T>
__device__ __forceinline__ void st4(T* p, const T (&v)[4]) {
  if constexpr (sizeof(T) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
    *reinterpret_cast<double2*>(p + 2) = make_double2(v[2], v[3]);
  }
}

// 1 / x: the exact quotient in FP64; in FP32 the correctly rounded reciprocal
// (the product then carries at most ~1.5 ulp, below the FP32 data's noise).
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

// Widening to FP64 for the partial sums: exact, on the integer pipe for FP32
// values (f64cvt.cuh; GB300 runs the hardware conversion on its FP64 pipe).
__device__ __forceinline__ double to_f64(double x) { return x; }
__device__ __forceinline__ double to_f64(float x) { return f32_to_f64(x); }

// An FP64 small-matrix entry in the data type T: for FP32 the same rounding as
// the hardware conversion, on the integer pipe.
template <typename T>
__device__ __forceinline__ T from_f64(double x) {
  if constexpr (sizeof(T) == 4) {
    return f64_to_f32_rn(x);
  } else {
    return x;
  }
}
__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }

// Sampled columns / rows of the transformed solution (Eq. g_for_p), one thread
// per output row: C(i, q) = (sum_k Fs(i,k) w_k Fo(J_q,k)) / (lambda_i + lambda_{J_q})
// for q < m.  The CTA stages B(k, q) = w_k Fo(J_q, k) for a chunk of KC x QC
// entries in shared memory (read by broadcast); each thread keeps QC sums in
// registers and reads its row's Fs(i, k) once per column chunk (coalesced
// across the warp); the outputs leave as one coalesced store per column.  Each
// sum runs over k in ascending order with one FMA per term, as the earlier
// tiled form did, so the values are the same bit for bit.
constexpr int XQ = 32;  // columns per register block
constexpr int XK = 32;  // k per shared-memory chunk

template <typename T>
__global__ void __launch_bounds__(NT) k_cross(TallGeom g, const SolveState* __restrict__ st_all, CrossArgs<T> a) {
  const int slot = slot_of(g, blockIdx.z >> 1), side = blockIdx.z & 1;
  if (slot < 0) return;
  const SolveState& st = st_all[slot];
  if (!st.active) return;
  const int m = st.cnt[1 - side];
  const int row = blockIdx.x * NT + threadIdx.x;
  if (blockIdx.x * NT >= g.n || m < 1) return;
  const int rf = st.rf;
  const T* Fs = a.F.at(slot, side);
  const T* Fo = a.F.at(slot, 1 - side);
  const int32_t* ix = a.idx.at(slot, 1 - side);
  const T* w = a.w + (int64_t)slot * a.wstride;
  T* A = a.A.at(slot, side);
  __shared__ __align__(16) T Bs[XK][XQ];
  __shared__ int jc[XQ];
  __shared__ T lamc[XQ];
  const bool live = row < g.n;
  const T li = live ? a.lam[row] : T(1);
  for (int q0 = 0; q0 < m; q0 += XQ) {
    const int qn = min(XQ, m - q0);
    __syncthreads();  // the previous block's jc / lamc are read no more
    if (threadIdx.x < XQ) {
      const int j = (threadIdx.x < qn) ? ix[q0 + threadIdx.x] : -1;
      jc[threadIdx.x] = j;
      lamc[threadIdx.x] = (j >= 0) ? a.lam[j] : T(1);
    }
    T acc[XQ];
#pragma unroll
    for (int q = 0; q < XQ; ++q) acc[q] = T(0);
    for (int k0 = 0; k0 < rf; k0 += XK) {
      const int kn = min(XK, rf - k0);
      __syncthreads();
      for (int e = threadIdx.x; e < XK * XQ; e += NT) {
        const int kk = e / XQ, q = e % XQ, k = k0 + kk;
        const int j = jc[q];
        Bs[kk][q] = (j >= 0 && kk < kn) ? w[k] * Fo[(int64_t)k * g.ld + j] : T(0);
      }
      __syncthreads();
      if (live) {
        // the row's values of 8 consecutive k are loaded before their FMAs
        for (int k8 = 0; k8 < kn; k8 += 8) {
          T av[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) av[u] = (k8 + u < kn) ? Fs[(int64_t)(k0 + k8 + u) * g.ld + row] : T(0);
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            if (k8 + u >= kn) break;
#pragma unroll
            for (int q = 0; q < XQ; q += 4) {
              if (q >= qn) break;  // the block's last columns (uniform across the CTA)
              T b[4];
              ld4<T>(&Bs[k8 + u][q], b);
#pragma unroll
              for (int t = 0; t < 4; ++t) acc[q + t] = fma(av[u], b[t], acc[q + t]);
            }
          }
        }
      }
    }
    if (live) {
#pragma unroll
      for (int q = 0; q < XQ; ++q)
        if (q < qn) A[(int64_t)(q0 + q) * g.ld + row] = acc[q] * recip(li + lamc[q]);
    } else if (row < g.ld) {
      // the padding rows n..ld-1 of each column hold zeros
      for (int q = 0; q < qn; ++q) A[(int64_t)(q0 + q) * g.ld + row] = T(0);
    }
  }
}

// Rows of one GEMM row tile, and row tiles per CTA.
constexpr int kGemmRows = 128;
constexpr int kGemmTiles = 4;

template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
  __device__ static void ld(const float* p, float (&v)[4]) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
  }
};
template <>
struct Vec4<double> {
  __device__ static void ld(const double* p, double (&v)[4]) {
    const double2 a = *reinterpret_cast<const double2*>(p);
    const double2 b = *reinterpret_cast<const double2*>(p + 2);
    v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
  }
};

// Out = In * Bm (or Zsub - In * Bm) for the CTA's kGemmTiles row tiles of
// kGemmRows rows, output columns [c0, c0 + TNW).  Bm is staged in shared
// memory in blocks of 64 rows of K (converted to T once per staging): with
// K <= 64 one staging serves all row tiles.  Each row tile streams In through
// shared memory in TK-deep slices: 256 threads, each RI consecutive rows x 4
// consecutive columns, operands read as 4-vectors.  The next slice (of this
// tile or the next) is loaded into registers, as 4-row vectors, while the
// current one is multiplied; the output is written as 4-row vectors.
template <typename T, int TNW>
__device__ __forceinline__ void gemm_block(const TallGeom& g, const T* __restrict__ X, const double* __restrict__ Bm,
                                           T* __restrict__ O, const T* __restrict__ Z, int mode, int mi, int mo,
                                           int rbase, int c0, bool vec, T (*As)[kGemmRows], T (*Bs)[64]) {
  constexpr int TX = TNW / 4;           // threads along columns
  constexpr int TY = NT / TX;           // threads along rows
  constexpr int RI = kGemmRows / TY;    // rows per thread
  constexpr int QV = kGemmRows / 4;     // 4-row vectors in a slice row
  constexpr int PV = TK * QV / NT;      // 4-row vectors per thread and slice
  static_assert(RI % 4 == 0, "rows per thread: whole 4-vectors");
  static_assert(PV * NT == TK * QV, "slice: whole vectors per thread");
  const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
  const int nkb = (mi + 63) / 64;
  T pf[PV][4];
  // Slice (rows r0.., K rows k0 .. k0 + TK - 1, valid below kend) into pf;
  // rows past n and K rows past kend read as zero.
  auto fetch = [&](int r0, int k0, int kend) {
#pragma unroll
    for (int v = 0; v < PV; ++v) {
      const int e = tid + NT * v, kk = e / QV, row = r0 + 4 * (e % QV), k = k0 + kk;
      const T* src = X + (int64_t)k * g.ld + row;
      if (vec && k < kend && row + 3 < g.n) {
        ld4<T>(src, pf[v]);
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) pf[v][u] = (k < kend && row + u < g.n) ? src[u] : (T)0;
      }
    }
  };
  fetch(rbase, 0, min(mi, 64));
  for (int tile = 0; tile < kGemmTiles; ++tile) {
    const int r0 = rbase + tile * kGemmRows;
    if (r0 >= g.n) break;
    T acc[RI][4];
#pragma unroll
    for (int i = 0; i < RI; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = (T)0;
    for (int kb = 0; kb < mi; kb += 64) {
      const int kend = min(mi, kb + 64);
      if (tile == 0 || nkb > 1) {
        __syncthreads();  // previous readers of Bs are done
        const int kpad = (kend - kb + TK - 1) / TK * TK;
        for (int e = tid; e < kpad * TNW; e += NT) {
          const int k = e % kpad, c = e / kpad;
          const int col = c0 + c;
          Bs[k][c] = (kb + k < kend && col < mo) ? from_f64<T>(Bm[(int64_t)col * g.M + kb + k]) : (T)0;
        }
      }
      for (int k0 = kb; k0 < kend; k0 += TK) {
#pragma unroll
        for (int v = 0; v < PV; ++v) {
          const int e = tid + NT * v;
          st4<T>(&As[e / QV][4 * (e % QV)], pf[v]);
        }
        if (k0 + TK < kend) {
          fetch(r0, k0 + TK, kend);
        } else if (kend < mi) {
          fetch(r0, kend, min(mi, kend + 64));
        } else if (tile + 1 < kGemmTiles && r0 + kGemmRows < g.n) {
          fetch(r0 + kGemmRows, 0, min(mi, 64));
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
          T av[RI], bv[4];
#pragma unroll
          for (int i = 0; i < RI; i += 4) {
            T v[4];
            Vec4<T>::ld(&As[kk][ty * RI + i], v);
#pragma unroll
            for (int u = 0; u < 4; ++u) av[i + u] = v[u];
          }
          Vec4<T>::ld(&Bs[k0 - kb + kk][tx * 4], bv);
#pragma unroll
          for (int i = 0; i < RI; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int col = c0 + tx * 4 + j;
      if (col >= mo) continue;
#pragma unroll
      for (int i = 0; i < RI; i += 4) {
        const int row = r0 + ty * RI + i;
        if (row >= g.n) continue;
        const int64_t o = (int64_t)col * g.ld + row;
        T v[4];
        if (vec && row + 3 < g.n) {
          if (mode == 1) {
            T z[4];
            ld4<T>(Z + o, z);
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = (T)(z[u] - acc[i + u][j]);
          } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = acc[i + u][j];
          }
          st4<T>(O + o, v);
        } else {
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (row + u < g.n) O[o + u] = (mode == 1) ? (T)(Z[o + u] - acc[i + u][j]) : acc[i + u][j];
        }
      }
    }
  }
  __syncthreads();  // the next column block restages Bs
}

// Out = In * Bm (or Zsub - In * Bm) for narrow products (mi <= KMAX, mo <= 64),
// thread per row: each thread holds R rows of In (KMAX values each, zero past
// mi) in registers and forms their outputs one column at a time against Bm^T,
// staged in shared memory once per CTA and read by broadcast.  Every output is
// the same FMA chain as in gemm_block (k = 0, 1, ... from zero; the zero
// padding of K adds exact zeros, which leave a sum unchanged), so both paths
// give identical results.  Loads and stores are coalesced along rows.
template <typename T, int KMAX, int R>
__device__ __forceinline__ void gemm_rows(const TallGeom& g, const T* __restrict__ X, const double* __restrict__ Bm,
                                          T* __restrict__ O, const T* __restrict__ Z, int mode, int mi, int mo,
                                          int rbase, T (*Bt)[KMAX]) {
  constexpr int kRows = kGemmRows * kGemmTiles;  // rows per CTA
  static_assert(kRows % (NT * R) == 0, "whole passes");
  const int tid = threadIdx.x;
  const int mi4 = (mi + 3) & ~3;
  for (int e = tid; e < mo * KMAX; e += NT) {
    const int k = e % KMAX, c = e / KMAX;
    Bt[c][k] = (k < mi) ? from_f64<T>(Bm[(int64_t)c * g.M + k]) : (T)0;
  }
  __syncthreads();
  for (int pass = 0; pass < kRows / (NT * R); ++pass) {
    int row[R];
    T x[R][KMAX];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      row[r] = rbase + pass * NT * R + r * NT + tid;
#pragma unroll
      for (int k = 0; k < KMAX; ++k) x[r][k] = (k < mi && row[r] < g.n) ? X[(int64_t)k * g.ld + row[r]] : (T)0;
    }
    for (int c = 0; c < mo; ++c) {
      T acc[R];
#pragma unroll
      for (int r = 0; r < R; ++r) acc[r] = (T)0;
#pragma unroll
      for (int k = 0; k < KMAX; k += 4) {
        if (k < mi4) {
          T b[4];
          ld4<T>(&Bt[c][k], b);
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int r = 0; r < R; ++r) acc[r] = fma(x[r][k + u], b[u], acc[r]);
        }
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (row[r] >= g.n) continue;
        const int64_t o = (int64_t)c * g.ld + row[r];
        O[o] = (mode == 1) ? (T)(Z[o] - acc[r]) : acc[r];
      }
    }
  }
}

// Thread-per-row products in a kernel of their own: mi <= 32 input columns and
// mo <= 64 outputs with RPT rows per thread (RPT = 2 halves the shared-memory
// reads per multiply-add, RPT = 1 halves the registers of that path), and
// (FP32) mi <= 64 with one row per thread.  Problems of other widths return at
// once here and are served by k_gemm_nn, which is launched only when the plan's
// index capacity allows such widths, so that the common case is one launch
// without the register-tiled paths' registers.
template <typename T>
__host__ __device__ constexpr bool gemm_rows_covers(int mi, int mo) {
  return mo <= 64 && (mi <= 32 || (sizeof(T) == 4 && mi <= 64));
}

template <typename T, int RPT>
__global__ void __launch_bounds__(NT, 2)
    k_gemm_narrow(TallGeom g, const SolveState* __restrict__ st_all, Strided<const T> in, int sel_in,
                  Strided<const double> bm, int sel_out, Strided<T> out, Strided<const T> zsub, int mode) {
  const int slot = slot_of(g, blockIdx.z >> 1), side = blockIdx.z & 1;
  if (slot < 0) return;
  const SolveState& st = st_all[slot];
  if (!st.active) return;
  const int mi = dim_of(st, side, sel_in), mo = dim_of(st, side, sel_out);
  const int rbase = blockIdx.x * kGemmRows * kGemmTiles;
  if (rbase >= g.n || mo < 1 || !gemm_rows_covers<T>(mi, mo)) return;
  __shared__ __align__(16) T Bs[64][64];
  const T* X = in.at(slot, side);
  const double* Bm = bm.at(slot, side);
  T* O = out.at(slot, side);
  const T* Z = (mode == 1) ? zsub.at(slot, side) : nullptr;
  if (mi <= 32) {
    gemm_rows<T, 32, RPT>(g, X, Bm, O, Z, mode, mi, mo, rbase, reinterpret_cast<T(*)[32]>(&Bs[0][0]));
  } else if constexpr (sizeof(T) == 4) {
    gemm_rows<T, 64, 1>(g, X, Bm, O, Z, mode, mi, mo, rbase, Bs);
  }
}

// Every width the thread-per-row kernel leaves: a CTA owns kGemmTiles x
// kGemmRows rows, register tiles, one 32-wide column block when mo <= 32,
// else 64-wide blocks.
template <typename T>
__global__ void __launch_bounds__(NT) k_gemm_nn(TallGeom g, const SolveState* __restrict__ st_all, Strided<const T> in,
                                                int sel_in, Strided<const double> bm, int sel_out, Strided<T> out,
                                                Strided<const T> zsub, int mode) {
  const int slot = slot_of(g, blockIdx.z >> 1), side = blockIdx.z & 1;
  if (slot < 0) return;
  const SolveState& st = st_all[slot];
  if (!st.active) return;
  const int mi = dim_of(st, side, sel_in), mo = dim_of(st, side, sel_out);
  const int rbase = blockIdx.x * kGemmRows * kGemmTiles;
  if (rbase >= g.n || mo < 1 || gemm_rows_covers<T>(mi, mo)) return;
  __shared__ __align__(16) T As[TK][kGemmRows];
  __shared__ __align__(16) T Bs[64][64];
  const T* X = in.at(slot, side);
  const double* Bm = bm.at(slot, side);
  T* O = out.at(slot, side);
  const T* Z = (mode == 1) ? zsub.at(slot, side) : nullptr;
  // 4-row vectors need 16-byte aligned columns (ld is a multiple of 32)
  const bool vec = ((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(O) |
                     reinterpret_cast<uintptr_t>(Z)) & 15) == 0 && (g.ld & 3) == 0;
  if (mo <= 32) {
    gemm_block<T, 32>(g, X, Bm, O, Z, mode, mi, mo, rbase, 0, vec, As, Bs);
  } else {
    for (int c0 = 0; c0 < mo; c0 += 64) gemm_block<T, 64>(g, X, Bm, O, Z, mode, mi, mo, rbase, c0, vec, As, Bs);
  }
}

// Tiled Gram partials for widths above kSmallGram: the CTA loops over the
// 64 x 64 output tiles (upper tiles only when symmetric) of its row block,
// accumulating in TA.
template <typename T, typename TA>
__device__ void gram_tiled(const TallGeom& g, const T* __restrict__ X, const T* __restrict__ Y, int mx, int my,
                           int rbeg, int rend, double* __restrict__ P, bool symmetric, unsigned char* smem) {
  T (*As)[TM + 1] = reinterpret_cast<T (*)[TM + 1]>(smem);
  T (*Bs)[TN + 1] = reinterpret_cast<T (*)[TN + 1]>(smem + sizeof(T) * TKG * (TM + 1));
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  for (int a0 = 0; a0 < mx; a0 += TM) {
    for (int b0 = symmetric ? a0 : 0; b0 < my; b0 += TN) {
      TA acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = (TA)0;
      for (int r = rbeg; r < rend; r += TKG) {
#pragma unroll
        for (int q = 0; q < (TKG * TM) / NT; ++q) {
          const int e = tid + NT * q;
          const int kk = e % TKG, c = e / TKG;
          const int row = r + kk;
          As[kk][c] = (row < rend && a0 + c < mx) ? X[(int64_t)(a0 + c) * g.ld + row] : (T)0;
          Bs[kk][c] = (row < rend && b0 + c < my) ? Y[(int64_t)(b0 + c) * g.ld + row] : (T)0;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < TKG; ++kk) {
          TA av[4], bv[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) av[i] = (TA)As[kk][ty + 16 * i];
#pragma unroll
          for (int j = 0; j < 4; ++j) bv[j] = (TA)Bs[kk][tx + 16 * j];
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int a = a0 + ty + 16 * i;
        if (a >= mx) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int b = b0 + tx + 16 * j;
          if (b < my) P[(int64_t)b * g.M + a] = to_f64(acc[i][j]);
        }
      }
    }
  }
}

// TS consecutive elements of a shared-memory row (16-byte aligned for TS = 4
// floats or 2 doubles, 32-byte for 4 doubles).
template <typename TA, int TS>
__device__ __forceinline__ void load_ts(const TA* p, TA (&v)[TS]) {
  if constexpr (sizeof(TA) == 4 && TS == 4) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
  } else if constexpr (sizeof(TA) == 8 && TS == 2) {
    const double2 q = *reinterpret_cast<const double2*>(p);
    v[0] = q.x, v[1] = q.y;
  } else {
#pragma unroll
    for (int u = 0; u < TS; ++u) v[u] = p[u];
  }
}

// Output tile t -> (ia, ib): upper tiles column by column when symmetric.
__device__ __forceinline__ void tile_coords(int t, bool symmetric, int tx, int& ia, int& ib) {
  if (symmetric) {
    ib = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
    while ((ib + 1) * (ib + 2) / 2 <= t) ++ib;
    while (ib * (ib + 1) / 2 > t) --ib;
    ia = t - ib * (ib + 1) / 2;
  } else {
    ia = t % tx;
    ib = t / tx;
  }
}

// Gram partials for small column counts (mx, my <= kSmallGram), register
// tiled: the output is cut into TS x TS tiles (upper tiles only when
// symmetric).  With at most NT tiles, every tile has one thread in each of
// NT / ntile row groups, which split the rows of each shared-memory chunk and
// add their sums in shared memory at the end; with more tiles than threads a
// thread owns up to TPT tiles over all rows.  Exits to the tiled kernel when
// either count exceeds kSmallGram.  TS = 4 for FP32 accumulation (16 FMAs per
// two 16-byte loads); TS = 2 with four tiles per thread for FP64 accumulation,
// whose pipe is the bound and which wastes fewer FMAs on diagonal and padding
// entries.  TA is the accumulation type: FP64 for every Gram of the FP64 path
// and for the first (ill-conditioned) CholeskyQR pass of the FP32 iterations,
// FP32 for the FP32 iterations' later passes and cross-Grams.
template <typename T, typename TA, int TS, int TPT>
__global__ void __launch_bounds__(NT) k_gram_small(TallGeom g, const SolveState* __restrict__ st_all,
                                                   Strided<const T> xs, int sel_x, Strided<const T> ys, int sel_y,
                                                   double* __restrict__ part, bool symmetric) {
  constexpr int KC = kSmallRows;          // rows per shared-memory chunk
  constexpr int LDS = kSmallGram + 4;     // padded row length (keeps 16-byte alignment)
  static_assert((kSmallGram / TS) * (kSmallGram / TS) <= NT * TPT, "tiles per thread");
  const int slot = slot_of(g, blockIdx.z >> 1), side = blockIdx.z & 1;
  if (slot < 0) return;
  const SolveState& st = st_all[slot];
  if (!st.active) return;
  const int mx = dim_of(st, side, sel_x), my = dim_of(st, side, sel_y);
  if (mx < 1 || my < 1) return;
  const int blk = blockIdx.x;
  const int rbeg = blk * g.rows_per_block;
  const int rend = min(g.n, rbeg + g.rows_per_block);
  const T* X = xs.at(slot, side);
  const T* Y = ys.at(slot, side);
  double* P = part + ((int64_t)(slot * 2 + side) * g.NB + blk) * (int64_t)g.M * g.M;
  // the chunk is staged in the accumulation type: each element is converted once
  constexpr size_t kTileBytes = 2 * KC * LDS * sizeof(TA);
  constexpr size_t kRedBytes = (size_t)NT * TS * TS * sizeof(TA);
  constexpr size_t kFallBytes = (size_t)TKG * (TM + 1 + TN + 1) * sizeof(T);
  constexpr size_t kSmem = kTileBytes > kRedBytes ? (kTileBytes > kFallBytes ? kTileBytes : kFallBytes)
                                                  : (kRedBytes > kFallBytes ? kRedBytes : kFallBytes);
  __shared__ __align__(16) unsigned char gsm[kSmem];
  if (mx > kSmallGram || my > kSmallGram) {
    gram_tiled<T, TA>(g, X, Y, mx, my, rbeg, rend, P, symmetric, gsm);
    return;
  }
  TA (*Xs)[LDS] = reinterpret_cast<TA (*)[LDS]>(gsm);
  TA (*Ys)[LDS] = reinterpret_cast<TA (*)[LDS]>(gsm + (size_t)KC * LDS * sizeof(TA));
  const bool same = symmetric;
  const int tx = (mx + TS - 1) / TS, ty = (my + TS - 1) / TS;
  const int ntile = same ? tx * (tx + 1) / 2 : tx * ty;
  const int G = ntile <= NT ? NT / ntile : 1;  // row groups
  const int tid = threadIdx.x;
  const int grp = ntile <= NT ? tid / ntile : 0;
  const int t0 = ntile <= NT ? tid - grp * ntile : tid;
  int ia[TPT], ib[TPT];
  bool own[TPT];
#pragma unroll
  for (int q = 0; q < TPT; ++q) {
    const int t = t0 + q * NT;
    own[q] = grp < G && t < ntile && (q == 0 || ntile > NT);
    ia[q] = ib[q] = 0;
    if (own[q]) tile_coords(t, same, tx, ia[q], ib[q]);
  }
  TA acc[TPT][TS][TS];
#pragma unroll
  for (int q = 0; q < TPT; ++q)
#pragma unroll
    for (int i = 0; i < TS; ++i)
#pragma unroll
      for (int j = 0; j < TS; ++j) acc[q][i][j] = (TA)0;
  const int wx = tx * TS, wy = ty * TS;  // padded widths (zero columns beyond mx, my)
  // The next chunk is fetched into registers while the current one is used.
  constexpr int PF = KC * kSmallGram / NT;  // elements per thread and chunk (8)
  T px[PF], py[PF];
  auto fetch = [&](int r) {
#pragma unroll
    for (int q = 0; q < PF; ++q) {
      const int e = tid + NT * q, kk = e % KC, c = e / KC, row = r + kk;
      px[q] = (c < mx && row < rend) ? X[(int64_t)c * g.ld + row] : (T)0;
      if (!same) py[q] = (c < my && row < rend) ? Y[(int64_t)c * g.ld + row] : (T)0;
    }
  };
  fetch(rbeg);
  for (int r = rbeg; r < rend; r += KC) {
#pragma unroll
    for (int q = 0; q < PF; ++q) {
      const int e = tid + NT * q, kk = e % KC, c = e / KC;
      if (c < wx) Xs[kk][c] = (TA)px[q];
      if (!same && c < wy) Ys[kk][c] = (TA)py[q];
    }
    __syncthreads();
    if (r + KC < rend) fetch(r + KC);
    const TA(*Bsrc)[LDS] = same ? Xs : Ys;
#pragma unroll
    for (int q = 0; q < TPT; ++q) {
      if (!own[q]) continue;
      for (int kk = grp; kk < KC; kk += G) {
        TA av[TS], bv[TS];
        load_ts<TA, TS>(&Xs[kk][TS * ia[q]], av);
        load_ts<TA, TS>(&Bsrc[kk][TS * ib[q]], bv);
#pragma unroll
        for (int i = 0; i < TS; ++i)
#pragma unroll
          for (int j = 0; j < TS; ++j) acc[q][i][j] = fma(av[i], bv[j], acc[q][i][j]);
      }
    }
    __syncthreads();
  }
  if (G == 1) {
    // one thread per tile: write directly
#pragma unroll
    for (int q = 0; q < TPT; ++q) {
      if (!own[q]) continue;
#pragma unroll
      for (int i = 0; i < TS; ++i)
#pragma unroll
        for (int j = 0; j < TS; ++j) {
          const int a = TS * ia[q] + i, b = TS * ib[q] + j;
          if (a < mx && b < my && (!same || a <= b)) P[(int64_t)b * g.M + a] = to_f64(acc[q][i][j]);
        }
    }
    return;
  }
  // sum the row groups' tiles (one tile per thread here): red[grp][t][TS*TS]
  TA* red = reinterpret_cast<TA*>(gsm);
  if (own[0]) {
#pragma unroll
    for (int i = 0; i < TS; ++i)
#pragma unroll
      for (int j = 0; j < TS; ++j) red[((size_t)grp * ntile + t0) * TS * TS + i * TS + j] = acc[0][i][j];
  }
  __syncthreads();
  for (int e = tid; e < ntile * TS * TS; e += NT) {
    const int tt = e / (TS * TS), ij = e % (TS * TS), i = ij / TS, j = ij % TS;
    TA v = (TA)0;
    for (int q = 0; q < G; ++q) v += red[((size_t)q * ntile + tt) * TS * TS + ij];
    int ta, tb;
    tile_coords(tt, same, tx, ta, tb);
    const int a = TS * ta + i, b = TS * tb + j;
    if (a < mx && b < my && (!same || a <= b)) P[(int64_t)b * g.M + a] = to_f64(v);
  }
}

// hi + lo += a * b without rounding the product: a*b = p + pe exactly (one FMA),
// p is added to hi by TwoSum (Knuth) and every rounding error goes to lo.  The
// _rn intrinsics keep the compiler from contracting or reordering the steps.
// (hi, lo) <- TwoSum(hi, lo): the same value with |lo| <= ulp(hi) / 2.
__device__ __forceinline__ void df_renorm(float& hi, float& lo) {
  const float s = __fadd_rn(hi, lo);
  const float bb = __fsub_rn(s, hi);
  lo = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(lo, bb));
  hi = s;
}

__device__ __forceinline__ void df_add_product(float a, float b, float& hi, float& lo) {
  const float p = __fmul_rn(a, b);
  const float pe = __fmaf_rn(a, b, -p);
  const float s = __fadd_rn(hi, p);
  const float bb = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(e, pe));
}

// Gram partials of FP32 data with near-FP64 accuracy on the FP32 pipe (the first,
// ill-conditioned CholeskyQR pass of the FP32 iterations).  Same tiling as
// k_gram_small<float, float, 4, 1>, but each entry is a double-float (hi, lo)
// sum of exact products, renormalised by TwoSum after every chunk so that lo
// stays within an ulp of hi: the relative error stays below ~n eps32^2 (6e-11
// at n = 4095) in the worst case, ~1e-13 typically.  Only the row groups'
// final sums touch GB300's FP64 pipe (1/64 of its FP32 pipe): each (hi, lo)
// pair is widened exactly on the integer pipe and the groups' values are added
// in FP64.  At most 85 registers per thread, three CTAs per SM.

__global__ void __launch_bounds__(NT, 3) k_gram_df(TallGeom g, const SolveState* __restrict__ st_all,
                                                Strided<const float> xs, int sel_x, double* __restrict__ part) {
  constexpr int KC = kSmallRows;
  constexpr int LDS = kSmallGram + 4;
  constexpr int TS = 4;
  const int slot = slot_of(g, blockIdx.z >> 1), side = blockIdx.z & 1;
  if (slot < 0) return;
  const SolveState& st = st_all[slot];
  if (!st.active) return;
  const int mx = dim_of(st, side, sel_x);
  if (mx < 1) return;
  const int blk = blockIdx.x;
  const int rbeg = blk * g.rows_per_block;
  const int rend = min(g.n, rbeg + g.rows_per_block);
  const float* X = xs.at(slot, side);
  double* P = part + ((int64_t)(slot * 2 + side) * g.NB + blk) * (int64_t)g.M * g.M;
  constexpr size_t kTileBytes = KC * LDS * sizeof(float);
  constexpr size_t kRedBytes = (size_t)NT * TS * TS * sizeof(double);
  constexpr size_t kFallBytes = (size_t)TKG * (TM + 1 + TN + 1) * sizeof(float);
  constexpr size_t kSmem = kRedBytes > kTileBytes ? (kRedBytes > kFallBytes ? kRedBytes : kFallBytes)
                                                  : (kTileBytes > kFallBytes ? kTileBytes : kFallBytes);
  __shared__ __align__(16) unsigned char gsm[kSmem];
  if (mx > kSmallGram) {
    gram_tiled<float, double>(g, X, X, mx, mx, rbeg, rend, P, true, gsm);
    return;
  }
  float (*Xs)[LDS] = reinterpret_cast<float (*)[LDS]>(gsm);
  const int tx = (mx + TS - 1) / TS;
  const int ntile = tx * (tx + 1) / 2;  // <= 136
  const int G = NT / ntile;
  const int tid = threadIdx.x;
  const int grp = tid / ntile, t0 = tid - grp * ntile;
  const bool own = grp < G;
  int ia = 0, ib = 0;
  if (own) tile_coords(t0, true, tx, ia, ib);
  float hi[TS][TS], lo[TS][TS];
#pragma unroll
  for (int i = 0; i < TS; ++i)
#pragma unroll
    for (int j = 0; j < TS; ++j) {
      hi[i][j] = 0.f;
      lo[i][j] = 0.f;
    }
  const int wx = tx * TS;
  constexpr int PF = KC * kSmallGram / NT;  // elements per thread and chunk (8)
  float px[PF];
  auto fetch = [&](int r) {
#pragma unroll
    for (int q = 0; q < PF; ++q) {
      const int e = tid + NT * q, kk = e % KC, c = e / KC, row = r + kk;
      px[q] = (c < mx && row < rend) ? X[(int64_t)c * g.ld + row] : 0.f;
    }
  };
  fetch(rbeg);
  for (int r = rbeg; r < rend; r += KC) {
#pragma unroll
    for (int q = 0; q < PF; ++q) {
      const int e = tid + NT * q, kk = e % KC, c = e / KC;
      if (c < wx) Xs[kk][c] = px[q];
    }
    __syncthreads();
    if (r + KC < rend) fetch(r + KC);
    if (own) {
      for (int kk = grp; kk < KC; kk += G) {
        float av[TS], bv[TS];
        load_ts<float, TS>(&Xs[kk][TS * ia], av);
        load_ts<float, TS>(&Xs[kk][TS * ib], bv);
#pragma unroll
        for (int i = 0; i < TS; ++i)
#pragma unroll
          for (int j = 0; j < TS; ++j) df_add_product(av[i], bv[j], hi[i][j], lo[i][j]);
      }
#pragma unroll
      for (int i = 0; i < TS; ++i)
#pragma unroll
        for (int j = 0; j < TS; ++j) df_renorm(hi[i][j], lo[i][j]);
    }
    __syncthreads();
  }
  if (G == 1) {
    if (own) {
#pragma unroll
      for (int i = 0; i < TS; ++i)
#pragma unroll
        for (int j = 0; j < TS; ++j) {
          const int a = TS * ia + i, b = TS * ib + j;
          if (a < mx && b < mx && a <= b) P[(int64_t)b * g.M + a] = f32_to_f64(hi[i][j]) + f32_to_f64(lo[i][j]);
        }
    }
    return;
  }
  // red[grp][tile][TS * TS]: each (hi, lo) sum as the exact FP64 value hi + lo
  double* red = reinterpret_cast<double*>(gsm);
  if (own) {
#pragma unroll
    for (int i = 0; i < TS; ++i)
#pragma unroll
      for (int j = 0; j < TS; ++j)
        red[((size_t)grp * ntile + t0) * TS * TS + i * TS + j] = f32_to_f64(hi[i][j]) + f32_to_f64(lo[i][j]);
  }
  __syncthreads();
  for (int e = tid; e < ntile * TS * TS; e += NT) {
    const int tt = e / (TS * TS), ij = e % (TS * TS), i = ij / TS, j = ij % TS;
    int ta, tb;
    tile_coords(tt, true, tx, ta, tb);
    const int a = TS * ta + i, b = TS * tb + j;
    if (a >= mx || b >= mx || a > b) continue;
    double v = 0.0;
    for (int q = 0; q < G; ++q) v += red[((size_t)q * ntile + tt) * TS * TS + ij];
    P[(int64_t)b * g.M + a] = v;
  }
}

__global__ void k_reduce(TallGeom g, const SolveState* __restrict__ st_all, int sel_x, int sel_y,
                         const double* __restrict__ part, Strided<double> G, bool symmetric) {
  const int slot = slot_of(g, blockIdx.y >> 1), side = blockIdx.y & 1;
  if (slot < 0) return;
  const SolveState& st = st_all[slot];
  if (!st.active) return;
  const int mx = dim_of(st, side, sel_x), my = dim_of(st, side, sel_y);
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int a = (int)(e % g.M), b = (int)(e / g.M);
  if (b >= g.M || a >= mx || b >= my) return;
  if (symmetric && b < a) return;
  const double* P = part + (int64_t)(slot * 2 + side) * g.NB * (int64_t)g.M * g.M + (int64_t)b * g.M + a;
  double s = 0.0;
  for (int blk = 0; blk < g.NB; ++blk) s += P[(int64_t)blk * g.M * g.M];
  double* out = G.at(slot, side);
  out[(int64_t)b * g.M + a] = s;
  if (symmetric) out[(int64_t)a * g.M + b] = s;
}

// Bitonic sort of (score desc, index asc) pairs in shared memory; len a power of two.
template <typename K>
__device__ inline bool before(K sa, int ia, K sb, int ib) {
  return (sa > sb) || (sa == sb && ia < ib);
}

template <typename K>
__device__ void bitonic_sort(K* key, int* idx, int len) {
  for (int size = 2; size <= len; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = threadIdx.x; t < len; t += blockDim.x) {
        const int p = t ^ stride;
        if (p > t) {
          const bool up = ((t & size) == 0);
          const bool t_first = before(key[t], idx[t], key[p], idx[p]);
          if (up != t_first) {
            const K k = key[t];
            key[t] = key[p];
            key[p] = k;
            const int i = idx[t];
            idx[t] = idx[p];
            idx[p] = i;
          }
        }
      }
      __syncthreads();
    }
  }
}

template <typename T>
__global__ void k_leverage(TallGeom g, const SolveState* __restrict__ st_all, Strided<const T> us, int sel,
                           double* __restrict__ cscore, int32_t* __restrict__ cidx, int cand_blocks,
                           int cand_per_block, int rows_per_cand_block, int sort_len, LevSample ls) {
  // Scores, their sums and the sort keys are in the data's precision (T): the
  // FP32 iterations keep them off the FP64 pipe.
  extern __shared__ unsigned char smem_raw[];
  T* key = reinterpret_cast<T*>(smem_raw);
  int* id = reinterpret_cast<int*>(key + sort_len);
  const int slot = slot_of(g, blockIdx.y >> 1), side = blockIdx.y & 1;
  if (slot < 0) return;
  const SolveState& st = st_all[slot];
  if (!st.active) return;
  const int c = dim_of(st, side, sel);
  const int blk = blockIdx.x;
  const int rbeg = blk * rows_per_cand_block;
  const int rend = min(g.n, rbeg + rows_per_cand_block);
  const T* U = us.at(slot, side);
  if (ls.on) {
    // Bernoulli: keep row i with probability min(1, c pi_i) = min(1, factor s_i).
    // Only the kept rows are sorted (best first, ties to the lower index): they
    // are appended to the front of key / id, then sorted over the next power
    // of two, which orders them exactly as a sort of the whole block would.
    __shared__ int kept;
    if (threadIdx.x == 0) kept = 0;
    __syncthreads();
    for (int t = threadIdx.x; t < sort_len; t += blockDim.x) {
      const int row = rbeg + t;
      if (row >= rend) continue;
      T s = T(0);
#pragma unroll 4
      for (int q = 0; q < c; ++q) {
        const T v = U[(int64_t)q * g.ld + row];
        s = fma(v, v, s);
      }
      const double pr = fmin(1.0, ls.factor * (double)s);
      if (philox_uniform(ls.seed, (uint32_t)(st.k + ls.k_ofs), (uint32_t)side, (uint32_t)row) < pr) {
        const int at = atomicAdd(&kept, 1);
        key[at] = s;
        id[at] = row;
      }
    }
    __syncthreads();
    const int nk = kept;
    int len = 1;
    while (len < nk) len <<= 1;
    for (int t = nk + threadIdx.x; t < len; t += blockDim.x) {
      key[t] = T(-1);
      id[t] = 0x7fffffff;
    }
    __syncthreads();
    bitonic_sort<T>(key, id, len);
    const int64_t base = ((int64_t)(slot * 2 + side) * cand_blocks + blk) * cand_per_block;
    for (int t = threadIdx.x; t < cand_per_block; t += blockDim.x) {
      const bool ok = t < nk;
      cscore[base + t] = ok ? (double)key[t] : -1.0;
      cidx[base + t] = ok ? id[t] : -1;
    }
    return;
  }
  for (int t = threadIdx.x; t < sort_len; t += blockDim.x) {
    const int row = rbeg + t;
    T s = T(-1);
    int ii = 0x7fffffff;
    if (row < rend) {
      s = T(0);
#pragma unroll 4
      for (int q = 0; q < c; ++q) {
        const T v = U[(int64_t)q * g.ld + row];
        s = fma(v, v, s);
      }
      ii = row;
    }
    key[t] = s;
    id[t] = ii;
  }
  __syncthreads();
  bitonic_sort<T>(key, id, sort_len);
  const int64_t base = ((int64_t)(slot * 2 + side) * cand_blocks + blk) * cand_per_block;
  for (int t = threadIdx.x; t < cand_per_block; t += blockDim.x) {
    const bool ok = (t < (ls.on ? cand_per_block : c)) && (t < sort_len) && key[t] >= T(0);
    cscore[base + t] = ok ? (double)key[t] : -1.0;
    cidx[base + t] = ok ? id[t] : -1;
  }
}

// ------------------------------------------------------------------ launches

static inline int cdiv(int a, int b) { return (a + b - 1) / b; }

template <typename T>
cudaError_t launch_cross(const TallGeom& g, const SolveState* st, const CrossArgs<T>& a, cudaStream_t s) {
  dim3 grid(cdiv(g.n, NT), 1, g.nslots * 2);
  k_cross<T><<<grid, NT, 0, s>>>(g, st, a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gemm_nn(const TallGeom& g, const SolveState* st, Strided<const T> in, int sel_in,
                           Strided<const double> bm, int sel_out, Strided<T> out, Strided<const T> zsub, int mode,
                           cudaStream_t s) {
  // the thread-per-row widths, then (when the index capacity allows wider
  // products) every other width, over the same problems
  const dim3 grid(cdiv(g.n, kGemmRows * kGemmTiles), 1, g.nslots * 2);
  const int rpt = g.gemm_rpt > 0 ? g.gemm_rpt : (sizeof(T) == 4 ? 2 : 1);
  if (rpt == 2)
    k_gemm_narrow<T, 2><<<grid, NT, 0, s>>>(g, st, in, sel_in, bm, sel_out, out, zsub, mode);
  else
    k_gemm_narrow<T, 1><<<grid, NT, 0, s>>>(g, st, in, sel_in, bm, sel_out, out, zsub, mode);
  if (gemm_wide_possible<T>(g.M)) k_gemm_nn<T><<<grid, NT, 0, s>>>(g, st, in, sel_in, bm, sel_out, out, zsub, mode);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gram(const TallGeom& g, const SolveState* st, Strided<const T> x, int sel_x,
                        Strided<const T> y, int sel_y, double* part, Strided<double> G, bool symmetric,
                        cudaStream_t s, bool acc64) {
  if (sizeof(T) == 4 && acc64 && symmetric && x.base == y.base)
    k_gram_df<<<dim3(g.NB, 1, g.nslots * 2), NT, 0, s>>>(g, st, Strided<const float>{(const float*)x.base,
                                                                                   x.side_stride, x.slot_stride},
                                                         sel_x, part);
  else if (acc64 || sizeof(T) == 8)
    k_gram_small<T, double, 2, 4><<<dim3(g.NB, 1, g.nslots * 2), NT, 0, s>>>(g, st, x, sel_x, y, sel_y, part,
                                                                             symmetric);
  else
    k_gram_small<T, float, 4, 1><<<dim3(g.NB, 1, g.nslots * 2), NT, 0, s>>>(g, st, x, sel_x, y, sel_y, part,
                                                                            symmetric);
  (void)G;
  return cudaGetLastError();
}

cudaError_t launch_reduce(const TallGeom& g, const SolveState* st, int sel_x, int sel_y, const double* part,
                          Strided<double> G, bool symmetric, cudaStream_t s) {
  dim3 rgrid(cdiv(g.M * g.M, 256), g.nslots * 2);
  k_reduce<<<rgrid, 256, 0, s>>>(g, st, sel_x, sel_y, part, G, symmetric);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_leverage(const TallGeom& g, SolveState* st, Strided<const T> U, int sel, double* cand_score,
                            int32_t* cand_idx, int cand_blocks, int cand_per_block, cudaStream_t s, LevSample ls) {
  const int rows = cdiv(g.n, cand_blocks);
  int len = 1;
  while (len < rows) len <<= 1;
  const size_t smem = (size_t)len * (sizeof(T) + sizeof(int));
  auto kern = k_leverage<T>;
  dim3 grid(cand_blocks, g.nslots * 2);
  kern<<<grid, 512, smem, s>>>(g, st, U, sel, cand_score, cand_idx, cand_blocks, cand_per_block, rows, len, ls);
  return cudaGetLastError();
}

cudaError_t tall_configure() {
  const int bytes = 8192 * (int)(sizeof(double) + sizeof(int));  // largest leverage sort
  cudaError_t e = cudaFuncSetAttribute(k_leverage<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_leverage<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  return e;
}

#define LRP_INST(T)                                                                                           \
  template cudaError_t launch_cross<T>(const TallGeom&, const SolveState*, const CrossArgs<T>&, cudaStream_t); \
  template cudaError_t launch_gemm_nn<T>(const TallGeom&, const SolveState*, Strided<const T>, int,          \
                                         Strided<const double>, int, Strided<T>, Strided<const T>, int,       \
                                         cudaStream_t);                                                        \
  template cudaError_t launch_gram<T>(const TallGeom&, const SolveState*, Strided<const T>, int,             \
                                      Strided<const T>, int, double*, Strided<double>, bool, cudaStream_t,    \
                                      bool);                                                                  \
  template cudaError_t launch_leverage<T>(const TallGeom&, SolveState*, Strided<const T>, int, double*,      \
                                          int32_t*, int, int, cudaStream_t, LevSample);
LRP_INST(double)
LRP_INST(float)
#undef LRP_INST

}  // namespace lrp
