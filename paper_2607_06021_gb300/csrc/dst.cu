// Orthonormal DST-I of columns (paper Sec. 3: Z_{ik} = sqrt(2/(n+1)) sin(i k pi/(n+1)),
// Z symmetric orthogonal, applied to n x r factors "in batches along dimensions
// independently without any global transpose", Sec. 1 / Sec. 3.2).
//
// Two methods, both written from the DFT definition.  N = n+1 <= 8192 (FP64,
// double-float) or 16384 (FP32): one column per group of threads in shared
// memory, through a real FFT of length N (a complex FFT of length N/2), see
// k_dst1_half.  Larger N: the odd extension y = [0, x_1..x_n, 0, -x_n..-x_1] of
// length 2N has DFT Y_k = -2i S_k, S_k = sum_j x_j sin(pi j k / N); packing
// z_j = y_{2j} + i y_{2j+1} (j < N) gives one complex FFT of length N, run as a
// four-step FFT through HBM (k_dst1_passA/B); the even/odd split E_k = (Z_k +
// conj Z_{N-k})/2, O_k = (Z_k - conj Z_{N-k})/(2i) recovers Y_k = E_k +
// e^{-i pi k/N} O_k, so S_k = -Im(Y_k)/2 and (Z x)_k = sqrt(2/N) S_k.
//
// The twiddle table e^{-i pi k/N} (length N, FP64, FP32 or double-float) is
// built once per size and stays cache-resident.
#include <cuda_runtime.h>
#include <math.h>

#include <type_traits>

#include "common.cuh"
#include "dfloat.cuh"
#include "dst.cuh"
#include "f64cvt.cuh"

namespace lrp {

template <typename T>
struct cplx {
  T re, im;
};

// An input element in the compute type.  FP64 data for an FP32 transform are
// rounded on the integer pipe (f64_to_f32_rn: the same value as the hardware
// conversion, without GB300's FP64 pipe).
template <typename TC, typename TIn>
__device__ __forceinline__ TC to_tc(TIn v) {
  if constexpr (std::is_same<TIn, double>::value && std::is_same<TC, float>::value) {
    return f64_to_f32_rn(v);
  } else {
    return TC(v);
  }
}

// An output element in the output type (the integer-pipe conversions again).
template <typename TOut, typename TC>
__device__ __forceinline__ TOut from_tc(TC v) {
  if constexpr (std::is_same<TOut, double>::value && std::is_same<TC, float>::value) {
    return f32_to_f64(v);
  } else if constexpr (std::is_same<TOut, float>::value && std::is_same<TC, double>::value) {
    return f64_to_f32_rn(v);
  } else {
    return (TOut)v;
  }
}

template <typename TC>
__global__ void k_twiddle(cplx<TC>* tw, int N) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  double s, c;
  sincospi((double)k / (double)N, &s, &c);  // e^{-i pi k / N}
  tw[k].re = (TC)c;
  tw[k].im = (TC)(-s);
}

// (a, c) <- (a + w c, a - w c), the operations of one radix-2 butterfly below.
template <typename TC>
__device__ __forceinline__ void butterfly(cplx<TC>& a, cplx<TC>& c, const cplx<TC>& w) {
  const TC tr = w.re * c.re - w.im * c.im;
  const TC ti = w.re * c.im + w.im * c.re;
  c.re = a.re - tr;
  c.im = a.im - ti;
  a.re = a.re + tr;
  a.im = a.im + ti;
}

// ---------------------------------------------------------------- shared memory
// For N = n+1 <= 8192 (FP64, double-float) or 16384 (FP32) one column is
// transformed in shared memory by a real FFT of HALF the length of the odd
// extension (written from the DFT definition; the pre-processing is the
// classical one for the sine transform, see e.g. Numerical Recipes, "sine
// transform").  With x_0 = x_N = 0, a_j = x_j + x_{N-j}, b_j = x_j - x_{N-j}:
//
//   u_j = sin(pi j / N) a_j + b_j / 2,                   j = 0..N-1,
//   U_k = sum_j u_j e^{-2 pi i j k / N} = R_k - i I_k,   k = 0..N/2,
//
// and the symmetries of a_j (even about N/2), b_j (odd) and the sines give
//
//   S_{2k}   = I_k,                      S_{2k+1} = S_{2k-1} + R_k,  S_1 = R_0 / 2,
//
// for S_k = sum_j x_j sin(pi j k / N); (Z x)_k = sqrt(2/N) S_k.  The real DFT
// U of length N is one complex FFT of length L = N/2 of v_m = u_{2m} + i
// u_{2m+1}, unpacked with U_k = E_k + e^{-2 pi i k/N} O_k, E_k = (V_k +
// conj V_{L-k}) / 2, O_k = (V_k - conj V_{L-k}) / (2i).  The odd outputs are a
// prefix sum, taken as a sequential sum over each thread's 8 consecutive terms
// plus a shuffle-tree scan of the thread totals (error ~ (8 + 2 log2 T) ulp of
// the partial sums).
//
// The complex FFT runs Stockham stages of radix 8 (a last radix-4 or radix-2
// stage when log2 L is not a multiple of 3): each thread holds 8 elements in
// registers per stage, so a stage is one read of the shared buffer, a barrier
// and one write; twiddles e^{-i pi u / N} come from the L1-resident table.
// T_c = L/8 threads serve one column; columns with L < 2048 share a CTA of 256
// threads (2048 / L columns).  Global loads and stores are coalesced along the
// column (the pre-processing reads x_j and x_{N-j} as a forward and a backward
// run; the outputs are staged in shared memory and written in order).
template <typename TC> struct TwVec;
template <> struct TwVec<float> { using V = float2; };
template <> struct TwVec<double> { using V = double2; };
template <> struct TwVec<dfloat> { using V = float4; };

template <typename TC>
__device__ __forceinline__ cplx<TC> tw_load(const cplx<TC>* __restrict__ tw, int k) {
  using V = typename TwVec<TC>::V;
  const V v = __ldg(reinterpret_cast<const V*>(tw) + k);
  cplx<TC> w;
  if constexpr (std::is_same<TC, dfloat>::value) {
    w.re = dfloat(v.x, v.y);
    w.im = dfloat(v.z, v.w);
  } else {
    w.re = v.x;
    w.im = v.y;
  }
  return w;
}

// e^{-i pi u / N} for any integer u >= 0 from the table e^{-i pi t / N}, t < N.
template <typename TC>
__device__ __forceinline__ cplx<TC> tw_any(const cplx<TC>* __restrict__ tw, int u, int N) {
  u &= 2 * N - 1;
  if (u < N) return tw_load(tw, u);
  const cplx<TC> w = tw_load(tw, u - N);
  return {-w.re, -w.im};
}

template <typename TC>
__device__ __forceinline__ cplx<TC> cmul(const cplx<TC>& a, const cplx<TC>& b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename TC>
__device__ __forceinline__ void bfly2(cplx<TC>& a, cplx<TC>& b) {
  const cplx<TC> t = a;
  a = {t.re + b.re, t.im + b.im};
  b = {t.re - b.re, t.im - b.im};
}
template <typename TC>
__device__ __forceinline__ cplx<TC> mul_mi(const cplx<TC>& a) {  // a * (-i)
  return {a.im, -a.re};
}

// In-register DFT of length R (2, 4 or 8), e^{-2 pi i / R}; a radix-2
// decimation-in-frequency network, outputs returned in natural order.
template <typename TC, int R>
__device__ __forceinline__ void dft_small(cplx<TC>* v) {
  if constexpr (R == 2) {
    bfly2(v[0], v[1]);
  } else if constexpr (R == 4) {
    bfly2(v[0], v[2]);
    bfly2(v[1], v[3]);
    v[3] = mul_mi(v[3]);
    bfly2(v[0], v[1]);
    bfly2(v[2], v[3]);
    const cplx<TC> t = v[1];
    v[1] = v[2];
    v[2] = t;
  } else {
    const TC c = TC(0.70710678118654752440);
    bfly2(v[0], v[4]);
    bfly2(v[1], v[5]);
    bfly2(v[2], v[6]);
    bfly2(v[3], v[7]);
    v[5] = {c * (v[5].re + v[5].im), c * (v[5].im - v[5].re)};     // * (1 - i)/sqrt(2)
    v[6] = mul_mi(v[6]);                                             // * (-i)
    v[7] = {c * (v[7].im - v[7].re), TC(0) - c * (v[7].re + v[7].im)};  // * (-1 - i)/sqrt(2)
    bfly2(v[0], v[2]);
    bfly2(v[1], v[3]);
    bfly2(v[4], v[6]);
    bfly2(v[5], v[7]);
    v[3] = mul_mi(v[3]);
    v[7] = mul_mi(v[7]);
    bfly2(v[0], v[1]);
    bfly2(v[2], v[3]);
    bfly2(v[4], v[5]);
    bfly2(v[6], v[7]);
    // bit-reversed -> natural: X0 v0, X1 v4, X2 v2, X3 v6, X4 v1, X5 v5, X6 v3, X7 v7
    cplx<TC> t = v[1];
    v[1] = v[4];
    v[4] = t;
    t = v[3];
    v[3] = v[6];
    v[6] = t;
  }
}

// Shared-memory index of complex element i: one element of padding after
// every 128 bytes, so that the strided writes of the early Stockham stages
// (stride R complex for Ns = 1, runs of 8 for Ns = 8) and the chunked scan
// reads spread over all banks.
template <typename TC>
__device__ __forceinline__ int zpad(int i) {
  constexpr int P = 128 / (int)sizeof(cplx<TC>);
  return i + i / P;
}

// Scalars of one column's shared memory: the padded complex buffer (L + 1
// elements, the extra one for zpad(L)) and the scan buffer (L + L/32).
template <typename TC>
__host__ __device__ constexpr int dst_half_col_scalars(int N) {
  return 2 * ((N / 2) + (N / 2) / (128 / (int)(2 * sizeof(TC))) + 1) + (N / 2) + (N / 2) / 32;
}

// One Stockham stage of radix R on the column's L complex values in z: the
// group's T_c = L/8 threads take butterflies j = t + q T_c (8/R each): inputs
// z[j + r L/R], twiddles e^{-2 pi i r k / (Ns R)} (k = j mod Ns), outputs
// z[(j - k) R + k + r Ns] (indices padded by zpad).  Reads complete before
// writes (barrier).
template <typename TC, int R>
__device__ __forceinline__ void stockham_stage(cplx<TC>* z, int L, int Ns, int N, int t, int Tc,
                                               const cplx<TC>* __restrict__ tw) {
  constexpr int P = 8 / R;
  cplx<TC> v[P][R];
#pragma unroll
  for (int q = 0; q < P; ++q) {
    const int j = t + q * Tc;
#pragma unroll
    for (int r = 0; r < R; ++r) v[q][r] = z[zpad<TC>(j + r * (L / R))];
  }
  __syncthreads();
  const int step = 2 * N / (Ns * R);  // e^{-2 pi i r k / (Ns R)} = e^{-i pi (r k step) / N}
#pragma unroll
  for (int q = 0; q < P; ++q) {
    const int j = t + q * Tc;
    const int k = j & (Ns - 1);
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) v[q][r] = cmul(v[q][r], tw_any(tw, r * k * step, N));
    }
    dft_small<TC, R>(v[q]);
    const int base = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) z[zpad<TC>(base + r * Ns)] = v[q][r];
  }
  __syncthreads();
}

template <typename TC>
__device__ __forceinline__ TC shfl_up_tc(TC v, int d, int width) {
  if constexpr (std::is_same<TC, dfloat>::value) {
    return dfloat(__shfl_up_sync(0xffffffffu, v.hi, d, width), __shfl_up_sync(0xffffffffu, v.lo, d, width));
  } else {
    return __shfl_up_sync(0xffffffffu, v, d, width);
  }
}
template <typename TC>
__device__ __forceinline__ TC shfl_idx_tc(TC v, int src, int width) {
  if constexpr (std::is_same<TC, dfloat>::value) {
    return dfloat(__shfl_sync(0xffffffffu, v.hi, src, width), __shfl_sync(0xffffffffu, v.lo, src, width));
  } else {
    return __shfl_sync(0xffffffffu, v, src, width);
  }
}

// Exclusive scan of one value per thread over a column group of Tc threads
// (Tc a power of two; groups are warp-aligned when Tc >= 32).  wt: shared
// scratch of 32 values per group.  Every thread of the CTA must call it.
template <typename TC>
__device__ __forceinline__ TC group_exclusive_scan(TC v, int t, int Tc, TC* wt) {
  const int width = Tc < 32 ? Tc : 32;
  const int lane = t & (width - 1);
  TC s = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    if (o < width) {
      const TC y = shfl_up_tc(s, o, width);
      if (lane >= o) s = s + y;
    }
  }
  TC ex = shfl_up_tc(s, 1, width);
  if (lane == 0) ex = TC(0);
  if (Tc > 32) {
    const int w = t >> 5, nw = Tc >> 5;
    if (lane == 31) wt[w] = s;
    __syncthreads();
    // inclusive scan of the warp totals in every warp, then the prefix before w
    TC a = (lane < nw) ? wt[lane] : TC(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const TC y = shfl_up_tc(a, o, 32);
      if (lane >= o) a = a + y;
    }
    TC before = shfl_idx_tc(a, (w > 0 ? w - 1 : 0), 32);
    if (w == 0) before = TC(0);
    ex = before + ex;
  } else {
    __syncthreads();  // keep the CTA's barrier count uniform across group sizes
  }
  return ex;
}

constexpr int kDstMinN = 128;  // smaller N: the direct O(N^2) sum (k_dst1_direct)

template <typename TC>
constexpr int dst_max_threads() { return sizeof(TC) == 4 ? 1024 : 512; }

// in/out pointers per (mat, slot); blockIdx.x = column group, .y = slot, .z = matrix.
template <typename TIn, typename TOut, typename TC>
__global__ void __launch_bounds__(dst_max_threads<TC>()) k_dst1_half(int n, int logL, int cols_per_cta,
                                                                   const DstBatch<TIn, TOut> job,
                                                                   const cplx<TC>* __restrict__ tw,
                                                                   double scale64) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = n + 1, L = N >> 1, Tc = L >> 3;
  const int g = threadIdx.x / Tc, t = threadIdx.x - g * Tc;
  const int slot = blockIdx.y, mat = blockIdx.z;
  const int col = blockIdx.x * cols_per_cta + g;
  // per column: z (L complex, padded: N + N/P scalars), R (L + L/32 scalars);
  // per group 32 scan values
  const int per_col = dst_half_col_scalars<TC>(N);
  TC* colbuf = reinterpret_cast<TC*>(smem_raw) + (int64_t)g * per_col;
  cplx<TC>* z = reinterpret_cast<cplx<TC>*>(colbuf);
  TC* Rb = colbuf + 2 * zpad<TC>(L);
  TC* wt = reinterpret_cast<TC*>(smem_raw) + (int64_t)cols_per_cta * per_col + 32 * g;
  int ncols = job.fixed_cols;
  if (job.ncols_dev) ncols = job.ncols_dev[slot * job.ncols_stride + mat * job.ncols_mat_stride];
  bool live = col < ncols;
  if (job.active_dev && job.require_active && job.active_dev[slot * job.active_stride] == 0) live = false;
  const TIn* x = job.in[mat * job.nslots + slot];
  TOut* y = job.out[mat * job.nslots + slot];
  if (x == nullptr || y == nullptr) live = false;
  // A CTA whose columns are all idle leaves before its first barrier; otherwise
  // idle groups run the barriers on zeros and store nothing.
  if (__syncthreads_count(live ? 1 : 0) == 0) return;
  if (live) {
    x += (int64_t)col * job.ld_in[mat * job.nslots + slot];
    y += (int64_t)col * job.ld_out[mat * job.nslots + slot];
  }
  // scalar u_j / output Y[i] lives in element i/2 (.re for even i, .im for odd)
  auto zs = [&](int i) -> TC& {
    cplx<TC>& c = z[zpad<TC>(i >> 1)];
    return (i & 1) ? c.im : c.re;
  };

  // Pre-processing: u_j and u_{N-j} for j = 1..N/2-1 (x_j = x[j-1]); u_0 = 0,
  // u_{N/2} = 2 x_{N/2}.  The thread's 16 loads are issued before any use.
  // (all 16 loads first, in the input type; the conversions, whose rare
  // branches would otherwise hold back the later loads, follow)
  const TC half = TC(0.5);
  TIn ra[8], rb[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int j = 1 + t + q * Tc;
    ra[q] = TIn(0);
    rb[q] = TIn(0);
    if (live && j < L) {
      ra[q] = x[j - 1];
      rb[q] = x[N - j - 1];
    }
  }
  TC xa[8], xb[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    xa[q] = to_tc<TC>(ra[q]);
    xb[q] = to_tc<TC>(rb[q]);
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int j = 1 + t + q * Tc;
    if (j < L) {
      const TC sj = TC(0) - tw_load(tw, j).im;  // sin(pi j / N)
      const TC a = xa[q] + xb[q], b = xa[q] - xb[q];
      zs(j) = sj * a + half * b;
      zs(N - j) = sj * a - half * b;
    }
  }
  if (t == 0) {
    zs(0) = TC(0);
    const TC xm = live ? to_tc<TC>(x[L - 1]) : TC(0);
    zs(L) = xm + xm;
  }
  __syncthreads();

  // Complex FFT of length L (natural order in, natural order out).
  int Ns = 1, bits = logL;
  for (; bits >= 3; bits -= 3, Ns <<= 3) stockham_stage<TC, 8>(z, L, Ns, N, t, Tc, tw);
  if (bits == 2) stockham_stage<TC, 4>(z, L, Ns, N, t, Tc, tw);
  else if (bits == 1) stockham_stage<TC, 2>(z, L, Ns, N, t, Tc, tw);

  // Unpack (strided k = t + e Tc): R_k, I_k of the real DFT of u.
  TC Rr[8], Ir[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int k = t + e * Tc;
    const cplx<TC> Vk = z[zpad<TC>(k)], Vm = z[zpad<TC>((L - k) & (L - 1))];
    const TC Er = (Vk.re + Vm.re) * half, Ei = (Vk.im - Vm.im) * half;
    const TC Or = (Vk.im + Vm.im) * half, Oi = (Vm.re - Vk.re) * half;  // (Vk - conj Vm) / (2i)
    const cplx<TC> w = tw_load(tw, 2 * k);                                // e^{-2 pi i k / N}
    Rr[e] = Er + (w.re * Or - w.im * Oi);
    Ir[e] = TC(0) - (Ei + (w.re * Oi + w.im * Or));
  }
  __syncthreads();
  // staged outputs: Y(k' - 1) = S_{k'}, in the scalar slots of z
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int k = t + e * Tc;
    if (k > 0) zs(2 * k - 1) = Ir[e];
    Rb[k + (k >> 5)] = (k == 0) ? Rr[e] * half : Rr[e];
  }
  __syncthreads();
  // S_{2k+1} = sum_{m <= k} R'_m over the thread's 8 consecutive k, then the
  // group's exclusive scan of the thread totals.
  TC acc[8];
  TC run = TC(0);
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int k = 8 * t + e;
    run = run + Rb[k + (k >> 5)];
    acc[e] = run;
  }
  const TC before = group_exclusive_scan(run, t, Tc, wt);
#pragma unroll
  for (int e = 0; e < 8; ++e) zs(2 * (8 * t + e)) = before + acc[e];
  __syncthreads();
  if (live) {
    const TC scale = to_tc<TC>(scale64);
    for (int i = t; i < n; i += Tc) y[i] = from_tc<TOut>(scale * zs(i));
  }
}

// Small N (< kDstMinN): one thread per output, the defining sum.
template <typename TIn, typename TOut, typename TC>
__global__ void k_dst1_direct(int n, const DstBatch<TIn, TOut> job, const cplx<TC>* __restrict__ tw,
                              double scale64) {
  const int N = n + 1;
  const int col = blockIdx.x, slot = blockIdx.y, mat = blockIdx.z;
  int ncols = job.fixed_cols;
  if (job.ncols_dev) ncols = job.ncols_dev[slot * job.ncols_stride + mat * job.ncols_mat_stride];
  if (col >= ncols) return;
  if (job.active_dev && job.require_active && job.active_dev[slot * job.active_stride] == 0) return;
  const TIn* x = job.in[mat * job.nslots + slot];
  TOut* y = job.out[mat * job.nslots + slot];
  if (x == nullptr || y == nullptr) return;
  x += (int64_t)col * job.ld_in[mat * job.nslots + slot];
  y += (int64_t)col * job.ld_out[mat * job.nslots + slot];
  const TC scale = to_tc<TC>(scale64);
  for (int k = 1 + threadIdx.x; k <= n; k += blockDim.x) {
    TC s = TC(0);
    for (int j = 1; j <= n; ++j) s = s + to_tc<TC>(x[j - 1]) * (TC(0) - tw_any(tw, j * k, N).im);  // sin(pi j k / N)
    y[k - 1] = from_tc<TOut>(scale * s);
  }
}

// ---------------------------------------------------------------- multi-pass
// For N = n+1 > 8192 the length-N complex FFT of the packed sequence runs as a
// four-step FFT through HBM: N = N1 * N2, j = j1 + N1 j2, k = k2 + N2 k1,
//   Y[k2][j1] = e^{-2 pi i j1 k2 / N} sum_{j2} z[j1 + N1 j2] e^{-2 pi i j2 k2 / N2}  (pass A)
//   Z[k2 + N2 k1] = sum_{j1} Y[k2][j1] e^{-2 pi i j1 k1 / N1}                       (pass B)
// Pass B handles the rows k2 = a and N2 - a together, so that the unpacking
// pairs (k, N - k) of one CTA never leave it.

// In-place radix-2 DIT FFT of length L = 2^logL held in shared memory (already in
// bit-reversed order); twiddle e^{-2 pi i m / L} = tw[2 m N / L] of the length-N table.
template <typename TC>
__device__ inline void blk_fft_bitrev(cplx<TC>* z, int logL, const cplx<TC>* __restrict__ tw, int N) {
  const int L = 1 << logL;
  for (int s = 1; s <= logL; ++s) {
    const int h = 1 << (s - 1);
    const int stride = (N / h);  // e^{-2 pi i pos / (2h)} = e^{-i pi pos / h} = tw[pos * N / h]
    for (int b = threadIdx.x; b < (L >> 1); b += blockDim.x) {
      const int pos = b & (h - 1);
      const int i0 = ((b >> (s - 1)) << s) + pos;
      const int i1 = i0 + h;
      const cplx<TC> w = tw[pos * stride];
      const cplx<TC> a = z[i0], c = z[i1];
      const TC tr = w.re * c.re - w.im * c.im;
      const TC ti = w.re * c.im + w.im * c.re;
      z[i1].re = a.re - tr;
      z[i1].im = a.im - ti;
      z[i0].re = a.re + tr;
      z[i0].im = a.im + ti;
    }
    __syncthreads();
  }
}

// e^{-2 pi i t / N} for 0 <= t < N from the table e^{-i pi k / N}, k < N.
template <typename TC>
__device__ inline cplx<TC> twiddle_full(const cplx<TC>* __restrict__ tw, int64_t t, int N) {
  int64_t k = 2 * t;
  if (k < N) return tw[k];
  const cplx<TC> w = tw[k - N];  // e^{-i pi k/N} = -e^{-i pi (k-N)/N}
  return {-w.re, -w.im};
}

// Packed sequence z_j (see k_dst1_smem) of column x.
template <typename TIn, typename TC>
__device__ inline cplx<TC> packed(const TIn* x, int j, int N) {
  const int half = N >> 1;
  TC re, im;
  if (j < half) {
    const int e = 2 * j, o = 2 * j + 1;
    re = (e == 0) ? (TC)0 : to_tc<TC>(x[e - 1]);
    im = to_tc<TC>(x[o - 1]);
  } else {
    const int e = 2 * N - 2 * j, o = 2 * N - 2 * j - 1;
    re = (e == N) ? (TC)0 : -to_tc<TC>(x[e - 1]);
    im = -to_tc<TC>(x[o - 1]);
  }
  return {re, im};
}

// Pass A: one CTA per (column, group of G consecutive j1).  Shared memory holds G
// sequences of length N2.  Output temp[col][k2 * N1 + j1].
template <typename TIn, typename TOut, typename TC>
__global__ void k_dst1_passA(int n, int logN1, int logN2, int G, int nmats, const DstBatch<TIn, TOut> job,
                             const cplx<TC>* __restrict__ tw, cplx<TC>* __restrict__ temp, int64_t temp_col_stride) {
  extern __shared__ unsigned char smem_raw[];
  cplx<TC>* z = reinterpret_cast<cplx<TC>*>(smem_raw);
  const int N = n + 1, N1 = 1 << logN1, N2 = 1 << logN2;
  const int col = blockIdx.y;
  const int slot = blockIdx.z / nmats, mat = blockIdx.z % nmats;
  int ncols = job.fixed_cols;
  if (job.ncols_dev) ncols = job.ncols_dev[slot * job.ncols_stride + mat * job.ncols_mat_stride];
  if (col >= ncols) return;
  const TIn* x = job.in[mat * job.nslots + slot];
  if (x == nullptr) return;
  x += (int64_t)col * job.ld_in[mat * job.nslots + slot];
  const int j1_0 = blockIdx.x * G;
  // load: element (g, j2) = z[j1_0 + g + N1 j2], stored at bit-reversed j2 of row g
  for (int e = threadIdx.x; e < G * N2; e += blockDim.x) {
    const int g = e % G, j2 = e / G;
    const int j = j1_0 + g + N1 * j2;
    z[g * N2 + (int)(__brev((unsigned)j2) >> (32 - logN2))] = packed<TIn, TC>(x, j, N);
  }
  __syncthreads();
  for (int g = 0; g < G; ++g) blk_fft_bitrev<TC>(z + g * N2, logN2, tw, N);
  // twiddle and store transposed
  cplx<TC>* out = temp + ((int64_t)(blockIdx.z * gridDim.y + col)) * temp_col_stride;
  for (int e = threadIdx.x; e < G * N2; e += blockDim.x) {
    const int g = e % G, k2 = e / G;
    const int j1 = j1_0 + g;
    const cplx<TC> v = z[g * N2 + k2];
    const cplx<TC> w = twiddle_full<TC>(tw, ((int64_t)j1 * k2) % N, N);
    out[(int64_t)k2 * N1 + j1] = {v.re * w.re - v.im * w.im, v.re * w.im + v.im * w.re};
  }
}

// Pass B: one CTA per (column, a in [0, N2/2]); rows a and N2 - a of length N1,
// FFT, then the DST unpacking of every pair (k, N - k) with k in row a.
template <typename TIn, typename TOut, typename TC>
__global__ void k_dst1_passB(int n, int logN1, int logN2, int nmats, const DstBatch<TIn, TOut> job,
                             const cplx<TC>* __restrict__ tw, const cplx<TC>* __restrict__ temp,
                             int64_t temp_col_stride, double scale64) {
  extern __shared__ unsigned char smem_raw[];
  cplx<TC>* z = reinterpret_cast<cplx<TC>*>(smem_raw);  // two rows of N1
  const int N = n + 1, N1 = 1 << logN1, N2 = 1 << logN2;
  const int col = blockIdx.y;
  const int slot = blockIdx.z / nmats, mat = blockIdx.z % nmats;
  int ncols = job.fixed_cols;
  if (job.ncols_dev) ncols = job.ncols_dev[slot * job.ncols_stride + mat * job.ncols_mat_stride];
  if (col >= ncols) return;
  TOut* y = job.out[mat * job.nslots + slot];
  if (y == nullptr || job.in[mat * job.nslots + slot] == nullptr) return;
  y += (int64_t)col * job.ld_out[mat * job.nslots + slot];
  const int a = blockIdx.x;
  const int b = (N2 - a) % N2;  // partner row (a = 0 and a = N2/2 pair with themselves)
  const cplx<TC>* in = temp + ((int64_t)(blockIdx.z * gridDim.y + col)) * temp_col_stride;
  for (int e = threadIdx.x; e < N1; e += blockDim.x) {
    const int p = (int)(__brev((unsigned)e) >> (32 - logN1));
    z[p] = in[(int64_t)a * N1 + e];
    z[N1 + p] = in[(int64_t)b * N1 + e];
  }
  __syncthreads();
  blk_fft_bitrev<TC>(z, logN1, tw, N);
  if (b != a) blk_fft_bitrev<TC>(z + N1, logN1, tw, N);
  // Z[a + N2 k1] = z[k1]; Z[b + N2 k1] = z[N1 + k1] (b == a: the same row).
  const cplx<TC>* zb = (b != a) ? z + N1 : z;
  const TC scale = to_tc<TC>(scale64);
  for (int k1 = threadIdx.x; k1 < N1; k1 += blockDim.x) {
    const int k = a + N2 * k1;
    if (k == 0) continue;
    const int m = N - k;  // lies in row b: m = b + N2 * k1m
    const int k1m = (m - b) / N2;
    const cplx<TC> Zk = z[k1], Zm = zb[k1m];
    const TC Ei = (Zk.im - Zm.im) * (TC)0.5;
    const TC Dr = (Zk.re - Zm.re) * (TC)0.5, Di = (Zk.im + Zm.im) * (TC)0.5;
    const TC Or = Di, Oi = -Dr;
    cplx<TC> w;
    if (k <= N / 2) {
      w = tw[k];
    } else {
      const cplx<TC> w2 = tw[N - k];  // e^{-i pi k/N} = -conj(e^{-i pi (N-k)/N})
      w = {-w2.re, w2.im};
    }
    const TC Yk_im = Ei + (w.re * Oi + w.im * Or);
    y[k - 1] = (TOut)(-(TC)0.5 * Yk_im * scale);
    if (b != a) {
      // partner m = N - k in row b: E_m = conj(E_k), O_m = (Z_m - conj Z_k)/(2i),
      // e^{-i pi m/N} = -conj(e^{-i pi k/N})
      const TC D2r = (Zm.re - Zk.re) * (TC)0.5, D2i = (Zm.im + Zk.im) * (TC)0.5;
      const TC O2r = D2i, O2i = -D2r;
      const cplx<TC> wm = {-w.re, w.im};
      const TC Ym_im = -Ei + (wm.re * O2i + wm.im * O2r);
      y[m - 1] = (TOut)(-(TC)0.5 * Ym_im * scale);
    }
  }
}

static int ilog2(int64_t v) {
  int l = 0;
  while ((int64_t(1) << l) < v) ++l;
  return l;
}

template <typename TC>
void* make_twiddles(int64_t N, cudaStream_t st) {
  void* p = nullptr;
  if (cudaMalloc(&p, sizeof(cplx<TC>) * (size_t)N) != cudaSuccess) return nullptr;
  k_twiddle<TC><<<(unsigned)((N + 255) / 256), 256, 0, st>>>((cplx<TC>*)p, (int)N);
  return p;
}

void* dst_make_twiddles(int64_t N, bool fp64, cudaStream_t st) {
  return fp64 ? make_twiddles<double>(N, st) : make_twiddles<float>(N, st);
}

void* dst_make_twiddles_df(int64_t N, cudaStream_t st) { return make_twiddles<dfloat>(N, st); }

size_t dst_smem_bytes(int64_t n, bool fp64) { return (size_t)(n + 1) * (fp64 ? 16 : 8); }

bool dst_smem_supported(int64_t n, bool fp64) {
  return dst_smem_bytes(n, fp64) <= 200 * 1024 && (n + 1) >= 2;
}

bool dst_supported(int64_t n) { return n >= 1 && n + 1 <= (int64_t(1) << 21); }

size_t dst_temp_bytes(int64_t n, bool fp64) {
  return dst_smem_supported(n, fp64) ? 0 : (size_t)(n + 1) * (fp64 ? 16 : 8);
}

// Shared memory of k_dst1_half: per column dst_half_col_scalars values, plus
// 32 scan values per column group.
template <typename TC>
static size_t dst_half_smem(int N, int cols_per_cta) {
  return sizeof(TC) * ((size_t)cols_per_cta * dst_half_col_scalars<TC>(N) + 32 * (size_t)cols_per_cta);
}

template <typename TIn, typename TOut, typename TC>
cudaError_t dst1_launch(int64_t n, const DstBatch<TIn, TOut>& job, int max_cols, int nslots, int nmats,
                        const void* tw, cudaStream_t st, void* temp, size_t temp_bytes, int cta_threads) {
  const int N = (int)(n + 1);
  const double scale64 = sqrt(2.0 / (double)N);  // the orthonormal scaling, once on the host
  if (!dst_smem_supported(n, sizeof(TC) == 8)) {
    // Multi-pass: N = N1 * N2 with N1 >= N2, both <= 2048 (N <= 2^22).
    const int logN = ilog2(N);
    const int logN1 = (logN + 1) / 2, logN2 = logN / 2;
    if (logN1 > 11) return cudaErrorInvalidValue;
    const int N1 = 1 << logN1, N2 = 1 << logN2;
    const size_t per_col = (size_t)N * sizeof(cplx<TC>);
    const size_t need = per_col * (size_t)max_cols * nslots * nmats;
    if (!temp || temp_bytes < need) return cudaErrorInvalidValue;
    // j1 values per pass-A CTA (coalesced row segments), bounded by 128 KB of shared memory
    int G = 8;
    while (G > 1 && (size_t)G * N2 * sizeof(cplx<TC>) > 128 * 1024) G >>= 1;
    if (max_cols <= 0 || nslots <= 0) return cudaSuccess;
    dim3 gA(N1 / G, max_cols, nslots * nmats);
    const size_t smemA = (size_t)G * N2 * sizeof(cplx<TC>);
    k_dst1_passA<TIn, TOut, TC><<<gA, 256, smemA, st>>>((int)n, logN1, logN2, G, nmats, job,
                                                         (const cplx<TC>*)tw, (cplx<TC>*)temp, (int64_t)N);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dim3 gB(N2 / 2 + 1, max_cols, nslots * nmats);
    const size_t smemB = 2 * (size_t)N1 * sizeof(cplx<TC>);
    k_dst1_passB<TIn, TOut, TC><<<gB, 256, smemB, st>>>((int)n, logN1, logN2, nmats, job,
                                                         (const cplx<TC>*)tw, (const cplx<TC>*)temp, (int64_t)N,
                                                         scale64);
    return cudaGetLastError();
  }
  if (max_cols <= 0 || nslots <= 0) return cudaSuccess;
  if (N < kDstMinN) {
    dim3 grid(max_cols, nslots, nmats);
    k_dst1_direct<TIn, TOut, TC><<<grid, 64, 0, st>>>((int)n, job, (const cplx<TC>*)tw, scale64);
    return cudaGetLastError();
  }
  const int L = N / 2, logL = ilog2(L);
  const int Tc = L / 8;
  // columns per CTA: the requested CTA size over the Tc threads of one column,
  // within the kernel's thread bound and the 200 KB of shared memory
  int want = cta_threads > 0 ? cta_threads : 256;
  if (want > dst_max_threads<TC>()) want = dst_max_threads<TC>();
  int cols_per_cta = Tc >= want ? 1 : want / Tc;
  while (cols_per_cta > 1 && dst_half_smem<TC>(N, cols_per_cta) > 200 * 1024) cols_per_cta >>= 1;
  const int threads = Tc * cols_per_cta;
  const size_t smem = dst_half_smem<TC>(N, cols_per_cta);
  dim3 grid((max_cols + cols_per_cta - 1) / cols_per_cta, nslots, nmats);
  k_dst1_half<TIn, TOut, TC><<<grid, threads, smem, st>>>((int)n, logL, cols_per_cta, job, (const cplx<TC>*)tw,
                                                           scale64);
  return cudaGetLastError();
}

cudaError_t dst_configure() {
  const int bytes = 200 * 1024;
  cudaError_t e = cudaSuccess;
#define LRP_CFG(K)                                                                              \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  LRP_CFG((k_dst1_passA<double, double, double>))
  LRP_CFG((k_dst1_passA<double, float, float>))
  LRP_CFG((k_dst1_passA<float, double, float>))
  LRP_CFG((k_dst1_passA<float, float, float>))
  LRP_CFG((k_dst1_passB<double, double, double>))
  LRP_CFG((k_dst1_passB<double, float, float>))
  LRP_CFG((k_dst1_passB<float, double, float>))
  LRP_CFG((k_dst1_passB<float, float, float>))
  LRP_CFG((k_dst1_half<double, double, double>))
  LRP_CFG((k_dst1_half<double, float, float>))
  LRP_CFG((k_dst1_half<float, double, float>))
  LRP_CFG((k_dst1_half<float, float, float>))
  LRP_CFG((k_dst1_half<double, double, dfloat>))
  LRP_CFG((k_dst1_passA<double, double, dfloat>))
  LRP_CFG((k_dst1_passB<double, double, dfloat>))
#undef LRP_CFG
  return e;
}

template cudaError_t dst1_launch<double, double, double>(int64_t, const DstBatch<double, double>&, int, int, int,
                                                         const void*, cudaStream_t, void*, size_t, int);
template cudaError_t dst1_launch<double, float, float>(int64_t, const DstBatch<double, float>&, int, int, int,
                                                       const void*, cudaStream_t, void*, size_t, int);
template cudaError_t dst1_launch<float, double, float>(int64_t, const DstBatch<float, double>&, int, int, int,
                                                       const void*, cudaStream_t, void*, size_t, int);
template cudaError_t dst1_launch<float, float, float>(int64_t, const DstBatch<float, float>&, int, int, int,
                                                     const void*, cudaStream_t, void*, size_t, int);
template cudaError_t dst1_launch<double, double, dfloat>(int64_t, const DstBatch<double, double>&, int, int, int,
                                                         const void*, cudaStream_t, void*, size_t, int);

}  // namespace lrp
