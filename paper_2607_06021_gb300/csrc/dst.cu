// Orthonormal DST-I of columns (paper Sec. 3: Z_{ik} = sqrt(2/(n+1)) sin(i k pi/(n+1)),
// Z symmetric orthogonal, applied to n x r factors "in batches along dimensions
// independently without any global transpose", Sec. 1 / Sec. 3.2).
//
// Method (standard real-FFT packing, written from the DFT definition): with
// N = n+1 a power of two, the odd extension y = [0, x_1..x_n, 0, -x_n..-x_1]
// of length 2N has DFT Y_k = -2i S_k, S_k = sum_j x_j sin(pi j k / N).  Packing
// z_j = y_{2j} + i y_{2j+1} (j < N) gives one complex FFT of length N; the
// even/odd split E_k = (Z_k + conj Z_{N-k})/2, O_k = (Z_k - conj Z_{N-k})/(2i)
// recovers Y_k = E_k + e^{-i pi k/N} O_k, so S_k = -Im(Y_k)/2 and
// (Z x)_k = sqrt(2/N) S_k.
//
// One CTA per column; the length-N complex sequence lives in shared memory
// (N * 2 * sizeof(T) bytes: 128 KB at N = 8192 in FP64).  Loads of the
// column-major input are contiguous; the twiddle table e^{-i pi k/N} (length N,
// FP64 or FP32) is built once per size and stays L2-resident.
#include <cuda_runtime.h>
#include <math.h>

#include <type_traits>

#include "common.cuh"
#include "dfloat.cuh"
#include "dst.cuh"

namespace lrp {

template <typename T>
struct cplx {
  T re, im;
};

template <typename TC>
__global__ void k_twiddle(cplx<TC>* tw, int N) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  double s, c;
  sincospi((double)k / (double)N, &s, &c);  // e^{-i pi k / N}
  tw[k].re = (TC)c;
  tw[k].im = (TC)(-s);
}

__device__ __forceinline__ int bitrev(int v, int bits) { return (int)(__brev((unsigned)v) >> (32 - bits)); }

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

// in_ptrs/out_ptrs: one column-0 pointer per slot; ncols_dev (or fixed_cols) gives
// the number of columns of each slot; blockIdx.x = column, blockIdx.y = slot,
// blockIdx.z selects one of two matrices of the slot (e.g. U and V).
template <typename TIn, typename TOut, typename TC>
__global__ void k_dst1_smem(int n, int logN, const DstBatch<TIn, TOut> job,
                            const cplx<TC>* __restrict__ tw) {
  extern __shared__ unsigned char smem_raw[];
  cplx<TC>* z = reinterpret_cast<cplx<TC>*>(smem_raw);
  const int N = n + 1;
  const int col = blockIdx.x;
  const int slot = blockIdx.y;
  const int mat = blockIdx.z;
  int ncols = job.fixed_cols;
  if (job.ncols_dev) ncols = job.ncols_dev[slot * job.ncols_stride + mat * job.ncols_mat_stride];
  if (job.active_dev && job.active_dev[slot * job.active_stride] == 0 && job.require_active) return;
  if (col >= ncols) return;
  const TIn* x = job.in[mat * job.nslots + slot] + (int64_t)col * job.ld_in[mat * job.nslots + slot];
  TOut* y = job.out[mat * job.nslots + slot] + (int64_t)col * job.ld_out[mat * job.nslots + slot];
  if (x == nullptr || y == nullptr) return;

  // Pack: z_j = y_{2j} + i y_{2j+1}; y_0 = y_N = 0, y_i = x_i (1 <= i <= n),
  // y_{2N-i} = -x_i.  x is 1-based in the formulas, x[i-1] in memory.
  const int half = N >> 1;
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    TC re, im;
    if (j < half) {
      const int e = 2 * j, o = 2 * j + 1;
      re = (e == 0) ? (TC)0 : (TC)x[e - 1];
      im = (TC)x[o - 1];
    } else {
      const int e = 2 * N - 2 * j, o = 2 * N - 2 * j - 1;  // e in [2, N], o in [1, N-1]
      re = (e == N) ? (TC)0 : -(TC)x[e - 1];
      im = -(TC)x[o - 1];
    }
    const int p = bitrev(j, logN);
    z[p].re = re;
    z[p].im = im;
  }
  __syncthreads();

  // Radix-2 decimation-in-time butterflies; twiddle e^{-2 pi i pos/(2h)} = tw[pos * N / h].
  int s = 1;
  if constexpr (std::is_same<TC, dfloat>::value) {
    // Double-float steps are explicitly rounded (nothing is contracted), so the
    // stages can go in pairs with the same operations: the elements i, i+h,
    // i+2h, i+3h of a 4h block take both stages' butterflies in registers,
    // with half the barriers and shared-memory round trips.
    for (; s + 1 <= logN; s += 2) {
      const int h = 1 << (s - 1);
      const int st0 = N >> (s - 1), st1 = N >> s;
      for (int b = threadIdx.x; b < (N >> 2); b += blockDim.x) {
        const int pos = b & (h - 1);
        const int i = ((b >> (s - 1)) << (s + 1)) + pos;
        cplx<TC> a0 = z[i], a1 = z[i + h], a2 = z[i + 2 * h], a3 = z[i + 3 * h];
        const cplx<TC> w0 = tw[pos * st0];
        butterfly(a0, a1, w0);
        butterfly(a2, a3, w0);
        const cplx<TC> w1 = tw[pos * st1], w2 = tw[(pos + h) * st1];
        butterfly(a0, a2, w1);
        butterfly(a1, a3, w2);
        z[i] = a0;
        z[i + h] = a1;
        z[i + 2 * h] = a2;
        z[i + 3 * h] = a3;
      }
      __syncthreads();
    }
  }
  for (; s <= logN; ++s) {
    const int h = 1 << (s - 1);
    const int stride = N >> (s - 1);  // N / h
    for (int b = threadIdx.x; b < half; b += blockDim.x) {
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

  // Unpack pairs (k, N-k), k = 1..N/2.
  const TC scale = (TC)sqrt(2.0 / (double)N);
  for (int k = 1 + threadIdx.x; k <= half; k += blockDim.x) {
    const int m = N - k;
    const cplx<TC> Zk = z[k], Zm = z[m];
    // E_k = (Zk + conj Zm)/2 ; O_k = (Zk - conj Zm)/(2i)
    const TC Er = (Zk.re + Zm.re) * (TC)0.5, Ei = (Zk.im - Zm.im) * (TC)0.5;
    const TC Dr = (Zk.re - Zm.re) * (TC)0.5, Di = (Zk.im + Zm.im) * (TC)0.5;  // (Zk - conj Zm)/2
    const TC Or = Di, Oi = -Dr;                                               // divide by i
    const cplx<TC> w = tw[k];
    // Y_k = E_k + w O_k; S_k = -Im(Y_k)/2
    const TC Yk_im = Ei + (w.re * Oi + w.im * Or);
    y[k - 1] = (TOut)(-(TC)0.5 * Yk_im * scale);
    if (m != k) {
      // E_{N-k} = conj(E_k); O_{N-k} = (Zm - conj Zk)/(2i) = conj(O_k) * (-1)... computed directly
      const TC Emi = -Ei;
      const TC D2r = (Zm.re - Zk.re) * (TC)0.5, D2i = (Zm.im + Zk.im) * (TC)0.5;
      const TC O2r = D2i, O2i = -D2r;
      const cplx<TC> w2 = {-w.re, w.im};  // e^{-i pi (N-k)/N} = -conj(e^{-i pi k/N})
      const TC Ym_im = Emi + (w2.re * O2i + w2.im * O2r);
      y[m - 1] = (TOut)(-(TC)0.5 * Ym_im * scale);
    }
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
    re = (e == 0) ? (TC)0 : (TC)x[e - 1];
    im = (TC)x[o - 1];
  } else {
    const int e = 2 * N - 2 * j, o = 2 * N - 2 * j - 1;
    re = (e == N) ? (TC)0 : -(TC)x[e - 1];
    im = -(TC)x[o - 1];
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
                             int64_t temp_col_stride) {
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
  const TC scale = (TC)sqrt(2.0 / (double)N);
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

template <typename TIn, typename TOut, typename TC>
cudaError_t dst1_launch(int64_t n, const DstBatch<TIn, TOut>& job, int max_cols, int nslots, int nmats,
                        const void* tw, cudaStream_t st, void* temp, size_t temp_bytes) {
  const int N = (int)(n + 1);
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
                                                         (const cplx<TC>*)tw, (const cplx<TC>*)temp, (int64_t)N);
    return cudaGetLastError();
  }
  const int logN = ilog2(N);
  const size_t smem = (size_t)N * sizeof(cplx<TC>);
  auto kern = k_dst1_smem<TIn, TOut, TC>;
  int threads = N >= 2048 ? 512 : (N >= 512 ? 256 : 128);
  dim3 grid(max_cols, nslots, nmats);
  if (max_cols <= 0 || nslots <= 0) return cudaSuccess;
  kern<<<grid, threads, smem, st>>>((int)n, logN, job, (const cplx<TC>*)tw);
  return cudaGetLastError();
}

cudaError_t dst_configure() {
  const int bytes = 200 * 1024;
  cudaError_t e = cudaFuncSetAttribute(k_dst1_smem<double, double, double>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_dst1_smem<double, float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_dst1_smem<float, double, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_dst1_smem<float, float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
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
  LRP_CFG((k_dst1_smem<double, double, dfloat>))
  LRP_CFG((k_dst1_passA<double, double, dfloat>))
  LRP_CFG((k_dst1_passB<double, double, dfloat>))
#undef LRP_CFG
  return e;
}

template cudaError_t dst1_launch<double, double, double>(int64_t, const DstBatch<double, double>&, int, int, int,
                                                         const void*, cudaStream_t, void*, size_t);
template cudaError_t dst1_launch<double, float, float>(int64_t, const DstBatch<double, float>&, int, int, int,
                                                       const void*, cudaStream_t, void*, size_t);
template cudaError_t dst1_launch<float, double, float>(int64_t, const DstBatch<float, double>&, int, int, int,
                                                       const void*, cudaStream_t, void*, size_t);
template cudaError_t dst1_launch<float, float, float>(int64_t, const DstBatch<float, float>&, int, int, int,
                                                     const void*, cudaStream_t, void*, size_t);
template cudaError_t dst1_launch<double, double, dfloat>(int64_t, const DstBatch<double, double>&, int, int, int,
                                                         const void*, cudaStream_t, void*, size_t);

}  // namespace lrp
