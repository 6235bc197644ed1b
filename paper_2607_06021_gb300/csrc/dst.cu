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

#include "common.cuh"
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
  for (int s = 1; s <= logN; ++s) {
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

size_t dst_smem_bytes(int64_t n, bool fp64) { return (size_t)(n + 1) * (fp64 ? 16 : 8); }

bool dst_smem_supported(int64_t n, bool fp64) {
  return dst_smem_bytes(n, fp64) <= 200 * 1024 && (n + 1) >= 2;
}

template <typename TIn, typename TOut, typename TC>
cudaError_t dst1_launch(int64_t n, const DstBatch<TIn, TOut>& job, int max_cols, int nslots, int nmats,
                        const void* tw, cudaStream_t st) {
  const int N = (int)(n + 1);
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
  return e;
}

template cudaError_t dst1_launch<double, double, double>(int64_t, const DstBatch<double, double>&, int, int, int,
                                                         const void*, cudaStream_t);
template cudaError_t dst1_launch<double, float, float>(int64_t, const DstBatch<double, float>&, int, int, int,
                                                       const void*, cudaStream_t);
template cudaError_t dst1_launch<float, double, float>(int64_t, const DstBatch<float, double>&, int, int, int,
                                                       const void*, cudaStream_t);
template cudaError_t dst1_launch<float, float, float>(int64_t, const DstBatch<float, float>&, int, int, int,
                                                     const void*, cudaStream_t);

}  // namespace lrp
