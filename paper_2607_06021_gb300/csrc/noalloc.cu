// lrp_dst1_noalloc: the orthonormal DST-I of lrp_dst1 without any device
// allocation.
//
// Some callers cannot allocate device memory when they call in: a host
// callback or plugin that runs while another framework owns the device memory
// pool, code that runs under a strict memory budget where every byte has been
// handed out up front, or a caller that must not trigger the implicit
// synchronisation cudaMalloc/cudaFree may cause.  lrp_dst1 keeps a small cache of
// device buffers (twiddle table, job descriptors) that it allocates on first use
// for each size; this variant puts that scratch in a fixed array that is part of
// the library image instead, so nothing is allocated at call time.
//
// The array is file-scope device memory of kNoallocScratchBytes (128 KiB + 256 B)
// on every device that loads the library, held until the process exits.  It
// holds the twiddle table e^{-i pi k/N} (N = n+1 <= 8192 complex doubles) and the
// job descriptor of the call.  Every call rewrites the parts it uses, and every
// call shares the one array: two calls whose work overlaps on the GPU (for
// example on two streams without ordering between them) race on it.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <mutex>
#include <string>

#include "common.cuh"
#include "dst.cuh"
#include "guard.cuh"

namespace lrp {
lrp_status set_error(lrp_status s, const std::string& msg);
}

using namespace lrp;

namespace {

constexpr int kNoallocMaxN = 8192;  // largest n+1 served (the shared-memory DST limit in FP64)
constexpr size_t kNoallocTwiddleBytes = (size_t)kNoallocMaxN * 2 * sizeof(double);
constexpr size_t kNoallocJobBytes = 256;  // 2 pointers + 2 leading dimensions, padded
constexpr size_t kNoallocScratchBytes = kNoallocTwiddleBytes + kNoallocJobBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// Device address of g_noalloc_scratch, fetched once per device.
struct ScratchAddr {
  std::mutex mu;
  void* ptr[64] = {};
};
ScratchAddr g_addr;

// Twiddles e^{-i pi k / N}, k < N, as (re, im) double pairs, plus the job
// descriptor (input pointer, output pointer, ldx, ldy) for one DST call.
__global__ void k_noalloc_prepare(double* tw, int N, const double* x, double* y, int64_t ldx, int64_t ldy,
                                  void** job) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < N) {
    double s, c;
    sincospi((double)k / (double)N, &s, &c);
    tw[2 * k] = c;
    tw[2 * k + 1] = -s;
  }
  if (k == 0) {
    job[0] = const_cast<double*>(x);
    job[1] = y;
    reinterpret_cast<int64_t*>(job)[2] = ldx;
    reinterpret_cast<int64_t*>(job)[3] = ldy;
  }
}

}  // namespace

extern "C" lrp_status lrp_dst1_noalloc(int64_t n, int32_t ncols, const double* d_X, int64_t ldx, double* d_Y,
                                       int64_t ldy, void* stream) {
  if (n < 1 || ((n + 1) & n) != 0) return set_error(LRP_EINVAL, "n+1 must be a power of two >= 2");
  if (n + 1 > kNoallocMaxN)
    return set_error(LRP_EINVAL, "lrp_dst1_noalloc serves n+1 <= 8192 (its fixed scratch holds one twiddle table "
                                 "of that length); use lrp_dst1 for larger n");
  if (ncols < 0 || !d_X || !d_Y || ldx < n || ldy < n) return set_error(LRP_EINVAL, "bad DST arguments");
  if (ncols == 0) return LRP_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return set_error(LRP_ECUDA, "no CUDA device");
  void* base = nullptr;
  {
    // First call on a device: look up the array's device address with that
    // device current (host code may not use the symbol itself as a pointer).
    std::lock_guard<std::mutex> lock(g_addr.mu);
    if (!g_addr.ptr[dev]) {
      SetupGuard guard;
      void* addr = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
      if (e != cudaSuccess)
        return set_error(LRP_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      // The DST kernel needs more than the default dynamic shared memory.  The
      // address is cached only once this has succeeded too, so a failed set-up
      // is retried in full by the next call.
      e = dst_configure();
      if (e != cudaSuccess) return set_error(LRP_ECUDA, std::string("kernel configuration: ") + cudaGetErrorString(e));
      g_addr.ptr[dev] = addr;
    }
    base = g_addr.ptr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  double* tw = reinterpret_cast<double*>(base);
  void** job = reinterpret_cast<void**>(static_cast<unsigned char*>(base) + kNoallocTwiddleBytes);
  const int N = (int)(n + 1);
  k_noalloc_prepare<<<(N + 255) / 256, 256, 0, s>>>(tw, N, d_X, d_Y, ldx, ldy, job);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(LRP_ECUDA, std::string("k_noalloc_prepare: ") + cudaGetErrorString(e));
  DstBatch<double, double> b;
  b.in = reinterpret_cast<const double* const*>(job + 0);
  b.out = reinterpret_cast<double* const*>(job + 1);
  b.ld_in = reinterpret_cast<const int64_t*>(job + 2);
  b.ld_out = reinterpret_cast<const int64_t*>(job + 3);
  b.nslots = 1;
  b.fixed_cols = ncols;
  b.ncols_dev = nullptr;
  b.ncols_stride = 0;
  b.ncols_mat_stride = 0;
  b.active_dev = nullptr;
  b.active_stride = 0;
  b.require_active = 0;
  e = dst1_launch<double, double, double>(n, b, ncols, 1, 1, tw, s);
  if (e != cudaSuccess) return set_error(LRP_ECUDA, std::string("dst1 launch: ") + cudaGetErrorString(e));
  return LRP_OK;
}
