// Compact copy of a batch's results: for each problem of the plan's most recent
// solve, the first rank columns of U and V and the first rank singular values,
// back to back in one device buffer, so that a host reads the results with
// one copy of their actual size instead of every problem's full capacity.
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "common.cuh"
#include "core.cuh"
#include "guard.cuh"
#include "solver.cuh"

namespace lrp {

// Offsets (in doubles) of each problem's block [U (n r) | S (r) | V (n r)] and
// their total in off[count], starting from *base_in (0 if null); one CTA,
// prefix sum over the problems.
__global__ void k_pack_offsets(const SolveState* __restrict__ st, int count, int64_t n, int64_t* __restrict__ off,
                               const int64_t* __restrict__ base_in) {
  __shared__ int64_t part[1024];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int64_t base = base_in ? *base_in : 0;
  __syncthreads();  // every thread has read the base before off[0] is written
  const int per = (count + nt - 1) / nt;
  const int b0 = tid * per, b1 = min(count, b0 + per);
  int64_t s = 0;
  for (int i = b0; i < b1; ++i) {
    const int r = st[i].valid ? st[i].r_out : 0;
    s += (2 * n + 1) * (int64_t)r;
  }
  part[tid] = s;
  __syncthreads();
  if (tid == 0) {
    int64_t acc = base;
    for (int t = 0; t < nt; ++t) {
      const int64_t v = part[t];
      part[t] = acc;
      acc += v;
    }
    off[count] = acc;
  }
  __syncthreads();
  int64_t o = part[tid];
  for (int i = b0; i < b1; ++i) {
    off[i] = o;
    const int r = st[i].valid ? st[i].r_out : 0;
    o += (2 * n + 1) * (int64_t)r;
  }
}

// Copies problem blockIdx.y's columns (rows split over blockIdx.x); blocks that
// would end beyond capacity are skipped (the caller sees off[count] > capacity).
__global__ void k_pack_copy(const SolveState* __restrict__ st, const ProblemDev* __restrict__ prob, int64_t n,
                            const int64_t* __restrict__ off, double* __restrict__ out, int64_t capacity) {
  const int i = blockIdx.y;
  if (!st[i].valid) return;
  const int r = st[i].r_out;
  const int64_t base = off[i];
  if (r < 1 || base + (2 * n + 1) * (int64_t)r > capacity) return;
  const ProblemDev& p = prob[i];
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double* U = out + base;
  double* S = U + n * (int64_t)r;
  double* V = S + r;
  if (row < n) {
    for (int t = 0; t < r; ++t) {
      U[(int64_t)t * n + row] = p.U[(int64_t)t * p.ldu + row];
      V[(int64_t)t * n + row] = p.V[(int64_t)t * p.ldv + row];
    }
  }
  if (blockIdx.x == 0)
    for (int t = threadIdx.x; t < r; t += blockDim.x) S[t] = p.S[t];
}

}  // namespace lrp

using namespace lrp;

extern "C" lrp_status lrp_plan_pack(lrp_plan_t p, double* d_packed, int64_t capacity, int64_t* d_offsets,
                                    void* stream) {
  if (!p || !d_offsets || (capacity > 0 && !d_packed) || capacity < 0)
    return set_error(LRP_EINVAL, "bad lrp_plan_pack arguments");
  std::lock_guard<std::mutex> lock(p->mu);
  const int count = p->last_count;
  if (count < 1) return set_error(LRP_EINVAL, "the plan has not solved a batch yet");
  cudaStream_t s = (cudaStream_t)stream;
  k_pack_offsets<<<1, 1024, 0, s>>>(p->st, count, p->n, d_offsets, nullptr);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    const dim3 grid((unsigned)((p->n + 255) / 256), (unsigned)count);
    k_pack_copy<<<grid, 256, 0, s>>>(p->st, p->prob_dev, p->n, d_offsets, d_packed, capacity);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return set_error(LRP_ECUDA, std::string("lrp_plan_pack: ") + cudaGetErrorString(e));
  p->stats.launches[LRP_K_OTHER] += 2;
  return LRP_OK;
}
