// Cross-DEIM on a matrix given by its entries: the test matrices of Sec. 4.1,
//   H(i, j) = 1 / (1 + i + j)                       (Hilbert, indices from 0)
//   K(i, j) = (|x_i + y_j| / 2)^5, x_i = -1 + 2 i / (n - 1), y_j likewise,
// both n x n.  Algorithm Cross-DEIM needs only sampled columns C = G(:, J) and
// rows R = G(I, :) (Algorithm scross), evaluated here from the formulas, so the
// matrix is never formed.  The initial guesses U_0, V_0 are the caller's and
// the result is the iterate's factors themselves (no transform), both moved by
// a batched column copy.
#include <cuda_runtime.h>

#include "common.cuh"
#include "matrix.cuh"

namespace lrp {

namespace {
constexpr int MR = 128;  // rows per CTA
constexpr int MC = 64;   // sampled indices per CTA
constexpr int MT = 256;
}  // namespace

__device__ __forceinline__ double matrix_entry(int kind, int n, int i, int j) {
  if (kind == LRP_MAT_HILBERT) return 1.0 / (1.0 + (double)i + (double)j);
  const double x = -1.0 + (2.0 * (double)i) / (double)(n - 1);
  const double y = -1.0 + (2.0 * (double)j) / (double)(n - 1);
  const double t = fabs(x + y) / 2.0;
  const double t2 = t * t;
  return t2 * t2 * t;
}

// Side 0: A(i, q) = G(i, J_q) (q < |J|); side 1: A(j, p) = G(I_p, j) (p < |I|).
__global__ void __launch_bounds__(MT) k_cross_matrix(TallGeom g, const SolveState* __restrict__ st_all, int kind,
                                                     Strided<double> A, Strided<const int32_t> idx) {
  const int slot = slot_of(g, blockIdx.z >> 1), side = blockIdx.z & 1;
  if (slot < 0) return;
  const SolveState& st = st_all[slot];
  if (!st.active) return;
  const int m = st.cnt[1 - side];
  const int r0 = blockIdx.x * MR, c0 = blockIdx.y * MC;
  if (c0 >= m || r0 >= g.n) return;
  __shared__ int sel[MC];
  const int32_t* ix = idx.at(slot, 1 - side);
  for (int t = threadIdx.x; t < MC; t += MT) sel[t] = (c0 + t < m) ? ix[c0 + t] : -1;
  __syncthreads();
  double* out = A.at(slot, side);
  const int cend = min(MC, m - c0);
  for (int e = threadIdx.x; e < MR * cend; e += MT) {
    const int i = r0 + e % MR, c = e / MR;
    if (i >= g.n) continue;
    const int s = sel[c];
    out[(int64_t)(c0 + c) * g.ld + i] = side == 0 ? matrix_entry(kind, g.n, i, s) : matrix_entry(kind, g.n, s, i);
  }
}

// out[mat][slot](:, c) = in[mat][slot](:, c) for c < ncols(slot, mat); null
// pointers are skipped.
__global__ void k_copy_cols(DstBatch<double, double> job, int n) {
  const int slot = blockIdx.z >> 1, mat = blockIdx.z & 1;
  const int c = blockIdx.y;
  const int ncols = job.ncols_dev ? job.ncols_dev[(int64_t)slot * job.ncols_stride + mat * job.ncols_mat_stride]
                                  : job.fixed_cols;
  if (c >= ncols) return;
  const int e = mat * job.nslots + slot;
  const double* src = job.in[e];
  double* dst = job.out[e];
  if (!src || !dst) return;
  const int64_t li = job.ld_in[e], lo = job.ld_out[e];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    dst[(int64_t)c * lo + i] = src[(int64_t)c * li + i];
}

cudaError_t launch_cross_matrix(const TallGeom& g, const SolveState* st, int kind, Strided<double> A,
                                Strided<const int32_t> idx, cudaStream_t s) {
  const dim3 grid((g.n + MR - 1) / MR, (g.M + MC - 1) / MC, g.nslots * 2);
  k_cross_matrix<<<grid, MT, 0, s>>>(g, st, kind, A, idx);
  return cudaGetLastError();
}

cudaError_t launch_copy_cols(const DstBatch<double, double>& job, int n, int max_cols, cudaStream_t s) {
  if (max_cols < 1 || job.nslots < 1) return cudaSuccess;
  const int bx = (n + 255) / 256 < 64 ? (n + 255) / 256 : 64;
  k_copy_cols<<<dim3(bx, max_cols, job.nslots * 2), 256, 0, s>>>(job, n);
  return cudaGetLastError();
}

}  // namespace lrp
