// QDEIM row selection (Sec. 2.2.1, Algorithm IS): the first c pivots of the
// column-pivoted QR of U^T, for an n x c factor U with orthonormal columns.
//
// Pivoted QR of U^T picks, at step j, the column of U^T (row of U) whose part
// orthogonal to the rows picked so far is longest.  Here that is computed
// row-wise: residual norms ||r_i||^2 = ||U(i,:)||^2 - sum_{l<j} (U(i,:) q_l)^2 are
// kept for every row, the pivot p_j is the row of largest residual norm (ties
// to the lower index, as for the leverage selection), and
// q_j = (U(p_j,:) - sum_{l<j} (U(p_j,:) q_l) q_l) / ||.|| extends the orthonormal
// basis of the picked rows.  Each step is two launches over all problems:
//   k_qdeim_pivot   one CTA per (problem, side): reduce the per-chunk best rows,
//                   form q_j (modified Gram-Schmidt, applied twice), record p_j;
//   k_qdeim_update  one CTA per 1024-row chunk: downdate the residual norms by
//                   (U(i,:) q_j)^2 and publish the chunk's best row.
// k_qdeim_emit hands the pivots to the index-set merge in pivot order.
#include <cuda_runtime.h>

#include "common.cuh"
#include "tall.cuh"

namespace lrp {

namespace {
constexpr int QT = 256;  // threads per CTA

// (score desc, row asc) maximum over a block; returns the winner in all threads.
__device__ void block_argmax(double& s, int& r, double* ss, int* rr) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    const double s2 = __shfl_xor_sync(0xffffffffu, s, o);
    const int r2 = __shfl_xor_sync(0xffffffffu, r, o);
    if (s2 > s || (s2 == s && r2 < r)) {
      s = s2;
      r = r2;
    }
  }
  if (lane == 0) {
    ss[wid] = s;
    rr[wid] = r;
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    s = lane < nw ? ss[lane] : -2.0;
    r = lane < nw ? rr[lane] : 0x7fffffff;
    for (int o = 16; o > 0; o >>= 1) {
      const double s2 = __shfl_xor_sync(0xffffffffu, s, o);
      const int r2 = __shfl_xor_sync(0xffffffffu, r, o);
      if (s2 > s || (s2 == s && r2 < r)) {
        s = s2;
        r = r2;
      }
    }
    if (lane == 0) {
      ss[0] = s;
      rr[0] = r;
    }
  }
  __syncthreads();
  s = ss[0];
  r = rr[0];
  __syncthreads();
}
}  // namespace

// Residual norms ||U(i,:)||^2 of the chunk's rows and the chunk's best row.
template <typename T>
__global__ void __launch_bounds__(QT) k_qdeim_init(TallGeom g, const SolveState* __restrict__ st_all,
                                                   Strided<const T> us, int sel, QdeimBufs q) {
  const int slot = slot_of(g, blockIdx.y >> 1), side = blockIdx.y & 1;
  if (slot < 0) return;
  const SolveState& st = st_all[slot];
  if (!st.active) return;
  const int c = dim_of(st, side, sel);
  const int ss_i = slot * 2 + side;
  const T* U = us.at(slot, side);
  double* qn = q.qn + (int64_t)ss_i * g.ld;
  const int rbeg = blockIdx.x * q.chunk_rows, rend = min(g.n, rbeg + q.chunk_rows);
  double best = -1.0;
  int brow = 0x7fffffff;
  for (int i = rbeg + threadIdx.x; i < rend; i += QT) {
    double s = 0.0;
    for (int k = 0; k < c; ++k) {
      const double v = (double)U[(int64_t)k * g.ld + i];
      s = fma(v, v, s);
    }
    qn[i] = s;
    if (s > best || (s == best && i < brow)) {
      best = s;
      brow = i;
    }
  }
  __shared__ double ss[QT / 32];
  __shared__ int rr[QT / 32];
  block_argmax(best, brow, ss, rr);
  if (threadIdx.x == 0) {
    const int64_t o = ((int64_t)ss_i * 2 + 0) * q.nchunk + blockIdx.x;
    q.cs[o] = best;
    q.ci[o] = brow;
  }
}

// Pivot j: the best row over all chunks and the next basis vector q_j.
template <typename T>
__global__ void __launch_bounds__(QT) k_qdeim_pivot(TallGeom g, const SolveState* __restrict__ st_all,
                                                    Strided<const T> us, int sel, QdeimBufs q, int j) {
  const int slot = slot_of(g, blockIdx.x >> 1), side = blockIdx.x & 1;
  if (slot < 0) return;
  const SolveState& st = st_all[slot];
  if (!st.active) return;
  const int c = dim_of(st, side, sel);
  if (j >= c) return;
  const int ss_i = slot * 2 + side;
  const int M = g.M;
  int32_t* piv = q.piv + (int64_t)ss_i * M;
  double best = -1.0;
  int brow = 0x7fffffff;
  const int64_t cb = ((int64_t)ss_i * 2 + (j & 1)) * q.nchunk;
  for (int t = threadIdx.x; t < q.nchunk; t += QT) {
    const double s = q.cs[cb + t];
    const int r = q.ci[cb + t];
    if (s > best || (s == best && r < brow)) {
      best = s;
      brow = r;
    }
  }
  __shared__ double ss[QT / 32];
  __shared__ int rr[QT / 32];
  block_argmax(best, brow, ss, rr);
  // no row left with a positive residual: the remaining pivots are void
  const bool none = !(best > 0.0) || brow < 0 || brow >= g.n;
  if (none) {
    if (threadIdx.x == 0) piv[j] = -1;
    return;
  }
  const T* U = us.at(slot, side);
  double* qv = q.qv + (int64_t)ss_i * M * M;  // row l: q_l (M entries)
  __shared__ double u[kMaxM];
  __shared__ double d[kMaxM];
  for (int k = threadIdx.x; k < c; k += QT) u[k] = (double)U[(int64_t)k * g.ld + brow];
  __syncthreads();
  for (int pass = 0; pass < 2; ++pass) {
    for (int l = 0; l < j; ++l) {
      // d_l = u . q_l (warp 0), then u -= d_l q_l
      if (threadIdx.x < 32) {
        double a = 0.0;
        for (int k = threadIdx.x; k < c; k += 32) a = fma(u[k], qv[(int64_t)l * M + k], a);
        a = warp_sum(a);
        if (threadIdx.x == 0) d[0] = a;
      }
      __syncthreads();
      const double dl = d[0];
      for (int k = threadIdx.x; k < c; k += QT) u[k] = fma(-dl, qv[(int64_t)l * M + k], u[k]);
      __syncthreads();
    }
  }
  if (threadIdx.x < 32) {
    double a = 0.0;
    for (int k = threadIdx.x; k < c; k += 32) a = fma(u[k], u[k], a);
    a = warp_sum(a);
    if (threadIdx.x == 0) d[1] = a;
  }
  __syncthreads();
  const double nrm = sqrt(d[1]);
  const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
  for (int k = threadIdx.x; k < c; k += QT) qv[(int64_t)j * M + k] = u[k] * inv;
  if (threadIdx.x == 0) piv[j] = brow;
}

// Downdate the chunk's residual norms by (U(i,:) q_j)^2; the picked row leaves.
template <typename T>
__global__ void __launch_bounds__(QT) k_qdeim_update(TallGeom g, const SolveState* __restrict__ st_all,
                                                     Strided<const T> us, int sel, QdeimBufs q, int j) {
  const int slot = slot_of(g, blockIdx.y >> 1), side = blockIdx.y & 1;
  if (slot < 0) return;
  const SolveState& st = st_all[slot];
  if (!st.active) return;
  const int c = dim_of(st, side, sel);
  if (j + 1 >= c) return;  // no later pivot reads these norms
  const int ss_i = slot * 2 + side;
  const int M = g.M;
  const int p = q.piv[(int64_t)ss_i * M + j];
  if (p < 0) return;  // void pivot: every later one is void too
  const T* U = us.at(slot, side);
  const double* qj = q.qv + (int64_t)ss_i * M * M + (int64_t)j * M;
  __shared__ double qs[kMaxM];
  for (int k = threadIdx.x; k < c; k += QT) qs[k] = qj[k];
  __syncthreads();
  double* qn = q.qn + (int64_t)ss_i * g.ld;
  const int rbeg = blockIdx.x * q.chunk_rows, rend = min(g.n, rbeg + q.chunk_rows);
  double best = -1.0;
  int brow = 0x7fffffff;
  for (int i = rbeg + threadIdx.x; i < rend; i += QT) {
    double s = qn[i];
    if (s >= 0.0) {
      if (i == p) {
        s = -1.0;  // picked
      } else {
        double a = 0.0;
        for (int k = 0; k < c; ++k) a = fma((double)U[(int64_t)k * g.ld + i], qs[k], a);
        s = fmax(s - a * a, 0.0);
      }
      qn[i] = s;
    }
    if (s > best || (s == best && i < brow)) {
      best = s;
      brow = i;
    }
  }
  __shared__ double ss[QT / 32];
  __shared__ int rr[QT / 32];
  block_argmax(best, brow, ss, rr);
  if (threadIdx.x == 0) {
    const int64_t o = ((int64_t)ss_i * 2 + ((j + 1) & 1)) * q.nchunk + blockIdx.x;
    q.cs[o] = best;
    q.ci[o] = brow;
  }
}

// The pivots as ranked candidates (block 0, scores c - j), every other candidate empty.
__global__ void k_qdeim_emit(TallGeom g, const SolveState* __restrict__ st_all, int sel, QdeimBufs q,
                             double* __restrict__ cscore, int32_t* __restrict__ cidx, int cand_blocks,
                             int cand_per_block) {
  const int slot = slot_of(g, blockIdx.x >> 1), side = blockIdx.x & 1;
  if (slot < 0) return;
  const SolveState& st = st_all[slot];
  if (!st.active) return;
  const int c = dim_of(st, side, sel);
  const int ss_i = slot * 2 + side;
  const int total = cand_blocks * cand_per_block;
  const int64_t base = (int64_t)ss_i * total;
  const int32_t* piv = q.piv + (int64_t)ss_i * g.M;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    int r = -1;
    if (t < c && t < cand_per_block) r = piv[t];
    cidx[base + t] = r;
    cscore[base + t] = r >= 0 ? (double)(c - t) : -1.0;
  }
}

template <typename T>
cudaError_t launch_qdeim(const TallGeom& g, const SolveState* st, Strided<const T> us, int sel, const QdeimBufs& q,
                         double* cscore, int32_t* cidx, int cand_blocks, int cand_per_block, int max_c,
                         cudaStream_t s) {
  const dim3 rows(q.nchunk, g.nslots * 2);
  k_qdeim_init<T><<<rows, QT, 0, s>>>(g, st, us, sel, q);
  for (int j = 0; j < max_c; ++j) {
    k_qdeim_pivot<T><<<g.nslots * 2, QT, 0, s>>>(g, st, us, sel, q, j);
    if (j + 1 < max_c) k_qdeim_update<T><<<rows, QT, 0, s>>>(g, st, us, sel, q, j);
  }
  k_qdeim_emit<<<g.nslots * 2, 256, 0, s>>>(g, st, sel, q, cscore, cidx, cand_blocks, cand_per_block);
  return cudaGetLastError();
}

template cudaError_t launch_qdeim<float>(const TallGeom&, const SolveState*, Strided<const float>, int,
                                         const QdeimBufs&, double*, int32_t*, int, int, int, cudaStream_t);
template cudaError_t launch_qdeim<double>(const TallGeom&, const SolveState*, Strided<const double>, int,
                                          const QdeimBufs&, double*, int32_t*, int, int, int, cudaStream_t);

}  // namespace lrp
