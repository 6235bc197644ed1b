// Tall-skinny kernels over all problems of a batch (see tall.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace lrp {

// Geometry shared by the tall kernels of one plan.
struct TallGeom {
  int n;        // rows
  int64_t ld;   // leading dimension of every n-row workspace matrix (>= n, multiple of 32)
  int M;        // capacity (m_cap): columns of n-row matrices, order of small matrices
  int nslots;   // batch slots launched (grid entries; see act)
  int NB;       // row blocks of the Gram partials
  int rows_per_block;  // ceil(n / NB) rounded up to 32
  // Slot of each launched entry: act[i] (-1: nothing to do), or the identity
  // when null.  The Cross-DEIM iterations launch over the compacted list of
  // the slots still active, so that finished slots cost no CTAs.
  const int32_t* act = nullptr;
  // Rows per thread of the narrow (thread-per-row) products, 1 or 2 (0: 2 for
  // FP32 data, 1 for FP64); a launch shape only, outputs do not depend on it.
  int gemm_rpt = 0;
};

__device__ __forceinline__ int slot_of(const TallGeom& g, int i) { return g.act ? g.act[i] : i; }

// Whether a tall product of data type T with index capacity M (every width is
// at most M) can need the register-tiled kernel: wider than the thread-per-row
// kernel's 32 input columns (64 for FP32) or 64 outputs.  Such products take a
// second launch.
template <typename T>
inline bool gemm_wide_possible(int M) {
  return M > (sizeof(T) == 4 ? 64 : 32);
}

template <typename T>
struct CrossArgs {
  Strided<const T> F;          // transformed RHS factors, n x rf, ld = geom.ld
  const T* w;                  // per slot: rf weights h^2 s_f (slot stride wstride)
  int wstride;
  const T* lam;                // eigenvalues lambda_1..lambda_n (shared)
  Strided<const int32_t> idx;  // index sets, M entries per (slot, side)
  Strided<T> A;                // out: n x M
};

template <typename T>
cudaError_t launch_cross(const TallGeom& g, const SolveState* st, const CrossArgs<T>& a, cudaStream_t s);

// Out[s] = In[s](:, :mi) * Bm[s](:mi, :mo)  (mode 0)  or  Out = Zsub - In * Bm  (mode 1).
// mi, mo come from the state through the DimSel codes; Bm is M x M col-major (ld M).
template <typename T>
cudaError_t launch_gemm_nn(const TallGeom& g, const SolveState* st, Strided<const T> in, int sel_in,
                           Strided<const double> bm, int sel_out, Strided<T> out, Strided<const T> zsub, int mode,
                           cudaStream_t s);

// part[s][blk] = X[s](rows of blk, :mx)^T Y[s](rows of blk, :my) in FP64 (launch_gram),
// then G[s] = sum over blk (launch_reduce).
template <typename T>
cudaError_t launch_gram(const TallGeom& g, const SolveState* st, Strided<const T> x, int sel_x,
                        Strided<const T> y, int sel_y, double* part, Strided<double> G, bool symmetric,
                        cudaStream_t s, bool acc64 = true);

cudaError_t launch_reduce(const TallGeom& g, const SolveState* st, int sel_x, int sel_y, const double* part,
                          Strided<double> G, bool symmetric, cudaStream_t s);

// Raises the dynamic shared-memory limit of the leverage kernels (once per device).
cudaError_t tall_configure();

// Work buffers of the QDEIM selection (per problem and side).
struct QdeimBufs {
  double* qn;        // [slots x 2][ld] residual row norms^2 (-1 once picked)
  double* qv;        // [slots x 2][M][M] row l: orthonormal direction q_l of the picked rows
  double* cs;        // [slots x 2][2][nchunk] best residual norm per row chunk (two step parities)
  int32_t* ci;       // [slots x 2][2][nchunk] its row
  int32_t* piv;      // [slots x 2][M] pivots in order (-1: none)
  int nchunk;        // row chunks of chunk_rows rows
  int chunk_rows;
};

// QDEIM (Algorithm IS): the first c = dim(sel) pivots of the column-pivoted QR of
// U[s](:, :c)^T, handed to the index-set merge as ranked candidates (block 0 of
// cand_score / cand_idx, in pivot order).  max_c bounds c over the batch (the
// plan's m_cap): 2 max_c + 1 launches.
template <typename T>
cudaError_t launch_qdeim(const TallGeom& g, const SolveState* st, Strided<const T> us, int sel, const QdeimBufs& q,
                         double* cscore, int32_t* cidx, int cand_blocks, int cand_per_block, int max_c,
                         cudaStream_t s);

// Double-float tall products on the FP32 pipe (dfmat.cu).  Out = A * Bm with A FP32
// (al.base == nullptr) or (hi, lo) planes, Bm FP64 (M x M, ld M); output FP64
// when o64.base is set, else (hi, lo) planes.  Gram partials of (hi, lo) data
// with at most 64 columns (then launch_reduce).
cudaError_t launch_gemm_dfx(const TallGeom& g, const SolveState* st, Strided<const float> ah, Strided<const float> al,
                            int sel_in, Strided<const double> bm, int sel_out, Strided<float> oh, Strided<float> ol,
                            Strided<double> o64, cudaStream_t s, bool tri = false);
cudaError_t launch_gram_dd(const TallGeom& g, const SolveState* st, Strided<const float> xh, Strided<const float> xl,
                           int sel, double* part, cudaStream_t s);

// Bernoulli form of Algorithm LeverageScores: when on, row i is a candidate
// with probability min(1, factor * ||U(i,:)||^2), keyed by its score.  The
// draw belongs to the iteration that uses the candidates: the slot's k plus
// k_ofs (0 before the first iteration, 1 at the end of iteration k).
struct LevSample {
  int on = 0;
  int k_ofs = 0;
  uint64_t seed = 0;
  double factor = 1.0;
};

// Leverage scores of U[s](:, :c) rows (c from sel) and per-block candidates:
// the top c rows, or the best cand_per_block sampled rows (Bernoulli).
template <typename T>
cudaError_t launch_leverage(const TallGeom& g, SolveState* st, Strided<const T> U, int sel,
                            double* cand_score, int32_t* cand_idx, int cand_blocks, int cand_per_block,
                            cudaStream_t s, LevSample ls = LevSample());

}  // namespace lrp
