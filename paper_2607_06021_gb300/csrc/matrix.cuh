// Cross-DEIM on the test matrices of Sec. 4.1 by entries (see matrix.cu).
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"
#include "dst.cuh"
#include "tall.cuh"

namespace lrp {

// Sampled columns (side 0) / rows (side 1) of the matrix `kind` (lrp_matrix)
// into A (n x |J| and n x |I|, leading dimension g.ld), from the index sets idx.
cudaError_t launch_cross_matrix(const TallGeom& g, const SolveState* st, int kind, Strided<double> A,
                                Strided<const int32_t> idx, cudaStream_t s);
// Batched column copy through the pointer tables of a DstBatch (the transform
// of the Poisson path is the identity here).
cudaError_t launch_copy_cols(const DstBatch<double, double>& job, int n, int max_cols, cudaStream_t s);

}  // namespace lrp
