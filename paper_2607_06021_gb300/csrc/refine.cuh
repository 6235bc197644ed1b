// Mixed-precision refinement kernels (see refine.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "core.cuh"

namespace lrp {

struct RefineArgs {
  int n;
  int64_t ld;
  int M;
  SolveState* st;
  const ProblemDev* prob;
  const double* lam;           // FP64 eigenvalues
  Strided<const double> Fh64;  // FP64 transformed right-hand side, n x rf
  Strided<const float> U32[2]; // FP32 ping-pong factors of the inner solves
  Strided<const double> U64;   // FP64 factors of the solution being refined (a second step), or base nullptr
  Strided<double> X;           // FP64 stacked blocks, n x M (CholeskyQR input)
  Strided<float> X32;          // FP32 stacked blocks (the sum's are FP32 values; the residual's the hi plane), or base nullptr
  Strided<float> X32lo;        // lo plane of the residual's stacked blocks in double-float, or base nullptr
  Strided<double> stash;       // FP64 copy of the trial factors Uh0 / Vh0
  Strided<double> Racc;        // FP64 R of the CholeskyQR passes
  Strided<double> P;           // FP64 inverse of the last pass's R
  Strided<double> Bf;          // out: small factors of the recompressed product
  const double* sig32;         // singular values of the FP32 solves: [slot][2][M]
  double* dvec;                // per slot M: diagonal weights of the stacked product
  double* s0;                  // per slot M: singular values of the trial solution
  double* sig_out;             // out: singular values of the recompressed product
  int64_t sig_out_stride;
  double* scratch;             // per slot >= 2 M^2 doubles
  int64_t scratch_stride;
  float* w32;                  // weights of the FP32 correction solve
  int wstride;
  double* acct;                // per slot LRP_K_COUNT x {flops, bytes} (see core.cuh)
  int NB;                      // Gram partial blocks of the plan
  double corr_tol;             // stop-test tolerance floor of the FP32 correction solve
  double final_tol;            // the solve's tolerance: the correction's absolute target is final_tol ||S0||
};

// Raises the dynamic shared-memory limit of the recompression kernels (once per device).
cudaError_t refine_configure();
cudaError_t launch_prepare_refine(const RefineArgs& a, int nslots, cudaStream_t s);
cudaError_t launch_assemble_residual(const RefineArgs& a, int nslots, cudaStream_t s);
cudaError_t launch_recompress(const RefineArgs& a, int nslots, int mode, double rel_tol, int rcap, cudaStream_t s);
cudaError_t launch_setup_correction(const RefineArgs& a, int nslots, cudaStream_t s);
template <typename TS, typename TD>
cudaError_t launch_convert(int n, int64_t ld, int nslots, const SolveState* st, Strided<const TS> src,
                           Strided<TD> dst, int sel, cudaStream_t s);
cudaError_t launch_prepare_sum(const RefineArgs& a, int nslots, cudaStream_t s);
cudaError_t launch_assemble_sum(const RefineArgs& a, int nslots, cudaStream_t s);
cudaError_t launch_final_state(const RefineArgs& a, int nslots, cudaStream_t s);
// Second refinement step: flag the problems whose first correction looks
// unreliable (count of flagged in *count) and hold the others out of it.
cudaError_t launch_check_refine(const RefineArgs& a, int nslots, int32_t* count, cudaStream_t s);
cudaError_t launch_prepare_refine2(const RefineArgs& a, int nslots, cudaStream_t s);
cudaError_t launch_release_held(const RefineArgs& a, int nslots, cudaStream_t s);

}  // namespace lrp
