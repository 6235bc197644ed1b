// Per-problem small dense kernels of the Cross-DEIM iteration (see core.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "dst.cuh"
#include "tall.cuh"

namespace lrp {

// Device-side description of one batch slot's caller buffers.
struct ProblemDev {
  int32_t rf;
  int32_t pad;
  const double* U_f;
  int64_t ldu_f;
  const double* s_f;
  const double* V_f;
  int64_t ldv_f;
  double* U;
  int64_t ldu;
  double* S;
  double* V;
  int64_t ldv;
  lrp_info* info;
  WarmDev* warm;   // warm-start record or nullptr
};

struct CoreParams {
  TallGeom g;
  SolveState* st;
  int max_iter;
  int r_max;
  double tol;          // Cross-DEIM epsilon (relative)
  double eps_data;     // unit roundoff of the tall data (in-loop cutoff scale)
  double shift_rel;    // pass-1 shift of shifted CholeskyQR, relative to trace(G)
  double drop_rel;     // Cholesky pivot drop threshold (relative to the pass's max diagonal)
  double redundancy;   // |diag R| threshold relative to max |diag R| (paper: 1e-12)
  uint64_t seed;
  int selector;        // lrp_selector
  double sample_factor;  // LRP_SEL_BERNOULLI: c / columns
  int noise_floor_stop;  // 1: the eta S_min term counts as met once S_min is at the data's noise floor
  int dst_df;          // 1: the back transform runs in double-float arithmetic (work accounting)
  int cand_blocks;     // leverage candidate blocks per side
  int cand_per_block;
  double* trace;       // [nslots][kTraceLen][kTraceWidth] per-iteration record, or nullptr
};

// Per-slot buffers used by the core kernels (all FP64 unless noted, M x M col-major).
template <typename T>
struct CoreBufs {
  Strided<double> G;      // reduced Gram (input of k_chol)
  Strided<double> Racc;   // accumulated R of the CholeskyQR passes
  Strided<double> P;      // inverse of this pass's R (applied by the tall GEMM)
  Strided<double> Bf;     // final small factor: U_k = Q2 * Bf
  Strided<double> X;      // cross-Gram U_k^T U_{k-1} (side 0), V_k^T V_{k-1} (side 1)
  Strided<double> GE;     // Gram of E = U_{k-1} - U_k X
  Strided<const T> Q2;    // n x M second-pass basis (gathered rows only)
  Strided<int32_t> idx;   // index sets (M per side)
  double* sig;            // per slot: 2 x M singular values (ping-pong by iteration parity)
  double* scratch;        // per slot: kCoreScratch * M * M doubles
  int64_t scratch_stride;
  double* cand_score;     // leverage candidates
  int32_t* cand_idx;
  const ProblemDev* prob; // per slot caller buffers
  double* acct;           // per slot: LRP_K_COUNT x {flops, bytes} of algorithmic work
};

// Algorithmic work of one Cross-DEIM iteration / of the setup, added to a slot's
// row of the accounting array (minimal flops and HBM bytes of each kernel class,
// independent of tiling waste).
__device__ void acct_iteration(double* row, int n, int p, int q, int r, int rp, int rf, int NB, int w);
__device__ void acct_setup(double* row, int n, int rf, int NB, int w);
__device__ void acct_back(double* row, int n, int r_out, int w);

constexpr int kCoreScratch = 12;  // M x M FP64 regions per slot

template <typename T>
cudaError_t launch_chol(const CoreParams& p, const CoreBufs<T>& b, int sel, int pass, cudaStream_t s);
template <typename T>
cudaError_t launch_core(const CoreParams& p, const CoreBufs<T>& b, int parity, cudaStream_t s);
template <typename T>
cudaError_t launch_select(const CoreParams& p, const CoreBufs<T>& b, int sel_c, cudaStream_t s);
template <typename T>
cudaError_t launch_stop(const CoreParams& p, const CoreBufs<T>& b, int parity, cudaStream_t s);
// Final truncation and per-slot back-transform job (pointer arrays of `back`
// are device memory written by the kernel); ubufs[2] are the ping-pong factor
// buffers (device array of two pointers).
template <typename T>
cudaError_t launch_finalize_impl(const CoreParams& p, const CoreBufs<T>& b, const DstBatch<T, double>& back,
                                 T* const* ubufs, int64_t side_stride, int64_t slot_stride, cudaStream_t s);

// Setup of each slot: state, h^2-scaled weights (type T) from the caller's s_f.
template <typename T>
cudaError_t launch_setup(const CoreParams& p, const ProblemDev* prob, T* w, int wstride, int nslots_active,
                         double* acct, cudaStream_t s);

// Raises the dynamic shared-memory limits of the per-problem kernels (once per process).
cudaError_t core_configure();

// Warm start: slots whose record holds a result replace U_{-1}, V_{-1} (in U1,
// the ping-pong buffer of iteration -1), the index sets and c0; store copies the
// final iterate (parity from the slot's iteration count) and sets into the record.
template <typename T>
cudaError_t launch_warm_load(const CoreParams& p, const CoreBufs<T>& b, Strided<T> U1, cudaStream_t s);
template <typename T>
cudaError_t launch_orth_keep(const CoreParams& p, const CoreBufs<T>& b, cudaStream_t s);
template <typename T>
cudaError_t launch_warm_store(const CoreParams& p, const CoreBufs<T>& b, T* const* ubufs, int64_t side_stride,
                              int64_t slot_stride, cudaStream_t s);

// Eigenvalues lambda_k = 4 sin^2(pi k / (2(n+1))), k = 1..n, in FP64 and FP32.
cudaError_t launch_eigenvalues(int n, double* lam64, float* lam32, cudaStream_t s);

// Number of active slots (written to a host-visible counter).
cudaError_t launch_count_active(const SolveState* st, int nslots, int32_t* out, int32_t* list, cudaStream_t s);
// Copies `bytes` (a multiple of 4, both ends 4-byte aligned) with a kernel on
// stream s.  The solve path moves its control data (job descriptors up, active
// counts down) this way, through the device aliases of mapped pinned host
// buffers, so that it never waits on a copy engine that a caller's bulk
// transfers on other streams hold.
cudaError_t launch_stage(const void* src, void* dst, size_t bytes, cudaStream_t s);
// Condition of a conditional if-node: *count > 0.
cudaError_t launch_cond_positive(const int32_t* count, cudaGraphConditionalHandle h, cudaStream_t s);
// Loop control of a device-side (conditional while-node) iteration loop.
cudaError_t launch_loop_begin(const int32_t* active, int32_t* trips, cudaGraphConditionalHandle h, cudaStream_t s);
cudaError_t launch_loop_next(const int32_t* active, int32_t* trips, int max_trips, cudaGraphConditionalHandle h,
                             cudaStream_t s);

}  // namespace lrp
