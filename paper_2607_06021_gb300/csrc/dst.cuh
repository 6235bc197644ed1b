// DST-I launch interface (see dst.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lrp {

// Device-resident description of a batch of column blocks to transform.
// Arrays in/out/ld_in/ld_out have nmats * nslots entries, index mat*nslots+slot.
template <typename TIn, typename TOut>
struct DstBatch {
  const TIn* const* in;
  TOut* const* out;
  const int64_t* ld_in;
  const int64_t* ld_out;
  int nslots;
  int fixed_cols;              // used when ncols_dev == nullptr
  const int32_t* ncols_dev;    // per-slot column counts (device), or nullptr
  int ncols_stride;            // int32 stride between slots in ncols_dev
  int ncols_mat_stride;        // int32 stride between the two matrices
  const int32_t* active_dev;   // optional per-slot flag; skip slots with 0 if require_active
  int active_stride;
  int require_active;
};

// Raises the dynamic shared-memory limit of the DST kernels (call once per process).
cudaError_t dst_configure();
void* dst_make_twiddles(int64_t N, bool fp64, cudaStream_t st);
// Double-float twiddles (for dst1_launch<..., dfloat>).
void* dst_make_twiddles_df(int64_t N, cudaStream_t st);
size_t dst_smem_bytes(int64_t n, bool fp64);
bool dst_smem_supported(int64_t n, bool fp64);
bool dst_supported(int64_t n);  // n+1 <= 2^21 (shared-memory or multi-pass)

// Bytes of HBM staging one column needs in the multi-pass DST (0 when the
// shared-memory kernel applies, n+1 <= 8192 in FP64 / 16384 in FP32).
size_t dst_temp_bytes(int64_t n, bool fp64);

// temp: staging of max_cols * nslots * nmats * dst_temp_bytes(n) bytes (multi-pass only).
// cta_threads: threads per CTA of the shared-memory kernel (256, 512 or 1024, capped
// at 512 for FP64 and double-float; 0: 256); each column's arithmetic is the same
// whatever the value.
template <typename TIn, typename TOut, typename TC>
cudaError_t dst1_launch(int64_t n, const DstBatch<TIn, TOut>& job, int max_cols, int nslots, int nmats,
                        const void* tw, cudaStream_t st, void* temp = nullptr, size_t temp_bytes = 0,
                        int cta_threads = 0);

}  // namespace lrp
