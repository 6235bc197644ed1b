// Shared definitions of the sm_103a kernels and the host driver.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lrp.h"

#ifndef LRP_MAX_M
#define LRP_MAX_M 256  // hard cap on index-set sizes and ranks (m_cap)
#endif

namespace lrp {

constexpr int kMaxM = LRP_MAX_M;
constexpr int kMaxRF = 256;
// Per-iteration trace (lrp_plan_set_trace): entries per slot, doubles per entry.
constexpr int kTraceLen = 96;  // LRP_TRACE_LEN
constexpr int kTraceWidth = 8;

// Per-problem iteration state, one per batch slot, in device memory.
// Side 0 is the row space (cross matrix C = What(:,J), factor U_k, index set
// I); side 1 is the column space (R^T = What(I,:)^T, factor V_k, index set J).
struct SolveState {
  int32_t active;        // 1 while the Cross-DEIM loop runs for this slot
  int32_t k;             // next iteration number
  int32_t cnt[2];        // |I|, |J|
  int32_t r;             // rank of the current iterate
  int32_t r_prev;        // rank of the previous iterate (0 = none)
  int32_t rf;            // right-hand-side rank
  int32_t flags;         // kFlag* bits
  int32_t iters;         // iterations done in this solve
  int32_t r_out;         // final rank
  int32_t r_star;        // tail-rule rank before the cap
  int32_t total_iters;   // across initial and refinement solves
  int32_t branch;        // scross branch taken (0: |J|<=|I|, 1: mirror)
  int32_t cnt_next[2];   // |I|, |J| after the redundancy removal (applied by k_stop,
                         // after the factor update has used the pre-removal sizes)
  int32_t mx[2];         // generic column counts of the refinement's tall matrices
  int32_t r0;            // rank of the trial solution being refined
  int32_t valid;         // slot holds a problem of this call
  int32_t rf0;           // rank of the caller's right-hand side
  int32_t upar;          // ping-pong parity of the FP32 iterate being stacked
  int32_t rd;            // rank of the correction
  int32_t first_converged;  // the first (FP32) solve met its stop test
  int32_t c0[2];         // columns of U_{-1}, V_{-1}: their numerical rank (cold) or the warm iterate's rank
  int32_t warm_ok;       // this solve may load a warm-start record
  double rho;
  double eta_smin;
  double snorm;          // ||S_k||_F
  double snorm_prev;
  double gram_trace[2];  // trace of the pass-1 Gram (shift scale)
  double tol;            // stop-test tolerance of the current solve (relative to ||S_k||)
  double tol_abs;        // > 0: also accept changes below tol_abs in absolute terms (correction solves)
  double rho_best;       // smallest rho of this solve after its first iteration (0: none yet)
  int32_t stall;         // iterations since rho last fell below half of rho_best
  int32_t is_corr;       // this solve is a refinement correction (mixed precision)
  double rho_jump;       // largest rho / rho_best seen after rho_best was first set
};

enum : int32_t {
  kFlagConverged = 1,
  kFlagRankCapped = 2,
  kFlagCapacity = 4,   // index set hit m_cap
  kFlagBadInput = 8,
  kFlagStalled = 16,   // FP32 solve stopped at its noise floor (change stopped halving)
  kFlagRolledBack = 32,  // a stalled FP32 solve returned its previous iterate
  kFlagRefinedTwice = 64,  // a second refinement step ran
  kFlagHeld = 128,     // internal: kept out of the second refinement step
};

// Size selectors for the generic tall kernels: which per-side dimension of
// the state a kernel's column count comes from.
enum DimSel : int32_t {
  kDimOther = 0,  // cnt[1-s]: columns of side s's cross matrix
  kDimR = 1,      // r
  kDimRPrev = 2,  // r_prev
  kDimRF = 3,     // rf
  kDimX = 4,      // mx[s]
  kDimC0 = 5,     // c0
};

__host__ __device__ inline int dim_of(const SolveState& st, int side, int sel) {
  switch (sel) {
    case kDimOther: return st.cnt[1 - side];
    case kDimR: return st.r;
    case kDimRPrev: return st.r_prev;
    case kDimX: return st.mx[side];
    case kDimC0: return st.c0[side];
    default: return st.rf;
  }
}

// Strided batch addressing: element (slot, side) of an array of equal blocks.
template <typename T>
struct Strided {
  T* base;
  int64_t side_stride;  // elements between side 0 and side 1
  int64_t slot_stride;  // elements between consecutive slots
  __host__ __device__ T* at(int slot, int side) const {
    return base + (int64_t)slot * slot_stride + (int64_t)side * side_stride;
  }
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum (blockDim.x a multiple of 32, <= 1024); `scratch` >= 32 doubles.
__device__ inline double block_sum(double v, double* scratch) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  const int nw = blockDim.x >> 5;
  double t = (threadIdx.x < nw) ? scratch[threadIdx.x] : 0.0;
  if (wid == 0) t = warp_sum(t);
  if (threadIdx.x == 0) scratch[0] = t;
  __syncthreads();
  double r = scratch[0];
  __syncthreads();
  return r;
}

__device__ inline double block_max(double v, double* scratch) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  const int nw = blockDim.x >> 5;
  double t = (threadIdx.x < nw) ? scratch[threadIdx.x] : -1.0e308;
  if (wid == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_xor_sync(0xffffffffu, t, o));
  }
  if (threadIdx.x == 0) scratch[0] = t;
  __syncthreads();
  double r = scratch[0];
  __syncthreads();
  return r;
}

// SplitMix64 output function (Steele, Lea, Flood, OOPSLA 2014): add the golden
// gamma, then two xor-shift-multiply rounds and a final xor-shift.
__host__ __device__ inline uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011): ten rounds of the
// 4x32 S-box (two 32 x 32 -> 64-bit products, xored with the other counter
// words and the key), the 2x32 key advanced by the Weyl increments before
// every round but the first.
__host__ __device__ inline void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0;
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = (uint32_t)p1;
    c[2] = n2;
    c[3] = (uint32_t)p0;
  }
}

// Uniform double in [0, 1) with 53 random bits for (row, iteration k, side):
// Philox4x32-10 with counter (row, k, side, 0) and key (low, high words of
// seed); (x0 >> 5) 2^26 + (x1 >> 6), scaled by 2^-53.
__host__ __device__ inline double philox_uniform(uint64_t seed, uint32_t k, uint32_t side, uint32_t row) {
  uint32_t c[4] = {row, k, side, 0u};
  philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  return ((double)(c[0] >> 5) * 67108864.0 + (double)(c[1] >> 6)) * (1.0 / 9007199254740992.0);
}

// Device part of a warm-start record (lrp_warm_t).
struct WarmDev {
  int32_t valid;      // holds a result
  int32_t cnt[2];     // |I|, |J|
  int32_t r;          // rank of the stored iterate
  int64_t ld;         // leading dimension of U
  int32_t* idx;       // 2 x M index sets
  double* U;          // 2 x (ld x M): transformed iterate Uh (side 0), Vh (side 1)
};

}  // namespace lrp
