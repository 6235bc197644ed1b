// Plan object and workspace layout (see solver.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "core.cuh"
#include "guard.cuh"

// Device allocations of one plan (released together).
struct DeviceArena {
  std::vector<void*> blocks;
  size_t total = 0;
  bool failed = false;
  bool measure = false;  // sizing pass: count bytes, allocate nothing
  void* raw(size_t bytes);
  template <typename T>
  T* get(size_t count) {
    return reinterpret_cast<T*>(raw(count * sizeof(T) + 1));
  }
  bool ok() const { return !failed; }
  void release();
};

namespace lrp {

// Launch buckets of the iteration graphs: the whole batch, then 1, 2, 4, ... slots.
constexpr int kGraphLevels = 18;

lrp_status set_error(lrp_status s, const std::string& msg);

struct PlanDims {
  int n;
  int64_t ld;          // leading dimension of n-row workspace matrices
  int B;               // batch slots
  int RF;              // right-hand-side rank capacity
  int M;               // index-set / rank capacity (m_cap)
  int NB;              // Gram partial row blocks
  int rows_per_block;
  int cand_blocks;     // leverage candidate blocks (<= 1024 rows each)
  int cand_per_block;
  int qdeim_chunks;    // QDEIM row chunks (0: leverage selection)
  int qdeim_rows;      // rows per QDEIM chunk
};

// HBM layout per batch slot b and side s (0 = rows/U/I, 1 = columns/V/J); every
// n-row matrix is column-major with leading dimension ld:
//   Fh   [b][s]  n x RF   transformed right-hand-side factor (Uhat_f, Vhat_f)
//   A    [b][s]  n x M    cross matrix C = What(:,J) / R^T = What(I,:)^T
//   Q1,Q2[b][s]  n x M    CholeskyQR pass outputs (Q = Q2 P3 implicitly)
//   U[2] [b][s]  n x M    current / previous factors U_k, V_k (ping-pong)
//   part [b][s][NB] M x M FP64 Gram partials; G, Racc, P, Bf, X, GE: M x M FP64
template <typename T>
struct Workspace {
  T* Fh = nullptr;
  T* w = nullptr;
  T* A = nullptr;
  T* Q1 = nullptr;
  T* Q2 = nullptr;
  T* U[2] = {nullptr, nullptr};
  double* part = nullptr;
  double* G = nullptr;
  double* Racc = nullptr;
  double* P = nullptr;
  double* Bf = nullptr;
  double* X = nullptr;
  double* GE = nullptr;
  double* sig = nullptr;
  double* scratch = nullptr;
  int32_t* idx = nullptr;
  double* cand_score = nullptr;
  int32_t* cand_idx = nullptr;
  T** back_in = nullptr;
  double** back_out = nullptr;
  int64_t* back_ldi = nullptr;
  int64_t* back_ldo = nullptr;
  T** ubufs = nullptr;
  const double** fwd_in = nullptr;
  T** fwd_out = nullptr;
  int64_t* fwd_ldi = nullptr;
  int64_t* fwd_ldo = nullptr;
  QdeimBufs qd{};  // QDEIM selection buffers (plans with the QDEIM selector only)
  int rf_cap = 0;  // columns of Fh (and entries of w) per slot and side
  // Captured CUDA graphs of one Cross-DEIM iteration: [0] the first iteration,
  // [1] odd iterations, [2] even iterations >= 2, [3] the initial bases; valid for
  // graph_count problems.  The second index is the launch bucket: level 0 the
  // whole batch, level l >= 1 a compacted list of 2^(l-1) active slots.
  int graph_count = -1;
  cudaGraphExec_t graphs[4][kGraphLevels] = {};
  int64_t graph_launches[4][kGraphLevels][LRP_K_COUNT] = {};
  void release_graphs();
  lrp_status allocate(const PlanDims& d, DeviceArena& arena, int rf_cap);
};

}  // namespace lrp

// Launch counts and optional CUDA-event timing per kernel class.
struct KernelStats {
  bool timing = false;
  int64_t launches[LRP_K_COUNT] = {};
  double ms[LRP_K_COUNT] = {};
  std::vector<cudaEvent_t> pool;
  struct Rec {
    int cls, e0, e1;
  };
  std::vector<Rec> pending;
  int next_event = 0;
  int take(cudaStream_t s);
  void drain();
  void release();
};

struct lrp_plan_s {
  int64_t n = 0;
  double tol = 0.0;
  int r_max = 0;
  lrp_opts opts;
  lrp::PlanDims dims;
  int device = 0;
  DeviceArena arena;
  lrp::SolveState* st = nullptr;
  double* lam64 = nullptr;
  float* lam32 = nullptr;
  void* tw64 = nullptr;
  void* tw32 = nullptr;
  void* twdf = nullptr;                  // double-float twiddles (mixed precision)
  lrp::ProblemDev* prob_dev = nullptr;
  lrp::ProblemDev* prob_host = nullptr;  // pinned
  void* host_ptrs = nullptr;             // pinned staging for DST job arrays
  int32_t* active_dev = nullptr;
  int32_t* act_list = nullptr;           // compacted active slots (written by k_count_active)
  double* acct = nullptr;                // [B][LRP_K_COUNT][2] algorithmic flops / bytes
  double* dvec = nullptr;                // [B][M] weights of the stacked refinement products
  unsigned char* dst_temp = nullptr;     // HBM staging of the multi-pass DST (n+1 > 8192)
  size_t dst_temp_bytes = 0;
  double* s0 = nullptr;                  // [B][M] singular values of the trial solution
  double mixed_inner_tol = 1e-4;         // FP32 Cross-DEIM tolerance (relative)
  int mixed_inner_max_iter = 12;         // iteration cap of each FP32 Cross-DEIM solve
  bool use_graphs = true;                // replay captured CUDA graphs of each iteration
  cudaStream_t cap_stream = nullptr;     // plan-owned stream used only for graph capture
  double mixed_redundancy = 1e-6;        // redundancy threshold on FP32 data
  double mixed_residual_tol = 1e-7;      // tail-rule truncation of the recompressed residual
  int32_t* active_host = nullptr;        // pinned
  // Device aliases of the mapped pinned buffers above (control data moves by
  // kernel, not by copy engine)
  lrp::ProblemDev* prob_host_dev = nullptr;
  void* host_ptrs_dev = nullptr;
  int32_t* active_host_dev = nullptr;
  lrp::Workspace<double> w64;
  lrp::Workspace<float> w32;
  KernelStats stats;
  bool any_warm = false;                 // the current call has warm-start records
  int last_count = 0;                    // problems of the most recent lrp_solve_batch
  double* trace_dev = nullptr;           // [B][kTraceLen][kTraceWidth], allocated on first use
  bool trace_on = false;
  // Device-side iteration loops (opts.loop_on_device): the whole solve is one
  // captured graph; its Cross-DEIM loops are conditional while-nodes.
  bool device_loop = false;
  bool capturing_solve = false;          // a whole-solve capture is open (no host sync or staging)
  cudaStream_t body_stream = nullptr;    // captures the loop bodies
  cudaStream_t if_stream = nullptr;      // captures the mixed path's second refinement step
  int32_t* loop_trips = nullptr;         // device: trips of the running device-side loop
  // Captured solves, one per (count, any_warm, trace_on), the least recently
  // used replaced: batches of varying size (a server's) each replay their own
  // graph instead of capturing and instantiating the whole solve again.
  struct SolveGraph {
    cudaGraphExec_t exec = nullptr;
    int key[3] = {-1, -1, -1};
    uint64_t used = 0;
    int64_t launches[LRP_K_COUNT] = {};  // kernel nodes of the captured solve (loop bodies once)
  };
  static constexpr int kSolveGraphs = 8;
  SolveGraph solve_graphs[kSolveGraphs];
  uint64_t solve_tick = 0;
  cudaEvent_t solve_done = nullptr;      // completion of the last enqueued solve
  std::mutex mu;
};

struct lrp_warm_s {
  lrp_plan_s* plan = nullptr;
  DeviceArena arena;
  lrp::WarmDev* dev = nullptr;
};
