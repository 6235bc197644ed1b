// Host driver and C ABI (include/lrp.h).
//
// A plan owns all device workspace for `batch` problems of one grid size n and
// runs the low-rank Poisson solve of the paper's Sec. 3.2: DST-I of the
// right-hand-side factors, Cross-DEIM (Algorithm "Cross-DEIM") on the
// transformed solution What = h^2 Fhat ./ (lambda_i + lambda_j) (Eq. g_for_p),
// final truncation and the back transform.  Every step runs in this library's
// kernels; the host only sequences launches and reads one device counter of
// still-iterating problems between iterations.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "core.cuh"
#include "dfloat.cuh"
#include "dst.cuh"
#include "matrix.cuh"
#include "refine.cuh"
#include "solver.cuh"
#include "tall.cuh"

namespace lrp {

thread_local std::string g_last_error;

std::shared_mutex& setup_mutex() {
  static std::shared_mutex m;
  return m;
}

lrp_status set_error(lrp_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

#define LRP_CUDA(call)                                                                              \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess)                                                                          \
      return set_error(LRP_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_) + " @" +        \
                                      std::to_string(__LINE__));                                    \
  } while (0)

// Brackets one library call that launches `nk` kernels of class `cls`.
#define LRP_LAUNCH(P, CLS, NK, S, call)                                                             \
  do {                                                                                              \
    int ev0_ = (P)->stats.timing ? (P)->stats.take(S) : -1;                                         \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess)                                                                          \
      return set_error(LRP_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_) + " @" +        \
                                      std::to_string(__LINE__));                                    \
    (P)->stats.launches[CLS] += (NK);                                                               \
    if (ev0_ >= 0) (P)->stats.pending.push_back({(CLS), ev0_, (P)->stats.take(S)});                 \
  } while (0)

// Kernel class of a tall product on data of type T.
template <typename T>
static constexpr int gemm_class() {
  return sizeof(T) == 4 ? LRP_K_GEMM_F32 : LRP_K_GEMM;
}

template <typename T>
lrp_status Workspace<T>::allocate(const PlanDims& d, DeviceArena& arena, int rfc) {
  const int64_t nm = d.ld * d.M;
  const int64_t MM = (int64_t)d.M * d.M;
  rf_cap = rfc;
  Fh = arena.get<T>((size_t)d.B * 2 * d.ld * rf_cap);
  w = arena.get<T>((size_t)d.B * rf_cap);
  A = arena.get<T>((size_t)d.B * 2 * nm);
  Q1 = arena.get<T>((size_t)d.B * 2 * nm);
  Q2 = arena.get<T>((size_t)d.B * 2 * nm);
  U[0] = arena.get<T>((size_t)d.B * 2 * nm);
  U[1] = arena.get<T>((size_t)d.B * 2 * nm);
  part = arena.get<double>((size_t)d.B * 2 * d.NB * MM);
  G = arena.get<double>((size_t)d.B * 2 * MM);
  Racc = arena.get<double>((size_t)d.B * 2 * MM);
  P = arena.get<double>((size_t)d.B * 2 * MM);
  Bf = arena.get<double>((size_t)d.B * 2 * MM);
  X = arena.get<double>((size_t)d.B * 2 * MM);
  GE = arena.get<double>((size_t)d.B * 2 * MM);
  sig = arena.get<double>((size_t)d.B * 2 * d.M);
  scratch = arena.get<double>((size_t)d.B * kCoreScratch * MM);
  idx = arena.get<int32_t>((size_t)d.B * 2 * d.M);
  cand_score = arena.get<double>((size_t)d.B * 2 * d.cand_blocks * d.cand_per_block);
  cand_idx = arena.get<int32_t>((size_t)d.B * 2 * d.cand_blocks * d.cand_per_block);
  if (d.qdeim_chunks > 0) {
    qd.nchunk = d.qdeim_chunks;
    qd.chunk_rows = d.qdeim_rows;
    qd.qn = arena.get<double>((size_t)d.B * 2 * d.ld);
    qd.qv = arena.get<double>((size_t)d.B * 2 * MM);
    qd.cs = arena.get<double>((size_t)d.B * 2 * 2 * d.qdeim_chunks);
    qd.ci = arena.get<int32_t>((size_t)d.B * 2 * 2 * d.qdeim_chunks);
    qd.piv = arena.get<int32_t>((size_t)d.B * 2 * d.M);
  }
  back_in = arena.get<T*>((size_t)2 * d.B);
  back_out = arena.get<double*>((size_t)2 * d.B);
  back_ldi = arena.get<int64_t>((size_t)2 * d.B);
  back_ldo = arena.get<int64_t>((size_t)2 * d.B);
  ubufs = arena.get<T*>(2);
  fwd_in = arena.get<const double*>((size_t)2 * d.B);
  fwd_out = arena.get<T*>((size_t)2 * d.B);
  fwd_ldi = arena.get<int64_t>((size_t)2 * d.B);
  fwd_ldo = arena.get<int64_t>((size_t)2 * d.B);
  if (!arena.ok()) return set_error(LRP_ENOMEM, "workspace allocation failed");
  if (arena.measure) return LRP_OK;
  T* ub[2] = {U[0], U[1]};
  LRP_CUDA(cudaMemcpy(ubufs, ub, sizeof(ub), cudaMemcpyHostToDevice));
  return LRP_OK;
}

template <typename T>
void Workspace<T>::release_graphs() {
  for (auto& row : graphs)
    for (auto& g : row)
      if (g) {
        cudaGraphExecDestroy(g);
        g = nullptr;
      }
  graph_count = -1;
}

template struct Workspace<double>;
template struct Workspace<float>;

}  // namespace lrp

using namespace lrp;

// ------------------------------------------------------------------- stats

int KernelStats::take(cudaStream_t s) {
  if (next_event >= (int)pool.size()) {
    cudaEvent_t e;
    SetupGuard guard;
    if (cudaEventCreate(&e) != cudaSuccess) return -1;
    pool.push_back(e);
  }
  const int i = next_event++;
  cudaEventRecord(pool[i], s);
  return i;
}

void KernelStats::drain() {
  for (const Rec& r : pending) {
    if (r.e0 < 0 || r.e1 < 0) continue;
    float ms_ = 0.f;
    if (cudaEventElapsedTime(&ms_, pool[r.e0], pool[r.e1]) == cudaSuccess) ms[r.cls] += ms_;
  }
  pending.clear();
  next_event = 0;
}

void KernelStats::release() {
  for (cudaEvent_t e : pool) cudaEventDestroy(e);
  pool.clear();
  pending.clear();
  next_event = 0;
}

extern "C" lrp_status lrp_plan_set_timing(lrp_plan_t p, int32_t enable) {
  if (!p) return set_error(LRP_EINVAL, "NULL plan");
  std::lock_guard<std::mutex> lock(p->mu);
  p->stats.timing = enable != 0;
  return LRP_OK;
}

extern "C" lrp_status lrp_plan_set_trace(lrp_plan_t p, int32_t enable) {
  if (!p) return set_error(LRP_EINVAL, "NULL plan");
  std::lock_guard<std::mutex> lock(p->mu);
  SetupGuard guard;
  const bool on = enable != 0;
  if (on && !p->trace_dev) {
    const size_t bytes = sizeof(double) * (size_t)p->dims.B * kTraceLen * kTraceWidth;
    if (cudaMalloc((void**)&p->trace_dev, bytes) != cudaSuccess) {
      p->trace_dev = nullptr;
      return set_error(LRP_ENOMEM, "trace allocation failed");
    }
    LRP_CUDA(cudaMemset(p->trace_dev, 0, bytes));
  }
  if (on != p->trace_on) {
    // captured iteration graphs hold the kernel parameters, trace pointer included
    p->w64.release_graphs();
    p->w32.release_graphs();
  }
  p->trace_on = on;
  return LRP_OK;
}

extern "C" lrp_status lrp_plan_trace(lrp_plan_t p, int32_t slot, double* out, int32_t max_entries,
                                     int32_t* n_entries) {
  if (!p || !out || !n_entries) return set_error(LRP_EINVAL, "NULL argument");
  if (slot < 0 || slot >= p->dims.B || max_entries < 0) return set_error(LRP_EINVAL, "slot out of range");
  std::lock_guard<std::mutex> lock(p->mu);
  SetupGuard guard;
  *n_entries = 0;
  if (!p->trace_dev) return set_error(LRP_EINVAL, "tracing was never enabled on this plan");
  LRP_CUDA(cudaDeviceSynchronize());
  SolveState h;
  LRP_CUDA(cudaMemcpy(&h, p->st + slot, sizeof(h), cudaMemcpyDeviceToHost));
  int cnt = h.total_iters < kTraceLen ? h.total_iters : kTraceLen;
  if (cnt > max_entries) cnt = max_entries;
  if (cnt > 0)
    LRP_CUDA(cudaMemcpy(out, p->trace_dev + (size_t)slot * kTraceLen * kTraceWidth,
                        sizeof(double) * kTraceWidth * cnt, cudaMemcpyDeviceToHost));
  *n_entries = cnt;
  return LRP_OK;
}

extern "C" lrp_status lrp_plan_kernel_stats(lrp_plan_t p, int32_t kclass, int64_t* launches, double* total_ms) {
  if (!p || !launches || !total_ms) return set_error(LRP_EINVAL, "NULL argument");
  if (kclass < -1 || kclass >= LRP_K_COUNT) return set_error(LRP_EINVAL, "kernel class out of range");
  std::lock_guard<std::mutex> lock(p->mu);
  SetupGuard guard;
  if (cudaDeviceSynchronize() != cudaSuccess) return set_error(LRP_ECUDA, "synchronize failed");
  p->stats.drain();
  int64_t l = 0;
  double t = 0.0;
  for (int c = 0; c < LRP_K_COUNT; ++c)
    if (kclass < 0 || c == kclass) {
      l += p->stats.launches[c];
      t += p->stats.ms[c];
    }
  *launches = l;
  *total_ms = t;
  return LRP_OK;
}

extern "C" lrp_status lrp_plan_kernel_work(lrp_plan_t p, int32_t kclass, double* flops, double* bytes) {
  if (!p || !flops || !bytes) return set_error(LRP_EINVAL, "NULL argument");
  if (kclass < -1 || kclass >= LRP_K_COUNT) return set_error(LRP_EINVAL, "kernel class out of range");
  std::lock_guard<std::mutex> lock(p->mu);
  SetupGuard guard;
  std::vector<double> h((size_t)p->dims.B * 2 * LRP_K_COUNT);
  LRP_CUDA(cudaDeviceSynchronize());
  LRP_CUDA(cudaMemcpy(h.data(), p->acct, sizeof(double) * h.size(), cudaMemcpyDeviceToHost));
  double f = 0.0, b = 0.0;
  for (int s = 0; s < p->dims.B; ++s)
    for (int c = 0; c < LRP_K_COUNT; ++c)
      if (kclass < 0 || c == kclass) {
        f += h[((size_t)s * LRP_K_COUNT + c) * 2];
        b += h[((size_t)s * LRP_K_COUNT + c) * 2 + 1];
      }
  *flops = f;
  *bytes = b;
  return LRP_OK;
}

extern "C" lrp_status lrp_plan_reset_stats(lrp_plan_t p) {
  if (!p) return set_error(LRP_EINVAL, "NULL plan");
  std::lock_guard<std::mutex> lock(p->mu);
  SetupGuard guard;
  cudaDeviceSynchronize();
  cudaMemset(p->acct, 0, sizeof(double) * (size_t)p->dims.B * 2 * LRP_K_COUNT);
  p->stats.drain();
  for (int c = 0; c < LRP_K_COUNT; ++c) {
    p->stats.launches[c] = 0;
    p->stats.ms[c] = 0.0;
  }
  return LRP_OK;
}

// ------------------------------------------------------------------- arena

void* DeviceArena::raw(size_t bytes) {
  if (failed) return nullptr;
  bytes = (bytes + 255) & ~(size_t)255;
  if (measure) {
    // sizing pass: count the bytes, hand out a placeholder that is never used
    total += bytes;
    return reinterpret_cast<void*>((uintptr_t)256);
  }
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    failed = true;
    cudaGetLastError();
    return nullptr;
  }
  cudaMemset(p, 0, bytes);
  blocks.push_back(p);
  total += bytes;
  return p;
}

void DeviceArena::release() {
  for (void* p : blocks) cudaFree(p);
  blocks.clear();
  total = 0;
}

// ------------------------------------------------------------------- plan

static bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

// Bytes of one region of a plan's pinned forward-DST staging (see forward_stage_host).
static size_t forward_stage_bytes(const PlanDims& d) { return (sizeof(void*) * 2 + sizeof(int64_t) * 2) * 2 * d.B; }

// Kernel attributes (dynamic shared-memory limits) are set once per device,
// never during a stream capture.
static lrp_status ensure_configured(int device) {
  static std::mutex cfg_mu;
  static uint64_t configured = 0;
  std::lock_guard<std::mutex> lock(cfg_mu);
  if (device >= 0 && device < 64 && (configured & (1ull << device))) return LRP_OK;
  cudaError_t e = dst_configure();
  if (e == cudaSuccess) e = core_configure();
  if (e == cudaSuccess) e = refine_configure();
  if (e == cudaSuccess) e = tall_configure();
  if (e != cudaSuccess) return set_error(LRP_ECUDA, std::string("kernel configuration: ") + cudaGetErrorString(e));
  if (device >= 0 && device < 64) configured |= (1ull << device);
  return LRP_OK;
}

extern "C" lrp_status lrp_default_opts(lrp_opts* o) {
  if (!o) return set_error(LRP_EINVAL, "opts is NULL");
  o->precision = LRP_FP64;
  o->selector = LRP_SEL_BERNOULLI;
  o->sample_factor = 1.0;
  o->matrix = LRP_MAT_POISSON;
  o->loop_on_device = 0;
  o->max_iter = 30;
  o->refine_steps = 2;
  o->max_rhs_rank = 64;
  o->batch = 1;
  o->m_cap = 0;
  o->check_every = 1;
  o->seed = 0;
  o->gemm_rows_per_thread = 0;
  o->dst_cta_threads = 0;
  return LRP_OK;
}

// Validated options and every size of the plan (no device work).
static lrp_status plan_setup_host(lrp_plan_s* p, int64_t n, double tol, int32_t max_rank, const lrp_opts* opts) {
  lrp_opts o;
  lrp_default_opts(&o);
  if (opts) o = *opts;
  const bool poisson = o.matrix == LRP_MAT_POISSON;
  if (n < 1 || (poisson && !is_pow2(n + 1))) return set_error(LRP_EINVAL, "n+1 must be a power of two >= 2");
  if (!poisson && n > (1 << 24)) return set_error(LRP_EINVAL, "n must be at most 2^24 for the test matrices");
  if (!(tol > 0.0) || !(tol < 1.0)) return set_error(LRP_EINVAL, "tol must be in (0, 1)");
  if (max_rank < 1) return set_error(LRP_EINVAL, "max_rank must be >= 1");
  if (o.max_iter < 1 || o.max_iter > 1000) return set_error(LRP_EINVAL, "max_iter out of range");
  if (o.max_rhs_rank < 1 || o.max_rhs_rank > kMaxRF) return set_error(LRP_EINVAL, "max_rhs_rank out of range");
  if (o.batch < 1 || o.batch > 65535) return set_error(LRP_EINVAL, "batch out of range");
  if (o.precision != LRP_FP64 && o.precision != LRP_MIXED) return set_error(LRP_EINVAL, "unknown precision");
  if (o.selector != LRP_SEL_LEVERAGE && o.selector != LRP_SEL_QDEIM && o.selector != LRP_SEL_BERNOULLI)
    return set_error(LRP_EINVAL, "unknown selector");
  if (!(o.sample_factor > 0.0) || !(o.sample_factor < 1e300)) return set_error(LRP_EINVAL, "sample_factor must be > 0");
  if (o.matrix != LRP_MAT_POISSON && o.matrix != LRP_MAT_HILBERT && o.matrix != LRP_MAT_K)
    return set_error(LRP_EINVAL, "unknown matrix");
  if (o.matrix != LRP_MAT_POISSON && o.precision != LRP_FP64)
    return set_error(LRP_EINVAL, "the test matrices are solved in FP64 only");
  if (o.matrix == LRP_MAT_K && n < 2) return set_error(LRP_EINVAL, "the K matrix needs n >= 2");
  if (o.check_every < 1) o.check_every = 1;
  if (o.loop_on_device != 0 && o.loop_on_device != 1) return set_error(LRP_EINVAL, "loop_on_device must be 0 or 1");
  if (o.gemm_rows_per_thread < 0 || o.gemm_rows_per_thread > 2)
    return set_error(LRP_EINVAL, "gemm_rows_per_thread must be 0, 1 or 2");
  if (o.dst_cta_threads != 0 && o.dst_cta_threads != 256 && o.dst_cta_threads != 512 && o.dst_cta_threads != 1024)
    return set_error(LRP_EINVAL, "dst_cta_threads must be 0, 256, 512 or 1024");
  const bool fp64 = (o.precision == LRP_FP64);
  if (poisson && !dst_supported(n)) return set_error(LRP_EINVAL, "n+1 must be at most 2^21");
  if (!fp64 && (o.refine_steps < 0 || o.refine_steps > 2))
    return set_error(LRP_EINVAL, "refine_steps must be 0, 1 or 2");
  p->n = n;
  p->tol = tol;
  p->mixed_inner_tol = 1e-4;
  p->mixed_redundancy = 1e-6;
  p->mixed_residual_tol = 1e-7;
  p->r_max = max_rank;
  p->opts = o;
  p->device_loop = o.loop_on_device != 0;
  PlanDims& d = p->dims;
  d.n = (int)n;
  d.ld = (n + 31) / 32 * 32;
  d.B = o.batch;
  d.RF = o.max_rhs_rank;
  int M = o.m_cap > 0 ? o.m_cap : 2 * max_rank + o.max_rhs_rank;
  if (M > kMaxM) M = kMaxM;
  if (M < o.max_rhs_rank) M = o.max_rhs_rank;  // the initial bases have r_f columns
  if (M < 2) M = 2;
  d.M = M;
  // Gram partial blocks: at least 512 rows each, at most 64 blocks.
  d.NB = (int)((n + 511) / 512);
  if (d.NB > 64) d.NB = 64;
  if (d.NB < 1) d.NB = 1;
  d.rows_per_block = (int)(((n + d.NB - 1) / d.NB + 31) / 32 * 32);
  d.NB = (int)((n + d.rows_per_block - 1) / d.rows_per_block);
  // Leverage candidate blocks: 1024 .. 8192 rows (sorted in shared memory), at
  // most ~128 blocks; k_select merges their top-c lists in bounded chunks.
  {
    int64_t rows = 1024;
    while (rows < 8192 && rows * 128 < n) rows <<= 1;
    d.cand_blocks = (int)((n + rows - 1) / rows);
  }
  d.cand_per_block = M;
  d.qdeim_rows = 1024;
  d.qdeim_chunks = (o.selector == LRP_SEL_QDEIM) ? (int)((n + d.qdeim_rows - 1) / d.qdeim_rows) : 0;
  if (!fp64 && d.M < d.RF + 2) return set_error(LRP_EINVAL, "mixed precision needs m_cap >= max_rhs_rank + 2");
  return LRP_OK;
}

// Every arena allocation of the plan, in one fixed order (also run as a
// sizing pass by lrp_plan_estimate_bytes).
static lrp_status plan_layout(lrp_plan_s* p) {
  const PlanDims& d = p->dims;
  const bool fp64 = (p->opts.precision == LRP_FP64);
  const int64_t n = p->n;
  const int max_rank = p->r_max;
  lrp_status s = LRP_OK;
  p->st = p->arena.get<SolveState>((size_t)d.B);
  p->lam64 = p->arena.get<double>((size_t)d.n);
  p->lam32 = p->arena.get<float>((size_t)d.n);
  p->prob_dev = p->arena.get<ProblemDev>((size_t)d.B);
  p->active_dev = p->arena.get<int32_t>(4);
  p->act_list = p->arena.get<int32_t>((size_t)d.B);
  p->acct = p->arena.get<double>((size_t)d.B * 2 * LRP_K_COUNT);
  p->dvec = p->arena.get<double>((size_t)d.B * d.M);
  if (p->opts.matrix == LRP_MAT_POISSON) {
    const size_t per_col = dst_temp_bytes(n, true);
    const int maxc = max_rank < d.M ? max_rank : d.M;
    const int cols = d.RF > maxc ? d.RF : maxc;
    p->dst_temp_bytes = per_col * (size_t)cols * d.B * 2;
    if (p->dst_temp_bytes) p->dst_temp = p->arena.get<unsigned char>(p->dst_temp_bytes);
  }
  p->s0 = p->arena.get<double>((size_t)d.B * d.M);
  p->loop_trips = p->arena.get<int32_t>(4);
  if (!p->arena.ok()) s = set_error(LRP_ENOMEM, "plan allocation failed");
  if (s == LRP_OK) s = p->w64.allocate(d, p->arena, d.RF);
  // the FP32 workspace also holds the recompressed residual (up to m_cap columns)
  if (s == LRP_OK && !fp64) s = p->w32.allocate(d, p->arena, d.RF > d.M ? d.RF : d.M);
  return s;
}

extern "C" lrp_status lrp_plan_estimate_bytes(int64_t n, double tol, int32_t max_rank, const lrp_opts* opts,
                                              size_t* bytes) {
  if (!bytes) return set_error(LRP_EINVAL, "bytes is NULL");
  *bytes = 0;
  lrp_plan_s* p = new (std::nothrow) lrp_plan_s();
  if (!p) return set_error(LRP_ENOMEM, "host allocation failed");
  p->arena.measure = true;
  lrp_status s = plan_setup_host(p, n, tol, max_rank, opts);
  if (s == LRP_OK) s = plan_layout(p);
  if (s == LRP_OK) *bytes = p->arena.total;
  delete p;
  return s;
}

static void plan_free(lrp_plan_s* p);

extern "C" lrp_status lrp_plan(lrp_plan_t* out, int64_t n, double tol, int32_t max_rank, const lrp_opts* opts) {
  if (!out) return set_error(LRP_EINVAL, "out is NULL");
  *out = nullptr;
  lrp_plan_s* p = new (std::nothrow) lrp_plan_s();
  if (!p) return set_error(LRP_ENOMEM, "host allocation failed");
  lrp_status s = plan_setup_host(p, n, tol, max_rank, opts);
  if (s != LRP_OK) {
    delete p;
    return s;
  }
  const PlanDims& d = p->dims;
  SetupGuard guard;
  if (cudaGetDevice(&p->device) != cudaSuccess) {
    delete p;
    return set_error(LRP_ECUDA, "no CUDA device");
  }
  s = ensure_configured(p->device);
  if (s != LRP_OK) {
    delete p;
    return s;
  }
  cudaStream_t st0 = nullptr;
  s = plan_layout(p);
  if (s == LRP_OK && p->opts.matrix == LRP_MAT_POISSON) {
    p->tw64 = dst_make_twiddles(n + 1, true, st0);
    p->tw32 = dst_make_twiddles(n + 1, false, st0);
    if (p->opts.precision == LRP_MIXED) p->twdf = dst_make_twiddles_df(n + 1, st0);
    if (!p->tw64 || !p->tw32 || (p->opts.precision == LRP_MIXED && !p->twdf))
      s = set_error(LRP_ENOMEM, "twiddle allocation failed");
  }
  if (s == LRP_OK) {
    cudaError_t e = launch_eigenvalues(d.n, p->lam64, p->lam32, st0);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&p->prob_host, sizeof(ProblemDev) * d.B);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&p->host_ptrs, forward_stage_bytes(d) * 2);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&p->active_host, sizeof(int32_t) * 4);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&p->prob_host_dev, p->prob_host, 0);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer(&p->host_ptrs_dev, p->host_ptrs, 0);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&p->active_host_dev, p->active_host, 0);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess && p->device_loop) e = cudaStreamCreateWithFlags(&p->body_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess && p->device_loop) e = cudaStreamCreateWithFlags(&p->if_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess && p->device_loop) e = cudaEventCreateWithFlags(&p->solve_done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) s = set_error(LRP_ECUDA, std::string("plan setup: ") + cudaGetErrorString(e));
  }
  if (s != LRP_OK) {
    plan_free(p);
    return s;
  }
  *out = p;
  return LRP_OK;
}

extern "C" lrp_status lrp_warm_create(lrp_plan_t p, lrp_warm_t* out) {
  if (!p || !out) return set_error(LRP_EINVAL, "NULL argument");
  *out = nullptr;
  lrp_warm_s* w = new (std::nothrow) lrp_warm_s();
  if (!w) return set_error(LRP_ENOMEM, "host allocation failed");
  w->plan = p;
  const PlanDims& d = p->dims;
  SetupGuard guard;
  WarmDev h;
  memset(&h, 0, sizeof(h));
  h.ld = d.ld;
  w->dev = w->arena.get<WarmDev>(1);
  h.idx = w->arena.get<int32_t>((size_t)2 * d.M);
  h.U = w->arena.get<double>((size_t)2 * d.ld * d.M);
  if (!w->arena.ok()) {
    w->arena.release();
    delete w;
    return set_error(LRP_ENOMEM, "warm-start record allocation failed");
  }
  if (cudaMemcpy(w->dev, &h, sizeof(h), cudaMemcpyHostToDevice) != cudaSuccess) {
    w->arena.release();
    delete w;
    return set_error(LRP_ECUDA, "warm-start record initialisation failed");
  }
  *out = w;
  return LRP_OK;
}

extern "C" lrp_status lrp_warm_reset(lrp_warm_t w) {
  if (!w) return set_error(LRP_EINVAL, "NULL record");
  SetupGuard guard;
  int32_t zero = 0;
  LRP_CUDA(cudaMemcpy(&w->dev->valid, &zero, sizeof(zero), cudaMemcpyHostToDevice));
  return LRP_OK;
}

extern "C" lrp_status lrp_warm_destroy(lrp_warm_t w) {
  if (!w) return LRP_OK;
  SetupGuard guard;
  cudaDeviceSynchronize();
  w->arena.release();
  delete w;
  return LRP_OK;
}

// Frees everything a plan holds; the caller holds the setup mutex.
static void plan_free(lrp_plan_s* p) {
  cudaDeviceSynchronize();
  if (p->trace_dev) cudaFree(p->trace_dev);
  p->arena.release();
  if (p->tw64) cudaFree(p->tw64);
  if (p->tw32) cudaFree(p->tw32);
  if (p->twdf) cudaFree(p->twdf);
  if (p->prob_host) cudaFreeHost(p->prob_host);
  if (p->host_ptrs) cudaFreeHost(p->host_ptrs);
  if (p->active_host) cudaFreeHost(p->active_host);
  p->stats.release();
  p->w64.release_graphs();
  p->w32.release_graphs();
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  for (auto& g : p->solve_graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  if (p->body_stream) cudaStreamDestroy(p->body_stream);
  if (p->if_stream) cudaStreamDestroy(p->if_stream);
  if (p->solve_done) cudaEventDestroy(p->solve_done);
  delete p;
}

extern "C" lrp_status lrp_plan_destroy(lrp_plan_t p) {
  if (!p) return LRP_OK;
  SetupGuard guard;
  plan_free(p);
  return LRP_OK;
}

extern "C" lrp_status lrp_plan_workspace_bytes(lrp_plan_t p, size_t* bytes) {
  if (!p || !bytes) return set_error(LRP_EINVAL, "NULL argument");
  *bytes = p->arena.total;
  return LRP_OK;
}

// ------------------------------------------------------------------- solve

namespace lrp {

// Kernels launched by one tall GEMM / Gram call (narrow and wide variants).
// launches of one tall product: the thread-per-row kernel, and the register-
// tiled one when the index capacity allows wider products
template <typename T = float>
static inline int gemm_kernels(const lrp_plan_s* p) { return gemm_wide_possible<T>(p->dims.M) ? 2 : 1; }
static inline int gram_kernels(const lrp_plan_s*) { return 1; }
static inline int dst_kernels(const lrp_plan_s* p) { return dst_smem_supported(p->n, true) ? 1 : 2; }

template <typename T>
static CoreBufs<T> make_core_bufs(lrp_plan_s* p, Workspace<T>& w) {
  const PlanDims& d = p->dims;
  const int64_t MM = (int64_t)d.M * d.M;
  const int64_t nm = d.ld * d.M;
  CoreBufs<T> b;
  b.G = {w.G, MM, 2 * MM};
  b.Racc = {w.Racc, MM, 2 * MM};
  b.P = {w.P, MM, 2 * MM};
  b.Bf = {w.Bf, MM, 2 * MM};
  b.X = {w.X, MM, 2 * MM};
  b.GE = {w.GE, MM, 2 * MM};
  b.Q2 = {w.Q2, nm, 2 * nm};
  b.idx = {w.idx, d.M, 2 * (int64_t)d.M};
  b.sig = w.sig;
  b.scratch = w.scratch;
  b.scratch_stride = kCoreScratch * MM;
  b.cand_score = w.cand_score;
  b.cand_idx = w.cand_idx;
  b.prob = p->prob_dev;
  b.acct = p->acct;
  return b;
}

template <typename T>
static Strided<const T> cs(const T* base, int64_t side, int64_t slot) {
  return Strided<const T>{base, side, slot};
}

// One CholeskyQR pass chain: Gram of X -> chol(pass 0, shifted) -> Q1 = X P,
// Gram -> chol(1) -> Q2 = Q1 P, Gram -> chol(2).  Leaves P3 in w.P, Q2 in w.Q2.
template <typename T>
static lrp_status gram_reduce(lrp_plan_s* p, const TallGeom& g, Strided<const T> x, int sx, Strided<const T> y,
                              int sy, double* part, Strided<double> G, bool sym, cudaStream_t s, bool acc64 = true) {
  // FP32 data run on the FP32 pipe (FP32 or double-float accumulation)
  const int cls = (sizeof(T) == 8) ? LRP_K_GRAM : (acc64 ? LRP_K_GRAM_DF : LRP_K_GRAM_F32);
  LRP_LAUNCH(p, cls, gram_kernels(p), s, launch_gram<T>(g, p->st, x, sx, y, sy, part, G, sym, s, acc64));
  LRP_LAUNCH(p, LRP_K_REDUCE, 1, s, launch_reduce(g, p->st, sx, sy, part, G, sym, s));
  return LRP_OK;
}

// Shifted CholeskyQR with `passes` (1..3) passes; Q = B P with B = X (1 pass),
// Q1 (2 passes) or Q2 (3 passes) and P the inverse R of the last pass (w.P).
template <typename T>
static lrp_status cholqr(lrp_plan_s* p, Workspace<T>& w, const TallGeom& g, const CoreParams& cp,
                         const CoreBufs<T>& cb, const T* X, int64_t side_stride, int64_t slot_stride, int sel,
                         cudaStream_t s, int passes) {
  const PlanDims& d = p->dims;
  const int64_t MM = (int64_t)d.M * d.M;
  const int64_t nm = d.ld * d.M;
  Strided<double> G{w.G, MM, 2 * MM};
  Strided<const double> P{w.P, MM, 2 * MM};
  const Strided<const T> none{nullptr, 0, 0};
  lrp_status st;
  if ((st = gram_reduce<T>(p, g, cs(X, side_stride, slot_stride), sel, cs(X, side_stride, slot_stride), sel, w.part,
                           G, true, s)))
    return st;
  LRP_LAUNCH(p, LRP_K_CHOL, 1, s, launch_chol<T>(cp, cb, sel, 0, s));
  if (passes < 2) return LRP_OK;
  LRP_LAUNCH(p, gemm_class<T>(), gemm_kernels<T>(p), s,
             launch_gemm_nn<T>(g, p->st, cs(X, side_stride, slot_stride), sel, P, sel, Strided<T>{w.Q1, nm, 2 * nm},
                               none, 0, s));
  // Later passes see a well-conditioned basis: FP32 data keep an FP32 Gram.
  const bool acc64 = sizeof(T) == 8;
  if ((st = gram_reduce<T>(p, g, cs<T>(w.Q1, nm, 2 * nm), sel, cs<T>(w.Q1, nm, 2 * nm), sel, w.part, G, true, s,
                           acc64)))
    return st;
  LRP_LAUNCH(p, LRP_K_CHOL, 1, s, launch_chol<T>(cp, cb, sel, 1, s));
  if (passes < 3) return LRP_OK;
  LRP_LAUNCH(p, gemm_class<T>(), gemm_kernels<T>(p), s,
             launch_gemm_nn<T>(g, p->st, cs<T>(w.Q1, nm, 2 * nm), sel, P, sel, Strided<T>{w.Q2, nm, 2 * nm}, none, 0,
                               s));
  if ((st = gram_reduce<T>(p, g, cs<T>(w.Q2, nm, 2 * nm), sel, cs<T>(w.Q2, nm, 2 * nm), sel, w.part, G, true, s,
                           acc64)))
    return st;
  LRP_LAUNCH(p, LRP_K_CHOL, 1, s, launch_chol<T>(cp, cb, sel, 2, s));
  return LRP_OK;
}

template <typename T>
static lrp_status cholqr3(lrp_plan_s* p, Workspace<T>& w, const TallGeom& g, const CoreParams& cp,
                          const CoreBufs<T>& cb, const T* X, int64_t side_stride, int64_t slot_stride, int sel,
                          cudaStream_t s) {
  return cholqr<T>(p, w, g, cp, cb, X, side_stride, slot_stride, sel, s, 3);
}

template <typename T>
static CoreParams make_core_params(lrp_plan_s* p, int count, double tol, double eps_data, double redundancy) {
  const PlanDims& d = p->dims;
  CoreParams cp;
  cp.g = TallGeom{d.n, d.ld, d.M, count, d.NB, d.rows_per_block};
  cp.g.gemm_rpt = p->opts.gemm_rows_per_thread;
  cp.st = p->st;
  cp.max_iter = p->opts.max_iter;
  cp.r_max = p->r_max;
  cp.tol = tol;
  cp.eps_data = eps_data;
  cp.shift_rel = 1e-15;
  cp.drop_rel = 64.0 * 2.220446049250313e-16;
  cp.redundancy = redundancy;
  cp.noise_floor_stop = 0;
  cp.dst_df = 0;
  cp.seed = p->opts.seed;
  cp.selector = p->opts.selector;
  cp.sample_factor = p->opts.sample_factor;
  cp.cand_blocks = d.cand_blocks;
  cp.cand_per_block = d.cand_per_block;
  cp.trace = p->trace_on ? p->trace_dev : nullptr;
  return cp;
}

// Pinned staging of one forward DST job: input/output pointers and leading
// dimensions of both factors of every slot.  Region 0 serves the iteration
// precision's transform, region 1 the mixed path's FP64 transform, so that a
// captured solve reads both from distinct host memory.

template <typename T>
static void forward_stage_host(lrp_plan_s* p, Workspace<T>& w, int count, int region) {
  const PlanDims& d = p->dims;
  const int64_t fm = d.ld * w.rf_cap;
  const double** hin = (const double**)((char*)p->host_ptrs + region * forward_stage_bytes(d));
  T** hout = (T**)(hin + 2 * d.B);
  int64_t* hldi = (int64_t*)(hout + 2 * d.B);
  int64_t* hldo = hldi + 2 * d.B;
  for (int mat = 0; mat < 2; ++mat)
    for (int sl = 0; sl < count; ++sl) {
      const ProblemDev& pr = p->prob_host[sl];
      hin[mat * count + sl] = mat == 0 ? pr.U_f : pr.V_f;
      hldi[mat * count + sl] = mat == 0 ? pr.ldu_f : pr.ldv_f;
      hout[mat * count + sl] = w.Fh + (int64_t)sl * 2 * fm + (int64_t)mat * fm;
      hldo[mat * count + sl] = d.ld;
    }
}

// Forward DST of the caller's factors into w.Fh (type T); with do_setup the
// per-slot state and the h^2-scaled weights are initialised too.
template <typename T>
static lrp_status phase_forward(lrp_plan_s* p, Workspace<T>& w, const CoreParams& cp, int count, bool do_setup, bool df,
                                cudaStream_t s, int region) {
  const PlanDims& d = p->dims;
  const double** hin = (const double**)((char*)p->host_ptrs + region * forward_stage_bytes(d));
  T** hout = (T**)(hin + 2 * d.B);
  int64_t* hldi = (int64_t*)(hout + 2 * d.B);
  int64_t* hldo = hldi + 2 * d.B;
  if (!p->capturing_solve) {
    // The pinned staging is reused by the next solve: wait for earlier copies from it.
    LRP_CUDA(cudaStreamSynchronize(s));
    forward_stage_host<T>(p, w, count, region);
  }
  // the device alias of a host staging address
  auto dev = [&](const void* h) {
    return static_cast<const void*>(static_cast<const char*>(p->host_ptrs_dev) +
                                    (static_cast<const char*>(h) - static_cast<const char*>(p->host_ptrs)));
  };
  LRP_LAUNCH(p, LRP_K_OTHER, 1, s, launch_stage(dev(hin), w.fwd_in, sizeof(void*) * 2 * count, s));
  LRP_LAUNCH(p, LRP_K_OTHER, 1, s, launch_stage(dev(hout), w.fwd_out, sizeof(void*) * 2 * count, s));
  LRP_LAUNCH(p, LRP_K_OTHER, 1, s, launch_stage(dev(hldi), w.fwd_ldi, sizeof(int64_t) * 2 * count, s));
  LRP_LAUNCH(p, LRP_K_OTHER, 1, s, launch_stage(dev(hldo), w.fwd_ldo, sizeof(int64_t) * 2 * count, s));
  if (do_setup)
    LRP_LAUNCH(p, LRP_K_OTHER, 1, s, launch_setup<T>(cp, p->prob_dev, w.w, w.rf_cap, count, p->acct, s));
  DstBatch<double, T> job;
  job.in = w.fwd_in;
  job.out = w.fwd_out;
  job.ld_in = w.fwd_ldi;
  job.ld_out = w.fwd_ldo;
  job.nslots = count;
  job.fixed_cols = 0;
  job.ncols_dev = &p->prob_dev[0].rf;
  job.ncols_stride = (int)(sizeof(ProblemDev) / sizeof(int32_t));
  job.ncols_mat_stride = 0;
  job.active_dev = nullptr;
  job.active_stride = 0;
  job.require_active = 0;
  if constexpr (sizeof(T) == 8) {
    if (p->opts.matrix != LRP_MAT_POISSON) {
      // a matrix given by entries: the initial guesses are used as they are
      LRP_LAUNCH(p, LRP_K_OTHER, 1, s, launch_copy_cols(job, d.n, d.RF, s));
      return LRP_OK;
    }
    if (df && p->twdf) {
      // FP64 data transformed in double-float arithmetic (mixed path)
      LRP_LAUNCH(p, LRP_K_DST_DF, dst_kernels(p), s,
                 (dst1_launch<double, double, dfloat>(d.n, job, d.RF, count, 2, p->twdf, s, p->dst_temp,
                                                      p->dst_temp_bytes, p->opts.dst_cta_threads)));
      return LRP_OK;
    }
  }
  const void* tw = (sizeof(T) == 8) ? p->tw64 : p->tw32;
  LRP_LAUNCH(p, LRP_K_DST, dst_kernels(p), s,
             (dst1_launch<double, T, T>(d.n, job, d.RF, count, 2, tw, s, p->dst_temp, p->dst_temp_bytes,
                                         p->opts.dst_cta_threads)));
  return LRP_OK;
}

// Row candidates for the next index-set enrichment from the current factors:
// leverage scores (Algorithm LeverageScores: top-c, the default, or Bernoulli
// sampling) or QDEIM pivots (Algorithm IS), all read by k_select.
template <typename T>
static lrp_status select_rows(lrp_plan_s* p, Workspace<T>& w, const TallGeom& g, Strided<const T> U, int sel,
                              cudaStream_t s) {
  const PlanDims& d = p->dims;
  if (p->opts.selector == LRP_SEL_QDEIM) {
    LRP_LAUNCH(p, LRP_K_LEVERAGE, 2 * d.M + 1, s,
               launch_qdeim<T>(g, p->st, U, sel, w.qd, w.cand_score, w.cand_idx, d.cand_blocks, d.cand_per_block,
                               d.M, s));
  } else {
    LevSample ls;
    if (p->opts.selector == LRP_SEL_BERNOULLI) {
      ls.on = 1;
      ls.k_ofs = (sel == kDimC0) ? 0 : 1;  // initial candidates: iteration 0
      ls.seed = p->opts.seed;
      ls.factor = p->opts.sample_factor;
    }
    LRP_LAUNCH(p, LRP_K_LEVERAGE, 1, s,
               launch_leverage<T>(g, p->st, U, sel, w.cand_score, w.cand_idx, d.cand_blocks, d.cand_per_block, s,
                                  ls));
  }
  return LRP_OK;
}

// Cross-DEIM (Algorithm Cross-DEIM) on the transformed right-hand side held in
// w.Fh / w.w: initial bases orth(Fh), then iterations until every slot stops.
// Runs `body` directly, or (when graphs are enabled and timing is off) replays
// a CUDA graph captured from it on first use for this batch count.
template <typename T, typename Body>
static lrp_status run_captured(lrp_plan_s* p, Workspace<T>& w, int count, int kind, int level, cudaStream_t s,
                               Body body) {
  if (!p->use_graphs || p->stats.timing || !p->cap_stream || p->capturing_solve) return body(s);
  if (w.graph_count != count) {
    SetupGuard guard;
    w.release_graphs();
    w.graph_count = count;
  }
  if (!w.graphs[kind][level]) {
    CaptureGuard capture;
    int64_t before[LRP_K_COUNT];
    for (int c = 0; c < LRP_K_COUNT; ++c) before[c] = p->stats.launches[c];
    // Captured on the plan's own stream (the caller's may be the legacy default
    // stream, which cannot be captured); the graph is launched on the caller's.
    LRP_CUDA(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal));
    lrp_status st = body(p->cap_stream);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(p->cap_stream, &graph);
    if (st != LRP_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (e != cudaSuccess) return set_error(LRP_ECUDA, std::string("stream capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&w.graphs[kind][level], graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      w.graphs[kind][level] = nullptr;
      return set_error(LRP_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    for (int c = 0; c < LRP_K_COUNT; ++c) {
      w.graph_launches[kind][level][c] = p->stats.launches[c] - before[c];
      p->stats.launches[c] = before[c];
    }
  }
  LRP_CUDA(cudaGraphLaunch(w.graphs[kind][level], s));
  for (int c = 0; c < LRP_K_COUNT; ++c) p->stats.launches[c] += w.graph_launches[kind][level][c];
  return LRP_OK;
}

// Cross-DEIM (Algorithm Cross-DEIM) on the transformed right-hand side held in
// w.Fh / w.w: initial bases orth(Fh), then iterations until every slot stops.
template <typename T>
static lrp_status phase_iterate(lrp_plan_s* p, Workspace<T>& w, const CoreParams& cp, int count, cudaStream_t s) {
  const PlanDims& d = p->dims;
  const int64_t MM = (int64_t)d.M * d.M;
  const int64_t nm = d.ld * d.M;
  const int64_t fm = d.ld * w.rf_cap;
  const TallGeom& g = cp.g;
  CoreBufs<T> cb = make_core_bufs<T>(p, w);
  const Strided<const T> none{nullptr, 0, 0};
  // U_{-1} = orth(Uhat_f), V_{-1} = orth(Vhat_f) and their leverage candidates.
  auto init = [&](cudaStream_t s) -> lrp_status {
    lrp_status st = cholqr3<T>(p, w, g, cp, cb, w.Fh, fm, 2 * fm, kDimRF, s);
    if (st) return st;
    LRP_LAUNCH(p, LRP_K_CHOL, 1, s, launch_orth_keep<T>(cp, cb, s));
    LRP_LAUNCH(p, gemm_class<T>(), gemm_kernels<T>(p), s,
               launch_gemm_nn<T>(g, p->st, cs<T>(w.Q2, nm, 2 * nm), kDimRF, Strided<const double>{w.P, MM, 2 * MM},
                                 kDimC0, Strided<T>{w.U[1], nm, 2 * nm}, none, 0, s));
    // Warm-started slots replace U_{-1}, V_{-1} and the index sets with their record.
    LRP_LAUNCH(p, LRP_K_OTHER, 1, s, launch_warm_load<T>(cp, cb, Strided<T>{w.U[1], nm, 2 * nm}, s));
    lrp_status sr = select_rows<T>(p, w, g, cs<T>(w.U[1], nm, 2 * nm), kDimC0, s);
    if (sr) return sr;
    // launch list of the first iteration
    LRP_LAUNCH(p, LRP_K_OTHER, 1, s, launch_count_active(p->st, count, p->active_dev, p->act_list, s));
    return LRP_OK;
  };
  lrp_status st0 = run_captured<T>(p, w, count, 3, 0, s, init);
  if (st0) return st0;
  Strided<double> Gx{w.X, MM, 2 * MM};
  Strided<double> Ge{w.GE, MM, 2 * MM};
  CrossArgs<T> ca;
  ca.F = {w.Fh, fm, 2 * fm};
  ca.w = w.w;
  ca.wstride = w.rf_cap;
  ca.lam = (sizeof(T) == 8) ? (const T*)p->lam64 : (const T*)p->lam32;
  ca.idx = {w.idx, d.M, 2 * (int64_t)d.M};
  ca.A = {w.A, nm, 2 * nm};
  // Each iteration launches over the compacted list of the slots still active
  // (k_count_active), in a bucket of the whole batch (level 0) or 2^(level-1)
  // entries, chosen from the count the host reads back.
  auto iteration = [&](int k, int level, cudaStream_t s) -> lrp_status {
    const int par = k & 1;
    CoreParams cpi = cp;
    cpi.g.act = p->act_list;
    cpi.g.nslots = level == 0 ? count : (1 << (level - 1));
    const TallGeom& gi = cpi.g;
    LRP_LAUNCH(p, LRP_K_SELECT, 1, s, launch_select<T>(cpi, cb, k == 0 ? kDimC0 : kDimR, s));
    if constexpr (sizeof(T) == 8) {
      if (p->opts.matrix != LRP_MAT_POISSON) {
        LRP_LAUNCH(p, LRP_K_CROSS, 1, s,
                   launch_cross_matrix(gi, p->st, p->opts.matrix, Strided<double>{(double*)w.A, nm, 2 * nm},
                                       Strided<const int32_t>{w.idx, d.M, 2 * (int64_t)d.M}, s));
      } else {
        LRP_LAUNCH(p, LRP_K_CROSS, 1, s, launch_cross<T>(gi, p->st, ca, s));
      }
    } else {
      LRP_LAUNCH(p, LRP_K_CROSS, 1, s, launch_cross<T>(gi, p->st, ca, s));
    }
    lrp_status st = cholqr3<T>(p, w, gi, cpi, cb, w.A, nm, 2 * nm, kDimOther, s);
    if (st) return st;
    LRP_LAUNCH(p, LRP_K_CORE, 1, s, launch_core<T>(cpi, cb, par, s));
    LRP_LAUNCH(p, gemm_class<T>(), gemm_kernels<T>(p), s,
               launch_gemm_nn<T>(gi, p->st, cs<T>(w.Q2, nm, 2 * nm), kDimOther,
                                 Strided<const double>{w.Bf, MM, 2 * MM}, kDimR, Strided<T>{w.U[par], nm, 2 * nm},
                                 none, 0, s));
    st = select_rows<T>(p, w, gi, cs<T>(w.U[par], nm, 2 * nm), kDimR, s);
    if (st) return st;
    if (k > 0) {
      // X = U_k^T U_{k-1}; E = U_{k-1} - U_k X; GE = E^T E  (terms of rho)
      st = gram_reduce<T>(p, gi, cs<T>(w.U[par], nm, 2 * nm), kDimR, cs<T>(w.U[1 - par], nm, 2 * nm), kDimRPrev,
                          w.part, Gx, false, s, sizeof(T) == 8);
      if (st) return st;
      LRP_LAUNCH(p, gemm_class<T>(), gemm_kernels<T>(p), s,
                 launch_gemm_nn<T>(gi, p->st, cs<T>(w.U[par], nm, 2 * nm), kDimR,
                                   Strided<const double>{w.X, MM, 2 * MM}, kDimRPrev,
                                   Strided<T>{w.Q1, nm, 2 * nm}, cs<T>(w.U[1 - par], nm, 2 * nm), 1, s));
      st = gram_reduce<T>(p, gi, cs<T>(w.Q1, nm, 2 * nm), kDimRPrev, cs<T>(w.Q1, nm, 2 * nm), kDimRPrev, w.part,
                          Ge, true, s, sizeof(T) == 8);
      if (st) return st;
    }
    LRP_LAUNCH(p, LRP_K_STOP, 1, s, launch_stop<T>(cpi, cb, par, s));
    LRP_LAUNCH(p, LRP_K_OTHER, 1, s, launch_count_active(p->st, count, p->active_dev, p->act_list, s));
    return LRP_OK;
  };
  if (p->capturing_solve) {
    // The loop runs on the device: iteration 0, then a conditional while-node
    // whose body is one odd and one even iteration (the kernels' parity is fixed
    // at capture); k_loop_next continues it while a problem is active.  Slots
    // that finish within a trip are skipped by every later kernel (their act
    // list entries are -1), and k_stop ends every slot at max_iter.
    lrp_status st = iteration(0, 0, s);
    if (st) return st;
    if (p->opts.max_iter < 2) return LRP_OK;
    const int max_trips = p->opts.max_iter / 2 + 1;
    cudaStreamCaptureStatus cst;
    cudaGraph_t graph = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    LRP_CUDA(cudaStreamGetCaptureInfo(s, &cst, nullptr, &graph, &deps, nullptr, &ndeps));
    cudaGraphConditionalHandle h;
    LRP_CUDA(cudaGraphConditionalHandleCreate(&h, graph, 0, 0));
    LRP_LAUNCH(p, LRP_K_OTHER, 1, s, launch_loop_begin(p->active_dev, p->loop_trips, h, s));
    LRP_CUDA(cudaStreamGetCaptureInfo(s, &cst, nullptr, &graph, &deps, nullptr, &ndeps));
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    LRP_CUDA(cudaGraphAddNode(&node, graph, deps, nullptr, ndeps, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    LRP_CUDA(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    LRP_CUDA(cudaStreamBeginCaptureToGraph(p->body_stream, body, nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal));
    st = iteration(1, 0, p->body_stream);
    if (st == LRP_OK) st = iteration(2, 0, p->body_stream);
    if (st == LRP_OK) {
      cudaError_t e = launch_loop_next(p->active_dev, p->loop_trips, max_trips, h, p->body_stream);
      if (e != cudaSuccess) st = set_error(LRP_ECUDA, std::string("loop control: ") + cudaGetErrorString(e));
    }
    cudaGraph_t captured = nullptr;
    cudaError_t e = cudaStreamEndCapture(p->body_stream, &captured);
    if (st) return st;
    if (e != cudaSuccess) return set_error(LRP_ECUDA, std::string("loop body capture: ") + cudaGetErrorString(e));
    return LRP_OK;
  }
  int level = 0;
  for (int k = 0; k < p->opts.max_iter; ++k) {
    const int kind = (k == 0) ? 0 : ((k & 1) ? 1 : 2);
    lrp_status st = run_captured<T>(p, w, count, kind, level, s,
                                    [&](cudaStream_t cs_) { return iteration(k, level, cs_); });
    if (st) return st;
    if ((k + 1) % p->opts.check_every == 0 || k + 1 == p->opts.max_iter) {
      LRP_LAUNCH(p, LRP_K_OTHER, 1, s, launch_stage(p->active_dev, p->active_host_dev, sizeof(int32_t), s));
      LRP_CUDA(cudaStreamSynchronize(s));
      const int na = *static_cast<volatile int32_t*>(p->active_host);
      if (na == 0) break;
      int b = 1, l = 1;
      while (b < na) {
        b <<= 1;
        ++l;
      }
      level = (b >= count || l >= kGraphLevels) ? 0 : l;
    }
  }
  return LRP_OK;
}

// Final truncation, singular values, info, then W factors = DST of the first r columns.
template <typename T>
static lrp_status phase_finalize(lrp_plan_s* p, Workspace<T>& w, const CoreParams& cp, int count, cudaStream_t s,
                                 bool df = false) {
  const PlanDims& d = p->dims;
  const int64_t nm = d.ld * d.M;
  CoreBufs<T> cb = make_core_bufs<T>(p, w);
  DstBatch<T, double> back;
  back.in = w.back_in;
  back.out = w.back_out;
  back.ld_in = w.back_ldi;
  back.ld_out = w.back_ldo;
  back.nslots = count;
  back.fixed_cols = 0;
  back.ncols_dev = &p->st[0].r_out;
  back.ncols_stride = (int)(sizeof(SolveState) / sizeof(int32_t));
  back.ncols_mat_stride = 0;
  back.active_dev = nullptr;
  back.active_stride = 0;
  back.require_active = 0;
  LRP_LAUNCH(p, LRP_K_OTHER, 1, s, launch_finalize_impl<T>(cp, cb, back, w.ubufs, nm, 2 * nm, s));
  const int maxc = p->r_max < d.M ? p->r_max : d.M;
  if constexpr (sizeof(T) == 8) {
    if (p->opts.matrix != LRP_MAT_POISSON) {
      LRP_LAUNCH(p, LRP_K_OTHER, 1, s, launch_copy_cols(back, d.n, maxc, s));
      return LRP_OK;
    }
    if (df && p->twdf) {
      LRP_LAUNCH(p, LRP_K_DST_DF, dst_kernels(p), s,
                 (dst1_launch<double, double, dfloat>(d.n, back, maxc, count, 2, p->twdf, s, p->dst_temp,
                                                      p->dst_temp_bytes, p->opts.dst_cta_threads)));
      return LRP_OK;
    }
  }
  const void* tw = (sizeof(T) == 8) ? p->tw64 : p->tw32;
  LRP_LAUNCH(p, LRP_K_DST, dst_kernels(p), s,
             (dst1_launch<T, double, T>(d.n, back, maxc, count, 2, tw, s, p->dst_temp, p->dst_temp_bytes,
                                         p->opts.dst_cta_threads)));
  return LRP_OK;
}

template <typename T>
static lrp_status warm_store(lrp_plan_s* p, Workspace<T>& w, const CoreParams& cp, cudaStream_t s) {
  if (!p->any_warm) return LRP_OK;
  const int64_t nm = p->dims.ld * p->dims.M;
  CoreBufs<T> cb = make_core_bufs<T>(p, w);
  LRP_LAUNCH(p, LRP_K_OTHER, 1, s, launch_warm_store<T>(cp, cb, w.ubufs, nm, 2 * nm, s));
  return LRP_OK;
}

static lrp_status run_fp64(lrp_plan_s* p, int count, cudaStream_t s) {
  CoreParams cp = make_core_params<double>(p, count, p->tol, 2.220446049250313e-16, 1e-12);
  lrp_status st;
  if ((st = phase_forward<double>(p, p->w64, cp, count, true, false, s, 0))) return st;
  if ((st = phase_iterate<double>(p, p->w64, cp, count, s))) return st;
  if ((st = warm_store<double>(p, p->w64, cp, s))) return st;
  return phase_finalize<double>(p, p->w64, cp, count, s);
}

static RefineArgs make_refine_args(lrp_plan_s* p) {
  const PlanDims& d = p->dims;
  const int64_t MM = (int64_t)d.M * d.M;
  const int64_t nm = d.ld * d.M;
  const int64_t fm = d.ld * d.RF;
  RefineArgs a;
  a.n = d.n;
  a.ld = d.ld;
  a.M = d.M;
  a.st = p->st;
  a.prob = p->prob_dev;
  a.lam = p->lam64;
  a.Fh64 = {p->w64.Fh, fm, 2 * fm};
  a.U32[0] = {p->w32.U[0], nm, 2 * nm};
  a.U32[1] = {p->w32.U[1], nm, 2 * nm};
  a.X = {p->w64.A, nm, 2 * nm};
  a.stash = {p->w64.U[1], nm, 2 * nm};
  a.Racc = {p->w64.Racc, MM, 2 * MM};
  a.P = {p->w64.P, MM, 2 * MM};
  a.Bf = {p->w64.Bf, MM, 2 * MM};
  a.sig32 = p->w32.sig;
  a.dvec = p->dvec;
  a.s0 = p->s0;
  a.sig_out = p->w64.sig;
  a.sig_out_stride = 2 * (int64_t)d.M;
  a.scratch = p->w64.scratch;
  a.scratch_stride = kCoreScratch * MM;
  a.w32 = p->w32.w;
  a.wstride = p->w32.rf_cap;
  a.acct = p->acct;
  a.NB = d.NB;
  a.corr_tol = p->tol;
  a.final_tol = p->tol;
  a.X32 = {nullptr, 0, 0};
  a.X32lo = {nullptr, 0, 0};
  a.U64 = {nullptr, 0, 0};
  return a;
}

// Mixed precision: FP32 Cross-DEIM to tol_in, FP64 residual recompression, an
// FP32 correction solve, FP64 recompression of the sum, FP64 back transform.
static lrp_status run_mixed(lrp_plan_s* p, int count, cudaStream_t s) {
  const PlanDims& d = p->dims;
  const int64_t MM = (int64_t)d.M * d.M;
  const int64_t nm = d.ld * d.M;
  const int64_t fm32 = d.ld * p->w32.rf_cap;
  const double eps32 = 1.1920928955078125e-07;
  const double tol_in = p->tol > p->mixed_inner_tol ? p->tol : p->mixed_inner_tol;
  CoreParams c32 = make_core_params<float>(p, count, tol_in, eps32, p->mixed_redundancy);
  c32.noise_floor_stop = 1;
  // the first pass's Gram is double-float (relative error ~1e-13, at worst
  // ~5e-10): its shift dominates that error
  c32.shift_rel = 1e-12;
  // FP32 solves whose change between iterates stalls above tol_in (FP32 noise in
  // the index updates) stop after a bounded number of iterations; the FP64
  // residual step corrects what they leave.
  c32.max_iter = p->opts.max_iter < p->mixed_inner_max_iter ? p->opts.max_iter : p->mixed_inner_max_iter;
  CoreParams c64 = make_core_params<double>(p, count, p->tol, 2.220446049250313e-16, 1e-12);
  c64.dst_df = 1;
  CoreBufs<double> cb64 = make_core_bufs<double>(p, p->w64);
  RefineArgs ra = make_refine_args(p);
  // The correction dW enters the sum at its own size ||dW|| ~ ||W - W0||, so
  // it is done once its change is below tol ||W0|| in absolute terms (the stop
  // test then uses tol ||S0|| / ||S_k||); FP32 resolves no better than tol_in.
  ra.corr_tol = tol_in;
  ra.final_tol = p->tol;
  const TallGeom& g = c64.g;
  const Strided<const double> none{nullptr, 0, 0};
  lrp_status st;
  if ((st = phase_forward<float>(p, p->w32, c32, count, true, false, s, 0))) return st;
  // FP64 transform of the right-hand side for the residual, in double-float
  if (p->opts.refine_steps > 0 && (st = phase_forward<double>(p, p->w64, c64, count, false, true, s, 1))) return st;
  if ((st = phase_iterate<float>(p, p->w32, c32, count, s))) return st;
  if ((st = warm_store<float>(p, p->w32, c32, s))) return st;
  // Without refinement the FP32 solution is the result (truncated at tol_in).
  if (p->opts.refine_steps == 0) return phase_finalize<float>(p, p->w32, c32, count, s);
  const int rcap_res = p->w32.rf_cap < d.M ? p->w32.rf_cap : d.M;
  // Step 0 refines the FP32 trial; step 1 (refine_steps == 2) refines the FP64
  // result of step 0 for the problems whose first correction looks unreliable
  // (k_check_refine), the others held out of it.
  auto refine_step = [&](int step, cudaStream_t s) -> lrp_status {
    RefineArgs rstep = ra;
    if (step) rstep.U64 = {p->w64.U[0], nm, 2 * nm};
    // Residual of the trial solution, recompressed with FP64 accuracy.  One
    // shifted-Cholesky pass: the residual only needs the accuracy of the FP32
    // correction solve, and its cancellation happens in the FP64 core.
    if (d.M <= 64) {
      // Stacked blocks as double-float (hi, lo) planes, Grams and products on
      // the FP32 pipe.  The stacked blocks are numerically rank deficient (the
      // residual is small because [Uh_f, Lambda Uh0, Uh0] nearly share a
      // span), so the first pass's shift (above the double-float Gram's
      // ~1e-13 relative error) leaves Q1 = X R1^{-1} far from orthonormal; a
      // second pass makes the residual's factors orthonormal, which is what
      // the FP32 correction solve evaluates its cross entries from.
      RefineArgs rr = rstep;
      rr.X32 = {p->w32.Q1, nm, 2 * nm};
      rr.X32lo = {p->w32.Q2, nm, 2 * nm};
      CoreParams c64r = c64;
      c64r.shift_rel = 1e-12;
      Strided<double> G64{p->w64.G, MM, 2 * MM};
      const Strided<const float> xh{p->w32.Q1, nm, 2 * nm}, xl{p->w32.Q2, nm, 2 * nm};
      // Q1 planes: the trial's FP32 factors are stashed by the assembly, so
      // the iteration factor buffers are free until the correction solve.
      const Strided<float> q1h{p->w32.A, nm, 2 * nm}, q1l{p->w32.U[0], nm, 2 * nm};
      const Strided<float> noo{nullptr, 0, 0};
      const Strided<double> no64{nullptr, 0, 0};
      if (step)
        LRP_LAUNCH(p, LRP_K_REFINE, 1, s, launch_prepare_refine2(rr, count, s));
      else
        LRP_LAUNCH(p, LRP_K_REFINE, 1, s, launch_prepare_refine(rr, count, s));
      LRP_LAUNCH(p, LRP_K_REFINE, 1, s, launch_assemble_residual(rr, count, s));
      LRP_LAUNCH(p, LRP_K_GRAM_DF, 1, s, launch_gram_dd(g, p->st, xh, xl, kDimX, p->w64.part, s));
      LRP_LAUNCH(p, LRP_K_REDUCE, 1, s, launch_reduce(g, p->st, kDimX, kDimX, p->w64.part, G64, true, s));
      LRP_LAUNCH(p, LRP_K_CHOL, 1, s, launch_chol<double>(c64r, cb64, kDimX, 0, s));
      LRP_LAUNCH(p, LRP_K_GEMM_DF, 1, s,
                 launch_gemm_dfx(g, p->st, xh, xl, kDimX, Strided<const double>{p->w64.P, MM, 2 * MM}, kDimX, q1h,
                                 q1l, no64, s, true));
      LRP_LAUNCH(p, LRP_K_GRAM_DF, 1, s,
                 launch_gram_dd(g, p->st, Strided<const float>{p->w32.A, nm, 2 * nm},
                                Strided<const float>{p->w32.U[0], nm, 2 * nm}, kDimX, p->w64.part, s));
      LRP_LAUNCH(p, LRP_K_REDUCE, 1, s, launch_reduce(g, p->st, kDimX, kDimX, p->w64.part, G64, true, s));
      LRP_LAUNCH(p, LRP_K_CHOL, 1, s, launch_chol<double>(c64r, cb64, kDimX, 1, s));
      LRP_LAUNCH(p, LRP_K_REFINE, 1, s, launch_recompress(rr, count, 0, p->mixed_residual_tol, rcap_res, s));
      // The residual's factors, rounded to FP32, are the correction solve's
      // right-hand side.
      LRP_LAUNCH(p, LRP_K_GEMM_DF, 1, s,
                 launch_gemm_dfx(g, p->st, Strided<const float>{p->w32.A, nm, 2 * nm},
                                 Strided<const float>{p->w32.U[0], nm, 2 * nm}, kDimX,
                                 Strided<const double>{p->w64.Bf, MM, 2 * MM}, kDimR,
                                 Strided<float>{p->w32.Fh, fm32, 2 * fm32}, noo, no64, s));
      LRP_LAUNCH(p, LRP_K_REFINE, 1, s, launch_setup_correction(ra, count, s));
    } else {
      if (step)
        LRP_LAUNCH(p, LRP_K_REFINE, 1, s, launch_prepare_refine2(rstep, count, s));
      else
        LRP_LAUNCH(p, LRP_K_REFINE, 1, s, launch_prepare_refine(rstep, count, s));
      LRP_LAUNCH(p, LRP_K_REFINE, 1, s, launch_assemble_residual(rstep, count, s));
      if ((st = cholqr<double>(p, p->w64, g, c64, cb64, p->w64.A, nm, 2 * nm, kDimX, s, 1))) return st;
      LRP_LAUNCH(p, LRP_K_REFINE, 1, s, launch_recompress(ra, count, 0, p->mixed_residual_tol, rcap_res, s));
      LRP_LAUNCH(p, LRP_K_GEMM, gemm_kernels<double>(p), s,
                 launch_gemm_nn<double>(g, p->st, cs<double>(p->w64.A, nm, 2 * nm), kDimX,
                                        Strided<const double>{p->w64.Bf, MM, 2 * MM}, kDimR,
                                        Strided<double>{p->w64.Q1, nm, 2 * nm}, none, 0, s));
      // FP32 correction solve on the residual (already in transformed variables).
      LRP_LAUNCH(p, LRP_K_REFINE, 1, s, launch_setup_correction(ra, count, s));
      LRP_LAUNCH(p, LRP_K_REFINE, 1, s,
                 (launch_convert<double, float>(d.n, d.ld, count, p->st, cs<double>(p->w64.Q1, nm, 2 * nm),
                                                Strided<float>{p->w32.Fh, fm32, 2 * fm32}, kDimRF, s)));
    }
    if ((st = phase_iterate<float>(p, p->w32, c32, count, s))) return st;
    // What1 = What0 + dWhat, recompressed.  Two passes: the stacked blocks are
    // two near-orthonormal bases, and the result is the output.
    if (d.M <= 64) {
      // Both blocks hold FP32 values (step 0), or the first block is the FP64
      // result of step 0 held as (hi, lo) planes (the lo plane in the free
      // right-hand-side buffer): double-float Grams and products on the FP32
      // pipe, FP64-accurate (~1e-13 relative), the first product kept as
      // (hi, lo) planes for the second pass.
      RefineArgs rs = ra;
      rs.X32 = {p->w32.A, nm, 2 * nm};
      if (step) rs.X32lo = {p->w32.Fh, fm32, 2 * fm32};
      const Strided<const float> a32{p->w32.A, nm, 2 * nm};
      const Strided<const float> nof{nullptr, 0, 0};
      const Strided<const float> a32lo = step ? Strided<const float>{p->w32.Fh, fm32, 2 * fm32} : nof;
      const Strided<float> q1h{p->w32.Q1, nm, 2 * nm}, q1l{p->w32.Q2, nm, 2 * nm}, noo{nullptr, 0, 0};
      const Strided<double> no64{nullptr, 0, 0};
      Strided<double> G64{p->w64.G, MM, 2 * MM};
      LRP_LAUNCH(p, LRP_K_REFINE, 1, s, launch_prepare_sum(rs, count, s));
      LRP_LAUNCH(p, LRP_K_REFINE, 1, s, launch_assemble_sum(rs, count, s));
      if (step) {
        LRP_LAUNCH(p, LRP_K_GRAM_DF, 1, s, launch_gram_dd(g, p->st, a32, a32lo, kDimX, p->w64.part, s));
        LRP_LAUNCH(p, LRP_K_REDUCE, 1, s, launch_reduce(g, p->st, kDimX, kDimX, p->w64.part, G64, true, s));
      } else if ((st = gram_reduce<float>(p, g, a32, kDimX, a32, kDimX, p->w64.part, G64, true, s, true))) {
        return st;
      }
      LRP_LAUNCH(p, LRP_K_CHOL, 1, s, launch_chol<double>(c64, cb64, kDimX, 0, s));
      LRP_LAUNCH(p, LRP_K_GEMM_DF, 1, s,
                 launch_gemm_dfx(g, p->st, a32, a32lo, kDimX, Strided<const double>{p->w64.P, MM, 2 * MM}, kDimX,
                                 q1h, q1l, no64, s, true));
      LRP_LAUNCH(p, LRP_K_GRAM_DF, 1, s,
                 launch_gram_dd(g, p->st, Strided<const float>{p->w32.Q1, nm, 2 * nm},
                                Strided<const float>{p->w32.Q2, nm, 2 * nm}, kDimX, p->w64.part, s));
      LRP_LAUNCH(p, LRP_K_REDUCE, 1, s, launch_reduce(g, p->st, kDimX, kDimX, p->w64.part, G64, true, s));
      LRP_LAUNCH(p, LRP_K_CHOL, 1, s, launch_chol<double>(c64, cb64, kDimX, 1, s));
      LRP_LAUNCH(p, LRP_K_REFINE, 1, s, launch_recompress(rs, count, 1, 0.0, d.M, s));
      LRP_LAUNCH(p, LRP_K_GEMM_DF, 1, s,
                 launch_gemm_dfx(g, p->st, Strided<const float>{p->w32.Q1, nm, 2 * nm},
                                 Strided<const float>{p->w32.Q2, nm, 2 * nm}, kDimX,
                                 Strided<const double>{p->w64.Bf, MM, 2 * MM}, kDimR, noo, noo,
                                 Strided<double>{p->w64.U[0], nm, 2 * nm}, s));
      (void)q1l;
    } else {
      LRP_LAUNCH(p, LRP_K_REFINE, 1, s, launch_prepare_sum(ra, count, s));
      LRP_LAUNCH(p, LRP_K_REFINE, 1, s, launch_assemble_sum(ra, count, s));
      if ((st = cholqr<double>(p, p->w64, g, c64, cb64, p->w64.A, nm, 2 * nm, kDimX, s, 2))) return st;
      LRP_LAUNCH(p, LRP_K_REFINE, 1, s, launch_recompress(ra, count, 1, 0.0, d.M, s));
      LRP_LAUNCH(p, LRP_K_GEMM, gemm_kernels<double>(p), s,
                 launch_gemm_nn<double>(g, p->st, cs<double>(p->w64.Q1, nm, 2 * nm), kDimX,
                                        Strided<const double>{p->w64.Bf, MM, 2 * MM}, kDimR,
                                        Strided<double>{p->w64.U[0], nm, 2 * nm}, none, 0, s));
    }
    return LRP_OK;
  };
  if ((st = refine_step(0, s))) return st;
  if (p->opts.refine_steps >= 2) {
    // The problems whose first step looks unreliable take a second one
    // (k_check_refine holds the others out); it runs when any is flagged: a
    // host decision, or a conditional node when the solve is one graph.
    LRP_CUDA(cudaMemsetAsync(p->active_dev, 0, sizeof(int32_t), s));
    LRP_LAUNCH(p, LRP_K_OTHER, 1, s, launch_check_refine(ra, count, p->active_dev, s));
    if (p->capturing_solve) {
      cudaStreamCaptureStatus cst;
      cudaGraph_t graph = nullptr;
      const cudaGraphNode_t* deps = nullptr;
      size_t ndeps = 0;
      LRP_CUDA(cudaStreamGetCaptureInfo(s, &cst, nullptr, &graph, &deps, nullptr, &ndeps));
      cudaGraphConditionalHandle h;
      LRP_CUDA(cudaGraphConditionalHandleCreate(&h, graph, 0, 0));
      LRP_LAUNCH(p, LRP_K_OTHER, 1, s, launch_cond_positive(p->active_dev, h, s));
      LRP_CUDA(cudaStreamGetCaptureInfo(s, &cst, nullptr, &graph, &deps, nullptr, &ndeps));
      cudaGraphNodeParams np = {};
      np.type = cudaGraphNodeTypeConditional;
      np.conditional.handle = h;
      np.conditional.type = cudaGraphCondTypeIf;
      np.conditional.size = 1;
      cudaGraphNode_t node;
      LRP_CUDA(cudaGraphAddNode(&node, graph, deps, nullptr, ndeps, &np));
      cudaGraph_t body = np.conditional.phGraph_out[0];
      LRP_CUDA(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
      LRP_CUDA(cudaStreamBeginCaptureToGraph(p->if_stream, body, nullptr, nullptr, 0,
                                             cudaStreamCaptureModeThreadLocal));
      st = refine_step(1, p->if_stream);
      cudaGraph_t captured = nullptr;
      const cudaError_t e = cudaStreamEndCapture(p->if_stream, &captured);
      if (st) return st;
      if (e != cudaSuccess) return set_error(LRP_ECUDA, std::string("second step capture: ") + cudaGetErrorString(e));
    } else {
      LRP_LAUNCH(p, LRP_K_OTHER, 1, s, launch_stage(p->active_dev, p->active_host_dev, sizeof(int32_t), s));
      LRP_CUDA(cudaStreamSynchronize(s));
      if (*static_cast<volatile int32_t*>(p->active_host) > 0 && (st = refine_step(1, s))) return st;
    }
    LRP_LAUNCH(p, LRP_K_OTHER, 1, s, launch_release_held(ra, count, s));
  }
  LRP_LAUNCH(p, LRP_K_OTHER, 1, s, launch_final_state(ra, count, s));
  return phase_finalize<double>(p, p->w64, c64, count, s, true);
}
}  // namespace lrp

namespace lrp {

// Enqueue the whole solve of `count` staged problems into the capturing
// stream s (device-side iteration loops).
lrp_status enqueue_solve(lrp_plan_s* p, int count, cudaStream_t s) {
  p->capturing_solve = true;
  const lrp_status st = (p->opts.precision == LRP_FP64) ? run_fp64(p, count, s) : run_mixed(p, count, s);
  p->capturing_solve = false;
  return st;
}

// Host staging of a device-loop solve: the forward DST job arrays (the problem
// descriptors are staged by lrp_solve_batch).
void stage_solve(lrp_plan_s* p, int count) {
  if (p->opts.precision == LRP_FP64) {
    forward_stage_host<double>(p, p->w64, count, 0);
  } else {
    forward_stage_host<float>(p, p->w32, count, 0);
    if (p->opts.refine_steps > 0) forward_stage_host<double>(p, p->w64, count, 1);
  }
}

// One graph launch per solve: captured on first use for (count, warm records,
// tracing), replayed on the caller's stream afterwards; up to kSolveGraphs such
// graphs are kept per plan.
static lrp_status solve_device(lrp_plan_s* p, int count, cudaStream_t s) {
  stage_solve(p, count);
  const int key[3] = {count, p->any_warm ? 1 : 0, p->trace_on ? 1 : 0};
  lrp_plan_s::SolveGraph* g = nullptr;
  lrp_plan_s::SolveGraph* victim = nullptr;  // an empty entry, else the least recently used
  for (auto& e : p->solve_graphs) {
    if (e.exec && e.key[0] == key[0] && e.key[1] == key[1] && e.key[2] == key[2]) {
      g = &e;
      break;
    }
    if (!victim || (victim->exec && (!e.exec || e.used < victim->used))) victim = &e;
  }
  if (!g) {
    g = victim;
    if (g->exec) {
      SetupGuard guard;
      cudaGraphExecDestroy(g->exec);
      g->exec = nullptr;
    }
    for (int i = 0; i < 3; ++i) g->key[i] = -1;
    int64_t before[LRP_K_COUNT];
    for (int c = 0; c < LRP_K_COUNT; ++c) before[c] = p->stats.launches[c];
    cudaGraph_t graph = nullptr;
    {
      CaptureGuard capture;
      LRP_CUDA(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal));
      const lrp_status st = enqueue_solve(p, count, p->cap_stream);
      const cudaError_t e = cudaStreamEndCapture(p->cap_stream, &graph);
      if (st != LRP_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
      }
      if (e != cudaSuccess) return set_error(LRP_ECUDA, std::string("solve capture: ") + cudaGetErrorString(e));
    }
    const cudaError_t e = cudaGraphInstantiate(&g->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      g->exec = nullptr;
      return set_error(LRP_ECUDA, std::string("solve graph instantiate: ") + cudaGetErrorString(e));
    }
    for (int c = 0; c < LRP_K_COUNT; ++c) {
      g->launches[c] = p->stats.launches[c] - before[c];
      p->stats.launches[c] = before[c];
    }
    for (int i = 0; i < 3; ++i) g->key[i] = key[i];
  }
  g->used = ++p->solve_tick;
  LRP_CUDA(cudaGraphLaunch(g->exec, s));
  LRP_CUDA(cudaEventRecord(p->solve_done, s));
  for (int c = 0; c < LRP_K_COUNT; ++c) p->stats.launches[c] += g->launches[c];
  return LRP_OK;
}

}  // namespace lrp

static lrp_status validate_problem(const lrp_plan_s* p, const lrp_problem& pr) {
  const int64_t n = p->n;
  if (pr.warm && pr.warm->plan != p) return set_error(LRP_EINVAL, "warm-start record belongs to another plan");
  if (pr.r_f < 1 || pr.r_f > p->dims.RF) return set_error(LRP_EINVAL, "r_f out of range [1, max_rhs_rank]");
  if (!pr.d_U_f || !pr.d_V_f || (!pr.d_s_f && p->opts.matrix == LRP_MAT_POISSON) || !pr.d_U || !pr.d_S || !pr.d_V)
    return set_error(LRP_EINVAL, "NULL factor pointer");
  if (pr.ldu_f < n || pr.ldv_f < n || pr.ldu < n || pr.ldv < n) return set_error(LRP_EINVAL, "leading dimension < n");
  return LRP_OK;
}

namespace lrp {

// Validate a batch and write its descriptors to the plan's pinned staging
// (the caller holds p->mu).  A device-loop solve returns before it has run, so
// its staging is rewritten only after the previous solve has finished with it.
lrp_status stage_problems(lrp_plan_s* p, int32_t count, const lrp_problem* hp) {
  if (count < 1 || count > p->dims.B) return set_error(LRP_EINVAL, "count out of range [1, batch]");
  for (int i = 0; i < count; ++i) {
    lrp_status s = validate_problem(p, hp[i]);
    if (s != LRP_OK) return s;
    for (int j = 0; j < i && hp[i].warm; ++j)
      if (hp[j].warm == hp[i].warm) return set_error(LRP_EINVAL, "one warm-start record used twice in a batch");
  }
  if (p->device_loop) LRP_CUDA(cudaEventSynchronize(p->solve_done));
  for (int i = 0; i < count; ++i) {
    ProblemDev& d = p->prob_host[i];
    d.rf = hp[i].r_f;
    d.pad = 0;
    d.U_f = hp[i].d_U_f;
    d.ldu_f = hp[i].ldu_f;
    d.s_f = hp[i].d_s_f;
    d.V_f = hp[i].d_V_f;
    d.ldv_f = hp[i].ldv_f;
    d.U = hp[i].d_U;
    d.ldu = hp[i].ldu;
    d.S = hp[i].d_S;
    d.V = hp[i].d_V;
    d.ldv = hp[i].ldv;
    d.info = hp[i].d_info;
    d.warm = hp[i].warm ? hp[i].warm->dev : nullptr;
  }
  p->any_warm = false;
  for (int i = 0; i < count; ++i) p->any_warm = p->any_warm || hp[i].warm != nullptr;
  p->last_count = count;
  return LRP_OK;
}

// The staged descriptors to device memory (a kernel reading the mapped pinned staging).
lrp_status launch_problems(lrp_plan_s* p, int32_t count, cudaStream_t s) {
  LRP_LAUNCH(p, LRP_K_OTHER, 1, s, launch_stage(p->prob_host_dev, p->prob_dev, sizeof(ProblemDev) * count, s));
  return LRP_OK;
}

}  // namespace lrp

extern "C" lrp_status lrp_solve_batch(lrp_plan_t p, int32_t count, const lrp_problem* hp, void* stream) {
  if (!p || !hp) return set_error(LRP_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lock(p->mu);
  lrp_status st = stage_problems(p, count, hp);
  if (st != LRP_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = launch_problems(p, count, s)) != LRP_OK) return st;
  if (p->device_loop && !p->stats.timing) return solve_device(p, count, s);
  if (p->opts.precision == LRP_FP64) return run_fp64(p, count, s);
  return run_mixed(p, count, s);
}

extern "C" lrp_status lrp_solve(lrp_plan_t p, int32_t r_f, const double* U_f, int64_t ldu_f, const double* s_f,
                                const double* V_f, int64_t ldv_f, double* U, int64_t ldu, double* S, double* V,
                                int64_t ldv, lrp_info* info, void* stream) {
  lrp_problem pr;
  memset(&pr, 0, sizeof(pr));
  pr.r_f = r_f;
  pr.d_U_f = U_f;
  pr.ldu_f = ldu_f;
  pr.d_s_f = s_f;
  pr.d_V_f = V_f;
  pr.ldv_f = ldv_f;
  pr.d_U = U;
  pr.ldu = ldu;
  pr.d_S = S;
  pr.d_V = V;
  pr.ldv = ldv;
  pr.d_info = info;
  return lrp_solve_batch(p, 1, &pr, stream);
}

extern "C" lrp_status lrp_dst1(int64_t n, int32_t ncols, const double* X, int64_t ldx, double* Y, int64_t ldy,
                               void* stream) {
  if (n < 1 || !is_pow2(n + 1)) return set_error(LRP_EINVAL, "n+1 must be a power of two >= 2");
  if (ncols < 0 || !X || !Y || ldx < n || ldy < n) return set_error(LRP_EINVAL, "bad DST arguments");
  if (!dst_supported(n)) return set_error(LRP_EINVAL, "n+1 must be at most 2^21");
  if (ncols == 0) return LRP_OK;
  cudaStream_t s = (cudaStream_t)stream;
  // Per-call job arrays: tiny device allocation kept for the lifetime of the process per n.
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  struct Cache {
    int64_t n = 0;
    int dev = -1;
    void* tw = nullptr;
    void* arrays = nullptr;
    void* temp = nullptr;
    size_t temp_bytes = 0;
  };
  static Cache cache[8];
  SetupGuard guard;  // the cache may allocate, free and synchronise
  int dev = 0;
  LRP_CUDA(cudaGetDevice(&dev));
  {
    lrp_status cs_ = ensure_configured(dev);
    if (cs_ != LRP_OK) return cs_;
  }
  Cache* c = nullptr;
  for (auto& e : cache)
    if (e.n == n && e.dev == dev) c = &e;
  if (!c) {
    for (auto& e : cache)
      if (e.n == 0) {
        c = &e;
        break;
      }
    if (!c) {
      c = &cache[0];
      cudaFree(c->tw);
      cudaFree(c->arrays);
      if (c->temp) cudaFree(c->temp);
      c->temp = nullptr;
      c->temp_bytes = 0;
    }
    c->n = n;
    c->dev = dev;
    c->tw = dst_make_twiddles(n + 1, true, nullptr);
    LRP_CUDA(cudaMalloc(&c->arrays, 4 * sizeof(void*)));
    LRP_CUDA(cudaDeviceSynchronize());
  }
  {
    const size_t need = dst_temp_bytes(n, true) * (size_t)ncols;
    if (need > c->temp_bytes) {
      if (c->temp) cudaFree(c->temp);
      c->temp = nullptr;
      c->temp_bytes = 0;
      LRP_CUDA(cudaMalloc(&c->temp, need));
      c->temp_bytes = need;
    }
  }
  const void* h[4] = {X, Y, (const void*)(intptr_t)ldx, (const void*)(intptr_t)ldy};
  LRP_CUDA(cudaMemcpyAsync(c->arrays, h, sizeof(h), cudaMemcpyHostToDevice, s));
  LRP_CUDA(cudaStreamSynchronize(s));  // h lives on this stack frame
  DstBatch<double, double> job;
  const void* const* arr = (const void* const*)c->arrays;
  job.in = (const double* const*)(arr + 0);
  job.out = (double* const*)(arr + 1);
  job.ld_in = (const int64_t*)(arr + 2);
  job.ld_out = (const int64_t*)(arr + 3);
  job.nslots = 1;
  job.fixed_cols = ncols;
  job.ncols_dev = nullptr;
  job.ncols_stride = 0;
  job.ncols_mat_stride = 0;
  job.active_dev = nullptr;
  job.active_stride = 0;
  job.require_active = 0;
  LRP_CUDA((dst1_launch<double, double, double>(n, job, ncols, 1, 1, c->tw, s, c->temp, c->temp_bytes)));
  return LRP_OK;
}

extern "C" const char* lrp_last_error(void) { return g_last_error.c_str(); }

extern "C" const char* lrp_status_string(lrp_status s) {
  switch (s) {
    case LRP_OK: return "LRP_OK";
    case LRP_EINVAL: return "LRP_EINVAL";
    case LRP_ENOMEM: return "LRP_ENOMEM";
    case LRP_ECUDA: return "LRP_ECUDA";
    case LRP_ETIMEDOUT: return "LRP_ETIMEDOUT";
    case LRP_NOT_CONVERGED: return "LRP_NOT_CONVERGED";
    case LRP_RANK_CAPPED: return "LRP_RANK_CAPPED";
    case LRP_EAGAIN: return "LRP_EAGAIN";
    case LRP_ECAPACITY: return "LRP_ECAPACITY";
  }
  return "LRP_UNKNOWN";
}

static_assert(sizeof(lrp_opts) == 64, "lrp_opts layout");
static_assert(sizeof(lrp_info) == 64, "lrp_info layout");
static_assert(sizeof(lrp_problem) == 104, "lrp_problem layout");
