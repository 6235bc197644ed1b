// A group of plans that solves one batch as several concurrent sub-batches.
//
// lrp_solve_batch drives a batch from the host (one readback of the active
// count per Cross-DEIM iteration), and many of its kernels are per-problem
// cores that occupy few SMs.  A group splits a batch over `lanes` plans, each
// with its own CUDA stream and its own host worker thread, so that the lanes'
// iterations interleave on the GPU and the latency-bound phases of one lane
// overlap the tall products of another.  The lanes start after the work the
// caller's stream holds when lrp_group_solve is called; the caller's stream
// waits for every lane before its later work.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <condition_variable>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"
#include "guard.cuh"
#include "solver.cuh"

namespace lrp {
__global__ void k_pack_offsets(const SolveState* __restrict__ st, int count, int64_t n, int64_t* __restrict__ off,
                               const int64_t* __restrict__ base_in);
__global__ void k_pack_copy(const SolveState* __restrict__ st, const ProblemDev* __restrict__ prob, int64_t n,
                            const int64_t* __restrict__ off, double* __restrict__ out, int64_t capacity);
}  // namespace lrp

using namespace lrp;

struct lrp_group_s {
  int device = 0;
  int lanes = 0;
  std::vector<lrp_plan_t> plans;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> done;
  cudaEvent_t start = nullptr;
  std::vector<std::thread> workers;
  std::mutex mu;
  std::condition_variable cv, done_cv;
  uint64_t job = 0;
  int pending = 0;
  bool stop = false;
  const lrp_problem* probs = nullptr;
  std::vector<int> first, count;
  std::vector<lrp_status> status;
  std::vector<std::string> error;
  std::mutex call_mu;  // one lrp_group_solve / pack at a time
};

static void group_worker(lrp_group_s* g, int lane) {
  cudaSetDevice(g->device);
  uint64_t seen = 0;
  std::unique_lock<std::mutex> lk(g->mu);
  for (;;) {
    g->cv.wait(lk, [&] { return g->stop || g->job != seen; });
    if (g->stop) break;
    seen = g->job;
    const lrp_problem* probs = g->probs + g->first[lane];
    const int cnt = g->count[lane];
    lk.unlock();
    lrp_status st = LRP_OK;
    std::string err;
    if (cnt > 0) {
      if (cudaStreamWaitEvent(g->streams[lane], g->start, 0) != cudaSuccess) {
        st = LRP_ECUDA;
        err = "group: stream wait failed";
      } else {
        st = lrp_solve_batch(g->plans[lane], cnt, probs, (void*)g->streams[lane]);
        if (st != LRP_OK) err = lrp_last_error();
      }
    }
    if (cudaEventRecord(g->done[lane], g->streams[lane]) != cudaSuccess && st == LRP_OK) {
      st = LRP_ECUDA;
      err = "group: event record failed";
    }
    lk.lock();
    g->status[lane] = st;
    g->error[lane] = err;
    if (--g->pending == 0) g->done_cv.notify_all();
  }
}

static void group_free(lrp_group_s* g) {
  {
    std::lock_guard<std::mutex> lk(g->mu);
    g->stop = true;
  }
  g->cv.notify_all();
  for (auto& t : g->workers) t.join();
  for (lrp_plan_t p : g->plans)
    if (p) lrp_plan_destroy(p);
  SetupGuard guard;
  for (cudaStream_t s : g->streams)
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : g->done)
    if (e) cudaEventDestroy(e);
  if (g->start) cudaEventDestroy(g->start);
  delete g;
}

extern "C" lrp_status lrp_group_create(lrp_group_t* out, int64_t n, double tol, int32_t max_rank,
                                       const lrp_opts* opts, int32_t lanes) {
  if (!out) return set_error(LRP_EINVAL, "out is NULL");
  *out = nullptr;
  if (lanes < 1 || lanes > 16) return set_error(LRP_EINVAL, "lanes must be in [1, 16]");
  lrp_opts o;
  lrp_default_opts(&o);
  if (opts) o = *opts;
  if (o.batch < lanes) return set_error(LRP_EINVAL, "batch must be >= lanes");
  lrp_group_s* g = new (std::nothrow) lrp_group_s();
  if (!g) return set_error(LRP_ENOMEM, "host allocation failed");
  if (cudaGetDevice(&g->device) != cudaSuccess) {
    delete g;
    return set_error(LRP_ECUDA, "no CUDA device");
  }
  g->lanes = lanes;
  g->first.assign(lanes, 0);
  g->count.assign(lanes, 0);
  g->status.assign(lanes, LRP_OK);
  g->error.assign(lanes, std::string());
  lrp_opts lo = o;
  lo.batch = (o.batch + lanes - 1) / lanes;
  for (int l = 0; l < lanes; ++l) {
    lrp_plan_t p = nullptr;
    lrp_status s = lrp_plan(&p, n, tol, max_rank, &lo);
    if (s != LRP_OK) {
      const std::string msg = lrp_last_error();
      group_free(g);
      return set_error(s, msg);
    }
    g->plans.push_back(p);
  }
  {
    SetupGuard guard;
    bool ok = cudaEventCreateWithFlags(&g->start, cudaEventDisableTiming) == cudaSuccess;
    for (int l = 0; l < lanes && ok; ++l) {
      cudaStream_t s = nullptr;
      cudaEvent_t e = nullptr;
      ok = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess &&
           cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
      g->streams.push_back(s);
      g->done.push_back(e);
    }
    if (!ok) {
      guard.lk.unlock();
      group_free(g);
      return set_error(LRP_ECUDA, "group stream/event creation failed");
    }
  }
  for (int l = 0; l < lanes; ++l) g->workers.emplace_back(group_worker, g, l);
  *out = g;
  return LRP_OK;
}

extern "C" lrp_status lrp_group_solve(lrp_group_t g, int32_t count, const lrp_problem* problems, void* stream) {
  if (!g || !problems) return set_error(LRP_EINVAL, "NULL argument");
  const int per = g->plans[0]->dims.B;
  if (count < 1 || count > per * g->lanes) return set_error(LRP_EINVAL, "count out of range [1, batch]");
  for (int i = 0; i < count; ++i)
    if (problems[i].warm) return set_error(LRP_EINVAL, "warm-start records are per plan: not accepted by a group");
  std::lock_guard<std::mutex> call(g->call_mu);
  cudaStream_t cs = (cudaStream_t)stream;
  if (cudaEventRecord(g->start, cs) != cudaSuccess) return set_error(LRP_ECUDA, "group: event record failed");
  {
    std::lock_guard<std::mutex> lk(g->mu);
    // contiguous, nearly equal shares
    int at = 0;
    for (int l = 0; l < g->lanes; ++l) {
      const int c = count / g->lanes + (l < count % g->lanes ? 1 : 0);
      g->first[l] = at;
      g->count[l] = c;
      at += c;
    }
    g->probs = problems;
    g->pending = g->lanes;
    ++g->job;
  }
  g->cv.notify_all();
  lrp_status st = LRP_OK;
  std::string err;
  {
    std::unique_lock<std::mutex> lk(g->mu);
    g->done_cv.wait(lk, [&] { return g->pending == 0; });
    for (int l = 0; l < g->lanes; ++l)
      if (g->status[l] != LRP_OK && st == LRP_OK) {
        st = g->status[l];
        err = g->error[l];
      }
  }
  for (int l = 0; l < g->lanes; ++l)
    if (cudaStreamWaitEvent(cs, g->done[l], 0) != cudaSuccess && st == LRP_OK) {
      st = LRP_ECUDA;
      err = "group: stream wait failed";
    }
  if (st != LRP_OK) return set_error(st, err);
  return LRP_OK;
}

extern "C" lrp_status lrp_group_plan(lrp_group_t g, int32_t lane, lrp_plan_t* out) {
  if (!g || !out || lane < 0 || lane >= g->lanes) return set_error(LRP_EINVAL, "bad lane");
  *out = g->plans[lane];
  return LRP_OK;
}

extern "C" lrp_status lrp_group_pack(lrp_group_t g, double* d_packed, int64_t capacity, int64_t* d_offsets,
                                     void* stream) {
  if (!g || !d_offsets || capacity < 0 || (capacity > 0 && !d_packed))
    return set_error(LRP_EINVAL, "bad lrp_group_pack arguments");
  std::lock_guard<std::mutex> call(g->call_mu);
  cudaStream_t s = (cudaStream_t)stream;
  // Lane by lane on the caller's stream: each lane's offsets start from the
  // previous lane's total (d_offsets[first]), so the blocks are back to back.
  for (int l = 0; l < g->lanes; ++l) {
    const int cnt = g->count[l];
    if (cnt < 1) continue;
    lrp_plan_s* p = g->plans[l];
    int64_t* off = d_offsets + g->first[l];
    k_pack_offsets<<<1, 1024, 0, s>>>(p->st, cnt, p->n, off, l > 0 ? off : nullptr);
    const dim3 grid((unsigned)((p->n + 255) / 256), (unsigned)cnt);
    k_pack_copy<<<grid, 256, 0, s>>>(p->st, p->prob_dev, p->n, off, d_packed, capacity);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(LRP_ECUDA, std::string("lrp_group_pack: ") + cudaGetErrorString(e));
  return LRP_OK;
}

extern "C" lrp_status lrp_group_destroy(lrp_group_t g) {
  if (!g) return LRP_OK;
  group_free(g);
  return LRP_OK;
}
