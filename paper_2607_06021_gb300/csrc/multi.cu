// Mixed grid sizes in one launch (include/lrp.h, lrp_multi_*).
//
// A set holds one plan per grid size n, each with device-side iteration loops.
// lrp_multi_solve sorts the problems of a call into their size's plan (the
// plans' problem descriptor arrays are the device work list) and runs every
// size's whole solve as one branch of a single CUDA graph: the branches fork
// from the caller's stream, run concurrently, and each continues its
// Cross-DEIM loops on the device (conditional while-nodes) while any of its
// problems is active.  The graph is captured on first use for each vector of
// per-size counts (and warm-record / trace use) and replayed afterwards.
#include <cuda_runtime.h>

#include <mutex>
#include <string>
#include <vector>

#include "solver.cuh"

namespace lrp {
lrp_status stage_problems(lrp_plan_s* p, int32_t count, const lrp_problem* hp);
lrp_status launch_problems(lrp_plan_s* p, int32_t count, cudaStream_t s);
lrp_status enqueue_solve(lrp_plan_s* p, int count, cudaStream_t s);
void stage_solve(lrp_plan_s* p, int count);
}  // namespace lrp

using namespace lrp;

struct lrp_multi_s {
  std::vector<lrp_plan_s*> plans;
  std::vector<int64_t> ns;
  cudaStream_t cap = nullptr;
  std::vector<cudaEvent_t> ev;  // [0] fork, [1 + b] join of size b
  cudaGraphExec_t exec = nullptr;
  std::vector<int> key;
  std::vector<std::vector<lrp_problem>> per;
  std::vector<int64_t> launches;  // [size][class] kernel nodes of the captured graph (loop bodies once)
  std::mutex mu;
};

static void multi_free(lrp_multi_s* m) {
  {
    SetupGuard guard;
    cudaDeviceSynchronize();
    if (m->exec) cudaGraphExecDestroy(m->exec);
    for (cudaEvent_t e : m->ev)
      if (e) cudaEventDestroy(e);
    if (m->cap) cudaStreamDestroy(m->cap);
  }
  for (lrp_plan_s* p : m->plans)
    if (p) lrp_plan_destroy(p);
  delete m;
}

extern "C" lrp_status lrp_multi_create(lrp_multi_t* out, int32_t nsizes, const int64_t* ns, const int32_t* batches,
                                       double tol, int32_t max_rank, const lrp_opts* opts) {
  if (!out || !ns || !batches || nsizes < 1 || nsizes > 64) return set_error(LRP_EINVAL, "bad size list");
  *out = nullptr;
  for (int i = 0; i < nsizes; ++i)
    for (int j = 0; j < i; ++j)
      if (ns[i] == ns[j]) return set_error(LRP_EINVAL, "a grid size is listed twice");
  lrp_opts o;
  lrp_default_opts(&o);
  if (opts) o = *opts;
  o.loop_on_device = 1;
  lrp_multi_s* m = new (std::nothrow) lrp_multi_s();
  if (!m) return set_error(LRP_ENOMEM, "host allocation failed");
  for (int i = 0; i < nsizes; ++i) {
    o.batch = batches[i];
    lrp_plan_t p = nullptr;
    const lrp_status st = lrp_plan(&p, ns[i], tol, max_rank, &o);
    if (st != LRP_OK) {
      multi_free(m);
      return st;
    }
    m->plans.push_back(p);
    m->ns.push_back(ns[i]);
  }
  m->per.resize(nsizes);
  m->launches.assign((size_t)nsizes * LRP_K_COUNT, 0);
  m->ev.assign(nsizes + 1, nullptr);
  {
    SetupGuard guard;
    cudaError_t e = cudaStreamCreateWithFlags(&m->cap, cudaStreamNonBlocking);
    for (int i = 0; i <= nsizes && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&m->ev[i], cudaEventDisableTiming);
    if (e != cudaSuccess) {
      multi_free(m);
      return set_error(LRP_ECUDA, std::string("multi setup: ") + cudaGetErrorString(e));
    }
  }
  *out = m;
  return LRP_OK;
}

extern "C" lrp_status lrp_multi_plan(lrp_multi_t m, int32_t size_index, lrp_plan_t* out) {
  if (!m || !out || size_index < 0 || size_index >= (int)m->plans.size()) return set_error(LRP_EINVAL, "bad argument");
  *out = m->plans[size_index];
  return LRP_OK;
}

extern "C" lrp_status lrp_multi_solve(lrp_multi_t m, int32_t count, const int64_t* ns, const lrp_problem* problems,
                                      void* stream) {
  if (!m || !ns || !problems || count < 1) return set_error(LRP_EINVAL, "bad argument");
  std::lock_guard<std::mutex> lock(m->mu);
  const int S = (int)m->plans.size();
  for (auto& v : m->per) v.clear();
  for (int i = 0; i < count; ++i) {
    int b = 0;
    while (b < S && m->ns[b] != ns[i]) ++b;
    if (b == S) return set_error(LRP_EINVAL, "problem " + std::to_string(i) + ": grid size not in the set");
    m->per[b].push_back(problems[i]);
  }
  std::vector<std::unique_lock<std::mutex>> locks;
  std::vector<int> key;
  for (int b = 0; b < S; ++b) {
    lrp_plan_s* p = m->plans[b];
    locks.emplace_back(p->mu);
    const int c = (int)m->per[b].size();
    if (c > 0) {
      const lrp_status st = stage_problems(p, c, m->per[b].data());
      if (st != LRP_OK) return st;
      stage_solve(p, c);
    }
    key.push_back(c);
    key.push_back(c > 0 && p->any_warm ? 1 : 0);
    key.push_back(p->trace_on ? 1 : 0);
  }
  if (!m->exec || key != m->key) {
    if (m->exec) {
      SetupGuard guard;
      cudaGraphExecDestroy(m->exec);
      m->exec = nullptr;
    }
    std::vector<int64_t> before((size_t)S * LRP_K_COUNT);
    for (int b = 0; b < S; ++b)
      for (int c = 0; c < LRP_K_COUNT; ++c) before[(size_t)b * LRP_K_COUNT + c] = m->plans[b]->stats.launches[c];
    cudaGraph_t graph = nullptr;
    {
      CaptureGuard capture;
      cudaError_t e = cudaStreamBeginCapture(m->cap, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return set_error(LRP_ECUDA, std::string("multi capture: ") + cudaGetErrorString(e));
      lrp_status st = LRP_OK;
      e = cudaEventRecord(m->ev[0], m->cap);
      for (int b = 0; b < S && st == LRP_OK && e == cudaSuccess; ++b) {
        const int c = (int)m->per[b].size();
        if (c == 0) continue;
        lrp_plan_s* p = m->plans[b];
        e = cudaStreamWaitEvent(p->cap_stream, m->ev[0], 0);
        if (e != cudaSuccess) break;
        st = launch_problems(p, c, p->cap_stream);
        if (st == LRP_OK) st = enqueue_solve(p, c, p->cap_stream);
        if (st != LRP_OK) break;
        e = cudaEventRecord(m->ev[1 + b], p->cap_stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(m->cap, m->ev[1 + b], 0);
      }
      const cudaError_t e2 = cudaStreamEndCapture(m->cap, &graph);
      if (st != LRP_OK || e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        if (st != LRP_OK) return st;
        return set_error(LRP_ECUDA, std::string("multi capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
      }
    }
    const cudaError_t e = cudaGraphInstantiate(&m->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      m->exec = nullptr;
      return set_error(LRP_ECUDA, std::string("multi graph instantiate: ") + cudaGetErrorString(e));
    }
    for (int b = 0; b < S; ++b) {
      lrp_plan_s* p = m->plans[b];
      for (int c = 0; c < LRP_K_COUNT; ++c) {
        m->launches[(size_t)b * LRP_K_COUNT + c] = p->stats.launches[c] - before[(size_t)b * LRP_K_COUNT + c];
        p->stats.launches[c] = before[(size_t)b * LRP_K_COUNT + c];
      }
      // the plan's own solve graphs are captured anew on their next use
      for (auto& sg : p->solve_graphs) sg.key[0] = -1;
    }
    m->key = key;
  }
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaGraphLaunch(m->exec, s);
  if (e != cudaSuccess) return set_error(LRP_ECUDA, std::string("multi launch: ") + cudaGetErrorString(e));
  for (int b = 0; b < S; ++b) {
    if (m->per[b].empty()) continue;
    lrp_plan_s* p = m->plans[b];
    e = cudaEventRecord(p->solve_done, s);
    if (e != cudaSuccess) return set_error(LRP_ECUDA, std::string("multi launch: ") + cudaGetErrorString(e));
    for (int c = 0; c < LRP_K_COUNT; ++c) p->stats.launches[c] += m->launches[(size_t)b * LRP_K_COUNT + c];
  }
  return LRP_OK;
}

extern "C" lrp_status lrp_multi_destroy(lrp_multi_t m) {
  if (!m) return LRP_OK;
  multi_free(m);
  return LRP_OK;
}
