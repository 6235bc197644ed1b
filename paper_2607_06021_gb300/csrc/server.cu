// Request server over the batched solver: admission by memory footprint,
// continuous batching per problem shape, warm-start records keyed by the
// caller, latency statistics.
//
// Requests carry host factors (copied at submission, so the caller may reuse
// its buffers at once) and host output buffers (written before the request
// completes).  Worker lanes, one host thread and one CUDA stream each, take the
// oldest waiting request that can start, gather up to a plan's batch of waiting
// requests of the same bucket (n, precision, tol, max_rank, right-hand-side
// rank class) in arrival order, and run them as one lrp_solve_batch call (one
// graph launch: the plans loop on the device).  A bucket may hold up to one
// plan per lane, so requests arriving while a batch of their bucket runs start
// on another lane instead of waiting for it.  Plans are created on first use,
// sized so that several fit the memory cap, and destroyed least recently used
// when a new one would not fit.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "guard.cuh"
#include "lrp.h"

namespace lrp {
lrp_status set_error(lrp_status s, const std::string& msg);
}
extern "C" const char* lrp_last_error(void);

static_assert(sizeof(lrp_server_opts) == 24, "lrp_server_opts layout");
static_assert(sizeof(lrp_request) == 88, "lrp_request layout");
static_assert(sizeof(lrp_result) == 32, "lrp_result layout");
static_assert(sizeof(lrp_server_stats) == 96, "lrp_server_stats layout");
using lrp::set_error;
using lrp::SetupGuard;

namespace {

using Clock = std::chrono::steady_clock;

double us_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::micro>(b - a).count();
}

struct BucketKey {
  int64_t n;
  int32_t precision;
  int32_t max_rank;
  int32_t rf_cap;
  double tol;
  bool operator==(const BucketKey& o) const {
    return n == o.n && precision == o.precision && max_rank == o.max_rank && rf_cap == o.rf_cap && tol == o.tol;
  }
};

// Right-hand-side rank class of a bucket: r_f rounded up to a multiple of 16,
// so that a stream of mixed ranks shares few plans while a plan's r_f capacity
// (and with it its workspace) stays close to its requests' ranks.
int rf_class(int r_f) { return (r_f + 15) / 16 * 16; }

// Index-set capacity of a bucket's plan.  FP64: 2 max_rank + r_f' (at most
// 256).  Mixed precision: 64 while the right-hand side leaves room for the
// index sets (r_f' + 16 <= 64), which keeps the refinement's recompressions in
// double-float arithmetic on the FP32 pipe; larger r_f' take r_f' + 16.
int m_cap_of(int max_rank, int rf_cap, int precision) {
  const int fp64 = std::min(2 * max_rank + rf_cap, 256);
  if (precision != LRP_MIXED) return fp64;
  return std::min(std::max(64, rf_cap + 16), std::max(fp64, rf_cap + 2));
}

struct Request {
  uint64_t ticket = 0;
  BucketKey key{};
  int32_t r_f = 0;
  uint64_t warm_key = 0;
  std::vector<double> in;  // U_f (n r_f) | s_f (r_f) | V_f (n r_f)
  double* U = nullptr;
  double* S = nullptr;
  double* V = nullptr;
  size_t footprint = 0;
  lrp_status solve_status = LRP_OK;  // status the solver reported for this problem
  Clock::time_point t_submit, t_start;
  bool done = false;
  lrp_result result{};
};

struct WarmEntry {
  lrp_warm_t rec = nullptr;
  bool filled = false;
  uint64_t last_used = 0;
};

struct PlanEntry {
  BucketKey key{};
  lrp_plan_t plan = nullptr;
  int B = 0;
  double* d_in = nullptr;   // per slot: U_f (n rf_cap) | s_f (rf_cap) | V_f (n rf_cap)
  double* d_out = nullptr;  // per slot: U (n max_rank) | S (max_rank) | V (n max_rank)
  lrp_info* d_info = nullptr;
  size_t in_stride = 0, out_stride = 0;
  size_t bytes = 0;          // plan arena + slot buffers
  size_t warm_bytes = 0;     // one warm-start record
  bool busy = false;
  uint64_t last_used = 0;
  std::unordered_map<uint64_t, WarmEntry> warm;
};

}  // namespace

struct lrp_server_s {
  lrp_server_opts opts{};
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;       // work for the lanes
  std::condition_variable done_cv;  // a request finished
  std::deque<Request*> queue;       // admitted, not started (arrival order)
  std::unordered_map<uint64_t, Request*> tickets;
  std::vector<PlanEntry*> plans;
  uint64_t next_ticket = 1;
  uint64_t clock = 0;               // LRU counter
  size_t admitted_bytes = 0;        // footprints of queued + running requests
  size_t device_bytes = 0;          // plans + warm records
  int running = 0;
  bool stop = false;
  int64_t submitted = 0, completed = 0, rejected = 0;
  std::vector<double> latencies;    // microseconds, completed requests
  std::vector<std::thread> lanes;
  std::string last_error;           // message of the most recent failed batch
};

namespace {

// Working-set estimate of one request (FP64 words): both right-hand-side
// factors, four n x m_cap blocks (cross matrix, two orthogonalisation passes,
// the factors) and the output factors, per side.
size_t request_footprint(int64_t n, int r_f, int max_rank, int precision = LRP_FP64) {
  const int m = m_cap_of(max_rank, rf_class(r_f), precision);
  return (size_t)8 * (size_t)n * (size_t)(2 * r_f + 4 * m + 2 * max_rank);
}

lrp_opts plan_opts(const BucketKey& k, int B) {
  lrp_opts o;
  lrp_default_opts(&o);
  o.precision = k.precision;
  o.max_rhs_rank = k.rf_cap;
  o.m_cap = m_cap_of(k.max_rank, k.rf_cap, k.precision);
  o.batch = B;
  // each batch is one graph launch whose iteration loops run on the device
  o.loop_on_device = 1;
  return o;
}

size_t slot_buffer_bytes(const BucketKey& k) {
  const size_t in = (size_t)(2 * k.n + 1) * k.rf_cap;
  const size_t out = (size_t)(2 * k.n + 1) * k.max_rank;
  return (in + out) * sizeof(double) + sizeof(lrp_info);
}

size_t warm_record_bytes(const BucketKey& k) {
  const size_t ld = (size_t)((k.n + 31) / 32 * 32);
  return (size_t)2 * ld * m_cap_of(k.max_rank, k.rf_cap, k.precision) * sizeof(double) + 4096;
}

// Batch slots of a bucket's plan: as many as fit a quarter of the memory cap.
lrp_status plan_batch(const lrp_server_opts& so, const BucketKey& k, int* B, size_t* bytes) {
  lrp_opts o1 = plan_opts(k, 1), o2 = plan_opts(k, 2);
  size_t b1 = 0, b2 = 0;
  lrp_status s = lrp_plan_estimate_bytes(k.n, k.tol, k.max_rank, &o1, &b1);
  if (s == LRP_OK) s = lrp_plan_estimate_bytes(k.n, k.tol, k.max_rank, &o2, &b2);
  if (s != LRP_OK) return s;
  const size_t per_slot = (b2 - b1) + slot_buffer_bytes(k);
  const size_t base = b1 - (b2 - b1);
  const size_t budget = (size_t)so.memory_cap_bytes / 4;
  int64_t fit = budget > base ? (int64_t)((budget - base) / per_slot) : 0;
  int b = (int)std::max<int64_t>(1, std::min<int64_t>(fit, so.max_batch));
  lrp_opts ob = plan_opts(k, b);
  size_t bb = 0;
  s = lrp_plan_estimate_bytes(k.n, k.tol, k.max_rank, &ob, &bb);
  if (s != LRP_OK) return s;
  *B = b;
  *bytes = bb + slot_buffer_bytes(k) * (size_t)b;
  return LRP_OK;
}

void destroy_entry(lrp_server_s* sv, PlanEntry* e) {
  for (auto& kv : e->warm) {
    if (kv.second.rec) lrp_warm_destroy(kv.second.rec);
    sv->device_bytes -= e->warm_bytes;
  }
  e->warm.clear();
  if (e->plan) lrp_plan_destroy(e->plan);
  {
    SetupGuard guard;
    if (e->d_in) cudaFree(e->d_in);
    if (e->d_out) cudaFree(e->d_out);
    if (e->d_info) cudaFree(e->d_info);
  }
  sv->device_bytes -= e->bytes;
  delete e;
}

// Make room for `need` more device bytes by destroying idle plans, least
// recently used first.  Called with the lock held.
bool make_room(lrp_server_s* sv, size_t need, const PlanEntry* keep) {
  while (sv->device_bytes + need > (size_t)sv->opts.memory_cap_bytes) {
    PlanEntry* victim = nullptr;
    for (PlanEntry* e : sv->plans)
      if (!e->busy && e != keep && (!victim || e->last_used < victim->last_used)) victim = e;
    if (!victim) return false;
    sv->plans.erase(std::find(sv->plans.begin(), sv->plans.end(), victim));
    destroy_entry(sv, victim);
  }
  return true;
}

// An idle plan of bucket k (nullptr if none); *count receives the bucket's plans.
PlanEntry* find_idle_plan(lrp_server_s* sv, const BucketKey& k, int* count = nullptr) {
  PlanEntry* idle = nullptr;
  int c = 0;
  for (PlanEntry* e : sv->plans)
    if (e->key == k) {
      ++c;
      if (!e->busy && !idle) idle = e;
    }
  if (count) *count = c;
  return idle;
}

// The first waiting request that can start now: its bucket has an idle plan,
// or fewer plans than there are lanes (a lane may build another one, so that
// requests arriving while a batch of their bucket runs need not wait for it).
// Lock held.
Request* next_runnable(lrp_server_s* sv) {
  for (Request* r : sv->queue) {
    int count = 0;
    if (find_idle_plan(sv, r->key, &count) || count < sv->opts.lanes) return r;
  }
  return nullptr;
}

void finish(lrp_server_s* sv, Request* r, lrp_status status) {
  r->result.status = status;
  r->result.latency_us = us_between(r->t_submit, Clock::now());
  r->result.queue_us = us_between(r->t_submit, r->t_start);
  r->done = true;
  sv->admitted_bytes -= r->footprint;
  sv->completed += 1;
  sv->latencies.push_back(r->result.latency_us);
}

// Creates the plan and slot buffers of an entry (lock not held; the entry is
// marked busy by the caller, so no other lane touches it).
lrp_status build_entry(lrp_server_s* sv, PlanEntry* e) {
  lrp_opts o = plan_opts(e->key, e->B);
  lrp_status s = lrp_plan(&e->plan, e->key.n, e->key.tol, e->key.max_rank, &o);
  if (s != LRP_OK) return s;
  e->in_stride = (size_t)(2 * e->key.n + 1) * e->key.rf_cap;
  e->out_stride = (size_t)(2 * e->key.n + 1) * e->key.max_rank;
  SetupGuard guard;
  if (cudaMalloc((void**)&e->d_in, sizeof(double) * e->in_stride * e->B) != cudaSuccess ||
      cudaMalloc((void**)&e->d_out, sizeof(double) * e->out_stride * e->B) != cudaSuccess ||
      cudaMalloc((void**)&e->d_info, sizeof(lrp_info) * e->B) != cudaSuccess) {
    cudaGetLastError();
    return set_error(LRP_ENOMEM, "server slot buffers");
  }
  return LRP_OK;
}

struct LaneBuffers {
  double* pinned = nullptr;
  size_t cap = 0;
  double* need(size_t count) {
    if (count <= cap) return pinned;
    SetupGuard guard;
    if (pinned) cudaFreeHost(pinned);
    pinned = nullptr;
    cap = 0;
    if (cudaMallocHost((void**)&pinned, count * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    cap = count;
    return pinned;
  }
  ~LaneBuffers() {
    SetupGuard guard;
    if (pinned) cudaFreeHost(pinned);
  }
};

// Runs one batch of the entry's bucket; the lock is not held.
lrp_status run_batch(lrp_server_s* sv, PlanEntry* e, std::vector<Request*>& batch,
                     std::vector<WarmEntry*>& warms, cudaStream_t s, LaneBuffers& lb) {
  const int64_t n = e->key.n;
  const int rfc = e->key.rf_cap, rmax = e->key.max_rank;
  const int cnt = (int)batch.size();
  size_t total_in = 0;
  for (Request* r : batch) total_in += r->in.size();
  double* pin = lb.need(total_in);
  if (!pin) return set_error(LRP_ENOMEM, "server pinned staging");
  std::vector<lrp_problem> probs(cnt);
  size_t off = 0;
  for (int i = 0; i < cnt; ++i) {
    Request* r = batch[i];
    const int rf = r->r_f;
    memcpy(pin + off, r->in.data(), r->in.size() * sizeof(double));
    double* base = e->d_in + e->in_stride * i;
    double* dU = base;
    double* ds = base + (size_t)n * rfc;
    double* dV = ds + rfc;
    cudaMemcpyAsync(dU, pin + off, sizeof(double) * n * rf, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(ds, pin + off + (size_t)n * rf, sizeof(double) * rf, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(dV, pin + off + (size_t)n * rf + rf, sizeof(double) * n * rf, cudaMemcpyHostToDevice, s);
    off += r->in.size();
    double* ob = e->d_out + e->out_stride * i;
    lrp_problem& p = probs[i];
    memset(&p, 0, sizeof(p));
    p.r_f = rf;
    p.d_U_f = dU;
    p.ldu_f = n;
    p.d_s_f = ds;
    p.d_V_f = dV;
    p.ldv_f = n;
    p.d_U = ob;
    p.ldu = n;
    p.d_S = ob + (size_t)n * rmax;
    p.d_V = ob + (size_t)n * rmax + rmax;
    p.ldv = n;
    p.d_info = e->d_info + i;
    p.warm = warms[i] ? warms[i]->rec : nullptr;
  }
  lrp_status st = lrp_solve_batch(e->plan, cnt, probs.data(), (void*)s);
  if (st != LRP_OK) return st;
  std::vector<lrp_info> info(cnt);
  if (cudaMemcpyAsync(info.data(), e->d_info, sizeof(lrp_info) * cnt, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return set_error(LRP_ECUDA, "server result copy");
  for (int i = 0; i < cnt; ++i) {
    Request* r = batch[i];
    const int rank = std::max(0, std::min(info[i].rank, rmax));
    const double* ob = e->d_out + e->out_stride * i;
    if (rank > 0) {
      cudaMemcpyAsync(r->U, ob, sizeof(double) * n * rank, cudaMemcpyDeviceToHost, s);
      cudaMemcpyAsync(r->S, ob + (size_t)n * rmax, sizeof(double) * rank, cudaMemcpyDeviceToHost, s);
      cudaMemcpyAsync(r->V, ob + (size_t)n * rmax + rmax, sizeof(double) * n * rank, cudaMemcpyDeviceToHost, s);
    }
    r->result.rank = rank;
    r->result.iterations = info[i].total_iterations;
    r->solve_status = (lrp_status)info[i].status;
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return set_error(LRP_ECUDA, "server result copy");
  return LRP_OK;
}

void lane_main(lrp_server_s* sv) {
  cudaSetDevice(sv->device);
  cudaStream_t s = nullptr;
  {
    SetupGuard guard;
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  }
  LaneBuffers lb;
  std::unique_lock<std::mutex> lk(sv->mu);
  for (;;) {
    sv->cv.wait(lk, [&] { return (sv->stop && sv->queue.empty()) || next_runnable(sv) != nullptr; });
    Request* head = next_runnable(sv);
    if (!head) {
      if (sv->stop && sv->queue.empty()) break;
      continue;
    }
    const BucketKey key = head->key;
    PlanEntry* e = find_idle_plan(sv, key);
    if (head->warm_key) {
      // prefer an idle plan of the bucket that holds the request's warm-start record
      for (PlanEntry* c : sv->plans)
        if (c->key == key && !c->busy && c->warm.count(head->warm_key)) {
          e = c;
          break;
        }
    }
    bool fresh = false;
    if (!e) {
      int B = 1;
      size_t bytes = 0;
      lrp_status ps = plan_batch(sv->opts, key, &B, &bytes);
      if (ps != LRP_OK) {
        // the bucket cannot be served: fail its waiting requests
        for (auto it = sv->queue.begin(); it != sv->queue.end();) {
          if ((*it)->key == key) {
            (*it)->t_start = Clock::now();
            finish(sv, *it, ps);
            it = sv->queue.erase(it);
          } else {
            ++it;
          }
        }
        sv->done_cv.notify_all();
        continue;
      }
      if (!make_room(sv, bytes, nullptr)) {
        // every other plan is busy: wait for one to finish
        sv->done_cv.wait_for(lk, std::chrono::milliseconds(5));
        continue;
      }
      e = new PlanEntry();
      e->key = key;
      e->B = B;
      e->bytes = bytes;
      e->warm_bytes = warm_record_bytes(key);
      sv->plans.push_back(e);
      sv->device_bytes += bytes;
      fresh = true;
    }
    e->busy = true;
    e->last_used = ++sv->clock;
    // Gather the batch: waiting requests of this bucket in arrival order, one
    // request per warm-start key.
    std::vector<Request*> batch;
    std::vector<uint64_t> keys;
    for (auto it = sv->queue.begin(); it != sv->queue.end() && (int)batch.size() < e->B;) {
      Request* r = *it;
      bool take = r->key == key;
      if (take && r->warm_key && std::find(keys.begin(), keys.end(), r->warm_key) != keys.end()) take = false;
      if (take) {
        if (r->warm_key) keys.push_back(r->warm_key);
        r->t_start = Clock::now();
        batch.push_back(r);
        it = sv->queue.erase(it);
      } else {
        ++it;
      }
    }
    sv->running += (int)batch.size();
    // Warm-start records: existing ones are reused, new keys get a record
    // while the per-plan capacity and the memory cap allow.
    std::vector<WarmEntry*> warms(batch.size(), nullptr);
    std::vector<WarmEntry*> fresh_warms;
    for (size_t i = 0; i < batch.size(); ++i) {
      const uint64_t wk = batch[i]->warm_key;
      if (!wk) continue;
      auto it = e->warm.find(wk);
      if (it != e->warm.end()) {
        warms[i] = &it->second;
        batch[i]->result.warm_used = it->second.filled ? 1 : 0;
        it->second.last_used = ++sv->clock;
        continue;
      }
      if ((int)e->warm.size() >= sv->opts.warm_capacity) {
        // drop this plan's least recently used record not in the batch
        auto victim = e->warm.end();
        for (auto jt = e->warm.begin(); jt != e->warm.end(); ++jt) {
          if (std::find(keys.begin(), keys.end(), jt->first) != keys.end()) continue;
          if (victim == e->warm.end() || jt->second.last_used < victim->second.last_used) victim = jt;
        }
        if (victim == e->warm.end()) continue;
        lrp_warm_destroy(victim->second.rec);
        e->warm.erase(victim);
        sv->device_bytes -= e->warm_bytes;
      }
      if (!make_room(sv, e->warm_bytes, e)) continue;
      WarmEntry& we = e->warm[wk];
      we.last_used = ++sv->clock;
      sv->device_bytes += e->warm_bytes;
      fresh_warms.push_back(&we);
      warms[i] = &we;
    }
    lk.unlock();
    lrp_status st = LRP_OK;
    if (fresh) st = build_entry(sv, e);
    for (WarmEntry* w : fresh_warms)
      if (st == LRP_OK && lrp_warm_create(e->plan, &w->rec) != LRP_OK) w->rec = nullptr;
    for (size_t i = 0; i < warms.size(); ++i)
      if (warms[i] && !warms[i]->rec) warms[i] = nullptr;
    if (st == LRP_OK) st = run_batch(sv, e, batch, warms, s, lb);
    const std::string err = (st != LRP_OK) ? std::string(lrp_last_error()) : std::string();
    lk.lock();
    if (st != LRP_OK) sv->last_error = err;
    for (size_t i = 0; i < batch.size(); ++i) {
      if (st == LRP_OK && warms[i]) warms[i]->filled = true;
      finish(sv, batch[i], st == LRP_OK ? batch[i]->solve_status : st);
    }
    // records whose creation failed are dropped again
    for (auto it = e->warm.begin(); it != e->warm.end();) {
      if (!it->second.rec) {
        sv->device_bytes -= e->warm_bytes;
        it = e->warm.erase(it);
      } else {
        ++it;
      }
    }
    sv->running -= (int)batch.size();
    e->busy = false;
    e->last_used = ++sv->clock;
    if (st != LRP_OK && fresh) {
      sv->plans.erase(std::find(sv->plans.begin(), sv->plans.end(), e));
      destroy_entry(sv, e);
    }
    sv->done_cv.notify_all();
    sv->cv.notify_all();
  }
  lk.unlock();
  cudaStreamSynchronize(s);
  SetupGuard guard;
  cudaStreamDestroy(s);
}

double percentile(std::vector<double> v, double q) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  // nearest rank
  size_t k = (size_t)std::ceil(q * (double)v.size());
  if (k < 1) k = 1;
  if (k > v.size()) k = v.size();
  return v[k - 1];
}

}  // namespace

extern "C" lrp_status lrp_server_default_opts(lrp_server_opts* o) {
  if (!o) return set_error(LRP_EINVAL, "NULL opts");
  memset(o, 0, sizeof(*o));
  o->memory_cap_bytes = (int64_t)40 << 30;
  o->lanes = 2;
  o->max_batch = 64;
  o->max_queue = 65536;
  o->warm_capacity = 64;
  return LRP_OK;
}

extern "C" size_t lrp_request_footprint(int64_t n, int32_t r_f, int32_t max_rank) {
  if (n < 1 || r_f < 1 || max_rank < 1) return 0;
  return request_footprint(n, r_f, max_rank);
}

extern "C" lrp_status lrp_server_create(lrp_server_t* out, const lrp_server_opts* opts) {
  if (!out) return set_error(LRP_EINVAL, "out is NULL");
  *out = nullptr;
  lrp_server_opts o;
  lrp_server_default_opts(&o);
  if (opts) o = *opts;
  if (o.memory_cap_bytes <= 0 || o.lanes < 1 || o.lanes > 16 || o.max_batch < 1 || o.max_queue < 1 ||
      o.warm_capacity < 0)
    return set_error(LRP_EINVAL, "server options out of range");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return set_error(LRP_ECUDA, "no CUDA device");
  lrp_server_s* sv = new (std::nothrow) lrp_server_s();
  if (!sv) return set_error(LRP_ENOMEM, "host allocation failed");
  sv->opts = o;
  sv->device = dev;
  for (int i = 0; i < o.lanes; ++i) sv->lanes.emplace_back(lane_main, sv);
  *out = sv;
  return LRP_OK;
}

extern "C" lrp_status lrp_submit(lrp_server_t sv, const lrp_request* req, uint64_t* ticket) {
  if (!sv || !req || !ticket) return set_error(LRP_EINVAL, "NULL argument");
  *ticket = 0;
  const int64_t n = req->n;
  if (n < 1 || ((n + 1) & n) != 0) return set_error(LRP_EINVAL, "n+1 must be a power of two");
  if (req->r_f < 1 || req->max_rank < 1 || !(req->tol > 0.0) || !(req->tol < 1.0))
    return set_error(LRP_EINVAL, "r_f, max_rank or tol out of range");
  if (req->precision != LRP_FP64 && req->precision != LRP_MIXED) return set_error(LRP_EINVAL, "unknown precision");
  if (!req->U_f || !req->s_f || !req->V_f || !req->U || !req->S || !req->V)
    return set_error(LRP_EINVAL, "NULL factor pointer");
  BucketKey key{n, req->precision, req->max_rank, rf_class(req->r_f), req->tol};
  {
    // a request whose plan cannot be built at all, or whose single-slot plan
    // exceeds the cap, is refused outright
    lrp_opts o = plan_opts(key, 1);
    size_t bytes = 0;
    lrp_status s = lrp_plan_estimate_bytes(n, req->tol, req->max_rank, &o, &bytes);
    if (s != LRP_OK) return s;
    if (bytes + slot_buffer_bytes(key) > (size_t)sv->opts.memory_cap_bytes)
      return set_error(LRP_ECAPACITY, "request exceeds the server memory cap");
  }
  const size_t fp = request_footprint(n, req->r_f, req->max_rank, req->precision);
  if (fp > (size_t)sv->opts.memory_cap_bytes) return set_error(LRP_ECAPACITY, "request exceeds the server memory cap");
  Request* r = new (std::nothrow) Request();
  if (!r) return set_error(LRP_ENOMEM, "host allocation failed");
  r->key = key;
  r->r_f = req->r_f;
  r->warm_key = req->warm_key;
  r->U = req->U;
  r->S = req->S;
  r->V = req->V;
  r->footprint = fp;
  try {
    r->in.resize((size_t)(2 * n + 1) * req->r_f);
  } catch (...) {
    delete r;
    return set_error(LRP_ENOMEM, "host allocation failed");
  }
  memcpy(r->in.data(), req->U_f, sizeof(double) * n * req->r_f);
  memcpy(r->in.data() + (size_t)n * req->r_f, req->s_f, sizeof(double) * req->r_f);
  memcpy(r->in.data() + (size_t)n * req->r_f + req->r_f, req->V_f, sizeof(double) * n * req->r_f);
  std::lock_guard<std::mutex> lock(sv->mu);
  if (sv->stop) {
    delete r;
    return set_error(LRP_EINVAL, "server is shutting down");
  }
  if ((int)sv->queue.size() >= sv->opts.max_queue || sv->admitted_bytes + fp > (size_t)sv->opts.memory_cap_bytes) {
    sv->rejected += 1;
    delete r;
    return LRP_EAGAIN;
  }
  r->ticket = sv->next_ticket++;
  r->t_submit = Clock::now();
  sv->admitted_bytes += fp;
  sv->submitted += 1;
  sv->tickets[r->ticket] = r;
  sv->queue.push_back(r);
  *ticket = r->ticket;
  sv->cv.notify_one();
  return LRP_OK;
}

static lrp_status take_result(lrp_server_s* sv, uint64_t ticket, lrp_result* out) {
  auto it = sv->tickets.find(ticket);
  if (it == sv->tickets.end()) return set_error(LRP_EINVAL, "unknown ticket");
  if (!it->second->done) return LRP_EAGAIN;
  *out = it->second->result;
  delete it->second;
  sv->tickets.erase(it);
  return LRP_OK;
}

extern "C" lrp_status lrp_poll(lrp_server_t sv, uint64_t ticket, lrp_result* out) {
  if (!sv || !out) return set_error(LRP_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lock(sv->mu);
  return take_result(sv, ticket, out);
}

extern "C" lrp_status lrp_wait(lrp_server_t sv, uint64_t ticket, lrp_result* out, int64_t timeout_us) {
  if (!sv || !out) return set_error(LRP_EINVAL, "NULL argument");
  std::unique_lock<std::mutex> lk(sv->mu);
  const auto deadline = Clock::now() + std::chrono::microseconds(timeout_us < 0 ? 0 : timeout_us);
  for (;;) {
    lrp_status s = take_result(sv, ticket, out);
    if (s != LRP_EAGAIN) return s;
    if (sv->done_cv.wait_until(lk, deadline) == std::cv_status::timeout) {
      s = take_result(sv, ticket, out);
      return s == LRP_EAGAIN ? LRP_ETIMEDOUT : s;
    }
  }
}

extern "C" lrp_status lrp_server_get_stats(lrp_server_t sv, lrp_server_stats* out) {
  if (!sv || !out) return set_error(LRP_EINVAL, "NULL argument");
  std::vector<double> lat;
  {
    std::lock_guard<std::mutex> lock(sv->mu);
    memset(out, 0, sizeof(*out));
    out->submitted = sv->submitted;
    out->completed = sv->completed;
    out->rejected = sv->rejected;
    out->queued = (int64_t)sv->queue.size();
    out->running = sv->running;
    out->plans = (int64_t)sv->plans.size();
    out->device_bytes = (int64_t)sv->device_bytes;
    out->admitted_bytes = (int64_t)sv->admitted_bytes;
    lat = sv->latencies;
  }
  if (!lat.empty()) {
    double sum = 0.0, mx = 0.0;
    for (double v : lat) {
      sum += v;
      mx = std::max(mx, v);
    }
    out->mean_us = sum / (double)lat.size();
    out->max_us = mx;
    out->p50_us = percentile(lat, 0.50);
    out->p99_us = percentile(lat, 0.99);
  }
  return LRP_OK;
}

extern "C" lrp_status lrp_server_last_error(lrp_server_t sv, char* buf, size_t len) {
  if (!sv || !buf || len == 0) return set_error(LRP_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lock(sv->mu);
  const size_t k = std::min(len - 1, sv->last_error.size());
  memcpy(buf, sv->last_error.data(), k);
  buf[k] = 0;
  return LRP_OK;
}

extern "C" lrp_status lrp_server_reset_stats(lrp_server_t sv) {
  if (!sv) return set_error(LRP_EINVAL, "NULL server");
  std::lock_guard<std::mutex> lock(sv->mu);
  sv->latencies.clear();
  sv->submitted = sv->completed = sv->rejected = 0;
  return LRP_OK;
}

extern "C" lrp_status lrp_server_destroy(lrp_server_t sv) {
  if (!sv) return LRP_OK;
  {
    std::lock_guard<std::mutex> lock(sv->mu);
    sv->stop = true;
  }
  sv->cv.notify_all();
  for (auto& t : sv->lanes) t.join();
  cudaSetDevice(sv->device);
  {
    SetupGuard guard;
    cudaDeviceSynchronize();
  }
  for (PlanEntry* e : sv->plans) destroy_entry(sv, e);
  sv->plans.clear();
  for (auto& kv : sv->tickets) delete kv.second;
  delete sv;
  return LRP_OK;
}
