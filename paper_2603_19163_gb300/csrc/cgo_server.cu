// Serving loop: continuous batching of solve requests.
//
// A host thread owns one non-blocking stream and a table of device slots.
// Between time slices it admits queued requests (first come, first served)
// into free slots while their device-memory footprint fits the budget,
// initialises their populations, rewrites the per-bucket work lists, then
// replays one captured slice (a persistent batched kernel per bucket on
// forked streams) that advances every resident request by up to its
// model's slice length (`slice_by_model`, else `slice_generations`).  The
// slice lasts as long as its slowest bucket, so cheap models may take more
// generations per slice.  Requests that reach their budget are retired and their
// waiters woken; requests that arrive mid-slice join at the next boundary.
// Populations, AOS weights, temperatures and generation counters stay in
// device memory across slices.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "cgo_host.h"

using namespace cgo;
using namespace cgo::host;

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
  uint64_t ticket = 0;
  cgo_problem *prob = nullptr;
  cgo_params params{};
  uint64_t seed = 0;
  uint32_t enabled = 0;
  Clock::time_point t_submit, t_done;
  int64_t bytes = 0;   // device memory charged against the budget
  int slot = -1, bucket = -1;
  int64_t g = 0;
  int64_t cost = 0;
  cgo_status status = CGO_OK;
  bool done = false;
  std::atomic<bool> cancel{false};  // cgo_cancel of a resident request
  KInst h{};
};

struct SBucket {
  int model, tri16, xf, wpm, warps;
  int64_t smem;
  int grid;
  int64_t slice;  // generations per slice of its requests
};

constexpr int kMaxBuckets = 16;

}  // namespace

struct cgo_server {
  cgo_server_cfg cfg{};
  int device = 0;
  std::thread th;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  uint64_t next_ticket = 1;
  std::deque<Req *> queue;
  std::unordered_map<uint64_t, Req *> reqs;
  std::vector<Req *> slot_req;
  std::vector<int> free_slots;
  int64_t hbm_used = 0;
  int active = 0;
  // device side (server thread only)
  cudaStream_t st = nullptr;
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> evs;
  KInst *d_k = nullptr;
  int *d_lists = nullptr, *d_counts = nullptr, *d_next = nullptr;
  std::vector<SBucket> buckets;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool dirty = true;
  int sms = 0;
  // counters
  uint64_t slices = 0, completed = 0;
  cgo_status fatal = CGO_OK;
  std::string fatal_msg;
};

namespace {

int64_t request_bytes(const cgo_problem *p, const cgo_params &q) {
  const int64_t P = q.population, len = p->len;
  int64_t data = 0;
  switch (p->model) {
    case TSP:
      data = (int64_t)p->n * p->n * 4 +
             (p->asym ? (int64_t)p->n * p->n : (int64_t)p->n * (p->n + 1) / 2) * (p->tri16 ? 2 : 4);
      break;
    case QAP: data = 2ll * p->n * p->n * 4; break;
    case KNAPSACK: data = 2ll * p->n * 4; break;
    case GAP: data = 2ll * p->m * p->n * 4 + 4ll * p->m; break;
    case CVRPTW: data = (int64_t)(p->n + 1) * (p->n + 1) * 4 + 16ll * (p->n + 1); break;
  }
  const int64_t pool = pool_size(p, q) * (len * 4 + 8);
  return data + 2 * P * len * 4 + 16 * P + 2 * (int64_t)sizeof(DevAos) + (int64_t)sizeof(DevSync) +
         pool;
}

cudaError_t capture_slice(cgo_server *S) {
  if (S->exec) cudaGraphExecDestroy(S->exec);
  if (S->graph) cudaGraphDestroy(S->graph);
  S->exec = nullptr;
  S->graph = nullptr;
  cudaStream_t cap = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) return e;
  e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  cudaError_t ce = cudaSuccess;
  if (e == cudaSuccess) {
    ce = cudaEventRecord(S->evs[kMaxBuckets], cap);
    for (size_t b = 0; b < S->buckets.size() && ce == cudaSuccess; ++b) {
      const SBucket &bk = S->buckets[b];
      ce = cudaStreamWaitEvent(S->side[b], S->evs[kMaxBuckets], 0);
      if (ce == cudaSuccess) ce = cudaMemsetAsync(S->d_next + b, 0, sizeof(int), S->side[b]);
      if (ce == cudaSuccess)
        ce = launch_batch(bk.model, bk.tri16, bk.xf, S->d_k, S->d_lists + b * S->cfg.max_slots,
                          S->d_counts + b, S->d_next + b, bk.warps, bk.wpm, bk.smem, bk.grid,
                          bk.slice, 10ull * 1000 * 1000 * 1000, S->side[b]);
      if (ce == cudaSuccess) ce = cudaEventRecord(S->evs[b], S->side[b]);
      if (ce == cudaSuccess) ce = cudaStreamWaitEvent(cap, S->evs[b], 0);
    }
    const cudaError_t ee = cudaStreamEndCapture(cap, &S->graph);
    e = ce != cudaSuccess ? ce : ee;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&S->exec, S->graph, 0);
  cudaStreamDestroy(cap);
  S->dirty = false;
  return e;
}

// generations per slice of a request of public model `model`
int64_t slice_of(const cgo_server *S, int model) {
  const int64_t v = model >= 0 && model < 5 ? S->cfg.slice_by_model[model] : 0;
  return v > 0 ? v : S->cfg.slice_generations;
}

// bucket of a request (created on first use; the graph is recaptured then)
int bucket_for(cgo_server *S, int model, int tri16, int xf, int wpm, int warps, int64_t smem,
               int64_t slice) {
  for (size_t b = 0; b < S->buckets.size(); ++b) {
    const SBucket &k = S->buckets[b];
    if (k.model == model && k.tri16 == tri16 && k.xf == xf && k.wpm == wpm && k.warps == warps &&
        k.smem == smem && k.slice == slice)
      return (int)b;
  }
  if ((int)S->buckets.size() >= kMaxBuckets) return -1;
  const int per_sm = batch_ctas_per_sm(model, tri16, xf, warps, wpm, smem);
  if (per_sm <= 0) return -1;
  S->buckets.push_back(SBucket{model, tri16, xf, wpm, warps, smem,
                               std::max(1, std::min(S->cfg.max_slots, per_sm * S->sms)), slice});
  S->dirty = true;
  return (int)S->buckets.size() - 1;
}

void fail_all(cgo_server *S, cgo_status st, const char *msg) {
  std::lock_guard<std::mutex> lk(S->mu);
  S->fatal = st;
  S->fatal_msg = msg;
  for (auto &kv : S->reqs) {
    Req *r = kv.second;
    if (!r->done) {
      r->done = true;
      r->status = st;
      r->prob->busy.store(0);
    }
  }
  S->queue.clear();
  S->cv_done.notify_all();
}

void server_loop(cgo_server *S) {
  cudaSetDevice(S->device);
  std::vector<Req *> admitted;
  std::vector<int> lists((size_t)kMaxBuckets * S->cfg.max_slots), counts(kMaxBuckets);
  for (;;) {
    admitted.clear();
    {
      std::unique_lock<std::mutex> lk(S->mu);
      if (S->active == 0 && S->queue.empty()) {
        if (S->stop) return;
        S->cv_work.wait_for(lk, std::chrono::milliseconds(20));
        continue;
      }
      // admission: FIFO, while a slot is free and the memory budget allows
      while (!S->queue.empty() && !S->free_slots.empty()) {
        Req *r = S->queue.front();
        if (S->active > 0 && S->hbm_used + r->bytes > S->cfg.hbm_budget_bytes) break;
        S->queue.pop_front();
        r->slot = S->free_slots.back();
        S->free_slots.pop_back();
        S->slot_req[(size_t)r->slot] = r;
        S->hbm_used += r->bytes;
        S->active++;
        admitted.push_back(r);
      }
      if (S->stop && S->queue.empty() && S->active == 0) return;
    }
    // set up the admitted requests: state, description, initial population
    for (Req *r : admitted) {
      cgo_problem *p = r->prob;
      cgo_status s = ensure_state(p, r->params.population);
      if (s == CGO_OK) s = ensure_pool(p, r->params);
      if (s != CGO_OK) {
        // this request ends with the allocation error; the others carry on
        std::lock_guard<std::mutex> lk(S->mu);
        r->status = s;
        r->done = true;
        r->t_done = Clock::now();
        S->slot_req[(size_t)r->slot] = nullptr;
        S->free_slots.push_back(r->slot);
        S->hbm_used -= r->bytes;
        S->active--;
        r->slot = -1;
        p->busy.store(0);
        S->cv_done.notify_all();
        continue;
      }
      p->params = r->params;
      p->seed = r->seed;
      p->enabled = r->enabled;
      p->g = 0;
      p->aos_cur = 0;
      KInst h = base_kinst(p);
      h.aos_in = h.aos_out = p->d_aos;
      h.G_total = r->params.generations;
      h.local_sync = 1;
      int wpm = 1, warps = 1;
      int64_t need = 0, cls = 0;
      if (batch_shape(p, r->params, h, &wpm, &warps, &need, &cls) != CGO_OK ||
          (r->bucket = bucket_for(S, h.model, p->tri16, takes_xf(h) != 0 ? 1 : 0, wpm, warps, cls,
                                  slice_of(S, p->model))) < 0) {
        fail_all(S, CGO_ERR_UNSUPPORTED, "no batched launch shape for a request");
        return;
      }
      r->h = h;
      cudaError_t e = cudaMemcpyAsync(S->d_k + r->slot, &r->h, sizeof(KInst), cudaMemcpyHostToDevice, S->st);
      if (e == cudaSuccess) e = launch_init(h, S->st);
      if (e == cudaSuccess) e = launch_init_aos(h, initial_aos(r->params, r->enabled), S->st);
      if (e != cudaSuccess) {
        fail_all(S, CGO_ERR_CUDA, cudaGetErrorString(e));
        return;
      }
    }
    // work lists of the resident requests that still have generations left
    std::fill(counts.begin(), counts.end(), 0);
    for (size_t sl = 0; sl < S->slot_req.size(); ++sl) {
      Req *r = S->slot_req[sl];
      if (!r || r->g >= r->params.generations || r->cancel.load()) continue;
      lists[(size_t)r->bucket * S->cfg.max_slots + (size_t)counts[(size_t)r->bucket]++] = (int)sl;
    }
    cudaError_t e = cudaSuccess;
    for (size_t b = 0; b < S->buckets.size() && e == cudaSuccess; ++b)
      if (counts[b] > 0)
        e = cudaMemcpyAsync(S->d_lists + b * S->cfg.max_slots, &lists[b * S->cfg.max_slots],
                            sizeof(int) * (size_t)counts[b], cudaMemcpyHostToDevice, S->st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(S->d_counts, counts.data(), sizeof(int) * kMaxBuckets, cudaMemcpyHostToDevice,
                          S->st);
    if (e == cudaSuccess && S->dirty) e = capture_slice(S);
    if (e == cudaSuccess) e = cudaGraphLaunch(S->exec, S->st);
    if (e == cudaSuccess) note_launches(S->buckets.size());
    if (e == cudaSuccess) e = cudaStreamSynchronize(S->st);
    if (e != cudaSuccess) {
      fail_all(S, CGO_ERR_CUDA, cudaGetErrorString(e));
      return;
    }
    S->slices++;
    // retire the requests that reached their budget
    const Clock::time_point now = Clock::now();
    std::vector<Req *> finished;
    std::vector<Req *> cancelled;
    for (Req *r : S->slot_req) {
      if (!r) continue;
      if (r->cancel.load()) {
        cancelled.push_back(r);
        continue;
      }
      r->g = std::min<int64_t>(r->params.generations, r->g + S->buckets[(size_t)r->bucket].slice);
      if (r->g >= r->params.generations) finished.push_back(r);
    }
    std::vector<DevAos> aos(finished.size());
    for (size_t i = 0; i < finished.size() && e == cudaSuccess; ++i)
      e = cudaMemcpyAsync(&aos[i], finished[i]->prob->d_aos, sizeof(DevAos), cudaMemcpyDeviceToHost, S->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(S->st);
    for (size_t i = 0; i < finished.size(); ++i) {
      finished[i]->cost = aos[i].elite_cost;
      finished[i]->status = e == cudaSuccess ? CGO_OK : CGO_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    for (Req *r : finished) {
      cgo_problem *p = r->prob;
      p->g = r->params.generations;
      p->has_state = r->status == CGO_OK;
      p->last_wpm = S->buckets[(size_t)r->bucket].wpm;
      p->last_ns = 1;
      p->last_warps = S->buckets[(size_t)r->bucket].warps;
      p->last_staging = r->h.shared_bytes > 0 ? STAGE_SMEM : STAGE_GLOBAL;
      p->busy.store(0);
      r->t_done = now;
      r->done = true;
      S->slot_req[(size_t)r->slot] = nullptr;
      S->free_slots.push_back(r->slot);
      S->hbm_used -= r->bytes;
      S->active--;
      S->completed++;
    }
    for (Req *r : cancelled) {
      r->prob->has_state = false;
      r->prob->busy.store(0);
      r->status = CGO_ERR_CANCELLED;
      r->t_done = now;
      r->done = true;
      S->slot_req[(size_t)r->slot] = nullptr;
      S->free_slots.push_back(r->slot);
      S->hbm_used -= r->bytes;
      S->active--;
    }
    if (!finished.empty() || !cancelled.empty()) S->cv_done.notify_all();
  }
}

}  // namespace

extern "C" {

cgo_status cgo_server_create(const cgo_server_cfg *cfg, cgo_server **out) {
  if (!out) return fail(CGO_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!cfg || (cfg->struct_size != sizeof(cgo_server_cfg) && cfg->struct_size != CGO_SERVER_CFG_SIZE_V1 &&
               cfg->struct_size != CGO_SERVER_CFG_SIZE_V2))
    return fail(CGO_ERR_INVALID, "cfg: struct_size must be sizeof(cgo_server_cfg)");
  cgo_server_cfg c{};
  memcpy(&c, cfg, cfg->struct_size);
  c.struct_size = sizeof c;
  if (c.max_queued < 0) return fail(CGO_ERR_INVALID, "max_queued < 0");
  for (int i = 0; i < 5; ++i)
    if (c.slice_by_model[i] < 0) return fail(CGO_ERR_INVALID, "slice_by_model < 0");
  cfg = &c;
  if (cfg->max_slots < 1 || cfg->max_slots > 65536) return fail(CGO_ERR_INVALID, "max_slots out of [1, 65536]");
  if (cfg->slice_generations < 1) return fail(CGO_ERR_INVALID, "slice_generations < 1");
  if (cfg->hbm_budget_bytes < 1) return fail(CGO_ERR_INVALID, "hbm_budget_bytes < 1");
  cgo_server *S = new cgo_server();
  S->cfg = *cfg;
  cudaGetDevice(&S->device);
  cudaDeviceGetAttribute(&S->sms, cudaDevAttrMultiProcessorCount, S->device);
  auto bail = [&](cudaError_t e) {
    cgo_server_destroy(S);
    return cuda_fail(e, "server setup");
  };
  cudaError_t e;
  if ((e = cudaStreamCreateWithFlags(&S->st, cudaStreamNonBlocking)) != cudaSuccess) return bail(e);
  S->side.assign(kMaxBuckets, nullptr);
  S->evs.assign(kMaxBuckets + 1, nullptr);
  for (int b = 0; b < kMaxBuckets; ++b)
    if ((e = cudaStreamCreateWithFlags(&S->side[(size_t)b], cudaStreamNonBlocking)) != cudaSuccess) return bail(e);
  for (int b = 0; b <= kMaxBuckets; ++b)
    if ((e = cudaEventCreateWithFlags(&S->evs[(size_t)b], cudaEventDisableTiming)) != cudaSuccess) return bail(e);
  const size_t ms = (size_t)cfg->max_slots;
  if ((e = cudaMalloc((void **)&S->d_k, sizeof(KInst) * ms)) != cudaSuccess ||
      (e = cudaMalloc((void **)&S->d_lists, sizeof(int) * ms * kMaxBuckets)) != cudaSuccess ||
      (e = cudaMalloc((void **)&S->d_counts, sizeof(int) * kMaxBuckets)) != cudaSuccess ||
      (e = cudaMalloc((void **)&S->d_next, sizeof(int) * kMaxBuckets)) != cudaSuccess)
    return bail(e);
  cudaMemset(S->d_counts, 0, sizeof(int) * kMaxBuckets);
  S->slot_req.assign(ms, nullptr);
  for (int i = cfg->max_slots - 1; i >= 0; --i) S->free_slots.push_back(i);
  S->th = std::thread(server_loop, S);
  *out = S;
  return CGO_OK;
}

cgo_status cgo_submit(cgo_server *S, cgo_problem *p, const cgo_params *qin, uint64_t seed,
                      uint64_t *ticket) {
  if (!S || !p || !ticket) return fail(CGO_ERR_INVALID, "NULL argument");
  if (p->device != S->device) return fail(CGO_ERR_INVALID, "problem lives on another device");
  cgo_params qq;
  cgo_status s = load_params(qin, &qq);
  if (s != CGO_OK) return s;
  const cgo_params *q = &qq;
  uint32_t en = 0;
  s = validate_params(p, q, &en);
  if (s != CGO_OK) return s;
  if (q->generations >= 0xFFFFFFFFll) return fail(CGO_ERR_INVALID, "too many generations");
  {
    KInst h = base_kinst(p);
    int wpm = 1, warps = 1;
    int64_t need = 0, cls = 0;
    if ((s = batch_shape(p, *q, h, &wpm, &warps, &need, &cls)) != CGO_OK) return s;
    if (need > S->cfg.smem_budget_bytes && S->cfg.smem_budget_bytes > 0)
      return fail(CGO_ERR_UNSUPPORTED, "request needs %lld bytes of shared memory; the budget is %lld",
                  (long long)need, (long long)S->cfg.smem_budget_bytes);
  }
  int z = 0;
  if (!p->busy.compare_exchange_strong(z, 1)) return fail(CGO_ERR_BUSY, "problem handle in use");
  Req *r = new Req();
  r->prob = p;
  r->params = *q;
  r->seed = seed;
  r->enabled = en;
  r->bytes = request_bytes(p, *q);
  r->t_submit = Clock::now();
  p->has_state = false;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop || S->fatal != CGO_OK) {
      p->busy.store(0);
      delete r;
      return fail(CGO_ERR_STATE, "server is stopping or failed");
    }
    if (S->cfg.max_queued > 0 && (int64_t)S->queue.size() >= S->cfg.max_queued) {
      p->busy.store(0);
      delete r;
      return fail(CGO_ERR_BUSY, "the submit queue holds %d requests (max_queued)", S->cfg.max_queued);
    }
    r->ticket = S->next_ticket++;
    S->reqs[r->ticket] = r;
    S->queue.push_back(r);
  }
  S->cv_work.notify_one();
  *ticket = r->ticket;
  return CGO_OK;
}

cgo_status cgo_wait(cgo_server *S, uint64_t ticket, int32_t timeout_ms, int64_t *cost,
                    double *latency_s) {
  if (!S) return fail(CGO_ERR_INVALID, "NULL server");
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return fail(CGO_ERR_INVALID, "unknown ticket %llu", (unsigned long long)ticket);
  Req *r = it->second;
  auto ready = [&] { return r->done; };
  if (timeout_ms < 0) S->cv_done.wait(lk, ready);
  else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
    return fail(CGO_ERR_TIMEOUT, "ticket %llu not finished", (unsigned long long)ticket);
  const cgo_status st = r->status;
  if (cost) *cost = r->cost;
  if (latency_s) *latency_s = std::chrono::duration<double>(r->t_done - r->t_submit).count();
  S->reqs.erase(it);
  delete r;
  if (st == CGO_ERR_CANCELLED) return fail(st, "ticket %llu was cancelled", (unsigned long long)ticket);
  if (st == CGO_ERR_NOMEM) return fail(st, "ticket %llu: no device memory for its state", (unsigned long long)ticket);
  if (st != CGO_OK) return fail(st, "request failed: %s", S->fatal_msg.c_str());
  return CGO_OK;
}

cgo_status cgo_cancel(cgo_server *S, uint64_t ticket) {
  if (!S) return fail(CGO_ERR_INVALID, "NULL server");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return fail(CGO_ERR_INVALID, "unknown ticket %llu", (unsigned long long)ticket);
  Req *r = it->second;
  if (r->done) return fail(CGO_ERR_STATE, "ticket %llu has finished", (unsigned long long)ticket);
  auto q = std::find(S->queue.begin(), S->queue.end(), r);
  if (q != S->queue.end()) {
    // not admitted yet: it finishes now
    S->queue.erase(q);
    r->prob->has_state = false;
    r->prob->busy.store(0);
    r->status = CGO_ERR_CANCELLED;
    r->t_done = Clock::now();
    r->done = true;
    S->cv_done.notify_all();
    return CGO_OK;
  }
  r->cancel.store(true);  // resident: retired at the next slice boundary
  return CGO_OK;
}

cgo_status cgo_server_stats(const cgo_server *S, cgo_server_info *out) {
  if (!S || !out || out->struct_size != sizeof(cgo_server_info)) return fail(CGO_ERR_INVALID, "bad arguments");
  cgo_server *M = const_cast<cgo_server *>(S);
  std::lock_guard<std::mutex> lk(M->mu);
  out->slices = (int64_t)S->slices;
  out->completed = (int64_t)S->completed;
  out->queued = (int32_t)S->queue.size();
  out->active = S->active;
  out->hbm_used_bytes = S->hbm_used;
  out->buckets = (int32_t)S->buckets.size();
  return CGO_OK;
}

cgo_status cgo_server_destroy(cgo_server *S) {
  if (!S) return CGO_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->th.joinable()) S->th.join();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    for (auto &kv : S->reqs) {
      Req *r = kv.second;
      if (!r->done) r->prob->busy.store(0);
      delete r;
    }
    S->reqs.clear();
  }
  if (S->exec) cudaGraphExecDestroy(S->exec);
  if (S->graph) cudaGraphDestroy(S->graph);
  for (auto x : S->side)
    if (x) cudaStreamDestroy(x);
  for (auto x : S->evs)
    if (x) cudaEventDestroy(x);
  if (S->st) cudaStreamDestroy(S->st);
  cudaFree(S->d_k);
  cudaFree(S->d_lists);
  cudaFree(S->d_counts);
  cudaFree(S->d_next);
  delete S;
  return CGO_OK;
}

}  // extern "C"
