// Host runtime and C ABI of the cgo library: validation, device copies of
// the instance data, search-state buffers, the launch-shape choice and the
// launch sequence init -> evolve (cooperative) -> finalize.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <climits>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "cgo_host.h"

using namespace cgo;
using namespace cgo::host;

namespace cgo {
namespace host {

thread_local std::string g_err;

cgo_status fail(cgo_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

cgo_status cuda_fail(cudaError_t e, const char *what) {
  if (e == cudaErrorMemoryAllocation) return fail(CGO_ERR_NOMEM, "%s: %s", what, cudaGetErrorString(e));
  return fail(CGO_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

int64_t pad16(int64_t b) { return (b + 15) & ~int64_t(15); }

int encoding_of(int model) {
  if (model == KNAPSACK) return CGO_ENC_BINARY;
  if (model == GAP) return CGO_ENC_INTEGER;
  return CGO_ENC_PERM;
}

}  // namespace host
}  // namespace cgo


namespace cgo {
namespace host {


// Per-thread, per-device non-blocking stream for the library's own
// allocations, copies and frees.  Allocation is stream-ordered
// (cudaMallocAsync from the device pool, which keeps freed memory cached),
// so creating or destroying a problem never waits for kernels other threads
// have in flight (a serving loop, for one).
cudaStream_t host_stream() {
  thread_local cudaStream_t streams[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!streams[dev]) {
    cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking);
    static std::mutex mu;
    static bool pool_set[64] = {};
    std::lock_guard<std::mutex> lk(mu);
    if (!pool_set[dev]) {
      cudaMemPool_t pool;
      if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
      }
      pool_set[dev] = true;
    }
  }
  return streams[dev];
}

cudaError_t copy_sync(void *dst, const void *src, size_t bytes, cudaMemcpyKind kind) {
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, kind, host_stream());
  return e != cudaSuccess ? e : cudaStreamSynchronize(host_stream());
}

// test hook: the n-th device allocation from now on fails (0 = off)
static std::atomic<int64_t> g_alloc_fail{0};
bool alloc_fails() {
  int64_t v = g_alloc_fail.load();
  while (v > 0)
    if (g_alloc_fail.compare_exchange_weak(v, v - 1)) return v == 1;
  return false;
}
cudaError_t lib_malloc_async(void **p, size_t bytes, cudaStream_t st) {
  if (alloc_fails()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMallocAsync(p, bytes, st);
}
cudaError_t dev_alloc(void **p, size_t bytes) { return lib_malloc_async(p, bytes, host_stream()); }
void dev_free(void *p) {
  if (p) cudaFreeAsync(p, host_stream());
}

cudaError_t copy_in(int32_t **dst, const int32_t *src, int64_t count, bool on_device) {
  const int64_t bytes = pad16(count * 4);
  cudaStream_t hs = host_stream();
  cudaError_t e = lib_malloc_async((void **)dst, (size_t)bytes, hs);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(*dst, 0, (size_t)bytes, hs);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(*dst, src, (size_t)(count * 4),
                      on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, hs);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(hs);
}

// host copy of caller data (for validation), whether it is on host or device
cgo_status host_copy(const int32_t *src, int64_t count, bool on_device, std::vector<int32_t> &out) {
  out.resize((size_t)count);
  if (count == 0) return CGO_OK;
  if (!src) return fail(CGO_ERR_INVALID, "missing data array");
  if (on_device) {
    CUDA_TRY(cudaMemcpyAsync(out.data(), src, (size_t)count * 4, cudaMemcpyDeviceToHost, host_stream()),
             "reading device data");
    CUDA_TRY(cudaStreamSynchronize(host_stream()), "reading device data");
  } else {
    memcpy(out.data(), src, (size_t)count * 4);
  }
  return CGO_OK;
}

int64_t absmax(const std::vector<int32_t> &v) {
  int64_t m = 0;
  for (int32_t x : v) m = std::max<int64_t>(m, x < 0 ? -(int64_t)x : (int64_t)x);
  return m;
}
int64_t maxval(const std::vector<int32_t> &v) {
  int64_t m = INT64_MIN;
  for (int32_t x : v) m = std::max<int64_t>(m, x);
  return m;
}
int64_t abssum(const std::vector<int32_t> &v) {
  int64_t s = 0;
  for (int32_t x : v) s += x < 0 ? -(int64_t)x : (int64_t)x;
  return s;
}

const double kLimit = 4.6e18;  // 2^62: every cost and delta fits in int64 with room
int64_t g_batch_slice = 2000;  // generations per batched time slice

void free_state(cgo_problem *p) {
  dev_free(p->d_cur);
  dev_free(p->d_bestsol);
  dev_free(p->d_cost);
  dev_free(p->d_best);
  dev_free(p->d_aos);
  dev_free(p->d_sync);
  p->d_cur = p->d_bestsol = nullptr;
  p->d_cost = p->d_best = nullptr;
  p->d_aos = nullptr;
  p->d_sync = nullptr;
  p->P_alloc = 0;
  p->has_state = false;
}

// Sec. 3.4.2: the orders of ascending and descending row sums, then of
// ascending and descending column sums, of an n x n matrix (ties: lower
// index first), appended to out.
void heuristic_perms(const std::vector<int32_t> &M, int64_t n, std::vector<int32_t> &out) {
  std::vector<int64_t> s((size_t)n);
  std::vector<int32_t> idx((size_t)n);
  for (int by_col = 0; by_col < 2; ++by_col) {
    for (int64_t i = 0; i < n; ++i) {
      int64_t t = 0;
      for (int64_t j = 0; j < n; ++j) t += by_col ? M[(size_t)(j * n + i)] : M[(size_t)(i * n + j)];
      s[(size_t)i] = t;
    }
    for (int desc = 0; desc < 2; ++desc) {
      for (int64_t i = 0; i < n; ++i) idx[(size_t)i] = (int32_t)i;
      std::stable_sort(idx.begin(), idx.end(), [&](int32_t x, int32_t y) {
        return desc ? s[(size_t)x] > s[(size_t)y] : s[(size_t)x] < s[(size_t)y];
      });
      out.insert(out.end(), idx.begin(), idx.end());
    }
  }
}

// rows of the scratch solution buffer: the start pool's entries (0: plain
// start), or with crossover three rows per member (its child, and its best
// as a crossover parent in two alternating rows), whichever is more
int64_t pool_size(const cgo_problem *p, const cgo_params &q) {
  const int64_t K = q.init_oversample > 1 ? q.init_oversample : 1;
  const int64_t H = q.init_heuristic ? p->n_heur : 0;
  const int64_t pool = (K > 1 || H > 0) ? K * q.population + H : 0;
  const int64_t cross = (q.cross_q16 > 0 && q.population >= 2) ? 3 * (int64_t)q.population : 0;
  return pool > cross ? pool : cross;
}

cgo_status ensure_pool(cgo_problem *p, const cgo_params &q) {
  const int64_t N = pool_size(p, q);
  if (N <= p->pool_cap) return CGO_OK;
  dev_free(p->d_pool);
  dev_free(p->d_pool_cost);
  p->d_pool = nullptr;
  p->d_pool_cost = nullptr;
  p->pool_cap = 0;
  cudaError_t e = dev_alloc((void **)&p->d_pool, (size_t)N * p->len * 4);
  if (e == cudaSuccess) e = dev_alloc((void **)&p->d_pool_cost, (size_t)N * 8);
  if (e == cudaSuccess) e = cudaStreamSynchronize(host_stream());
  if (e != cudaSuccess) {
    dev_free(p->d_pool);
    dev_free(p->d_pool_cost);
    p->d_pool = nullptr;
    p->d_pool_cost = nullptr;
    return cuda_fail(e, "start pool");
  }
  p->pool_cap = N;
  return CGO_OK;
}

cgo_status ensure_state(cgo_problem *p, int P) {
  if (p->P_alloc == P && p->d_cur) return CGO_OK;
  free_state(p);
  const size_t sol = (size_t)P * p->len * 4;
  cudaError_t e = dev_alloc((void **)&p->d_cur, sol);
  if (e == cudaSuccess) e = dev_alloc((void **)&p->d_bestsol, sol);
  if (e == cudaSuccess) e = dev_alloc((void **)&p->d_cost, (size_t)P * 8);
  if (e == cudaSuccess) e = dev_alloc((void **)&p->d_best, (size_t)P * 8);
  if (e == cudaSuccess) e = dev_alloc((void **)&p->d_aos, 2 * sizeof(DevAos));
  if (e == cudaSuccess) e = dev_alloc((void **)&p->d_sync, sizeof(DevSync));
  if (e == cudaSuccess) e = cudaMemsetAsync(p->d_aos, 0, 2 * sizeof(DevAos), host_stream());
  if (e == cudaSuccess) e = cudaStreamSynchronize(host_stream());
  if (e != cudaSuccess) {
    free_state(p);  // nothing half-allocated stays behind
    return cuda_fail(e, "state alloc");
  }
  p->P_alloc = P;
  return CGO_OK;
}

// a solution of this problem's encoding (checked before it reaches a kernel)
bool valid_solution(const cgo_problem *p, const int32_t *x) {
  const int enc = encoding_of(p->model);
  if (enc == CGO_ENC_PERM) {
    std::vector<char> seen((size_t)p->len, 0);
    for (int i = 0; i < p->len; ++i) {
      if (x[i] < 0 || x[i] >= p->len || seen[(size_t)x[i]]) return false;
      seen[(size_t)x[i]] = 1;
    }
    return true;
  }
  const int lo = enc == CGO_ENC_BINARY ? 0 : p->lb, hi = enc == CGO_ENC_BINARY ? 1 : p->ub;
  for (int i = 0; i < p->len; ++i)
    if (x[i] < lo || x[i] > hi) return false;
  return true;
}

uint32_t applicable_mask(const cgo_problem *p) {
  const int enc = encoding_of(p->model);
  const uint32_t seg = p->len >= 2 ? 1u << SEGMENT : 0u;
  if (enc == CGO_ENC_BINARY) return (1u << FLIP) | seg;
  if (enc == CGO_ENC_INTEGER) return (1u << PERTURB) | seg;
  uint32_t m = (1u << SWAP) | (1u << TWO_OPT) | (1u << INSERT) | (1u << THREE_OPT);
  if (p->len >= 4) m |= 1u << OR_OPT;
  // the row level: CVRPTW's routes, at least two of them
  if (p->model == CVRPTW && p->len - p->n + 1 >= 2)
    m |= (1u << ROW_SWAP) | (1u << ROW_MERGE) | (1u << ROW_SPLIT);
  return m;
}

cgo_status load_params(const cgo_params *in, cgo_params *out) {
  if (!in) return fail(CGO_ERR_INVALID, "NULL params");
  if (in->struct_size == sizeof(cgo_params)) {
    *out = *in;
    return CGO_OK;
  }
  if (in->struct_size == CGO_PARAMS_SIZE_V1) {
    // the earlier fields only (its tail padding overlaps the appended ones)
    memset(out, 0, sizeof *out);
    memcpy(out, in, offsetof(cgo_params, row_w0_q16));
    out->struct_size = sizeof(cgo_params);
    out->op_mask &= (1u << CGO_NOPS) - 1u;
    for (int i = 0; i < CGO_NROW; ++i) out->row_cap_q16[i] = 65536u;
    return CGO_OK;
  }
  return fail(CGO_ERR_INVALID, "params: struct_size must be sizeof(cgo_params) or CGO_PARAMS_SIZE_V1");
}

cgo_status validate_params(const cgo_problem *p, const cgo_params *q, uint32_t *enabled) {
  if (!q || q->struct_size != sizeof(cgo_params))
    return fail(CGO_ERR_INVALID, "params: struct_size must be sizeof(cgo_params)");
  if (q->population < 1 || q->population > 65536) return fail(CGO_ERR_INVALID, "population out of [1, 65536]");
  if (q->candidates < 1 || q->candidates > 4096) return fail(CGO_ERR_INVALID, "candidates out of [1, 4096]");
  if (q->generations < 0) return fail(CGO_ERR_INVALID, "generations < 0");
  const uint32_t en = q->op_mask & applicable_mask(p);
  if (!en) return fail(CGO_ERR_INVALID, "no operator of this encoding is enabled");
  uint64_t ws = 0;
  for (int i = 0; i < kNops; ++i) {
    if (!((en >> i) & 1u)) continue;
    if (op_w0(*q, i) > 65536u) return fail(CGO_ERR_INVALID, "operator weight > 1.0");
    if (op_capq(*q, i) < q->w_floor_q16) return fail(CGO_ERR_INVALID, "operator cap below floor");
    ws += op_w0(*q, i);
  }
  if (ws == 0) return fail(CGO_ERR_INVALID, "enabled operator weights sum to zero");
  uint64_t ks = 0;
  for (int i = 0; i < 3; ++i) {
    if (q->k_w0_q16[i] > 65536u) return fail(CGO_ERR_INVALID, "K weight > 1.0");
    ks += q->k_w0_q16[i];
  }
  if (ks == 0) return fail(CGO_ERR_INVALID, "K weights sum to zero");
  if (q->aos_interval < 1) return fail(CGO_ERR_INVALID, "aos_interval < 1");
  if ((uint64_t)q->population * q->candidates * 3ull * q->aos_interval >= (1ull << 32))
    return fail(CGO_ERR_INVALID, "population*candidates*3*aos_interval must be < 2^32");
  if (q->ema_alpha_q16 > 65536u) return fail(CGO_ERR_INVALID, "ema_alpha > 1.0");
  if (q->w_floor_q16 < 8u) return fail(CGO_ERR_INVALID, "w_floor must be >= 8 (Q16)");
  if (q->w_cap_q16 < q->w_floor_q16 || q->w_cap_q16 > 65536u)
    return fail(CGO_ERR_INVALID, "w_cap must be in [w_floor, 65536]");
  if (q->alpha_q32 > (1ull << 32)) return fail(CGO_ERR_INVALID, "alpha > 1.0");
  if (q->elite_period > 0 && q->elite_period % q->aos_interval != 0)
    return fail(CGO_ERR_UNSUPPORTED, "elite_period must be a multiple of aos_interval on the GPU");
  if (q->init_oversample > 64) return fail(CGO_ERR_INVALID, "init_oversample must be <= 64");
  if ((uint64_t)(q->init_oversample > 1 ? q->init_oversample : 1) * q->population > 16384u)
    return fail(CGO_ERR_INVALID, "init_oversample * population must be <= 16384");
  if (q->init_heuristic > 1) return fail(CGO_ERR_INVALID, "init_heuristic must be 0 or 1");
  if (q->cross_q16 > 65536u) return fail(CGO_ERR_INVALID, "cross_q16 must be <= 65536");
  if (q->islands > 1 && q->migrate_period > 0) {
    if ((uint32_t)q->population % q->islands != 0)
      return fail(CGO_ERR_INVALID, "islands must divide the population");
    if (q->migrate_period % q->aos_interval != 0)
      return fail(CGO_ERR_UNSUPPORTED, "migrate_period must be a multiple of aos_interval on the GPU");
    if (q->migrate_strategy > 2) return fail(CGO_ERR_INVALID, "migrate_strategy must be 0, 1 or 2");
    if (q->migrate_strategy != 0 &&
        (q->migrate_n < 1 || q->migrate_n > (uint32_t)q->population / q->islands))
      return fail(CGO_ERR_INVALID, "migrate_n must be in [1, population / islands]");
  }
  *enabled = en;
  return CGO_OK;
}

KInst base_kinst(const cgo_problem *p) {
  KInst h;
  memset(&h, 0, sizeof h);
  h.model = (p->model == TSP && p->asym) ? (int32_t)ATSP : p->model;
  h.n = p->n;
  h.len = p->len;
  h.m = p->m;
  h.capacity = p->capacity;
  h.lam0 = p->lam0;
  h.lam1 = p->lam1;
  h.wdist = p->wdist;
  h.wveh = p->wveh;
  h.wlong = p->wlong;
  h.lex_n = p->lex_n;
  for (int i = 0; i < 3; ++i) {
    h.lex_obj[i] = p->lex_obj[i];
    h.lex_w[i] = p->lex_w[i];
    h.lex_R[i] = p->lex_R[i];
    h.lex_sh[i] = p->lex_sh[i];
  }
  h.lb = p->lb;
  h.ub = p->ub;
  h.tag = p->tag;
  h.tri16 = p->tri16;
  h.mat0 = p->d_mat0;
  h.mat1 = p->d_mat1;
  h.vec0 = p->d_vec[0];
  h.vec1 = p->d_vec[1];
  h.vec2 = p->d_vec[2];
  h.vec3 = p->d_vec[3];
  h.tri = p->d_tri;
  h.node = p->d_node;
  h.cv32 = p->cv32;
  const cgo_params &q = p->params;
  h.P = q.population;
  h.members = q.population;
  h.C = q.candidates;
  h.U = q.aos_interval;
  h.E = q.elite_period;
  h.alpha = q.alpha_q32;
  h.ema_a = q.ema_alpha_q16;
  h.w_floor = q.w_floor_q16;
  h.w_cap = q.w_cap_q16;
  h.stag_limit = q.stag_limit;
  for (int i = 0; i < kNops; ++i) h.op_cap[i] = op_capq(q, i);
  h.enabled = p->enabled;
  h.seed = p->seed;
  h.cur = p->d_cur;
  h.bestsol = p->d_bestsol;
  h.cost = p->d_cost;
  h.best = p->d_best;
  h.sync = p->d_sync;
  const bool mig = q.islands > 1 && q.migrate_period > 0;
  h.islands = mig ? (int32_t)q.islands : 1;
  h.mperiod = mig ? q.migrate_period : 0u;
  h.mstrat = (int32_t)q.migrate_strategy;
  h.mN = q.migrate_n;
  h.cross_q16 = q.population >= 2 ? q.cross_q16 : 0u;
  h.K_over = q.init_oversample > 1 ? (int32_t)q.init_oversample : 1;
  h.n_heur = q.init_heuristic ? p->n_heur : 0;
  h.heur = p->d_heur;
  h.pool_sol = p->d_pool;
  h.pool_cost = p->d_pool_cost;
  return h;
}

// Launch shape: warps per member generation (candidates split across
// them), generations in flight, members per CTA and staging mode.  Prefers
// two generations in flight where a lane holds one candidate, and one member
// per CTA (most SMs, least shared-memory pressure); grows the CTA only when
// the population would not be co-resident otherwise.
cgo_status choose_launch(cgo_problem *p, KInst &h, int *warps_out, int *wpm_out, int *ns_out,
                         int64_t *smem_out) {
  const int64_t optin = max_smem_optin();
  const int P = h.P, C = h.C;
  int wpm = p->wpm_override;
  if (wpm == 0) wpm = C >= 128 ? 4 : (C >= 64 ? 2 : 1);
  // a later generation in flight holds one candidate's counts per lane; three
  // or four in flight take 4 warps per generation (migration and crossover
  // kernels take at most two)
  auto ns_ok = [&](int ns) {
    if (ns == 1) return true;
    if (C > 32 * wpm) return false;
    if (ns == 2) return 2 * wpm <= kMaxWarps;
    // three or four: one member per CTA of four warps each, no window code;
    // the asymmetric TSP keeps one or two
    return wpm == 4 && !takes_xf(h) && h.model != ATSP;
  };
  int ns_try[4] = {2, 1, 0, 0}, nns = 2;
  if (p->ns_override > 0) {
    if (!ns_ok(p->ns_override))
      return fail(CGO_ERR_UNSUPPORTED,
                  "%d generations in flight need C <= 32 * warps_per_member (and, for 3 or 4, "
                  "warps_per_member = 4 without migration or crossover, and a symmetric TSP "
                  "matrix)",
                  p->ns_override);
    ns_try[0] = p->ns_override;
    nns = 1;
  } else if (!ns_ok(2)) {
    ns_try[0] = 1;
    nns = 1;
  }
  int fit_seen = 0, grid_seen = 0;
  for (int t = 0; t < nns; ++t) {
    const int ns = ns_try[t];
    const int max_warps = ns > 2 ? kMaxWarpsDeep : kMaxWarps;
    for (int mpc = 1; mpc * wpm * ns <= max_warps; mpc *= 2) {
      if (ns > 2 && mpc > 1) break;  // one member per CTA
      const int warps = mpc * wpm * ns;
      if (p->warps_override > 0 && warps != p->warps_override) continue;
      const int64_t staged = evolve_smem_bytes(h, warps, wpm, ns, true);
      const int64_t global = evolve_smem_bytes(h, warps, wpm, ns, false);
      bool use_smem = staged <= optin;
      if (p->staging_override == STAGE_GLOBAL) use_smem = false;
      if (p->staging_override == STAGE_SMEM && !use_smem) continue;
      const int64_t need = use_smem ? staged : global;
      if (need > optin) continue;
      h.shared_bytes = use_smem ? instance_data_bytes(h) : 0;
      const int grid = (P + mpc - 1) / mpc;
      const int fit = max_coresident_ctas(h, warps, wpm, ns, need);
      fit_seen = fit;
      grid_seen = grid;
      if (fit >= grid) {
        *warps_out = warps;
        *wpm_out = wpm;
        *ns_out = ns;
        *smem_out = need;
        p->last_warps = warps;
        p->last_wpm = wpm;
        p->last_ns = ns;
        p->last_staging = use_smem ? STAGE_SMEM : STAGE_GLOBAL;
        return CGO_OK;
      }
    }
  }
  if (grid_seen)
    return fail(CGO_ERR_UNSUPPORTED, "population %d needs %d co-resident CTAs; the GPU holds %d", P,
                grid_seen, fit_seen);
  return fail(CGO_ERR_UNSUPPORTED,
              "no launch shape fits (solution length %d, requested warps %d, staging %d)", p->len,
              p->warps_override, p->staging_override);
}

cgo_status check_sync_error(cgo_problem *p, cudaStream_t st) {
  uint32_t err = 0;
  CUDA_TRY(cudaMemcpyAsync(&err, &p->d_sync->error, 4, cudaMemcpyDeviceToHost, st), "reading status");
  CUDA_TRY(cudaStreamSynchronize(st), "synchronising stream");
  if (err) {
    p->has_state = false;
    return fail(CGO_ERR_TIMEOUT, "a member barrier timed out (flags 0x%x); search state discarded", err);
  }
  return CGO_OK;
}

cgo_status run_generations(cgo_problem *p, int64_t G, cudaStream_t st) {
  if (G == 0) return CGO_OK;
  if (p->g + G >= 0xFFFFFFFFll) return fail(CGO_ERR_INVALID, "generation index would exceed 2^32 - 2");
  // crossover needs three scratch rows per member
  if (p->params.cross_q16 > 0 && p->params.population >= 2 &&
      p->pool_cap < 3 * (int64_t)p->params.population)
    return fail(CGO_ERR_STATE, "no crossover buffer for this population");
  KInst h = base_kinst(p);
  int warps = 0, wpm = 1, ns = 1;
  int64_t smem = 0;
  cgo_status s = choose_launch(p, h, &warps, &wpm, &ns, &smem);
  if (s != CGO_OK) return s;
  h.members = p->params.population + (int)p->phantom_members;  // test hook adds phantoms
  h.g_begin = p->g;
  h.g_end = p->g + G;
  h.aos_in = p->d_aos + p->aos_cur;
  h.aos_out = p->d_aos + (1 - p->aos_cur);
  CUDA_TRY(cudaMemsetAsync(p->d_sync, 0, sizeof(DevSync), st), "sync reset");
  CUDA_TRY(cudaMemsetAsync(p->d_sync->elite, 0x7F, sizeof(p->d_sync->elite), st), "sync reset");
  if (!p->ev0) {
    CUDA_TRY(cudaEventCreate(&p->ev0), "event");
    CUDA_TRY(cudaEventCreate(&p->ev1), "event");
  }
  CUDA_TRY(cudaEventRecord(p->ev0, st), "event");
  CUDA_TRY(launch_evolve_single(h, warps, wpm, ns, smem, p->timeout_ns, st), "evolve launch");
  CUDA_TRY(cudaEventRecord(p->ev1, st), "event");
  p->timed = true;
  p->timed_gens = G;
  CUDA_TRY(launch_finalize(h, st), "finalize launch");
  s = check_sync_error(p, st);
  if (s != CGO_OK) return s;
  p->aos_cur = 1 - p->aos_cur;
  p->g += G;
  return CGO_OK;
}

// ------------------------------------------------ allocation-free solve
// Scratch of cgo_solve_static: a fixed device array that every GPU loading
// this library holds until the process exits.  Host code must not use the
// symbol's name as an address: it resolves the device address once per
// device with cudaGetSymbolAddress and passes that pointer to the kernels.
constexpr size_t kStaticScratchBytes = size_t(8) << 20;
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void *g_static_ptr[kMaxDevices] = {};

// Batched instances: every member in one CTA; one warp per member by
// default (many members per CTA keep the SMs busy).  The shared-memory size
// class (1/8, 1/4, 1/2 or all of the budget) groups instances into launches.
cgo_status batch_shape(cgo_problem *p, const cgo_params &q, KInst &h, int *wpm_out, int *warps_out,
                       int64_t *smem_out, int64_t *class_out) {
  const int64_t optin = max_smem_optin() - 1024;  // the kernel's static shared memory
  const int wpm = p->wpm_override > 0 ? p->wpm_override : 1;
  int warps = p->warps_override > 0 ? p->warps_override : kMaxWarps;
  warps = std::max(wpm, std::min(warps, q.population * wpm));
  warps = std::min(warps, kMaxWarps) / wpm * wpm;
  const int64_t staged = batch_smem_bytes(h, warps, wpm, true);
  const int64_t global = batch_smem_bytes(h, warps, wpm, false);
  const bool use_smem = staged <= optin && p->staging_override != STAGE_GLOBAL;
  if (p->staging_override == STAGE_SMEM && !use_smem)
    return fail(CGO_ERR_UNSUPPORTED, "instance data do not fit in shared memory");
  const int64_t need = use_smem ? staged : global;
  if (need > optin)
    return fail(CGO_ERR_UNSUPPORTED, "population %d x length %d does not fit in one CTA", q.population,
                p->len);
  h.shared_bytes = use_smem ? instance_data_bytes(h) : 0;
  int64_t cls = optin;
  for (int64_t c = optin / 8; c < optin; c *= 2)
    if (need <= c) {
      cls = c;
      break;
    }
  *wpm_out = wpm;
  *warps_out = warps;
  *smem_out = need;
  *class_out = cls;
  return CGO_OK;
}

DevAos initial_aos(const cgo_params &q, uint32_t en) {
  DevAos a;
  memset(&a, 0, sizeof a);
  a.T = q.T0_q32;
  for (int k = 0; k < kNops; ++k) a.w_op[k] = ((en >> k) & 1u) ? op_w0(q, k) : 0u;
  for (int k = 0; k < 3; ++k) a.w_k[k] = q.k_w0_q16[k];
  return a;
}

}  // namespace host
}  // namespace cgo

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

namespace cgo {
namespace host {

cgo_status static_scratch(void **out) {
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev), "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(CGO_ERR_UNSUPPORTED, "device ordinal %d >= %d", dev, kMaxDevices);
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_ptr[dev]) {
    void *ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the static scratch");
    g_static_ptr[dev] = ptr;
  }
  *out = g_static_ptr[dev];
  return CGO_OK;
}

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace host
}  // namespace cgo

extern "C" {

const char *cgo_last_error(void) { return g_err.c_str(); }

const char *cgo_version(void) { return "cgo 0.1 (sm_103a)"; }

cgo_status cgo_gather_peak(int32_t kind, int32_t log2_elements, double *gathers_per_s,
                           double *kernel_ms) {
  if (!gathers_per_s) return fail(CGO_ERR_INVALID, "gathers_per_s is NULL");
  if (kind == 0 ? (log2_elements < 10 || log2_elements > 16)
                : (kind != 1 || log2_elements < 10 || log2_elements > 28))
    return fail(CGO_ERR_INVALID, "kind %d with 2^%d elements is not measured", kind, log2_elements);
  CUDA_TRY(measure_gather_peak(kind, log2_elements, gathers_per_s, kernel_ms), "gather peak");
  return CGO_OK;
}

cgo_status cgo_kernel_launches(uint64_t *out) {
  if (!out) return fail(CGO_ERR_INVALID, "out is NULL");
  *out = launches_total();
  return CGO_OK;
}

// [R37] CVRPTW's lexicographic mode.  The kernels keep computing one integer
// cost per route set, with power-of-two weights that pack the objectives
// into separate bit fields of it: distance in bits [0, a), vehicles used in
// [a, b), the longest route's distance in [b, c) (when it is an objective)
// and the penalty from bit c on.  The kernels read the fields back and turn
// them into the key of the lexicographic order (bucketed objectives in mixed
// radix), which is the cost the search works with.
static int bits_for(int64_t x) {
  int b = 0;
  while (b < 62 && (x >> b) != 0) ++b;
  return b;
}

cgo_status set_lexicographic(cgo_problem *p, const cgo_problem_desc *d, const std::vector<int32_t> &travel,
                             double pen_max) {
  if (d->lex_n < 0 || d->lex_n > 3) return fail(CGO_ERR_INVALID, "lex_n must be in [0, 3]");
  if (d->weight_distance != 0 || d->weight_vehicles != 0 || d->weight_longest != 0)
    return fail(CGO_ERR_INVALID, "the lexicographic mode takes no objective weights");
  int64_t maxd = 0;
  for (int32_t t : travel) {
    if (t < 0) return fail(CGO_ERR_INVALID, "the lexicographic mode needs travel times >= 0");
    maxd = std::max<int64_t>(maxd, t);
  }
  bool seen[3] = {false, false, false};
  for (int i = 0; i < d->lex_n; ++i) {
    const int o = d->lex_obj[i];
    if (o < 0 || o > 2 || seen[o]) return fail(CGO_ERR_INVALID, "lex_obj: each objective at most once");
    if (d->lex_tol[i] < 0) return fail(CGO_ERR_INVALID, "lex_tol must be >= 0");
    seen[o] = true;
  }
  const int64_t dmax = ((int64_t)p->n + p->V) * maxd;
  const int a = bits_for(dmax), b = a + bits_for(p->V), c = b + (seen[2] ? bits_for(dmax) : 0);
  // the packed cost, the shifted penalty weights and the key stay below 2^62
  const double top = std::ldexp(1.0, c);
  if (c > 61 || (pen_max + 1.0) * top > kLimit || (double)p->lam0 * top > kLimit ||
      (double)p->lam1 * top > kLimit)
    return fail(CGO_ERR_UNSUPPORTED, "the objectives of this instance do not fit the packed cost");
  double radix = 1.0;
  p->lex_n = d->lex_n;
  for (int i = 0; i < 3; ++i) {
    const bool on = i < d->lex_n;
    const int o = on ? d->lex_obj[i] : 0;
    const int64_t w = on ? d->lex_tol[i] + 1 : 1;
    const int64_t omax = o == 1 ? (int64_t)p->V : dmax;
    p->lex_obj[i] = o;
    p->lex_w[i] = w;
    p->lex_R[i] = on ? omax / w + 1 : 1;
    radix *= (double)p->lex_R[i];
  }
  if ((pen_max + 1.0) * radix > kLimit)
    return fail(CGO_ERR_UNSUPPORTED, "the lexicographic key of this instance could exceed 2^62");
  p->lex_sh[0] = a;
  p->lex_sh[1] = b;
  p->lex_sh[2] = c;
  p->wdist = 1;
  p->wveh = (int64_t)1 << a;
  p->wlong = seen[2] ? (int64_t)1 << b : 0;
  p->lam0 <<= c;
  p->lam1 <<= c;
  return CGO_OK;
}

cgo_status cgo_problem_create(const cgo_problem_desc *d, cgo_problem **out) {
  if (!out) return fail(CGO_ERR_INVALID, "out is NULL");
  *out = nullptr;
  cgo_problem_desc dd;
  if (!d || (d->struct_size != sizeof(cgo_problem_desc) && d->struct_size != CGO_DESC_SIZE_V1 &&
             d->struct_size != CGO_DESC_SIZE_V2))
    return fail(CGO_ERR_INVALID, "desc: struct_size must be sizeof(cgo_problem_desc)");
  memset(&dd, 0, sizeof dd);
  memcpy(&dd, d, d->struct_size);  // an earlier description has the fields appended since off
  d = &dd;
  if (d->model < CGO_TSP || d->model > CGO_CVRPTW) return fail(CGO_ERR_INVALID, "unknown model");
  if (d->encoding != encoding_of(d->model))
    return fail(CGO_ERR_INVALID, "encoding %d does not match model %d", d->encoding, d->model);
  if (d->n < 2) return fail(CGO_ERR_INVALID, "n must be >= 2");
  const bool dev = d->pointers_on_device != 0;
  const int64_t n = d->n;
  if (d->model == CGO_CVRPTW && d->vehicles < 1) return fail(CGO_ERR_INVALID, "CVRPTW needs vehicles >= 1");
  const int64_t len64 = d->model == CGO_CVRPTW ? n + d->vehicles - 1 : n;
  if (len64 > 65535) return fail(CGO_ERR_INVALID, "solution length must be <= 65535");
  const int len = (int)len64;

  cgo_problem *p = new cgo_problem();
  cudaGetDevice(&p->device);
  p->model = d->model;
  p->n = (int)n;
  p->len = len;
  p->V = d->vehicles;
  p->tag = d->instance_tag;
  p->lam0 = d->penalty0;
  p->lam1 = d->penalty1;
  p->capacity = d->capacity;
  auto bail = [&](cgo_status s) {
    cgo_problem_destroy(p);
    return s;
  };
  std::vector<int32_t> a, b, c;
  cgo_status s;
  switch (d->model) {
    case CGO_TSP: {
      if ((s = host_copy(d->mat0, n * n, dev, a)) != CGO_OK) return bail(s);
      for (int64_t i = 0; i < n && !p->asym; ++i)
        for (int64_t j = i + 1; j < n; ++j)
          if (a[i * n + j] != a[j * n + i]) {
            p->asym = 1;  // the kernels' ATSP path: the full matrix, piece deltas
            break;
          }
      const int64_t mx = absmax(a);
      if ((double)mx * (double)n > kLimit) return bail(fail(CGO_ERR_INVALID, "distances could overflow"));
      p->tri16 = mx <= 32767 ? 1 : 0;
      cudaError_t e = copy_in(&p->d_mat0, a.data(), n * n, false);
      if (e != cudaSuccess) return bail(cuda_fail(e, "copying D"));
      if (p->asym) {
        // the full matrix in the kernels' element width
        const int64_t fb = pad16(n * n * (p->tri16 ? 2 : 4));
        std::vector<int16_t> h16;
        if (p->tri16) {
          h16.resize((size_t)(n * n));
          for (int64_t t = 0; t < n * n; ++t) h16[(size_t)t] = (int16_t)a[(size_t)t];
        }
        if ((e = dev_alloc(&p->d_tri, (size_t)fb)) != cudaSuccess) return bail(cuda_fail(e, "matrix"));
        if ((e = cudaMemcpyAsync(p->d_tri, p->tri16 ? (const void *)h16.data() : (const void *)a.data(),
                                 (size_t)(n * n * (p->tri16 ? 2 : 4)), cudaMemcpyHostToDevice,
                                 host_stream())) != cudaSuccess)
          return bail(cuda_fail(e, "matrix"));
      } else {
        const int64_t tb = pad16(n * (n + 1) / 2 * (p->tri16 ? 2 : 4));
        if ((e = dev_alloc(&p->d_tri, (size_t)tb)) != cudaSuccess) return bail(cuda_fail(e, "triangle"));
        if ((e = cudaMemsetAsync(p->d_tri, 0, (size_t)tb, host_stream())) != cudaSuccess) return bail(cuda_fail(e, "triangle"));
        if ((e = build_triangle(p->d_mat0, (int)n, p->tri16, p->d_tri, host_stream())) != cudaSuccess)
          return bail(cuda_fail(e, "triangle"));
      }
      if ((e = cudaStreamSynchronize(host_stream())) != cudaSuccess) return bail(cuda_fail(e, "triangle"));
      std::vector<int32_t> hp;
      heuristic_perms(a, n, hp);
      if ((e = copy_in(&p->d_heur, hp.data(), (int64_t)hp.size(), false)) != cudaSuccess)
        return bail(cuda_fail(e, "start permutations"));
      p->n_heur = 4;
      break;
    }
    case CGO_QAP: {
      if ((s = host_copy(d->mat0, n * n, dev, a)) != CGO_OK) return bail(s);
      if ((s = host_copy(d->mat1, n * n, dev, b)) != CGO_OK) return bail(s);
      const double mf = (double)absmax(a), md = (double)absmax(b);
      if (mf * md * (double)std::max<int64_t>(n * n, 16 * n) * 4.0 > kLimit)
        return bail(fail(CGO_ERR_INVALID, "flow x distance could overflow int64"));
      // a swap delta is 2n + 2 products of differences (each |.| <= 4 mf md)
      p->cv32 = (double)(2 * n + 2) * 4.0 * mf * md < 2.0e9 ? 1 : 0;
      {
        std::vector<int32_t> hp;
        heuristic_perms(a, n, hp);
        heuristic_perms(b, n, hp);
        cudaError_t e = copy_in(&p->d_heur, hp.data(), (int64_t)hp.size(), false);
        if (e != cudaSuccess) return bail(cuda_fail(e, "start permutations"));
        p->n_heur = 8;
      }
      cudaError_t e;
      if ((e = copy_in(&p->d_mat0, a.data(), n * n, false)) != cudaSuccess) return bail(cuda_fail(e, "copy F"));
      if ((e = copy_in(&p->d_mat1, b.data(), n * n, false)) != cudaSuccess) return bail(cuda_fail(e, "copy D"));
      break;
    }
    case CGO_KNAPSACK: {
      if ((s = host_copy(d->vec0, n, dev, a)) != CGO_OK) return bail(s);
      if ((s = host_copy(d->vec1, n, dev, b)) != CGO_OK) return bail(s);
      if (d->penalty0 < 0) return bail(fail(CGO_ERR_INVALID, "penalty0 < 0"));
      p->lam0 = d->penalty0 > 0 ? d->penalty0 : 1 + std::max<int64_t>(0, maxval(b));
      if ((double)p->lam0 * ((double)abssum(a) + std::fabs((double)d->capacity)) + (double)abssum(b) > kLimit)
        return bail(fail(CGO_ERR_INVALID, "penalty x weights could overflow int64"));
      cudaError_t e;
      if ((e = copy_in(&p->d_vec[0], a.data(), n, false)) != cudaSuccess) return bail(cuda_fail(e, "copy w"));
      if ((e = copy_in(&p->d_vec[1], b.data(), n, false)) != cudaSuccess) return bail(cuda_fail(e, "copy v"));
      break;
    }
    case CGO_CVRPTW: {
      const int64_t N = n + 1;
      std::vector<int32_t> v[4];
      if ((s = host_copy(d->mat0, N * N, dev, a)) != CGO_OK) return bail(s);
      const int32_t *src[4] = {d->vec0, d->vec1, d->vec2, d->vec3};
      for (int k = 0; k < 4; ++k)
        if ((s = host_copy(src[k], N, dev, v[k])) != CGO_OK) return bail(s);
      if (d->penalty0 < 0 || d->penalty1 < 0) return bail(fail(CGO_ERR_INVALID, "penalties < 0"));
      p->lam0 = d->penalty0 > 0 ? d->penalty0 : 100;
      p->lam1 = d->penalty1 > 0 ? d->penalty1 : 100;
      if (d->weight_distance < 0 || d->weight_vehicles < 0 || d->weight_longest < 0)
        return bail(fail(CGO_ERR_INVALID, "objective weights < 0"));
      p->wdist = d->weight_distance > 0 ? d->weight_distance : 1;
      p->wveh = d->weight_vehicles;
      p->wlong = d->weight_longest;
      // bound every route quantity: time, lateness, distance, load
      const double maxd = (double)absmax(a), tmax = (double)absmax(v[1]) + (double)N * (maxd + (double)absmax(v[3]));
      const double late = (double)N * (tmax + (double)absmax(v[2]));
      if ((double)p->lam1 * late + (double)p->lam0 * ((double)abssum(v[0]) + std::fabs((double)d->capacity) * N) +
              (double)(p->wdist + p->wlong) * (double)(len + 1) * maxd + (double)p->wveh * (double)d->vehicles >
          kLimit)
        return bail(fail(CGO_ERR_INVALID, "CVRPTW data could overflow an int64 cost"));
      // route quantities (time, lateness, distance, load) fit in int32?
      p->cv32 = (late < 2.0e9 && (double)abssum(v[0]) < 2.0e9 && (double)N * maxd < 2.0e9) ? 1 : 0;
      if (d->lex_n != 0 && (s = set_lexicographic(p, d, a, (double)p->lam0 * (double)abssum(v[0]) +
                                                              (double)p->lam1 * late)) != CGO_OK)
        return bail(s);
      std::vector<int4> node((size_t)N);
      for (int64_t k = 0; k < N; ++k) node[(size_t)k] = make_int4(v[1][(size_t)k], v[2][(size_t)k], v[3][(size_t)k], v[0][(size_t)k]);
      cudaError_t e;
      if ((e = copy_in(&p->d_mat0, a.data(), N * N, false)) != cudaSuccess) return bail(cuda_fail(e, "copy d"));
      for (int k = 0; k < 4; ++k)
        if ((e = copy_in(&p->d_vec[k], v[k].data(), N, false)) != cudaSuccess) return bail(cuda_fail(e, "copy vectors"));
      if ((e = copy_in((int32_t **)&p->d_node, (const int32_t *)node.data(), 4 * N, false)) != cudaSuccess)
        return bail(cuda_fail(e, "copy nodes"));
      break;
    }
    case CGO_GAP: {
      if (d->m < 2 || d->m > kMaxAgents) return bail(fail(CGO_ERR_INVALID, "GAP needs 2 <= m <= %d", kMaxAgents));
      p->m = d->m;
      p->lb = 0;
      p->ub = d->m - 1;
      const int64_t mn = (int64_t)d->m * n;
      if ((s = host_copy(d->mat0, mn, dev, a)) != CGO_OK) return bail(s);
      if ((s = host_copy(d->mat1, mn, dev, b)) != CGO_OK) return bail(s);
      if ((s = host_copy(d->vec0, d->m, dev, c)) != CGO_OK) return bail(s);
      if (d->penalty0 < 0) return bail(fail(CGO_ERR_INVALID, "penalty0 < 0"));
      p->lam0 = d->penalty0 > 0 ? d->penalty0 : 1 + std::max<int64_t>(0, maxval(a));
      if ((double)p->lam0 * ((double)abssum(b) + (double)abssum(c)) + (double)abssum(a) > kLimit)
        return bail(fail(CGO_ERR_INVALID, "penalty x requirements could overflow int64"));
      cudaError_t e;
      if ((e = copy_in(&p->d_mat0, a.data(), mn, false)) != cudaSuccess) return bail(cuda_fail(e, "copy c"));
      if ((e = copy_in(&p->d_mat1, b.data(), mn, false)) != cudaSuccess) return bail(cuda_fail(e, "copy r"));
      if ((e = copy_in(&p->d_vec[0], c.data(), d->m, false)) != cudaSuccess) return bail(cuda_fail(e, "copy cap"));
      break;
    }
  }
  *out = p;
  return CGO_OK;
}

cgo_status cgo_problem_destroy(cgo_problem *p) {
  if (!p) return CGO_OK;
  free_state(p);
  if (p->ev0) cudaEventDestroy(p->ev0);
  if (p->ev1) cudaEventDestroy(p->ev1);
  dev_free(p->d_mat0);
  dev_free(p->d_mat1);
  for (int i = 0; i < 4; ++i) dev_free(p->d_vec[i]);
  dev_free(p->d_tri);
  dev_free(p->d_node);
  dev_free(p->d_heur);
  dev_free(p->d_pool);
  dev_free(p->d_pool_cost);
  delete p;
  return CGO_OK;
}

cgo_status cgo_solution_length(const cgo_problem *p, int32_t *out) {
  if (!p || !out) return fail(CGO_ERR_INVALID, "NULL argument");
  *out = p->len;
  return CGO_OK;
}

cgo_status cgo_params_default(const cgo_problem *p, cgo_params *out) {
  if (!p || !out) return fail(CGO_ERR_INVALID, "NULL argument");
  const bool v1 = out->struct_size == CGO_PARAMS_SIZE_V1;
  cgo_params full;
  cgo_params *q = &full;
  memset(q, 0, sizeof *q);
  q->struct_size = sizeof(cgo_params);
  q->population = 32;
  q->candidates = 128;
  q->generations = 2000;
  const uint32_t app = applicable_mask(p);
  // 3-opt, the segment operators of the binary / integer sets and the row
  // level are off by default
  const uint32_t en =
      app & ~((1u << THREE_OPT) | (1u << SEGMENT) | (1u << ROW_SWAP) | (1u << ROW_MERGE) | (1u << ROW_SPLIT));
  q->op_mask = en;
  // Table "weight_preset": O(1) operators 1.0; or-opt and 3-opt by scale of
  // the length, seg_flip / seg_reset with or-opt's segment-level preset; the
  // normaliser is taken over the default mask
  uint64_t S = 0;
  uint32_t w[kNops] = {0};
  for (int i = 0; i < kNops; ++i) {
    if (!((app >> i) & 1u)) continue;
    w[i] = 65536u;
    if (i == OR_OPT) w[i] = p->len <= 100 ? 52429u : (p->len <= 250 ? 45875u : 19661u);
    if (i == THREE_OPT) w[i] = p->len <= 100 ? 32768u : (p->len <= 250 ? 19661u : 3277u);
    if (i == SEGMENT) w[i] = p->len <= 100 ? 52429u : (p->len <= 250 ? 45875u : 19661u);
    if ((en >> i) & 1u) S += w[i];
  }
  // (the row level takes the O(1) prior 1.0: the table scales only the
  // operators of higher complexity)
  for (int i = 0; i < kNops; ++i) {
    const uint32_t wi = (uint32_t)(((uint64_t)w[i] << 16) / S);
    if (i < CGO_NOPS) {
      q->op_w0_q16[i] = wi;
      q->op_cap_q16[i] = 65536u;
    } else {
      q->row_w0_q16[i - CGO_NOPS] = wi;
      q->row_cap_q16[i - CGO_NOPS] = 65536u;
    }
  }
  q->k_w0_q16[0] = 52429u;
  q->k_w0_q16[1] = 9830u;
  q->k_w0_q16[2] = 3277u;
  q->T0_q32 = 100ull << 32;
  q->alpha_q32 = 4290672329ull;  // round(0.999 * 2^32)
  q->aos_interval = 10;
  q->ema_alpha_q16 = 52429u;
  q->w_floor_q16 = 3277u;
  q->w_cap_q16 = 39322u;
  q->stag_limit = 5;
  q->elite_period = 0;
  q->init_oversample = 1;
  q->init_heuristic = 0;
  q->islands = 1;
  q->migrate_period = 0;
  q->migrate_strategy = 0;
  q->migrate_n = 1;
  q->cross_q16 = 0;
  if (v1) {
    memcpy(out, q, offsetof(cgo_params, row_w0_q16));
    out->struct_size = CGO_PARAMS_SIZE_V1;
  } else {
    *out = *q;
  }
  return CGO_OK;
}

cgo_status cgo_set_launch(cgo_problem *p, const cgo_launch *l) {
  if (!p || !l || l->struct_size != sizeof(cgo_launch)) return fail(CGO_ERR_INVALID, "bad launch struct");
  if (l->gens_in_flight < 0 || l->gens_in_flight > 4)
    return fail(CGO_ERR_INVALID, "gens_in_flight must be in [0, 4]");
  const int max_warps = l->gens_in_flight > 2 ? kMaxWarpsDeep : kMaxWarps;
  if (l->warps_per_cta < 0 || l->warps_per_cta > max_warps)
    return fail(CGO_ERR_INVALID, "warps_per_cta must be in [0, %d]", max_warps);
  if (l->warps_per_member != 0 && l->warps_per_member != 1 && l->warps_per_member != 2 &&
      l->warps_per_member != 4)
    return fail(CGO_ERR_INVALID, "warps_per_member must be 0, 1, 2 or 4");
  if (l->gens_in_flight > 2 && l->warps_per_member != 4 && l->warps_per_member != 0)
    return fail(CGO_ERR_INVALID, "3 or 4 generations in flight take warps_per_member = 4");
  const int unit = (l->warps_per_member > 0 ? l->warps_per_member : 1) *
                   (l->gens_in_flight > 0 ? l->gens_in_flight : 1);
  if (l->warps_per_cta > 0 && l->warps_per_cta % unit)
    return fail(CGO_ERR_INVALID, "warps_per_cta must be a multiple of warps_per_member * gens_in_flight");
  if (l->staging < 0 || l->staging > 2) return fail(CGO_ERR_INVALID, "staging must be 0, 1 or 2");
  p->warps_override = l->warps_per_cta;
  p->wpm_override = l->warps_per_member;
  p->staging_override = l->staging;
  p->ns_override = l->gens_in_flight;
  return CGO_OK;
}

cgo_status cgo_get_launch(const cgo_problem *p, cgo_launch *l) {
  if (!p || !l) return fail(CGO_ERR_INVALID, "NULL argument");
  l->struct_size = sizeof(cgo_launch);
  l->warps_per_cta = p->last_warps;
  l->warps_per_member = p->last_wpm;
  l->staging = p->last_staging;
  l->gens_in_flight = p->last_ns;
  return CGO_OK;
}

cgo_status cgo_solve(cgo_problem *p, const cgo_params *qin, uint64_t seed, void *stream) {
  if (!p) return fail(CGO_ERR_INVALID, "NULL problem");
  Guard gd(p);
  if (!gd.ok) return fail(CGO_ERR_BUSY, "problem handle in use");
  cudaSetDevice(p->device);
  cgo_params qq;
  cgo_status s = load_params(qin, &qq);
  if (s != CGO_OK) return s;
  const cgo_params *q = &qq;
  uint32_t en = 0;
  s = validate_params(p, q, &en);
  if (s != CGO_OK) return s;
  if ((s = ensure_state(p, q->population)) != CGO_OK) return s;
  if ((s = ensure_pool(p, *q)) != CGO_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  p->params = *q;
  p->seed = seed;
  p->enabled = en;
  p->g = 0;
  p->aos_cur = 0;
  p->has_state = false;
  KInst h = base_kinst(p);
  CUDA_TRY(launch_init(h, st), "init launch");
  const DevAos a0 = initial_aos(*q, en);
  h.aos_out = p->d_aos;
  CUDA_TRY(launch_init_aos(h, a0, st), "init launch");
  CUDA_TRY(cudaStreamSynchronize(st), "init");
  p->has_state = true;
  return run_generations(p, q->generations, st);
}

cgo_status cgo_solve_continue(cgo_problem *p, int64_t G, void *stream) {
  if (!p) return fail(CGO_ERR_INVALID, "NULL problem");
  Guard gd(p);
  if (!gd.ok) return fail(CGO_ERR_BUSY, "problem handle in use");
  if (!p->has_state) return fail(CGO_ERR_STATE, "no search state: call cgo_solve first");
  if (G < 0) return fail(CGO_ERR_INVALID, "generations < 0");
  cudaSetDevice(p->device);
  return run_generations(p, G, (cudaStream_t)stream);
}

cgo_status cgo_last_kernel_time(const cgo_problem *p, double *ms, int64_t *generations) {
  if (!p || !ms) return fail(CGO_ERR_INVALID, "NULL argument");
  if (!p->timed) return fail(CGO_ERR_STATE, "no evolve launch yet");
  float f = 0.f;
  CUDA_TRY(cudaEventElapsedTime(&f, p->ev0, p->ev1), "event time");
  *ms = f;
  if (generations) *generations = p->timed_gens;
  return CGO_OK;
}

cgo_status cgo_best(const cgo_problem *p, int32_t *out_sol, int32_t cap, int64_t *out_cost) {
  if (!p) return fail(CGO_ERR_INVALID, "NULL problem");
  Guard gd(p);
  if (!gd.ok) return fail(CGO_ERR_BUSY, "problem handle in use");
  if (!p->has_state) return fail(CGO_ERR_STATE, "no search state: call cgo_solve first");
  if (out_sol && cap < p->len) return fail(CGO_ERR_INVALID, "cap %d < solution length %d", cap, p->len);
  cudaSetDevice(p->device);
  DevAos a;
  CUDA_TRY(copy_sync(&a, p->d_aos + p->aos_cur, sizeof a, cudaMemcpyDeviceToHost), "reading elite");
  if (out_cost) *out_cost = a.elite_cost;
  if (out_sol)
    CUDA_TRY(copy_sync(out_sol, p->d_bestsol + (int64_t)a.elite * p->len, (size_t)p->len * 4,
                        cudaMemcpyDeviceToHost),
             "reading elite");
  return CGO_OK;
}

// ------------------------------------------------ state as a byte buffer
namespace {
constexpr uint32_t kBlobMagic = 0x314F4743u;  // "CGO1"
constexpr uint32_t kBlobVersion = 1;
struct BlobHead {
  uint32_t magic, version, population, length;
  int64_t generation;
  uint64_t T_q32;
  uint32_t w_op[CGO_NOPS_ALL], w_k[3], stag, pad;
  int64_t elite_prev;
  uint32_t u_op[CGO_NOPS_ALL], v_op[CGO_NOPS_ALL], u_k[3], v_k[3];
};
size_t blob_bytes(int P, int len) { return sizeof(BlobHead) + (size_t)P * len * 8 + (size_t)P * 16; }
}  // namespace

cgo_status cgo_state_export(const cgo_problem *p, void *buf, size_t cap, size_t *used) {
  if (!p || !used) return fail(CGO_ERR_INVALID, "NULL argument");
  if (!p->has_state) return fail(CGO_ERR_STATE, "no search state");
  const int P = p->params.population, len = p->len;
  *used = blob_bytes(P, len);
  if (!buf || cap < *used) return fail(CGO_ERR_INVALID, "buffer of %zu bytes; the state needs %zu", cap, *used);
  unsigned char *b = (unsigned char *)buf;
  BlobHead h;
  memset(&h, 0, sizeof h);
  cgo_state s;
  memset(&s, 0, sizeof s);
  s.struct_size = sizeof s;
  s.cur = (int32_t *)(b + sizeof h);
  s.best_sol = s.cur + (size_t)P * len;
  s.cost = (int64_t *)(s.best_sol + (size_t)P * len);
  s.best_cost = s.cost + P;
  cgo_status st = cgo_state_get(p, &s);
  if (st != CGO_OK) return st;
  h.magic = kBlobMagic;
  h.version = kBlobVersion;
  h.population = (uint32_t)P;
  h.length = (uint32_t)len;
  h.generation = s.generation;
  h.T_q32 = s.T_q32;
  for (int i = 0; i < CGO_NOPS_ALL; ++i) {
    const bool row = i >= CGO_NOPS;
    h.w_op[i] = row ? s.w_row_q16[i - CGO_NOPS] : s.w_op_q16[i];
    h.u_op[i] = row ? s.u_row[i - CGO_NOPS] : s.u_op[i];
    h.v_op[i] = row ? s.v_row[i - CGO_NOPS] : s.v_op[i];
  }
  for (int i = 0; i < 3; ++i) {
    h.w_k[i] = s.w_k_q16[i];
    h.u_k[i] = s.u_k[i];
    h.v_k[i] = s.v_k[i];
  }
  h.stag = s.stag;
  h.elite_prev = s.elite_prev;
  memcpy(b, &h, sizeof h);
  return CGO_OK;
}

cgo_status cgo_state_import(cgo_problem *p, const cgo_params *q, uint64_t seed, const void *buf,
                            size_t blen) {
  if (!p || !buf) return fail(CGO_ERR_INVALID, "NULL argument");
  BlobHead h;
  if (blen < sizeof h) return fail(CGO_ERR_INVALID, "buffer shorter than the state header");
  memcpy(&h, buf, sizeof h);
  if (h.magic != kBlobMagic) return fail(CGO_ERR_INVALID, "not a cgo state buffer");
  if (h.version != kBlobVersion) return fail(CGO_ERR_INVALID, "state format version %u, expected %u", h.version, kBlobVersion);
  if (h.length != (uint32_t)p->len) return fail(CGO_ERR_INVALID, "state of length %u for a problem of length %d", h.length, p->len);
  if (h.population < 1 || h.population > 65536 || blen < blob_bytes((int)h.population, p->len))
    return fail(CGO_ERR_INVALID, "truncated state buffer");
  const int P = (int)h.population, len = p->len;
  const unsigned char *b = (const unsigned char *)buf;
  std::vector<int32_t> cur((size_t)P * len), best((size_t)P * len);
  std::vector<int64_t> cost((size_t)P), bcost((size_t)P);
  memcpy(cur.data(), b + sizeof h, cur.size() * 4);
  memcpy(best.data(), b + sizeof h + cur.size() * 4, best.size() * 4);
  memcpy(cost.data(), b + sizeof h + 2 * cur.size() * 4, (size_t)P * 8);
  memcpy(bcost.data(), b + sizeof h + 2 * cur.size() * 4 + (size_t)P * 8, (size_t)P * 8);
  cgo_state s;
  memset(&s, 0, sizeof s);
  s.struct_size = sizeof s;
  s.population = P;
  s.length = len;
  s.generation = h.generation;
  s.T_q32 = h.T_q32;
  for (int i = 0; i < CGO_NOPS_ALL; ++i) {
    if (i < CGO_NOPS) {
      s.w_op_q16[i] = h.w_op[i];
      s.u_op[i] = h.u_op[i];
      s.v_op[i] = h.v_op[i];
    } else {
      s.w_row_q16[i - CGO_NOPS] = h.w_op[i];
      s.u_row[i - CGO_NOPS] = h.u_op[i];
      s.v_row[i - CGO_NOPS] = h.v_op[i];
    }
  }
  for (int i = 0; i < 3; ++i) {
    s.w_k_q16[i] = h.w_k[i];
    s.u_k[i] = h.u_k[i];
    s.v_k[i] = h.v_k[i];
  }
  s.stag = h.stag;
  s.elite_prev = h.elite_prev;
  s.cur = cur.data();
  s.best_sol = best.data();
  s.cost = cost.data();
  s.best_cost = bcost.data();
  return cgo_state_set(p, q, seed, &s);
}

cgo_status cgo_op_counts(const cgo_problem *p, uint64_t *out, int32_t cap) {
  if (!p || !out) return fail(CGO_ERR_INVALID, "NULL argument");
  if (cap < kStats) return fail(CGO_ERR_INVALID, "cap %d < %d", cap, kStats);
  Guard gd(p);
  if (!gd.ok) return fail(CGO_ERR_BUSY, "problem handle in use");
  if (!p->has_state) return fail(CGO_ERR_STATE, "no search state");
  cudaSetDevice(p->device);
  DevAos a;
  CUDA_TRY(copy_sync(&a, p->d_aos + p->aos_cur, sizeof a, cudaMemcpyDeviceToHost), "reading counts");
  for (int i = 0; i < kStats; ++i) out[i] = a.cum[i] + a.pend[i];
  return CGO_OK;
}

cgo_status cgo_best_rows(const cgo_problem *p, int32_t *out_rows, int32_t cap, int32_t *row_lengths,
                         int32_t max_rows, int32_t *out_rows_count, int64_t *out_cost) {
  if (!p || !out_rows || !row_lengths || !out_rows_count) return fail(CGO_ERR_INVALID, "NULL argument");
  const bool cv = p->model == CVRPTW;
  const int rows = cv ? p->len - p->n + 1 : 1, elems = cv ? p->n : p->len;
  if (cap < elems) return fail(CGO_ERR_INVALID, "cap %d < %d elements", cap, elems);
  if (max_rows < rows) return fail(CGO_ERR_INVALID, "max_rows %d < %d rows", max_rows, rows);
  std::vector<int32_t> seq((size_t)p->len);
  int64_t c = 0;
  const cgo_status s = cgo_best(p, seq.data(), p->len, &c);
  if (s != CGO_OK) return s;
  int o = 0, r = 0;
  for (int r0 = 0; r0 < rows; ++r0) row_lengths[r0] = 0;
  for (int q = 0; q < p->len; ++q) {
    if (cv && seq[(size_t)q] >= p->n) {
      ++r;  // a separator closes route r
      continue;
    }
    out_rows[o++] = seq[(size_t)q];
    row_lengths[r]++;
  }
  *out_rows_count = rows;
  if (out_cost) *out_cost = c;
  return CGO_OK;
}

cgo_status cgo_state_get(const cgo_problem *p, cgo_state *o) {
  if (!p || !o || (o->struct_size != sizeof(cgo_state) && o->struct_size != CGO_STATE_SIZE_V1))
    return fail(CGO_ERR_INVALID, "bad state struct");
  const bool has_rows = o->struct_size == sizeof(cgo_state);
  Guard gd(p);
  if (!gd.ok) return fail(CGO_ERR_BUSY, "problem handle in use");
  if (!p->has_state) return fail(CGO_ERR_STATE, "no search state");
  cudaSetDevice(p->device);
  DevAos a;
  CUDA_TRY(copy_sync(&a, p->d_aos + p->aos_cur, sizeof a, cudaMemcpyDeviceToHost), "reading state");
  const int P = p->params.population;
  o->population = P;
  o->length = p->len;
  o->generation = a.g;
  o->T_q32 = a.T;
  for (int i = 0; i < kNops; ++i) {
    if (i < CGO_NOPS) {
      o->w_op_q16[i] = a.w_op[i];
      o->u_op[i] = a.pend[i];
      o->v_op[i] = a.pend[kStatV + i];
    } else if (has_rows) {
      o->w_row_q16[i - CGO_NOPS] = a.w_op[i];
      o->u_row[i - CGO_NOPS] = a.pend[i];
      o->v_row[i - CGO_NOPS] = a.pend[kStatV + i];
    }
  }
  for (int i = 0; i < 3; ++i) {
    o->w_k_q16[i] = a.w_k[i];
    o->u_k[i] = a.pend[kStatUK + i];
    o->v_k[i] = a.pend[kStatVK + i];
  }
  o->stag = a.stag;
  o->elite_prev = a.elite_prev;
  const size_t sb = (size_t)P * p->len * 4;
  if (o->cur) CUDA_TRY(copy_sync(o->cur, p->d_cur, sb, cudaMemcpyDeviceToHost), "reading state");
  if (o->best_sol) CUDA_TRY(copy_sync(o->best_sol, p->d_bestsol, sb, cudaMemcpyDeviceToHost), "reading state");
  if (o->cost) CUDA_TRY(copy_sync(o->cost, p->d_cost, (size_t)P * 8, cudaMemcpyDeviceToHost), "reading state");
  if (o->best_cost) CUDA_TRY(copy_sync(o->best_cost, p->d_best, (size_t)P * 8, cudaMemcpyDeviceToHost), "reading state");
  return CGO_OK;
}

cgo_status cgo_state_set(cgo_problem *p, const cgo_params *qin, uint64_t seed, const cgo_state *in) {
  if (!p || !in || (in->struct_size != sizeof(cgo_state) && in->struct_size != CGO_STATE_SIZE_V1))
    return fail(CGO_ERR_INVALID, "bad state struct");
  Guard gd(p);
  if (!gd.ok) return fail(CGO_ERR_BUSY, "problem handle in use");
  cudaSetDevice(p->device);
  cgo_params qq;
  cgo_status s = load_params(qin, &qq);
  if (s != CGO_OK) return s;
  const cgo_params *q = &qq;
  uint32_t en = 0;
  s = validate_params(p, q, &en);
  if (s != CGO_OK) return s;
  const bool has_rows = in->struct_size == sizeof(cgo_state);
  if (!has_rows && (en >> CGO_NOPS))
    return fail(CGO_ERR_INVALID, "a state without the row level cannot resume a search with row operators");
  if (in->population != q->population || in->length != p->len)
    return fail(CGO_ERR_INVALID, "state shape does not match params/problem");
  if (!in->cur || !in->best_sol || !in->cost || !in->best_cost)
    return fail(CGO_ERR_INVALID, "all four state arrays are required");
  if (in->generation < 0 || in->generation >= 0xFFFFFFFFll) return fail(CGO_ERR_INVALID, "bad generation");
  const int P = q->population;
  for (int r = 0; r < 2 * P; ++r) {
    const int32_t *x = (r < P ? in->cur : in->best_sol) + (int64_t)(r % P) * p->len;
    if (!valid_solution(p, x)) return fail(CGO_ERR_INVALID, "state row %d is not a valid solution", r);
  }
  if ((s = ensure_state(p, q->population)) != CGO_OK) return s;
  if ((s = ensure_pool(p, *q)) != CGO_OK) return s;
  const size_t sb = (size_t)P * p->len * 4;
  CUDA_TRY(copy_sync(p->d_cur, in->cur, sb, cudaMemcpyHostToDevice), "writing state");
  CUDA_TRY(copy_sync(p->d_bestsol, in->best_sol, sb, cudaMemcpyHostToDevice), "writing state");
  CUDA_TRY(copy_sync(p->d_cost, in->cost, (size_t)P * 8, cudaMemcpyHostToDevice), "writing state");
  CUDA_TRY(copy_sync(p->d_best, in->best_cost, (size_t)P * 8, cudaMemcpyHostToDevice), "writing state");
  DevAos a;
  memset(&a, 0, sizeof a);
  a.T = in->T_q32;
  a.g = in->generation;
  for (int i = 0; i < kNops; ++i) {
    const bool row = i >= CGO_NOPS;
    a.w_op[i] = row ? (has_rows ? in->w_row_q16[i - CGO_NOPS] : 0u) : in->w_op_q16[i];
    a.pend[i] = row ? (has_rows ? in->u_row[i - CGO_NOPS] : 0u) : in->u_op[i];
    a.pend[kStatV + i] = row ? (has_rows ? in->v_row[i - CGO_NOPS] : 0u) : in->v_op[i];
  }
  for (int i = 0; i < 3; ++i) {
    a.w_k[i] = in->w_k_q16[i];
    a.pend[kStatUK + i] = in->u_k[i];
    a.pend[kStatVK + i] = in->v_k[i];
  }
  a.stag = in->stag;
  a.elite_prev = in->elite_prev;
  int e = 0;
  for (int i = 1; i < P; ++i)
    if (in->best_cost[i] < in->best_cost[e]) e = i;
  a.elite = e;
  a.elite_cost = in->best_cost[e];
  CUDA_TRY(copy_sync(p->d_aos, &a, sizeof a, cudaMemcpyHostToDevice), "writing state");
  p->params = *q;
  p->seed = seed;
  p->enabled = en;
  p->g = in->generation;
  p->aos_cur = 0;
  p->has_state = true;
  return CGO_OK;
}

cgo_status cgo_solve_batch(cgo_problem *const *probs, const cgo_params *per_in, const uint64_t *seeds,
                           int32_t count, void *stream) {
  if (count < 0 || (count > 0 && (!probs || !per_in || !seeds))) return fail(CGO_ERR_INVALID, "bad batch arguments");
  if (count == 0) return CGO_OK;
  cudaStream_t st = (cudaStream_t)stream;
  // every handle distinct and free
  std::vector<std::unique_ptr<Guard>> guards;
  guards.reserve((size_t)count);
  for (int32_t i = 0; i < count; ++i) {
    if (!probs[i]) return fail(CGO_ERR_INVALID, "problem %d is NULL", i);
    guards.emplace_back(new Guard(probs[i]));
    if (!guards.back()->ok) return fail(CGO_ERR_BUSY, "problem %d is in use (or repeated in the batch)", i);
  }
  int dev = 0;
  cudaGetDevice(&dev);
  // validate, allocate state, and describe each problem
  std::vector<KInst> hk((size_t)count);
  std::vector<DevAos> a0((size_t)count);
  std::vector<int> bucket_of((size_t)count);
  struct Bucket {
    int model, tri16, xf, wpm, warps;
    int64_t smem;
    std::vector<int> members;
  };
  std::vector<Bucket> buckets;
  int64_t Gmax = 0;
  // per_prob is an array of structs of one size: the current or the earlier one
  const size_t stride = per_in[0].struct_size == CGO_PARAMS_SIZE_V1 ? CGO_PARAMS_SIZE_V1
                                                                     : sizeof(cgo_params);
  std::vector<cgo_params> per((size_t)count);
  for (int32_t i = 0; i < count; ++i) {
    cgo_status s = load_params((const cgo_params *)((const char *)per_in + (size_t)i * stride),
                               &per[(size_t)i]);
    if (s != CGO_OK) return s;
  }
  for (int32_t i = 0; i < count; ++i) {
    cgo_problem *p = probs[i];
    if (p->device != dev) return fail(CGO_ERR_INVALID, "problem %d lives on another device", i);
    uint32_t en = 0;
    cgo_status s = validate_params(p, &per[i], &en);
    if (s != CGO_OK) return s;
    if (per[i].generations >= 0xFFFFFFFFll) return fail(CGO_ERR_INVALID, "problem %d: too many generations", i);
    if ((s = ensure_state(p, per[i].population)) != CGO_OK) return s;
    if ((s = ensure_pool(p, per[i])) != CGO_OK) return s;
    p->params = per[i];
    p->seed = seeds[i];
    p->enabled = en;
    p->g = 0;
    p->aos_cur = 0;
    p->has_state = false;
    KInst h = base_kinst(p);
    h.aos_in = h.aos_out = p->d_aos;
    h.G_total = per[i].generations;
    h.local_sync = 1;
    int wpm = 1, warps = 1;
    int64_t need = 0, cls = 0;
    if ((s = batch_shape(p, per[i], h, &wpm, &warps, &need, &cls)) != CGO_OK)
      return fail(s, "problem %d: %s", i, cgo_last_error());
    int b = -1;
    const int xf = takes_xf(h) != 0 ? 1 : 0;  // batched kernels: one set with both steps
    for (size_t k = 0; k < buckets.size(); ++k)
      if (buckets[k].model == h.model && buckets[k].tri16 == p->tri16 && buckets[k].xf == xf &&
          buckets[k].wpm == wpm && buckets[k].warps == warps && buckets[k].smem == cls)
        b = (int)k;
    if (b < 0) {
      buckets.push_back(Bucket{h.model, p->tri16, xf, wpm, warps, cls, {}});  // the kernels' model
      b = (int)buckets.size() - 1;
    }
    buckets[(size_t)b].members.push_back(i);
    hk[(size_t)i] = h;
    a0[(size_t)i] = initial_aos(per[i], en);
    Gmax = std::max<int64_t>(Gmax, per[i].generations);
  }
  // device copies of the descriptions, work lists and counters
  const size_t nb = buckets.size();
  KInst *d_k = nullptr;
  DevAos *d_a0 = nullptr;
  int *d_lists = nullptr, *d_next = nullptr, *d_counts = nullptr;
  auto release = [&]() {
    if (d_k) cudaFreeAsync(d_k, st);
    if (d_a0) cudaFreeAsync(d_a0, st);
    if (d_lists) cudaFreeAsync(d_lists, st);
    if (d_next) cudaFreeAsync(d_next, st);
    if (d_counts) cudaFreeAsync(d_counts, st);
  };
  std::vector<int> lists, counts;
  std::vector<size_t> list_off;
  for (auto &bk : buckets) {
    // longest first: larger instances start early, small ones fill the tail
    std::stable_sort(bk.members.begin(), bk.members.end(), [&](int x, int y) {
      const double wx = (double)probs[x]->len * per[x].population * per[x].generations;
      const double wy = (double)probs[y]->len * per[y].population * per[y].generations;
      return wx > wy;
    });
    list_off.push_back(lists.size());
    counts.push_back((int)bk.members.size());
    lists.insert(lists.end(), bk.members.begin(), bk.members.end());
  }
  cudaError_t e;
  if ((e = lib_malloc_async((void **)&d_k, sizeof(KInst) * (size_t)count, st)) != cudaSuccess ||
      (e = lib_malloc_async((void **)&d_a0, sizeof(DevAos) * (size_t)count, st)) != cudaSuccess ||
      (e = lib_malloc_async((void **)&d_lists, sizeof(int) * lists.size(), st)) != cudaSuccess ||
      (e = lib_malloc_async((void **)&d_next, sizeof(int) * nb, st)) != cudaSuccess ||
      (e = lib_malloc_async((void **)&d_counts, sizeof(int) * nb, st)) != cudaSuccess) {
    release();
    return cuda_fail(e, "batch descriptors");
  }
  if ((e = cudaMemcpyAsync(d_k, hk.data(), sizeof(KInst) * (size_t)count, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(d_a0, a0.data(), sizeof(DevAos) * (size_t)count, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(d_lists, lists.data(), sizeof(int) * lists.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(d_counts, counts.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = launch_init_batch(d_k, d_a0, count, st)) != cudaSuccess) {
    release();
    return cuda_fail(e, "batch init");
  }
  // one slice: every bucket's persistent kernel, concurrently on forked
  // streams; captured once as a CUDA graph and replayed
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t slice = std::max<int64_t>(1, std::min<int64_t>(Gmax, g_batch_slice));
  const int64_t nslices = Gmax > 0 ? (Gmax + slice - 1) / slice : 0;
  std::vector<cudaStream_t> side(nb, nullptr);
  std::vector<cudaEvent_t> evs(nb + 1, nullptr);
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  auto cleanup = [&]() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    for (auto &x : side)
      if (x) cudaStreamDestroy(x);
    for (auto &x : evs)
      if (x) cudaEventDestroy(x);
    release();
  };
  for (size_t b = 0; b < nb; ++b) {
    if ((e = cudaStreamCreateWithFlags(&side[b], cudaStreamNonBlocking)) != cudaSuccess) break;
    if ((e = cudaEventCreateWithFlags(&evs[b], cudaEventDisableTiming)) != cudaSuccess) break;
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&evs[nb], cudaEventDisableTiming);
  // grid per bucket: as many CTAs as fit, at most one per instance
  std::vector<int> grids(nb, 0);
  for (size_t b = 0; b < nb && e == cudaSuccess; ++b) {
    const Bucket &bk = buckets[b];
    const int per_sm = batch_ctas_per_sm(bk.model, bk.tri16, bk.xf, bk.warps, bk.wpm, bk.smem);
    if (per_sm <= 0) {
      cleanup();
      return fail(CGO_ERR_UNSUPPORTED, "no CTA of the batched kernel fits (model %d)", bk.model);
    }
    grids[b] = std::max(1, std::min<int>((int)bk.members.size(), per_sm * sms));
  }
  if (e == cudaSuccess && nslices > 0) {
    cudaStream_t cap = nullptr;
    e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaEvent_t fork = evs[nb];
      cudaError_t ce = cudaEventRecord(fork, cap);
      for (size_t b = 0; b < nb && ce == cudaSuccess; ++b) {
        const Bucket &bk = buckets[b];
        ce = cudaStreamWaitEvent(side[b], fork, 0);
        if (ce == cudaSuccess) ce = cudaMemsetAsync(d_next + b, 0, sizeof(int), side[b]);
        if (ce == cudaSuccess)
          ce = launch_batch(bk.model, bk.tri16, bk.xf, d_k, d_lists + list_off[b], d_counts + b,
                            d_next + b, bk.warps, bk.wpm, bk.smem, grids[b], slice,
                            probs[0]->timeout_ns, side[b]);
        if (ce == cudaSuccess) ce = cudaEventRecord(evs[b], side[b]);
        if (ce == cudaSuccess) ce = cudaStreamWaitEvent(cap, evs[b], 0);
      }
      const cudaError_t ee = cudaStreamEndCapture(cap, &graph);
      e = ce != cudaSuccess ? ce : ee;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    for (int64_t k = 0; k < nslices && e == cudaSuccess; ++k) {
      e = cudaGraphLaunch(exec, st);
      if (e == cudaSuccess) note_launches(nb);
    }
    if (cap) cudaStreamDestroy(cap);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cleanup();
    return cuda_fail(e, "batched solve");
  }
  cleanup();
  for (int32_t i = 0; i < count; ++i) {
    probs[i]->g = per[i].generations;
    probs[i]->has_state = true;
    probs[i]->last_warps = buckets[(size_t)0].warps;
  }
  for (size_t b = 0; b < nb; ++b)
    for (int i : buckets[b].members) {
      probs[i]->last_warps = buckets[b].warps;
      probs[i]->last_wpm = buckets[b].wpm;
      probs[i]->last_ns = 1;
      probs[i]->last_staging = hk[(size_t)i].shared_bytes > 0 ? STAGE_SMEM : STAGE_GLOBAL;
    }
  return CGO_OK;
}

cgo_status cgo_solve_static(const cgo_problem_desc *d, const cgo_params *q, uint64_t seed,
                            int32_t *out_best_sol, int64_t *out_best_cost, void *stream) {
  cgo_problem_desc dd;
  if (!d || (d->struct_size != sizeof(cgo_problem_desc) && d->struct_size != CGO_DESC_SIZE_V1 &&
             d->struct_size != CGO_DESC_SIZE_V2))
    return fail(CGO_ERR_INVALID, "desc: struct_size must be sizeof(cgo_problem_desc)");
  memset(&dd, 0, sizeof dd);
  memcpy(&dd, d, d->struct_size);  // an earlier description has no longest-route weight
  d = &dd;
  if (d->model != CGO_TSP || d->encoding != CGO_ENC_PERM)
    return fail(CGO_ERR_UNSUPPORTED, "the allocation-free solve supports TSP only");
  if (!d->pointers_on_device || !d->mat0)
    return fail(CGO_ERR_INVALID, "the allocation-free solve needs the distance matrix on the device");
  if (!out_best_sol || !out_best_cost) return fail(CGO_ERR_INVALID, "output buffers are required");
  if (d->n < 2 || d->n > 65535) return fail(CGO_ERR_INVALID, "n must be in [2, 65535]");
  cgo_params qq;
  {
    const cgo_status ls = load_params(q, &qq);
    if (ls != CGO_OK) return ls;
  }
  q = &qq;
  if (q->generations >= 0xFFFFFFFFll) return fail(CGO_ERR_INVALID, "too many generations");
  cgo_problem p;  // a description on the stack: no device state of its own
  CUDA_TRY(cudaGetDevice(&p.device), "current device");
  p.model = TSP;
  p.n = p.len = d->n;
  p.tag = d->instance_tag;
  uint32_t en = 0;
  cgo_status s = validate_params(&p, q, &en);
  if (s != CGO_OK) return s;
  if (q->init_oversample > 1 || q->init_heuristic)
    return fail(CGO_ERR_UNSUPPORTED, "the allocation-free solve starts from the plain random population");
  if (q->cross_q16 > 0)
    return fail(CGO_ERR_UNSUPPORTED, "the allocation-free solve has no buffer for crossover children");
  const int n = d->n, P = q->population;
  // carve the scratch; the triangle is sized for int32 entries (worst case)
  const size_t tri_b = up256((size_t)n * (n + 1) / 2 * 4 + 16);
  const size_t sol_b = up256((size_t)P * n * 4);
  const size_t need = tri_b + 2 * sol_b + 2 * up256((size_t)P * 8) + up256(2 * sizeof(DevAos)) +
                      up256(sizeof(DevSync)) + 256;
  if (need > kStaticScratchBytes)
    return fail(CGO_ERR_INVALID,
                "n=%d, population=%d need %zu bytes of scratch; the allocation-free solve has %zu", n,
                P, need, kStaticScratchBytes);
  void *base = nullptr;
  if ((s = static_scratch(&base)) != CGO_OK) return s;
  unsigned char *b = (unsigned char *)base;
  void *tri = b;
  b += tri_b;
  int32_t *cur = (int32_t *)b;
  b += sol_b;
  int32_t *bestsol = (int32_t *)b;
  b += sol_b;
  int64_t *cost = (int64_t *)b;
  b += up256((size_t)P * 8);
  int64_t *best = (int64_t *)b;
  b += up256((size_t)P * 8);
  DevAos *aos = (DevAos *)b;
  b += up256(2 * sizeof(DevAos));
  DevSync *sync = (DevSync *)b;
  b += up256(sizeof(DevSync));
  uint32_t *flags = (uint32_t *)b;
  cudaStream_t st = (cudaStream_t)stream;
  // the array keeps the previous call's contents: clear what starts at zero
  CUDA_TRY(cudaMemsetAsync(flags, 0, 16, st), "scratch reset");
  CUDA_TRY(launch_tsp_check(d->mat0, n, flags, st), "matrix check");
  uint32_t hf[2] = {0, 0};
  CUDA_TRY(cudaMemcpyAsync(hf, flags, sizeof hf, cudaMemcpyDeviceToHost, st), "matrix check");
  CUDA_TRY(cudaStreamSynchronize(st), "matrix check");
  if (hf[0]) return fail(CGO_ERR_UNSUPPORTED, "the allocation-free solve needs a symmetric distance matrix");
  p.tri16 = hf[1] <= 32767u ? 1 : 0;
  CUDA_TRY(cudaMemsetAsync(tri, 0, tri_b, st), "scratch reset");
  CUDA_TRY(build_triangle(d->mat0, n, p.tri16, tri, st), "triangle");
  p.d_mat0 = const_cast<int32_t *>(d->mat0);
  p.d_tri = tri;
  p.params = *q;
  p.seed = seed;
  p.enabled = en;
  p.d_cur = cur;
  p.d_bestsol = bestsol;
  p.d_cost = cost;
  p.d_best = best;
  p.d_aos = aos;
  p.d_sync = sync;
  KInst h = base_kinst(&p);
  CUDA_TRY(launch_init(h, st), "init launch");
  DevAos a0;
  memset(&a0, 0, sizeof a0);
  a0.T = q->T0_q32;
  for (int i = 0; i < kNops; ++i) a0.w_op[i] = ((en >> i) & 1u) ? op_w0(*q, i) : 0u;
  for (int i = 0; i < 3; ++i) a0.w_k[i] = q->k_w0_q16[i];
  h.aos_out = aos;
  CUDA_TRY(launch_init_aos(h, a0, st), "init launch");
  int cur_aos = 0;
  if (q->generations > 0) {
    int warps = 0, wpm = 1, ns = 1;
    int64_t smem = 0;
    h = base_kinst(&p);
    if ((s = choose_launch(&p, h, &warps, &wpm, &ns, &smem)) != CGO_OK) {
      // leave no queued work behind in the shared array
      cudaStreamSynchronize(st);
      return s;
    }
    h.g_begin = 0;
    h.g_end = q->generations;
    h.aos_in = aos;
    h.aos_out = aos + 1;
    CUDA_TRY(cudaMemsetAsync(sync, 0, sizeof(DevSync), st), "scratch reset");
    CUDA_TRY(cudaMemsetAsync(sync->elite, 0x7F, sizeof(sync->elite), st), "scratch reset");
    CUDA_TRY(launch_evolve_single(h, warps, wpm, ns, smem, p.timeout_ns, st), "evolve launch");
    CUDA_TRY(launch_finalize(h, st), "finalize launch");
    cur_aos = 1;
  }
  CUDA_TRY(launch_copy_elite(aos + cur_aos, bestsol, n, out_best_sol, out_best_cost, st), "copy elite");
  uint32_t err = 0;
  if (q->generations > 0)
    CUDA_TRY(cudaMemcpyAsync(&err, &sync->error, 4, cudaMemcpyDeviceToHost, st), "reading status");
  CUDA_TRY(cudaStreamSynchronize(st), "synchronising stream");
  if (err) return fail(CGO_ERR_TIMEOUT, "a member barrier timed out (flags 0x%x)", err);
  return CGO_OK;
}

/* Test-only fault injection: what = 1 adds `value` phantom members to every member barrier,
 * so the barrier cannot complete and the bounded wait must give up;
 * what = 2 sets the barrier wait limit to `value` milliseconds. */
cgo_status cgo_debug_inject(cgo_problem *p, int32_t what, int64_t value) {
  if (!p && what != 3 && what != 4) return fail(CGO_ERR_INVALID, "NULL problem");
  if (what == 1) {
    if (value < 0 || value > 1024) return fail(CGO_ERR_INVALID, "phantom members out of range");
    p->phantom_members = (uint32_t)value;
  } else if (what == 2) {
    if (value < 1 || value > 600000) return fail(CGO_ERR_INVALID, "timeout out of range");
    p->timeout_ns = (uint64_t)value * 1000000ull;
  } else if (what == 3) {
    if (value < 1 || value > (1ll << 31)) return fail(CGO_ERR_INVALID, "slice out of range");
    g_batch_slice = value;
  } else if (what == 4) {
    if (value < 0 || value > (1ll << 31)) return fail(CGO_ERR_INVALID, "allocation index out of range");
    g_alloc_fail.store(value);
  } else {
    return fail(CGO_ERR_INVALID, "unknown injection");
  }
  return CGO_OK;
}

}  // extern "C"
