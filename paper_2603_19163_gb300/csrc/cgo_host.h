// Host-runtime internals shared by the C-ABI translation units (the single
// and batched solves in cgo_api.cu, the serving loop in cgo_server.cu).
#pragma once
#include <atomic>
#include <cstdint>
#include <string>

#include "cgo.h"
#include "cgo_internal.h"

// A problem handle: device copies of the instance, the search state of its
// last solve, launch-shape overrides and test hooks.
struct cgo_problem {
  int device = 0;
  int model = 0, n = 0, len = 0, m = 0, V = 0;
  int64_t capacity = 0, lam0 = 0, lam1 = 0;
  int64_t wdist = 1, wveh = 0;  // CVRPTW objective weights
  int64_t wlong = 0;            // CVRPTW: weight of the longest route
  int asym = 0;                 // TSP with an asymmetric matrix (the kernels' ATSP path)
  // CVRPTW lexicographic mode: objectives, bucket widths, radices and the
  // bit positions of the packed cost's fields
  int lex_n = 0;
  int lex_obj[3] = {0, 0, 0};
  int64_t lex_w[3] = {1, 1, 1}, lex_R[3] = {1, 1, 1};
  int lex_sh[3] = {0, 0, 0};
  int lb = 0, ub = 0;
  uint32_t tag = 0;
  int32_t *d_mat0 = nullptr, *d_mat1 = nullptr, *d_vec[4] = {nullptr, nullptr, nullptr, nullptr};
  void *d_tri = nullptr;
  int tri16 = 0;
  int4 *d_node = nullptr;  // CVRPTW packed node data
  int cv32 = 0;
  // search state
  bool has_state = false;
  cgo_params params{};
  uint64_t seed = 0;
  uint32_t enabled = 0;
  int P_alloc = 0;
  int32_t *d_cur = nullptr, *d_bestsol = nullptr;
  int64_t *d_cost = nullptr, *d_best = nullptr;
  cgo::DevAos *d_aos = nullptr;  // [2]
  cgo::DevSync *d_sync = nullptr;
  // start pool (oversampled / heuristic start)
  int32_t *d_heur = nullptr;     // heuristic start permutations, n_heur x n
  int n_heur = 0;
  int32_t *d_pool = nullptr;
  int64_t *d_pool_cost = nullptr;
  int64_t pool_cap = 0;
  int aos_cur = 0;
  int64_t g = 0;
  // launch shape
  int warps_override = 0, wpm_override = 0, staging_override = 0, ns_override = 0;
  int last_warps = 0, last_wpm = 0, last_staging = 0, last_ns = 0;
  // events around the last evolve launch (kernel time on the launching stream)
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  bool timed = false;
  int64_t timed_gens = 0;
  // test-only fault injection
  uint32_t phantom_members = 0;
  uint64_t timeout_ns = 10ull * 1000 * 1000 * 1000;
  std::atomic<int> busy{0};
};

namespace cgo {
namespace host {

cgo_status fail(cgo_status s, const char *fmt, ...);
cgo_status cuda_fail(cudaError_t e, const char *what);
int encoding_of(int model);
int64_t pad16(int64_t b);
extern int64_t g_batch_slice;

// Exclusive use of a handle for the duration of a call (ok = false if busy).
struct Guard {
  cgo_problem *p;
  bool ok;
  explicit Guard(const cgo_problem *q) : p(const_cast<cgo_problem *>(q)) {
    int z = 0;
    ok = p->busy.compare_exchange_strong(z, 1);
  }
  ~Guard() {
    if (ok) p->busy.store(0);
  }
};

cudaStream_t host_stream();
// A cgo_params of the current or the earlier size (CGO_PARAMS_SIZE_V1, without
// the row level) as a full current struct; the earlier size leaves the row
// operators off.
cgo_status load_params(const cgo_params *in, cgo_params *out);
// weight / cap of operator slot i (0 .. kNops - 1)
inline uint32_t op_w0(const cgo_params &q, int i) {
  return i < CGO_NOPS ? q.op_w0_q16[i] : q.row_w0_q16[i - CGO_NOPS];
}
inline uint32_t op_capq(const cgo_params &q, int i) {
  return i < CGO_NOPS ? q.op_cap_q16[i] : q.row_cap_q16[i - CGO_NOPS];
}
// q must be a current-size struct (load_params)
cgo_status validate_params(const cgo_problem *p, const cgo_params *q, uint32_t *enabled);
cgo_status ensure_state(cgo_problem *p, int P);
int64_t pool_size(const cgo_problem *p, const cgo_params &q);
cgo_status ensure_pool(cgo_problem *p, const cgo_params &q);
KInst base_kinst(const cgo_problem *p);
// launch shape of a batched (CTA-local) instance: warps per member, warps
// per CTA, shared memory of a unit; fails if the instance cannot fit a CTA
cgo_status batch_shape(cgo_problem *p, const cgo_params &q, KInst &h, int *wpm, int *warps,
                       int64_t *smem, int64_t *smem_class);
DevAos initial_aos(const cgo_params &q, uint32_t enabled);

}  // namespace host
}  // namespace cgo

#define CUDA_TRY(call, what)                              \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cgo::host::cuda_fail(e_, what); \
  } while (0)
