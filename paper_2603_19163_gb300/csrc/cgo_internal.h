// Internal structures shared by the host runtime (cgo_api.cu) and the
// kernels (cgo_kernels.cu).  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace cgo {

constexpr int kNops = 11;      // operator slots (cgo_op), the row level in 8 .. 10
// window counts, one per lane of a warp: u_op[kNops] at lanes 0.., v_op at
// kStatV.., u_k[3] at kStatUK.., v_k[3] at kStatVK..
constexpr int kStatV = kNops, kStatUK = 2 * kNops, kStatVK = 2 * kNops + 3;
constexpr int kStats = 2 * kNops + 6;
static_assert(kStats <= 32, "window counts must fit the lanes of a warp");
constexpr int kMaxWarps = 8;    // warps per CTA (kernel launch bound 256 threads)
// warps per CTA of a single solve with 3 or 4 generations in flight (one
// member of 4 warps per generation; launch bound 32 x that)
constexpr int kMaxWarpsDeep = 16;
constexpr int kMaxAgents = 64;  // GAP agents

// ATSP: the TSP of an asymmetric matrix (the kernels' own model id; the
// public model stays CGO_TSP)
enum Model { TSP = 0, QAP = 1, KNAPSACK = 2, GAP = 3, CVRPTW = 4, ATSP = 5 };
enum Op { SWAP = 0, TWO_OPT = 1, INSERT = 2, OR_OPT = 3, FLIP = 4, PERTURB = 5, THREE_OPT = 6,
          SEGMENT = 7 /* seg_flip (binary), seg_reset (integer) */,
          ROW_SWAP = 8, ROW_MERGE = 9, ROW_SPLIT = 10 /* CVRPTW's routes */ };
enum Staging { STAGE_AUTO = 0, STAGE_SMEM = 1, STAGE_GLOBAL = 2 };

// Per-instance search scalars (device memory, double-buffered in/out per launch).
struct DevAos {
  uint64_t T;                 // Q32.32
  int64_t g;                  // generations completed
  uint32_t w_op[kNops];       // Q16, global operator ids
  uint32_t w_k[3];
  uint32_t stag;
  uint32_t pad0;
  int64_t elite_prev;
  uint32_t pend[kStats];      // counts of the open (incomplete) AOS window
  int32_t elite;              // member index of the elite (after finalize)
  int32_t pad1;
  int64_t elite_cost;
  uint64_t cum[kStats];       // counts of every closed window since the solve began
                              // (reported to the caller; the search never reads them)
};

// Per-launch synchronisation block (zeroed/reset by the host before a launch).
struct DevSync {
  uint32_t arrive;            // members arrived at window barriers (cumulative)
  uint32_t error;             // bit 0: timeout, bit 1: invalid state
  uint32_t acc[2][32];        // window count accumulators, cumulative per slot
  int64_t elite[2];           // atomicMin of member bests per slot
  uint32_t pend_out[kStats];  // counts of a window left open at the end
  uint32_t pad[10];
};

// One instance's work for a launch.  Lives in device memory.
struct KInst {
  // instance
  int32_t model, n, len, m;
  int64_t capacity, lam0, lam1;
  int64_t wdist, wveh;  // CVRPTW objective weights (distance, vehicles used)
  int64_t wlong;        // CVRPTW: weight of the longest route's distance (0 = off)
  // CVRPTW lexicographic mode (lex_n > 0): the cost is the key of the
  // order; the packed route cost's fields start at bits 0, lex_sh[0..2]
  int32_t lex_n, lex_obj[3], lex_sh[3];
  int64_t lex_w[3], lex_R[3];
  int32_t lb, ub;
  uint32_t tag;
  int32_t tri16;              // TSP triangle stored as int16
  const int32_t *mat0, *mat1, *vec0, *vec1, *vec2, *vec3;
  const void *tri;            // TSP upper triangle (row-major, i <= j)
  const int4 *node;           // CVRPTW: per node {ready, due, service, demand}
  int32_t cv32;               // 32-bit delta arithmetic is exact: CVRPTW route
                              // quantities, QAP swap deltas
  int32_t pad3;
  int64_t shared_bytes;       // bytes of instance data staged per CTA (0 = global)
  // parameters
  int32_t P, C;
  int32_t members;            // barrier arrivals expected per window (= P)
  int32_t pad1;
  uint32_t U, E;
  uint64_t alpha;
  uint32_t ema_a, w_floor, w_cap, stag_limit;
  uint32_t op_cap[kNops];
  uint32_t enabled;           // effective enabled-operator mask
  uint32_t pad0;
  uint64_t seed;
  // launch range
  int64_t g_begin, g_end;
  int64_t G_total;            // batched slices: generations of the whole solve
  int32_t local_sync;         // 1: all members in one CTA, barriers are CTA-local
  int32_t pad2;
  // state
  int32_t *cur, *bestsol;
  int64_t *cost, *best;
  const DevAos *aos_in;
  DevAos *aos_out;
  DevSync *sync;
  // oversampled / heuristic start (pool of K*P random starts + n_heur
  // permutations, the P cheapest become the members)
  int32_t K_over, n_heur;
  // islands and migration
  int32_t islands, mstrat;
  uint32_t mperiod, mN;
  // crossover probability per window (Q16); pool_sol rows 0..P-1 hold the
  // children of models without a shared-memory child, rows P..3P-1 the
  // members' bests as crossover parents (two alternating sets of P rows)
  uint32_t cross_q16;
  const int32_t *heur;        // n_heur x n
  int32_t *pool_sol;          // (K*P + n_heur) x len, or 3P x len with crossover
  int64_t *pool_cost;
};

// host-side launchers (cgo_kernels.cu)
cudaError_t launch_init(const KInst &h, cudaStream_t st);
cudaError_t launch_init_aos(const KInst &h, const DevAos &a0, cudaStream_t st);
cudaError_t launch_evolve_single(const KInst &h, int warps, int wpm, int ns, int64_t smem_bytes,
                                 uint64_t timeout_ns, cudaStream_t st);
cudaError_t launch_finalize(const KInst &h, cudaStream_t st);
cudaError_t build_triangle(const int32_t *d_mat, int n, int tri16, void *d_tri,
                           cudaStream_t st);
cudaError_t launch_tsp_check(const int32_t *d_mat, int n, uint32_t *d_flags, cudaStream_t st);
cudaError_t launch_copy_elite(const DevAos *d_aos, const int32_t *d_bestsol, int len,
                              int32_t *out_sol, int64_t *out_cost, cudaStream_t st);
cudaError_t launch_init_batch(const KInst *d_insts, const DevAos *d_a0s, int count, cudaStream_t st);
// batched kernels: xf = 1 for instances that take island migration or crossover
int batch_ctas_per_sm(int model, int tri16, int xf, int warps, int wpm, int64_t smem_bytes);
cudaError_t launch_batch(int model, int tri16, int xf, const KInst *d_insts, const int *d_list,
                         const int *d_count, int *d_next, int warps, int wpm, int64_t smem_bytes,
                         int grid, int64_t slice, uint64_t timeout_ns, cudaStream_t st);
// whether an instance's search takes island migration or crossover
// (2: migration, and crossover if any; 1: crossover alone; 0: neither)
inline int takes_xf(const KInst &h) { return h.islands > 1 ? 2 : (h.cross_q16 > 0 ? 1 : 0); }
int64_t batch_smem_bytes(const KInst &h, int warps, int wpm, bool staged);
// shared-memory needs of the evolve kernel
int64_t smem_per_warp(const KInst &h);
int64_t instance_data_bytes(const KInst &h);
int64_t evolve_smem_bytes(const KInst &h, int warps, int wpm, int ns, bool staged);
int64_t smem_instance(const KInst &h);
int max_coresident_ctas(const KInst &h, int warps, int wpm, int ns, int64_t smem_bytes);
int64_t max_smem_optin();
// random-gather rate microbenchmark (kind 0: 16-bit gathers from a shared
// buffer of 2^log2n elements, one CTA per SM; kind 1: 32-bit gathers from a
// global buffer of 2^log2n elements)
cudaError_t measure_gather_peak(int kind, int log2n, double *per_s, double *ms);
// process-wide count of kernels launched by the library
void note_launches(uint64_t n);
uint64_t launches_total();

}  // namespace cgo
