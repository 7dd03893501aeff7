/*
 * cgo — GB300-native population search for combinatorial optimisation.
 *
 * C ABI of the per-solution search generation of cuGenOpt (arxiv 2603.19163):
 * for every solution of a population, in parallel, each generation draws a
 * K-step neighbourhood move from the adaptively weighted operator set,
 * evaluates its exact integer cost delta against the instance data, applies
 * Metropolis acceptance with geometric cooling and updates the two-level
 * adaptive-operator-selection (AOS) weights and the elite
 * (Alg. "evolve", Alg. "aos", Eq. "ema", Sec. 3.2-3.4 and 4.2).
 *
 * Conventions (every entry point):
 *  - returns a cgo_status; no C++ exception and no abort crosses the ABI;
 *  - on a non-OK status, cgo_last_error() returns a message for this thread;
 *  - all sizes are element counts unless stated; all integers are exact;
 *  - `cuda_stream` is a cudaStream_t (NULL = the legacy default stream); the
 *    call enqueues its work there and waits for it before returning;
 *  - a handle may be used by one thread at a time; a call on a handle that
 *    is already in use returns CGO_ERR_BUSY.
 * The library runs only on the GPU (sm_103a); it has no CPU fallback.
 */
#ifndef CGO_H
#define CGO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CGO_OK = 0,
  CGO_ERR_INVALID = 1,      /* an argument violates the documented limits */
  CGO_ERR_NOMEM = 2,        /* device or host allocation failed */
  CGO_ERR_CUDA = 3,         /* a CUDA runtime call failed (message has the error) */
  CGO_ERR_UNSUPPORTED = 4,  /* valid, but outside what the GPU path implements */
  CGO_ERR_TIMEOUT = 5,      /* a bounded device-side wait gave up */
  CGO_ERR_BUSY = 6,         /* the handle (or server slot) is in use */
  CGO_ERR_STATE = 7,        /* no search state yet, or it was lost to an error */
  CGO_ERR_CANCELLED = 8     /* the request was cancelled (cgo_cancel) */
} cgo_status;

/* Encodings (Sec. 3.1.1). */
typedef enum { CGO_ENC_PERM = 0, CGO_ENC_BINARY = 1, CGO_ENC_INTEGER = 2 } cgo_encoding;

/* Cost models.  Costs are int64 and minimised.
 *  TSP      perm of n cities; sum of D[a_k][a_(k+1) mod n]; mat0 = D (n*n).
 *           D may be asymmetric (the tour's direction then counts; the
 *           library keeps the full matrix instead of its triangle).
 *  QAP      perm of n; sum_i sum_j F[i][j]*D[a_i][a_j]; mat0 = F, mat1 = D (n*n).
 *           F and D may be asymmetric with a non-zero diagonal.
 *  KNAPSACK binary n; -sum v x + lambda*max(0, sum w x - capacity);
 *           vec0 = w, vec1 = v (n); lambda = penalty0, or 1 + max v if 0.
 *  GAP      integer n jobs in [0, m-1]; sum_j c[x_j][j] +
 *           lambda * sum_a max(0, load_a - cap_a), load_a = sum_{x_j=a} r[a][j];
 *           mat0 = c, mat1 = r (m*n, row = agent), vec0 = cap (m);
 *           lambda = penalty0, or 1 + max c if 0.
 *  CVRPTW   perm of n + vehicles - 1 symbols: s < n is customer s+1, s >= n
 *           ends a route.  Node 0 is the depot.  mat0 = travel (n+1)^2,
 *           vec0..vec3 = demand, ready, due, service (n+1 each).  Per route
 *           from the depot at t = 0: t = max(t + d, ready), late +=
 *           max(0, t - due), t += service; back at the depot t += d, late +=
 *           max(0, t - due_0); a route with no customer costs nothing.
 *           cost = distance + penalty0*sum max(0, load - capacity)
 *           + penalty1*late (each 100 if 0). */
typedef enum { CGO_TSP = 0, CGO_QAP = 1, CGO_KNAPSACK = 2, CGO_GAP = 3, CGO_CVRPTW = 4 } cgo_model;

/* Operators (Table "operators").  Bit i of cgo_params.op_mask enables op i. */
typedef enum {
  CGO_OP_SWAP = 0,     /* perm: exchange a[i], a[j] */
  CGO_OP_TWO_OPT = 1,  /* perm: reverse a[min(i,j) .. max(i,j)] */
  CGO_OP_INSERT = 2,   /* perm: remove a[i], re-insert so it lands at index j */
  CGO_OP_OR_OPT = 3,   /* perm: move a block of 2 or 3 elements (needs length >= 4) */
  CGO_OP_FLIP = 4,     /* binary: x_i ^= 1 */
  CGO_OP_PERTURB = 5,  /* integer: x_i <- another value of [lb, ub] */
  CGO_OP_THREE_OPT = 6, /* perm: exchange the adjacent segments a[i..j-1], a[j..k-1] at three
                          distinct cut points i < j < k of 0..length (segment level,
                          Table "operators"); off in the default mask */
  /* slot 7 holds the segment-level operator of the binary and of the integer
     set (Table "operators"): a segment of L = min(2 + (x & 1), length)
     elements from i = pos(a, length - L + 1); needs length >= 2; off in the
     default mask */
  CGO_OP_SEG_FLIP = 7,  /* binary: flip every element of the segment */
  CGO_OP_SEG_RESET = 7, /* integer: add one offset d = 1 + pos(b, R - 1) to every element of
                           the segment, modulo the range R (the random reset's rule) */
  /* row level (Table "operators"; Sec. 3.1's multi-row solutions): the rows
     of CVRPTW's separator encoding are its V routes, route r running from
     just after the r-th separator to the next one; they need V >= 2 and
     are off in the default mask */
  CGO_OP_ROW_SWAP = 8,  /* routes r1 = pos(a, V), r2 = pos(b, V - 1) stepped over r1 exchange
                           their customers */
  CGO_OP_ROW_MERGE = 9, /* r = pos(a, V - 1): route r takes route r + 1's customers (the
                           separator between them moves to the end of route r + 1) */
  CGO_OP_ROW_SPLIT = 10 /* r = pos(a, V): with c >= 2 customers on r and an empty route, the
                           separator of the lowest-index empty route moves inside r after its
                           first 1 + pos(b, c - 1) customers; otherwise nothing changes */
} cgo_op;

/* operator slots in cgo_params.op_w0_q16 / op_cap_q16 and cgo_state's
   arrays (slots 0 .. 7); the row level's slots 8 .. 10 have arrays of their
   own appended to those structs */
#define CGO_NOPS 8
#define CGO_NROW 3
#define CGO_NOPS_ALL (CGO_NOPS + CGO_NROW)

typedef struct cgo_problem cgo_problem;  /* opaque; owns device copies + search state */

/* Problem statement (Sec. 3.1: encoding, size, data, constraints). */
typedef struct {
  uint32_t struct_size;        /* = sizeof(cgo_problem_desc) */
  int32_t encoding;            /* must be the model's encoding (cgo_encoding) */
  int32_t model;               /* cgo_model */
  int32_t n;                   /* 2 <= n; solution length <= 65535 */
  const int32_t *mat0, *mat1;  /* row-major matrices, see cgo_model */
  const int32_t *vec0, *vec1, *vec2, *vec3;
  int64_t capacity;            /* knapsack capacity; CVRPTW vehicle capacity */
  int32_t lb, ub;              /* integer bounds (GAP: ignored, [0, m-1]) */
  int32_t m;                   /* GAP agents, 2 <= m <= 64 */
  int32_t vehicles;            /* CVRPTW vehicles, >= 1 */
  int64_t penalty0, penalty1;  /* lambdas; 0 = default */
  int32_t pointers_on_device;  /* 0: host pointers; 1: device pointers (e.g. a
                                  torch tensor's data_ptr) on the current device */
  uint32_t instance_tag;       /* word 1 of every Philox counter of this instance */
  /* CVRPTW objective weights (Sec. 6.8, weighted mode; a weight above every
     difference of the lower-priority terms gives the lexicographic order):
     cost = weight_distance * distance + penalties + weight_vehicles * routes
     that visit a customer.  0 = default (1 and 0); other models ignore them. */
  int64_t weight_distance, weight_vehicles;
  /* --- appended --- */
  /* CVRPTW: weight of the longest route's distance (the third objective of
     Sec. 6.8's tri-objective VRP; 0 = off): cost += weight_longest * the
     largest distance driven by one vehicle */
  int64_t weight_longest;
  /* --- appended --- */
  /* CVRPTW lexicographic mode (Sec. 6.8, Table "lexicographic_mode"): the
     first lex_n (0 = off, the weighted cost above; 1..3) entries of lex_obj
     name the objectives in priority order (CGO_LEX_DISTANCE,
     CGO_LEX_VEHICLES, CGO_LEX_LONGEST, each at most once), lex_tol their
     tolerances (>= 0).  Solutions compare by their penalty (penalty0 *
     capacity excess + penalty1 * lateness) first, then by each objective o
     in buckets of width tol + 1 (values in one bucket tie and the next
     objective decides).  The cost is then this order's key:
       key = ((penalty * R_1 + o_1 / (tol_1 + 1)) * R_2 + o_2 / (tol_2 + 1)) ...
       R_i = omax_i / (tol_i + 1) + 1, omax = (n + vehicles) * the largest
       travel time for the two distances, vehicles for the vehicle count.
     Needs travel times >= 0 and the three weights left at 0; a mode whose
     key could exceed 2^62 returns CGO_ERR_UNSUPPORTED. */
  int32_t lex_n;
  int32_t lex_obj[3];
  int64_t lex_tol[3];
} cgo_problem_desc;

/* The size of cgo_problem_desc before weight_longest was appended (accepted
 * by the calls that take a description: no longest-route term). */
#define CGO_DESC_SIZE_V1 ((uint32_t)offsetof(cgo_problem_desc, weight_longest))
/* The size before the lexicographic mode was appended (accepted: mode off). */
#define CGO_DESC_SIZE_V2 ((uint32_t)offsetof(cgo_problem_desc, lex_n))

/* CVRPTW objectives of the lexicographic mode. */
enum { CGO_LEX_DISTANCE = 0, CGO_LEX_VEHICLES = 1, CGO_LEX_LONGEST = 2 };

/* Search parameters.  Fixed point: Q16 weights (65536 = 1.0), Q32.32
 * temperature, Q0.32 cooling factor. */
typedef struct {
  uint32_t struct_size;        /* = sizeof(cgo_params) */
  int32_t population;          /* P, 1 .. 65536 */
  int32_t candidates;          /* C per solution per generation, 1 .. 4096 (paper T = 128) */
  int64_t generations;         /* G for cgo_solve; >= 0 */
  uint32_t op_mask;            /* enabled operators (bits of cgo_op) */
  uint32_t op_w0_q16[CGO_NOPS];/* initial operator weights (disabled ops ignored) */
  uint32_t k_w0_q16[3];        /* initial K-step weights for k = 1, 2, 3 */
  uint64_t T0_q32;             /* initial temperature */
  uint64_t alpha_q32;          /* cooling: T <- (T * alpha) >> 32 each generation */
  uint32_t aos_interval;       /* U: AOS update after every U-th generation, >= 1 */
  uint32_t ema_alpha_q16;      /* EMA a of Eq. "ema", <= 65536 */
  uint32_t w_floor_q16;        /* w_floor, >= 8 */
  uint32_t w_cap_q16;          /* w_cap, >= w_floor */
  uint32_t op_cap_q16[CGO_NOPS];/* per-operator caps (>= w_floor for enabled ops) */
  uint32_t stag_limit;         /* AOS updates without elite gain before the K reset; 0 = off */
  uint32_t elite_period;       /* E: elite injection after every E-th generation; 0 = off;
                                  the GPU path needs E to be a multiple of U */
  uint32_t init_oversample;    /* K of the oversampled start (Sec. 3.4.1): K*P random
                                  starts, the P cheapest kept; 0 or 1 = plain start;
                                  K <= 64 and K*P <= 16384 */
  uint32_t init_heuristic;     /* 1: the row/column-sum permutations of each square
                                  data matrix (Sec. 3.4.2; TSP, QAP) join the pool */
  uint32_t islands;            /* I islands of P/I consecutive members (Sec. 3.4.3);
                                  0 or 1 = one population; I divides P */
  uint32_t migrate_period;     /* migration after every such generation (a multiple of
                                  aos_interval on the GPU); 0 = off */
  uint32_t migrate_strategy;   /* 0 ring: each island's best to the next island's worst;
                                  1 top-N: the population's N best to every island's N
                                  worst; 2 hybrid: ring and top-N alternate */
  uint32_t migrate_n;          /* N of top-N, 1 .. P/I */
  uint32_t cross_q16;          /* crossover probability per member and AOS window, Q16
                                  (<= 65536; 0 = off): order crossover for permutations,
                                  uniform crossover for binary / integer vectors (Table
                                  "operators", crossover level) with another member's best */
  /* --- appended: the row level (operator slots 8 .. 10) --- */
  uint32_t row_w0_q16[CGO_NROW];  /* initial weights of CGO_OP_ROW_SWAP .. _SPLIT */
  uint32_t row_cap_q16[CGO_NROW]; /* their caps */
} cgo_params;

/* The size of cgo_params and cgo_state before the row-level fields were
 * appended.  Calls that take these structs accept that size too: an
 * earlier cgo_params leaves the row operators off, an earlier cgo_state
 * carries no row-level weights or counts (so it cannot be written back
 * while row operators are on).  cgo_params_default fills the earlier
 * layout when the caller sets struct_size to it before the call.  (Both
 * sizes are the earlier structs' sizeof, tail padding included.) */
#define CGO_PARAMS_SIZE_V1 ((uint32_t)((offsetof(cgo_params, row_w0_q16) + 7u) & ~(size_t)7u))
#define CGO_STATE_SIZE_V1 ((uint32_t)((offsetof(cgo_state, w_row_q16) + 7u) & ~(size_t)7u))

/* Full search state (checkpoint).  Scalars are filled/read by value; the
 * four arrays are caller-owned host buffers (NULL = skip on get). */
typedef struct {
  uint32_t struct_size;        /* = sizeof(cgo_state) */
  int32_t population, length;  /* P and the solution length */
  int64_t generation;          /* generations completed */
  uint64_t T_q32;
  uint32_t w_op_q16[CGO_NOPS], w_k_q16[3];
  uint32_t stag;               /* AOS updates since the elite last improved */
  int64_t elite_prev;          /* elite cost at the last AOS update */
  uint32_t u_op[CGO_NOPS], v_op[CGO_NOPS], u_k[3], v_k[3]; /* counts of the open window */
  int32_t *cur;                /* [P * length] current solutions */
  int32_t *best_sol;           /* [P * length] best solution of each member */
  int64_t *cost;               /* [P] current costs */
  int64_t *best_cost;          /* [P] best costs */
  /* --- appended: the row level (operator slots 8 .. 10) --- */
  uint32_t w_row_q16[CGO_NROW];
  uint32_t u_row[CGO_NROW], v_row[CGO_NROW];  /* counts of the open window */
} cgo_state;

/* Launch shape (the autotuner's choice, or a caller override).  The C
 * candidates of a member's generation are split over warps_per_member warps.
 * With gens_in_flight = s > 1 a member has s such warp sets: set i evaluates
 * generation g + i against the same solution, which stands unless an
 * earlier generation of the set accepts a move (the later ones are then
 * evaluated again); the results are the same either way.  A CTA holds
 * warps_per_cta / (warps_per_member * gens_in_flight) members.  Launch
 * shapes never change results. */
typedef struct {
  uint32_t struct_size;        /* = sizeof(cgo_launch) */
  int32_t warps_per_cta;       /* 0 = auto; else 1 .. 8 (1 .. 16 with 3 or 4
                                  generations in flight), a multiple of
                                  warps_per_member * gens_in_flight */
  int32_t warps_per_member;    /* 0 = auto; else 1, 2 or 4 */
  int32_t staging;             /* 0 = auto, 1 = instance data in shared memory,
                                  2 = instance data read through L2 */
  int32_t gens_in_flight;      /* 0 = auto; 1 .. 4 for single solves with at
                                  most 32 * warps_per_member candidates (3 and 4
                                  with warps_per_member = 4 and neither island
                                  migration nor crossover, not for an asymmetric
                                  TSP matrix); batched solves use 1 */
} cgo_launch;

/* Create a problem: validates the description and deep-copies the data to
 * the current device, so the caller may free its arrays on return.
 * Errors: CGO_ERR_INVALID (sizes, encoding/model mismatch, data that could
 * overflow an int64 cost), CGO_ERR_NOMEM, CGO_ERR_CUDA.  *out is NULL on
 * error. */
cgo_status cgo_problem_create(const cgo_problem_desc *desc, cgo_problem **out);

/* Free the problem and its device memory.  NULL is accepted. */
cgo_status cgo_problem_destroy(cgo_problem *prob);

/* Default parameters for this problem: P = 32, C = 128, G = 2000, every
 * operator of the encoding enabled with the L1 profile priors (Sec. 4.1,
 * Table "weight_preset": O(1) operators 1.0, or-opt 0.80/0.70/0.30 for
 * solution length <= 100 / <= 250 / > 250, normalised to Q16),
 * K weights (0.8, 0.15, 0.05), T0 = 100, alpha = 0.999, U = 10 (I = 10,
 * Sec. 4.2.2), EMA a = 0.8, floor 0.05, cap 0.6, stagnation after 5
 * updates, no elite injection.  3-opt, the segment operators and the row
 * operators are off in the default mask; their priors are filled in (the
 * row level takes the O(1) prior 1.0), normalised with the default set.
 * out->struct_size = CGO_PARAMS_SIZE_V1 before the call asks for the earlier
 * layout; otherwise the current one is written. */
cgo_status cgo_params_default(const cgo_problem *prob, cgo_params *out);

/* Override the launch shape (warps per CTA, staging mode) used by the next
 * solves of this problem; results do not depend on it. */
cgo_status cgo_set_launch(cgo_problem *prob, const cgo_launch *launch);
/* The launch shape the last solve used (after autotuning). */
cgo_status cgo_get_launch(const cgo_problem *prob, cgo_launch *out);

/* Initialise a population from `seed` (Philox key) and run
 * params->generations generations (Alg. "evolve" + Alg. "aos").
 * Replaces any previous state of the handle.  Waits for completion. */
cgo_status cgo_solve(cgo_problem *prob, const cgo_params *params, uint64_t seed,
                     void *cuda_stream);

/* Run `generations` more generations of the current state (same params and
 * seed).  Splitting a solve this way gives bit-identical results. */
cgo_status cgo_solve_continue(cgo_problem *prob, int64_t generations, void *cuda_stream);

/* Copy the instance elite (lowest best cost, ties to the lowest member
 * index) to host memory: out_sol gets `length` int32 values (cap >= length,
 * else CGO_ERR_INVALID); out_cost its cost.  Either pointer may be NULL.
 * CGO_ERR_STATE before the first solve. */
cgo_status cgo_best(const cgo_problem *prob, int32_t *out_sol, int32_t cap, int64_t *out_cost);

/* Device time of the last evolve-kernel launch of this problem, measured
 * with CUDA events recorded on the launching stream just before and after
 * it, and the generations that launch ran.  CGO_ERR_STATE if none yet. */
cgo_status cgo_last_kernel_time(const cgo_problem *prob, double *ms, int64_t *generations);

/* The elite as a multi-row solution (Sec. 3.1: rows of variable length,
 * "dim2_sizes", over a partition of the elements; the Perm-Partition
 * structure).  CVRPTW's rows are its vehicles' routes: the separator
 * sequence the search works on is this solution laid out flat, route r
 * running from just after the r-th separator to the next one.  Fills
 * out_rows with the customers (0 .. n-1) row after row (cap >= n),
 * row_lengths[r] with each row's length (max_rows >= vehicles) and
 * *out_rows_count with the number of rows (vehicles; empty routes are rows
 * of length 0) and *out_cost with the elite's cost.  Other models have one
 * row: the whole solution.  Host buffers; CGO_ERR_INVALID for short
 * buffers, CGO_ERR_STATE before the first solve. */
cgo_status cgo_best_rows(const cgo_problem *prob, int32_t *out_rows, int32_t cap,
                         int32_t *row_lengths, int32_t max_rows, int32_t *out_rows_count,
                         int64_t *out_cost);

/* Solution length of this problem (n, or n + vehicles - 1 for CVRPTW). */
cgo_status cgo_solution_length(const cgo_problem *prob, int32_t *out_len);

/* Read the full search state into `out` (struct_size set by the caller;
 * population and length are filled in; arrays copied if non-NULL). */
cgo_status cgo_state_get(const cgo_problem *prob, cgo_state *out);

/* Replace the search state (resume from a checkpoint taken with
 * cgo_state_get under the same params and seed).  All four arrays are
 * required.  Costs are taken as given. */
cgo_status cgo_state_set(cgo_problem *prob, const cgo_params *params, uint64_t seed,
                         const cgo_state *state);

/* The search state as one opaque, versioned byte buffer (a checkpoint
 * file's contents): a header (magic "CGO1", format version, population,
 * solution length, generation), the scalars of cgo_state including the row
 * level, then the four arrays.  cgo_state_export writes it into buf (cap
 * bytes; *used gets the size, which is also returned with
 * CGO_ERR_INVALID when cap is too small or buf is NULL, so a first call can
 * size the buffer).  cgo_state_import checks the header and resumes from
 * it exactly as cgo_state_set would (CGO_ERR_INVALID for a foreign, older
 * or truncated buffer, or one whose shape does not match the problem and
 * params).  Host buffers; both calls synchronise. */
cgo_status cgo_state_export(const cgo_problem *prob, void *buf, size_t cap, size_t *used);
cgo_status cgo_state_import(cgo_problem *prob, const cgo_params *params, uint64_t seed,
                            const void *buf, size_t len);

/* Operator statistics of the search so far (Sec. 4.2.2 counts the uses of
 * every operator and how many improved, for the AOS update; this call sums
 * them over every generation since the last cgo_solve or cgo_state_set,
 * closed AOS windows and the open one).  out[0..10]: steps that applied
 * operator slot i (cgo_op order, CGO_NOPS_ALL slots); out[11..21]: of those,
 * steps of an improving candidate (delta < 0); out[22..24]: candidates of
 * k = 1, 2, 3 steps; out[25..27]: of those, improving candidates.
 * cap >= 28, else CGO_ERR_INVALID; CGO_ERR_STATE before any solve.  The
 * counts are the ones the AOS update reads, so sum(out[22..24]) =
 * population x candidates x generations. */
cgo_status cgo_op_counts(const cgo_problem *prob, uint64_t *out, int32_t cap);

/* Batched solve: `count` independent problems (different models and sizes
 * allowed) advance together in persistent kernels; problem i uses
 * per_prob[i] and seeds[i].  The paper has no counterpart: it solves one
 * problem per launch; this is the library's batching interface.  Each result is bit-identical to cgo_solve of
 * that problem alone.  All members of a problem share one CTA: its
 * solutions (and, for CVRPTW, route caches) must fit the shared memory of
 * one CTA beside the staged instance data, else CGO_ERR_UNSUPPORTED. */
cgo_status cgo_solve_batch(cgo_problem *const *probs, const cgo_params *per_prob,
                           const uint64_t *seeds, int32_t count, void *cuda_stream);

/* Allocation-free TSP solve, for callers that cannot allocate device memory
 * themselves or through the library (for example code running where
 * cudaMalloc is not allowed, or a host that must keep GPU memory use fixed
 * after start-up).  The paper has no counterpart: it is an interface
 * variant of cgo_solve for TSP.
 *
 * The caller passes the inputs and the outputs; this call allocates nothing
 * (no cudaMalloc, cudaFree or allocating library routine).  Its working
 * memory is one file-scope device array of 8 MiB inside the library, which
 * every GPU that loads the library holds until the process exits.  The
 * problem must fit in it: a request larger than the array (roughly
 * 2n^2 + 8*population*n bytes) returns CGO_ERR_INVALID before any GPU work.
 *
 * desc:          TSP (CGO_ENC_PERM), pointers_on_device = 1, mat0 = the
 *                n*n int32 distance matrix in device memory (symmetric,
 *                else CGO_ERR_UNSUPPORTED); other fields as in
 *                cgo_problem_create.
 * params, seed:  as in cgo_solve; the result equals cgo_solve followed by
 *                cgo_best for the same inputs.
 * out_best_sol:  device buffer of n int32: the elite solution.
 * out_best_cost: device buffer of one int64: its cost.
 * The call synchronises cuda_stream twice (after checking the matrix, and at
 * the end), so its work is complete when it returns.  Argument errors
 * (sizes, generations, parameters) are returned before any GPU work.
 *
 * The first call on a device resolves the array's device address
 * (cudaGetSymbolAddress) with that device current, so make that first call
 * before any stream capture.  Every call shares the same array and leaves
 * its contents behind: calls that overlap on the GPU (other threads or
 * streams) race with each other and must be serialised by the caller. */
cgo_status cgo_solve_static(const cgo_problem_desc *desc, const cgo_params *params, uint64_t seed,
                            int32_t *out_best_sol, int64_t *out_best_cost, void *cuda_stream);

/* ------------------------------------------------------------- serving
 * Continuous batching of solve requests (a request loop on a host thread of
 * the library).  Submitted requests are admitted first come, first served,
 * into device slots as slots and device memory free up; all resident
 * requests advance together by `slice_generations` per time slice in
 * persistent batched kernels replayed from a CUDA graph, and requests that
 * arrive during a slice join at the next slice boundary.  Populations, AOS
 * state and generation counters stay in device memory across slices.  Each
 * result is bit-identical to cgo_solve of the same problem alone.  The paper
 * has no counterpart: this is the library's serving interface. */
typedef struct cgo_server cgo_server;

typedef struct {
  uint32_t struct_size;        /* = sizeof(cgo_server_cfg) */
  int32_t max_slots;           /* requests resident on the device at once, 1 .. 65536 */
  int64_t hbm_budget_bytes;    /* device memory (instance data + search state) of
                                  resident requests; a request waits until it fits
                                  (one request is always admitted when none is resident) */
  int64_t smem_budget_bytes;   /* largest shared-memory footprint of one request (0 = the
                                  CTA limit); larger requests are refused at submit */
  int64_t slice_generations;   /* generations per time slice, >= 1 */
  /* --- appended --- */
  int32_t max_queued;          /* requests waiting for admission at most; cgo_submit
                                  returns CGO_ERR_BUSY beyond it (0 = no bound) */
  int32_t reserved;            /* 0 */
  /* --- appended --- */
  int64_t slice_by_model[5];   /* generations per slice for the requests of each model,
                                  indexed by cgo_model (an asymmetric TSP counts as TSP);
                                  0 = slice_generations.  Every bucket advances in each
                                  slice and the slice lasts as long as its slowest
                                  bucket, so a model whose requests cost little per
                                  generation can take more generations per slice and
                                  finish in fewer slices.  Results do not depend on it. */
} cgo_server_cfg;

/* The size of cgo_server_cfg before max_queued was appended (accepted by
 * cgo_server_create: no queue bound). */
#define CGO_SERVER_CFG_SIZE_V1 ((uint32_t)offsetof(cgo_server_cfg, max_queued))
/* The size before slice_by_model was appended (accepted: every model takes
 * slice_generations). */
#define CGO_SERVER_CFG_SIZE_V2 ((uint32_t)offsetof(cgo_server_cfg, slice_by_model))

typedef struct {
  uint32_t struct_size;        /* = sizeof(cgo_server_info) */
  int32_t queued, active, buckets;
  int64_t slices, completed, hbm_used_bytes;
} cgo_server_info;

/* Start a server on the current device (its thread owns a non-blocking
 * stream).  Errors: CGO_ERR_INVALID, CGO_ERR_NOMEM, CGO_ERR_CUDA. */
cgo_status cgo_server_create(const cgo_server_cfg *cfg, cgo_server **out);

/* Queue a solve of `prob` (created on the server's device) with params and
 * seed; the handle is in use (CGO_ERR_BUSY for other calls) until the
 * request finishes, after which it holds the final state (cgo_best,
 * cgo_state_get).  Validation errors are returned here; a request whose
 * shared-memory footprint exceeds the budget returns CGO_ERR_UNSUPPORTED;
 * CGO_ERR_BUSY when max_queued requests already wait for admission.  A
 * request whose device state cannot be allocated at admission finishes with
 * CGO_ERR_NOMEM (cgo_wait returns it); the server carries on with the rest. */
cgo_status cgo_submit(cgo_server *srv, cgo_problem *prob, const cgo_params *params, uint64_t seed,
                      uint64_t *ticket);

/* Wait for a ticket (timeout_ms < 0: forever).  On CGO_OK fills the elite
 * cost and the latency from submit to completion (seconds) and forgets the
 * ticket; CGO_ERR_TIMEOUT leaves it pending.  Each ticket is waited once.
 * A cancelled request returns CGO_ERR_CANCELLED (and is forgotten). */
cgo_status cgo_wait(cgo_server *srv, uint64_t ticket, int32_t timeout_ms, int64_t *cost,
                    double *latency_s);

/* Cancel a request.  A request still waiting for admission finishes at
 * once; a resident one runs no further slice and finishes at the next slice
 * boundary, freeing its slot and memory.  Its handle keeps no search state
 * (CGO_ERR_STATE from cgo_best) and is free again once the request has
 * finished.  CGO_ERR_INVALID for an unknown ticket, CGO_ERR_STATE if it has
 * already finished.  The serving loop has no counterpart in the paper. */
cgo_status cgo_cancel(cgo_server *srv, uint64_t ticket);

/* Counters of the request loop. */
cgo_status cgo_server_stats(const cgo_server *srv, cgo_server_info *out);

/* Finish every queued and resident request, stop the loop and free the
 * server.  Tickets not yet waited are forgotten.  NULL is accepted. */
cgo_status cgo_server_destroy(cgo_server *srv);

/* Message for the last non-OK status returned on this thread ("" if none). */
const char *cgo_last_error(void);

/* Library version string. */
const char *cgo_version(void);

/* Random-gather rate of this GPU, the denominator of the gather roofline
 * the benchmark reports; it has no counterpart in the method.  kind 0:
 * 16-bit gathers from a shared-memory buffer of 2^log2_elements entries
 * (10 <= log2_elements <= 16), one 1024-thread CTA per SM; kind 1: 32-bit
 * gathers from a global buffer of 2^log2_elements entries (10 .. 28; served
 * by L2 when it fits).  Indices are independent linear-congruential
 * sequences, eight per thread.  Synchronous on the calling thread's device;
 * allocates and frees its own buffers.  gathers_per_s, kernel_ms: host
 * pointers (kernel_ms may be NULL).  CGO_ERR_INVALID for other sizes or
 * kinds, CGO_ERR_CUDA on a CUDA error. */
cgo_status cgo_gather_peak(int32_t kind, int32_t log2_elements, double *gathers_per_s,
                           double *kernel_ms);

/* Number of kernels this library has launched in this process, on any
 * device and from any thread (a replayed graph adds its kernel nodes).  A
 * monotone counter for accounting; it has no counterpart in the method.
 * out: host pointer; CGO_ERR_INVALID if NULL. */
cgo_status cgo_kernel_launches(uint64_t *out);

/* Testing hook (host-side fault injection; never faults the GPU).
 * what = 1: `value` phantom members (0 .. 1024) are added to every member
 *           barrier of the next solves, so no barrier can complete and the
 *           bounded device wait must give up: the solve returns
 *           CGO_ERR_TIMEOUT and the handle's search state is discarded;
 * what = 2: the device wait limit becomes `value` milliseconds (default
 *           10000);
 * what = 3: batched solves advance in time slices of `value` generations
 *           (default 2000; process-wide, prob may be NULL).  Results do not
 *           depend on it;
 * what = 4: the value-th device allocation the library makes from now on
 *           (1 = the next one) fails as out of memory, without allocating;
 *           0 disarms it (process-wide, prob may be NULL).
 * Errors: CGO_ERR_INVALID for an unknown `what` or a value out of range. */
cgo_status cgo_debug_inject(cgo_problem *prob, int32_t what, int64_t value);

#ifdef __cplusplus
}
#endif

#endif /* CGO_H */
