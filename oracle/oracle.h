/*
 * CPU oracle for the per-solution search generation of cuGenOpt
 * (arxiv 2603.19163).  TEST INFRASTRUCTURE ONLY: the test-suite, the smoke
 * check and the benchmark's CPU-baseline leg use it to check and time the
 * CUDA library; the library itself never links, loads or calls it.
 *
 * It is a plain, slow, literal restatement of
 *   - Alg. "evolve" (Sec. 3.2.3): per-candidate K-step move sampling, delta
 *     f(s') - f(s), block argmin, Metropolis acceptance, cooling;
 *   - Alg. "aos" and Eq. "ema" (Sec. 4.2.2): two-level AOS statistics, EMA
 *     weight update, clamping, normalisation, stagnation reset (Sec. 4.2.3);
 *   - elite tracking and elite injection (Sec. 3.4.3);
 *   - the three encodings (Sec. 3.1.1) and the element/segment operators of
 *     Table "operators" (swap, reverse, insert, or-opt, flip, random reset);
 * with the fixed-point readings listed in the design notes (counter-based
 * Philox4x32-10 random stream, Q32.32 temperature, Q16 weights, integer
 * logarithm for the acceptance test).  Candidate deltas are computed by the
 * definition: the candidate is built on a literal copy of the solution and
 * both costs are evaluated in full.
 *
 * It shares no code, header or table with the CUDA library.
 */
#ifndef CGO_ORACLE_H
#define CGO_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_TSP = 0, ORC_QAP = 1, ORC_KNAPSACK = 2, ORC_GAP = 3, ORC_CVRPTW = 4 };
enum { ORC_SWAP = 0, ORC_TWO_OPT = 1, ORC_INSERT = 2, ORC_OR_OPT = 3,
       ORC_FLIP = 4, ORC_PERTURB = 5, ORC_THREE_OPT = 6,
       ORC_SEGMENT = 7, /* binary: seg_flip; integer: seg_reset [R28] */
       /* row level of CVRPTW's separator encoding [R31, R32] */
       ORC_ROW_SWAP = 8, ORC_ROW_MERGE = 9, ORC_ROW_SPLIT = 10,
       ORC_NOPS = 11 };
/* counts per member per generation: u_op, v_op (ORC_NOPS each), u_k, v_k */
enum { ORC_NSTATS = 2 * ORC_NOPS + 6 };

typedef struct {
  int32_t model;      /* ORC_TSP ... ORC_CVRPTW */
  int32_t n;          /* cities / facilities / items / jobs / customers */
  int32_t m;          /* GAP: agents */
  int32_t vehicles;   /* CVRPTW: V */
  const int32_t *mat0, *mat1;
  const int32_t *vec0, *vec1, *vec2, *vec3;
  int64_t capacity;   /* knapsack capacity, CVRPTW vehicle capacity Q */
  int32_t lb, ub;     /* integer-encoding bounds (GAP: 0 .. m-1) */
  int64_t penalty0, penalty1; /* 0 = default lambda */
  uint32_t tag;       /* instance tag (Philox counter word 1) */
  int64_t weight0, weight1; /* CVRPTW objective weights: distance (0 = 1), vehicles used */
  int64_t weight2;          /* CVRPTW: weight of the longest route's distance [R34] (0 = off) */
  /* CVRPTW lexicographic mode [R37] (Sec. 6.8, Table "lexicographic_mode"):
   * lex_n objectives in priority order (0 distance, 1 vehicles used, 2 the
   * longest route's distance), each with an integer tolerance; lex_n = 0
   * keeps the weighted cost.  lex_dmax = (n + vehicles) * the largest travel
   * time, the bound on the distances that sets the key's radices. */
  int32_t lex_n;
  int32_t lex_obj[3];
  int64_t lex_tol[3];
  int64_t lex_dmax;
} orc_instance;

typedef struct {
  int32_t P, C;
  uint32_t op_mask;
  uint32_t w_op[ORC_NOPS], w_k[3];
  uint64_t T0, alpha;              /* Q32.32, Q0.32 */
  uint32_t U, ema_a, w_floor, w_cap, op_cap[ORC_NOPS], stag_limit, elite_period;
  uint32_t init_oversample;        /* K of the oversampled start (Sec. 3.4.1); 0 or 1 = off */
  uint32_t init_heuristic;         /* 1 = add the row/column-sum permutations (Sec. 3.4.2) */
  uint32_t islands;                /* islands (Sec. 3.4.3); 0 or 1 = one population */
  uint32_t migrate_period;         /* migration after every such generation; 0 = off */
  uint32_t migrate_strategy;       /* 0 ring, 1 global top-N, 2 hybrid (alternating) */
  uint32_t migrate_n;              /* N of the top-N strategy */
  uint32_t cross_q16;              /* crossover probability per member and AOS window
                                      (Table "operators", crossover level); 0 = off */
} orc_params;

/* Complete search state.  Arrays are caller-owned: cur/best_sol P*len,
 * cost/best_cost P. */
typedef struct {
  int32_t P, len;
  int64_t g;                        /* generations completed */
  uint64_t T;                       /* current temperature, Q32.32 */
  uint32_t w_op[ORC_NOPS], w_k[3];  /* current AOS weights, Q16 */
  uint32_t stag;                    /* updates without elite improvement */
  int64_t elite_prev;               /* elite cost at the last AOS update */
  uint32_t u_op[ORC_NOPS], v_op[ORC_NOPS], u_k[3], v_k[3]; /* open window */
  int32_t *cur, *best_sol;
  int64_t *cost, *best_cost;
  /* the same counts summed over every generation since init (statistics for
   * the caller; the search never reads them) */
  uint64_t all_u_op[ORC_NOPS], all_v_op[ORC_NOPS], all_u_k[3], all_v_k[3];
} orc_state;

/* building blocks, exported for the oracle's own pin tests */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
uint32_t orc_pos(uint32_t h16, uint32_t m);
int32_t orc_wsample(const uint32_t *w, int32_t count, uint32_t word);
uint64_t orc_log2_q32(uint32_t A);
uint64_t orc_exp_q32(uint32_t A);
int32_t orc_accept(int64_t delta, uint64_t T, uint32_t A);
uint64_t orc_cool(uint64_t T, uint64_t alpha);
int32_t orc_apply_move(const orc_instance *in, int32_t op, uint32_t a, uint32_t b,
                       uint32_t x, int32_t *sol, int32_t len);
void orc_aos_level(uint32_t *w, const uint32_t *u, const uint32_t *v, const int32_t *enabled,
                   const uint32_t *cap_i, int32_t count, uint32_t a, uint32_t w_floor,
                   uint32_t w_cap);

/* defaults: the L1 profile priors (Table "weight_preset") and the readings of
 * the unstated AOS/annealing constants */
void orc_params_default(const orc_instance *in, orc_params *pr);
int32_t orc_solution_length(const orc_instance *in);
int64_t orc_cost(const orc_instance *in, const int32_t *sol);
int32_t orc_valid(const orc_instance *in, const int32_t *sol);
int32_t orc_enabled_ops(const orc_instance *in, uint32_t op_mask, int32_t enabled[ORC_NOPS]);

/* population init (seeded Philox) + exact costs; state arrays must be sized */
int32_t orc_init(const orc_instance *in, const orc_params *pr, uint64_t seed, orc_state *st);
/* run `generations` more generations from the state (threads <= 0: all cores) */
int32_t orc_run(const orc_instance *in, const orc_params *pr, uint64_t seed, orc_state *st,
                int64_t generations, int32_t threads);
/* index of the instance elite (lowest best cost, ties to the lowest index) */
int32_t orc_elite(const orc_state *st);
/* one migration between islands on the state as it stands (the step the
 * search takes after every migrate_period-th generation); exported for the
 * oracle's own pins.  Returns -1 for invalid island parameters. */
int32_t orc_migrate(const orc_params *pr, orc_state *st);
/* Row operators [R31] of CVRPTW's separator encoding (rows = routes; Table
 * "operators", row level): kind 0 row_swap, 1 row_merge, 2 row_split, drawn
 * from the 16-bit fields a, b; edits s in place (an identity when the row
 * operator has nothing to do).  The search applies them as operator slots
 * ORC_ROW_SWAP .. ORC_ROW_SPLIT [R32].  Returns -1 for other models, -2 unless
 * len = n + V - 1 with exactly V - 1 separators, -3 when memory runs out. */
int32_t orc_row_move(const orc_instance *in, int32_t kind, uint32_t a, uint32_t b, int32_t *s,
                     int32_t len);
/* order crossover [R29]: child keeps A[lo..hi] in place and fills positions
 * hi+1, ..., len-1, 0, ..., lo-1 with the elements of B outside that segment,
 * in B's order from B[hi+1] on (wrapping); 0 <= lo <= hi < len */
void orc_ox(const int32_t *A, const int32_t *B, int32_t len, int32_t lo, int32_t hi,
            int32_t *child);
/* One crossover step of the whole population at the state's generation
 * (normally run by orc_run at each AOS window end); 0 or -1. */
int32_t orc_crossover(const orc_instance *in, const orc_params *pr, uint64_t seed,
                      orc_state *st);
/* the attribute-agnostic start permutations of an instance (TSP: D; QAP: F,
 * then D): per matrix the orders of ascending and descending row sums, then
 * ascending and descending column sums.  out: 8 * n entries; returns their
 * number of permutations (0 for other models). */
int32_t orc_heuristic_perms(const orc_instance *in, int32_t *out);
/* OpenMP threads the oracle would use for `threads` */
int32_t orc_threads(int32_t threads);

#ifdef __cplusplus
}
#endif
#endif
