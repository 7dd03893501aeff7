/*
 * CPU oracle for cuGenOpt's per-solution search generation (arxiv 2603.19163).
 *
 * TEST INFRASTRUCTURE: only the tests, the smoke check and the benchmark's
 * CPU-baseline leg load this file's library.  The CUDA library never does.
 *
 * Plain, slow and literal by design: every candidate is built on a copy of
 * the current solution and its cost is evaluated in full.  Function headers
 * name the passage of the paper each one restates; the fixed-point readings
 * (marked [R#]) are the ones this project pins where the paper is silent.
 */
#include "oracle.h"

#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;

/* ------------------------------------------------------------------ RNG [R1]
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplications with
 * the Weyl key schedule.  The paper names no generator (it fixes seeds only,
 * Sec. 6.1); a counter-based one keyed by (instance, solution, generation)
 * makes the trajectory independent of thread scheduling. */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; r++) {
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
    uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
    uint32_t y1 = (uint32_t)p1;
    uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
    uint32_t y3 = (uint32_t)p0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* counter = (w0, tag, p, g), key = (lo32(seed), hi32(seed)) [R1] */
static void draw(uint32_t w0, uint32_t tag, uint32_t p, uint32_t g, uint64_t seed,
                 uint32_t out[4]) {
  uint32_t ctr[4] = {w0, tag, p, g};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  orc_philox(ctr, key, out);
}

#define KIND_MOVE 0u
#define KIND_ACCEPT 1u
#define KIND_INIT 2u
#define KIND_CROSS 3u
#define W0(cand, step, kind) ((uint32_t)(cand) | ((uint32_t)(step) << 20) | ((uint32_t)(kind) << 24))
#define INIT_GEN 0xFFFFFFFFu

/* -------------------------------------------------------- index mapping [R2] */
/* pos(h16, m) = floor(h16 * m / 2^16): a 16-bit field scaled to [0, m). */
uint32_t orc_pos(uint32_t h16, uint32_t m) { return (uint32_t)(((uint64_t)h16 * m) >> 16); }

/* Roulette-wheel choice from weights (Sec. 4.2.1, "sample from w"):
 * r = floor(word * sum(w) / 2^32); first i with r < w_0 + ... + w_i. */
int32_t orc_wsample(const uint32_t *w, int32_t count, uint32_t word) {
  uint64_t W = 0;
  for (int32_t i = 0; i < count; i++) W += w[i];
  uint64_t r = ((uint64_t)word * W) >> 32;
  uint64_t acc = 0;
  for (int32_t i = 0; i < count; i++) {
    acc += w[i];
    if (r < acc) return i;
  }
  return -1; /* all weights zero */
}

/* ------------------------------------------------- acceptance test [R7]
 * Alg. "evolve" accepts the best candidate when delta < 0 or
 * rand() < exp(-delta / T).  Restated in integers: with u = (A+1)/2^32,
 * rand() < exp(-delta/T)  <=>  delta < T * (-ln u).  -log2(u) is computed in
 * Q32 by the bit-by-bit squaring method (C. S. Turner, "A Fast Binary
 * Logarithm Algorithm", IEEE Signal Processing Magazine, 2010), then scaled
 * by ln 2 in Q32. */
uint64_t orc_log2_q32(uint32_t A) {
  /* returns -log2((A+1)/2^32) in Q32 */
  uint64_t y = (uint64_t)A + 1;        /* 1 .. 2^32 */
  int e = 0;
  while ((y >> (e + 1)) != 0) e++;     /* e = floor(log2 y) */
  uint64_t z = y << (62 - e);          /* y / 2^e in Q2.62, in [1, 2) */
  uint32_t frac = 0;
  for (int i = 1; i <= 32; i++) {
    z = (uint64_t)(((u128)z * z) >> 62);
    if (z >= (1ull << 63)) {
      z >>= 1;
      frac |= 1u << (32 - i);
    }
  }
  uint64_t log2y = ((uint64_t)e << 32) + frac;   /* log2(y) in Q32 (truncated) */
  return (32ull << 32) - log2y;                  /* 32 - log2(y) = -log2(u) */
}

#define LN2_Q32 2977044472ull /* round(ln 2 * 2^32) */

uint64_t orc_exp_q32(uint32_t A) {
  return (uint64_t)(((u128)orc_log2_q32(A) * LN2_Q32) >> 32); /* -ln(u), Q32 */
}

int32_t orc_accept(int64_t delta, uint64_t T, uint32_t A) {
  if (delta <= 0) return 1;
  u128 lhs = (u128)(uint64_t)delta << 64;       /* delta, Q64 */
  u128 rhs = (u128)T * (u128)orc_exp_q32(A);    /* T (Q32) * E (Q32) */
  return lhs < rhs;
}

/* geometric cooling T <- alpha * T (Alg. "evolve", last line) [R8] */
uint64_t orc_cool(uint64_t T, uint64_t alpha) { return (uint64_t)(((u128)T * alpha) >> 32); }

/* --------------------------------------------------------- instances [R16] */
int32_t orc_solution_length(const orc_instance *in) {
  if (in->model == ORC_CVRPTW) return in->n + in->vehicles - 1; /* separators */
  return in->n;
}

static int32_t encoding_of(int32_t model) {
  if (model == ORC_KNAPSACK) return 1;   /* binary (Sec. 3.1.1) */
  if (model == ORC_GAP) return 2;        /* integer */
  return 0;                              /* permutation */
}

static void int_bounds(const orc_instance *in, int32_t *lb, int32_t *ub) {
  if (in->model == ORC_GAP) { *lb = 0; *ub = in->m - 1; return; }
  *lb = in->lb; *ub = in->ub;
}

static int64_t over(int64_t x) { return x > 0 ? x : 0; }

/* TSP: sum of D[a_k][a_(k+1) mod n] (Listing "tsp", in integers) */
static int64_t cost_tsp(const orc_instance *in, const int32_t *x) {
  int32_t n = in->n;
  int64_t s = 0;
  for (int32_t k = 0; k < n; k++) s += in->mat0[(int64_t)x[k] * n + x[(k + 1) % n]];
  return s;
}

/* QAP (Koopmans-Beckmann): sum_i sum_j F[i][j] * D[a_i][a_j] */
static int64_t cost_qap(const orc_instance *in, const int32_t *x) {
  int32_t n = in->n;
  int64_t s = 0;
  for (int32_t i = 0; i < n; i++)
    for (int32_t j = 0; j < n; j++)
      s += (int64_t)in->mat0[(int64_t)i * n + j] * in->mat1[(int64_t)x[i] * n + x[j]];
  return s;
}

/* knapsack as minimisation: -sum v x + lambda * max(0, sum w x - cap),
 * lambda = 1 + max v unless given (objective + penalty, Sec. 3.1.3) */
static int64_t cost_knapsack(const orc_instance *in, const int32_t *x) {
  int64_t W = 0, V = 0, vmax = 0;
  for (int32_t i = 0; i < in->n; i++) {
    if (in->vec1[i] > vmax) vmax = in->vec1[i];
    if (x[i]) { W += in->vec0[i]; V += in->vec1[i]; }
  }
  int64_t lam = in->penalty0 > 0 ? in->penalty0 : 1 + vmax;
  return -V + lam * over(W - in->capacity);
}

/* GAP: sum_j c[x_j][j] + lambda * sum_a max(0, load_a - cap_a) */
static int64_t cost_gap(const orc_instance *in, const int32_t *x) {
  int32_t n = in->n, m = in->m;
  int64_t cmax = 0;
  for (int64_t i = 0; i < (int64_t)m * n; i++)
    if (in->mat0[i] > cmax) cmax = in->mat0[i];
  int64_t lam = in->penalty0 > 0 ? in->penalty0 : 1 + cmax;
  int64_t s = 0;
  for (int32_t j = 0; j < n; j++) s += in->mat0[(int64_t)x[j] * n + j];
  for (int32_t a = 0; a < m; a++) {
    int64_t load = 0;
    for (int32_t j = 0; j < n; j++)
      if (x[j] == a) load += in->mat1[(int64_t)a * n + j];
    s += lam * over(load - in->vec0[a]);
  }
  return s;
}

/* [R37] CVRPTW's lexicographic key (Sec. 6.8, Table "lexicographic_mode"):
 * the penalty first, then the prioritised objectives in order, objective i
 * in buckets of width tol_i + 1 (values in one bucket tie and the next
 * objective decides), as one integer in mixed radix:
 *   key = (((pen * R_1 + q_1) * R_2 + q_2) ...),  q_i = o_i / (tol_i + 1),
 *   R_i = omax_i / (tol_i + 1) + 1,
 * omax = lex_dmax for the two distances and the fleet size for vehicles. */
static int64_t lex_key(const orc_instance *in, int64_t pen, int64_t dist, int64_t used,
                       int64_t longest) {
  int64_t key = pen;
  for (int32_t i = 0; i < in->lex_n; i++) {
    int32_t obj = in->lex_obj[i];
    int64_t o = obj == 0 ? dist : (obj == 1 ? used : longest);
    int64_t omax = obj == 1 ? (int64_t)in->vehicles : in->lex_dmax;
    int64_t w = in->lex_tol[i] + 1;
    key = key * (omax / w + 1) + o / w;
  }
  return key;
}

/* CVRPTW, separator encoding: symbols < n are customers 1..n, symbols >= n
 * end a route.  Per route from the depot at t = 0: arrive t = max(t + d,
 * ready); late += max(0, t - due); t += service; load += demand; back at the
 * depot t += d(last, 0), late += max(0, t - due_0).  A route with no customer
 * costs nothing.
 * cost = distance + lambda_cap * sum max(0, load - Q) + lambda_tw * late,
 * with the objective weights of [R30] and [R34] (longest route), or the
 * lexicographic key of [R37]. */
static int64_t cost_cvrptw(const orc_instance *in, const int32_t *x) {
  int32_t n = in->n, len = orc_solution_length(in), N = n + 1;
  const int32_t *d = in->mat0, *dem = in->vec0, *rdy = in->vec1, *due = in->vec2,
                *svc = in->vec3;
  int64_t lcap = in->penalty0 > 0 ? in->penalty0 : 100;
  int64_t ltw = in->penalty1 > 0 ? in->penalty1 : 100;
  /* [R30] weighted objectives (Sec. 6.8): distance and vehicles used */
  int64_t wd = in->weight0 > 0 ? in->weight0 : 1, wv = in->weight1;
  /* [R34] the third objective of Sec. 6.8's tri-objective VRP: the longest
   * route, as the largest distance driven by one vehicle */
  int64_t wl = in->weight2, longest = 0;
  int64_t dist = 0, capx = 0, late = 0, used = 0;
  int32_t k = 0;
  while (k <= len) {
    /* one route: symbols until a separator or the end */
    int64_t t = 0, load = 0, rd = 0;
    int32_t prev = 0;
    while (k < len && x[k] < n) {
      int32_t c = x[k] + 1;
      int64_t dd = d[(int64_t)prev * N + c];
      dist += dd;
      rd += dd;
      t = t + dd > rdy[c] ? t + dd : rdy[c];
      late += over(t - due[c]);
      t += svc[c];
      load += dem[c];
      prev = c;
      k++;
    }
    if (prev != 0) { /* a route that visits no customer costs nothing */
      int64_t back = d[(int64_t)prev * N + 0];
      dist += back;
      rd += back;
      if (rd > longest) longest = rd;
      t += back;
      late += over(t - due[0]);
      capx += over(load - in->capacity);
      used++;
    }
    k++; /* skip the separator (or step past the end) */
  }
  if (in->lex_n > 0) return lex_key(in, lcap * capx + ltw * late, dist, used, longest);
  return wd * dist + lcap * capx + ltw * late + wv * used + wl * longest;
}

int64_t orc_cost(const orc_instance *in, const int32_t *sol) {
  switch (in->model) {
    case ORC_TSP: return cost_tsp(in, sol);
    case ORC_QAP: return cost_qap(in, sol);
    case ORC_KNAPSACK: return cost_knapsack(in, sol);
    case ORC_GAP: return cost_gap(in, sol);
    case ORC_CVRPTW: return cost_cvrptw(in, sol);
  }
  return 0;
}

int32_t orc_valid(const orc_instance *in, const int32_t *sol) {
  int32_t len = orc_solution_length(in), enc = encoding_of(in->model);
  if (enc == 0) {
    char *seen = (char *)calloc((size_t)len, 1);
    int ok = 1;
    for (int32_t i = 0; i < len && ok; i++) {
      if (sol[i] < 0 || sol[i] >= len || seen[sol[i]]) ok = 0;
      else seen[sol[i]] = 1;
    }
    free(seen);
    return ok;
  }
  int32_t lb = 0, ub = 1;
  if (enc == 2) int_bounds(in, &lb, &ub);
  for (int32_t i = 0; i < len; i++)
    if (sol[i] < lb || sol[i] > ub) return 0;
  return 1;
}

/* Operators per encoding (Table "operators"): permutation -> swap, reverse
 * (2-opt), insert, or-opt, 3-opt; binary -> flip, seg_flip; integer ->
 * random reset, seg_reset; the row level (row_swap, row_merge, row_split)
 * applies to CVRPTW, whose rows are its V >= 2 routes [R32]. */
int32_t orc_enabled_ops(const orc_instance *in, uint32_t op_mask, int32_t enabled[ORC_NOPS]) {
  int32_t enc = encoding_of(in->model), len = orc_solution_length(in), count = 0;
  for (int32_t i = 0; i < ORC_NOPS; i++) {
    int32_t ok = 0;
    if (enc == 0 && i <= ORC_OR_OPT) ok = (i == ORC_OR_OPT) ? (len >= 4) : 1; /* [R3] */
    if (enc == 0 && i == ORC_THREE_OPT) ok = 1;                                /* [R26] */
    if (enc == 1 && i == ORC_FLIP) ok = 1;
    if (enc == 2 && i == ORC_PERTURB) ok = 1;
    if (enc != 0 && i == ORC_SEGMENT) ok = (len >= 2);                         /* [R28] */
    if (i >= ORC_ROW_SWAP) ok = in->model == ORC_CVRPTW && in->vehicles >= 2;  /* [R32] */
    enabled[i] = ok && ((op_mask >> i) & 1u);
    count += enabled[i];
  }
  return count;
}

/* ------------------------------------------------------------- moves [R3,R4]
 * Each operator reads two 16-bit position fields (a, b) and one extra word x
 * and edits the array in place (a literal copy of the current solution). */
static void pick_ij(uint32_t a, uint32_t b, int32_t len, int32_t *i, int32_t *j) {
  *i = (int32_t)orc_pos(a, (uint32_t)len);
  *j = (int32_t)orc_pos(b, (uint32_t)(len - 1));
  if (*j >= *i) (*j)++; /* j != i */
}

int32_t orc_apply_move(const orc_instance *in, int32_t op, uint32_t a, uint32_t b, uint32_t x,
                       int32_t *s, int32_t len) {
  int32_t i, j;
  if (op >= ORC_ROW_SWAP && op <= ORC_ROW_SPLIT)   /* [R32] the row level */
    return orc_row_move(in, op - ORC_ROW_SWAP, a, b, s, len) == 0 ? 0 : -1;
  switch (op) {
    case ORC_SWAP: { /* exchange two elements */
      pick_ij(a, b, len, &i, &j);
      int32_t t = s[i]; s[i] = s[j]; s[j] = t;
      return 0;
    }
    case ORC_TWO_OPT: { /* reverse the segment between them (inclusive) */
      pick_ij(a, b, len, &i, &j);
      int32_t lo = i < j ? i : j, hi = i < j ? j : i;
      while (lo < hi) { int32_t t = s[lo]; s[lo] = s[hi]; s[hi] = t; lo++; hi--; }
      return 0;
    }
    case ORC_INSERT: { /* remove s[i]; re-insert it so that it ends at index j */
      pick_ij(a, b, len, &i, &j);
      int32_t v = s[i];
      for (int32_t k = i; k < len - 1; k++) s[k] = s[k + 1];   /* remove */
      for (int32_t k = len - 1; k > j; k--) s[k] = s[k - 1];   /* open slot j */
      s[j] = v;
      return 0;
    }
    case ORC_OR_OPT: { /* move a block of L = 2 + (x & 1) elements */
      if (len < 4) return -1;
      int32_t L = 2 + (int32_t)(x & 1u);
      i = (int32_t)orc_pos(a, (uint32_t)(len - L + 1));          /* block start */
      int32_t q = (int32_t)orc_pos(b, (uint32_t)(len - L));       /* slot in rest */
      if (q >= i) q++;                                           /* not back in place */
      int32_t blk[3], *rest = (int32_t *)malloc(sizeof(int32_t) * (size_t)len);
      for (int32_t k = 0; k < L; k++) blk[k] = s[i + k];
      int32_t r = 0;
      for (int32_t k = 0; k < len; k++)
        if (k < i || k >= i + L) rest[r++] = s[k];
      int32_t o = 0;
      for (int32_t k = 0; k < q; k++) s[o++] = rest[k];           /* rest before q */
      for (int32_t k = 0; k < L; k++) s[o++] = blk[k];            /* the block */
      for (int32_t k = q; k < len - L; k++) s[o++] = rest[k];     /* rest from q */
      free(rest);
      return 0;
    }
    case ORC_THREE_OPT: { /* [R26] exchange the adjacent segments [i,j) and [j,k) */
      /* three distinct cut points of 0..len: from len+1, len and len-1 values,
       * each later draw skipping the points already taken */
      int32_t c1 = (int32_t)orc_pos(a, (uint32_t)(len + 1));
      int32_t c2 = (int32_t)orc_pos(b, (uint32_t)len);
      if (c2 >= c1) c2++;
      int32_t lo = c1 < c2 ? c1 : c2, hi = c1 < c2 ? c2 : c1;
      int32_t c3 = (int32_t)orc_pos(x >> 16, (uint32_t)(len - 1));
      if (c3 >= lo) c3++;
      if (c3 >= hi) c3++;
      int32_t ci = lo < c3 ? lo : c3;
      int32_t ck = hi > c3 ? hi : c3;
      int32_t cj = c1 + c2 + c3 - ci - ck;
      int32_t *t = (int32_t *)malloc(sizeof(int32_t) * (size_t)len);
      int32_t o = 0;
      for (int32_t q = 0; q < ci; q++) t[o++] = s[q];
      for (int32_t q = cj; q < ck; q++) t[o++] = s[q];
      for (int32_t q = ci; q < cj; q++) t[o++] = s[q];
      for (int32_t q = ck; q < len; q++) t[o++] = s[q];
      memcpy(s, t, sizeof(int32_t) * (size_t)len);
      free(t);
      return 0;
    }
    case ORC_FLIP: { /* x_i ^= 1 */
      i = (int32_t)orc_pos(a, (uint32_t)len);
      s[i] ^= 1;
      return 0;
    }
    case ORC_PERTURB: { /* random reset to a different value in [lb, ub] */
      int32_t lb, ub;
      int_bounds(in, &lb, &ub);
      int64_t R = (int64_t)ub - lb + 1;
      i = (int32_t)orc_pos(a, (uint32_t)len);
      int64_t d = 1 + (int64_t)orc_pos(b, (uint32_t)(R - 1));
      s[i] = (int32_t)(lb + (((int64_t)s[i] - lb + d) % R));
      return 0;
    }
    case ORC_SEGMENT: { /* [R28] a segment of L = 2 + (x & 1) elements (at most len) */
      if (len < 2) return -1;
      int32_t L = 2 + (int32_t)(x & 1u);
      if (L > len) L = len;
      i = (int32_t)orc_pos(a, (uint32_t)(len - L + 1));          /* segment start */
      if (encoding_of(in->model) == 1) {                          /* seg_flip */
        for (int32_t q = i; q < i + L; q++) s[q] ^= 1;
      } else {                                                    /* seg_reset */
        int32_t lb, ub;
        int_bounds(in, &lb, &ub);
        int64_t R = (int64_t)ub - lb + 1;
        int64_t d = 1 + (int64_t)orc_pos(b, (uint32_t)(R - 1));  /* one offset for all */
        for (int32_t q = i; q < i + L; q++) s[q] = (int32_t)(lb + (((int64_t)s[q] - lb + d) % R));
      }
      return 0;
    }
  }
  return -1;
}

/* ----------------------------------------------------------- AOS [R9-R12]
 * Eq. "ema": w <- a*w + (1-a)*(v/(u+eps) + w_floor), clamped to
 * [w_floor, min(w_cap, cap_i)] and normalised (Sec. 4.2.2), all in Q16 with
 * eps = 1 (ratio = v*2^16 / (u+1)) and floor division. */
void orc_aos_level(uint32_t *w, const uint32_t *u, const uint32_t *v, const int32_t *enabled,
                   const uint32_t *cap_i, int32_t count, uint32_t a, uint32_t w_floor,
                   uint32_t w_cap) {
  uint64_t S = 0;
  for (int32_t i = 0; i < count; i++) {
    if (!enabled[i]) continue;
    uint64_t ratio = ((uint64_t)v[i] << 16) / ((uint64_t)u[i] + 1);
    uint64_t nw = ((uint64_t)a * w[i] + (uint64_t)(65536u - a) * (ratio + w_floor)) >> 16;
    uint64_t hi = w_cap < cap_i[i] ? w_cap : cap_i[i];
    if (nw > hi) nw = hi;
    if (nw < w_floor) nw = w_floor;
    w[i] = (uint32_t)nw;
    S += nw;
  }
  for (int32_t i = 0; i < count; i++)
    if (enabled[i]) w[i] = (uint32_t)(((uint64_t)w[i] << 16) / S);
}

/* K-step weights after a stagnation reset (Sec. 4.2.3): (0.8, 0.15, 0.05) */
static const uint32_t K_RESET[3] = {52429u, 9830u, 3277u};

/* Defaults [R11, R14].  L1 priors (Sec. 4.1, Table "weight_preset"): O(1)
 * operators start at 1.0; or-opt at 0.80 / 0.70 / 0.30 for solution length
 * <= 100 / <= 250 / > 250; normalised to Q16 by floor division.  K-step
 * weights (0.8, 0.15, 0.05) (Sec. 4.2.3).  T0 = 100, alpha = 0.999,
 * I = 10, EMA a = 0.8, floor 0.05, cap 0.6, stagnation after 5 updates,
 * elite injection off. */
void orc_params_default(const orc_instance *in, orc_params *pr) {
  int32_t en[ORC_NOPS], len = orc_solution_length(in);
  memset(pr, 0, sizeof *pr);
  pr->P = 32;
  pr->C = 128;
  pr->op_mask = 0x3Fu;
  /* priors of every applicable operator (Table "weight_preset"); the
   * normaliser is taken over the default mask (3-opt, the segment and the
   * row operators off by default).  The row operators take the O(1) prior
   * 1.0: the table scales only the listed high-complexity operators [R32]. */
  int32_t app[ORC_NOPS];
  orc_enabled_ops(in, pr->op_mask, en);
  orc_enabled_ops(in, (1u << ORC_NOPS) - 1u, app);
  uint64_t S = 0;
  for (int32_t i = 0; i < ORC_NOPS; i++) {
    uint32_t w = 0;
    if (app[i]) {
      w = 65536u;
      if (i == ORC_OR_OPT) w = len <= 100 ? 52429u : (len <= 250 ? 45875u : 19661u);
      if (i == ORC_THREE_OPT) w = len <= 100 ? 32768u : (len <= 250 ? 19661u : 3277u);
      /* [R28] segment-level operators of the binary and integer sets take
       * the segment-level (or-opt) preset */
      if (i == ORC_SEGMENT) w = len <= 100 ? 52429u : (len <= 250 ? 45875u : 19661u);
    }
    pr->w_op[i] = w;
    if (en[i]) S += w;
    pr->op_cap[i] = 65536u;
  }
  for (int32_t i = 0; i < ORC_NOPS; i++) pr->w_op[i] = (uint32_t)(((uint64_t)pr->w_op[i] << 16) / S);
  pr->w_k[0] = 52429u; pr->w_k[1] = 9830u; pr->w_k[2] = 3277u;
  pr->T0 = 100ull << 32;
  pr->alpha = 4290672329ull;
  pr->U = 10;
  pr->ema_a = 52429u;
  pr->w_floor = 3277u;
  pr->w_cap = 39322u;
  pr->stag_limit = 5;
  pr->elite_period = 0;
  pr->init_oversample = 1;
  pr->init_heuristic = 0;
  pr->islands = 1;
  pr->migrate_period = 0;
  pr->migrate_strategy = 0;
  pr->migrate_n = 1;
}

/* ------------------------------------------------------------- init [R15] */
/* Random start j (member j of a plain start, candidate j of an oversampled
 * one): Fisher-Yates for permutations, one draw per entry otherwise. */
static void random_start(const orc_instance *in, uint32_t j, uint64_t seed, int32_t enc,
                         int32_t lb, int32_t ub, int32_t *x, int32_t len) {
  uint32_t R[4];
  if (enc == 0) { /* Fisher-Yates, i = len-1 .. 1, j = floor(word*(i+1)/2^32) */
    for (int32_t i = 0; i < len; i++) x[i] = i;
    for (int32_t i = len - 1; i >= 1; i--) {
      int32_t d = len - 1 - i;
      draw(W0(d / 4, 0, KIND_INIT), in->tag, j, INIT_GEN, seed, R);
      int32_t r = (int32_t)(((uint64_t)R[d % 4] * (uint64_t)(i + 1)) >> 32);
      int32_t t = x[i]; x[i] = x[r]; x[r] = t;
    }
  } else {
    for (int32_t i = 0; i < len; i++) {
      draw(W0(i / 4, 0, KIND_INIT), in->tag, j, INIT_GEN, seed, R);
      uint32_t w = R[i % 4];
      if (enc == 1) x[i] = (int32_t)(w & 1u);
      else x[i] = lb + (int32_t)(((uint64_t)w * (uint64_t)((int64_t)ub - lb + 1)) >> 32);
    }
  }
}

/* sort keys: (key, index) ascending */
typedef struct { int64_t key; int64_t idx; } orc_keyed;
static int keyed_less(const void *a, const void *b) {
  const orc_keyed *x = (const orc_keyed *)a, *y = (const orc_keyed *)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  return x->idx < y->idx ? -1 : (x->idx > y->idx ? 1 : 0);
}

/* Sec. 3.4.2: per n x n data matrix, sort the elements by row sum and by
 * column sum, ascending and descending (ties: lower index first). */
int32_t orc_heuristic_perms(const orc_instance *in, int32_t *out) {
  const int32_t n = in->n;
  const int32_t *mats[2] = {in->mat0, in->mat1};
  int32_t nm = in->model == ORC_TSP ? 1 : (in->model == ORC_QAP ? 2 : 0), H = 0;
  orc_keyed *k = (orc_keyed *)malloc(sizeof(orc_keyed) * (size_t)n);
  for (int32_t t = 0; t < nm; t++) {
    const int32_t *M = mats[t];
    for (int32_t by_col = 0; by_col < 2; by_col++) {
      for (int32_t desc = 0; desc < 2; desc++) {
        for (int32_t i = 0; i < n; i++) {
          int64_t s = 0;
          for (int32_t j = 0; j < n; j++) s += by_col ? M[(int64_t)j * n + i] : M[(int64_t)i * n + j];
          k[i].key = desc ? -s : s;
          k[i].idx = i;
        }
        qsort(k, (size_t)n, sizeof(orc_keyed), keyed_less);
        for (int32_t i = 0; i < n; i++) out[(int64_t)H * n + i] = (int32_t)k[i].idx;
        H++;
      }
    }
  }
  free(k);
  return H;
}

int32_t orc_init(const orc_instance *in, const orc_params *pr, uint64_t seed, orc_state *st) {
  int32_t len = orc_solution_length(in), enc = encoding_of(in->model);
  int32_t en[ORC_NOPS];
  if (pr->P < 1 || len < 2) return -1;
  orc_enabled_ops(in, pr->op_mask, en);
  st->P = pr->P;
  st->len = len;
  st->g = 0;
  st->T = pr->T0;
  for (int32_t i = 0; i < ORC_NOPS; i++) {
    st->w_op[i] = en[i] ? pr->w_op[i] : 0u;
    st->u_op[i] = st->v_op[i] = 0;
  }
  for (int32_t i = 0; i < 3; i++) { st->w_k[i] = pr->w_k[i]; st->u_k[i] = st->v_k[i] = 0; }
  for (int32_t i = 0; i < ORC_NOPS; i++) st->all_u_op[i] = st->all_v_op[i] = 0;
  for (int32_t i = 0; i < 3; i++) st->all_u_k[i] = st->all_v_k[i] = 0;
  st->stag = 0;
  int32_t lb = 0, ub = 1;
  if (enc == 2) int_bounds(in, &lb, &ub);
  const int64_t K = pr->init_oversample > 1 ? pr->init_oversample : 1;
  int32_t *heur = NULL, H = 0;
  if (pr->init_heuristic) {
    heur = (int32_t *)malloc(sizeof(int32_t) * 8 * (size_t)in->n);
    H = orc_heuristic_perms(in, heur);
  }
  if (K == 1 && H == 0) {
    /* plain start: member p is random start p */
    for (int32_t p = 0; p < pr->P; p++) {
      int32_t *x = st->cur + (int64_t)p * len;
      random_start(in, (uint32_t)p, seed, enc, lb, ub, x, len);
      st->cost[p] = orc_cost(in, x);
      st->best_cost[p] = st->cost[p];
      memcpy(st->best_sol + (int64_t)p * len, x, sizeof(int32_t) * (size_t)len);
    }
  } else {
    /* Sec. 3.4.1: K*P random starts and the heuristic permutations form a
     * pool; the members are its P cheapest, in order of (cost, pool index) */
    const int64_t N = K * pr->P + H;
    int32_t *pool = (int32_t *)malloc(sizeof(int32_t) * (size_t)(N * len));
    orc_keyed *order = (orc_keyed *)malloc(sizeof(orc_keyed) * (size_t)N);
    for (int64_t j = 0; j < N; j++) {
      int32_t *x = pool + j * len;
      if (j < K * pr->P) random_start(in, (uint32_t)j, seed, enc, lb, ub, x, len);
      else memcpy(x, heur + (j - K * pr->P) * in->n, sizeof(int32_t) * (size_t)len);
      order[j].key = orc_cost(in, x);
      order[j].idx = j;
    }
    qsort(order, (size_t)N, sizeof(orc_keyed), keyed_less);
    for (int32_t p = 0; p < pr->P; p++) {
      const int32_t *x = pool + order[p].idx * len;
      memcpy(st->cur + (int64_t)p * len, x, sizeof(int32_t) * (size_t)len);
      memcpy(st->best_sol + (int64_t)p * len, x, sizeof(int32_t) * (size_t)len);
      st->cost[p] = st->best_cost[p] = order[p].key;
    }
    free(pool);
    free(order);
  }
  free(heur);
  st->elite_prev = st->best_cost[orc_elite(st)];
  return 0;
}

int32_t orc_elite(const orc_state *st) {
  int32_t e = 0;
  for (int32_t p = 1; p < st->P; p++)
    if (st->best_cost[p] < st->best_cost[e]) e = p;
  return e;
}

int32_t orc_threads(int32_t threads) {
#ifdef _OPENMP
  return threads > 0 ? threads : omp_get_max_threads();
#else
  (void)threads;
  return 1;
#endif
}

/* ---------------------------------------------------- one generation of one
 * solution: Alg. "evolve" for block p.  Writes its AOS counts to u/v/uk/vk.
 * Pinned by generations worked by hand (step draws, k from word r3, the
 * argmin's tie rule, every candidate's counts, the acceptance draw; a TSP
 * and a GAP case, tests/golden/generation.json). */
static void evolve_one(const orc_instance *in, const orc_params *pr, uint64_t seed,
                       orc_state *st, int32_t p, const uint32_t *w_op, const uint32_t *w_k,
                       uint64_t T, uint32_t g, int32_t *work, int64_t *delta, int32_t *ops,
                       int32_t *ks, uint32_t *u, uint32_t *v, uint32_t *uk, uint32_t *vk) {
  int32_t len = st->len, C = pr->C;
  int32_t *s = st->cur + (int64_t)p * len;
  int64_t fs = orc_cost(in, s);
  uint32_t R[4], R0[4];
  for (int32_t c = 0; c < C; c++) {
    /* each "thread" t: sample k from w_K, copy s, apply k sampled operators */
    memcpy(work, s, sizeof(int32_t) * (size_t)len);
    draw(W0(c, 0, KIND_MOVE), in->tag, (uint32_t)p, g, seed, R0);
    int32_t k = 1 + orc_wsample(w_k, 3, R0[3]);
    for (int32_t t = 0; t < k; t++) {
      if (t == 0) memcpy(R, R0, sizeof R);
      else draw(W0(c, t, KIND_MOVE), in->tag, (uint32_t)p, g, seed, R);
      int32_t op = orc_wsample(w_op, ORC_NOPS, R[0]);
      orc_apply_move(in, op, R[1] >> 16, R[1] & 0xFFFFu, R[2], work, len);
      ops[c * 3 + t] = op;
    }
    ks[c] = k;
    delta[c] = orc_cost(in, work) - fs;   /* delta_t = f(s_t) - f(s) */
  }
  /* block reduction: t* = argmin delta, ties to the lowest index [R5] */
  int32_t cs = 0;
  for (int32_t c = 1; c < C; c++)
    if (delta[c] < delta[cs]) cs = c;
  /* AOS statistics: usage and improvement of every sampled operator [R6] */
  for (int32_t c = 0; c < C; c++) {
    int32_t imp = delta[c] < 0;
    for (int32_t t = 0; t < ks[c]; t++) { u[ops[c * 3 + t]]++; v[ops[c * 3 + t]] += imp; }
    uk[ks[c] - 1]++;
    vk[ks[c] - 1] += imp;
  }
  /* thread 0: Metropolis acceptance */
  draw(W0(0, 0, KIND_ACCEPT), in->tag, (uint32_t)p, g, seed, R);
  if (orc_accept(delta[cs], T, R[0])) {
    /* s <- s_t*: rebuild the winning candidate on s itself */
    for (int32_t t = 0; t < ks[cs]; t++) {
      if (t == 0) draw(W0(cs, 0, KIND_MOVE), in->tag, (uint32_t)p, g, seed, R);
      else draw(W0(cs, t, KIND_MOVE), in->tag, (uint32_t)p, g, seed, R);
      orc_apply_move(in, ops[cs * 3 + t], R[1] >> 16, R[1] & 0xFFFFu, R[2], s, len);
    }
    st->cost[p] += delta[cs];
    if (st->cost[p] < st->best_cost[p]) { /* elite of this solution */
      st->best_cost[p] = st->cost[p];
      memcpy(st->best_sol + (int64_t)p * len, s, sizeof(int32_t) * (size_t)len);
    }
  }
}

/* Alg. "aos" body, run after every U-th generation */
static void aos_update(const orc_instance *in, const orc_params *pr, orc_state *st) {
  int32_t en[ORC_NOPS], enk[3] = {1, 1, 1};
  uint32_t capk[3] = {65536u, 65536u, 65536u};
  orc_enabled_ops(in, pr->op_mask, en);
  orc_aos_level(st->w_op, st->u_op, st->v_op, en, pr->op_cap, ORC_NOPS, pr->ema_a, pr->w_floor,
                pr->w_cap);
  orc_aos_level(st->w_k, st->u_k, st->v_k, enk, capk, 3, pr->ema_a, pr->w_floor, pr->w_cap);
  for (int32_t i = 0; i < ORC_NOPS; i++) st->u_op[i] = st->v_op[i] = 0;
  for (int32_t i = 0; i < 3; i++) st->u_k[i] = st->v_k[i] = 0;
  /* stagnation detection (Sec. 4.2.3) [R12] */
  int64_t elite = st->best_cost[orc_elite(st)];
  if (elite < st->elite_prev) st->stag = 0;
  else st->stag++;
  st->elite_prev = elite;
  if (pr->stag_limit > 0 && st->stag >= pr->stag_limit) {
    for (int32_t i = 0; i < 3; i++) st->w_k[i] = K_RESET[i];
    st->stag = 0;
  }
}

/* elite injection (Sec. 3.4.3): the worst current solution (highest cost,
 * ties to the lowest index) becomes a copy of the instance elite [R13] */
/* [R27] islands and migration (Sec. 3.4.3): island i holds members
 * [i*P/I, (i+1)*P/I).  A migrant replaces a member's current solution by a
 * source member's best solution (the rule of elite injection); sources and
 * targets are chosen on the state before any replacement.
 *   ring:  the best member of island i-1 (mod I) -> the worst of island i;
 *   top-N: the N best members of the population -> the N worst of every
 *          island, j-th best to j-th worst;
 *   hybrid: ring at odd-numbered migrations (g / period odd), top-N at even.
 * best = lowest (best cost, index); worst = highest (cost, -index). */
static void replace_member(orc_state *st, int32_t target, const int32_t *sol, int64_t cost) {
  const int32_t len = st->len;
  memcpy(st->cur + (int64_t)target * len, sol, sizeof(int32_t) * (size_t)len);
  st->cost[target] = cost;
  if (cost < st->best_cost[target]) {
    st->best_cost[target] = cost;
    memcpy(st->best_sol + (int64_t)target * len, sol, sizeof(int32_t) * (size_t)len);
  }
}

/* the k-th worst member (0 = worst) of [lo, hi) by (cost desc, index asc) */
static int32_t kth_worst(const int64_t *cost, int32_t lo, int32_t hi, int32_t k) {
  int32_t *taken = (int32_t *)calloc((size_t)(hi - lo), sizeof(int32_t)), w = -1;
  for (int32_t r = 0; r <= k; r++) {
    w = -1;
    for (int32_t q = lo; q < hi; q++)
      if (!taken[q - lo] && (w < 0 || cost[q] > cost[w])) w = q;
    taken[w - lo] = 1;
  }
  free(taken);
  return w;
}

static void migrate(const orc_params *pr, orc_state *st) {
  const int32_t P = st->P, I = (int32_t)pr->islands, S = P / I, len = st->len;
  const int64_t event = st->g / pr->migrate_period;
  const int32_t ring = pr->migrate_strategy == 0 || (pr->migrate_strategy == 2 && (event & 1));
  /* snapshot of the state the sources are taken from */
  int32_t *bsol = (int32_t *)malloc(sizeof(int32_t) * (size_t)P * len);
  int64_t *bcost = (int64_t *)malloc(sizeof(int64_t) * (size_t)P);
  int64_t *ccost = (int64_t *)malloc(sizeof(int64_t) * (size_t)P);
  memcpy(bsol, st->best_sol, sizeof(int32_t) * (size_t)P * len);
  memcpy(bcost, st->best_cost, sizeof(int64_t) * (size_t)P);
  memcpy(ccost, st->cost, sizeof(int64_t) * (size_t)P);
  if (ring) {
    for (int32_t i = 0; i < I; i++) {
      const int32_t from = (i + I - 1) % I;
      int32_t b = from * S;
      for (int32_t q = from * S; q < (from + 1) * S; q++)
        if (bcost[q] < bcost[b]) b = q;
      const int32_t t = kth_worst(ccost, i * S, (i + 1) * S, 0);
      replace_member(st, t, bsol + (int64_t)b * len, bcost[b]);
    }
  } else {
    const int32_t N = (int32_t)pr->migrate_n;
    int32_t *src = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    int32_t *taken = (int32_t *)calloc((size_t)P, sizeof(int32_t));
    for (int32_t j = 0; j < N; j++) {   /* the N best, by (best cost, index) */
      int32_t b = -1;
      for (int32_t q = 0; q < P; q++)
        if (!taken[q] && (b < 0 || bcost[q] < bcost[b])) b = q;
      taken[b] = 1;
      src[j] = b;
    }
    for (int32_t i = 0; i < I; i++)
      for (int32_t j = 0; j < N; j++) {
        const int32_t t = kth_worst(ccost, i * S, (i + 1) * S, j);
        replace_member(st, t, bsol + (int64_t)src[j] * len, bcost[src[j]]);
      }
    free(src);
    free(taken);
  }
  free(bsol);
  free(bcost);
  free(ccost);
}

int32_t orc_migrate(const orc_params *pr, orc_state *st) {
  if (pr->islands < 2 || pr->migrate_period < 1 || (uint32_t)st->P % pr->islands != 0 ||
      pr->migrate_strategy > 2 ||
      (pr->migrate_strategy != 0 && (pr->migrate_n < 1 || pr->migrate_n > (uint32_t)st->P / pr->islands)))
    return -1;
  migrate(pr, st);
  return 0;
}

/* [R31] row operators (Table "operators", row level; the paper names
 * row_swap, row_split and row_merge and says nothing more).  Rows are the V
 * routes of the separator encoding: route r spans [b_r, e_r) with b_0 = 0,
 * e_r = the r-th separator's position (e_(V-1) = len), b_r = e_(r-1) + 1.
 *   row_swap:  r1 = pos(a, V), r2 = pos(b, V-1) stepped over r1; the two
 *              routes' contents exchange places.
 *   row_merge: r = pos(a, V-1); the separator ending route r moves to the
 *              end of route r+1, so r takes r+1's customers and an empty
 *              route follows it.
 *   row_split: r = pos(a, V); with c >= 2 customers on r and an empty route
 *              z (the lowest-index one), the separator that closes z (or,
 *              for the last route, opens it) moves inside r, after its first
 *              k = 1 + pos(b, c-1) customers.  Otherwise nothing changes. */
/* Route r spans [bb[r], ee[r]).  Returns -2 unless s holds exactly V-1
 * separators (symbols >= n). */
static int32_t route_bounds(const int32_t *s, int32_t len, int32_t n, int32_t *bb, int32_t *ee,
                            int32_t V) {
  int32_t r = 0;
  bb[0] = 0;
  for (int32_t q = 0; q < len; q++)
    if (s[q] >= n) {
      if (r == V - 1) return -2;
      ee[r] = q;
      bb[++r] = q + 1;
    }
  if (r != V - 1) return -2;
  ee[V - 1] = len;
  return 0;
}

static void move_element(int32_t *s, int32_t from, int32_t to) {
  /* remove s[from]; re-insert it so that it lands at index to */
  const int32_t v = s[from];
  if (from < to)
    for (int32_t k = from; k < to; k++) s[k] = s[k + 1];
  else
    for (int32_t k = from; k > to; k--) s[k] = s[k - 1];
  s[to] = v;
}

int32_t orc_row_move(const orc_instance *in, int32_t kind, uint32_t a, uint32_t b, int32_t *s,
                     int32_t len) {
  if (in->model != ORC_CVRPTW) return -1;
  const int32_t n = in->n, V = in->vehicles;
  if (len != n + V - 1) return -2;
  if (V < 2) return 0;
  int32_t *bb = (int32_t *)malloc(sizeof(int32_t) * (size_t)V);
  int32_t *ee = (int32_t *)malloc(sizeof(int32_t) * (size_t)V);
  int32_t *t = (int32_t *)malloc(sizeof(int32_t) * (size_t)len);
  if (!bb || !ee || !t || route_bounds(s, len, n, bb, ee, V) != 0) {
    free(bb);
    free(ee);
    free(t);
    return !bb || !ee || !t ? -3 : -2;
  }
  if (kind == 0) {                                      /* row_swap */
    int32_t r1 = (int32_t)orc_pos(a, (uint32_t)V), r2 = (int32_t)orc_pos(b, (uint32_t)(V - 1));
    if (r2 >= r1) r2++;
    const int32_t lo = r1 < r2 ? r1 : r2, hi = r1 < r2 ? r2 : r1;
    int32_t o = 0;
    for (int32_t q = 0; q < bb[lo]; q++) t[o++] = s[q];
    for (int32_t q = bb[hi]; q < ee[hi]; q++) t[o++] = s[q];
    for (int32_t q = ee[lo]; q < bb[hi]; q++) t[o++] = s[q];
    for (int32_t q = bb[lo]; q < ee[lo]; q++) t[o++] = s[q];
    for (int32_t q = ee[hi]; q < len; q++) t[o++] = s[q];
    memcpy(s, t, sizeof(int32_t) * (size_t)len);
  } else if (kind == 1) {                               /* row_merge */
    const int32_t r = (int32_t)orc_pos(a, (uint32_t)(V - 1));
    move_element(s, ee[r], ee[r + 1] - 1);
  } else {                                              /* row_split */
    const int32_t r = (int32_t)orc_pos(a, (uint32_t)V), c = ee[r] - bb[r];
    int32_t z = -1;
    for (int32_t q = 0; q < V && z < 0; q++)
      if (ee[q] == bb[q]) z = q;
    if (c >= 2 && z >= 0) {
      const int32_t k = 1 + (int32_t)orc_pos(b, (uint32_t)(c - 1));
      const int32_t from = z < V - 1 ? ee[z] : bb[z] - 1;  /* the separator that goes */
      const int32_t gap = bb[r] + k;                        /* before s[gap] */
      move_element(s, from, from < gap ? gap - 1 : gap);
    }
  }
  free(bb);
  free(ee);
  free(t);
  return 0;
}

/* [R29] crossover (Table "operators", crossover level: OX for permutations,
 * uniform crossover for binary and integer vectors), taken after every AOS
 * update and migration, before elite injection.  With R = Philox(0 | 3<<24,
 * tag, p, g): member p crosses when hi16(R.r0) < cross_q16, with partner
 * q = (p + 1 + pos(hi16(R.r1), P-1)) mod P.  The parents are p's current
 * solution A and q's best solution B, both as they stood before any
 * crossover of this window.
 *   OX: cut points i = pos(hi16(R.r2), n), j = pos(lo16(R.r2), n-1) + (j >= i),
 *       lo = min, hi = max; the child keeps A[lo..hi] in place and fills the
 *       positions hi+1, ..., n-1, 0, ..., lo-1 with the elements of B that
 *       are not in A[lo..hi], in B's order from B[hi+1] on (wrapping).
 *   uniform: element k comes from B when bit k mod 32 of word (k/32) mod 4
 *       of Philox((k/128) | 1<<20 | 3<<24, tag, p, g) is set, else from A.
 * The child's cost is evaluated in full; it replaces A under the Metropolis
 * rule [R7] at the current temperature with the variate R.r3, and lowers
 * p's best like an accepted move. */
void orc_ox(const int32_t *A, const int32_t *B, int32_t len, int32_t lo, int32_t hi,
            int32_t *child) {
  char *mark = (char *)calloc((size_t)len, 1);
  for (int32_t k = lo; k <= hi; k++) {
    child[k] = A[k];
    mark[A[k]] = 1;
  }
  int32_t o = (hi + 1) % len;                           /* next free position */
  for (int32_t t = 0; t < len; t++) {
    const int32_t e = B[(hi + 1 + t) % len];
    if (!mark[e]) {
      child[o] = e;
      o = (o + 1) % len;
    }
  }
  free(mark);
}

static void crossover(const orc_instance *in, const orc_params *pr, uint64_t seed,
                      orc_state *st) {
  const int32_t P = st->P, len = st->len, enc = encoding_of(in->model);
  const uint32_t g = (uint32_t)st->g;
  int32_t *bsol = (int32_t *)malloc(sizeof(int32_t) * (size_t)P * len);
  int32_t *child = (int32_t *)malloc(sizeof(int32_t) * (size_t)len);
  memcpy(bsol, st->best_sol, sizeof(int32_t) * (size_t)P * len);
  for (int32_t p = 0; p < P; p++) {
    uint32_t R[4];
    draw(W0(0, 0, KIND_CROSS), in->tag, (uint32_t)p, g, seed, R);
    if ((R[0] >> 16) >= pr->cross_q16) continue;
    const int32_t q = (p + 1 + (int32_t)orc_pos(R[1] >> 16, (uint32_t)(P - 1))) % P;
    const int32_t *A = st->cur + (int64_t)p * len, *B = bsol + (int64_t)q * len;
    if (enc == 0) {                                     /* OX */
      int32_t i = (int32_t)orc_pos(R[2] >> 16, (uint32_t)len);
      int32_t j = (int32_t)orc_pos(R[2] & 0xFFFFu, (uint32_t)(len - 1));
      if (j >= i) j++;
      orc_ox(A, B, len, i < j ? i : j, i < j ? j : i, child);
    } else {                                            /* uniform */
      uint32_t Q[4] = {0, 0, 0, 0};
      for (int32_t k = 0; k < len; k++) {
        if (k % 128 == 0) draw(W0(k / 128, 1, KIND_CROSS), in->tag, (uint32_t)p, g, seed, Q);
        child[k] = ((Q[(k / 32) % 4] >> (k % 32)) & 1u) ? B[k] : A[k];
      }
    }
    const int64_t c = orc_cost(in, child);
    if (orc_accept(c - st->cost[p], st->T, R[3])) {
      memcpy(st->cur + (int64_t)p * len, child, sizeof(int32_t) * (size_t)len);
      st->cost[p] = c;
      if (c < st->best_cost[p]) {
        st->best_cost[p] = c;
        memcpy(st->best_sol + (int64_t)p * len, child, sizeof(int32_t) * (size_t)len);
      }
    }
  }
  free(bsol);
  free(child);
}

int32_t orc_crossover(const orc_instance *in, const orc_params *pr, uint64_t seed,
                      orc_state *st) {
  if (pr->cross_q16 > 65536u) return -1;
  if (st->P >= 2 && pr->cross_q16 > 0) crossover(in, pr, seed, st);
  return 0;
}

static void inject(orc_state *st) {
  int32_t e = orc_elite(st), wv = 0, len = st->len;
  for (int32_t p = 1; p < st->P; p++)
    if (st->cost[p] > st->cost[wv]) wv = p;
  memcpy(st->cur + (int64_t)wv * len, st->best_sol + (int64_t)e * len,
         sizeof(int32_t) * (size_t)len);
  st->cost[wv] = st->best_cost[e];
  if (st->cost[wv] < st->best_cost[wv]) {
    st->best_cost[wv] = st->cost[wv];
    memcpy(st->best_sol + (int64_t)wv * len, st->cur + (int64_t)wv * len,
           sizeof(int32_t) * (size_t)len);
  }
}

int32_t orc_run(const orc_instance *in, const orc_params *pr, uint64_t seed, orc_state *st,
                int64_t generations, int32_t threads) {
  int32_t P = st->P, len = st->len, C = pr->C;
  if (C < 1 || pr->U < 1) return -1;
  if (pr->islands > 1 && pr->migrate_period > 0 &&
      ((uint32_t)P % pr->islands != 0 || pr->migrate_strategy > 2 ||
       (pr->migrate_strategy != 0 && (pr->migrate_n < 1 || pr->migrate_n > (uint32_t)P / pr->islands))))
    return -1;
  if (pr->cross_q16 > 65536u) return -1;
  uint32_t *cnt = (uint32_t *)calloc((size_t)P * ORC_NSTATS, sizeof(uint32_t));
  int32_t nthreads = orc_threads(threads);
  for (int64_t it = 0; it < generations; it++) {
    uint32_t g = (uint32_t)st->g;
    memset(cnt, 0, sizeof(uint32_t) * (size_t)P * ORC_NSTATS);
#pragma omp parallel num_threads(nthreads)
    {
      int32_t *work = (int32_t *)malloc(sizeof(int32_t) * (size_t)len);
      int64_t *delta = (int64_t *)malloc(sizeof(int64_t) * (size_t)C);
      int32_t *ops = (int32_t *)malloc(sizeof(int32_t) * (size_t)C * 3);
      int32_t *ks = (int32_t *)malloc(sizeof(int32_t) * (size_t)C);
#pragma omp for schedule(dynamic, 1)
      for (int32_t p = 0; p < P; p++) {
        uint32_t *c = cnt + (int64_t)p * ORC_NSTATS;
        evolve_one(in, pr, seed, st, p, st->w_op, st->w_k, st->T, g, work, delta, ops, ks, c,
                   c + ORC_NOPS, c + 2 * ORC_NOPS, c + 2 * ORC_NOPS + 3);
      }
      free(work); free(delta); free(ops); free(ks);
    }
    for (int32_t p = 0; p < P; p++) {
      const uint32_t *c = cnt + (int64_t)p * ORC_NSTATS;
      const uint32_t *cv = c + ORC_NOPS, *ck = c + 2 * ORC_NOPS, *cvk = ck + 3;
      for (int32_t i = 0; i < ORC_NOPS; i++) { st->u_op[i] += c[i]; st->v_op[i] += cv[i]; }
      for (int32_t i = 0; i < 3; i++) { st->u_k[i] += ck[i]; st->v_k[i] += cvk[i]; }
      for (int32_t i = 0; i < ORC_NOPS; i++) { st->all_u_op[i] += c[i]; st->all_v_op[i] += cv[i]; }
      for (int32_t i = 0; i < 3; i++) { st->all_u_k[i] += ck[i]; st->all_v_k[i] += cvk[i]; }
    }
    st->T = orc_cool(st->T, pr->alpha);
    st->g++;
    if (st->g % pr->U == 0) aos_update(in, pr, st);
    if (pr->islands > 1 && pr->migrate_period > 0 && st->g % pr->migrate_period == 0) migrate(pr, st);
    if (pr->cross_q16 > 0 && P >= 2 && st->g % pr->U == 0) crossover(in, pr, seed, st);
    if (pr->elite_period > 0 && st->g % pr->elite_period == 0) inject(st);
  }
  free(cnt);
  return 0;
}
