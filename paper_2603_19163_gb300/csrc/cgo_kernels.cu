// Kernels of the per-solution search generation (sm_103a).
//
// One warp evolves one population member at a time (a CTA holds a few
// members; a warp may own several).  Per generation the 32 lanes evaluate the
// C candidates (C/32 per lane): each draws k from w_K and k operators from
// w_S (Alg. "evolve"), and the cost delta of the k-step composite move is
// computed exactly from the instance data without materialising it.  A warp
// argmin picks the best candidate (ties to the lowest index), the Metropolis
// test uses a pre-drawn Exp(1) variate, and the winner is applied in place.
// After every U-th generation the members of an instance meet at a barrier
// (global-memory counters, bounded wait) where the AOS counts are summed and
// every warp applies Eq. "ema", the stagnation rule and, when due, elite
// injection (Alg. "aos", Sec. 3.4.3, 4.2).
#include <atomic>
#include <climits>
#include <type_traits>
#include <mutex>
#include <set>
#include <utility>
#include <cooperative_groups.h>

#include "cgo_device.cuh"

namespace cgo {
#ifdef CGO_UNIT
// a kernel unit keeps its copies of the device code local
namespace {
#endif

// ---------------------------------------------------------------- layout
// Solutions in shared memory use compact elements: permutation symbols
// (< 65536) as uint16, binary values and agent indices (< 256) as uint8.
using PermEl = uint16_t;
using ByteEl = uint8_t;
__host__ __device__ inline int sol_esize(int model) {
  return (model == KNAPSACK || model == GAP) ? 1 : 2;
}
template <int MODEL>
struct SolEl {
  using T = PermEl;
};
template <>
struct SolEl<KNAPSACK> {
  using T = ByteEl;
};
template <>
struct SolEl<GAP> {
  using T = ByteEl;
};

struct SolScal {
  long long cost, best, aw, av;  // aw/av: knapsack sum of weights / values
};

struct Layout {
  int64_t inst, sol_off, sol_stride, scr_off, scr_stride, scal_off, snap_off, load_off, aux_off,
      aux_stride, part_off, total;
};

__host__ __device__ inline int64_t align16(int64_t x) { return (x + 15) & ~int64_t(15); }

// per member group of nw warps: two buffers of per-warp partial argmins
// (16 B each), a flag (16 B), two buffers of per-warp winner moves (64 B
// each) and each warp's window counts (32 x 4 B)
__host__ __device__ inline int64_t group_bytes(int nw) { return 2 * nw * 16 + 16 + 2 * nw * 64 + nw * 128; }

// CVRPTW route cache of one member: route-cost prefix sums (len + 2 int64),
// the next / previous separator of every position (len + 1, len int32) and
// the separators' positions in order with the lowest-index empty route
// (len + 1 int32)
// (+ with the longest-route objective: prefix and suffix maxima of the route
// distances, len + 2 int64 each)
__host__ __device__ inline int64_t cv_aux_bytes(int len, bool cvmax = false) {
  return align16(8 * (int64_t)(len + 2) + 4 * (int64_t)(len + 1) + 4 * (int64_t)len +
                 4 * (int64_t)(len + 1)) +
         (cvmax ? align16(16 * (int64_t)(len + 2)) : 0);
}

// Shared memory of one CTA: [instance data][members' solutions][one scratch
// array per member group (permutations: a solution row and a bitmask)]
// [member scalars][parent-row costs][GAP loads][CVRPTW route caches / ATSP
// prefix sums]
// [per-group partials]
__host__ __device__ inline Layout make_layout(int64_t inst_bytes, int len, int m, int nsol,
                                              int warps, int wpm, int model, bool cvmax = false) {
  Layout L;
  const int groups = warps / wpm;
  L.inst = align16(inst_bytes);
  L.sol_stride = align16((int64_t)len * sol_esize(model));
  L.sol_off = L.inst;
  L.scr_off = L.sol_off + (int64_t)nsol * L.sol_stride;
  const bool perm = (model == TSP || model == QAP || model == CVRPTW || model == ATSP);
  // a permutation's scratch row, then a bitmask of len bits (crossover)
  L.scr_stride = perm ? L.sol_stride + align16(4 * (int64_t)((len + 31) / 32)) : 0;
  L.scal_off = L.scr_off + (int64_t)groups * L.scr_stride;
  // per member, the best cost held by each of its two crossover-parent rows
  L.snap_off = L.scal_off + align16((int64_t)nsol * 32);
  L.load_off = L.snap_off + align16((int64_t)nsol * 16);
  L.aux_off = L.load_off + (model == GAP ? align16((int64_t)nsol * m * 8) : 0);
  L.aux_stride = model == CVRPTW ? cv_aux_bytes(len, cvmax)
                                 : (model == ATSP ? align16(16 * (int64_t)(len + 1)) : 0);
  L.part_off = L.aux_off + (int64_t)nsol * L.aux_stride;
  L.total = L.part_off + (int64_t)groups * group_bytes(wpm);
  return L;
}

#ifndef CGO_UNIT
int64_t instance_data_bytes(const KInst &h) {
  switch (h.model) {
    case TSP: return align16((int64_t)h.n * (h.n + 1) / 2 * (h.tri16 ? 2 : 4));
    case ATSP: return align16((int64_t)h.n * h.n * (h.tri16 ? 2 : 4));
    case QAP: return 4 * align16((int64_t)h.n * (h.n | 1) * 4);  // F, D and their transposes
    case KNAPSACK: return 2 * align16((int64_t)h.n * 4);
    case GAP: return 2 * align16((int64_t)h.m * h.n * 4) + align16((int64_t)h.m * 4);
    case CVRPTW: {
      const int64_t N = h.n + 1;
      return align16(N * N * 4) + N * 16;
    }
  }
  return 0;
}

int64_t smem_instance(const KInst &h) { return instance_data_bytes(h); }
int64_t smem_per_warp(const KInst &h) {
  Layout a = make_layout(0, h.len, h.m, 1, 1, 1, h.model, h.wlong > 0);
  return a.total;
}
#endif

// ------------------------------------------------------------- instance view
struct View {
  int n, len, m;
  long long cap, lam0;
  uint32_t tag, k0, k1;
  const void *tri;
  int n2m1;
  const int32_t *F, *D;        // QAP (row stride qs)
  const int32_t *FT, *DT;      // QAP transposes when staged (else null)
  int qs;
  const int32_t *w, *v;        // knapsack
  const int32_t *gc, *gr, *gcap;  // GAP
  const int32_t *rd, *dem, *rdy, *due, *svc;  // CVRPTW: travel (n+1)^2, vectors n+1
  const int4 *node;                           // CVRPTW: {ready, due, service, demand}
  long long lam1;
  long long wd, wv;  // CVRPTW objective weights (distance, vehicles used)
  long long wl;      // CVRPTW: weight of the longest route's distance
  const KInst *ki;   // the instance (the CVRPTW lexicographic mode's constants)
  bool cv32;
  bool t3;   // 3-opt enabled for this instance
  bool t16;  // TSP / ATSP matrix entries stored as int16
  bool seg;  // seg_flip / seg_reset enabled for this instance
};

template <int NO>
struct Stats {
  uint32_t u[NO], v[NO], uk[3], vk[3];
};

template <int NO>
__device__ __forceinline__ void stats_zero(Stats<NO> &s) {
#pragma unroll
  for (int i = 0; i < NO; ++i) s.u[i] = s.v[i] = 0;
#pragma unroll
  for (int i = 0; i < 3; ++i) s.uk[i] = s.vk[i] = 0;
}

// What one candidate adds to the window counts, packed in a word: the local
// operator of each of its three steps (bits 4t..4t+3, 15 = step not taken),
// its step count k (bits 12-13) and whether it improves (bit 14).  A record
// is added to the counts only once its generation is decided on the solution
// it was evaluated against.
__device__ __forceinline__ uint32_t stats_record(int op0, int op1, int op2, int k, uint32_t imp) {
  const uint32_t a = op0 < 0 ? 15u : (uint32_t)op0, b = op1 < 0 ? 15u : (uint32_t)op1,
                 c = op2 < 0 ? 15u : (uint32_t)op2;
  return a | (b << 4) | (c << 8) | ((uint32_t)k << 12) | (imp << 14);
}

constexpr uint32_t kNoRecord = 0xFFFu;  // no step taken, k = 0

// Window counts of one member kept in bytes while it evolves (one byte per
// operator or k level, uses and improvements apart), added to the full
// counts when its window ends; valid while a lane counts at most 255 uses of
// one kind in a member window (3 * candidates per lane * U <= 255).
struct PackedStats {
  uint32_t u, v;    // local operators 0..3, one byte each
  uint32_t uk, vk;  // k levels 1..3 in bytes 0..2, local operator 4 in byte 3
  uint32_t u2, v2;  // local operators 5..7 (the row level of CVRPTW)
};

template <int NO>
__device__ __forceinline__ void packed_add(PackedStats &s, uint32_t rec) {
  const uint32_t imp = (rec >> 14) & 1u, k = (rec >> 12) & 3u;
  uint32_t inc = 0, inck = k ? 1u << (8u * (k - 1u)) : 0u, inc2 = 0;
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    const uint32_t op = (rec >> (4 * t)) & 15u;
    inc += op < 4u ? 1u << (8u * op) : 0u;
    inck += op == 4u ? 1u << 24 : 0u;
    if constexpr (NO > 5) inc2 += (op >= 5u && op < 8u) ? 1u << (8u * (op - 5u)) : 0u;
  }
  s.u += inc;
  s.v += imp ? inc : 0u;
  s.uk += inck;
  s.vk += imp ? inck : 0u;
  if constexpr (NO > 5) {
    s.u2 += inc2;
    s.v2 += imp ? inc2 : 0u;
  }
}

template <int NO>
__device__ __forceinline__ void packed_flush(Stats<NO> &st, PackedStats &s) {
#pragma unroll
  for (int i = 0; i < NO; ++i) {
    st.u[i] += (i < 4 ? s.u >> (8 * i) : (i == 4 ? s.uk >> 24 : s.u2 >> (8 * (i - 5)))) & 0xFFu;
    st.v[i] += (i < 4 ? s.v >> (8 * i) : (i == 4 ? s.vk >> 24 : s.v2 >> (8 * (i - 5)))) & 0xFFu;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    st.uk[i] += (s.uk >> (8 * i)) & 0xFFu;
    st.vk[i] += (s.vk >> (8 * i)) & 0xFFu;
  }
  s.u = s.v = s.uk = s.vk = s.u2 = s.v2 = 0u;
}

template <int NO>
__device__ __forceinline__ void stats_add(Stats<NO> &s, uint32_t rec) {
  const uint32_t imp = (rec >> 14) & 1u, k = (rec >> 12) & 3u;
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    const uint32_t op = (rec >> (4 * t)) & 15u;
#pragma unroll
    for (int i = 0; i < NO; ++i) {
      const uint32_t hit = (op == (uint32_t)i);
      s.u[i] += hit;
      s.v[i] += hit & imp;
    }
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const uint32_t hit = (k == (uint32_t)(i + 1));
    s.uk[i] += hit;
    s.vk[i] += hit & imp;
  }
}

// per-encoding operator set: local op l is global op glob(l) (permutations:
// swap, 2-opt, insertion, or-opt, 3-opt; CVRPTW's separator sequence adds the
// row level: row_swap, row_merge, row_split; binary: flip, seg_flip; integer:
// reset, seg_reset), in the order of the global slots
struct PermOps {
  static constexpr int NO = 5;
  __host__ __device__ static constexpr int glob(int l) { return l < 4 ? l : (int)THREE_OPT; }
};
template <int MODEL>
struct Enc : PermOps {};
template <>
struct Enc<CVRPTW> {
  static constexpr int NO = 8;
  __host__ __device__ static constexpr int glob(int l) {
    return l < 4 ? l : (l == 4 ? (int)THREE_OPT : (int)ROW_SWAP + (l - 5));
  }
};
template <>
struct Enc<KNAPSACK> {
  static constexpr int NO = 2;
  __host__ __device__ static constexpr int glob(int l) { return l == 0 ? (int)FLIP : (int)SEGMENT; }
};
template <>
struct Enc<GAP> {
  static constexpr int NO = 2;
  __host__ __device__ static constexpr int glob(int l) { return l == 0 ? (int)PERTURB : (int)SEGMENT; }
};

// [R28] elements a step of the binary / integer sets touches: 1 for the
// element operator, min(2 + (x & 1), n) for the segment operator; the
// segment starts at pos(a, n - L + 1) (the element operator's pos(a, n))
constexpr int kSegMax = 3;
__device__ __forceinline__ int seg_len(int op, uint32_t x, int n) {
  return op == 0 ? 1 : min(2 + (int)(x & 1u), n);
}

template <int NO>
struct Weights {
  // prefix sums only (the roulette's thresholds): op[i] = cop[i] - cop[i-1]
  uint32_t cop[NO], ck[3];
  uint32_t Wop, Wk;
};

// the prefix sums and totals of both levels from the weights (when the
// weights change, i.e. once per window), and the weights back
template <int NO>
__device__ __forceinline__ void weights_set(Weights<NO> &w, const uint32_t (&op)[NO],
                                            const uint32_t (&k)[3]) {
  w.Wop = 0;
#pragma unroll
  for (int i = 0; i < NO; ++i) {
    w.Wop += op[i];
    w.cop[i] = w.Wop;
  }
  w.ck[0] = k[0];
  w.ck[1] = w.ck[0] + k[1];
  w.ck[2] = w.ck[1] + k[2];
  w.Wk = w.ck[2];
}

template <int NO>
__device__ __forceinline__ void weights_get(const Weights<NO> &w, uint32_t (&op)[NO],
                                            uint32_t (&k)[3]) {
#pragma unroll
  for (int i = 0; i < NO; ++i) op[i] = w.cop[i] - (i ? w.cop[i - 1] : 0u);
  k[0] = w.ck[0];
  k[1] = w.ck[1] - w.ck[0];
  k[2] = w.ck[2] - w.ck[1];
}

__device__ __forceinline__ long long overp(long long x) { return x > 0 ? x : 0; }

// ---------------------------------------------------------------- TSP
// D(x, y) of the symmetric matrix is the upper-triangle entry of
// (min, max) at offset a (2n - 1 - a) / 2 + b.

// element at position q of the array after the np prior moves (p0 first)
__device__ __forceinline__ int vlook(const PermEl *sol, int q, const PMove &p0, const PMove &p1,
                                     int np) {
  if (np >= 2) q = perm_inv(p1, q);
  if (np >= 1) q = perm_inv(p0, q);
  return sol[q];
}

// Symmetric-TSP delta of one move on the (virtual) array (evaluated by
// tsp_three_steps below for all three steps at once).  The cyclic tour
// is R A M B (R = P4 P0 joined around the end) and becomes R B M A (or
// R A^r for 2-opt).  Pieces keep their internal edges (D is symmetric), so
// only junction edges change.  With r_l / r_f the elements just before A and
// just after B in the cyclic tour:
//   2-opt:      d(r_l,A_l) + d(A_f,r_f) - d(r_l,A_f) - d(A_l,r_f)
//   exchange:   d(r_l,B_f) + d(A_l,r_f) - d(r_l,A_f) - d(B_l,r_f) + mid,
//     M empty:  mid = d(B_l,A_f) - d(A_l,B_f)
//     M:        mid = d(B_l,M_f) + d(M_l,A_f) - d(A_l,M_f) - d(M_l,B_f)
// When R is empty (A starts the array and B ends it) the tour is A M B and
// the delta is 0 except for an exchange with M non-empty:
//   d(B_l,M_f) + d(M_l,A_f) + d(A_l,B_f) - d(A_l,M_f) - d(M_l,B_f) - d(B_l,A_f).

// ---------------------------------------------------------------- QAP
// Swap of positions r, s on the (virtual) permutation pi: O(n) delta of
// sum_ij F[i][j] D[pi_i][pi_j] for general (asymmetric, non-zero diagonal)
// F and D.
// Q: the arithmetic type (int when the host proved every partial sum fits).
template <class Q>
__device__ __forceinline__ long long qap_step_t(const View &X, const PermEl *sol, const PMove &mv,
                                                const PMove &p0, const PMove &p1, int np) {
  const int n = X.n;
  const int r = mv.b1, s = mv.b3;
  const int pr = vlook(sol, r, p0, p1, np), ps = vlook(sol, s, p0, p1, np);
  const int32_t *F = X.F, *D = X.D;
  const int qs = X.qs;
  const int32_t *Fr = F + (size_t)r * qs, *Fs = F + (size_t)s * qs;
  const int32_t *Dr = D + (size_t)pr * qs, *Ds = D + (size_t)ps * qs;
  Q acc = 0;
  if (X.FT) {
    // F[k][r] = FT[r][k], D[pk][ps] = DT[ps][pk]: every read is a row read,
    // lanes on different rows of an odd stride hit different banks
    const int32_t *FTr = X.FT + (size_t)r * qs, *FTs = X.FT + (size_t)s * qs;
    const int32_t *DTr = X.DT + (size_t)pr * qs, *DTs = X.DT + (size_t)ps * qs;
    for (int k = 0; k < n; ++k) {
      const int pk = vlook(sol, k, p0, p1, np);
      const Q t1 = ((Q)Fr[k] - (Q)Fs[k]) * ((Q)Ds[pk] - (Q)Dr[pk]);
      const Q t2 = ((Q)FTr[k] - (Q)FTs[k]) * ((Q)DTs[pk] - (Q)DTr[pk]);
      acc += (k != r && k != s) ? t1 + t2 : (Q)0;
    }
  } else {
    for (int k = 0; k < n; ++k) {
      const int pk = vlook(sol, k, p0, p1, np);
      const Q t1 = ((Q)Fr[k] - (Q)Fs[k]) * ((Q)Ds[pk] - (Q)Dr[pk]);
      const int32_t *Fk = F + (size_t)k * qs, *Dk = D + (size_t)pk * qs;
      const Q t2 = ((Q)Fk[r] - (Q)Fk[s]) * ((Q)Dk[ps] - (Q)Dk[pr]);
      acc += (k != r && k != s) ? t1 + t2 : (Q)0;
    }
  }
  acc += ((Q)Fr[r] - (Q)Fs[s]) * ((Q)Ds[ps] - (Q)Dr[pr]);
  acc += ((Q)Fr[s] - (Q)Fs[r]) * ((Q)Ds[pr] - (Q)Dr[ps]);
  return (long long)acc;
}

__device__ long long qap_step(const View &X, const PermEl *sol, const PMove &mv,
                              const PMove &p0, const PMove &p1, int np) {
  return X.cv32 ? qap_step_t<int>(X, sol, mv, p0, p1, np)
                : qap_step_t<long long>(X, sol, mv, p0, p1, np);
}

// Any other permutation move (2-opt, insertion, or-opt, 3-opt) on the
// (virtual) permutation V: only the positions H = [b1, b4) change, so
//   delta = sum_{i in H} sum_j F[i][j] (D[V'_i][V'_j] - D[V_i][V_j])
//         + sum_{i not in H} sum_{j in H} F[i][j] (D[V_i][V'_j] - D[V_i][V_j]),
// with V'_q = V_{inv(q)} (64-bit arithmetic: O(n |H|) terms).  H is taken
// in chunks of up to 32 positions whose old and new values are looked up
// once; the rows of a chunk are summed column by column, so each column's
// values are looked up once per chunk too.
__device__ long long qap_block_step(const View &X, const PermEl *sol, const PMove &mv,
                                    const PMove &p0, const PMove &p1, int np) {
  constexpr int kChunk = 32;
  const int n = X.n, lo = mv.b1, hi = mv.b4, qs = X.qs;
  const int32_t *F = X.F, *D = X.D;
  auto V = [&](int q) { return vlook(sol, q, p0, p1, np); };
  int vH[kChunk], wH[kChunk];
  long long acc = 0;
  for (int c0 = lo; c0 < hi; c0 += kChunk) {
    const int len = min(hi - c0, kChunk);
    for (int t = 0; t < len; ++t) {
      vH[t] = V(c0 + t);
      wH[t] = V(perm_inv(mv, c0 + t));
    }
    // rows in the chunk, every column
    for (int j = 0; j < n; ++j) {
      const int vj = V(j), wj = (j >= lo && j < hi) ? V(perm_inv(mv, j)) : vj;
      const int32_t *Fj = F + (size_t)c0 * qs + j;
      for (int t = 0; t < len; ++t)
        acc += (long long)Fj[(size_t)t * qs] *
               ((long long)D[(size_t)wH[t] * qs + wj] - (long long)D[(size_t)vH[t] * qs + vj]);
    }
    // rows outside H, the chunk's columns
    for (int i = 0; i < n; ++i) {
      if (i >= lo && i < hi) continue;
      const int vi = V(i);
      const int32_t *Fi = F + (size_t)i * qs + c0, *Dv = D + (size_t)vi * qs;
      for (int t = 0; t < len; ++t) acc += (long long)Fi[t] * ((long long)Dv[wH[t]] - (long long)Dv[vH[t]]);
    }
  }
  return acc;
}

// ---------------------------------------------------------------- CVRPTW
// Cost of the whole routes in positions [L, R) of a separator-encoded
// sequence (symbols < n are customers 1..n, others end a route); R acts as
// a separator.  Per route from the depot at t = 0: t = max(t + d, ready),
// late += max(0, t - due), t += service; back at the depot t += d and
// late += max(0, t - due_0); empty routes cost nothing.  A route that visits
// a customer costs wd * distance + penalties + wv (R30's objective weights).
// Up to three jumps (from separator position jf_i to separator position
// jt_i, in increasing order) leave out whole routes known to cancel.
struct Jumps {
  int f0 = INT_MAX, t0 = 0, f1 = INT_MAX, t1 = 0, f2 = INT_MAX, t2 = 0;
};

template <class Look, class Q>
__device__ __forceinline__ long long cvrptw_routes_t(const View &X, Look V, int L, int R,
                                                     Jumps J = Jumps(), long long *mx = nullptr) {
  const int n = X.n, N = n + 1;
  long long total = 0;
  Q t = 0, load = 0, dist = 0, late = 0;
  int prev = 0;
  for (int q = L; q <= R; ++q) {
    // one body for customers and separators (a separator is the trip back
    // to the depot, node 0), so lanes at either kind of position stay together
    const int sym = q < R ? V(q) : n;
    const bool sep = sym >= n;
    const int c = sep ? 0 : sym + 1;
    const int4 nd = X.node[c];  // ready, due, service, demand (depot: its due)
    const Q dd = (Q)X.rd[(size_t)prev * N + c];
    dist += dd;
    const Q arr = t + dd;
    t = sep ? arr : max(arr, (Q)nd.x);
    late += max(t - (Q)nd.y, (Q)0);
    t += sep ? (Q)0 : (Q)nd.z;
    load += sep ? (Q)0 : (Q)nd.w;
    if (sep) {
      if (prev != 0) {
        total += X.wd * (long long)dist + X.lam0 * overp((long long)load - X.cap) +
                 X.lam1 * (long long)late + X.wv;
        if (mx) *mx = max(*mx, (long long)dist);
      }
      t = load = dist = late = 0;
      prev = 0;
      if (q == J.f0) {
        q = J.t0;
        J.f0 = J.f1;
        J.t0 = J.t1;
        J.f1 = J.f2;
        J.t1 = J.t2;
        J.f2 = INT_MAX;
      }
    } else {
      prev = c;
    }
  }
  return total;
}

template <class Look>
__device__ __forceinline__ long long cvrptw_routes(const View &X, Look V, int L, int R, bool q32,
                                                   Jumps J = Jumps(), long long *mx = nullptr) {
  return q32 ? cvrptw_routes_t<Look, int>(X, V, L, R, J, mx)
             : cvrptw_routes_t<Look, long long>(X, V, L, R, J, mx);
}

// Route cache of one member's (actual) sequence: cum[q] = cost of the routes
// ended by a terminator (separator, or the virtual one at len) before q;
// nxt[q] = first separator at or after q (len if none, nxt[len] = len);
// prv[q] = last separator at or before q (-1 if none); sep[r] = position of
// the r-th separator (r < V - 1) and sep[len] = the lowest-index empty route
// (-1 if none).
// With the longest-route objective also pmx[q] = the largest distance of a
// route that ends (at its terminator) before q and smx[q] = that of a route
// that starts at or after q (q = 0 .. len + 1; 0 where there is none).
struct CvAux {
  long long *cum;
  int *nxt, *prv, *sep;
  long long *pmx, *smx;
};

__device__ __forceinline__ CvAux cv_aux_at(unsigned char *p, int len, bool cvmax = false) {
  CvAux a;
  a.cum = (long long *)p;
  a.nxt = (int *)(p + 8 * (int64_t)(len + 2));
  a.prv = a.nxt + (len + 1);
  a.sep = a.prv + len;
  a.pmx = a.smx = nullptr;
  if (cvmax) {
    a.pmx = (long long *)(p + cv_aux_bytes(len));
    a.smx = a.pmx + (len + 2);
  }
  return a;
}

// Rebuild the cache after the member's sequence changed (one warp of the
// group; the group waits for it).
template <class El, class G_t>
__device__ void cv_build(const View &X, const El *sol, const CvAux &a, const G_t &G) {
  const int m = X.len, n = X.n, lane = threadIdx.x & 31;
  if (G.gw == 0) {
    int carry = -1;
    for (int base = 0; base < m; base += 32) {
      const int q = base + lane;
      int v = (q < m && (int)sol[q] >= n) ? q : -1;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const int u = __shfl_up_sync(kFull, v, off);
        if (lane >= off) v = max(v, u);
      }
      v = max(v, carry);
      if (q < m) a.prv[q] = v;
      carry = __shfl_sync(kFull, v, 31);
    }
    carry = m;
    for (int top = m - 1; top >= 0; top -= 32) {
      const int q = top - lane;
      int v = (q >= 0 && (int)sol[q] >= n) ? q : m;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const int u = __shfl_up_sync(kFull, v, off);
        if (lane >= off) v = min(v, u);
      }
      v = min(v, carry);
      if (q >= 0) a.nxt[q] = v;
      carry = __shfl_sync(kFull, v, 31);
    }
    if (lane == 0) a.nxt[m] = m;
    for (int q = lane; q <= m + 1; q += 32) a.cum[q] = 0;
    // separators in order, and the lowest-index empty route: route r runs
    // from just after separator r - 1 (from 0 for r = 0) to separator r (to
    // len for the last one)
    int rank = 0, zmin = INT_MAX;
    for (int base = 0; base < m; base += 32) {
      const int q = base + lane;
      const bool sp = q < m && (int)sol[q] >= n;
      const uint32_t bal = __ballot_sync(kFull, sp);
      const int r = rank + __popc(bal & ((1u << lane) - 1u));
      if (sp) {
        a.sep[r] = q;
        // route r is empty when it starts here (q = 0, or a separator before)
        if (q == 0 || (int)sol[q - 1] >= n) zmin = min(zmin, r);
      }
      rank += __popc(bal);
    }
    // the last route is empty when the sequence ends with a separator
    if (lane == 0 && m > 0 && (int)sol[m - 1] >= n) zmin = min(zmin, rank);
    zmin = __reduce_min_sync(kFull, zmin);
    if (lane == 0) a.sep[m] = zmin == INT_MAX ? -1 : zmin;
    __syncwarp();
    if (a.pmx)
      for (int q = lane; q <= m + 1; q += 32) a.pmx[q] = a.smx[q] = 0;
    __syncwarp();
    // each non-empty route's cost, stored one past its terminator (and its
    // distance at the same place and at its start, for the maxima)
    for (int q = lane; q < m; q += 32) {
      if ((q == 0 || (int)sol[q - 1] >= n) && (int)sol[q] < n) {
        const int s = a.nxt[q];
        long long rd = 0;
        a.cum[s + 1] = cvrptw_routes(X, [&](int r) { return (int)sol[r]; }, q, s, X.cv32, Jumps(),
                                     a.pmx ? &rd : nullptr);
        if (a.pmx) {
          a.pmx[s + 1] = rd;
          a.smx[q] = rd;
        }
      }
    }
    __syncwarp();
    if (a.pmx) {
      // prefix maxima over pmx, suffix maxima over smx
      long long c1 = 0;
      for (int base = 0; base <= m + 1; base += 32) {
        const int q = base + lane;
        long long v = q <= m + 1 ? a.pmx[q] : 0ll;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
          const long long u = __shfl_up_sync(kFull, v, off);
          if (lane >= off) v = max(v, u);
        }
        v = max(v, c1);
        __syncwarp();
        if (q <= m + 1) a.pmx[q] = v;
        c1 = __shfl_sync(kFull, v, 31);
      }
      long long c2s = 0;
      for (int top = m + 1; top >= 0; top -= 32) {
        const int q = top - lane;
        long long v = q >= 0 ? a.smx[q] : 0ll;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
          const long long u = __shfl_up_sync(kFull, v, off);
          if (lane >= off) v = max(v, u);
        }
        v = max(v, c2s);
        __syncwarp();
        if (q >= 0) a.smx[q] = v;
        c2s = __shfl_sync(kFull, v, 31);
      }
      __syncwarp();
    }
    long long c2 = 0;
    for (int base = 0; base <= m + 1; base += 32) {
      const int q = base + lane;
      long long v = q <= m + 1 ? a.cum[q] : 0ll;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const long long u = __shfl_up_sync(kFull, v, off);
        if (lane >= off) v += u;
      }
      v += c2;
      __syncwarp();
      if (q <= m + 1) a.cum[q] = v;
      c2 = __shfl_sync(kFull, v, 31);
    }
  }
  G.sync();
}

// Delta of a first step (on the actual sequence) from the cache: the old
// routes' cost is a difference of prefix sums; when no piece is reversed,
// the routes that lie wholly inside one moved piece are the same before and
// after and are left out of both sides; only the new routes are walked.
__device__ long long cvrptw_step0(const View &X, const PermEl *sol, const PMove &mv,
                                  const CvAux &a) {
  const int b1 = mv.b1, b2 = mv.b2, b3 = mv.b3, b4 = mv.b4;
  const int L = b1 > 0 ? a.prv[b1 - 1] + 1 : 0;
  const int R = a.nxt[b4];
  long long old = a.cum[R + 1] - a.cum[L];
  if (X.wl > 0) {
    // the longest route: the routes outside [L, R] keep their distances
    // (prefix / suffix maxima); the new ones over [L, R] are walked whole
    long long mx = max(a.pmx[L], a.smx[R + 1]);
    auto Vn = [&](int q) { return (int)sol[perm_inv(mv, q)]; };
    const long long nw = cvrptw_routes(X, Vn, L, R, X.cv32, Jumps(), &mx);
    return nw - old + X.wl * (mx - a.pmx[X.len + 1]);
  }
  Jumps J;
  if (!mv.rev) {
    const int lb = b4 - b3, lm = b3 - b2;
    // new order: B at b1, M at b1 + lb, A at b1 + lb + lm
    int nj = 0;
    const int x1s[3] = {b3, b2, b1}, x2s[3] = {b4, b3, b2}, nb[3] = {b1, b1 + lb, b1 + lb + lm};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int x1 = x1s[i], x2 = x2s[i];
      if (x2 > x1) {
        const int f = a.nxt[x1];
        if (f < x2) {
          const int l = a.prv[x2 - 1];
          if (l > f) {
            old -= a.cum[l + 1] - a.cum[f + 1];
            const int jf = nb[i] + (f - x1), jt = nb[i] + (l - x1);
            if (nj == 0) {
              J.f0 = jf;
              J.t0 = jt;
            } else if (nj == 1) {
              J.f1 = jf;
              J.t1 = jt;
            } else {
              J.f2 = jf;
              J.t2 = jt;
            }
            ++nj;
          }
        }
      }
    }
  }
  auto Vn = [&](int q) { return (int)sol[perm_inv(mv, q)]; };
  return cvrptw_routes(X, Vn, L, R, X.cv32, J) - old;
}

// The moves of one candidate, kept by the lane that may win the argmin so
// that the group can apply it without redrawing.
struct CandMoves {
  PMove m[3];
  int k;
};

// ---------------------------------------------------------------- ATSP
// TSP of an asymmetric matrix (Sec. 3.1's TSP asks no symmetry of D).  A
// reversed piece of the tour changes the direction of its inner edges, so
// the junction delta of the symmetric case does not hold.  Each member
// keeps the prefix sums of its tour's forward and backward edge costs:
// F[q] = sum_{i<q} D[s_i][s_(i+1)], B[q] = sum_{i<q} D[s_(i+1)][s_i]
// (q < len) and F[len] = the whole cyclic tour.  A candidate's k moves turn
// the tour into at most 13 pieces of the current one, each traversed forward
// or backward; its cost is the pieces' inner edges (from the prefix sums)
// plus the edges that join them.
struct TsAux {
  long long *F, *B;
};
__device__ __forceinline__ TsAux ts_aux_at(unsigned char *p, int len) {
  TsAux a;
  a.F = (long long *)p;
  a.B = a.F + (len + 1);
  return a;
}

template <bool T16>
__device__ __forceinline__ long long dfull(const View &X, int a, int b) {
  const size_t i = (size_t)a * X.n + b;
  return T16 ? (long long)((const int16_t *)X.tri)[i] : (long long)((const int32_t *)X.tri)[i];
}

template <bool T16, class El, class G_t>
__device__ void ts_build(const View &X, const El *sol, const TsAux &a, const G_t &G) {
  const int m = X.len, lane = threadIdx.x & 31;
  if (G.gw == 0) {
    long long cf = 0, cb = 0;
    for (int base = 0; base < m; base += 32) {
      const int q = base + lane;
      long long f = 0, b = 0;
      if (q + 1 < m) {
        f = dfull<T16>(X, (int)sol[q], (int)sol[q + 1]);
        b = dfull<T16>(X, (int)sol[q + 1], (int)sol[q]);
      }
      // inclusive scans, then shifted by one position (exclusive prefix)
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const long long uf = __shfl_up_sync(kFull, f, off), ub = __shfl_up_sync(kFull, b, off);
        if (lane >= off) {
          f += uf;
          b += ub;
        }
      }
      if (q + 1 < m) {
        a.F[q + 1] = cf + f;
        a.B[q + 1] = cb + b;
      }
      cf += __shfl_sync(kFull, f, 31);
      cb += __shfl_sync(kFull, b, 31);
    }
    __syncwarp();
    if (lane == 0) {
      a.F[0] = 0;
      a.B[0] = 0;
      a.F[m] = (m > 1 ? a.F[m - 1] : 0) + dfull<T16>(X, (int)sol[m - 1], (int)sol[0]);
    }
  }
  G.sync();
}

struct Piece {
  int s, e, r;  // positions s .. e of the current tour, traversed backward when r
};
constexpr int kMaxPieces = 16;

// cut the piece holding virtual position x (0 < x < len) so that a piece starts there
__device__ __forceinline__ void piece_split(Piece *pc, int &np, int x) {
  int vs = 0;
  for (int i = 0; i < np; ++i) {
    const int L = pc[i].e - pc[i].s + 1;
    if (x > vs && x < vs + L) {
      for (int j = np; j > i + 1; --j) pc[j] = pc[j - 1];
      const int c = x - vs;  // elements of the first part
      Piece a = pc[i], b = pc[i];
      if (!pc[i].r) {
        a.e = a.s + c - 1;
        b.s = a.s + c;
      } else {
        a.s = pc[i].e - c + 1;  // backward: the first part is the top c positions
        b.e = pc[i].e - c;
      }
      pc[i] = a;
      pc[i + 1] = b;
      ++np;
      return;
    }
    vs += L;
  }
}

// the pieces after one cut-and-reorder move P0 A M B P4 -> P0 B M A' P4
__device__ void piece_move(Piece *pc, int &np, const PMove &mv, int m) {
  const int cuts[4] = {mv.b1, mv.b2, mv.b3, mv.b4};
#pragma unroll
  for (int t = 0; t < 4; ++t)
    if (cuts[t] > 0 && cuts[t] < m) piece_split(pc, np, cuts[t]);
  int cls[kMaxPieces];
  int vs = 0;
  for (int i = 0; i < np; ++i) {
    cls[i] = vs < mv.b1 ? 0 : (vs < mv.b2 ? 1 : (vs < mv.b3 ? 2 : (vs < mv.b4 ? 3 : 4)));
    vs += pc[i].e - pc[i].s + 1;
  }
  Piece out[kMaxPieces];
  int no = 0;
  const int order[5] = {0, 3, 2, 1, 4};
#pragma unroll
  for (int o = 0; o < 5; ++o) {
    const int c = order[o];
    const bool flip = c == 1 && mv.rev;
    for (int t = 0; t < np; ++t) {
      const int i = flip ? np - 1 - t : t;
      if (cls[i] != c) continue;
      out[no] = pc[i];
      if (flip) out[no].r ^= 1;
      ++no;
    }
  }
  for (int i = 0; i < no; ++i) pc[i] = out[i];
  np = no;
}

// delta of the k-step candidate: cost of the new cyclic tour minus F[len]
template <bool T16>
__device__ long long atsp_delta(const View &X, const PermEl *sol, const TsAux &a, const CandMoves &cm,
                                int k) {
  const int m = X.len;
  Piece pc[kMaxPieces];
  int np = 1;
  pc[0] = Piece{0, m - 1, 0};
  for (int t = 0; t < k; ++t) piece_move(pc, np, cm.m[t], m);
  long long total = 0;
  for (int i = 0; i < np; ++i) {
    const Piece p = pc[i], q = pc[i + 1 < np ? i + 1 : 0];
    total += p.r ? a.B[p.e] - a.B[p.s] : a.F[p.e] - a.F[p.s];
    total += dfull<T16>(X, (int)sol[p.r ? p.s : p.e], (int)sol[q.r ? q.e : q.s]);
  }
  return total - a.F[m];
}

// rebuild a member's cache after its solution changed (CVRPTW's route
// cache, ATSP's edge-cost prefix sums; nothing for the other models)
template <int MODEL, class El, class G_t>
__device__ __forceinline__ void model_aux_build(const View &X, const El *sol, unsigned char *auxp,
                                                int len, const G_t &G) {
  if constexpr (MODEL == CVRPTW) {
    cv_build(X, sol, cv_aux_at(auxp, len, X.wl > 0), G);
  } else if constexpr (MODEL == ATSP) {
    if (X.t16) ts_build<true>(X, sol, ts_aux_at(auxp, len), G);
    else ts_build<false>(X, sol, ts_aux_at(auxp, len), G);
  }
}

// ------------------------------------------------- candidate evaluation
// The three steps of a TSP candidate, evaluated in phases across the steps
// (positions, inverse maps, solution loads, triangle gathers, sums) so that
// independent work is adjacent in program order.  With the int16 triangle
// every junction sum fits comfortably in 32 bits.
template <bool T16>
__device__ __forceinline__ long long tsp_three_steps(const View &X, const PermEl *sol,
                                                     const CandMoves &cm, int k) {
  using Acc = typename std::conditional<T16, int, long long>::type;
  const int m = X.len;
  int pos[3][8];
  bool rev[3], mn[3], remp[3];
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    const PMove &mv = cm.m[t];
    rev[t] = mv.rev != 0;
    mn[t] = mv.b3 > mv.b2;
    remp[t] = (mv.b1 == 0) && (mv.b4 == m);
    pos[t][0] = mv.b1 == 0 ? m - 1 : mv.b1 - 1;  // r_l
    pos[t][1] = mv.b4 == m ? 0 : mv.b4;          // r_f
    pos[t][2] = mv.b1;                           // A_f
    pos[t][3] = mv.b2 - 1;                       // A_l
    pos[t][4] = min(mv.b3, m - 1);               // B_f
    pos[t][5] = max(mv.b4 - 1, 0);               // B_l
    pos[t][6] = min(mv.b2, m - 1);               // M_f
    pos[t][7] = max(mv.b3 - 1, 0);               // M_l
  }
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    pos[1][e] = perm_inv(cm.m[0], pos[1][e]);
    pos[2][e] = perm_inv(cm.m[0], perm_inv(cm.m[1], pos[2][e]));
  }
  int v[3][8];
#pragma unroll
  for (int t = 0; t < 3; ++t)
#pragma unroll
    for (int e = 0; e < 8; ++e) v[t][e] = sol[pos[t][e]];
  // gather pairs: (rl,x1) (y2,rf) (rl,af) (z4,rf) (bl,mf|af) (ml,af) (al,mf|bf) (ml,bf).
  // With R empty (the move spans the whole tour) the junctions with R do not
  // exist: pairs 0 and 2 become (al,bf) and (bl,af), pairs 1 and 3 cancel.
  uint32_t idx[3][8];
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    const int rl = v[t][0], rf = v[t][1], af = v[t][2], al = v[t][3], bf = v[t][4], bl = v[t][5],
              mf = v[t][6], ml = v[t][7];
    const bool re = remp[t];
    const int px[8] = {re ? al : rl, rev[t] ? af : al, re ? bl : rl, re ? (rev[t] ? af : al) : (rev[t] ? al : bl),
                       bl, ml, al, ml};
    const int py[8] = {re ? bf : (rev[t] ? al : bf), rf, af, rf, mn[t] ? mf : af, af, mn[t] ? mf : bf, bf};
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int a = min(px[e], py[e]), b = max(px[e], py[e]);
      idx[t][e] = (((uint32_t)a * (uint32_t)(X.n2m1 - a)) >> 1) + (uint32_t)b;
    }
  }
  Acc dv[3][8];
#pragma unroll
  for (int t = 0; t < 3; ++t)
#pragma unroll
    for (int e = 0; e < 8; ++e)
      dv[t][e] = T16 ? (Acc)((const int16_t *)X.tri)[idx[t][e]] : (Acc)((const int32_t *)X.tri)[idx[t][e]];
  long long total = 0;
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    const Acc mid_n = dv[t][4] + (mn[t] ? dv[t][5] : (Acc)0);
    const Acc mid_o = dv[t][6] + (mn[t] ? dv[t][7] : (Acc)0);
    Acc d = dv[t][0] + dv[t][1] - dv[t][2] - dv[t][3] + (rev[t] ? (Acc)0 : mid_n - mid_o);
    // R empty: a reversal or an exchange of two pieces is a rotation of the
    // cycle (no change); three pieces B M A change three junctions
    d = (remp[t] && (rev[t] || !mn[t])) ? (Acc)0 : d;
    total += (t < k) ? (long long)d : 0ll;
  }
  return total;
}

// ------------------------------------------------- row level [R31, R32]
// The rows of CVRPTW's separator sequence are its V routes: route r spans
// [b_r, e_r), b_0 = 0, e_r = the r-th separator's position (e_(V-1) = len),
// b_r = e_(r-1) + 1.  Each row operator is a cut-and-reorder move once the
// bounds of the routes it names are known: row_swap exchanges two routes'
// contents (P0 B M A P4 with A, B the routes), row_merge and row_split move
// one separator (an insertion).
struct RouteBounds {
  int b[2], e[2];  // the routes the operator names
  int z, zb, ze;   // the lowest-index empty route (z = -1 if none) and its bounds
};

// element i removed and re-inserted so that it lands at index j
__device__ __forceinline__ PMove insert_move(int i, int j) {
  return i < j ? PMove{i, i + 1, i + 1, j + 1, 0} : PMove{j, i, i, i + 1, 0};
}

// the routes a row operator (local 5 swap, 6 merge, 7 split) names
__device__ __forceinline__ void row_routes(int op, uint32_t r1, int V, int &ra, int &rb) {
  const uint32_t a = r1 >> 16, b = r1 & 0xFFFFu;
  if (op == 5) {
    const int x = posm(a, (uint32_t)V);
    int y = posm(b, (uint32_t)(V - 1));
    y += (y >= x);
    ra = min(x, y);
    rb = max(x, y);
  } else if (op == 6) {
    ra = posm(a, (uint32_t)(V - 1));
    rb = ra + 1;
  } else {
    ra = posm(a, (uint32_t)V);
    rb = -1;
  }
}

__device__ __forceinline__ PMove row_move(int op, uint32_t r1, int V, const RouteBounds &S) {
  if (op == 5) return PMove{S.b[0], S.e[0], S.b[1], S.e[1], 0};
  if (op == 6) return insert_move(S.e[0], S.e[1] - 1);
  const int c = S.e[0] - S.b[0];
  if (c >= 2 && S.z >= 0) {
    const int k = 1 + posm(r1 & 0xFFFFu, (uint32_t)(c - 1));
    // the separator that closes the empty route (opens it, for the last one)
    const int from = S.z < V - 1 ? S.ze : S.zb - 1;
    const int gap = S.b[0] + k;  // it goes before the element now at gap
    return insert_move(from, from < gap ? gap - 1 : gap);
  }
  return PMove{0, 0, 0, 0, 0};  // nothing to split: identity
}

// bounds on the actual sequence, from the route cache
__device__ __forceinline__ RouteBounds row_bounds_cached(const CvAux &a, int len, int V, int ra,
                                                         int rb) {
  auto bb = [&](int r) { return r == 0 ? 0 : a.sep[r - 1] + 1; };
  auto ee = [&](int r) { return r == V - 1 ? len : a.sep[r]; };
  RouteBounds S;
  S.b[0] = bb(ra);
  S.e[0] = ee(ra);
  S.b[1] = rb >= 0 ? bb(rb) : 0;
  S.e[1] = rb >= 0 ? ee(rb) : 0;
  S.z = a.sep[len];
  S.zb = S.z >= 0 ? bb(S.z) : 0;
  S.ze = S.z >= 0 ? ee(S.z) : 0;
  return S;
}

// bounds on the sequence as earlier steps left it (position q holds Vq(q)):
// one pass over the positions
template <class Look>
__device__ RouteBounds row_bounds_scan(Look Vq, int n, int len, int ra, int rb) {
  RouteBounds S;
  S.b[0] = S.e[0] = S.b[1] = S.e[1] = 0;
  S.z = -1;
  S.zb = S.ze = 0;
  int r = 0, start = 0;
  for (int q = 0; q <= len; ++q) {
    if (q < len && Vq(q) < n) continue;
    // route r spans [start, q)
    if (r == ra) {
      S.b[0] = start;
      S.e[0] = q;
    }
    if (r == rb) {
      S.b[1] = start;
      S.e[1] = q;
    }
    if (S.z < 0 && q == start) {
      S.z = r;
      S.zb = start;
      S.ze = q;
    }
    ++r;
    start = q + 1;
  }
  return S;
}

// Delta of a CVRPTW candidate of k >= 2 steps on the actual sequence: the
// routes over the hull of the moves' ranges, walked in the final sequence
// (position q of it holds sol[inv_1(.. inv_k(q))]), minus their cached cost.
__device__ long long cvrptw_composite(const View &X, const PermEl *sol, const CandMoves &cm,
                                      const CvAux &a) {
  const int k = cm.k;
  int lo = min(cm.m[0].b1, cm.m[1].b1), hi = max(cm.m[0].b4, cm.m[1].b4);
  if (k >= 3) {
    lo = min(lo, cm.m[2].b1);
    hi = max(hi, cm.m[2].b4);
  }
  const int L = lo > 0 ? a.prv[lo - 1] + 1 : 0;
  const int R = a.nxt[hi];
  const long long old = a.cum[R + 1] - a.cum[L];
  auto Vf = [&](int q) {
    if (k >= 3) q = perm_inv(cm.m[2], q);
    q = perm_inv(cm.m[1], q);
    return (int)sol[perm_inv(cm.m[0], q)];
  };
  if (X.wl > 0) {
    long long mx = max(a.pmx[L], a.smx[R + 1]);
    const long long nw = cvrptw_routes(X, Vf, L, R, X.cv32, Jumps(), &mx);
    return nw - old + X.wl * (mx - a.pmx[X.len + 1]);
  }
  return cvrptw_routes(X, Vf, L, R, X.cv32) - old;
}

// [R37] CVRPTW's lexicographic key from a packed route cost: the fields
// (distance, vehicles used, longest route, penalty from the top) are read
// back and each prioritised objective goes in as its bucket, in mixed radix
__device__ __forceinline__ long long lex_key(const KInst &K, long long P) {
  const unsigned long long u = (unsigned long long)P;
  const int a = K.lex_sh[0], b = K.lex_sh[1], c = K.lex_sh[2];
  const long long o[3] = {(long long)(u & ((1ull << a) - 1ull)),
                          (long long)((u >> a) & ((1ull << (b - a)) - 1ull)),
                          (long long)((u >> b) & ((1ull << (c - b)) - 1ull))};
  long long key = (long long)(u >> c);
  for (int i = 0; i < K.lex_n; ++i) key = key * K.lex_R[i] + o[K.lex_obj[i]] / K.lex_w[i];
  return key;
}

// CVRPTW candidate.  One step: from the route cache; k steps: every changed
// position lies in the hull of the moves' ranges (a move permutes only inside
// its own range), so the routes over that hull are walked once in the final
// sequence against their cached old cost.  With `defer` set, a candidate
// whose walk may be long is not evaluated and its class is returned (0: it
// was evaluated): 1 for k >= 2 steps (the hull of the moves), 2 and 3 for one
// step whose routes over [L, R] are walked whole (a reversal, or any move
// with the longest-route objective) at more than kWalkDefer positions,
// 2 above kWalkLong.  A warp then evaluates its long candidates together,
// the longest first, instead of paying its longest walk in every slot.
constexpr int kWalkDefer = 24, kWalkLong = 64;

__device__ __forceinline__ int candidate_cvrptw(const View &X, const PermEl *sol,
                                                const Weights<Enc<CVRPTW>::NO> &W, uint32_t c,
                                                uint32_t p, uint32_t g, bool defer, long long &d,
                                                uint32_t &rec, CandMoves &cm, const CvAux &aux) {
  const uint4 R0 = philox(ctr_word(c, 0, kKindMove), X.tag, p, g, X.k0, X.k1);
  const int k = 1 + wpick(W.ck, W.Wk, R0.w);
  if (defer && k >= 2) return 1;
  int ops[3] = {-1, -1, -1};
  cm.k = k;
  cm.m[1] = cm.m[2] = PMove{0, 0, 0, 0, 0};
  const int V = X.len - X.n + 1;
  ops[0] = wpick(W.cop, W.Wop, R0.x);
  if (ops[0] >= 5) {
    int ra, rb;
    row_routes(ops[0], R0.y, V, ra, rb);
    cm.m[0] = row_move(ops[0], R0.y, V, row_bounds_cached(aux, X.len, V, ra, rb));
  } else {
    cm.m[0] = X.t3 ? perm_decode<true>(ops[0], R0.y, R0.z, X.len)
                   : perm_decode<false>(ops[0], R0.y, R0.z, X.len);
  }
  if (k == 1) {
    if (defer && (cm.m[0].rev || X.wl > 0)) {
      const int L = cm.m[0].b1 > 0 ? aux.prv[cm.m[0].b1 - 1] + 1 : 0;
      const int w = aux.nxt[cm.m[0].b4] - L + 1;
      if (w > kWalkDefer) return w > kWalkLong ? 2 : 3;
    }
    d = cvrptw_step0(X, sol, cm.m[0], aux);
  } else {
#pragma unroll
    for (int t = 1; t < 3; ++t) {
      if (t < k) {
        const uint4 R = philox(ctr_word(c, (uint32_t)t, kKindMove), X.tag, p, g, X.k0, X.k1);
        ops[t] = wpick(W.cop, W.Wop, R.x);
        if (ops[t] >= 5) {
          // the routes of the sequence as the earlier steps left it
          int ra, rb;
          row_routes(ops[t], R.y, V, ra, rb);
          auto Vq = [&](int q) {
            if (t == 2) q = perm_inv(cm.m[1], q);
            return (int)sol[perm_inv(cm.m[0], q)];
          };
          cm.m[t] = row_move(ops[t], R.y, V, row_bounds_scan(Vq, X.n, X.len, ra, rb));
        } else {
          cm.m[t] = X.t3 ? perm_decode<true>(ops[t], R.y, R.z, X.len)
                         : perm_decode<false>(ops[t], R.y, R.z, X.len);
        }
      }
    }
    d = cvrptw_composite(X, sol, cm, aux);
  }
  if (X.ki->lex_n > 0) {
    // the change of the key: the packed cost of the current routes is in the cache
    const long long cur = aux.cum[X.len + 1] + (X.wl > 0 ? X.wl * aux.pmx[X.len + 1] : 0ll);
    d = lex_key(*X.ki, cur + d) - lex_key(*X.ki, cur);
  }
  rec = stats_record(ops[0], ops[1], ops[2], k, d < 0);
  return 0;
}

// Candidate c: all three steps are drawn and decoded, and the delta of every
// step is computed (each needs only the decoded earlier moves, not their
// deltas), so the steps overlap; k selects how many count.
template <int MODEL, bool T16>
__device__ __forceinline__ long long candidate_perm(const View &X, const PermEl *sol,
                                                    const Weights<Enc<MODEL>::NO> &W, uint32_t c,
                                                    uint32_t p,
                                                    uint32_t g, uint32_t &rec, CandMoves &cm,
                                                    const CvAux &aux) {
  if constexpr (MODEL == CVRPTW) {
    long long d = 0;
    candidate_cvrptw(X, sol, W, c, p, g, false, d, rec, cm, aux);
    return d;
  }
  if constexpr (MODEL == ATSP) {
    // the k steps' moves, then the tour they give as pieces of this one
    const uint4 R0 = philox(ctr_word(c, 0, kKindMove), X.tag, p, g, X.k0, X.k1);
    const int k = 1 + wpick(W.ck, W.Wk, R0.w);
    int ops[3] = {-1, -1, -1};
    cm.k = k;
    cm.m[1] = cm.m[2] = PMove{0, 0, 0, 0, 0};
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      if (t < k) {
        const uint4 R = t == 0 ? R0 : philox(ctr_word(c, (uint32_t)t, kKindMove), X.tag, p, g, X.k0, X.k1);
        ops[t] = wpick(W.cop, W.Wop, R.x);
        cm.m[t] = X.t3 ? perm_decode<true>(ops[t], R.y, R.z, X.len)
                       : perm_decode<false>(ops[t], R.y, R.z, X.len);
      }
    }
    const long long d = atsp_delta<T16>(X, sol, ts_aux_at((unsigned char *)aux.cum, X.len), cm, k);
    rec = stats_record(ops[0], ops[1], ops[2], k, d < 0);
    return d;
  }
  if constexpr (MODEL == QAP) {
    // O(n) deltas: evaluate only the k steps that count
    const uint4 R0 = philox(ctr_word(c, 0, kKindMove), X.tag, p, g, X.k0, X.k1);
    const int k = 1 + wpick(W.ck, W.Wk, R0.w);
    int ops[3] = {-1, -1, -1};
    long long d = 0;
    cm.k = k;
    cm.m[1] = cm.m[2] = PMove{0, 0, 0, 0, 0};
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      if (t < k) {
        const uint4 R = t == 0 ? R0 : philox(ctr_word(c, (uint32_t)t, kKindMove), X.tag, p, g, X.k0, X.k1);
        ops[t] = wpick(W.cop, W.Wop, R.x);
        cm.m[t] = X.t3 ? perm_decode<true>(ops[t], R.y, R.z, X.len)
                       : perm_decode<false>(ops[t], R.y, R.z, X.len);
        d += ops[t] == SWAP ? qap_step(X, sol, cm.m[t], cm.m[0], cm.m[1], t)
                            : qap_block_step(X, sol, cm.m[t], cm.m[0], cm.m[1], t);
      }
    }
    rec = stats_record(ops[0], ops[1], ops[2], k, d < 0);
    return d;
  }
  uint4 R0, R1, R2;
  philox3(ctr_word(c, 0, kKindMove), ctr_word(c, 1, kKindMove), ctr_word(c, 2, kKindMove), X.tag,
          p, g, X.k0, X.k1, R0, R1, R2);
  const int k = 1 + wpick(W.ck, W.Wk, R0.w);
  const int op0 = wpick(W.cop, W.Wop, R0.x);
  const int op1 = wpick(W.cop, W.Wop, R1.x);
  const int op2 = wpick(W.cop, W.Wop, R2.x);
  if (X.t3) {
    cm.m[0] = perm_decode<true>(op0, R0.y, R0.z, X.len);
    cm.m[1] = perm_decode<true>(op1, R1.y, R1.z, X.len);
    cm.m[2] = perm_decode<true>(op2, R2.y, R2.z, X.len);
  } else {
    cm.m[0] = perm_decode<false>(op0, R0.y, R0.z, X.len);
    cm.m[1] = perm_decode<false>(op1, R1.y, R1.z, X.len);
    cm.m[2] = perm_decode<false>(op2, R2.y, R2.z, X.len);
  }
  cm.k = k;
  const long long d = tsp_three_steps<T16>(X, sol, cm, k);
  rec = stats_record(op0, k >= 2 ? op1 : -1, k >= 3 ? op2 : -1, k, d < 0);
  return d;
}

// Knapsack with the flip alone: k flips on x (a flip of an index flipped
// earlier in the same candidate undoes it); delta from the running
// weight/value sums.
__device__ long long candidate_knap_flip(const View &X, const ByteEl *x, const Weights<2> &W,
                                         long long W0, long long V0, uint32_t c, uint32_t p,
                                         uint32_t g, uint32_t &rec) {
  const uint4 R0 = philox(ctr_word(c, 0, kKindMove), X.tag, p, g, X.k0, X.k1);
  const int k = 1 + wpick(W.ck, W.Wk, R0.w);
  long long Wt = W0, Vt = V0;
  int i0 = -1, i1 = -1;
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    if (t < k) {
      const uint4 R = t == 0 ? R0 : philox(ctr_word(c, t, kKindMove), X.tag, p, g, X.k0, X.k1);
      const int i = posm(R.y >> 16, (uint32_t)X.n);
      const int xi = x[i] ^ (int)(i == i0) ^ (int)(i == i1);
      const long long wi = X.w[i], vi = X.v[i];
      Wt += xi ? -wi : wi;
      Vt += xi ? -vi : vi;
      if (t == 0) i0 = i;
      else if (t == 1) i1 = i;
    }
  }
  const long long d = (-Vt + X.lam0 * overp(Wt - X.cap)) - (-V0 + X.lam0 * overp(W0 - X.cap));
  rec = stats_record(0, k >= 2 ? 0 : -1, k >= 3 ? 0 : -1, k, d < 0);
  return d;
}

// Knapsack with seg_flip enabled: k flips or segment flips on x (an element an
// earlier step of the same candidate covered is read with that flip applied).
__device__ long long candidate_knap_seg(const View &X, const ByteEl *x, const Weights<2> &W,
                                        long long W0, long long V0, uint32_t c, uint32_t p,
                                        uint32_t g, uint32_t &rec) {
  const uint4 R0 = philox(ctr_word(c, 0, kKindMove), X.tag, p, g, X.k0, X.k1);
  const int k = 1 + wpick(W.ck, W.Wk, R0.w);
  long long Wt = W0, Vt = V0;
  int s0 = 0, e0 = 0, s1 = 0, e1 = 0;  // [start, end) of steps 0 and 1
  int op[3] = {0, 0, 0};
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    if (t < k) {
      const uint4 R = t == 0 ? R0 : philox(ctr_word(c, t, kKindMove), X.tag, p, g, X.k0, X.k1);
      op[t] = wpick(W.cop, W.Wop, R.x);
      const int L = seg_len(op[t], R.z, X.n);
      const int i = posm(R.y >> 16, (uint32_t)(X.n - L + 1));
#pragma unroll
      for (int e = 0; e < kSegMax; ++e) {
        if (e < L) {
          const int q = i + e;
          const int xi = x[q] ^ (int)(t >= 1 && q >= s0 && q < e0) ^ (int)(t >= 2 && q >= s1 && q < e1);
          const long long wi = X.w[q], vi = X.v[q];
          Wt += xi ? -wi : wi;
          Vt += xi ? -vi : vi;
        }
      }
      if (t == 0) {
        s0 = i;
        e0 = i + L;
      } else if (t == 1) {
        s1 = i;
        e1 = i + L;
      }
    }
  }
  const long long d = (-Vt + X.lam0 * overp(Wt - X.cap)) - (-V0 + X.lam0 * overp(W0 - X.cap));
  rec = stats_record(op[0], k >= 2 ? op[1] : -1, k >= 3 ? op[2] : -1, k, d < 0);
  return d;
}

__device__ __forceinline__ long long candidate_knap(const View &X, const ByteEl *x,
                                                    const Weights<2> &W, long long W0, long long V0,
                                                    uint32_t c, uint32_t p, uint32_t g,
                                                    uint32_t &rec) {
  return X.seg ? candidate_knap_seg(X, x, W, W0, V0, c, p, g, rec)
               : candidate_knap_flip(X, x, W, W0, V0, c, p, g, rec);
}

// GAP with the random reset alone: k resets of a job's agent; loads of
// touched agents tracked through small override lists.
__device__ long long candidate_gap_reset(const View &X, const ByteEl *x, const long long *loads,
                                         const Weights<2> &W, uint32_t c, uint32_t p, uint32_t g,
                                         uint32_t &rec) {
  const uint4 R0 = philox(ctr_word(c, 0, kKindMove), X.tag, p, g, X.k0, X.k1);
  const int k = 1 + wpick(W.ck, W.Wk, R0.w);
  const int n = X.n, m = X.m;
  int xj[2] = {-1, -1}, xv[2] = {0, 0};
  int la[4] = {-1, -1, -1, -1};
  long long lv[4] = {0, 0, 0, 0};
  long long d = 0;
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    if (t < k) {
      const uint4 R = t == 0 ? R0 : philox(ctr_word(c, t, kKindMove), X.tag, p, g, X.k0, X.k1);
      const int j = posm(R.y >> 16, (uint32_t)n);
      const int dd = 1 + posm(R.y & 0xFFFFu, (uint32_t)(m - 1));
      int ao = x[j];
#pragma unroll
      for (int q = 0; q < 2; ++q)
        if (q < t && xj[q] == j) ao = xv[q];
      const int an = (ao + dd) % m;
      long long Lo = loads[ao], Ln = loads[an];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (q < 2 * t && la[q] == ao) Lo = lv[q];
        if (q < 2 * t && la[q] == an) Ln = lv[q];
      }
      const long long ro = X.gr[(size_t)ao * n + j], rn = X.gr[(size_t)an * n + j];
      const long long co = X.gcap[ao], cn = X.gcap[an];
      d += (long long)X.gc[(size_t)an * n + j] - X.gc[(size_t)ao * n + j];
      d += X.lam0 * (overp(Lo - ro - co) - overp(Lo - co) + overp(Ln + rn - cn) - overp(Ln - cn));
      if (t < 2) {
        xj[t] = j;
        xv[t] = an;
        la[2 * t] = ao;
        lv[2 * t] = Lo - ro;
        la[2 * t + 1] = an;
        lv[2 * t + 1] = Ln + rn;
      }
    }
  }
  rec = stats_record(0, k >= 2 ? 0 : -1, k >= 3 ? 0 : -1, k, d < 0);
  return d;
}

// GAP with seg_reset enabled: k steps, each a random reset of one job or of a segment of jobs by one
// offset [R28].  The move is taken as its sequence of single-job
// reassignments (steps in order, jobs in index order); the delta is the sum
// of their exact deltas (the costs telescope).  A job's agent before step t
// is its stored agent plus the offsets of the earlier steps covering it; an
// agent's load before a reassignment is its stored load plus the changes of
// the earlier reassignments, found by scanning them.
struct GapSteps {
  int s0, s1, s2, l0, l1, l2, d0, d1, d2;  // start, length, offset of each step
  __device__ __forceinline__ int agent_before(const ByteEl *x, int j, int t, int m) const {
    int a = x[j] + ((t >= 1 && j >= s0 && j < s0 + l0) ? d0 : 0) +
            ((t >= 2 && j >= s1 && j < s1 + l1) ? d1 : 0);
    a -= a >= 2 * m ? 2 * m : 0;
    return a - (a >= m ? m : 0);
  }
  // reassignment u (0 .. l0+l1+l2-1): its step, job and offset
  __device__ __forceinline__ void at(int u, int &t, int &j, int &d) const {
    t = (u >= l0) + (u >= l0 + l1);
    j = t == 0 ? s0 + u : (t == 1 ? s1 + u - l0 : s2 + u - l0 - l1);
    d = t == 0 ? d0 : (t == 1 ? d1 : d2);
  }
};

__device__ long long candidate_gap_seg(const View &X, const ByteEl *x, const long long *loads,
                                       const Weights<2> &W, uint32_t c, uint32_t p, uint32_t g,
                                       uint32_t &rec) {
  const uint4 R0 = philox(ctr_word(c, 0, kKindMove), X.tag, p, g, X.k0, X.k1);
  const int k = 1 + wpick(W.ck, W.Wk, R0.w);
  const int n = X.n, m = X.m;
  GapSteps S{0, 0, 0, 0, 0, 0, 0, 0, 0};
  int op[3] = {0, 0, 0};
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    if (t < k) {
      const uint4 R = t == 0 ? R0 : philox(ctr_word(c, t, kKindMove), X.tag, p, g, X.k0, X.k1);
      op[t] = wpick(W.cop, W.Wop, R.x);
      const int L = seg_len(op[t], R.z, n);
      const int i = posm(R.y >> 16, (uint32_t)(n - L + 1));
      const int dd = 1 + posm(R.y & 0xFFFFu, (uint32_t)(m - 1));
      if (t == 0) { S.s0 = i; S.l0 = L; S.d0 = dd; }
      else if (t == 1) { S.s1 = i; S.l1 = L; S.d1 = dd; }
      else { S.s2 = i; S.l2 = L; S.d2 = dd; }
    }
  }
  long long d = 0;
  const int V = S.l0 + S.l1 + S.l2;
  // the reassignments already taken: job << 16 | new agent << 8 | old agent
  // (both loops unrolled so that the array stays in registers)
  uint32_t done[3 * kSegMax];
#pragma unroll
  for (int u = 0; u < 3 * kSegMax; ++u) {
    if (u >= V) break;
    int t, j, dd;
    S.at(u, t, j, dd);
    const int ao = S.agent_before(x, j, t, m);
    const int an = ao + dd - (ao + dd >= m ? m : 0);
    long long Lo = loads[ao], Ln = loads[an];
#pragma unroll
    for (int v = 0; v < u; ++v) {
      const uint32_t w = done[v];
      const int bo = (int)(w & 0xFFu), bn = (int)((w >> 8) & 0xFFu), j2 = (int)(w >> 16);
      if (bo == ao) Lo -= X.gr[(size_t)ao * n + j2];
      else if (bn == ao) Lo += X.gr[(size_t)ao * n + j2];
      if (bo == an) Ln -= X.gr[(size_t)an * n + j2];
      else if (bn == an) Ln += X.gr[(size_t)an * n + j2];
    }
    done[u] = (uint32_t)ao | ((uint32_t)an << 8) | ((uint32_t)j << 16);
    const long long ro = X.gr[(size_t)ao * n + j], rn = X.gr[(size_t)an * n + j];
    const long long co = X.gcap[ao], cn = X.gcap[an];
    d += (long long)X.gc[(size_t)an * n + j] - X.gc[(size_t)ao * n + j];
    d += X.lam0 * (overp(Lo - ro - co) - overp(Lo - co) + overp(Ln + rn - cn) - overp(Ln - cn));
  }
  rec = stats_record(op[0], k >= 2 ? op[1] : -1, k >= 3 ? op[2] : -1, k, d < 0);
  return d;
}

__device__ __forceinline__ long long candidate_gap(const View &X, const ByteEl *x,
                                                   const long long *loads, const Weights<2> &W,
                                                   uint32_t c, uint32_t p, uint32_t g,
                                                   uint32_t &rec) {
  return X.seg ? candidate_gap_seg(X, x, loads, W, c, p, g, rec)
               : candidate_gap_reset(X, x, loads, W, c, p, g, rec);
}

// ------------------------------------------------------------ member group
// WPM warps evolve one member together: each evaluates its share of the C
// candidates, partial argmins meet in shared memory behind a named barrier,
// and the winner is applied by the whole group.
struct Group {
  int wpm, gw, grp, tig, nthr;  // warps per member, warp in group, group, thread in group
  __device__ __forceinline__ void sync() const {
    if (wpm == 1) __syncwarp();
    else asm volatile("bar.sync %0, %1;" ::"r"(1 + grp), "r"(nthr) : "memory");
  }
};

// --------------------------------------------------------------- apply
// Materialise one permutation move in place (group-cooperative): positions
// that change are gathered through the inverse map into the scratch array,
// then written back.  Only A and B move when they have equal lengths.
__device__ void perm_materialise(PermEl *sol, PermEl *scr, const PMove &mv, const Group &G) {
  const int la = mv.b2 - mv.b1, lb = mv.b4 - mv.b3;
  const bool ends = !mv.rev && la == lb;
  const int cnt = ends ? 2 * la : mv.b4 - mv.b1;
  for (int e = G.tig; e < cnt; e += G.nthr) {
    const int q = ends ? (e < la ? mv.b1 + e : mv.b3 + (e - la)) : mv.b1 + e;
    scr[q] = sol[perm_inv(mv, q)];
  }
  G.sync();
  for (int e = G.tig; e < cnt; e += G.nthr) {
    const int q = ends ? (e < la ? mv.b1 + e : mv.b3 + (e - la)) : mv.b1 + e;
    sol[q] = scr[q];
  }
  G.sync();
}

template <int NO>
__device__ __forceinline__ int regen_k(const View &X, const Weights<NO> &W, uint32_t c,
                                       uint32_t p, uint32_t g, uint4 &R0) {
  R0 = philox(ctr_word(c, 0, kKindMove), X.tag, p, g, X.k0, X.k1);
  return 1 + wpick(W.ck, W.Wk, R0.w);
}

__device__ void apply_perm(PermEl *sol, PermEl *scr, const CandMoves &cm, const Group &G) {
  for (int t = 0; t < cm.k; ++t) perm_materialise(sol, scr, cm.m[t], G);
}

__device__ void apply_knap(const View &X, ByteEl *x, const Weights<2> &W, uint32_t c,
                           uint32_t p, uint32_t g, const Group &G, long long &aw, long long &av) {
  uint4 R0;
  const int k = regen_k(X, W, c, p, g, R0);
  for (int t = 0; t < k; ++t) {
    const uint4 R = t == 0 ? R0 : philox(ctr_word(c, t, kKindMove), X.tag, p, g, X.k0, X.k1);
    const int L = seg_len(wpick(W.cop, W.Wop, R.x), R.z, X.n);
    const int i = posm(R.y >> 16, (uint32_t)(X.n - L + 1));
    int xs[kSegMax];
#pragma unroll
    for (int e = 0; e < kSegMax; ++e) xs[e] = e < L ? x[i + e] : 0;
    G.sync();
#pragma unroll
    for (int e = 0; e < kSegMax; ++e) {
      if (e < L) {
        if (G.tig == 0) x[i + e] = (ByteEl)(xs[e] ^ 1);
        aw += xs[e] ? -(long long)X.w[i + e] : (long long)X.w[i + e];
        av += xs[e] ? -(long long)X.v[i + e] : (long long)X.v[i + e];
      }
    }
    G.sync();
  }
}

__device__ void apply_gap(const View &X, ByteEl *x, long long *loads, const Weights<2> &W,
                          uint32_t c, uint32_t p, uint32_t g, const Group &G) {
  uint4 R0;
  const int k = regen_k(X, W, c, p, g, R0);
  G.sync();
  if (G.tig == 0) {
    for (int t = 0; t < k; ++t) {
      const uint4 R = t == 0 ? R0 : philox(ctr_word(c, t, kKindMove), X.tag, p, g, X.k0, X.k1);
      const int L = seg_len(wpick(W.cop, W.Wop, R.x), R.z, X.n);
      const int i = posm(R.y >> 16, (uint32_t)(X.n - L + 1));
      const int dd = 1 + posm(R.y & 0xFFFFu, (uint32_t)(X.m - 1));
      for (int j = i; j < i + L; ++j) {
        const int ao = x[j];
        const int an = (ao + dd) % X.m;
        x[j] = (ByteEl)an;
        loads[ao] -= X.gr[(size_t)ao * X.n + j];
        loads[an] += X.gr[(size_t)an * X.n + j];
      }
    }
  }
  G.sync();
}

// auxiliary sums of one member (knapsack W/V, GAP loads), computed by the
// group's first warp and left in shared memory
template <class El>
__device__ void aux_init(int model, const View &X, const El *x, SolScal *sc,
                         long long *loads, const Group &G) {
  const int lane = threadIdx.x & 31;
  if (G.gw == 0) {
    if (model == KNAPSACK) {
      long long W = 0, V = 0;
      for (int i = lane; i < X.n; i += 32)
        if (x[i]) {
          W += X.w[i];
          V += X.v[i];
        }
#pragma unroll
      for (int off = 16; off; off >>= 1) {
        W += __shfl_xor_sync(kFull, W, off);
        V += __shfl_xor_sync(kFull, V, off);
      }
      if (lane == 0) {
        sc->aw = W;
        sc->av = V;
      }
    } else if (model == GAP) {
      for (int a = 0; a < X.m; ++a) {
        long long L = 0;
        for (int j = lane; j < X.n; j += 32)
          if (x[j] == a) L += X.gr[(size_t)a * X.n + j];
#pragma unroll
        for (int off = 16; off; off >>= 1) L += __shfl_xor_sync(kFull, L, off);
        if (lane == 0) loads[a] = L;
      }
    }
  }
  G.sync();
}

// ------------------------------------------------------ window barrier
// All members of the instance arrive (counting members), then wait until
// the arrival count reaches members * (barrier index + 1).  The wait is
// bounded: on timeout (or another warp's error) it raises the error flag and
// returns false so the kernel can exit.  Called by one warp per group.
__device__ bool member_barrier(DevSync *S, uint32_t arrivals, uint32_t target, uint64_t timeout_ns,
                               int lane) {
  __syncwarp();
  int ok = 1;
  if (lane == 0) {
    add_release(&S->arrive, arrivals);
    const uint64_t t0 = global_ns();
    for (;;) {
      if (ld_acquire(&S->arrive) >= target) break;
      if (ld_relaxed(&S->error)) {
        ok = 0;
        break;
      }
      if (global_ns() - t0 > timeout_ns) {
        atomicOr(&S->error, 1u);
        ok = 0;
        break;
      }
      __nanosleep(32);
    }
  }
  ok = __shfl_sync(kFull, ok, 0);
  __syncwarp();
  return ok != 0;
}

__device__ __forceinline__ void cta_bar(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Barrier id of the members of a CTA-local instance (groups use 1..8).
constexpr int kLocalBar = 15;

// group-wide barrier wait: the group's first warp waits, the group follows.
// CTA-local instances (nact > 0) meet at a named barrier of all active threads.
// Ordering: bar.sync orders every thread's prior memory accesses for the
// threads of the CTA (release/acquire at CTA scope), so a CTA-local barrier
// needs no fence; across CTAs the arriving thread adds with release semantics
// at gpu scope (cumulative over what the group's barriers ordered before it)
// and the poller reads with acquire loads.
__device__ bool group_barrier(DevSync *S, uint32_t arrivals, uint32_t target, uint64_t timeout_ns,
                              const Group &G, int *flag, int nact) {
  if (nact > 0) {
    cta_bar(kLocalBar, nact);
    return true;
  }
  G.sync();
  if (G.gw == 0) {
    const bool ok = member_barrier(S, arrivals, target, timeout_ns, threadIdx.x & 31);
    if ((threadIdx.x & 31) == 0) *flag = ok ? 1 : 0;
  }
  G.sync();
  const int ok = *flag;
  G.sync();
  return ok != 0;
}

struct __align__(16) Partial {
  long long d;
  int c, pad;
};

__device__ long long full_cost(const KInst &I, const int32_t *x);

// [R29] the first loads of member p's order crossover at the window ending
// at g (its partner's parent row, positions hi+1+4t .. +3 for group thread t)
__device__ __forceinline__ void cross_first_loads(const KInst &I, const uint4 &R, int p, uint32_t g,
                                                  int tig, int (&el)[4]) {
  const int P = I.P, len = I.len;
  int q = p + 1 + posm(R.y >> 16, (uint32_t)(P - 1));
  q -= q >= P ? P : 0;
  const int i = posm(R.z >> 16, (uint32_t)len);
  int j = posm(R.z & 0xFFFFu, (uint32_t)(len - 1));
  j += j >= i ? 1 : 0;
  const int hi = max(i, j);
  const int32_t *B = I.pool_sol + ((int64_t)P * (1 + (int64_t)((g / I.U) & 1u)) + q) * len;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int idx = 4 * tig + u;
    el[u] = -1;
    if (idx < len) {
      int bi = hi + 1 + idx;
      bi -= bi >= len ? len : 0;
      el[u] = __ldcg(B + bi);
    }
  }
}

// [R29] the crossover parents of a window: each member's best solution as
// it stands at the barrier before the crossovers, in the parent row of the
// window's parity (rows P + b*P + p of the scratch buffer).  The search
// writes a best that it lowers into the coming window's row at once; this
// copies the best in only when the row does not hold it yet (a best changes
// only by decreasing, so its cost identifies it).  A row of parity b is read
// by the crossovers of one window and written again only after the barrier
// of the next window, which every member reaches once its reads are over;
// so no barrier is needed after the crossovers themselves.
__device__ void snapshot_best(const KInst &I, unsigned char *smem, const Layout &Lo, const Group &G,
                              int p0, int mine, int ngroups, uint32_t b) {
  const SolScal *scal = (const SolScal *)(smem + Lo.scal_off);
  long long *snap = (long long *)(smem + Lo.snap_off);
  const int len = I.len;
  for (int e = 0; e < mine; ++e) {
    const int ls = G.grp + e * ngroups, p = p0 + ls;
    const long long bc = scal[ls].best;
    if (snap[2 * ls + (int)b] == bc) continue;
    const int32_t *src = I.bestsol + (int64_t)p * len;
    int32_t *dst = I.pool_sol + ((int64_t)I.P * (1 + (int64_t)b) + p) * len;
    for (int i = G.tig; i < len; i += G.nthr) dst[i] = __ldcg(src + i);
    G.sync();
    if (G.tig == 0) snap[2 * ls + (int)b] = bc;
  }
  G.sync();
}

// [R27] migration at a window end (its two phases and barriers), kept out of
// line so that the generation loop's register allocation does not carry it.
// Returns the number of barriers passed, or -1 when one timed out.
template <int MODEL, int NW>
__device__ __noinline__ int window_migrate(const KInst &I, const View X, unsigned char *smem,
                                           const Layout Lo, const Group G, int p0, int mine,
                                           int ngroups, uint32_t g, uint32_t nb,
                                           uint64_t timeout_ns, int nact, bool more, bool snap) {
  using El = typename SolEl<MODEL>::T;
  const int lane = threadIdx.x & 31, len = I.len, P = I.P;
  DevSync *S = I.sync;
  SolScal *scal = (SolScal *)(smem + Lo.scal_off);
  unsigned char *gmem = smem + Lo.part_off + (int64_t)G.grp * group_bytes(NW);
  int *flag = (int *)(gmem + 2 * NW * sizeof(Partial));
  const uint32_t nb0 = nb;
  // [R27] islands of S consecutive members (Sec. 3.4.3).  Phase 1: every
  // target takes its source's best solution as its current one, in shared
  // memory only, so that all sources are read as they stood at the window
  // end.  Phase 2, after a barrier: bests a migrant improved go to global
  // memory and every member's cost and best are published again.
  const int S_ = P / I.islands;
  const bool ring = I.mstrat == 0 || (I.mstrat == 2 && ((g / I.mperiod) & 1u));
  const int need = ring ? 1 : (int)I.mN;
  const long long *gc = (const long long *)I.cost, *gb = (const long long *)I.best;
  for (int e = 0; e < mine; ++e) {
    const int ls = G.grp + e * ngroups, p = p0 + ls;
    const int isl = p / S_, lo = isl * S_;
    // the member's rank in its island, worst first: (cost desc, index asc)
    const long long cp = ld_relaxed64(gc + p);
    int r = 0;
    for (int q = lo + lane; q < lo + S_; q += 32) {
      const long long cq = ld_relaxed64(gc + q);
      r += (cq > cp || (cq == cp && q < p)) ? 1 : 0;
    }
    r = __reduce_add_sync(kFull, r);
    if (r >= need) continue;
    // its source: ring, the best of the previous island; top-N, the r-th
    // best of the population by (best, index), found by r + 1 successor scans
    long long kb = LLONG_MIN;
    int ki = -1;
    const int qlo = ring ? ((isl + I.islands - 1) % I.islands) * S_ : 0;
    const int qhi = ring ? qlo + S_ : P;
    for (int j = 0; j <= (ring ? 0 : r); ++j) {
      long long bb = LLONG_MAX;
      int be = INT_MAX;
      for (int q = qlo + lane; q < qhi; q += 32) {
        const long long b = ld_relaxed64(gb + q);
        if ((b > kb || (b == kb && q > ki)) && b < bb) {
          bb = b;
          be = q;
        }
      }
      warp_argmin(bb, be);
      kb = bb;
      ki = be;
    }
    El *sol = (El *)(smem + Lo.sol_off + (int64_t)ls * Lo.sol_stride);
    const int32_t *src = I.bestsol + (int64_t)ki * len;
    for (int i = G.tig; i < len; i += G.nthr) sol[i] = (El)__ldcg(src + i);
    G.sync();
    SolScal sc = scal[ls];
    sc.cost = kb;
    sc.best = min(sc.best, kb);
    G.sync();
    if (G.tig == 0) scal[ls] = sc;
    G.sync();
    aux_init(MODEL, X, sol, &scal[ls], (long long *)(smem + Lo.load_off) + (int64_t)ls * X.m, G);
    model_aux_build<MODEL>(X, sol, smem + Lo.aux_off + (int64_t)ls * Lo.aux_stride, len, G);
  }
  if (!group_barrier(S, (uint32_t)mine, (uint32_t)I.members * (nb + 1), timeout_ns, G, flag, nact))
    return -1;
  ++nb;
  for (int e = 0; e < mine; ++e) {
    const int ls = G.grp + e * ngroups, p = p0 + ls;
    if (scal[ls].best < ld_relaxed64(gb + p)) {
      const El *sol = (const El *)(smem + Lo.sol_off + (int64_t)ls * Lo.sol_stride);
      int32_t *dst = I.bestsol + (int64_t)p * len;
      for (int i = G.tig; i < len; i += G.nthr) dst[i] = sol[i];
    }
  }
  G.sync();
  if (G.tig == 0) {
    for (int e = 0; e < mine; ++e) {
      const int ls = G.grp + e * ngroups;
      I.cost[p0 + ls] = scal[ls].cost;
      I.best[p0 + ls] = scal[ls].best;
    }
  }
  // crossovers follow: their parents are the bests after migration
  if (snap) snapshot_best(I, smem, Lo, G, p0, mine, ngroups, (g / I.U) & 1u);
  if (more) {
    if (!group_barrier(S, (uint32_t)mine, (uint32_t)I.members * (nb + 1), timeout_ns, G, flag, nact))
      return -1;
    ++nb;
  }
  return (int)(nb - nb0);
}

// sum of one value over a member group (every thread gets the total)
template <int NW>
__device__ __forceinline__ long long group_sum(long long v, const Group &G, Partial *part) {
#pragma unroll
  for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
  G.sync();
  if ((threadIdx.x & 31) == 0) part[G.gw].d = v;
  G.sync();
  long long t = 0;
#pragma unroll
  for (int w = 0; w < NW; ++w) t += part[w].d;
  G.sync();
  return t;
}

// exact cost of a binary or integer crossover child held in global memory
// (R16), computed by the member group together
template <int MODEL, int NW>
__device__ long long child_cost(const KInst &I, const int32_t *x, const Group &G, Partial *part) {
  const int n = I.n, lane = threadIdx.x & 31;
  static_assert(MODEL == KNAPSACK || MODEL == GAP, "permutation children are costed by perm_cost");
  if constexpr (MODEL == KNAPSACK) {
    long long W = 0, V = 0;
    for (int k = G.tig; k < n; k += G.nthr)
      if (__ldcg(x + k)) {
        W += I.vec0[k];
        V += I.vec1[k];
      }
    W = group_sum<NW>(W, G, part);
    V = group_sum<NW>(V, G, part);
    return -V + I.lam0 * overp(W - I.capacity);
  } else if constexpr (MODEL == GAP) {
    long long s = 0;
    for (int j = G.tig; j < n; j += G.nthr) s += I.mat0[(size_t)__ldcg(x + j) * n + j];
    s = group_sum<NW>(s, G, part);
    // loads: the group's warps take the agents in turn
    long long pen = 0;
    for (int a = G.gw; a < I.m; a += NW) {
      long long L = 0;
      for (int j = lane; j < n; j += 32)
        if (__ldcg(x + j) == a) L += I.mat1[(size_t)a * n + j];
#pragma unroll
      for (int off = 16; off; off >>= 1) L += __shfl_xor_sync(kFull, L, off);
      pen += overp(L - I.vec0[a]);
    }
    // every lane of a warp holds its warp's penalty sum; count it once
    pen = group_sum<NW>(lane == 0 ? pen : 0, G, part);
    return s + I.lam0 * pen;
  }
}

// largest of one value over a member group (every thread gets it)
template <int NW>
__device__ __forceinline__ long long group_max(long long v, const Group &G, Partial *part) {
#pragma unroll
  for (int off = 16; off; off >>= 1) v = max(v, __shfl_xor_sync(kFull, v, off));
  G.sync();
  if ((threadIdx.x & 31) == 0) part[G.gw].d = v;
  G.sync();
  long long t = LLONG_MIN;
#pragma unroll
  for (int w = 0; w < NW; ++w) t = max(t, part[w].d);
  G.sync();
  return t;
}

// exact cost (R16) of a permutation held in shared memory, read through the
// kernel's view of the instance, computed by the member group together;
// CVRPTW's routes are walked in parallel (one thread per route)
template <int MODEL, int NW>
__device__ long long perm_cost(const View &X, const PermEl *x, const Group &G, Partial *part) {
  const int len = X.len;
  long long s = 0;
  if constexpr (MODEL == TSP) {
    for (int k = G.tig; k < len; k += G.nthr) {
      const int a = (int)x[k], b = (int)x[k + 1 == len ? 0 : k + 1];
      const int lo = min(a, b), hi = max(a, b);
      const uint32_t i = (((uint32_t)lo * (uint32_t)(X.n2m1 - lo)) >> 1) + (uint32_t)hi;
      s += X.t16 ? (long long)((const int16_t *)X.tri)[i] : (long long)((const int32_t *)X.tri)[i];
    }
    return group_sum<NW>(s, G, part);
  } else if constexpr (MODEL == ATSP) {
    for (int k = G.tig; k < len; k += G.nthr) {
      const int a = (int)x[k], b = (int)x[k + 1 == len ? 0 : k + 1];
      s += X.t16 ? dfull<true>(X, a, b) : dfull<false>(X, a, b);
    }
    return group_sum<NW>(s, G, part);
  } else if constexpr (MODEL == QAP) {
    const int n = X.n, qs = X.qs;
    for (int i = G.tig; i < n; i += G.nthr) {
      const int32_t *Fi = X.F + (size_t)i * qs, *Dx = X.D + (size_t)x[i] * qs;
      for (int j = 0; j < n; ++j) s += (long long)Fi[j] * (long long)Dx[x[j]];
    }
    return group_sum<NW>(s, G, part);
  } else {
    static_assert(MODEL == CVRPTW, "permutation models only");
    const int n = X.n;
    long long mx = 0;
    for (int q = G.tig; q < len; q += G.nthr) {
      if ((q == 0 || (int)x[q - 1] >= n) && (int)x[q] < n) {
        int e = q + 1;
        while (e < len && (int)x[e] < n) ++e;
        long long rd = 0;
        s += cvrptw_routes(X, [&](int r) { return (int)x[r]; }, q, e, X.cv32, Jumps(),
                           X.wl > 0 ? &rd : nullptr);
        mx = max(mx, rd);
      }
    }
    s = group_sum<NW>(s, G, part);
    if (X.wl > 0) s += X.wl * group_max<NW>(mx, G, part);
    return X.ki->lex_n > 0 ? lex_key(*X.ki, s) : s;
  }
}

// [R29] crossover at a window end, out of line like migration: each member
// crosses, with probability cross_q16 / 2^16, with another member's best as
// it stood before the window's crossovers (its parent row).  A permutation
// child is built and costed in the group's shared scratch row; the others
// in the member's global scratch row.  A best lowered by a child is written
// at once (also into the member's other parent row).  The caller calls it
// only for groups with a member that crosses; it is inlined (an out-of-line
// call saves registers to local memory, which beside a large shared-memory
// instance spills to L2).
template <int MODEL, int NW>
__device__ __forceinline__ void window_cross(const KInst &I, const View X, unsigned char *smem,
                                          const Layout Lo, const Group G, int p0, int mine,
                                          int ngroups, uint32_t g, uint64_t T, uint4 R0,
                                          const int (&el0)[4], bool have_el0) {
  constexpr bool PERM = (MODEL == TSP || MODEL == QAP || MODEL == CVRPTW || MODEL == ATSP);
  using El = typename SolEl<MODEL>::T;
  const int lane = threadIdx.x & 31, len = I.len, P = I.P;
  SolScal *scal = (SolScal *)(smem + Lo.scal_off);
  El *scr = (El *)(smem + Lo.scr_off + (int64_t)G.grp * Lo.scr_stride);
  unsigned char *gmem = smem + Lo.part_off + (int64_t)G.grp * group_bytes(NW);
  Partial *part = (Partial *)gmem;
  const uint32_t b = (g / I.U) & 1u;
  int *wt = (int *)part;  // per-warp counts of the order crossover's compaction
  for (int e = 0; e < mine; ++e) {
    const int ls = G.grp + e * ngroups, p = p0 + ls;
    const uint4 R =
        e == 0 ? R0 : philox(ctr_word(0, 0, kKindCross), X.tag, (uint32_t)p, g, X.k0, X.k1);
    if ((R.x >> 16) >= I.cross_q16) continue;
    int q = p + 1 + posm(R.y >> 16, (uint32_t)(P - 1));
    q -= q >= P ? P : 0;
    const int32_t *B = I.pool_sol + ((int64_t)P * (1 + (int64_t)b) + q) * len;
    El *A = (El *)(smem + Lo.sol_off + (int64_t)ls * Lo.sol_stride);
    long long cc;
    bool took;
    if constexpr (PERM) {
      // order crossover: A[lo..hi] stays; the other positions, from hi+1
      // on (wrapping), take B's elements outside that segment in B's order
      El *child = scr;
      uint32_t *mark = (uint32_t *)((unsigned char *)scr + Lo.sol_stride);  // len bits
      int i = posm(R.z >> 16, (uint32_t)len), j = posm(R.z & 0xFFFFu, (uint32_t)(len - 1));
      j += j >= i ? 1 : 0;
      const int lo = min(i, j), hi = max(i, j);
      // thread t of the group takes B's positions hi+1+c0+4t .. +3 (wrapping):
      // the kept ones go, in order, to the child's positions from hi+1 on.
      // The first chunk's loads are issued before the segment is marked (the
      // first member's by the caller, right after the window barrier).
      int el[4];
      auto load_chunk = [&](int c0) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int idx = c0 + 4 * G.tig + u;
          el[u] = -1;
          if (idx < len) {
            int bi = hi + 1 + idx;
            bi -= bi >= len ? len : 0;
            el[u] = __ldcg(B + bi);
          }
        }
      };
      if (e == 0 && have_el0) {
#pragma unroll
        for (int u = 0; u < 4; ++u) el[u] = el0[u];
      } else {
        load_chunk(0);
      }
      // the bitmask is all zero between crossovers (cleared at the load of
      // the members and after each use)
      for (int k = lo + G.tig; k <= hi; k += G.nthr) {
        const int a = (int)A[k];
        atomicOr(&mark[a >> 5], 1u << (a & 31));
        child[k] = A[k];
      }
      G.sync();
      int base = 0;
      for (int c0 = 0; c0 < len; c0 += 4 * G.nthr) {
        int cnt = 0;
        unsigned km = 0u;
        if (c0 > 0) load_chunk(c0);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int a = el[u];
          if ((unsigned)a < (unsigned)len && !((mark[a >> 5] >> (a & 31)) & 1u)) {
            km |= 1u << u;
            ++cnt;
          }
        }
        int incl = cnt;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
          const int v = __shfl_up_sync(kFull, incl, off);
          if (lane >= off) incl += v;
        }
        if (lane == 31) wt[G.gw] = incl;
        G.sync();
        int off = 0, tot = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
          const int v = wt[w];
          off += w < G.gw ? v : 0;
          tot += v;
        }
        int pos = base + off + incl - cnt;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if ((km >> u) & 1u) {
            int d = hi + 1 + pos;
            d -= d >= len ? len : 0;
            child[d] = (El)el[u];
            ++pos;
          }
        }
        base += tot;
        G.sync();
      }
      for (int k = lo + G.tig; k <= hi; k += G.nthr) mark[(int)child[k] >> 5] = 0u;
      cc = perm_cost<MODEL, NW>(X, child, G, part);
      took = accept_move(cc - scal[ls].cost, T, exp_variate_q32(R.w));
      if (took)
        for (int k = G.tig; k < len; k += G.nthr) A[k] = child[k];
    } else {
      // uniform crossover: element k from B where bit k of the stream is set
      int32_t *child = I.pool_sol + (int64_t)p * len;
      for (int k = G.tig; k < len; k += G.nthr) {
        const uint4 Q = philox(ctr_word((uint32_t)k >> 7, 1, kKindCross), X.tag, (uint32_t)p, g,
                               X.k0, X.k1);
        const int wsel = (k >> 5) & 3;
        const uint32_t w = wsel == 0 ? Q.x : wsel == 1 ? Q.y : wsel == 2 ? Q.z : Q.w;
        child[k] = ((w >> (k & 31)) & 1u) ? __ldcg(B + k) : (int32_t)A[k];
      }
      G.sync();
      cc = child_cost<MODEL, NW>(I, child, G, part);
      took = accept_move(cc - scal[ls].cost, T, exp_variate_q32(R.w));
      if (took)
        for (int k = G.tig; k < len; k += G.nthr) A[k] = (El)__ldcg(child + k);
    }
    if (took) {
      G.sync();
      SolScal sc = scal[ls];
      const bool lowered = cc < sc.best;
      sc.cost = cc;
      sc.best = min(sc.best, cc);
      if (lowered) {
        // the new best to global memory, and into the parent row of the next
        // crossover window (its readers finished before this window's barrier)
        int32_t *dst = I.bestsol + (int64_t)p * len;
        int32_t *pr = I.pool_sol + ((int64_t)P * (2 - (int64_t)b) + p) * len;
        for (int k = G.tig; k < len; k += G.nthr) {
          const int32_t v = (int32_t)A[k];
          dst[k] = v;
          pr[k] = v;
        }
      }
      G.sync();
      if (G.tig == 0) {
        scal[ls] = sc;
        if (lowered) ((long long *)(smem + Lo.snap_off))[2 * ls + (1 - (int)b)] = sc.best;
      }
      G.sync();
      aux_init(MODEL, X, A, &scal[ls], (long long *)(smem + Lo.load_off) + (int64_t)ls * X.m, G);
      model_aux_build<MODEL>(X, A, smem + Lo.aux_off + (int64_t)ls * Lo.aux_stride, len, G);
    }
  }
}

// ---------------------------------------------------------- evolve unit
// XF: the population steps beyond AOS and injection compiled in: 0 none,
// 1 crossover, 2 island migration and crossover.  Solves take the kernels
// with no more of that code than they use, whose generation loop then
// allocates registers alone.
template <int MODEL, bool T16, int WPM, int NS, int XF>
__device__ void evolve_members(const KInst &I, const View &X, unsigned char *smem, const Layout &Lo,
                               int p0, int nsol, int warps, uint64_t timeout_ns) {
  constexpr int NO = Enc<MODEL>::NO;
  constexpr bool PERM = (MODEL == TSP || MODEL == QAP || MODEL == CVRPTW || MODEL == ATSP);
  using El = typename SolEl<MODEL>::T;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // a member group: NS generation slots of WPM warps each (slot s evaluates
  // generation g + s of every step against the same solution)
  constexpr int NW = WPM * NS;
  Group G;
  G.wpm = NW;
  G.gw = wid % NW;
  G.grp = wid / NW;
  G.nthr = NW * 32;
  G.tig = G.gw * 32 + lane;
  const int gslot = G.gw / WPM, gwi = G.gw % WPM;
  const int ngroups = warps / NW;
  const int mine = nsol > G.grp ? (nsol - G.grp + ngroups - 1) / ngroups : 0;
  if (mine == 0) return;
  const int len = I.len, P = I.P, C = I.C;
  DevSync *S = I.sync;
  El *scr = (El *)(smem + Lo.scr_off + (int64_t)G.grp * Lo.scr_stride);
  SolScal *scal = (SolScal *)(smem + Lo.scal_off);
  unsigned char *gmem = smem + Lo.part_off + (int64_t)G.grp * group_bytes(NW);
  Partial *part = (Partial *)gmem;
  int *flag = (int *)(gmem + 2 * NW * sizeof(Partial));
  CandMoves *mvw = (CandMoves *)(gmem + 2 * NW * sizeof(Partial) + 16);
  uint32_t *cnt_smem = (uint32_t *)(gmem + 2 * NW * sizeof(Partial) + 16 + 2 * NW * sizeof(CandMoves));

  // load this group's members (and clear the group's crossover bitmask)
  if constexpr (PERM)
    for (int k = G.tig; k < (len + 31) >> 5; k += G.nthr)
      ((uint32_t *)((unsigned char *)scr + Lo.sol_stride))[k] = 0u;
  for (int e = 0; e < mine; ++e) {
    const int ls = G.grp + e * ngroups, p = p0 + ls;
    El *sol = (El *)(smem + Lo.sol_off + (int64_t)ls * Lo.sol_stride);
    const int32_t *src = I.cur + (int64_t)p * len;
    for (int i = G.tig; i < len; i += G.nthr) sol[i] = (El)src[i];
    if (G.tig == 0) {
      scal[ls].cost = I.cost[p];
      scal[ls].best = I.best[p];
      scal[ls].aw = scal[ls].av = 0;
      long long *snap = (long long *)(smem + Lo.snap_off) + 2 * (int64_t)ls;
      snap[0] = snap[1] = LLONG_MIN;  // the parent rows hold nothing of this launch yet
    }
    G.sync();
    aux_init(MODEL, X, sol, &scal[ls], (long long *)(smem + Lo.load_off) + (int64_t)ls * X.m, G);
    model_aux_build<MODEL>(X, sol, smem + Lo.aux_off + (int64_t)ls * Lo.aux_stride, len, G);
  }

  // instance-wide scalars (identical in every warp)
  // CTA-local instance: every active thread of the CTA takes part in barriers
  const int nact = I.local_sync ? min(ngroups, nsol) * NW * 32 : 0;
  const DevAos *A = I.aos_in;
  uint64_t T = A->T;
  Weights<NO> W;
  uint32_t capl[NO];
  {
    uint32_t wo[NO], wk[3];
#pragma unroll
    for (int l = 0; l < NO; ++l) {
      wo[l] = A->w_op[Enc<MODEL>::glob(l)];
      capl[l] = I.op_cap[Enc<MODEL>::glob(l)];
    }
    wk[0] = A->w_k[0];
    wk[1] = A->w_k[1];
    wk[2] = A->w_k[2];
    weights_set(W, wo, wk);
  }
  uint32_t en_local = 0;
#pragma unroll
  for (int l = 0; l < NO; ++l) en_local |= ((I.enabled >> Enc<MODEL>::glob(l)) & 1u) << l;
  uint32_t stag = A->stag;
  long long elite_prev = A->elite_prev;
  uint32_t pend = lane < kStats ? A->pend[lane] : 0u;
  // the first warp of member 0 keeps the cumulative window counts
  const bool cum_owner = p0 + G.grp == 0 && G.gw == 0;
  if (cum_owner && lane < kStats && I.aos_out != A) I.aos_out->cum[lane] = A->cum[lane];
  // the instance scalars are updated in place by a CTA-local unit: everyone
  // reads them before anyone can write them back
  if (nact > 0) cta_bar(kLocalBar, nact);
  bool pend_used = false;
  uint32_t prev_acc[2] = {0u, 0u};
  uint32_t nb = 0, wi = 0, gpar = 0;
  Stats<NO> st;
  stats_zero(st);
  const int span = WPM * 32;
  const int cpl = (C + span - 1) / span;
  const bool packed = 96ull * (uint64_t)cpl * (uint64_t)I.U * (uint64_t)mine < 65536ull;
  // a member's window counts in bytes while it evolves (PackedStats): a lane
  // counts at most cpl candidates a generation, or 2 cpl where CVRPTW gathers
  // its long candidates over the warp's lanes (in place, then one per round)
  const uint64_t lane_cands =
      (MODEL == CVRPTW && NS == 1 && cpl > 1 && cpl <= 8) ? 2ull * (uint64_t)cpl : (uint64_t)cpl;
  const bool bytec = 3ull * lane_cands * (uint64_t)I.U <= 255ull;
  PackedStats ps{0u, 0u, 0u, 0u, 0u, 0u};
  auto count = [&](uint32_t rec) {
    if (bytec) packed_add<NO>(ps, rec);
    else stats_add(st, rec);
  };

  // generations are below 2^32 (checked on the host), so window arithmetic
  // is 32-bit
  const uint32_t U = (uint32_t)I.U, gend = (uint32_t)I.g_end;
  // acceptance variates of one aligned block of 32 generations, lane q
  // holding generation 32 * eblk + q; kept across windows while the group
  // evolves a single member
  uint64_t Ereg = 0;
  int64_t eblk = -1;
  uint32_t g = (uint32_t)I.g_begin;
  while (g < gend) {
    const uint32_t wend = min(gend, (g / U + 1u) * U);
    const uint64_t Tw = T;
    long long minbest = LLONG_MAX;
    for (int e = 0; e < mine; ++e) {
      const int ls = G.grp + e * ngroups;
      const uint32_t p = (uint32_t)(p0 + ls);
      El *sol = (El *)(smem + Lo.sol_off + (int64_t)ls * Lo.sol_stride);
      long long *loads = (long long *)(smem + Lo.load_off) + (int64_t)ls * X.m;
      const CvAux cva = cv_aux_at(smem + Lo.aux_off + (int64_t)ls * Lo.aux_stride, len, X.wl > 0);
      SolScal sc = scal[ls];
      const long long best0 = sc.best;
      T = Tw;
      if (mine > 1) eblk = -1;
      uint32_t gg = g;
      while (gg < wend) {
        // evaluate: slot s takes generation gg + s (slots past the window idle)
        const uint32_t gm = gg + (uint32_t)gslot;
        // temperatures of the step's generations do not depend on it
        uint64_t Tq[NS + 1];
        Tq[0] = T;
#pragma unroll
        for (int s2 = 0; s2 < NS; ++s2) Tq[s2 + 1] = cool(Tq[s2], I.alpha);
        // largest worsening each generation could accept (with the largest
        // variate): delta * 2^64 < T * Emax  <=>  delta <= hi - (lo == 0)
        long long thr[NS];
#pragma unroll
        for (int s2 = 0; s2 < NS; ++s2) {
          const uint64_t hi = __umul64hi(Tq[s2], kExpVariateMax), lo = Tq[s2] * kExpVariateMax;
          thr[s2] = (long long)(hi - (lo == 0ull ? 1ull : 0ull));
        }
        long long bd = LLONG_MAX;
        int bc = INT_MAX;
        CandMoves cbest;
        // a later slot's counts wait for its generation to be decided (lanes
        // without a candidate hold the empty record)
        uint32_t held = kNoRecord;
        bool done = false;
        if constexpr (MODEL == CVRPTW && NS == 1) {
          if (gm < wend && cpl > 1 && cpl <= 8) {
            // candidates with short walks in place; the long ones (multi-step
            // candidates, long reversals: about a third) gathered over the
            // warp's lanes by class, longest class first, so that the long
            // walks are paid in a few rounds of similar lengths rather than
            // in every slot.  cpack: the class of the lane's candidate in
            // each slot, 2 bits a slot.
            uint32_t cpack = 0u;
            int nl = 0;
#pragma unroll
            for (int slot = 0; slot < 8; ++slot) {
              if (slot < cpl) {
                const int c = slot * span + gwi * 32 + lane;
                int cls = 0;
                if (c < C) {
                  long long d;
                  uint32_t rec;
                  CandMoves cm;
                  cls = candidate_cvrptw(X, sol, W, c, p, gm, true, d, rec, cm, cva);
                  if (cls == 0) {
                    count(rec);
                    if (d < bd || (d == bd && c < bc)) {
                      bd = d;
                      bc = c;
                      cbest = cm;
                    }
                  }
                }
                cpack |= (uint32_t)cls << (2 * slot);
                nl += cls != 0;
              }
            }
            const int n2 = (int)__reduce_add_sync(kFull, (uint32_t)nl);
            for (int base = 0; base < n2; base += 32) {
              // entry i of the gathered list: class 1 first, slots in order,
              // lanes in order within a slot
              const int i = base + lane;
              int c = 0, acc = 0;
#pragma unroll
              for (int q = 1; q <= 3; ++q)
#pragma unroll
                for (int slot = 0; slot < 8; ++slot) {
                  if (slot < cpl) {
                    const uint32_t b = __ballot_sync(kFull, ((cpack >> (2 * slot)) & 3u) == (uint32_t)q);
                    const int cnt = __popc(b);
                    if (i >= acc && i < acc + cnt)
                      c = slot * span + gwi * 32 + (int)__fns(b, 0u, i - acc + 1);
                    acc += cnt;
                  }
                }
              if (i < n2) {
                long long d;
                uint32_t rec;
                CandMoves cm;
                candidate_cvrptw(X, sol, W, c, p, gm, false, d, rec, cm, cva);
                count(rec);
                if (d < bd || (d == bd && c < bc)) {
                  bd = d;
                  bc = c;
                  cbest = cm;
                }
              }
            }
            done = true;
          }
        }
        if (gm < wend && !done) {
          for (int slot = 0; slot < cpl; ++slot) {
            const int c = slot * span + gwi * 32 + lane;
            if (c < C) {
              long long d;
              uint32_t rec;
              CandMoves cm;
              if constexpr (PERM) d = candidate_perm<MODEL, T16>(X, sol, W, c, p, gm, rec, cm, cva);
              else if constexpr (MODEL == KNAPSACK)
                d = candidate_knap(X, sol, W, sc.aw, sc.av, c, p, gm, rec);
              else d = candidate_gap(X, sol, loads, W, c, p, gm, rec);
              if (gslot == 0) count(rec);
              else held = rec;  // NS > 1 runs with one candidate per lane
              if (d < bd || (d == bd && c < bc)) {
                bd = d;
                bc = c;
                if constexpr (PERM) cbest = cm;
              }
            }
          }
        }
        const int mybc = bc;
        warp_argmin(bd, bc);
        // each warp publishes its minimum and (permutations) the moves of the
        // lane that holds it
        Partial *pp = part + gpar * NW;
        CandMoves *mv = mvw + gpar * NW;
        if constexpr (PERM)
          if (mybc == bc && bc != INT_MAX) mv[G.gw] = cbest;
        if constexpr (NW > 1) {
          if (lane == 0) {
            pp[G.gw].d = bd;
            pp[G.gw].c = bc;
          }
        }
        G.sync();
        gpar ^= 1u;
        // every slot's minimum over its warps: all partials read at once
        // (one 16-byte load each), then a pairwise tree
        long long ds[NS];
        int cs[NS], ws[NS];
#pragma unroll
        for (int s2 = 0; s2 < NS; ++s2) {
          ds[s2] = bd;
          cs[s2] = bc;
          ws[s2] = G.gw;
          if constexpr (NW > 1) {
            long long dq[WPM];
            int cq[WPM], wq[WPM];
#pragma unroll
            for (int q = 0; q < WPM; ++q) {
              const int4 v = *reinterpret_cast<const int4 *>(pp + s2 * WPM + q);
              dq[q] = (long long)(((uint64_t)(uint32_t)v.y << 32) | (uint32_t)v.x);
              cq[q] = v.z;
              wq[q] = s2 * WPM + q;
            }
#pragma unroll
            for (int h = 1; h < WPM; h *= 2)
#pragma unroll
              for (int q = 0; q + h < WPM; q += 2 * h)
                if (dq[q + h] < dq[q] || (dq[q + h] == dq[q] && cq[q + h] < cq[q])) {
                  dq[q] = dq[q + h];
                  cq[q] = cq[q + h];
                  wq[q] = wq[q + h];
                }
            ds[s2] = dq[0];
            cs[s2] = cq[0];
            ws[s2] = wq[0];
          }
        }
        // decide generations gg, gg + 1, ... in order; an accepted move ends
        // the step (later slots evaluated the old solution)
        uint32_t adv = 0;
#pragma unroll
        for (int s2 = 0; s2 < NS; ++s2) {
          const uint32_t gs = gg + (uint32_t)s2;
          if (gs >= wend) break;
          const long long d = ds[s2];
          const int c = cs[s2], w = ws[s2];
          if (s2 > 0 && gslot == s2) count(held);
          // the variate is drawn only when it can decide: a worsening move that
          // even the largest variate would reject is rejected without it
          bool acc = d <= 0;
          if (!acc && d <= thr[s2]) {
            if ((int64_t)(gs >> 5) != eblk) {
              eblk = gs >> 5;
              const uint4 Ra = philox(ctr_word(0, 0, kKindAccept), X.tag, p, (gs & ~31u) + lane,
                                      X.k0, X.k1);
              Ereg = exp_variate_q32(Ra.x);
            }
            acc = accept_move(d, Tq[s2], __shfl_sync(kFull, Ereg, gs & 31u));
          }
          T = Tq[s2 + 1];
          adv = (uint32_t)s2 + 1u;
          if (acc) {
            if constexpr (PERM) {
              apply_perm(sol, scr, mv[w], G);
              model_aux_build<MODEL>(X, sol, (unsigned char *)cva.cum, len, G);
            }
            else if constexpr (MODEL == KNAPSACK) apply_knap(X, sol, W, c, p, gs, G, sc.aw, sc.av);
            else apply_gap(X, sol, loads, W, c, p, gs, G);
            sc.cost += d;
            if (sc.cost < sc.best) {
              sc.best = sc.cost;
              int32_t *dst = I.bestsol + (int64_t)p * len;
              for (int i = G.tig; i < len; i += G.nthr) dst[i] = sol[i];
              if constexpr (XF) {
                // [R29] and into the parent row of the coming crossover window
                if (I.cross_q16 > 0) {
                  int32_t *pr =
                      I.pool_sol + ((int64_t)P * (1 + (int64_t)((g / U + 1u) & 1u)) + p) * len;
                  for (int i = G.tig; i < len; i += G.nthr) pr[i] = sol[i];
                }
              }
            }
            break;
          }
        }
        gg += adv;
      }
      if (bytec) packed_flush(st, ps);
      G.sync();
      if (G.tig == 0) {
        scal[ls] = sc;
        if constexpr (XF)
          if (I.cross_q16 > 0 && sc.best < best0)
            ((long long *)(smem + Lo.snap_off))[2 * ls + (int)((g / U + 1u) & 1u)] = sc.best;
      }
      G.sync();
      minbest = min(minbest, sc.best);
    }
    g = wend;
    if (g % U != 0) continue;  // only at the very end of a launch

    // ------------------------------------------------ AOS window end
    const bool inject = I.E > 0 && (g % (uint32_t)I.E) == 0;
    const bool migr = XF == 2 && I.islands > 1 && (g % I.mperiod) == 0;
    const bool cross = XF != 0 && I.cross_q16 > 0;
    uint32_t tot[NO * 2 + 6];
    if (packed) {
      // a lane counts at most 3 * cpl * U * mine uses per window, so the warp
      // totals of a (uses, improvements) pair fit 16 bits each
#pragma unroll
      for (int l = 0; l < NO; ++l) {
        const uint32_t t = __reduce_add_sync(kFull, st.u[l] | (st.v[l] << 16));
        tot[l] = t & 0xFFFFu;
        tot[NO + l] = t >> 16;
      }
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const uint32_t t = __reduce_add_sync(kFull, st.uk[i] | (st.vk[i] << 16));
        tot[2 * NO + i] = t & 0xFFFFu;
        tot[2 * NO + 3 + i] = t >> 16;
      }
    } else {
#pragma unroll
      for (int l = 0; l < NO; ++l) {
        tot[l] = __reduce_add_sync(kFull, st.u[l]);
        tot[NO + l] = __reduce_add_sync(kFull, st.v[l]);
      }
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        tot[2 * NO + i] = __reduce_add_sync(kFull, st.uk[i]);
        tot[2 * NO + 3 + i] = __reduce_add_sync(kFull, st.vk[i]);
      }
    }
    uint32_t my = 0;
#pragma unroll
    for (int l = 0; l < NO; ++l) {
      my = (lane == Enc<MODEL>::glob(l)) ? tot[l] : my;
      my = (lane == kStatV + Enc<MODEL>::glob(l)) ? tot[NO + l] : my;
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      my = (lane == kStatUK + i) ? tot[2 * NO + i] : my;
      my = (lane == kStatVK + i) ? tot[2 * NO + 3 + i] : my;
    }
    const int slot = wi & 1;
    if constexpr (NW > 1) {
      // the group's warps add their counts in shared memory; one warp publishes
      cnt_smem[G.gw * 32 + lane] = my;
      G.sync();
      if (G.gw == 0) {
#pragma unroll
        for (int w = 1; w < NW; ++w) my += cnt_smem[w * 32 + lane];
      }
      G.sync();
    }
    if (G.gw == 0 && lane < kStats && my) atomicAdd(&S->acc[slot][lane], my);
    if (G.gw == 0 && lane == 0) atomicMin((long long *)&S->elite[slot], minbest);
    if ((inject || migr) && G.tig == 0) {
      for (int e = 0; e < mine; ++e) {
        const int ls = G.grp + e * ngroups;
        I.cost[p0 + ls] = scal[ls].cost;
        I.best[p0 + ls] = scal[ls].best;
      }
    }
    // crossover parents (after migration instead, when the window migrates)
    if constexpr (XF)
      if (cross && !migr) snapshot_best(I, smem, Lo, G, p0, mine, ngroups, (g / I.U) & 1u);
    if (!group_barrier(S, (uint32_t)mine, (uint32_t)I.members * (nb + 1), timeout_ns, G, flag, nact))
      return;
    ++nb;
    uint32_t cum = lane < kStats ? ld_relaxed(&S->acc[slot][lane]) : 0u;
    const long long elite = ld_relaxed64((const long long *)&S->elite[slot]);
    // [R29] the members' crossover draws, and the first loads of the first
    // member's parent row (final now unless migration comes first), while
    // the window's totals are on their way
    bool cany = false;
    uint4 cR0 = make_uint4(0u, 0u, 0u, 0u);
    int cel[4] = {-1, -1, -1, -1};
    if constexpr (XF) {
      if (cross) {
        for (int e = 0; e < mine; ++e) {
          const uint4 R = philox(ctr_word(0, 0, kKindCross), X.tag,
                                 (uint32_t)(p0 + G.grp + e * ngroups), g, X.k0, X.k1);
          if (e == 0) cR0 = R;
          cany = cany || (R.x >> 16) < I.cross_q16;
        }
        if constexpr (PERM)
          if (!migr && (cR0.x >> 16) < I.cross_q16)
            cross_first_loads(I, cR0, p0 + G.grp, g, G.tig, cel);
      }
    }
    uint32_t total = cum - prev_acc[slot];
    prev_acc[slot] = cum;
    if (!pend_used) total += pend;
    pend_used = true;
    if (cum_owner && lane < kStats) I.aos_out->cum[lane] += total;
    ++wi;

    uint32_t wo[NO], wk[3];
    weights_get(W, wo, wk);
    aos_update_lanes<Enc<MODEL>>(wo, wk, total, en_local, capl, I.ema_a, I.w_floor, I.w_cap);
    if (elite < elite_prev) stag = 0;
    else ++stag;
    elite_prev = elite;
    if (I.stag_limit > 0 && stag >= I.stag_limit) {
      wk[0] = 52429u;
      wk[1] = 9830u;
      wk[2] = 3277u;
      stag = 0;
    }
    weights_set(W, wo, wk);
    stats_zero(st);

    if constexpr (XF) {
      if constexpr (XF == 2) {
        if (migr) {
          const int nbar = window_migrate<MODEL, NW>(I, X, smem, Lo, G, p0, mine, ngroups, g, nb,
                                                     timeout_ns, nact, inject || cross, cross);
          if (nbar < 0) return;
          nb += (uint32_t)nbar;
        }
      }
      if (cross) {
        // [R29] the crossovers of a group that has a member crossing
        if (cany)
          window_cross<MODEL, NW>(I, X, smem, Lo, G, p0, mine, ngroups, g, T, cR0, cel, !migr);
        if (inject) {
          // injection reads every member's cost and best after the crossovers
          if (G.tig == 0) {
            for (int e = 0; e < mine; ++e) {
              const int ls = G.grp + e * ngroups;
              I.cost[p0 + ls] = scal[ls].cost;
              I.best[p0 + ls] = scal[ls].best;
            }
          }
          if (!group_barrier(S, (uint32_t)mine, (uint32_t)I.members * (nb + 1), timeout_ns, G, flag,
                             nact))
            return;
          ++nb;
        }
      }
    }

    if (inject) {
      // elite = lowest best (lowest index on ties), worst = highest cost
      long long bb = LLONG_MAX, nwc = LLONG_MAX;
      int be = INT_MAX, wq = INT_MAX;
      for (int q = lane; q < P; q += 32) {
        const long long b = ld_relaxed64((const long long *)I.best + q);
        const long long cq = ld_relaxed64((const long long *)I.cost + q);
        if (b < bb) {
          bb = b;
          be = q;
        }
        if (-cq < nwc) {
          nwc = -cq;
          wq = q;
        }
      }
      warp_argmin(bb, be);
      warp_argmin(nwc, wq);
      const int lw = wq - p0;
      if (lw >= 0 && lw < nsol && (lw % ngroups) == G.grp) {
        El *sol = (El *)(smem + Lo.sol_off + (int64_t)lw * Lo.sol_stride);
        const int32_t *src = I.bestsol + (int64_t)be * len;
        for (int i = G.tig; i < len; i += G.nthr) sol[i] = (El)__ldcg(src + i);
        G.sync();
        SolScal sc = scal[lw];
        sc.cost = bb;
        if (bb < sc.best) {
          sc.best = bb;
          int32_t *dst = I.bestsol + (int64_t)wq * len;
          for (int i = G.tig; i < len; i += G.nthr) dst[i] = sol[i];
        }
        G.sync();
        if (G.tig == 0) scal[lw] = sc;
        G.sync();
        aux_init(MODEL, X, sol, &scal[lw], (long long *)(smem + Lo.load_off) + (int64_t)lw * X.m, G);
        model_aux_build<MODEL>(X, sol, smem + Lo.aux_off + (int64_t)lw * Lo.aux_stride, len, G);
      }
      if (!group_barrier(S, (uint32_t)mine, (uint32_t)I.members * (nb + 1), timeout_ns, G, flag, nact))
        return;
      ++nb;
    }
  }

  // ------------------------------------------------ write back
  for (int e = 0; e < mine; ++e) {
    const int ls = G.grp + e * ngroups, p = p0 + ls;
    const El *sol = (const El *)(smem + Lo.sol_off + (int64_t)ls * Lo.sol_stride);
    int32_t *dst = I.cur + (int64_t)p * len;
    for (int i = G.tig; i < len; i += G.nthr) dst[i] = sol[i];
    if (G.tig == 0) {
      I.cost[p] = scal[ls].cost;
      I.best[p] = scal[ls].best;
    }
  }
  // counts of a window left open by this launch
  if (I.g_end % I.U != 0) {
    uint32_t my = 0;
#pragma unroll
    for (int l = 0; l < NO; ++l) {
      const uint32_t tu = __reduce_add_sync(kFull, st.u[l]), tv = __reduce_add_sync(kFull, st.v[l]);
      my = (lane == Enc<MODEL>::glob(l)) ? tu : my;
      my = (lane == kStatV + Enc<MODEL>::glob(l)) ? tv : my;
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const uint32_t tu = __reduce_add_sync(kFull, st.uk[i]), tv = __reduce_add_sync(kFull, st.vk[i]);
      my = (lane == kStatUK + i) ? tu : my;
      my = (lane == kStatVK + i) ? tv : my;
    }
    if (p0 + G.grp == 0 && G.gw == 0 && !pend_used) my += pend;
    if (lane < kStats && my) atomicAdd(&S->pend_out[lane], my);
  }
  if (nact > 0) {
    // CTA-local finalize: elite and the open window's counts
    __threadfence();
    cta_bar(kLocalBar, nact);
    if (p0 + G.grp == 0 && G.gw == 0) {
      long long bb = LLONG_MAX;
      int be = INT_MAX;
      for (int q = lane; q < P; q += 32) {
        const long long b = ld_relaxed64((const long long *)I.best + q);
        if (b < bb) {
          bb = b;
          be = q;
        }
      }
      warp_argmin(bb, be);
      if (lane < kStats) I.aos_out->pend[lane] = ld_relaxed(&S->pend_out[lane]);
      if (lane == 0) {
        I.aos_out->elite = be;
        I.aos_out->elite_cost = bb;
      }
    }
  }
  if (p0 + G.grp == 0 && G.tig == 0) {
    DevAos *O = I.aos_out;
    O->T = T;
    O->g = I.g_end;
    for (int i = 0; i < kNops; ++i) O->w_op[i] = 0;
    uint32_t wo[NO], wk[3];
    weights_get(W, wo, wk);
#pragma unroll
    for (int l = 0; l < NO; ++l) O->w_op[Enc<MODEL>::glob(l)] = wo[l];
    O->w_k[0] = wk[0];
    O->w_k[1] = wk[1];
    O->w_k[2] = wk[2];
    O->stag = stag;
    O->elite_prev = elite_prev;
  }
}

// stage this unit's instance data into shared memory (or point at global)
__device__ View make_view(const KInst &I, unsigned char *smem, bool staged) {
  View X;
  X.n = I.n;
  X.len = I.len;
  X.m = I.m;
  X.cap = I.capacity;
  X.lam0 = I.lam0;
  X.tag = I.tag;
  X.k0 = (uint32_t)I.seed;
  X.k1 = (uint32_t)(I.seed >> 32);
  X.n2m1 = 2 * I.n - 1;
  X.tri = I.tri;
  X.F = I.mat0;
  X.D = I.mat1;
  X.FT = X.DT = nullptr;
  X.qs = I.n;
  X.w = I.vec0;
  X.v = I.vec1;
  X.gc = I.mat0;
  X.gr = I.mat1;
  X.gcap = I.vec0;
  X.rd = I.mat0;
  X.dem = I.vec0;
  X.rdy = I.vec1;
  X.due = I.vec2;
  X.svc = I.vec3;
  X.node = I.node;
  X.cv32 = I.cv32 != 0;
  X.t3 = ((I.enabled >> THREE_OPT) & 1u) != 0;
  X.t16 = I.tri16 != 0;
  X.seg = ((I.enabled >> SEGMENT) & 1u) != 0;
  X.lam1 = I.lam1;
  X.wd = I.wdist;
  X.wv = I.wveh;
  X.wl = I.wlong;
  X.ki = &I;
  if (!staged) return X;
  auto copy = [&](const void *src, int64_t bytes, int64_t off) {
    const int4 *s = (const int4 *)src;
    int4 *d = (int4 *)(smem + off);
    const int64_t n16 = align16(bytes) / 16;
    for (int64_t i = threadIdx.x; i < n16; i += blockDim.x) d[i] = s[i];
    return (const void *)(smem + off);
  };
  switch (I.model) {
    case TSP:
      X.tri = copy(I.tri, (int64_t)I.n * (I.n + 1) / 2 * (I.tri16 ? 2 : 4), 0);
      break;
    case ATSP:
      X.tri = copy(I.tri, (int64_t)I.n * I.n * (I.tri16 ? 2 : 4), 0);
      break;
    case QAP: {
      // rows re-strided to an odd length so that lanes reading different rows
      // at the same column hit different banks
      // (and transposed, so that the column reads of the delta are row reads)
      const int n = I.n, qs = I.n | 1;
      const int64_t b = align16((int64_t)n * qs * 4);
      int32_t *Fs = (int32_t *)smem, *Ds = (int32_t *)(smem + b);
      int32_t *FTs = (int32_t *)(smem + 2 * b), *DTs = (int32_t *)(smem + 3 * b);
      for (int64_t t = threadIdx.x; t < (int64_t)n * n; t += blockDim.x) {
        const int i = (int)(t / n), j = (int)(t % n);
        const int32_t f = I.mat0[t], d = I.mat1[t];
        Fs[(int64_t)i * qs + j] = f;
        Ds[(int64_t)i * qs + j] = d;
        FTs[(int64_t)j * qs + i] = f;
        DTs[(int64_t)j * qs + i] = d;
      }
      X.F = Fs;
      X.D = Ds;
      X.FT = FTs;
      X.DT = DTs;
      X.qs = qs;
      break;
    }
    case KNAPSACK: {
      const int64_t b = align16((int64_t)I.n * 4);
      X.w = (const int32_t *)copy(I.vec0, b, 0);
      X.v = (const int32_t *)copy(I.vec1, b, b);
      break;
    }
    case CVRPTW: {
      const int64_t N = I.n + 1, b = align16(N * N * 4);
      X.rd = (const int32_t *)copy(I.mat0, b, 0);
      X.node = (const int4 *)copy(I.node, N * 16, b);
      break;
    }
    case GAP: {
      const int64_t b = align16((int64_t)I.m * I.n * 4);
      X.gc = (const int32_t *)copy(I.mat0, b, 0);
      X.gr = (const int32_t *)copy(I.mat1, b, b);
      X.gcap = (const int32_t *)copy(I.vec0, (int64_t)I.m * 4, 2 * b);
      break;
    }
  }
  return X;
}

// Single solve: CTA b covers members [b * groups, (b+1) * groups) of the
// instance, one member per group of WPM warps (cooperative launch, so that
// all members are resident together for the window barriers).
template <int MODEL, bool T16, int WPM, int NS, int XF>
__global__ void __launch_bounds__((WPM * NS > kMaxWarps ? WPM * NS : kMaxWarps) * 32, 1)
    evolve_kernel(const __grid_constant__ KInst I, int warps, uint64_t timeout_ns) {
  extern __shared__ __align__(16) unsigned char smem[];
  const bool staged = I.shared_bytes > 0;
  const View X = make_view(I, smem, staged);
  __syncthreads();
  const int groups = warps / (WPM * NS);
  const int p0 = blockIdx.x * groups;
  const int nsol = min(groups, I.P - p0);
  const Layout Lo = make_layout(staged ? I.shared_bytes : 0, I.len, I.m, groups, warps, WPM * NS,
                                I.model, I.wlong > 0);
  evolve_members<MODEL, T16, WPM, NS, XF>(I, X, smem, Lo, p0, nsol, warps, timeout_ns);
}

// Batched persistent kernel: each CTA takes the next instance of the work
// list, stages its data, and evolves all of its members (groups of WPM warps
// loop over them) for up to `slice` generations, with CTA-local window
// barriers; the instance's scalars are updated in place.  Instances that
// have reached their generation budget are skipped.
template <int MODEL, bool T16, int WPM, int XF>
__global__ void __launch_bounds__(kMaxWarps * 32, 1)
    batch_kernel(const KInst *__restrict__ insts, const int *__restrict__ list,
                 const int *__restrict__ count_ptr, int *next, int warps, int64_t slice,
                 uint64_t timeout_ns) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ KInst sI;
  __shared__ int su;
  const int count = *count_ptr;
  for (;;) {
    if (threadIdx.x == 0) su = atomicAdd(next, 1);
    __syncthreads();
    const int u = su;
    if (u >= count) return;
    if (threadIdx.x == 0) {
      sI = insts[list[u]];
      const int64_t g0 = sI.aos_in->g;
      sI.g_begin = g0;
      sI.g_end = min(sI.G_total, g0 + slice);
      sI.local_sync = 1;
      // reset this instance's window-barrier block
      DevSync *S = sI.sync;
      S->error = 0;
      for (int i = 0; i < 32; ++i) S->acc[0][i] = S->acc[1][i] = 0;
      S->elite[0] = S->elite[1] = LLONG_MAX;
      for (int i = 0; i < kStats; ++i) S->pend_out[i] = 0;
      __threadfence();
    }
    __syncthreads();
    const KInst &I = sI;
    if (I.g_begin < I.g_end) {
      const bool staged = I.shared_bytes > 0;
      const View X = make_view(I, smem, staged);
      __syncthreads();
      const int groups = warps / WPM;
      const Layout Lo =
          make_layout(staged ? I.shared_bytes : 0, I.len, I.m, I.P, warps, WPM, I.model, I.wlong > 0);
      evolve_members<MODEL, T16, WPM, 1, XF>(I, X, smem, Lo, 0, I.P, warps, timeout_ns);
      (void)groups;
    }
    __syncthreads();
  }
}

// the host reserves 1 KB of each CTA's shared memory for these statics
static_assert(sizeof(KInst) + 16 <= 1024, "static shared memory of batch_kernel exceeds its reserve");

// ---------------------------------------------------------------- init
__device__ long long full_cost(const KInst &I, const int32_t *x) {
  const int n = I.n;
  long long s = 0;
  switch (I.model) {
    case TSP:
    case ATSP:
      for (int k = 0; k < n; ++k) s += I.mat0[(size_t)x[k] * n + x[(k + 1) % n]];
      return s;
    case QAP:
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
          s += (long long)I.mat0[(size_t)i * n + j] * I.mat1[(size_t)x[i] * n + x[j]];
      return s;
    case KNAPSACK: {
      long long W = 0, V = 0;
      for (int i = 0; i < n; ++i)
        if (x[i]) {
          W += I.vec0[i];
          V += I.vec1[i];
        }
      return -V + I.lam0 * overp(W - I.capacity);
    }
    case CVRPTW: {
      View X;
      X.n = n;
      X.cap = I.capacity;
      X.lam0 = I.lam0;
      X.lam1 = I.lam1;
      X.wd = I.wdist;
      X.wv = I.wveh;
      X.rd = I.mat0;
      X.node = I.node;
      long long mx = 0;
      const long long c = cvrptw_routes(X, [&](int q) { return (int)x[q]; }, 0, I.len, false, Jumps(),
                                        I.wlong > 0 ? &mx : nullptr);
      return I.lex_n > 0 ? lex_key(I, c + I.wlong * mx) : c + I.wlong * mx;
    }
    case GAP: {
      for (int j = 0; j < n; ++j) s += I.mat0[(size_t)x[j] * n + j];
      for (int a = 0; a < I.m; ++a) {
        long long L = 0;
        for (int j = 0; j < n; ++j)
          if (x[j] == a) L += I.mat1[(size_t)a * n + j];
        s += I.lam0 * overp(L - I.vec0[a]);
      }
      return s;
    }
  }
  return 0;
}

// The kernels of one (model, matrix width, population-step code) set, by
// launch shape: one or two generations in flight with 1, 2 or 4 warps per
// generation, three or four with 4 (not with the population-step code, nor
// for the asymmetric TSP); batched kernels with 1, 2 or 4 warps per member.
// EM / BM select the shapes a translation unit instantiates (bit i of EM:
// (wpm, ns) = (1,1) (2,1) (4,1) (1,2) (2,2) (4,2) (4,3) (4,4); bit i of BM:
// wpm = 1, 2, 4); a shape outside them gives nullptr.
#define CGO_EV(WPM_, NS_, BIT_)                                            \
  if constexpr (((EM >> BIT_) & 1u) != 0u)                                 \
    if (wpm == WPM_ && ns == NS_) return (const void *)evolve_kernel<MODEL, T16, WPM_, NS_, XF>;
template <int MODEL, bool T16, int XF, unsigned EM = 0xFFu>
static const void *evolve_set(int wpm, int ns) {
  if (wpm != 2 && wpm != 4) wpm = 1;
  if constexpr (MODEL != ATSP && !XF) {
    CGO_EV(4, 3, 6)
    CGO_EV(4, 4, 7)
  }
  CGO_EV(1, 1, 0)
  CGO_EV(2, 1, 1)
  CGO_EV(4, 1, 2)
  CGO_EV(1, 2, 3)
  CGO_EV(2, 2, 4)
  CGO_EV(4, 2, 5)
  return nullptr;
}
#undef CGO_EV

template <int MODEL, bool T16, int XF, unsigned BM = 0x7u>
static const void *batch_set(int wpm) {
  if constexpr ((BM & 4u) != 0u)
    if (wpm == 4) return (const void *)batch_kernel<MODEL, T16, 4, XF>;
  if constexpr ((BM & 2u) != 0u)
    if (wpm == 2) return (const void *)batch_kernel<MODEL, T16, 2, XF>;
  if constexpr ((BM & 1u) != 0u)
    if (wpm != 2 && wpm != 4) return (const void *)batch_kernel<MODEL, T16, 1, XF>;
  return nullptr;
}

#ifndef CGO_UNIT
// Philox-seeded Fisher-Yates / random bits / random integers for member p,
// then its exact cost
// Random start j (member j of a plain start, candidate j of a start pool):
// Fisher-Yates for permutations, one draw per entry otherwise.
__device__ void random_start(const KInst &I, int p, int32_t *x) {
  const int len = I.len;
  const uint32_t k0 = (uint32_t)I.seed, k1 = (uint32_t)(I.seed >> 32);
  const bool perm = (I.model == TSP || I.model == QAP || I.model == CVRPTW || I.model == ATSP);
  if (perm) {
    for (int i = 0; i < len; ++i) x[i] = i;
    uint4 R = make_uint4(0, 0, 0, 0);
    for (int i = len - 1; i >= 1; --i) {
      const int d = len - 1 - i;
      if ((d & 3) == 0) R = philox(ctr_word((uint32_t)(d >> 2), 0, kKindInit), I.tag, (uint32_t)p,
                                   kInitGen, k0, k1);
      const uint32_t w = (d & 3) == 0 ? R.x : (d & 3) == 1 ? R.y : (d & 3) == 2 ? R.z : R.w;
      const int j = (int)(((uint64_t)w * (uint64_t)(i + 1)) >> 32);
      const int t = x[i];
      x[i] = x[j];
      x[j] = t;
    }
  } else {
    const int lb = I.model == GAP ? 0 : I.lb;
    const int ub = I.model == GAP ? I.m - 1 : I.ub;
    const uint64_t R = (uint64_t)((int64_t)ub - lb + 1);
    uint4 Q = make_uint4(0, 0, 0, 0);
    for (int i = 0; i < len; ++i) {
      if ((i & 3) == 0) Q = philox(ctr_word((uint32_t)(i >> 2), 0, kKindInit), I.tag, (uint32_t)p,
                                   kInitGen, k0, k1);
      const uint32_t w = (i & 3) == 0 ? Q.x : (i & 3) == 1 ? Q.y : (i & 3) == 2 ? Q.z : Q.w;
      if (I.model == KNAPSACK) x[i] = (int32_t)(w & 1u);
      else x[i] = lb + (int32_t)(((uint64_t)w * R) >> 32);
    }
  }
}

__device__ void init_member(const KInst &I, int p) {
  const int len = I.len;
  int32_t *x = I.cur + (int64_t)p * len;
  random_start(I, p, x);
  const long long c = full_cost(I, x);
  I.cost[p] = c;
  I.best[p] = c;
  int32_t *b = I.bestsol + (int64_t)p * len;
  for (int i = 0; i < len; ++i) b[i] = x[i];
}

// Start pool (Sec. 3.4.1-3.4.2): K*P random starts, then the heuristic
// permutations; the members are the P cheapest in order of (cost, index).
__device__ __forceinline__ bool pool_start(const KInst &I) { return I.K_over > 1 || I.n_heur > 0; }
__device__ __forceinline__ int pool_entries(const KInst &I) { return I.K_over * I.P + I.n_heur; }

__device__ void pool_fill(const KInst &I, int j) {
  const int len = I.len, R = I.K_over * I.P;
  int32_t *x = I.pool_sol + (int64_t)j * len;
  if (j < R) random_start(I, j, x);
  else
    for (int i = 0; i < len; ++i) x[i] = I.heur[(int64_t)(j - R) * I.n + i];
  I.pool_cost[j] = full_cost(I, x);
}

// entry j's rank among all entries; the P best become members 0 .. P-1
__device__ void pool_select(const KInst &I, int j) {
  const int N = pool_entries(I), len = I.len;
  const long long cj = I.pool_cost[j];
  int rank = 0;
  for (int i = 0; i < N; ++i) {
    const long long ci = I.pool_cost[i];
    rank += (ci < cj || (ci == cj && i < j)) ? 1 : 0;
  }
  if (rank >= I.P) return;
  const int32_t *x = I.pool_sol + (int64_t)j * len;
  int32_t *c = I.cur + (int64_t)rank * len, *b = I.bestsol + (int64_t)rank * len;
  for (int i = 0; i < len; ++i) c[i] = b[i] = x[i];
  I.cost[rank] = I.best[rank] = cj;
}

// one thread per member
__global__ void init_kernel(const __grid_constant__ KInst I) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < I.P) init_member(I, p);
}

// one thread per pool entry: build and cost it, then (second launch) rank it
__global__ void init_pool_fill_kernel(const __grid_constant__ KInst I) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < pool_entries(I)) pool_fill(I, j);
}

__global__ void init_pool_select_kernel(const __grid_constant__ KInst I) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < pool_entries(I)) pool_select(I, j);
}

// batched: one block per instance, threads over its members (or its pool)
__global__ void init_batch_kernel(const KInst *__restrict__ insts) {
  const KInst &I = insts[blockIdx.x];
  if (pool_start(I)) {
    const int N = pool_entries(I);
    for (int j = threadIdx.x; j < N; j += blockDim.x) pool_fill(I, j);
    __syncthreads();
    for (int j = threadIdx.x; j < N; j += blockDim.x) pool_select(I, j);
  } else {
    for (int p = threadIdx.x; p < I.P; p += blockDim.x) init_member(I, p);
  }
}

// elite = lowest best cost, lowest index on ties (one block)
__device__ void block_elite(const KInst &I, int &e_out, long long &c_out) {
  __shared__ long long sb[32];
  __shared__ int se[32];
  long long bb = LLONG_MAX;
  int be = INT_MAX;
  for (int q = threadIdx.x; q < I.P; q += blockDim.x) {
    const long long b = I.best[q];
    if (b < bb) {
      bb = b;
      be = q;
    }
  }
  warp_argmin(bb, be);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    sb[wid] = bb;
    se[wid] = be;
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    bb = lane < nw ? sb[lane] : LLONG_MAX;
    be = lane < nw ? se[lane] : INT_MAX;
    warp_argmin(bb, be);
  }
  e_out = be;
  c_out = bb;
}

// batched: one block per instance; a0s[b] holds the initial scalars
__global__ void init_aos_batch_kernel(const KInst *__restrict__ insts, const DevAos *__restrict__ a0s) {
  const KInst &I = insts[blockIdx.x];
  int e;
  long long c;
  block_elite(I, e, c);
  if (threadIdx.x == 0) {
    DevAos a0 = a0s[blockIdx.x];
    a0.elite = e;
    a0.elite_cost = c;
    a0.elite_prev = c;
    *I.aos_out = a0;
  }
}

__global__ void init_aos_kernel(const __grid_constant__ KInst I, DevAos a0) {
  int e;
  long long c;
  block_elite(I, e, c);
  if (threadIdx.x == 0) {
    a0.elite = e;
    a0.elite_cost = c;
    a0.elite_prev = c;
    *I.aos_out = a0;
  }
}

__global__ void finalize_kernel(const __grid_constant__ KInst I) {
  int e;
  long long c;
  block_elite(I, e, c);
  if (threadIdx.x == 0) {
    I.aos_out->elite = e;
    I.aos_out->elite_cost = c;
  }
  if (threadIdx.x < kStats) I.aos_out->pend[threadIdx.x] = I.sync->pend_out[threadIdx.x];
}

__global__ void triangle_kernel(const int32_t *__restrict__ mat, int n, int tri16, void *tri) {
  const int64_t total = (int64_t)n * n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / n), j = (int)(t % n);
    if (j < i) continue;
    const uint32_t idx = (((uint32_t)i * (uint32_t)(2 * n - 1 - i)) >> 1) + (uint32_t)j;
    if (tri16) ((int16_t *)tri)[idx] = (int16_t)mat[t];
    else ((int32_t *)tri)[idx] = mat[t];
  }
}

// flags[0]: 1 if D is asymmetric; flags[1]: max |D| (for the triangle width)
__global__ void tsp_check_kernel(const int32_t *__restrict__ mat, int n, uint32_t *flags) {
  const int64_t total = (int64_t)n * n;
  uint32_t asym = 0, mx = 0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / n), j = (int)(t % n);
    const int32_t v = mat[t];
    asym |= (uint32_t)(v != mat[(int64_t)j * n + i]);
    const uint32_t a = v < 0 ? (uint32_t)(-(int64_t)v) : (uint32_t)v;
    mx = max(mx, a);
  }
  if (asym) atomicOr(&flags[0], 1u);
  atomicMax(&flags[1], mx);
}

// copy the elite member's best solution and cost to caller buffers
__global__ void copy_elite_kernel(const DevAos *aos, const int32_t *bestsol, int len, int32_t *out_sol,
                                  int64_t *out_cost) {
  const int e = aos->elite;
  for (int i = threadIdx.x; i < len; i += blockDim.x) out_sol[i] = bestsol[(int64_t)e * len + i];
  if (threadIdx.x == 0) *out_cost = aos->elite_cost;
}

// ------------------------------------------------------------ launchers
// Kernels this library has put on a device (every launch that returned
// success; the kernels of a replayed graph are added by the replaying code).
static std::atomic<uint64_t> g_launches{0};
void note_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
uint64_t launches_total() { return g_launches.load(std::memory_order_relaxed); }
static cudaError_t counted(cudaError_t e, uint64_t n = 1) {
  if (e == cudaSuccess) note_launches(n);
  return e;
}

cudaError_t launch_tsp_check(const int32_t *d_mat, int n, uint32_t *d_flags, cudaStream_t st) {
  const int64_t total = (int64_t)n * n;
  const int blocks = (int)min((int64_t)1024, (total + 255) / 256);
  tsp_check_kernel<<<blocks, 256, 0, st>>>(d_mat, n, d_flags);
  return counted(cudaGetLastError());
}

cudaError_t launch_copy_elite(const DevAos *d_aos, const int32_t *d_bestsol, int len,
                              int32_t *out_sol, int64_t *out_cost, cudaStream_t st) {
  copy_elite_kernel<<<1, 256, 0, st>>>(d_aos, d_bestsol, len, out_sol, out_cost);
  return counted(cudaGetLastError());
}

cudaError_t launch_init(const KInst &h, cudaStream_t st) {
  const int threads = 128;
  if (h.K_over > 1 || h.n_heur > 0) {
    const int N = h.K_over * h.P + h.n_heur, blocks = (N + threads - 1) / threads;
    init_pool_fill_kernel<<<blocks, threads, 0, st>>>(h);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    init_pool_select_kernel<<<blocks, threads, 0, st>>>(h);
    return counted(cudaGetLastError(), 2);
  }
  const int blocks = (h.P + threads - 1) / threads;
  init_kernel<<<blocks, threads, 0, st>>>(h);
  return counted(cudaGetLastError());
}

cudaError_t launch_init_aos(const KInst &h, const DevAos &a0, cudaStream_t st) {
  init_aos_kernel<<<1, 256, 0, st>>>(h, a0);
  return counted(cudaGetLastError());
}

cudaError_t launch_init_batch(const KInst *d_insts, const DevAos *d_a0s, int count, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  init_batch_kernel<<<count, 128, 0, st>>>(d_insts);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  init_aos_batch_kernel<<<count, 256, 0, st>>>(d_insts, d_a0s);
  return counted(cudaGetLastError(), 2);
}

cudaError_t launch_finalize(const KInst &h, cudaStream_t st) {
  finalize_kernel<<<1, 256, 0, st>>>(h);
  return counted(cudaGetLastError());
}

cudaError_t build_triangle(const int32_t *d_mat, int n, int tri16, void *d_tri, cudaStream_t st) {
  const int64_t total = (int64_t)n * n;
  const int blocks = (int)min((int64_t)1024, (total + 255) / 256);
  triangle_kernel<<<blocks, 256, 0, st>>>(d_mat, n, tri16, d_tri);
  return counted(cudaGetLastError());
}


// The kernel sets are instantiated in translation units of their own, which
// compile in parallel: this file again, compiled with CGO_UNIT and the unit's
// sets defined (the unit table in build.py names them, at most two per
// unit); this unit keeps the
// set the benchmark's single solve runs (TSP, int16 triangle, without the
// population steps).  A unit returns nullptr for shapes it does not hold.
#define CGO_UNIT_DECL(NAME)                        \
  const void *unit_evolve_##NAME(int wpm, int ns); \
  const void *unit_batch_##NAME(int wpm);
CGO_UNIT_DECL(p_tsp32)
CGO_UNIT_DECL(p_atsp16)
CGO_UNIT_DECL(p_atsp32)
CGO_UNIT_DECL(p_qap)
CGO_UNIT_DECL(p_knapsack)
CGO_UNIT_DECL(p_gap)
CGO_UNIT_DECL(p_cvrptw_a)
CGO_UNIT_DECL(p_cvrptw_b)
CGO_UNIT_DECL(p_cvrptw_c)
CGO_UNIT_DECL(p_cvrptw_d)
CGO_UNIT_DECL(p_cvrptw_e)
CGO_UNIT_DECL(c_tsp16)
CGO_UNIT_DECL(c_tsp32)
CGO_UNIT_DECL(c_atsp16)
CGO_UNIT_DECL(c_atsp32)
CGO_UNIT_DECL(c_qap)
CGO_UNIT_DECL(c_knapsack)
CGO_UNIT_DECL(c_gap)
CGO_UNIT_DECL(c_cvrptw_a)
CGO_UNIT_DECL(c_cvrptw_b)
CGO_UNIT_DECL(c_cvrptw_c)
CGO_UNIT_DECL(x_tsp16)
CGO_UNIT_DECL(x_tsp32)
CGO_UNIT_DECL(x_atsp16)
CGO_UNIT_DECL(x_atsp32)
CGO_UNIT_DECL(x_qap)
CGO_UNIT_DECL(x_knapsack)
CGO_UNIT_DECL(x_gap)
CGO_UNIT_DECL(x_cvrptw_a)
CGO_UNIT_DECL(x_cvrptw_b)
CGO_UNIT_DECL(x_cvrptw_c)
CGO_UNIT_DECL(x_cvrptw_d)
CGO_UNIT_DECL(x_cvrptw_e)
#undef CGO_UNIT_DECL

// the first unit of a list that holds the shape
template <class... F>
static const void *first_evolve(int wpm, int ns, F... units) {
  const void *r = nullptr;
  ((r = r ? r : units(wpm, ns)), ...);
  return r;
}
template <class... F>
static const void *first_batch(int wpm, F... units) {
  const void *r = nullptr;
  ((r = r ? r : units(wpm)), ...);
  return r;
}

// the kernel of a single solve: with the crossover code (the c_ sets) or
// the migration and crossover code (the x_ sets) only when the solve takes
// them
static const void *pick_evolve(const KInst &h, int wpm, int ns) {
  const int xf = takes_xf(h);
  const bool t16 = h.tri16 != 0;
  switch (h.model) {
    case TSP:
      if (xf == 2) return t16 ? unit_evolve_x_tsp16(wpm, ns) : unit_evolve_x_tsp32(wpm, ns);
      if (xf == 1) return t16 ? unit_evolve_c_tsp16(wpm, ns) : unit_evolve_c_tsp32(wpm, ns);
      return t16 ? evolve_set<TSP, true, 0>(wpm, ns) : unit_evolve_p_tsp32(wpm, ns);
    case ATSP:
      if (xf == 2) return t16 ? unit_evolve_x_atsp16(wpm, ns) : unit_evolve_x_atsp32(wpm, ns);
      if (xf == 1) return t16 ? unit_evolve_c_atsp16(wpm, ns) : unit_evolve_c_atsp32(wpm, ns);
      return t16 ? unit_evolve_p_atsp16(wpm, ns) : unit_evolve_p_atsp32(wpm, ns);
    case QAP:
      return xf == 2 ? unit_evolve_x_qap(wpm, ns)
                     : (xf == 1 ? unit_evolve_c_qap(wpm, ns) : unit_evolve_p_qap(wpm, ns));
    case CVRPTW:
      if (xf == 2)
        return first_evolve(wpm, ns, unit_evolve_x_cvrptw_a, unit_evolve_x_cvrptw_b,
                            unit_evolve_x_cvrptw_c);
      if (xf == 1)
        return first_evolve(wpm, ns, unit_evolve_c_cvrptw_a, unit_evolve_c_cvrptw_b,
                            unit_evolve_c_cvrptw_c);
      return first_evolve(wpm, ns, unit_evolve_p_cvrptw_a, unit_evolve_p_cvrptw_b,
                          unit_evolve_p_cvrptw_c, unit_evolve_p_cvrptw_d);
    case KNAPSACK:
      return xf == 2 ? unit_evolve_x_knapsack(wpm, ns)
                     : (xf == 1 ? unit_evolve_c_knapsack(wpm, ns) : unit_evolve_p_knapsack(wpm, ns));
    case GAP:
      return xf == 2 ? unit_evolve_x_gap(wpm, ns)
                     : (xf == 1 ? unit_evolve_c_gap(wpm, ns) : unit_evolve_p_gap(wpm, ns));
  }
  return nullptr;
}

int64_t max_smem_optin() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return v;
}

// A kernel function's dynamic shared-memory limit is process-wide state, so
// it is raised once per device to the most the device allows and never set
// per launch: launches of one function with different sizes (the nodes of a
// captured graph, other host threads, a profiler replaying a node) must not
// see a smaller limit that was set for someone else.
static cudaError_t open_smem(const void *fn) {
  static std::mutex mu;
  static std::set<std::pair<int, const void *>> done;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  if (done.count({dev, fn})) return cudaSuccess;
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, fn);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(max_smem_optin() - (int64_t)fa.sharedSizeBytes));
  if (e == cudaSuccess) done.insert({dev, fn});
  return e;
}

int max_coresident_ctas(const KInst &h, int warps, int wpm, int ns, int64_t smem_bytes) {
  const void *fn = pick_evolve(h, wpm, ns);
  if (!fn) return 0;
  if (open_smem(fn) != cudaSuccess) return 0;
  int per_sm = 0, dev = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, warps * 32, (size_t)smem_bytes) !=
      cudaSuccess)
    return 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return per_sm * sms;
}

cudaError_t launch_evolve_single(const KInst &h, int warps, int wpm, int ns, int64_t smem_bytes,
                                 uint64_t timeout_ns, cudaStream_t st) {
  const void *fn = pick_evolve(h, wpm, ns);
  if (!fn) return cudaErrorInvalidValue;
  cudaError_t e = open_smem(fn);
  if (e != cudaSuccess) return e;
  const int groups = warps / (wpm * ns);
  const int grid = (h.P + groups - 1) / groups;
  KInst hi = h;
  void *args[] = {(void *)&hi, (void *)&warps, (void *)&timeout_ns};
  return counted(
      cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(warps * 32), args, (size_t)smem_bytes, st));
}


// the batched kernel of a bucket: with the migration and crossover code
// (the x_ sets) for instances that take either
static const void *pick_batch(int model, int tri16, int xf, int wpm) {
  switch (model) {
    case TSP:
      if (xf) return tri16 ? unit_batch_x_tsp16(wpm) : unit_batch_x_tsp32(wpm);
      return tri16 ? batch_set<TSP, true, 0>(wpm) : unit_batch_p_tsp32(wpm);
    case ATSP:
      if (xf) return tri16 ? unit_batch_x_atsp16(wpm) : unit_batch_x_atsp32(wpm);
      return tri16 ? unit_batch_p_atsp16(wpm) : unit_batch_p_atsp32(wpm);
    case QAP: return xf ? unit_batch_x_qap(wpm) : unit_batch_p_qap(wpm);
    case CVRPTW:
      return xf ? first_batch(wpm, unit_batch_x_cvrptw_d, unit_batch_x_cvrptw_e)
                : first_batch(wpm, unit_batch_p_cvrptw_e);
    case KNAPSACK: return xf ? unit_batch_x_knapsack(wpm) : unit_batch_p_knapsack(wpm);
    case GAP: return xf ? unit_batch_x_gap(wpm) : unit_batch_p_gap(wpm);
  }
  return nullptr;
}

int batch_ctas_per_sm(int model, int tri16, int xf, int warps, int wpm, int64_t smem_bytes) {
  const void *fn = pick_batch(model, tri16, xf, wpm);
  if (!fn) return 0;
  if (open_smem(fn) != cudaSuccess) return 0;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, warps * 32, (size_t)smem_bytes) !=
      cudaSuccess)
    return 0;
  return per_sm;
}

cudaError_t launch_batch(int model, int tri16, int xf, const KInst *d_insts, const int *d_list,
                         const int *d_count, int *d_next, int warps, int wpm, int64_t smem_bytes,
                         int grid, int64_t slice, uint64_t timeout_ns, cudaStream_t st) {
  const void *fn = pick_batch(model, tri16, xf, wpm);
  if (!fn) return cudaErrorInvalidValue;
  cudaError_t e = open_smem(fn);
  if (e != cudaSuccess) return e;
  void *args[] = {(void *)&d_insts, (void *)&d_list, (void *)&d_count, (void *)&d_next,
                  (void *)&warps, (void *)&slice, (void *)&timeout_ns};
  return cudaLaunchKernel(fn, dim3(grid), dim3(warps * 32), args, (size_t)smem_bytes, st);
}

// shared memory of a batched unit: all P members of an instance in one CTA
int64_t batch_smem_bytes(const KInst &h, int warps, int wpm, bool staged) {
  const Layout L =
      make_layout(staged ? instance_data_bytes(h) : 0, h.len, h.m, h.P, warps, wpm, h.model, h.wlong > 0);
  return L.total;
}

int64_t evolve_smem_bytes(const KInst &h, int warps, int wpm, int ns, bool staged) {
  const Layout L = make_layout(staged ? instance_data_bytes(h) : 0, h.len, h.m, warps / (wpm * ns),
                               warps, wpm * ns, h.model, h.wlong > 0);
  return L.total;
}

#else  // CGO_UNIT: a kernel unit exports the kernel sets it instantiates
}  // namespace
// set i of the unit: CGO_UNIT_S<i>_NAME, _MODEL, _T16, _EM, _BM (compiler
// definitions, one value each)
#define CGO_UNIT_SET_(NAME, MODEL, T16, EM, BM)                                \
  const void *unit_evolve_##NAME(int wpm, int ns) {                            \
    return evolve_set<MODEL, T16, CGO_UNIT_XF, EM>(wpm, ns);                   \
  }                                                                            \
  const void *unit_batch_##NAME(int wpm) { return batch_set<MODEL, T16, CGO_UNIT_XF, BM>(wpm); }
#define CGO_UNIT_SET(NAME, MODEL, T16, EM, BM) CGO_UNIT_SET_(NAME, MODEL, T16, EM, BM)
CGO_UNIT_SET(CGO_UNIT_S1_NAME, CGO_UNIT_S1_MODEL, CGO_UNIT_S1_T16, CGO_UNIT_S1_EM, CGO_UNIT_S1_BM)
#ifdef CGO_UNIT_S2_NAME
CGO_UNIT_SET(CGO_UNIT_S2_NAME, CGO_UNIT_S2_MODEL, CGO_UNIT_S2_T16, CGO_UNIT_S2_EM, CGO_UNIT_S2_BM)
#endif
#undef CGO_UNIT_SET
#undef CGO_UNIT_SET_
#endif  // CGO_UNIT

}  // namespace cgo
