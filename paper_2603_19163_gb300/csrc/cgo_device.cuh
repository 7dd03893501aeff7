// Device primitives of the search generation: counter-based random numbers,
// index mapping, roulette choice, the integer acceptance test, cooling, the
// Q16 AOS update, warp reductions and the permutation-move algebra.
#pragma once
#include <stdint.h>
#include <climits>

#include "cgo_internal.h"

namespace cgo {

constexpr unsigned kFull = 0xffffffffu;
constexpr uint32_t kKindMove = 0u, kKindAccept = 1u, kKindInit = 2u, kKindCross = 3u;
constexpr uint32_t kInitGen = 0xFFFFFFFFu;

__device__ __forceinline__ uint32_t ctr_word(uint32_t cand, uint32_t step, uint32_t kind) {
  return cand | (step << 20) | (kind << 24);
}

// Philox4x32-10 (Salmon et al., SC'11): counter (c0..c3), key (k0, k1).
__device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                        uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    c0 = hi1 ^ c1 ^ k0;
    c2 = hi0 ^ c3 ^ k1;
    c1 = lo1;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return make_uint4(c0, c1, c2, c3);
}

// Three Philox4x32-10 blocks whose counters differ only in word 0, advanced
// round by round so that the three dependency chains sit next to each other
// in program order (warps issue in order; this is what lets them overlap).
__device__ __forceinline__ void philox3(uint32_t a0, uint32_t b0, uint32_t e0, uint32_t c1,
                                        uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1,
                                        uint4 &A, uint4 &B, uint4 &E) {
  uint32_t a[4] = {a0, c1, c2, c3}, b[4] = {b0, c1, c2, c3}, e[4] = {e0, c1, c2, c3};
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t alo0 = 0xD2511F53u * a[0], ahi0 = __umulhi(0xD2511F53u, a[0]);
    const uint32_t blo0 = 0xD2511F53u * b[0], bhi0 = __umulhi(0xD2511F53u, b[0]);
    const uint32_t elo0 = 0xD2511F53u * e[0], ehi0 = __umulhi(0xD2511F53u, e[0]);
    const uint32_t alo1 = 0xCD9E8D57u * a[2], ahi1 = __umulhi(0xCD9E8D57u, a[2]);
    const uint32_t blo1 = 0xCD9E8D57u * b[2], bhi1 = __umulhi(0xCD9E8D57u, b[2]);
    const uint32_t elo1 = 0xCD9E8D57u * e[2], ehi1 = __umulhi(0xCD9E8D57u, e[2]);
    a[0] = ahi1 ^ a[1] ^ k0;
    b[0] = bhi1 ^ b[1] ^ k0;
    e[0] = ehi1 ^ e[1] ^ k0;
    a[2] = ahi0 ^ a[3] ^ k1;
    b[2] = bhi0 ^ b[3] ^ k1;
    e[2] = ehi0 ^ e[3] ^ k1;
    a[1] = alo1;
    b[1] = blo1;
    e[1] = elo1;
    a[3] = alo0;
    b[3] = blo0;
    e[3] = elo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  A = make_uint4(a[0], a[1], a[2], a[3]);
  B = make_uint4(b[0], b[1], b[2], b[3]);
  E = make_uint4(e[0], e[1], e[2], e[3]);
}

// A 16-bit field scaled to [0, m): floor(h * m / 2^16), m <= 65536.
__device__ __forceinline__ int posm(uint32_t h16, uint32_t m) { return (int)((h16 * m) >> 16); }

// Roulette choice: r = floor(word * W / 2^32), first i with r < w_0 + .. + w_i.
// Counting the prefix sums cum_i = w_0 + .. + w_i that are <= r gives that
// index (the sums do not decrease).
template <int N>
__device__ __forceinline__ int wpick(const uint32_t (&cum)[N], uint32_t W, uint32_t word) {
  const uint32_t r = __umulhi(word, W);
  int idx = 0;
#pragma unroll
  for (int i = 0; i < N; ++i) idx += (r >= cum[i]);
  return idx;
}

// -ln(u) in Q32 for u = (A + 1) / 2^32: the binary logarithm digit by digit
// (repeated squaring of the Q2.62 mantissa, C. S. Turner, IEEE SPM 2010),
// then times round(ln 2 * 2^32).
__device__ __forceinline__ uint64_t exp_variate_q32(uint32_t A) {
  const uint64_t y = (uint64_t)A + 1ull;
  const int e = 63 - __clzll((long long)y);
  uint64_t z = y << (62 - e);
  uint32_t frac = 0;
#pragma unroll 8
  for (int i = 1; i <= 32; ++i) {
    const uint64_t lo = z * z, hi = __umul64hi(z, z);
    z = (hi << 2) | (lo >> 62);
    const uint32_t bit = (uint32_t)(z >> 63);
    z >>= bit;
    frac |= bit << (32 - i);
  }
  const uint64_t L = (32ull << 32) - (((uint64_t)e << 32) + frac);
  const uint64_t lo = L * 2977044472ull, hi = __umul64hi(L, 2977044472ull);
  return (hi << 32) | (lo >> 32);
}

// The largest value exp_variate_q32 returns (A = 0: log2 term 32).
constexpr uint64_t kExpVariateMax = 32ull * 2977044472ull;

// Metropolis test in integers: accept iff delta <= 0 or delta < T * E.
__device__ __forceinline__ bool accept_move(long long delta, uint64_t T, uint64_t E) {
  if (delta <= 0) return true;
  const uint64_t hi = __umul64hi(T, E), lo = T * E;
  const uint64_t d = (uint64_t)delta;
  return d < hi || (d == hi && lo != 0ull);
}

__device__ __forceinline__ uint64_t cool(uint64_t T, uint64_t alpha) {
  return (__umul64hi(T, alpha) << 32) | ((T * alpha) >> 32);
}

// Eq. "ema" on one level, Q16: w <- (a*w + (1-a)*(v/(u+1) + floor)) >> 16,
// clamped to [floor, min(cap, cap_i)], then w <- w * 2^16 / sum(w).
template <int N>
__device__ __forceinline__ void aos_level(uint32_t (&w)[N], const uint32_t (&u)[N],
                                          const uint32_t (&v)[N], uint32_t enabled,
                                          const uint32_t (&capi)[N], uint32_t a,
                                          uint32_t wfloor, uint32_t wcap) {
  uint64_t S = 0;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    if ((enabled >> i) & 1u) {
      const uint64_t ratio = ((uint64_t)v[i] << 16) / ((uint64_t)u[i] + 1ull);
      uint64_t nw = ((uint64_t)a * w[i] + (uint64_t)(65536u - a) * (ratio + wfloor)) >> 16;
      const uint64_t hi = wcap < capi[i] ? wcap : capi[i];
      nw = nw > hi ? hi : nw;
      nw = nw < wfloor ? wfloor : nw;
      w[i] = (uint32_t)nw;
      S += nw;
    }
  }
#pragma unroll
  for (int i = 0; i < N; ++i)
    if ((enabled >> i) & 1u) w[i] = (uint32_t)(((uint64_t)w[i] << 16) / S);
}

// floor(num / den), den >= 1, in integer arithmetic (double precision is
// a slow unit on this GPU)
__device__ __forceinline__ uint64_t udiv_exact(uint64_t num, uint64_t den) {
  return num <= 0xFFFFFFFFull && den <= 0xFFFFFFFFull ? (uint64_t)((uint32_t)num / (uint32_t)den)
                                                      : num / den;
}

// Eq. "ema" for both levels at once, one lane per weight: lanes 0..NO-1
// hold the operator weights, lanes 24..26 the K weights; u/v are read from
// the lanes that hold the window totals (u_op at lane o, v_op at kStatV + o,
// u_k at kStatUK + i, v_k at kStatVK + i, o the global operator E::glob(l)
// of local operator l).  Every lane ends with the new weights.
template <class E>
__device__ __forceinline__ void aos_update_lanes(uint32_t (&wop)[E::NO], uint32_t (&wk)[3],
                                                 uint32_t total, uint32_t en_local,
                                                 const uint32_t (&capl)[E::NO], uint32_t a,
                                                 uint32_t wfloor, uint32_t wcap) {
  constexpr int NO = E::NO;
  const int lane = threadIdx.x & 31;
  const bool is_op = lane < NO, is_k = lane >= 24 && lane < 27;
  const int li = is_op ? lane : lane - 24;
  int go = 0;
#pragma unroll
  for (int l = 0; l < NO; ++l) go = li == l ? E::glob(l) : go;
  static_assert(NO <= 24, "operator lanes must stay below the K lanes");
  const uint32_t u = __shfl_sync(kFull, total, is_op ? go : (is_k ? kStatUK + li : 0));
  const uint32_t v = __shfl_sync(kFull, total, is_op ? kStatV + go : (is_k ? kStatVK + li : 0));
  uint32_t w = 0, cap = 65536u;
  bool en = false;
#pragma unroll
  for (int l = 0; l < NO; ++l)
    if (is_op && li == l) {
      w = wop[l];
      cap = capl[l];
      en = (en_local >> l) & 1u;
    }
#pragma unroll
  for (int i = 0; i < 3; ++i)
    if (is_k && li == i) {
      w = wk[i];
      en = true;
    }
  uint64_t nw = 0;
  if (en) {
    const uint64_t ratio = udiv_exact((uint64_t)v << 16, (uint64_t)u + 1ull);
    nw = ((uint64_t)a * w + (uint64_t)(65536u - a) * (ratio + wfloor)) >> 16;
    const uint64_t hi = wcap < cap ? wcap : cap;
    nw = nw > hi ? hi : nw;
    nw = nw < wfloor ? wfloor : nw;
  }
  const uint32_t s_op = __reduce_add_sync(kFull, is_op ? (uint32_t)nw : 0u);
  const uint32_t s_k = __reduce_add_sync(kFull, is_k ? (uint32_t)nw : 0u);
  const uint32_t mine = en ? (uint32_t)udiv_exact(nw << 16, is_op ? s_op : s_k) : w;
#pragma unroll
  for (int l = 0; l < NO; ++l) wop[l] = __shfl_sync(kFull, mine, l);
#pragma unroll
  for (int i = 0; i < 3; ++i) wk[i] = __shfl_sync(kFull, mine, 24 + i);
}

// Lexicographic (delta, index) minimum over the warp; every lane gets it.
// Signed 64-bit order is (signed high word, unsigned low word), so three
// warp reductions (high, low among the lanes holding the high minimum, index
// among the lanes holding both) give the minimum pair.
__device__ __forceinline__ void warp_argmin(long long &d, int &c) {
  const int hi = (int)(d >> 32);
  const uint32_t lo = (uint32_t)d;
  const int hmin = __reduce_min_sync(kFull, hi);
  const uint32_t lmin = __reduce_min_sync(kFull, hi == hmin ? lo : 0xFFFFFFFFu);
  const int cmin = __reduce_min_sync(kFull, (hi == hmin && lo == lmin) ? c : INT_MAX);
  d = (long long)(((uint64_t)(uint32_t)hmin << 32) | lmin);
  c = cmin;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// arrival at a barrier: everything this thread (and, through the barrier
// that preceded it, its warp) did before is visible to whoever observes the add
__device__ __forceinline__ void add_release(uint32_t *p, uint32_t v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ long long ld_relaxed64(const long long *p) {
  long long v;
  asm volatile("ld.relaxed.gpu.global.s64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// ---------------------------------------------------------------------------
// Permutation moves as "cut and reorder" of an array of length m.
// Five pieces P0 = [0,b1), A = [b1,b2), M = [b2,b3), B = [b3,b4), P4 = [b4,m);
// the move produces P0 B M A' P4, with A' = A reversed when rev is set
// (2-opt uses A only, with M and B empty).
//   swap(lo,hi)        A=[lo], M=(lo,hi), B=[hi]
//   2-opt(lo,hi)       A=[lo..hi] reversed
//   insert(i -> j)     i<j: A=[i], B=(i,j];  i>j: A=[j,i), B=[i]
//   or-opt(i, L, q)    q<i: A=[q,i), B=[i,i+L);  q>i: A=[i,i+L), B=[i+L,q+L)
struct PMove {
  int b1, b2, b3, b4;
  int rev;
};

template <bool T3>
__device__ __forceinline__ PMove perm_decode(int op, uint32_t r1, uint32_t r2, int m) {
  // every variant is computed and the operator selects one (no branches:
  // lanes of a warp draw different operators)
  const uint32_t a = r1 >> 16, b = r1 & 0xFFFFu;
  const int L = 2 + (int)(r2 & 1u);
  const int io = posm(a, (uint32_t)(m - L + 1));
  int q = posm(b, (uint32_t)(m - L));
  q += (q >= io);
  const int i = posm(a, (uint32_t)m);
  int j = posm(b, (uint32_t)(m - 1));
  j += (j >= i);
  const int lo = min(i, j), hi = max(i, j);
  const bool ob = q < io;
  // local operator 4 of a permutation is 3-opt: three distinct cut points of
  // 0..m (from m+1, m and m-1 values, each later draw stepping over the
  // points already taken); the segments between them change places.  Its
  // variant is compiled in only where the instance enables it (T3), so
  // other instances run the same straight-line code as without it.
  const bool oo = op == OR_OPT, sw = op == SWAP, two = op == TWO_OPT, fw = i < j;
  bool t3 = false;
  int ci = 0, cj = 0, ck = 0;
  if constexpr (T3) {
    t3 = op == 4;
    const int c1 = posm(a, (uint32_t)(m + 1));
    int c2 = posm(b, (uint32_t)m);
    c2 += (c2 >= c1);
    const int clo = min(c1, c2), chi = max(c1, c2);
    int c3 = posm(r2 >> 16, (uint32_t)(m - 1));
    c3 += (c3 >= clo);
    c3 += (c3 >= chi);
    ci = min(clo, c3);
    ck = max(chi, c3);
    cj = c1 + c2 + c3 - ci - ck;
  }
  PMove mv;
  const int o1 = ob ? q : io, o2 = ob ? io : io + L, o4 = ob ? io + L : q + L;
  const int p1 = (sw || two) ? lo : (fw ? i : j);
  const int p2 = sw ? lo + 1 : (two ? hi + 1 : (fw ? i + 1 : i));
  const int p3 = sw ? hi : (two ? hi + 1 : (fw ? i + 1 : i));
  const int p4 = sw ? hi + 1 : (two ? hi + 1 : (fw ? j + 1 : i + 1));
  mv.b1 = t3 ? ci : (oo ? o1 : p1);
  mv.b2 = t3 ? cj : (oo ? o2 : p2);
  mv.b3 = t3 ? cj : (oo ? o2 : p3);
  mv.b4 = t3 ? ck : (oo ? o4 : p4);
  mv.rev = (!oo && !t3 && two) ? 1 : 0;
  return mv;
}

// Position in the array before the move of the element at position q after
// it (branch-free).
// Inside [b1, b4) the new array reads B, then M, then A: position q comes
// from q + (b3 - b1) below b1 + |B|, from q + (b2 - b1 - |B|) below
// b1 + |B| + |M|, else from q - |B| - |M|; a reversal reads b1 + b2 - 1 - q.
__device__ __forceinline__ int perm_inv(const PMove &mv, int q) {
  const int lb = mv.b4 - mv.b3, lm = mv.b3 - mv.b2;
  const int t1 = mv.b1 + lb, t2 = t1 + lm;
  const bool in = q >= mv.b1 && q < mv.b4;
  int add = q < t1 ? mv.b3 - mv.b1 : (q < t2 ? mv.b2 - mv.b1 - lb : -(lb + lm));
  add = in ? add : 0;
  const int r = q + add;
  return (in && mv.rev) ? mv.b1 + mv.b2 - 1 - q : r;
}

}  // namespace cgo
