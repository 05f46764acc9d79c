// lp_scan_dev.cuh -- device helpers of the wedge scan shared by the scan
// kernels (lp_scan.cu) and the expand-and-count large tier (lp_expand.cu):
// keys of Eq. 1-9, wedge loops, shared-memory tables, candidate sinks and
// the scoring passes.  Header-only (inline device code).
#pragma once

#include <float.h>
#include <limits.h>
#include <math.h>

#include <type_traits>

#include "lp_internal.cuh"

namespace lp {

#define FULLMASK 0xffffffffu

__device__ __forceinline__ u32 hash_slot(int key, int logcap) {
  return ((u32)key * 0x9E3779B1u) >> (32 - logcap);
}

// Dense-window layout: counter i sits at position swz(i) (an involution that
// keeps each aligned block of 32).  Hub lists step through the window with
// near-constant strides; without it those strides fall on a few banks.
__device__ __forceinline__ int swz(int i) { return i ^ ((i >> 5) & 31); }

__host__ __device__ __forceinline__ int ceil_log2(u64 x) {
  int l = 0;
  while ((1ull << l) < x) ++l;
  return l;
}

// Fixed-point weight that an intermediary of degree db adds (Algorithm 1,
// scanEdges: 1/log|Gamma_b| for AA, 1/|Gamma_b| for RA), rounded to
// nearest at fixbits fraction bits.  Intermediaries have degree >= 2.
__device__ __forceinline__ u64 fixed_weight(int measure, int db, int fixbits) {
  if (db < 2) return 0;
  if (measure == LP_RA) return __double2ull_rn(ldexp(1.0, fixbits) / (double)db);
  return __double2ull_rn(ldexp(1.0, fixbits) / log((double)db));
}

// Weight that intermediary b of degree db adds to each of its wedges: 1 for
// the count measures, the table entry for AA and RA (no FP64 in the scan).
template <typename V>
__device__ __forceinline__ V arc_weight(const ScanArgs& A, int db) {
  if (sizeof(V) == 8) return (V)__ldg(A.wt + db);
  return (V)1;
}

// Exact ordering key num/den of Eq. 1-7 (Salton through its square); for AA
// and RA the fixed-point sum over 1.
__device__ __forceinline__ void make_key(int measure, u64 v, u64 da, u64 dc, u64& num, u64& den) {
  num = v;
  den = 1;
  switch (measure) {
    case LP_JC: den = da + dc - v; break;
    case LP_SI: den = da + dc; break;
    case LP_SC: num = v * v; den = da * dc; break;
    case LP_HP: den = da < dc ? da : dc; break;
    case LP_HD: den = da > dc ? da : dc; break;
    case LP_LHN: den = da * dc; break;
    default: break;
  }
}

__device__ __forceinline__ bool needs_dc(int measure) {
  return measure != LP_CN && measure != LP_AA && measure != LP_RA;
}

// FP64 value of a score from its key (the same IEEE operations as the
// definitions: one correctly rounded division, Salton through a square root).
__device__ __forceinline__ double key_value(int measure, u64 num, u64 den, u64 cn, int fixbits) {
  if (measure == LP_AA || measure == LP_RA) return ldexp(__ull2double_rn(num), -fixbits);
  if (measure == LP_SC) return __ddiv_rn(__ull2double_rn(cn), __dsqrt_rn(__ull2double_rn(den)));
  return __ddiv_rn(__ull2double_rn(num), __ull2double_rn(den));
}

// ------------------------------------------------------- wedge loops ------

// First index in idx[l, r) whose value is >= key (lists are sorted).
__device__ __forceinline__ int lower_bound_g(const int* __restrict__ idx, int l, int r, int key) {
  while (l < r) {
    const int m = (l + r) >> 1;
    if (__ldg(idx + m) < key) l = m + 1; else r = m;
  }
  return l;
}

// First index in idx[l, r) whose value is >= key.  The ids of an adjacency
// list spread over the id range roughly evenly, so up to three interpolation
// probes narrow the range before the bisection: fewer dependent loads than
// bisection alone on long lists, and never more than three extra.
__device__ __forceinline__ int lower_bound_interp(const int* __restrict__ idx, int l, int r,
                                                  int key) {
  if (l >= r) return l;
  int vl = __ldg(idx + l);
  if (vl >= key) return l;
  int vr = __ldg(idx + r - 1);
  if (vr < key) return r;
  int lo = l, hi = r - 1;  // idx[lo] < key <= idx[hi]
  for (int it = 0; it < 3 && hi - lo > 16; ++it) {
    int g = lo + (int)(((long long)(key - vl) * (long long)(hi - lo)) / (long long)(vr - vl));
    g = max(lo + 1, min(hi - 1, g));
    const int v = __ldg(idx + g);
    if (v < key) {
      lo = g;
      vl = v;
    } else {
      hi = g;
      vr = v;
    }
  }
  return lower_bound_g(idx, lo + 1, hi, key);
}

constexpr int kLongArc = 64;

// The warp holds up to 32 arcs (lane j: suffix start s_j, length len_j,
// weight w_j).  Calls f(c, w) once for every one of the sum(len) wedges.
template <typename V, typename F>
__device__ __forceinline__ void scan_arcs(int s, int len, V w, const int* __restrict__ idx, F&& f) {
  const int lane = lane_id();
  // long suffixes: the whole warp streams one suffix, four loads per lane
  u32 lm = __ballot_sync(FULLMASK, len >= kLongArc);
  while (lm) {
    const int j = __ffs(lm) - 1;
    lm &= lm - 1;
    const int sj = __shfl_sync(FULLMASK, s, j);
    const int lj = __shfl_sync(FULLMASK, len, j);
    const V wj = __shfl_sync(FULLMASK, w, j);
    const int* p = idx + sj;
    int i = lane;
    for (; i + 96 < lj; i += 128) {
      const int c0 = __ldg(p + i), c1 = __ldg(p + i + 32), c2 = __ldg(p + i + 64),
                c3 = __ldg(p + i + 96);
      f(c0, wj);
      f(c1, wj);
      f(c2, wj);
      f(c3, wj);
    }
    for (; i < lj; i += 32) f(__ldg(p + i), wj);
  }
  if (len >= kLongArc) len = 0;
  // short suffixes: concatenated, two 32-wedge windows per step
  int incl = len;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(FULLMASK, incl, o);
    if (lane >= o) incl += t;
  }
  const int total = __shfl_sync(FULLMASK, incl, 31);
  const int excl = incl - len;
  for (int base = 0; base < total; base += 64) {
    const int p0 = base + lane, p1 = base + 32 + lane;
    int j0 = 0, j1 = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
      const int e0 = __shfl_sync(FULLMASK, excl, j0 + step);
      const int e1 = __shfl_sync(FULLMASK, excl, j1 + step);
      if (e0 <= p0) j0 += step;
      if (e1 <= p1) j1 += step;
    }
    const int s0 = __shfl_sync(FULLMASK, s, j0) - __shfl_sync(FULLMASK, excl, j0);
    const int s1 = __shfl_sync(FULLMASK, s, j1) - __shfl_sync(FULLMASK, excl, j1);
    const V w0 = __shfl_sync(FULLMASK, w, j0);
    const V w1 = __shfl_sync(FULLMASK, w, j1);
    int c0 = 0, c1 = 0;
    if (p0 < total) c0 = __ldg(idx + s0 + p0);
    if (p1 < total) c1 = __ldg(idx + s1 + p1);
    if (p0 < total) f(c0, w0);
    if (p1 < total) f(c1, w1);
  }
}

// ----------------------------------------------------------- hash tables --

// Shared-memory accumulate.  A 64-bit value is added as two 32-bit atomics:
// the low word, then the high word plus the carry out of the low word (the
// 32-bit shared atomics run several times faster than the 64-bit one).  The
// value is exact once all adds are done, since each wrap of the low word is
// paid by the add that caused it; nothing reads it before then.  Returns the
// old low word (0 on the first add to a zero counter).
template <typename V>
__device__ __forceinline__ u32 shared_add(V* p, V w) {
  if (sizeof(V) == 8) {
    u32* q = reinterpret_cast<u32*>(p);
    const u32 l = (u32)w, h = (u32)((u64)w >> 32);
    const u32 old = atomicAdd(q, l);
    const u32 hc = h + ((old + l < old) ? 1u : 0u);
    if (hc) atomicAdd(q + 1, hc);
    return old;
  }
  return atomicAdd(reinterpret_cast<u32*>(p), (u32)w);
}

// Add w to key c (stored as c + 1).  Returns 1 if c was new, 0 if it
// existed, 2 if no free slot came within max_probe probes (by default the
// whole table).  Tables that may fill pass fill_probes(logcap): a probe run
// of a quarter of the table, at most 256 slots (linear probing,
// multiplicative hash), means it is about three quarters full or more, and
// the caller splits the range, so no shared distinct-key counter is needed.
__device__ __forceinline__ u32 fill_probes(int logcap) {
  return min(256u, (1u << logcap) >> 2);
}
template <typename V>
__device__ __forceinline__ int hash_add(int* keys, V* vals, int logcap, int c, V w,
                                       u32 max_probe = 0xffffffffu) {
  const u32 mask = (1u << logcap) - 1u;
  const int key = c + 1;
  u32 h = hash_slot(key, logcap);
  const u32 np = min(mask, max_probe - 1u);
  for (u32 probe = 0; probe <= np; ++probe) {
    const int k = ((volatile int*)keys)[h];
    if (k == key) {
      shared_add<V>(&vals[h], w);
      return 0;
    }
    if (k == kEmpty) {
      const int old = atomicCAS(&keys[h], kEmpty, key);
      if (old == kEmpty || old == key) {
        shared_add<V>(&vals[h], w);
        return old == kEmpty ? 1 : 0;
      }
    }
    h = (h + 1u) & mask;
  }
  return 2;
}

// Clear the value of key b if present (first-order exclusion).
template <typename V>
__device__ __forceinline__ void hash_kill(int* keys, V* vals, int logcap, int b) {
  const u32 mask = (1u << logcap) - 1u;
  const int key = b + 1;
  u32 h = hash_slot(key, logcap);
  for (u32 probe = 0; probe <= mask; ++probe) {
    const int k = keys[h];
    if (k == key) {
      vals[h] = 0;
      return;
    }
    if (k == kEmpty) return;
    h = (h + 1u) & mask;
  }
}

// ------------------------------------------------------ candidate sinks --

// Global mode: warp-aggregated append of passing candidates to the selection
// buffer.  Returns true if any lane's entry did not fit.
__device__ __forceinline__ bool admit_global(const ScanArgs& A, bool pass, u64 num, u64 den, int u,
                                             int v) {
  const u32 mask = __ballot_sync(FULLMASK, pass);
  if (mask == 0) return false;
  const int lane = lane_id();
  const int leader = __ffs(mask) - 1;
  u64 base = 0;
  if (lane == leader) base = atomicAdd(&A.ctr->cand_cnt, (u64)__popc(mask));
  base = __shfl_sync(FULLMASK, base, leader);
  bool bad = false;
  if (pass) {
    const u64 pos = base + __popc(mask & ((1u << lane) - 1u));
    if (pos < A.buf_cap) {
      Cand c;
      c.num = num;
      c.den = den;
      c.u = u;
      c.v = v;
      A.buf[pos] = c;
    } else {
      bad = true;
    }
  }
  return __any_sync(FULLMASK, bad);
}

// Per-source top-k list in shared memory, kept sorted by (score desc, c asc).
__device__ __forceinline__ bool ent_before(const TopEnt& x, const TopEnt& y) {
  return before(x.num, x.den, x.c, 0, y.num, y.den, y.c, 0);
}

// Warp-cooperative insertion of x (same value in every lane) into top[0..cnt).
__device__ __forceinline__ void top_insert(TopEnt* top, int& cnt, int k, const TopEnt& x) {
  const int lane = lane_id();
  int nb = 0;
  for (int j = lane; j < cnt; j += 32) nb += ent_before(top[j], x) ? 1 : 0;
  const int pos = __reduce_add_sync(FULLMASK, (u32)nb);
  if (pos >= k) return;
  const int ncnt = cnt + 1 < k ? cnt + 1 : k;
  // move [pos, ncnt - 1) one to the right, highest chunk first
  const int nmove = ncnt - 1 - pos;
  for (int c0 = ((nmove - 1) / 32) * 32; c0 >= 0 && nmove > 0; c0 -= 32) {
    const int j = pos + c0 + lane;
    TopEnt t;
    const bool act = (c0 + lane) < nmove;
    if (act) t = top[j];
    __syncwarp();
    if (act) top[j + 1] = t;
    __syncwarp();
  }
  if (lane == 0) top[pos] = x;
  __syncwarp();
  cnt = ncnt;
}

// Offer one candidate per lane (pass = lane has one) to the warp's list.
__device__ __forceinline__ void top_offer(TopEnt* top, int& cnt, int k, bool has, const TopEnt& x) {
  bool pass = has;
  if (pass && cnt >= k) pass = ent_before(x, top[k - 1]);
  u32 mask = __ballot_sync(FULLMASK, pass);
  while (mask) {
    const int src = __ffs(mask) - 1;
    mask &= mask - 1;
    TopEnt y;
    y.num = __shfl_sync(FULLMASK, x.num, src);
    y.den = __shfl_sync(FULLMASK, x.den, src);
    y.c = __shfl_sync(FULLMASK, x.c, src);
    y.cn = __shfl_sync(FULLMASK, x.cn, src);
    top_insert(top, cnt, k, y);
  }
}

// Position of the n-th (0-based) set bit of mask (mask has more than n bits).
__device__ __forceinline__ int nth_set_bit(u32 mask, int n) {
  int pos = 0;
#pragma unroll
  for (int w = 16; w > 0; w >>= 1) {
    const int cnt = __popc(mask & ((1u << w) - 1u));
    if (cnt <= n) {
      n -= cnt;
      mask >>= w;
      pos += w;
    }
  }
  return pos;
}

// The measures that read |Gamma_c| do not increase with it, and |Gamma_c| is
// at least the count v (each counted intermediary is a neighbour of c), so
// the key taken with |Gamma_c| = v bounds the true key from above.  True when
// that bound already ranks strictly below tn/td: the pair cannot pass and
// |Gamma_c| need not be read.
__device__ __forceinline__ bool bound_below(int measure, u64 v, u64 da, u64 tn, u64 td) {
  u64 un, ud;
  make_key(measure, v, da, v, un, ud);
  const u64 lh = __umul64hi(un, td), ll = un * td;
  const u64 rh = __umul64hi(tn, ud), rl = tn * ud;
  return lh < rh || (lh == rh && ll < rl);
}

// Key of candidate c (count or fixed-point sum v) and whether it can enter the
// selection: S_th (strict), then in the global mode the admission threshold
// T, in the per-source mode the warp's full top-k list (bound test only; the
// exact test is top_offer's).
template <typename V, int MODE>
__device__ __forceinline__ bool key_passes(const ScanArgs& A, const Thresh& T, int a, u64 da,
                                           int c, V v, const TopEnt* top, int tcnt, u64& num,
                                           u64& den, int dc_in = -1) {
  u64 dc = 0;
  if (needs_dc(A.measure)) {
    if (MODE == 0 && T.valid && bound_below(A.measure, (u64)v, da, T.num, T.den)) return false;
    if (MODE == 1 && tcnt >= A.k &&
        bound_below(A.measure, (u64)v, da, top[A.k - 1].num, top[A.k - 1].den))
      return false;
    dc = dc_in >= 0 ? (u64)dc_in : (u64)__ldg(A.deg + c);
  }
  make_key(A.measure, (u64)v, da, dc, num, den);
  bool pass = !A.thr_check || key_value(A.measure, num, den, (u64)v, A.fixbits) > A.threshold;
  if (MODE == 0 && pass && T.valid) pass = before(num, den, a, c, T.num, T.den, T.u, T.v);
  return pass;
}

// Global mode with a valid admission threshold T: the smallest count (or
// fixed-point sum) v that can still reach T for a source of degree da.  Every
// key grows with v, and for the measures that read |Gamma_c| the bound of
// bound_below does too, so the counters below the floor are rejected by one
// comparison.  Counts never exceed da (each counted intermediary is a
// neighbour of the source); da + 1 means no counter can pass.
__device__ __forceinline__ u64 count_floor(int measure, u64 da, const Thresh& T) {
  if (!T.valid) return 1;
  if (!needs_dc(measure)) return (T.num + T.den - 1) / T.den;  // key = v / 1
  u64 lo = 1, hi = da + 1;
  while (lo < hi) {
    const u64 mid = (lo + hi) >> 1;
    if (bound_below(measure, mid, da, T.num, T.den)) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Score the live entries among four table slots per lane (value 0 = empty or
// dead): the live ones are first gathered across the warp, then scored 32 at
// a time with every lane busy.  Returns true if the global buffer
// overflowed.
template <typename V, int MODE>
__device__ __forceinline__ bool score_chunk(const ScanArgs& A, const Thresh& T, int a, u64 da,
                                            const int (&c4)[4], const V (&v4)[4], TopEnt* top,
                                            int& tcnt, u64& n_cand) {
  const int lane = lane_id();
  u32 m[4];
  int pre[5];
  pre[0] = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    m[j] = __ballot_sync(FULLMASK, v4[j] != 0);
    pre[j + 1] = pre[j] + __popc(m[j]);
  }
  const int L = pre[4];
  bool fail = false;
  for (int r0 = 0; r0 < L; r0 += 32) {
    const int t = r0 + lane;
    const int j = (t >= pre[1]) + (t >= pre[2]) + (t >= pre[3]);
    const u32 mj = j == 0 ? m[0] : (j == 1 ? m[1] : (j == 2 ? m[2] : m[3]));
    const int src = t < L ? nth_set_bit(mj, t - pre[j]) : 0;
    int c = 0;
    V v = 0;
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      const int cc = __shfl_sync(FULLMASK, c4[jj], src);
      const V vv = __shfl_sync(FULLMASK, v4[jj], src);
      if (jj == j) {
        c = cc;
        v = vv;
      }
    }
    const bool live = t < L;
    u64 num = 0, den = 1;
    bool pass = false;
    if (live) {
      ++n_cand;
      pass = key_passes<V, MODE>(A, T, a, da, c, v, top, tcnt, num, den);
    }
    if (MODE == 0) {
      fail |= admit_global(A, pass, num, den, a, c);
    } else {
      TopEnt x;
      x.num = num;
      x.den = den;
      x.c = c;
      x.cn = sizeof(V) == 8 ? 0 : (int)v;
      top_offer(top, tcnt, A.k, pass, x);
    }
  }
  return fail;
}

// Score one candidate per lane (live: the lane has one) and hand it to the
// sink; warp-collective.  Returns true if the global buffer overflowed.
template <typename V, int MODE>
__device__ __forceinline__ bool score_one(const ScanArgs& A, const Thresh& T, int a, u64 da,
                                          bool live, int c, V v, TopEnt* top, int& tcnt,
                                          u64& n_cand, int dc_in = -1) {
  u64 num = 0, den = 1;
  bool pass = false;
  if (live) {
    ++n_cand;
    pass = key_passes<V, MODE>(A, T, a, da, c, v, top, tcnt, num, den, dc_in);
  }
  if (MODE == 0) return admit_global(A, pass, num, den, a, c);
  TopEnt x;
  x.num = num;
  x.den = den;
  x.c = c;
  x.cn = sizeof(V) == 8 ? 0 : (int)v;
  top_offer(top, tcnt, A.k, pass, x);
  return false;
}

template <typename V>
__device__ __forceinline__ void load4(const V* p, V (&v)[4]);
template <typename V>
__device__ __forceinline__ void zero4(V* p);

// Score the 128-slot hash chunk [base0, base0 + 128) of a table (lane l owns
// slots 4l..4l+3; slots at or beyond nslots are absent) and leave it empty.
// The live entries are first packed to the front of the chunk in place, so
// they are scored 32 at a time with every lane busy.
template <typename V, int MODE>
__device__ __forceinline__ bool score_hash_chunk(const ScanArgs& A, const Thresh& T, int a, u64 da,
                                                 int* keys, V* vals, int base0, int nslots,
                                                 TopEnt* top, int& tcnt, u64& n_cand) {
  const int lane = lane_id();
  const int base = base0 + lane * 4;
  int4 k4 = make_int4(0, 0, 0, 0);
  V v4[4] = {0, 0, 0, 0};
  if (base < nslots) {
    k4 = *reinterpret_cast<const int4*>(keys + base);
    load4<V>(vals + base, v4);
  }
  const int kk[4] = {k4.x, k4.y, k4.z, k4.w};
  int nl = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) nl += (v4[j] != 0) ? 1 : 0;
  int incl = nl;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(FULLMASK, incl, o);
    if (lane >= o) incl += t;
  }
  const int L = __shfl_sync(FULLMASK, incl, 31);
  __syncwarp();
  if (L > 0) {
    int pos = base0 + incl - nl;
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (v4[j] != 0) {
        keys[pos] = kk[j];
        vals[pos] = v4[j];
        ++pos;
      }
  }
  __syncwarp();
  bool fail = false;
  for (int r0 = 0; r0 < L; r0 += 32) {
    const int t = r0 + lane;
    const bool live = t < L;
    const int c = live ? keys[base0 + t] - 1 : 0;
    const V v = live ? vals[base0 + t] : (V)0;
    fail |= score_one<V, MODE>(A, T, a, da, live, c, v, top, tcnt, n_cand);
  }
  __syncwarp();
  if (base < nslots) {
    *reinterpret_cast<int4*>(keys + base) = make_int4(0, 0, 0, 0);
    zero4<V>(vals + base);
  }
  __syncwarp();
  return fail;
}

// Score the touched counters of 32 bitmap words [w0, w0 + 32) of a dense
// window (words at or beyond nwords are absent), clearing counters and bits.
// Bit i marks the counter of vertex lg + i, held at position swz(i).
// The set bits are first numbered across the warp (prefix sum of the word
// popcounts), so every round scores 32 touched counters whatever their
// spread over the words.
template <typename V, int MODE>
__device__ __forceinline__ bool score_dense_words(const ScanArgs& A, const Thresh& T, int a, u64 da,
                                                  V* dense, u32* bits, int w0, int nwords, int lg,
                                                  TopEnt* top, int& tcnt, u64& n_cand) {
  const int lane = lane_id();
  const int wi = w0 + lane;
  u32 w = 0;
  if (wi < nwords) {
    w = bits[wi];
    if (w) bits[wi] = 0;
  }
  const int cnt = __popc(w);
  int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(FULLMASK, incl, o);
    if (lane >= o) incl += t;
  }
  const int L = __shfl_sync(FULLMASK, incl, 31);
  const int excl = incl - cnt;
  bool fail = false;
  for (int r0 = 0; r0 < L; r0 += 32) {  // warp-uniform trips
    const int t = r0 + lane;
    // owner: the last lane j with excl_j <= t (it has a set bit when t < L)
    int j = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
      const int e = __shfl_sync(FULLMASK, excl, j + step);
      if (e <= t) j += step;
    }
    const u32 wj = __shfl_sync(FULLMASK, w, j);
    const int ej = __shfl_sync(FULLMASK, excl, j);
    bool live = false;
    int c = 0;
    V v = 0;
    if (t < L) {
      const int i = (w0 + j) * 32 + nth_set_bit(wj, t - ej);
      v = dense[swz(i)];
      dense[swz(i)] = 0;
      c = lg + i;
      live = v != 0;  // 0: a first-order neighbour cleared by the exclusion
    }
    fail |= score_one<V, MODE>(A, T, a, da, live, c, v, top, tcnt, n_cand);
  }
  return fail;
}

// Global mode, large tier: counters at or above the count floor ("survivors")
// still need the exact test, most of them |Gamma_c| too.  Each warp queues
// them in registers (lane i holds entry i; qn entries, warp-uniform), the
// degree load issued as the entry is queued, and tests 32 at a time, so the
// loads overlap the scan instead of stalling it.
template <typename V>
__device__ __forceinline__ bool survivors_flush(const ScanArgs& A, const Thresh& T, int a, u64 da,
                                                int& qn, int qc, V qv, int qd) {
  u64 unused = 0;
  int tcnt = 0;
  const bool fail =
      score_one<V, 0>(A, T, a, da, lane_id() < qn, qc, qv, nullptr, tcnt, unused, qd);
  qn = 0;
  return fail;
}

template <typename V>
__device__ __forceinline__ bool survivors_push(const ScanArgs& A, const Thresh& T, int a, u64 da,
                                               bool live, int c, V v, int& qn, int& qc, V& qv,
                                               int& qd) {
  const u32 m = __ballot_sync(FULLMASK, live);
  if (m == 0) return false;
  const int k = __popc(m);
  bool fail = false;
  if (qn + k > 32) fail = survivors_flush<V>(A, T, a, da, qn, qc, qv, qd);
  const int t = lane_id() - qn;  // this lane receives new entry t
  const bool recv = t >= 0 && t < k;
  const int src = recv ? nth_set_bit(m, t) : lane_id();
  const int nc = __shfl_sync(FULLMASK, c, src);
  const V nv = __shfl_sync(FULLMASK, v, src);
  if (recv) {
    qc = nc;
    qv = nv;
    qd = needs_dc(A.measure) ? __ldg(A.deg + nc) : 0;
  }
  qn += k;
  return fail;
}

// Global mode: 128 consecutive dense counters per warp (positions [base0,
// base0 + 128), four per lane), cleared; the ones at or above vmin are queued.
// Position p holds the counter of vertex lg + swz(p).
template <typename V>
__device__ __forceinline__ bool score_dense_linear(const ScanArgs& A, const Thresh& T, int a,
                                                   u64 da, V* dense, int base0, int npos, int lg,
                                                   u64 vmin, u64& n_cand, int& qn, int& qc,
                                                   V& qv, int& qd) {
  const int base = base0 + lane_id() * 4;
  V v4[4] = {0, 0, 0, 0};
  if (base < npos) {
    load4<V>(dense + base, v4);
    if ((v4[0] | v4[1] | v4[2] | v4[3]) != 0) zero4<V>(dense + base);
  }
  bool any = false;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    n_cand += v4[j] != 0 ? 1 : 0;
    any |= v4[j] != 0 && (u64)v4[j] >= vmin;
  }
  if (!__any_sync(FULLMASK, any)) return false;
  bool fail = false;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const bool live = v4[j] != 0 && (u64)v4[j] >= vmin;
    fail |= survivors_push<V>(A, T, a, da, live, lg + swz(base + j), v4[j], qn, qc, qv, qd);
  }
  return fail;
}

// Lane-parallel tests on packed counters (SWAR).  nonzero8 / nonzero16: the
// number of nonzero 8-bit / 16-bit lanes of x (a lane's low bits plus the
// all-ones low mask reach its top bit iff they are nonzero; OR-ing x covers a
// set top bit; no carry leaves the lane).  any_ge8: whether some 8-bit lane
// of x is >= m (1 <= m <= 256): every byte, widened to a 16-bit lane, plus
// 256 - m reaches bit 8 iff byte >= m, and stays below 2^16.
__device__ __forceinline__ int nonzero8(u32 x) {
  return __popc((((x & 0x7f7f7f7fu) + 0x7f7f7f7fu) | x) & 0x80808080u);
}
__device__ __forceinline__ int nonzero16(u32 x) {
  return __popc((((x & 0x7fff7fffu) + 0x7fff7fffu) | x) & 0x80008000u);
}
__device__ __forceinline__ bool any_ge8(u32 x, u32 cth) {
  const u32 e = x & 0x00ff00ffu, o = (x >> 8) & 0x00ff00ffu;
  return (((e + cth) | (o + cth)) & 0x01000100u) != 0;
}

// The same for 8-bit counters, four per word (sources of degree <= 255): 256
// positions per warp, eight per lane.
__device__ __forceinline__ bool score_dense8_linear(const ScanArgs& A, const Thresh& T, int a,
                                                    u64 da, u32* words, int base0, int npos,
                                                    int lg, u64 vmin, u64& n_cand, int& qn,
                                                    int& qc, u32& qv, int& qd) {
  const int base = base0 + lane_id() * 8;
  uint2 w = make_uint2(0, 0);
  if (base < npos) {
    w = *reinterpret_cast<const uint2*>(words + (base >> 2));
    if ((w.x | w.y) != 0) *reinterpret_cast<uint2*>(words + (base >> 2)) = make_uint2(0, 0);
  }
  n_cand += (u64)(nonzero8(w.x) + nonzero8(w.y));
  const u32 m = (u32)min(max(vmin, (u64)1), (u64)256);  // counters are nonzero and below 256
  const u32 cth = (256u - m) * 0x00010001u;
  if (!__any_sync(FULLMASK, any_ge8(w.x, cth) || any_ge8(w.y, cth))) return false;
  bool fail = false;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const u32 v = ((j < 4 ? w.x : w.y) >> ((j & 3) << 3)) & 0xffu;
    const bool live = v >= m;
    fail |= survivors_push<u32>(A, T, a, da, live, lg + swz(base + j), v, qn, qc, qv, qd);
  }
  return fail;
}

// Mark of a first-order neighbour in the high word of a 64-bit counter pair:
// added (not stored) during the insert phase, so its order against the
// inserts does not matter.
constexpr u32 kFirstOrder64 = 0x80000000u;

// The same for 64-bit counters kept as two arrays of 32-bit halves (position
// p: low word lo[p], high word hi[p]), so the low-word atomics of the scan
// spread over all banks.
__device__ __forceinline__ bool score_dense64_linear(const ScanArgs& A, const Thresh& T, int a,
                                                     u64 da, u32* lo, u32* hi, int base0, int npos,
                                                     int lg, u64 vmin, u64& n_cand, int& qn,
                                                     int& qc, u64& qv, int& qd) {
  const int base = base0 + lane_id() * 4;
  uint4 l4 = make_uint4(0, 0, 0, 0), h4 = make_uint4(0, 0, 0, 0);
  if (base < npos) {
    l4 = *reinterpret_cast<const uint4*>(lo + base);
    h4 = *reinterpret_cast<const uint4*>(hi + base);
    if ((l4.x | l4.y | l4.z | l4.w | h4.x | h4.y | h4.z | h4.w) != 0) {
      *reinterpret_cast<uint4*>(lo + base) = make_uint4(0, 0, 0, 0);
      *reinterpret_cast<uint4*>(hi + base) = make_uint4(0, 0, 0, 0);
    }
  }
  // a first-order neighbour carries the mark kFirstOrder64 in its high word
  // (real sums stay below 2^63); it is neither a candidate nor scored
  const u32 hw[4] = {h4.x, h4.y, h4.z, h4.w};
  const u64 v4[4] = {(u64)l4.x | ((u64)h4.x << 32), (u64)l4.y | ((u64)h4.y << 32),
                     (u64)l4.z | ((u64)h4.z << 32), (u64)l4.w | ((u64)h4.w << 32)};
  const u64 vm = max(vmin, (u64)1);
  bool any = false;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const bool first = (hw[j] & kFirstOrder64) != 0;
    n_cand += v4[j] != 0 && !first ? 1 : 0;
    any |= !first && v4[j] >= vm;
  }
  if (!__any_sync(FULLMASK, any)) return false;
  bool fail = false;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const bool live = (hw[j] & kFirstOrder64) == 0 && v4[j] >= vm;
    fail |= survivors_push<u64>(A, T, a, da, live, lg + swz(base + j), v4[j], qn, qc, qv, qd);
  }
  return fail;
}

// The same for 16-bit counters, two per word (count measures, counts below
// 2^16): 256 positions per warp, eight per lane.
__device__ __forceinline__ bool score_dense16_linear(const ScanArgs& A, const Thresh& T, int a,
                                                     u64 da, u32* words, int base0, int npos,
                                                     int lg, u64 vmin, u64& n_cand, int& qn,
                                                     int& qc, u32& qv, int& qd) {
  const int base = base0 + lane_id() * 8;
  uint4 w = make_uint4(0, 0, 0, 0);
  if (base < npos) {
    w = *reinterpret_cast<const uint4*>(words + (base >> 1));
    if ((w.x | w.y | w.z | w.w) != 0)
      *reinterpret_cast<uint4*>(words + (base >> 1)) = make_uint4(0, 0, 0, 0);
  }
  n_cand += (u64)(nonzero16(w.x) + nonzero16(w.y) + nonzero16(w.z) + nonzero16(w.w));
  const u32 m = (u32)min(max(vmin, (u64)1), (u64)65536);  // counters are nonzero
  auto top = [](u32 x) { return max(x & 0xffffu, x >> 16); };
  if (!__any_sync(FULLMASK, max(max(top(w.x), top(w.y)), max(top(w.z), top(w.w))) >= m))
    return false;
  const u32 ww[4] = {w.x, w.y, w.z, w.w};
  bool fail = false;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const u32 v = (ww[j >> 1] >> ((j & 1) << 4)) & 0xffffu;
    const bool live = v >= m;
    fail |= survivors_push<u32>(A, T, a, da, live, lg + swz(base + j), v, qn, qc, qv, qd);
  }
  return fail;
}

// Global mode: the 128-slot hash chunk [base0, base0 + 128), cleared; the
// live slots at or above vmin are queued.
template <typename V>
__device__ __forceinline__ bool score_hash_linear(const ScanArgs& A, const Thresh& T, int a,
                                                  u64 da, int* keys, V* vals, int base0, int nslots,
                                                  u64 vmin, u64& n_cand, int& qn, int& qc, V& qv,
                                                  int& qd) {
  const int base = base0 + lane_id() * 4;
  int4 k4 = make_int4(0, 0, 0, 0);
  V v4[4] = {0, 0, 0, 0};
  if (base < nslots) {
    k4 = *reinterpret_cast<const int4*>(keys + base);
    if ((k4.x | k4.y | k4.z | k4.w) != 0) {
      load4<V>(vals + base, v4);
      *reinterpret_cast<int4*>(keys + base) = make_int4(0, 0, 0, 0);
      zero4<V>(vals + base);
    }
  }
  const int kk[4] = {k4.x, k4.y, k4.z, k4.w};
  bool any = false;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    n_cand += v4[j] != 0 ? 1 : 0;
    any |= v4[j] != 0 && (u64)v4[j] >= vmin;
  }
  if (!__any_sync(FULLMASK, any)) return false;
  bool fail = false;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const bool live = v4[j] != 0 && (u64)v4[j] >= vmin;
    fail |= survivors_push<V>(A, T, a, da, live, kk[j] - 1, v4[j], qn, qc, qv, qd);
  }
  return fail;
}

// Vector loads / stores of four consecutive table slots.
template <typename V>
__device__ __forceinline__ void load4(const V* p, V (&v)[4]) {
  if (sizeof(V) == 8) {
    const ulonglong2 a = reinterpret_cast<const ulonglong2*>(p)[0];
    const ulonglong2 b = reinterpret_cast<const ulonglong2*>(p)[1];
    v[0] = (V)a.x;
    v[1] = (V)a.y;
    v[2] = (V)b.x;
    v[3] = (V)b.y;
  } else {
    const uint4 a = *reinterpret_cast<const uint4*>(p);
    v[0] = (V)a.x;
    v[1] = (V)a.y;
    v[2] = (V)a.z;
    v[3] = (V)a.w;
  }
}

template <typename V>
__device__ __forceinline__ void zero4(V* p) {
  if (sizeof(V) == 8) {
    reinterpret_cast<ulonglong2*>(p)[0] = make_ulonglong2(0, 0);
    reinterpret_cast<ulonglong2*>(p)[1] = make_ulonglong2(0, 0);
  } else {
    *reinterpret_cast<uint4*>(p) = make_uint4(0, 0, 0, 0);
  }
}

// Sum over the common neighbours b of (u, v) with |Gamma_b| <= cap of 1
// (wt null: the count) or of wt[|Gamma_b|] (the AA / RA fixed-point weight,
// so the sum is the key the scan accumulated: integer addition does not
// depend on the order).  One warp per pair; every lane returns the total.
// x is the endpoint of smaller degree.  Short Gamma_x (or a much longer
// Gamma_y): each lane takes elements b of Gamma_x (hub test from the arc
// table) and looks the other endpoint up in the shorter of Gamma_b and
// Gamma_y.  Two long lists of similar length: a merge-path intersection
// across the lanes.
__device__ __forceinline__ u64 pair_common(int u, int v, const int* __restrict__ off,
                                           const int* __restrict__ idx,
                                           const int* __restrict__ deg,
                                           const Arc* __restrict__ arc, int cap,
                                           const u64* __restrict__ wt) {
  const int lane = lane_id();
  int x = u, y = v;
  if (off[x + 1] - off[x] > off[y + 1] - off[y]) {
    const int t = x;
    x = y;
    y = t;
  }
  const int xs = off[x], xe = off[x + 1];
  const int ys = off[y], ye = off[y + 1];
  const int dy = ye - ys;
  const int dx = xe - xs;
  u64 c = 0;
  if (dx <= 64 || dy > 16 * dx || cap < 256) {
    // short Gamma_x, a much longer Gamma_y or a low hub limit (most b are
    // skipped without a search): look each b of Gamma_x up
    for (int e = xs + lane; e < xe; e += 32) {
      const Arc t = arc[e];  // b = t.w, |Gamma_b| = t.z, Gamma_b ends at t.y
      const int b = t.w, db = t.z;
      if (db > cap) continue;
      bool hit;
      if (db <= dy) {
        const int be = t.y, bs = be - db;
        const int p = lower_bound_interp(idx, bs, be, y);
        hit = p < be && __ldg(idx + p) == y;
      } else {
        const int p = lower_bound_interp(idx, ys, ye, b);
        hit = p < ye && __ldg(idx + p) == b;
      }
      if (hit) c += wt ? __ldg(wt + db) : 1ull;
    }
  } else {
    // comparable long lists: both walked in 32-element tiles, one element
    // per lane.  Each lane looks its Gamma_x element up in the current Gamma_y
    // tile (binary search over the lanes); then the tile with the smaller last
    // element moves on (both on a tie), with the next tiles already loading.
    // A common element is in both tiles during exactly one step.
    const int* X = idx + xs;
    const int* Y = idx + ys;
    int i = 0, j = 0;
    int xv = lane < dx ? __ldg(X + lane) : INT_MAX;
    int yv = lane < dy ? __ldg(Y + lane) : INT_MAX;
    int xn = 32 + lane < dx ? __ldg(X + 32 + lane) : INT_MAX;
    int yn = 32 + lane < dy ? __ldg(Y + 32 + lane) : INT_MAX;
    while (i < dx && j < dy) {  // warp-uniform
      int p = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1)
        if (__shfl_sync(FULLMASK, yv, p + step - 1) < xv) p += step;
      const int yp = __shfl_sync(FULLMASK, yv, p);  // every lane takes part
      bool hit = xv != INT_MAX && yp == xv;
      int db = 0;
      if (hit && (cap < INT_MAX || wt)) {
        db = __ldg(deg + xv);
        hit = db <= cap;
      }
      if (hit) c += wt ? __ldg(wt + db) : 1ull;
      const int lx = __shfl_sync(FULLMASK, xv, 31), ly = __shfl_sync(FULLMASK, yv, 31);
      if (lx <= ly) {
        i += 32;
        xv = xn;
        xn = i + 32 + lane < dx ? __ldg(X + i + 32 + lane) : INT_MAX;
      }
      if (ly <= lx) {
        j += 32;
        yv = yn;
        yn = j + 32 + lane < dy ? __ldg(Y + j + 32 + lane) : INT_MAX;
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(FULLMASK, c, o);
  return c;
}

}  // namespace lp
