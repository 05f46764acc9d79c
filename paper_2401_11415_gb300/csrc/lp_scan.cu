// lp_scan.cu -- work estimate, binning and the wedge-scan kernels.
//
// For every source a the scan accumulates, for each second-order vertex c,
// the paths a -> b -> c through intermediaries b with |Gamma_b| <= L_H
// (Algorithm 1: the loop over G.out(a) with the hub test, then scanEdges;
// Sections 4.1.1-4.1.3 and 4.2.1).  It then drops the first-order neighbours
// of a (Section 4.1.4), scores each surviving c with Eq. 1-9 (Section 4.1.5)
// and hands the pair to the selection (Section 4.1.6).
//
// GPU design (replaces the paper's OpenMP loop with per-thread dense tables):
//  * k_estimate: 32 sources per warp (one per lane; sources of high degree
//    are summed by the whole warp) compute the exact wedge count W(a) from
//    the per-arc table -- hub arcs add nothing and their adjacency lists are
//    never read -- and bin each source:
//      - W <= 256: warp tier, a per-warp shared-memory table of 2W..4W slots;
//      - W <= 1024: medium tier, one 4-warp CTA with a 2048-slot table;
//      - W <= 8192: one 32-warp CTA item over the whole vertex range;
//      - larger: the c-range is cut into items; each item is a 32-warp CTA
//        with either a shared-memory hash (split by vertex id, a binary search
//        per arc finds the sub-range) or dense shared-memory counters over an
//        id window (hubs whose second-order set is a large part of the graph).
//    Queue appends and statistics are aggregated per warp.
//  * Wedge loops: a warp holds 32 arcs (one int4 per lane).  Suffixes of 64
//    or more ids are streamed by the whole warp with four loads in flight per
//    lane; the short ones are concatenated (prefix sum over the lanes) and
//    walked 32 wedges at a time, two windows per step, so every lane issues
//    coalesced reads whatever the intermediary degrees are.
//  * Tables hold key c + 1 (0 = empty) and are left all-zero after each
//    source, so no table is cleared before use.  Counts are u32 (CN family);
//    AA and RA accumulate u64 fixed-point weights round(2^F / ln|Gamma_b|)
//    and round(2^F / |Gamma_b|): integer addition is associative, so the
//    sums do not depend on thread order.
#include <float.h>
#include <limits.h>
#include <math.h>

#include <algorithm>
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

// The graph's weight tables, by degree: wt[d] (AA) and wt[dmax + 1 + d] (RA).
__global__ void k_build_weights(int dmax, int fixbits, u64* __restrict__ wt) {
  for (int d = blockIdx.x * blockDim.x + threadIdx.x; d <= dmax; d += gridDim.x * blockDim.x) {
    wt[d] = fixed_weight(LP_AA, d, fixbits);
    wt[(size_t)dmax + 1 + d] = fixed_weight(LP_RA, d, fixbits);
  }
}

cudaError_t launch_build_weights(int dmax, int fixbits, u64* wt, cudaStream_t st) {
  const int threads = 256;
  const int blocks = (int)std::min<long long>(((long long)dmax + threads) / threads, 4096);
  k_build_weights<<<blocks, threads, 0, st>>>(dmax, fixbits, wt);
  return cudaGetLastError();
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

// --------------------------------------------------------------- estimate --

struct TierStats {
  u64 w[3], a[3], k[3];
  u64 dense;
};

// Per record r (global mode: source r; per-source mode: sources[r]).
// Warp records: {r, lo, hi, W | 1<<30}.  Medium and large items:
// {r, lo, hi, kind | logcap << 8}.  grp[r] = (first item, item count) in the
// per-source mode.
template <int MODE, bool V64>
__global__ void __launch_bounds__(256) k_estimate(ScanArgs A, int n_rec, int4* __restrict__ warpq,
                                                  int4* __restrict__ medq,
                                                  int4* __restrict__ itemq, u64 itemq_cap,
                                                  int2* __restrict__ grp) {
  const int lane = lane_id();
  const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const u32 lt = (1u << lane) - 1u;
  TierStats ts;
  for (int i = 0; i < 3; ++i) ts.w[i] = ts.a[i] = ts.k[i] = 0;
  ts.dense = 0;
  for (int base = gwarp * 32; base < n_rec; base += nwarps * 32) {
    const bool valid = base + lane < n_rec;
    // global mode: the record is the source itself (within the range)
    const int r = MODE ? base + lane : A.rec_base + base + lane;
    int a = 0, e0 = 0, e1 = 0;
    if (valid) {
      a = MODE ? A.sources[r] : r;
      e0 = A.off[a];
      e1 = A.off[a + 1];
    }
    u64 W = 0;
    u32 kept = 0;
    // the second-order ids span [nlo, nhi]: each kept list (or suffix) is
    // sorted, so its first and last ids bound it
    int nlo = INT_MAX, nhi = -1;
    auto span_arc = [&](const Arc& t, int& l, int& h) {
      const int s0 = MODE ? t.y - t.z : t.x + 1;
      if (s0 < t.y) {
        l = min(l, __ldg(A.idx + s0));
        h = max(h, __ldg(A.idx + t.y - 1));
      }
    };
    const bool small = valid && (e1 - e0) <= 64;
    if (small) {
      for (int e = e0; e < e1; ++e) {
        const Arc t = A.arc[e];
        if (t.z <= A.cap) {
          W += MODE ? (u64)(t.z - 1) : (u64)(t.y - t.x - 1);
          ++kept;
          span_arc(t, nlo, nhi);
        }
      }
    }
    u32 big = __ballot_sync(FULLMASK, valid && !small);
    while (big) {
      const int j = __ffs(big) - 1;
      big &= big - 1;
      const int j0 = __shfl_sync(FULLMASK, e0, j), j1 = __shfl_sync(FULLMASK, e1, j);
      u64 Wj = 0;
      u32 kj = 0;
      int lj = INT_MAX, hj = -1;
      // four arcs per lane at a time, so that a hub's walk keeps eight
      // independent list reads in flight instead of two dependent ones
      int e = j0 + lane;
      for (; e + 96 < j1; e += 128) {
        Arc t[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) t[u] = A.arc[e + 32 * u];
        int l4[4], h4[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int s0 = MODE ? t[u].y - t[u].z : t[u].x + 1;
          const bool use = t[u].z <= A.cap && s0 < t[u].y;
          l4[u] = use ? __ldg(A.idx + s0) : INT_MAX;
          h4[u] = use ? __ldg(A.idx + t[u].y - 1) : -1;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (t[u].z <= A.cap) {
            Wj += MODE ? (u64)(t[u].z - 1) : (u64)(t[u].y - t[u].x - 1);
            ++kj;
          }
          lj = min(lj, l4[u]);
          hj = max(hj, h4[u]);
        }
      }
      for (; e < j1; e += 32) {
        const Arc t = A.arc[e];
        if (t.z <= A.cap) {
          Wj += MODE ? (u64)(t.z - 1) : (u64)(t.y - t.x - 1);
          ++kj;
          span_arc(t, lj, hj);
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        Wj += __shfl_xor_sync(FULLMASK, Wj, o);
        kj += __shfl_xor_sync(FULLMASK, kj, o);
      }
      lj = __reduce_min_sync(FULLMASK, lj);
      hj = __reduce_max_sync(FULLMASK, hj);
      if (lane == j) {
        W = Wj;
        kept = kj;
        nlo = lj;
        nhi = hj;
      }
    }
    // binning (items cover only the source's second-order id range)
    const int lo = W > 0 ? max(MODE ? 0 : a + 1, nlo) : (MODE ? 0 : a + 1);
    const int hi = W > 0 ? min(A.n, nhi + 1) : A.n;
    int tier = -1;
    if (valid && W > 0) tier = W <= (u64)A.warp_max ? 0 : (W <= (u64)A.med_max ? 1 : 2);
    if (tier >= 0) {
      ts.w[tier] += W;
      ts.a[tier] += (u64)(e1 - e0);
      ts.k[tier] += kept;
    }
    if (MODE && valid) {
      grp[r] = make_int2(-1, 0);
      if (W == 0) A.out_cnt[r] = 0;
    }
    // warp tier
    {
      const u32 m = __ballot_sync(FULLMASK, tier == 0);
      if (m) {
        const int leader = __ffs(m) - 1;
        u64 q = 0;
        if (lane == leader) q = atomicAdd(&A.ctr->nwarp, (u64)__popc(m));
        q = __shfl_sync(FULLMASK, q, leader);
        if (tier == 0) warpq[q + __popc(m & lt)] = make_int4(r, lo, hi, (int)W | (1 << 30));
      }
    }
    // medium tier
    {
      const u32 m = __ballot_sync(FULLMASK, tier == 1);
      if (m) {
        const int leader = __ffs(m) - 1;
        u64 q = 0;
        if (lane == leader) q = atomicAdd(&A.ctr->nmed, (u64)__popc(m));
        q = __shfl_sync(FULLMASK, q, leader);
        if (tier == 1) {
          const int logcap = max(6, min(11, ceil_log2(2 * W)));
          const int kind = MODE ? kItemSingle : 0;
          medq[q + __popc(m & lt)] =
              make_int4(r, lo, hi, kind | kItemWhole | (logcap << 8) | (1 << 29));
        }
      }
    }
    // large tier: P items per source
    int P = 0, kind = 0, logcap = 0, Gd = 1, bspan = A.big_span;
    u64 nsub = 1;  // hash items: sub-ranges of the source
    if (tier == 2) {
      const u64 span = (u64)(hi - lo);
      if (W <= (u64)A.cta_max) {
        P = 1;
        logcap = max(10, ceil_log2(2 * W));
      } else {
        // 16-bit dense counters hold twice as many 8-bit ones; a count never
        // exceeds the kept arcs of the source
        const bool d8 = MODE == 0 && A.dense16 && kept <= 255;
        bspan = d8 ? 2 * A.big_span : A.big_span;
        const u64 sh = (W + A.split_target - 1) / A.split_target;
        const u64 sd = (span + bspan - 1) / bspan;
        const u64 pdi = max((u64)1, min(sd, (W + A.item_wedges - 1) / A.item_wedges));
        // relative costs (measured on R-MAT sweeps): a dense window is
        // scanned whole, a split hash item re-reads every arc; in the global
        // mode a dense 64-bit window holds an eighth of the ids of an 8-bit
        // one, which tips AA / RA further towards hash items
        const double hw = (MODE == 0 && V64) ? 0.6 : 1.0;
        const double cost_h =
            hw * ((double)sh * (kept * 24.0 + (1 << A.split_logcap) / 4.0) + W * 3.0);
        const double cost_d =
            (double)sd * (kept * 2.0 + bspan / 8.0) + (double)W + (double)pdi * kept * 24.0;
        logcap = A.split_logcap;
        if (cost_d < cost_h || A.no_split) {  // dense items never overflow
          Gd = (int)min((sd + pdi - 1) / pdi, (u64)kMaxSweep);
          P = (int)((sd + Gd - 1) / Gd);
          kind = kItemDense | (d8 ? kItemD8 : 0);
        } else {
          // sub-ranges of about split_target wedges; in the global mode an
          // item sweeps Gd consecutive ones (per-arc cursors carried from
          // range to range), items of about item_wedges wedges
          const u64 ps = min(sh, span);
          const u64 ph = MODE == 0 ? max((u64)1, min(ps, (W + A.item_wedges - 1) / A.item_wedges)) : ps;
          Gd = (int)min((ps + ph - 1) / ph, (u64)kMaxSweep);
          P = (int)((ps + Gd - 1) / Gd);
          nsub = ps;
        }
      }
      if (MODE && P == 1) kind |= kItemSingle;
      if (P == 1) kind |= kItemWhole;
      if (kind & kItemDense) ts.dense += (u64)P;
    }
    int incl = P;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(FULLMASK, incl, o);
      if (lane >= o) incl += t;
    }
    const int total = __shfl_sync(FULLMASK, incl, 31);
    if (total) {
      u64 q = 0;
      if (lane == 31) q = atomicAdd(&A.ctr->nitem, (u64)total);
      q = __shfl_sync(FULLMASK, q, 31);
      const u64 first = q + (u64)(incl - P);
      if (P && first + P <= itemq_cap) {  // else the host re-runs with a larger queue
        if (MODE) grp[r] = make_int2((int)first, P);
        const u64 span = (u64)(hi - lo);
        for (int p = 0; p < P; ++p) {
          int l2, h2;
          int gcount = 1;
          if (kind & kItemDense) {
            l2 = lo + (int)min(span, (u64)p * Gd * bspan);
            h2 = lo + (int)min(span, (u64)(p + 1) * Gd * bspan);
            gcount = (h2 - l2 + bspan - 1) / bspan;
          } else {
            const u64 s0 = (u64)p * Gd, s1 = min(nsub, (u64)(p + 1) * Gd);
            l2 = lo + (int)((span * s0) / nsub);
            h2 = lo + (int)((span * s1) / nsub);
            gcount = (int)(s1 - s0);
          }
          itemq[first + p] = make_int4(r, l2, h2, kind | (logcap << 8) | ((gcount - 1) << 16));
        }
      }
    }
  }
  // statistics, one set of atomics per warp
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ts.w[i] += __shfl_xor_sync(FULLMASK, ts.w[i], o);
      ts.a[i] += __shfl_xor_sync(FULLMASK, ts.a[i], o);
      ts.k[i] += __shfl_xor_sync(FULLMASK, ts.k[i], o);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ts.dense += __shfl_xor_sync(FULLMASK, ts.dense, o);
  if (lane == 0) {
    u64 w = 0, a = 0, k = 0;
    for (int i = 0; i < 3; ++i) {
      if (ts.w[i]) atomicAdd(&A.ctr->tier_wedges[i], ts.w[i]);
      if (ts.a[i]) atomicAdd(&A.ctr->tier_arcs[i], ts.a[i]);
      if (ts.k[i]) atomicAdd(&A.ctr->tier_kept[i], ts.k[i]);
      w += ts.w[i];
      a += ts.a[i];
      k += ts.k[i];
    }
    if (w) atomicAdd(&A.ctr->wedges, w);
    if (a) atomicAdd(&A.ctr->scanned_arcs, a);
    if (k) atomicAdd(&A.ctr->kept_arcs, k);
    if (ts.dense) atomicAdd(&A.ctr->dense_items, ts.dense);
  }
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
// existed, 2 if the table had no free slot (bounded probe count).
template <typename V>
__device__ __forceinline__ int hash_add(int* keys, V* vals, int logcap, int c, V w) {
  const u32 mask = (1u << logcap) - 1u;
  const int key = c + 1;
  u32 h = hash_slot(key, logcap);
  for (u32 probe = 0; probe <= mask; ++probe) {
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

// The floors of every source degree 0..dmax for the current threshold (one
// thread per degree); rewritten whenever the threshold changes.
__global__ void k_count_floor(int measure, int dmax, const Thresh* __restrict__ thresh,
                              u64* __restrict__ floor) {
  const Thresh T = *thresh;
  for (int d = blockIdx.x * blockDim.x + threadIdx.x; d <= dmax; d += gridDim.x * blockDim.x)
    floor[d] = count_floor(measure, (u64)d, T);
}

cudaError_t launch_count_floor(int measure, int dmax, const Thresh* thresh, u64* floor,
                               cudaStream_t st) {
  const int threads = 256;
  const int blocks = (int)std::min<long long>(((long long)dmax + threads) / threads, 4096);
  k_count_floor<<<blocks, threads, 0, st>>>(measure, dmax, thresh, floor);
  return cudaGetLastError();
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

// ------------------------------------------------------------ warp tier ---

template <bool V64, int MODE>
__global__ void __launch_bounds__(kWarpTierThreads) k_scan_warp(ScanArgs A, const int4* __restrict__ q,
                                                                u64 nq) {
  typedef typename std::conditional<V64, u64, u32>::type V;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = lane_id();
  const int wid = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  int* keys = reinterpret_cast<int*>(smem) + wid * kWarpSlots;
  V* vals = reinterpret_cast<V*>(smem + (size_t)nw * kWarpSlots * 4) + wid * kWarpSlots;
  TopEnt* top = reinterpret_cast<TopEnt*>(smem + (size_t)nw * kWarpSlots * (4 + sizeof(V))) +
                wid * (MODE ? A.k : 0);
  for (int i = lane * 4; i < kWarpSlots; i += 128) {
    *reinterpret_cast<int4*>(keys + i) = make_int4(0, 0, 0, 0);
    zero4<V>(vals + i);
  }
  __syncwarp();
  Thresh T;
  if (MODE == 0) T = *A.thresh;
  u64 n_cand = 0;
  // claims with one record of look-ahead; a claimed record is always
  // processed (once the buffer is full it fails and is re-queued)
  u64 next = 0;
  if (lane == 0) {
    if (MODE == 0 && *(volatile u32*)&A.ctr->full) next = ~0ull;
    else next = atomicAdd(&A.ctr->claim_w, 1ull);
  }
  next = __shfl_sync(FULLMASK, next, 0);
  while (next < nq) {
    const u64 qi = next;
    const int4 rec = q[qi];
    if (lane == 0) {
      if (MODE == 0 && *(volatile u32*)&A.ctr->full) next = ~0ull;
      else next = atomicAdd(&A.ctr->claim_w, 1ull);
    }
    const int r = rec.x;
    const int a = MODE ? A.sources[r] : r;
    const int W = rec.w & 0xffff;
    const int logcap = max(7, ceil_log2(2 * (u64)W));
    const int nslots = 1 << logcap;
    const int e0 = A.off[a], e1 = A.off[a + 1];
    for (int eb = e0; eb < e1; eb += 32) {
      const int e = eb + lane;
      int s = 0, len = 0;
      V w = 0;
      if (e < e1) {
        const Arc t = A.arc[e];
        if (t.z <= A.cap) {
          if (MODE == 0) {
            s = t.x + 1;
            len = t.y - s;
          } else {
            s = t.y - t.z;
            len = t.z;
          }
          if (len > 0) w = arc_weight<V>(A, t.z);
        }
      }
      scan_arcs<V>(s, len, w, A.idx, [&](int c, V wc) {
        if (MODE == 1 && c == a) return;
        hash_add<V>(keys, vals, logcap, c, wc);
      });
    }
    __syncwarp();
    for (int e = e0 + lane; e < e1; e += 32) {
      const int b = __ldg(A.idx + e);
      if (MODE == 1 || b > a) hash_kill<V>(keys, vals, logcap, b);
    }
    __syncwarp();
    const u64 da = (u64)(e1 - e0);
    bool fail = false;
    int tcnt = 0;
    for (int base0 = 0; base0 < nslots; base0 += 128)
      fail |= score_hash_chunk<V, MODE>(A, T, a, da, keys, vals, base0, nslots, top, tcnt, n_cand);
    __syncwarp();
    next = __shfl_sync(FULLMASK, next, 0);
    if (MODE == 0) {
      if (fail && lane == 0) {
        A.ctr->full = 1u;
        const u64 f = atomicAdd(&A.ctr->nfailed, 1ull);
        if (f < A.failed_cap) A.failed[f] = rec;
        else A.ctr->error = 1u;
      }
    } else {
      for (int j = lane; j < tcnt; j += 32) A.out_top[(u64)r * A.k + j] = top[j];
      if (lane == 0) A.out_cnt[r] = tcnt;
    }
    __syncwarp();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) n_cand += __shfl_xor_sync(FULLMASK, n_cand, o);
  if (lane == 0 && n_cand) atomicAdd(&A.ctr->candidates, n_cand);
}

// ------------------------------------------------------------- CTA items ---

// THREADS threads cooperate on one item (medium tier: 128 threads and a
// 2048-slot table; large tier: 1024 threads, tables and dense windows in
// table_bytes of shared memory).
template <bool V64, int MODE, int THREADS>
__global__ void __launch_bounds__(THREADS, (THREADS >= 512 ? 1 : 8)) k_scan_cta(ScanArgs A, const int4* __restrict__ q,
                                                          u64 nq, int table_bytes,
                                                          u64* __restrict__ claim) {
  typedef typename std::conditional<V64, u64, u32>::type V;
  constexpr int NW = THREADS / 32;
  extern __shared__ __align__(16) unsigned char smem[];
  const int max_slots = 1 << (ceil_log2((u64)table_bytes / (4 + sizeof(V)) + 1) - 1);
  int* keys = reinterpret_cast<int*>(smem);
  V* vals = reinterpret_cast<V*>(smem + (size_t)max_slots * 4);
  V* dense = reinterpret_cast<V*>(smem);
  TopEnt* tops = reinterpret_cast<TopEnt*>(smem + table_bytes);
  __shared__ int4 s_rec;
  __shared__ u64 s_next;
  __shared__ int s_ndistinct;
  __shared__ int s_overflow;
  __shared__ int s_fail;
  __shared__ int s_tcnt[NW];

  const int lane = lane_id();
  const int wid = threadIdx.x >> 5;
  for (int i = threadIdx.x * 16; i < table_bytes; i += THREADS * 16)
    *reinterpret_cast<int4*>(smem + i) = make_int4(0, 0, 0, 0);
  Thresh T;
  if (MODE == 0) T = *A.thresh;
  u64 n_cand = 0;
  if (threadIdx.x == 0) {
    if (MODE == 0 && *(volatile u32*)&A.ctr->full) s_next = ~0ull;
    else s_next = atomicAdd(claim, 1ull);
  }
  __syncthreads();
  for (;;) {
    const u64 qi = s_next;
    if (qi >= nq) break;
    if (threadIdx.x == 0) {
      s_rec = q[qi];
      s_ndistinct = 0;
      s_overflow = 0;
      s_fail = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {  // look-ahead claim, read after the item
      if (MODE == 0 && *(volatile u32*)&A.ctr->full) s_next = ~0ull;
      else s_next = atomicAdd(claim, 1ull);
    }
    const int4 rec = s_rec;
    const int r = rec.x;
    const int a = MODE ? A.sources[r] : r;
    const int lo = rec.y, hi = rec.z;
    const bool is_dense = (rec.w & kItemDense) != 0;
    const int logcap = (rec.w >> 8) & 0xff;
    const int nslots = 1 << logcap;
    const int limit = (nslots * 3) / 4;
    const bool full_range = (rec.w & kItemWhole) || ((lo <= (MODE ? 0 : a + 1)) && hi >= A.n);
    const int span = hi - lo;
    const int e0 = A.off[a], e1 = A.off[a + 1];
    for (int eb = e0 + wid * 32; eb < e1; eb += NW * 32) {
      const int e = eb + lane;
      int s = 0, len = 0;
      V w = 0;
      if (e < e1) {
        const Arc t = A.arc[e];
        if (t.z <= A.cap) {
          int s0, s1;
          if (MODE == 0) {
            s0 = t.x + 1;
            s1 = t.y;
          } else {
            s0 = t.y - t.z;
            s1 = t.y;
          }
          if (!full_range && s0 < s1) {
            s0 = lower_bound_g(A.idx, s0, s1, lo);
            s1 = lower_bound_g(A.idx, s0, s1, hi);
          }
          s = s0;
          len = s1 - s0;
          if (len > 0) w = arc_weight<V>(A, t.z);
        }
      }
      if (is_dense) {
        scan_arcs<V>(s, len, w, A.idx, [&](int c, V wc) {
          if (MODE == 1 && c == a) return;
          shared_add<V>(&dense[c - lo], wc);
        });
      } else {
        scan_arcs<V>(s, len, w, A.idx, [&](int c, V wc) {
          if (MODE == 1 && c == a) return;
          if (*(volatile int*)&s_overflow) return;
          const int rc = hash_add<V>(keys, vals, logcap, c, wc);
          if (rc == 1) {
            if (atomicAdd(&s_ndistinct, 1) >= limit) s_overflow = 1;
          } else if (rc == 2) {
            s_overflow = 1;
          }
        });
        if (__any_sync(FULLMASK, *(volatile int*)&s_overflow != 0)) break;
      }
    }
    __syncthreads();
    if (!is_dense && s_overflow) {
      // give the item back for splitting; leave the table empty
      for (int i = threadIdx.x * 4; i < nslots; i += THREADS * 4) {
        *reinterpret_cast<int4*>(keys + i) = make_int4(0, 0, 0, 0);
        zero4<V>(vals + i);
      }
      if (threadIdx.x == 0) {
        const u64 f = atomicAdd(&A.ctr->nsplit, 1ull);
        if (f < A.split_cap) A.split[f] = rec;
        else A.ctr->error = 2u;
      }
      __syncthreads();
      continue;
    }
    // drop first-order neighbours inside [lo, hi)
    for (int e = e0 + threadIdx.x; e < e1; e += THREADS) {
      const int b = __ldg(A.idx + e);
      if (b < lo || b >= hi || (MODE == 0 && b <= a)) continue;
      if (is_dense) dense[b - lo] = 0;
      else hash_kill<V>(keys, vals, logcap, b);
    }
    __syncthreads();
    // score and select: 4 consecutive slots per lane and step
    const u64 da = (u64)(e1 - e0);
    const int nscan = is_dense ? ((span + 3) & ~3) : nslots;
    bool fail = false;
    TopEnt* top = tops + wid * (MODE ? A.k : 0);
    int tcnt = 0;
    for (int base0 = wid * 128; base0 < nscan; base0 += THREADS * 4) {  // warp-uniform trips
      if (is_dense) {
        const int base = base0 + lane * 4;
        int c4[4] = {0, 0, 0, 0};
        V v4[4] = {0, 0, 0, 0};
        if (base < nscan) {
          load4<V>(dense + base, v4);
          zero4<V>(dense + base);
#pragma unroll
          for (int j = 0; j < 4; ++j) c4[j] = lo + base + j;
        }
        fail |= score_chunk<V, MODE>(A, T, a, da, c4, v4, top, tcnt, n_cand);
      } else {
        fail |= score_hash_chunk<V, MODE>(A, T, a, da, keys, vals, base0, nslots, top, tcnt,
                                          n_cand);
      }
    }
    if (MODE == 0) {
      if (fail && lane == 0) s_fail = 1;
      __syncthreads();
      if (threadIdx.x == 0 && s_fail) {
        A.ctr->full = 1u;
        const u64 f = atomicAdd(&A.ctr->nfailed, 1ull);
        if (f < A.failed_cap) A.failed[f] = rec;
        else A.ctr->error = 1u;
      }
    } else {
      if (lane == 0) s_tcnt[wid] = tcnt;
      __syncthreads();
      if (wid == 0) {
        int cnt = s_tcnt[0];
        for (int w2 = 1; w2 < NW; ++w2) {
          const TopEnt* other = tops + w2 * A.k;
          const int oc = s_tcnt[w2];
          for (int j = 0; j < oc; ++j) {
            const TopEnt x = other[j];
            if (cnt >= A.k && !ent_before(x, top[A.k - 1])) break;  // sorted: rest is worse
            top_insert(top, cnt, A.k, x);
          }
        }
        if (rec.w & kItemSingle) {
          for (int j = lane; j < cnt; j += 32) A.out_top[(u64)r * A.k + j] = top[j];
          if (lane == 0) A.out_cnt[r] = cnt;
        } else {
          u64 p = 0;
          if (lane == 0) p = A.partial_by_item ? qi : atomicAdd(&A.ctr->npartial, 1ull);
          p = __shfl_sync(FULLMASK, p, 0);
          if (p < A.partial_cap) {
            for (int j = lane; j < cnt; j += 32) A.partial[p * A.k + j] = top[j];
            if (lane == 0) A.partial_hdr[p] = make_int2(r, cnt);
          } else if (lane == 0) {
            A.ctr->error = 3u;
          }
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) n_cand += __shfl_xor_sync(FULLMASK, n_cand, o);
  if (lane == 0 && n_cand) atomicAdd(&A.ctr->candidates, n_cand);
}

// ------------------------------------------------------------ large tier ---

// Shared memory of a large-tier CTA of THREADS threads beyond its table
// (big_extra_smem(THREADS) bytes): a window-boundary table of
// big_bounds(THREADS) positions, then a queue of THREADS segments (prefix,
// start, length, weight): entries [0, THREADS / 2) hold segments of kPiece or
// more wedges, cut into pieces of their own; entries [THREADS / 2, THREADS)
// shorter ones, laid end to end and cut into pieces across segments.
__host__ __device__ constexpr int big_bounds(int threads) { return 3 * threads; }
constexpr int kPiece = 128;  // wedges per piece
constexpr int kPerLane = kPiece / 32;
constexpr int kLongSeg = 64; // segments at least this long are shared as pieces
constexpr int kShortSeg = 8; // the same when the item has at most one arc per thread

// First index in idx[l, r) whose value is >= key, searching outward from l.
__device__ __forceinline__ int lower_bound_gallop(const int* __restrict__ idx, int l, int r,
                                                  int key) {
  if (l >= r || __ldg(idx + l) >= key) return l;
  int prev = l, step = 1;
  while (true) {
    const int cur = l + step;
    if (cur >= r) return lower_bound_g(idx, prev + 1, r, key);
    if (__ldg(idx + cur) >= key) return lower_bound_g(idx, prev + 1, cur, key);
    prev = cur;
    step <<= 1;
  }
}

// Exclusive CTA-wide prefix sums of two ints per thread (ex, ey) and their
// totals (tx, ty).  One barrier; wtot (one int2 per warp) must not be written
// again before every thread has passed a later barrier.
template <int THREADS>
__device__ __forceinline__ void block_scan2(int x, int y, int& ex, int& ey, int& tx, int& ty,
                                            int2* wtot) {
  constexpr int NW = THREADS / 32;
  const int lane = lane_id();
  const int wid = threadIdx.x >> 5;
  int ix = x, iy = y;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int ux = __shfl_up_sync(FULLMASK, ix, o);
    const int uy = __shfl_up_sync(FULLMASK, iy, o);
    if (lane >= o) {
      ix += ux;
      iy += uy;
    }
  }
  if (lane == 31) wtot[wid] = make_int2(ix, iy);
  __syncthreads();
  const int2 t = lane < NW ? wtot[lane] : make_int2(0, 0);
  int sx = t.x, sy = t.y;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int ux = __shfl_up_sync(FULLMASK, sx, o);
    const int uy = __shfl_up_sync(FULLMASK, sy, o);
    if (lane >= o) {
      sx += ux;
      sy += uy;
    }
  }
  ex = __shfl_sync(FULLMASK, sx - t.x, wid) + ix - x;
  ey = __shfl_sync(FULLMASK, sy - t.y, wid) + iy - y;
  tx = __shfl_sync(FULLMASK, sx, NW - 1);
  ty = __shfl_sync(FULLMASK, sy, NW - 1);
}

// Last j in [lo, hi) with p[j] <= key (p ascending, p[lo] <= key).
__device__ __forceinline__ int last_le(const int* p, int lo, int hi, int key) {
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (p[mid] <= key) lo = mid; else hi = mid;
  }
  return lo;
}

// One CTA per item.  A hash item is one vertex range; a dense item sweeps G
// consecutive windows of at most A.big_span vertices.  Each arc's segment (the
// part of its suffix inside the range) comes from a boundary table filled once
// per item when it fits (independent binary searches, one per thread), from a
// cursor carried between windows, or from a binary search.  Warps take 32 arcs
// at a time and walk the short segments at once; segments of kLongSeg or more
// wedges are queued, laid end to end by a CTA prefix sum and dealt to all
// warps in pieces of kPiece wedges, so a source with a few long intermediary
// lists still keeps every warp busy.
template <bool V64, int MODE, int THREADS>
__global__ void __launch_bounds__(THREADS, 1024 / THREADS) k_scan_big(ScanArgs A, const int4* __restrict__ q,
                                                                      u64 nq, int table_bytes,
                                                                      u64* __restrict__ claim) {
  typedef typename std::conditional<V64, u64, u32>::type V;
  constexpr int NW = THREADS / 32;
  constexpr int NB = big_bounds(THREADS);
  extern __shared__ __align__(16) unsigned char smem[];
  const int max_slots = 1 << (ceil_log2((u64)table_bytes / (4 + sizeof(V)) + 1) - 1);
  int* keys = reinterpret_cast<int*>(smem);
  V* vals = reinterpret_cast<V*>(smem + (size_t)max_slots * 4);
  V* dense = reinterpret_cast<V*>(smem);
  u32* dbits = reinterpret_cast<u32*>(smem + (size_t)A.big_span * sizeof(V));  // touched bits
  int* bnd = reinterpret_cast<int*>(smem + table_bytes);  // boundaries or cursors
  int* c_p = bnd + NB;                                    // queued segment: prefix
  int* c_s = c_p + THREADS;                               // start (short: start - prefix)
  int* c_l = c_s + THREADS;                               // length
  u64* c_w = reinterpret_cast<u64*>(c_l + THREADS);       // weight
  TopEnt* tops = reinterpret_cast<TopEnt*>(c_w + THREADS);
  constexpr int H = THREADS / 2;                          // long entries [0, H), short [H, 2H)
  __shared__ int4 s_rec;
  __shared__ u64 s_next;
  __shared__ int s_ndistinct, s_overflow, s_fail, s_qnl, s_qns;
  __shared__ int s_tcnt[NW];
  __shared__ int2 s_wtot[NW];
  // optional phase profile (thread 0's clock): 0 item setup and boundary
  // table, 1 arc segments and short walks, 3 long-segment pieces, 4
  // exclusion and scoring, 5 item end; 2 is the whole time of dense items
  // (also counted in the others)
  long long t_prof[6] = {0, 0, 0, 0, 0, 0};
  long long t_last = clock64();
  const bool prof = A.prof != nullptr && threadIdx.x == 0;
#define LP_PHASE(i)                        \
  do {                                     \
    if (prof) {                            \
      const long long t_now = clock64();   \
      t_prof[i] += t_now - t_last;         \
      t_last = t_now;                      \
    }                                      \
  } while (0)

  const int lane = lane_id();
  const int wid = threadIdx.x >> 5;
  // global mode, count measures: dense windows of 16-bit counters; AA / RA:
  // 64-bit counters as two arrays of halves (low words, then high words)
  const bool d16 = MODE == 0 && !V64 && A.dense16;
  u32* dlo = reinterpret_cast<u32*>(smem);
  u32* dhi = dlo + A.big_span;
  for (int i = threadIdx.x * 16; i < table_bytes; i += THREADS * 16)
    *reinterpret_cast<int4*>(smem + i) = make_int4(0, 0, 0, 0);
  Thresh T;
  if (MODE == 0) T = *A.thresh;
  u64 n_cand = 0;
  if (threadIdx.x == 0) {
    if (MODE == 0 && *(volatile u32*)&A.ctr->full) s_next = ~0ull;
    else s_next = atomicAdd(claim, 1ull);
  }
  __syncthreads();
  for (;;) {
    const u64 qi = s_next;
    if (qi >= nq) break;
    const long long t_item = prof ? clock64() : 0;
    if (threadIdx.x == 0) {
      s_rec = q[qi];
      s_fail = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {  // look-ahead claim, read after the item
      if (MODE == 0 && *(volatile u32*)&A.ctr->full) s_next = ~0ull;
      else s_next = atomicAdd(claim, 1ull);
    }
    const int4 rec = s_rec;
    const int r = rec.x;
    const int a = MODE ? A.sources[r] : r;
    const int lo = rec.y, hi = rec.z;
    const bool is_dense = (rec.w & kItemDense) != 0;
    const bool d8 = d16 && (rec.w & kItemD8) != 0;  // 8-bit counters for this item
    const int logcap = (rec.w >> 8) & 0xff;
    // dense items sweep G windows; global-mode hash items G ranges
    const int G = (is_dense || MODE == 0) ? ((rec.w >> 16) & 0xfff) + 1 : 1;
    const int nslots = 1 << logcap;
    const int limit = (nslots * 3) / 4;
    const int span = hi - lo;
    const int e0 = A.off[a], e1 = A.off[a + 1];
    const int K = e1 - e0;
    // dense sweeps: all window boundaries of every arc up front when they
    // fit (independent binary searches, one per thread), else a cursor per
    // arc carried from window to window
    const bool pre = G > 1 && (long long)K * (G + 1) <= NB;
    const bool use_cur = G > 1 && !pre && K <= NB;
    // more arcs than the shared table holds: the cursors live in this CTA's
    // slice of a device scratch array (same arc, same thread every window)
    const bool use_gcur = G > 1 && K > NB && A.gcur != nullptr && (int)blockIdx.x < A.gcur_ctas;
    int* gcur = use_gcur ? A.gcur + (size_t)blockIdx.x * (size_t)A.gcur_stride : nullptr;
    if (pre) {
      for (int q2 = threadIdx.x; q2 < K * (G + 1); q2 += THREADS) {
        const int j = q2 / (G + 1);
        const int gg = q2 - j * (G + 1);
        const Arc t = A.arc[e0 + j];
        const int s0 = MODE ? t.y - t.z : t.x + 1;
        const int key = lo + (int)(((u64)span * (u64)gg) / (u64)G);
        bnd[q2] = (t.z <= A.cap && s0 < t.y) ? lower_bound_interp(A.idx, s0, t.y, key) : s0;
      }
      __syncthreads();
    }
    const u64 da = (u64)K;
    const u64 vmin = MODE == 0 && T.valid ? __ldg(A.vfloor + K) : 1;
    TopEnt* top = tops + wid * (MODE ? A.k : 0);
    int tcnt = 0;
    bool fail = false;
    bool overflowed = false;
    int g_over = 0;  // the range that overflowed (ranges before it are done)
    for (int g = 0; g < G; ++g) {
      const int lg = lo + (int)(((u64)span * (u64)g) / (u64)G);
      const int hg = lo + (int)(((u64)span * (u64)(g + 1)) / (u64)G);
      const bool full_range =
          G == 1 && ((rec.w & kItemWhole) || (lo <= (MODE ? 0 : a + 1) && hi >= A.n));
      if (threadIdx.x == 0) {
        s_ndistinct = 0;
        s_overflow = 0;
        s_qnl = 0;
        s_qns = 0;
      }
      __syncthreads();
      LP_PHASE(0);
      auto insert = [&](int c, V wc) {
        if (MODE == 1 && c == a) return;
        if (is_dense) {
          const int i = c - lg;
          if (MODE == 0) {  // scored by a linear scan: no touched bits
            if (sizeof(V) == 8) {  // split halves: low word, then high word plus carry
              const int p = swz(i);
              const u32 l = (u32)wc, h = (u32)((u64)wc >> 32);
              const u32 old = atomicAdd(dlo + p, l);
              const u32 hc = h + ((old + l < old) ? 1u : 0u);
              if (hc) atomicAdd(dhi + p, hc);
            } else if (d8) {  // count measures: the weight is 1
              const int p = swz(i);
              atomicAdd(reinterpret_cast<u32*>(dense) + (p >> 2), 1u << ((p & 3) << 3));
            } else if (d16) {
              const int p = swz(i);
              atomicAdd(reinterpret_cast<u32*>(dense) + (p >> 1), 1u << ((p & 1) << 4));
            } else {
              atomicAdd(reinterpret_cast<u32*>(&dense[swz(i)]), (u32)wc);
            }
          } else if (shared_add<V>(&dense[swz(i)], wc) == 0) {
            // the first add sees a zero low word (a later wrap to zero only
            // sets the bit again)
            atomicOr(&dbits[i >> 5], 1u << (i & 31));
          }
        } else {
          if (*(volatile int*)&s_overflow) return;
          const int rc = hash_add<V>(keys, vals, logcap, c, wc);
          if (rc == 1) {
            if (atomicAdd(&s_ndistinct, 1) >= limit) s_overflow = 1;
          } else if (rc == 2) {
            s_overflow = 1;
          }
        }
      };
      // phase A: one arc per thread, THREADS arcs at a time, dealt round-robin
      // to the warps (arc eb + lane * NW + wid) so that a source with few arcs
      // still spreads them over every warp; short segments are walked at once
      // (concatenated across the lanes), longer ones are queued for phase B.
      // With at most one arc per thread all but the shortest are queued.
      const int long_seg = K <= THREADS ? kShortSeg : kLongSeg;
      // global-mode 64-bit dense windows mark the first-order neighbours in
      // this pass (every arc of the source comes by) instead of a clearing
      // pass after the inserts
      const bool mark_first = MODE == 0 && V64 && is_dense;
      for (int eb = 0; eb < K; eb += THREADS) {  // CTA-uniform trips
        const int j = eb + lane * NW + wid;
        int st = 0, len = 0;
        V w = 0;
        if (j < K) {
          const Arc t = A.arc[e0 + j];
          if (mark_first && t.w >= lg && t.w < hg && t.w > a)
            atomicAdd(dhi + swz(t.w - lg), kFirstOrder64);
          if (t.z <= A.cap) {
            int s0 = MODE ? t.y - t.z : t.x + 1, s1 = t.y;
            if (s0 < s1) {
              if (pre) {
                s0 = bnd[j * (G + 1) + g];
                s1 = bnd[j * (G + 1) + g + 1];
              } else if (!full_range) {
                const int b0 = (use_cur && g > 0)    ? bnd[j]
                               : (use_gcur && g > 0) ? gcur[j]
                                                     : lower_bound_interp(A.idx, s0, s1, lg);
                const int b1 = (use_cur || use_gcur) ? lower_bound_gallop(A.idx, b0, s1, hg)
                                                     : lower_bound_interp(A.idx, b0, s1, hg);
                if (use_cur) bnd[j] = b1;
                if (use_gcur) gcur[j] = b1;
                s0 = b0;
                s1 = b1;
              }
            }
            st = s0;
            len = s1 > s0 ? s1 - s0 : 0;
            if (len > 0) w = arc_weight<V>(A, t.z);
          }
        }
        if (len >= long_seg) {  // queue it (a full queue: the warp walks it below)
          const bool lng = len >= kPiece;
          const int slot = atomicAdd(lng ? &s_qnl : &s_qns, 1);
          if (slot < H) {
            const int q2 = lng ? slot : H + slot;
            c_s[q2] = st;
            c_l[q2] = len;
            c_w[q2] = (u64)w;
            len = 0;
          }
        }
        scan_arcs<V>(st, len, w, A.idx, insert);
        if (!is_dense && __any_sync(FULLMASK, *(volatile int*)&s_overflow != 0)) break;
      }
      __syncthreads();
      LP_PHASE(1);
      // phase B: the queued segments in pieces of kPiece wedges dealt to the
      // warps: the long ones piece by piece (one segment per piece, so a
      // warp streams it), then the short ones end to end
      const int nl = min(s_qnl, H), ns = min(s_qns, H);
      if (nl + ns > 0 && (is_dense || !s_overflow)) {  // CTA-uniform
        const int t = threadIdx.x;
        const bool is_l = t < nl, is_s = t >= H && t < H + ns;
        int ex, ey, npl, tsw;
        block_scan2<THREADS>(is_l ? (c_l[t] + kPiece - 1) / kPiece : 0, is_s ? c_l[t] : 0, ex, ey,
                             npl, tsw, s_wtot);
        if (is_l) c_p[t] = ex;  // first piece of the segment
        if (is_s) {             // first wedge of the segment in the concatenation
          c_p[t] = ey;
          c_s[t] -= ey;
        }
        __syncthreads();
        const int npieces = npl + (tsw + kPiece - 1) / kPiece;
        for (int p = wid; p < npieces; p += NW) {  // warp-uniform trips
          int c8[kPerLane], j8[kPerLane];
          if (p < npl) {
            const int j = last_le(c_p, 0, nl, p);
            const int off = (p - c_p[j]) * kPiece;
            const int plen = min(kPiece, c_l[j] - off);
            const int* src = A.idx + c_s[j] + off;
#pragma unroll
            for (int u = 0; u < kPerLane; ++u) {
              c8[u] = lane + 32 * u < plen ? __ldg(src + lane + 32 * u) : -1;
              j8[u] = j;
            }
          } else {
            const int i0 = (p - npl) * kPiece + lane;
            int jj = i0 < tsw ? last_le(c_p, H, H + ns, i0) : H;
#pragma unroll
            for (int u = 0; u < kPerLane; ++u) {
              const int i = i0 + 32 * u;
              c8[u] = -1;
              if (i < tsw) {
                // i - 32 lay in segment jj and segments are not empty, so i
                // lies in one of the segments jj .. jj + 32
                if (jj + 1 < H + ns && c_p[jj + 1] <= i) jj = last_le(c_p, jj + 1, min(H + ns, jj + 33), i);
                c8[u] = __ldg(A.idx + c_s[jj] + i);
              }
              j8[u] = jj;
            }
          }
#pragma unroll
          for (int u = 0; u < kPerLane; ++u)
            if (c8[u] >= 0) insert(c8[u], V64 ? (V)c_w[j8[u]] : (V)1);
          if (!is_dense && __any_sync(FULLMASK, *(volatile int*)&s_overflow != 0)) break;
        }
        __syncthreads();
      }
      LP_PHASE(3);
      if (!is_dense && s_overflow) {
        // give the range back for splitting; leave the table empty
        for (int i = threadIdx.x * 4; i < nslots; i += THREADS * 4) {
          *reinterpret_cast<int4*>(keys + i) = make_int4(0, 0, 0, 0);
          zero4<V>(vals + i);
        }
        overflowed = true;
        g_over = g;
        __syncthreads();
        break;  // the rest of the item goes back for splitting
      }
      // drop first-order neighbours inside [lg, hg) (marked above in the
      // global-mode 64-bit dense windows; the last phase ended with a barrier)
      if (!(MODE == 0 && V64 && is_dense)) {
      for (int e = e0 + threadIdx.x; e < e1; e += THREADS) {
        const int b = __ldg(A.idx + e);
        if (b < lg || b >= hg || (MODE == 0 && b <= a)) continue;
        if (is_dense && d8) {
          const int p = swz(b - lg);
          atomicAnd(reinterpret_cast<u32*>(dense) + (p >> 2), ~(0xffu << ((p & 3) << 3)));
        } else if (is_dense && d16) {
          const int p = swz(b - lg);
          atomicAnd(reinterpret_cast<u32*>(dense) + (p >> 1), ~(0xffffu << ((p & 1) << 4)));
        } else if (is_dense) {
          dense[swz(b - lg)] = 0;
        }
        else hash_kill<V>(keys, vals, logcap, b);
      }
      __syncthreads();
      }
      // score and select.  Global mode: every counter or slot once, the ones
      // below the count floor only counted.  Per-source mode: the touched
      // counters (dense) or the packed live slots (hash).
      if (MODE == 0 && (is_dense || T.valid)) {
        int qn = 0, qc = 0, qd = 0;
        V qv = 0;
        if (is_dense && d8) {
          const int npos = (hg - lg + 31) & ~31;
          u32 qv8 = (u32)qv;
          for (int base0 = wid * 256; base0 < npos; base0 += THREADS * 8)  // warp-uniform trips
            fail |= score_dense8_linear(A, T, a, da, reinterpret_cast<u32*>(dense), base0, npos,
                                        lg, vmin, n_cand, qn, qc, qv8, qd);
          qv = (V)qv8;
        } else if (is_dense && d16) {
          const int npos = (hg - lg + 31) & ~31;
          u32 qv16 = (u32)qv;
          for (int base0 = wid * 256; base0 < npos; base0 += THREADS * 8)  // warp-uniform trips
            fail |= score_dense16_linear(A, T, a, da, reinterpret_cast<u32*>(dense), base0, npos,
                                         lg, vmin, n_cand, qn, qc, qv16, qd);
          qv = (V)qv16;
        } else if (is_dense && V64) {
          const int npos = (hg - lg + 31) & ~31;
          u64 qv64 = (u64)qv;
          for (int base0 = wid * 128; base0 < npos; base0 += THREADS * 4)  // warp-uniform trips
            fail |= score_dense64_linear(A, T, a, da, dlo, dhi, base0, npos, lg, vmin, n_cand, qn,
                                         qc, qv64, qd);
          qv = (V)qv64;
        } else if (is_dense) {
          const int npos = (hg - lg + 31) & ~31;
          for (int base0 = wid * 128; base0 < npos; base0 += THREADS * 4)  // warp-uniform trips
            fail |= score_dense_linear<V>(A, T, a, da, dense, base0, npos, lg, vmin, n_cand, qn,
                                          qc, qv, qd);
        } else {
          for (int base0 = wid * 128; base0 < nslots; base0 += THREADS * 4)
            fail |= score_hash_linear<V>(A, T, a, da, keys, vals, base0, nslots, vmin, n_cand, qn,
                                         qc, qv, qd);
        }
        if (qn > 0) fail |= survivors_flush<V>(A, T, a, da, qn, qc, qv, qd);
      } else if (is_dense) {
        const int nwords = (hg - lg + 31) >> 5;
        for (int w0 = wid * 32; w0 < nwords; w0 += THREADS)  // warp-uniform trips
          fail |= score_dense_words<V, MODE>(A, T, a, da, dense, dbits, w0, nwords, lg, top, tcnt,
                                             n_cand);
      } else {
        for (int base0 = wid * 128; base0 < nslots; base0 += THREADS * 4)
          fail |= score_hash_chunk<V, MODE>(A, T, a, da, keys, vals, base0, nslots, top, tcnt,
                                            n_cand);
      }
      __syncthreads();
      LP_PHASE(4);
    }
    if (overflowed) {
      if (threadIdx.x == 0) {
        // hand back [start of the overflowed range, hi) with its G - g_over ranges
        int4 back = rec;
        back.y = lo + (int)(((u64)span * (u64)g_over) / (u64)G);
        back.w = (rec.w & 0xffff) | ((G - g_over - 1) << 16);
        const u64 f = atomicAdd(&A.ctr->nsplit, 1ull);
        if (f < A.split_cap) A.split[f] = back;
        else A.ctr->error = 2u;
      }
      __syncthreads();
      continue;
    }
    if (MODE == 0) {
      if (fail && lane == 0) s_fail = 1;
      __syncthreads();
      if (threadIdx.x == 0 && s_fail) {
        A.ctr->full = 1u;
        const u64 f = atomicAdd(&A.ctr->nfailed, 1ull);
        if (f < A.failed_cap) A.failed[f] = rec;
        else A.ctr->error = 1u;
      }
    } else {
      if (lane == 0) s_tcnt[wid] = tcnt;
      __syncthreads();
      if (wid == 0) {
        int cnt = s_tcnt[0];
        for (int w2 = 1; w2 < NW; ++w2) {
          const TopEnt* other = tops + w2 * A.k;
          const int oc = s_tcnt[w2];
          for (int j = 0; j < oc; ++j) {
            const TopEnt x = other[j];
            if (cnt >= A.k && !ent_before(x, top[A.k - 1])) break;  // sorted: rest is worse
            top_insert(top, cnt, A.k, x);
          }
        }
        if (rec.w & kItemSingle) {
          for (int j = lane; j < cnt; j += 32) A.out_top[(u64)r * A.k + j] = top[j];
          if (lane == 0) A.out_cnt[r] = cnt;
        } else {
          u64 p = 0;
          if (lane == 0) p = A.partial_by_item ? qi : atomicAdd(&A.ctr->npartial, 1ull);
          p = __shfl_sync(FULLMASK, p, 0);
          if (p < A.partial_cap) {
            for (int j = lane; j < cnt; j += 32) A.partial[p * A.k + j] = top[j];
            if (lane == 0) A.partial_hdr[p] = make_int2(r, cnt);
          } else if (lane == 0) {
            A.ctr->error = 3u;
          }
        }
      }
    }
    __syncthreads();
    LP_PHASE(5);
    if (prof && is_dense) t_prof[2] += clock64() - t_item;
  }
#undef LP_PHASE
  if (prof)
    for (int i = 0; i < 6; ++i) atomicAdd(&A.prof[i], (u64)t_prof[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) n_cand += __shfl_xor_sync(FULLMASK, n_cand, o);
  if (lane == 0 && n_cand) atomicAdd(&A.ctr->candidates, n_cand);
}

// --------------------------------------------------- per-source merging ---

// For each record with several items: merge their partial lists.  grp_list
// holds (record, first partial position in `order`, number of partials);
// order lists partial slot ids grouped by record.
__global__ void k_merge_partials(const int4* __restrict__ grp_list, int ngrp,
                                 const int* __restrict__ order, const TopEnt* __restrict__ partial,
                                 const int2* __restrict__ hdr, int k, TopEnt* __restrict__ out_top,
                                 int* __restrict__ out_cnt) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = lane_id();
  const int wid = threadIdx.x >> 5;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  TopEnt* top = reinterpret_cast<TopEnt*>(smem) + wid * k;
  if (gw >= ngrp) return;
  const int4 g = grp_list[gw];
  int cnt = 0;
  for (int i = 0; i < g.z; ++i) {
    const int p = order[g.y + i];
    const int pc = hdr[p].y;
    for (int j0 = 0; j0 < pc; j0 += 32) {
      const int j = j0 + lane;
      TopEnt x;
      const bool has = j < pc;
      if (has) x = partial[(u64)p * k + j];
      else {
        x.num = 0;
        x.den = 1;
        x.c = 0;
        x.cn = 0;
      }
      top_offer(top, cnt, k, has, x);
    }
  }
  for (int j = lane; j < cnt; j += 32) out_top[(u64)g.x * k + j] = top[j];
  if (lane == 0) out_cnt[g.x] = cnt;
}

// ------------------------------------------------------------ emitting ---

__device__ __forceinline__ u64 isqrt64(u64 x) {
  u64 r = (u64)sqrt((double)x);
  while (r * r > x) --r;
  while ((r + 1) * (r + 1) <= x) ++r;
  return r;
}

__device__ __forceinline__ lp_link make_link(int measure, int u, int v, u64 num, u64 den, u64 cn,
                                             int fixbits) {
  lp_link L;
  L.u = u;
  L.v = v;
  L.score = (float)key_value(measure, num, den, cn, fixbits);
  L.cn = (int)cn;
  return L;
}

// Global mode: sorted candidates -> links.
__global__ void k_emit_global(const Cand* __restrict__ c, u64 n, int measure, int fixbits,
                              lp_link* __restrict__ out) {
  const u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Cand x = c[i];
  u64 cn = x.num;
  if (measure == LP_SC) cn = isqrt64(x.num);
  if (measure == LP_AA || measure == LP_RA) cn = 0;
  out[i] = make_link(measure, x.u, x.v, x.num, x.den, cn, fixbits);
}

// Per-source mode: lists -> links (rows of k).
__global__ void k_emit_sources(const TopEnt* __restrict__ top, const int* __restrict__ cnt,
                               const int* __restrict__ sources, int n_src, int k, int measure,
                               int fixbits, lp_link* __restrict__ out) {
  const u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (u64)n_src * k) return;
  const int r = (int)(i / k), j = (int)(i % k);
  if (j >= cnt[r]) {  // unused entry of the row: a fixed filler
    lp_link L;
    L.u = -1;
    L.v = -1;
    L.score = 0.f;
    L.cn = 0;
    out[i] = L;
    return;
  }
  const TopEnt x = top[i];
  out[i] = make_link(measure, sources[r], x.c, x.num, x.den, (u64)x.cn, fixbits);
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

// Common neighbours of AA / RA links (whose tables hold weight sums rather
// than counts), one warp per link.
__global__ void k_pair_cn(lp_link* __restrict__ links, const int* __restrict__ cnt_rows, int k,
                          u64 n, const int* __restrict__ off, const int* __restrict__ idx,
                          const int* __restrict__ deg, const Arc* __restrict__ arc, int cap) {
  const u64 gw = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (gw >= n) return;
  if (cnt_rows && (int)(gw % k) >= cnt_rows[gw / k]) return;
  const lp_link L = links[gw];
  const u64 c = pair_common(L.u, L.v, off, idx, deg, arc, cap, nullptr);
  if (lane_id() == 0) links[gw].cn = (int)c;
}

// Exact selection keys of global-mode links (u < v): the count measures'
// rational from the link's common-neighbour count and the two degrees (Eq.
// 1-7), AA / RA's fixed-point sum rebuilt from the graph (Eq. 8-9).  One warp
// per link.
__global__ void k_link_keys(const lp_link* __restrict__ links, u64 n, int measure,
                            const int* __restrict__ off, const int* __restrict__ idx,
                            const int* __restrict__ deg, const Arc* __restrict__ arc, int cap,
                            const u64* __restrict__ wt, Cand* __restrict__ out) {
  const u64 gw = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (gw >= n) return;
  const lp_link L = links[gw];
  Cand x;
  x.u = L.u;
  x.v = L.v;
  if (measure == LP_AA || measure == LP_RA) {
    x.num = pair_common(L.u, L.v, off, idx, deg, arc, cap, wt);
    x.den = 1;
  } else {
    make_key(measure, (u64)L.cn, (u64)__ldg(deg + L.u), (u64)__ldg(deg + L.v), x.num, x.den);
  }
  if (lane_id() == 0) out[gw] = x;
}

// ------------------------------------------------------------ launchers ---

static int g_nsm = 0;
static int num_sms() {
  if (g_nsm == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_nsm, cudaDevAttrMultiProcessorCount, dev);
    if (g_nsm <= 0) g_nsm = 1;
  }
  return g_nsm;
}

// Allow kern the device's whole opt-in shared memory.  The value is the same
// on every call, so threads launching it concurrently with different dynamic
// sizes cannot race on the attribute (a smaller size set by one thread would
// make another thread's larger launch fail).
template <typename Kern>
static cudaError_t allow_max_smem(Kern kern) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kern);
  if (e != cudaSuccess) return e;
  int dev = 0, optin = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              optin - (int)fa.sharedSizeBytes);
}

cudaError_t launch_estimate2(const ScanArgs& A, int n_rec, int4* warpq, int4* medq, int4* itemq,
                             u64 itemq_cap, int2* grp, cudaStream_t st) {
  if (n_rec <= 0) return cudaSuccess;
  const int threads = 256;
  const u64 groups = ((u64)n_rec + 31) / 32;
  const int blocks = (int)max((u64)1, min((u64)num_sms() * 8, (groups * 32 + threads - 1) / threads));
  const bool v64 = A.measure == LP_AA || A.measure == LP_RA;
  if (A.mode == 0) {
    if (v64) k_estimate<0, true><<<blocks, threads, 0, st>>>(A, n_rec, warpq, medq, itemq, itemq_cap, grp);
    else k_estimate<0, false><<<blocks, threads, 0, st>>>(A, n_rec, warpq, medq, itemq, itemq_cap, grp);
  } else {
    if (v64) k_estimate<1, true><<<blocks, threads, 0, st>>>(A, n_rec, warpq, medq, itemq, itemq_cap, grp);
    else k_estimate<1, false><<<blocks, threads, 0, st>>>(A, n_rec, warpq, medq, itemq, itemq_cap, grp);
  }
  return cudaGetLastError();
}

template <bool V64, int MODE>
static cudaError_t launch_warp_t(const ScanArgs& A, const int4* q, u64 nq, cudaStream_t st) {
  typedef typename std::conditional<V64, u64, u32>::type V;
  const int nw = kWarpTierThreads / 32;
  const size_t smem = (size_t)nw * kWarpSlots * (4 + sizeof(V)) +
                      (MODE ? (size_t)nw * A.k * sizeof(TopEnt) : 0);
  auto kern = k_scan_warp<V64, MODE>;
  cudaError_t e = allow_max_smem(kern);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kWarpTierThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const u64 want = (nq + nw - 1) / nw;
  const int blocks = (int)max((u64)1, min((u64)num_sms() * per_sm, want));
  kern<<<blocks, kWarpTierThreads, smem, st>>>(A, q, nq);
  return cudaGetLastError();
}

cudaError_t launch_scan_warp(const ScanArgs& A, const int4* q, u64 nq, cudaStream_t st) {
  if (nq == 0) return cudaSuccess;
  const bool v64 = A.measure == LP_AA || A.measure == LP_RA;
  if (A.mode == 0) return v64 ? launch_warp_t<true, 0>(A, q, nq, st) : launch_warp_t<false, 0>(A, q, nq, st);
  return v64 ? launch_warp_t<true, 1>(A, q, nq, st) : launch_warp_t<false, 1>(A, q, nq, st);
}

template <bool V64, int MODE, int THREADS>
static cudaError_t launch_cta_t(const ScanArgs& A, const int4* q, u64 nq, int table_bytes,
                                u64* claim, cudaStream_t st) {
  const size_t smem = (size_t)table_bytes + (MODE ? (size_t)(THREADS / 32) * A.k * sizeof(TopEnt) : 0);
  auto kern = k_scan_cta<V64, MODE, THREADS>;
  cudaError_t e = allow_max_smem(kern);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, THREADS, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const int blocks = (int)max((u64)1, min((u64)num_sms() * per_sm, nq));
  kern<<<blocks, THREADS, smem, st>>>(A, q, nq, table_bytes, claim);
  return cudaGetLastError();
}

template <bool V64, int MODE, int THREADS>
static cudaError_t launch_big_t(const ScanArgs& A, const int4* q, u64 nq, cudaStream_t st) {
  static_assert(big_extra_smem(THREADS) == big_bounds(THREADS) * 4 + THREADS * (4 + 4 + 4 + 8),
                "large-tier shared memory layout");
  const int tb = A.big_bytes;
  const size_t smem = (size_t)tb + big_extra_smem(THREADS) +
                      (MODE ? (size_t)(THREADS / 32) * A.k * sizeof(TopEnt) : 0);
  auto kern = k_scan_big<V64, MODE, THREADS>;
  cudaError_t e = allow_max_smem(kern);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, THREADS, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const int blocks = (int)max((u64)1, min((u64)num_sms() * per_sm, nq));
  kern<<<blocks, THREADS, smem, st>>>(A, q, nq, tb, &A.ctr->claim_c);
  return cudaGetLastError();
}

template <bool V64, int MODE>
static cudaError_t launch_big_v(const ScanArgs& A, const int4* q, u64 nq, cudaStream_t st) {
  if (A.big_threads == 512) return launch_big_t<V64, MODE, 512>(A, q, nq, st);
  return launch_big_t<V64, MODE, 1024>(A, q, nq, st);
}

cudaError_t launch_scan_cta(const ScanArgs& A, const int4* q, u64 nq, cudaStream_t st) {
  if (nq == 0) return cudaSuccess;
  const bool v64 = A.measure == LP_AA || A.measure == LP_RA;
  if (A.mode == 0) return v64 ? launch_big_v<true, 0>(A, q, nq, st) : launch_big_v<false, 0>(A, q, nq, st);
  return v64 ? launch_big_v<true, 1>(A, q, nq, st) : launch_big_v<false, 1>(A, q, nq, st);
}

cudaError_t launch_scan_med(const ScanArgs& A, const int4* q, u64 nq, cudaStream_t st) {
  if (nq == 0) return cudaSuccess;
  const bool v64 = A.measure == LP_AA || A.measure == LP_RA;
  u64* claim = &A.ctr->claim_m;
  const int tb = kMedSlots * (v64 ? 12 : 8);
  if (A.mode == 0)
    return v64 ? launch_cta_t<true, 0, kMedThreads>(A, q, nq, tb, claim, st)
               : launch_cta_t<false, 0, kMedThreads>(A, q, nq, tb, claim, st);
  return v64 ? launch_cta_t<true, 1, kMedThreads>(A, q, nq, tb, claim, st)
             : launch_cta_t<false, 1, kMedThreads>(A, q, nq, tb, claim, st);
}

// Load the code of every kernel the per-source mode launches, without
// launching any (cudaFuncGetAttributes loads a kernel that lazy module loading
// has not loaded yet; loading can allocate device memory for the code).
cudaError_t preload_sources_kernels() {
  cudaFuncAttributes fa;
  cudaError_t e = cudaSuccess;
  auto get = [&](auto kern) {
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kern);
  };
  auto big = [&](auto kern) {
    if (e == cudaSuccess) e = allow_max_smem(kern);
  };
  get(k_estimate<1, false>);
  get(k_estimate<1, true>);
  big(k_scan_warp<false, 1>);
  big(k_scan_warp<true, 1>);
  big(k_scan_cta<false, 1, kMedThreads>);
  big(k_scan_cta<true, 1, kMedThreads>);
  big(k_scan_big<false, 1, 512>);
  big(k_scan_big<true, 1, 512>);
  big(k_scan_big<false, 1, 1024>);
  big(k_scan_big<true, 1, 1024>);
  get(k_merge_partials);
  get(k_emit_sources);
  get(k_pair_cn);
  return e;
}

cudaError_t launch_merge_partials(const int4* grp_list, int ngrp, const int* order,
                                  const TopEnt* partial, const int2* hdr, int k, TopEnt* out_top,
                                  int* out_cnt, cudaStream_t st) {
  if (ngrp <= 0) return cudaSuccess;
  const int threads = 128;
  const size_t smem = (size_t)(threads / 32) * k * sizeof(TopEnt);
  const int blocks = (ngrp * 32 + threads - 1) / threads;
  k_merge_partials<<<blocks, threads, smem, st>>>(grp_list, ngrp, order, partial, hdr, k, out_top,
                                                   out_cnt);
  return cudaGetLastError();
}

cudaError_t launch_emit_global(const Cand* c, u64 n, int measure, int fixbits, lp_link* out,
                               cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_emit_global<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(c, n, measure, fixbits, out);
  return cudaGetLastError();
}

cudaError_t launch_emit_sources(const TopEnt* top, const int* cnt, const int* sources, int n_src,
                                int k, int measure, int fixbits, lp_link* out, cudaStream_t st) {
  const u64 n = (u64)n_src * k;
  if (n == 0) return cudaSuccess;
  k_emit_sources<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(top, cnt, sources, n_src, k, measure,
                                                               fixbits, out);
  return cudaGetLastError();
}

cudaError_t launch_link_keys(const lp_link* links, u64 n, int measure, const int* off,
                             const int* idx, const int* deg, const Arc* arc, int cap,
                             const u64* wt, Cand* out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const u64 threads = 256;
  k_link_keys<<<(unsigned)((n * 32 + threads - 1) / threads), (unsigned)threads, 0, st>>>(
      links, n, measure, off, idx, deg, arc, cap, wt, out);
  return cudaGetLastError();
}

cudaError_t launch_pair_cn(lp_link* links, const int* cnt_rows, int k, u64 n, const int* off,
                           const int* idx, const int* deg, const Arc* arc, int cap,
                           cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const u64 threads = 256;
  k_pair_cn<<<(unsigned)((n * 32 + threads - 1) / threads), (unsigned)threads, 0, st>>>(
      links, cnt_rows, k, n, off, idx, deg, arc, cap);
  return cudaGetLastError();
}

}  // namespace lp
