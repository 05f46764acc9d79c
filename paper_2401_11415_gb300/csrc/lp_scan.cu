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
//  * k_estimate: one warp per source computes the exact wedge count W(a)
//    from the per-arc table (hub arcs contribute nothing and their adjacency
//    lists are never read) and bins the source:
//      - W <= 512: warp tier, a per-warp open-addressing table in shared
//        memory sized 2W..4W slots;
//      - W <= 8192: one CTA item over the whole vertex range;
//      - larger: the c-range is cut into items; each item is a CTA with either
//        a shared-memory hash (split by vertex id, binary search per arc for
//        the sub-range) or a dense shared-memory counter array over an id
//        window (hubs whose second-order set is a large part of the graph).
//  * k_scan_warp / k_scan_cta: the wedge loop is flattened per warp: 32 arcs
//    are loaded (one int4 per lane), their suffix lengths prefix-summed with
//    shuffles, and the warp walks the concatenated suffixes 32 wedges at a
//    time, so every lane reads one coalesced neighbour id per step whatever
//    the intermediary degrees are.
//  * Counts are u32 (CN family).  AA and RA accumulate u64 fixed-point
//    weights round(2^F / ln|Gamma_b|) and round(2^F / |Gamma_b|): integer
//    addition is associative, so results do not depend on thread order.
#include <float.h>
#include <math.h>

#include "lp_internal.cuh"

namespace lp {

#define FULLMASK 0xffffffffu

__device__ __forceinline__ u32 hash_slot(int c, int logcap) {
  return ((u32)c * 0x9E3779B1u) >> (32 - logcap);
}

__host__ __device__ __forceinline__ int ceil_log2(u64 x) {
  int l = 0;
  while ((1ull << l) < x) ++l;
  return l;
}

// Fixed-point weight that intermediary b of degree db adds (Algorithm 1,
// scanEdges: 1/log|Gamma_b| for AA, 1/|Gamma_b| for RA, 1 otherwise).
template <typename V>
__device__ __forceinline__ V arc_weight(int measure, int db, int fixbits) {
  if (sizeof(V) == 8) {
    if (measure == LP_RA) return (V)__double2ull_rn(ldexp(1.0, fixbits) / (double)db);
    return (V)__double2ull_rn(ldexp(1.0, fixbits) / log((double)db));
  }
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

// Per record r (global mode: source r; per-source mode: sources[r]): exact
// wedge count and binning.  Warp records: {r, lo, hi, W | 1<<30}.  CTA items:
// {r, lo, hi, kind | logcap << 8}.  grp[r] = (first item, item count) in the
// per-source mode.
template <int MODE, bool V64>
__global__ void k_estimate(ScanArgs A, int n_rec, int4* __restrict__ warpq,
                           int4* __restrict__ itemq, u64 itemq_cap, int2* __restrict__ grp) {
  const int lane = lane_id();
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int dense_span = (V64 ? kCtaSmem / 8 : kCtaSmem / 4);
  for (int r = warp; r < n_rec; r += nwarps) {
    const int a = MODE ? A.sources[r] : r;
    const int e0 = A.off[a], e1 = A.off[a + 1];
    u64 W = 0;
    u32 kept = 0;
    for (int e = e0 + lane; e < e1; e += 32) {
      const Arc t = A.arc[e];
      if (t.z <= A.cap) {
        W += MODE ? (u64)(t.z - 1) : (u64)(t.y - t.x - 1);
        ++kept;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      W += __shfl_xor_sync(FULLMASK, W, o);
      kept += __shfl_xor_sync(FULLMASK, kept, o);
    }
    if (lane != 0) continue;
    atomicAdd(&A.ctr->wedges, W);
    atomicAdd(&A.ctr->kept_arcs, (u64)kept);
    atomicAdd(&A.ctr->scanned_arcs, (u64)(e1 - e0));
    const int lo = MODE ? 0 : a + 1;
    const int hi = A.n;
    if (MODE) grp[r] = make_int2(-1, 0);
    if (W == 0) {
      if (MODE) A.out_cnt[r] = 0;
      continue;
    }
    const int tier = W <= (u64)A.warp_max ? 0 : 1;
    atomicAdd(&A.ctr->tier_wedges[tier], W);
    atomicAdd(&A.ctr->tier_arcs[tier], (u64)(e1 - e0));
    atomicAdd(&A.ctr->tier_kept[tier], (u64)kept);
    if (tier == 0) {
      const u64 q = atomicAdd(&A.ctr->nwarp, 1ull);
      warpq[q] = make_int4(r, lo, hi, (int)W | (1 << 30));
      continue;
    }
    int P, kind, logcap;
    const u64 span = (u64)(hi - lo);
    if (W <= (u64)A.cta_max) {
      P = 1;
      kind = 0;
      logcap = max(10, ceil_log2(2 * W));
    } else {
      const u64 ph = (W + A.split_target - 1) / A.split_target;
      const u64 pd = (span + dense_span - 1) / dense_span;
      const double cost_h = (double)ph * kept * 24.0 + (double)W * 4.0;
      const double cost_d = (double)pd * ((double)kept * 24.0 + dense_span / 4.0) + (double)W;
      logcap = A.split_logcap;
      if (cost_d < cost_h) {
        P = (int)pd;
        kind = kItemDense;
      } else {
        P = (int)min(ph, span);
        kind = 0;
      }
    }
    if (MODE && P == 1) kind |= kItemSingle;
    const u64 base = atomicAdd(&A.ctr->nitem, (u64)P);
    if (kind & kItemDense) atomicAdd(&A.ctr->dense_items, (u64)P);
    if (base + P > itemq_cap) continue;  // host re-runs with a larger queue
    if (MODE) grp[r] = make_int2((int)base, P);
    for (int p = 0; p < P; ++p) {
      int l2, h2;
      if (kind & kItemDense) {
        l2 = lo + p * dense_span;
        h2 = min(hi, l2 + dense_span);
      } else {
        l2 = lo + (int)((span * (u64)p) / (u64)P);
        h2 = lo + (int)((span * (u64)(p + 1)) / (u64)P);
      }
      itemq[base + p] = make_int4(r, l2, h2, kind | (logcap << 8));
    }
  }
}

// ------------------------------------------------------- wedge flattening --

// The warp holds up to 32 arcs (lane j: suffix start s_j, length len_j,
// weight w_j).  Calls f(c, w) once for each of the sum(len) wedges, lane p
// of window `base` taking wedge base + p, so neighbour ids are read with
// consecutive addresses inside each suffix.
template <typename V, typename F>
__device__ __forceinline__ void flat_scan(int s, int len, V w, const int* __restrict__ idx,
                                          F&& f) {
  const int lane = lane_id();
  int incl = len;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(FULLMASK, incl, o);
    if (lane >= o) incl += t;
  }
  const int total = __shfl_sync(FULLMASK, incl, 31);
  const int excl = incl - len;
  for (int base = 0; base < total; base += 32) {
    const int p = base + lane;
    int j = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
      const int ej = __shfl_sync(FULLMASK, excl, j + step);
      if (ej <= p) j += step;
    }
    const int sj = __shfl_sync(FULLMASK, s, j);
    const int ej = __shfl_sync(FULLMASK, excl, j);
    const V wj = __shfl_sync(FULLMASK, w, j);
    if (p < total) f(__ldg(idx + sj + (p - ej)), wj);
  }
}

// First index in idx[l, r) whose value is >= key (lists are sorted).
__device__ __forceinline__ int lower_bound_g(const int* __restrict__ idx, int l, int r, int key) {
  while (l < r) {
    const int m = (l + r) >> 1;
    if (__ldg(idx + m) < key) l = m + 1; else r = m;
  }
  return l;
}

// ----------------------------------------------------------- hash tables --

// Add w to key c.  Returns 1 if c was new, 0 if it existed, 2 if the table
// had no free slot (bounded probe count).
template <typename V>
__device__ __forceinline__ int hash_add(int* keys, V* vals, int logcap, int c, V w) {
  const u32 mask = (1u << logcap) - 1u;
  u32 h = hash_slot(c, logcap);
  for (u32 probe = 0; probe <= mask; ++probe) {
    const int k = ((volatile int*)keys)[h];
    if (k == c) {
      atomicAdd(&vals[h], w);
      return 0;
    }
    if (k == kEmpty) {
      const int old = atomicCAS(&keys[h], kEmpty, c);
      if (old == kEmpty || old == c) {
        atomicAdd(&vals[h], w);
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
  u32 h = hash_slot(b, logcap);
  for (u32 probe = 0; probe <= mask; ++probe) {
    const int k = keys[h];
    if (k == b) {
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
  for (int i = lane; i < kWarpSlots; i += 32) {
    keys[i] = kEmpty;
    vals[i] = 0;
  }
  __syncwarp();
  Thresh T;
  if (MODE == 0) T = *A.thresh;
  const bool dc_needed = needs_dc(A.measure);
  u64 n_cand = 0;
  for (;;) {
    u64 qi = 0;
    if (lane == 0) {
      if (MODE == 0 && *(volatile u32*)&A.ctr->full) qi = ~0ull;
      else qi = atomicAdd(&A.ctr->claim_w, 1ull);
    }
    qi = __shfl_sync(FULLMASK, qi, 0);
    if (qi >= nq) break;
    const int4 rec = q[qi];
    const int r = rec.x;
    const int a = MODE ? A.sources[r] : r;
    const int W = rec.w & 0xffff;
    const int logcap = max(5, ceil_log2(2 * (u64)W));
    const int nslots = 1 << logcap;
    const int e0 = A.off[a], e1 = A.off[a + 1];
    // scan
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
          if (len > 0) w = arc_weight<V>(A.measure, t.z, A.fixbits);
        }
      }
      flat_scan<V>(s, len, w, A.idx, [&](int c, V wc) {
        if (MODE == 1 && c == a) return;
        hash_add<V>(keys, vals, logcap, c, wc);
      });
    }
    __syncwarp();
    // drop first-order neighbours
    for (int e = e0 + lane; e < e1; e += 32) {
      const int b = __ldg(A.idx + e);
      if (MODE == 1 || b > a) hash_kill<V>(keys, vals, logcap, b);
    }
    __syncwarp();
    // score and select
    const u64 da = (u64)(e1 - e0);
    bool fail = false;
    int tcnt = 0;
    for (int base = 0; base < nslots; base += 32) {
      const int slot = base + lane;
      const int c = keys[slot];
      const V v = vals[slot];
      keys[slot] = kEmpty;
      vals[slot] = 0;
      const bool live = (c != kEmpty) && (v != 0);
      u64 num = 0, den = 1;
      bool pass = false;
      if (live) {
        ++n_cand;
        const u64 dc = dc_needed ? (u64)__ldg(A.deg + c) : 0;
        make_key(A.measure, (u64)v, da, dc, num, den);
        pass = !A.thr_check || key_value(A.measure, num, den, (u64)v, A.fixbits) > A.threshold;
        if (MODE == 0 && pass && T.valid) pass = before(num, den, a, c, T.num, T.den, T.u, T.v);
      }
      if (MODE == 0) {
        fail |= admit_global(A, pass, num, den, a, c);
      } else {
        TopEnt x;
        x.num = num;
        x.den = den;
        x.c = c;
        x.cn = V64 ? 0 : (int)v;
        top_offer(top, tcnt, A.k, pass, x);
      }
    }
    __syncwarp();
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
  // per-warp candidate count
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) n_cand += __shfl_xor_sync(FULLMASK, n_cand, o);
  if (lane == 0 && n_cand) atomicAdd(&A.ctr->candidates, n_cand);
}

// ------------------------------------------------------------- CTA items ---

template <bool V64, int MODE>
__global__ void __launch_bounds__(kCtaThreads, 1) k_scan_cta(ScanArgs A, const int4* __restrict__ q,
                                                             u64 nq) {
  typedef typename std::conditional<V64, u64, u32>::type V;
  extern __shared__ __align__(16) unsigned char smem[];
  int* keys = reinterpret_cast<int*>(smem);
  V* vals = reinterpret_cast<V*>(smem + kCtaSlots * 4);
  V* dense = reinterpret_cast<V*>(smem);
  TopEnt* tops = reinterpret_cast<TopEnt*>(smem + kCtaSmem);
  __shared__ int4 s_rec;
  __shared__ u64 s_qi;
  __shared__ int s_ndistinct;
  __shared__ int s_overflow;
  __shared__ int s_fail;
  __shared__ int s_tcnt[kCtaWarps];

  const int lane = lane_id();
  const int wid = threadIdx.x >> 5;
  Thresh T;
  if (MODE == 0) T = *A.thresh;
  const bool dc_needed = needs_dc(A.measure);
  u64 n_cand = 0;
  for (;;) {
    if (threadIdx.x == 0) {
      u64 qi;
      if (MODE == 0 && *(volatile u32*)&A.ctr->full) qi = ~0ull;
      else qi = atomicAdd(&A.ctr->claim_c, 1ull);
      s_qi = qi;
      if (qi < nq) s_rec = q[qi];
      s_ndistinct = 0;
      s_overflow = 0;
      s_fail = 0;
    }
    __syncthreads();
    if (s_qi >= nq) break;
    const int4 rec = s_rec;
    const int r = rec.x;
    const int a = MODE ? A.sources[r] : r;
    const int lo = rec.y, hi = rec.z;
    const bool is_dense = (rec.w & kItemDense) != 0;
    const int logcap = (rec.w >> 8) & 0xff;
    const int nslots = 1 << logcap;
    const int limit = (nslots * 3) / 4;
    const bool full_range = (lo <= (MODE ? 0 : a + 1)) && hi >= A.n;
    const int span = hi - lo;
    // initialise the table / counters
    if (is_dense) {
      for (int i = threadIdx.x; i < span; i += blockDim.x) dense[i] = 0;
    } else {
      for (int i = threadIdx.x; i < nslots; i += blockDim.x) {
        keys[i] = kEmpty;
        vals[i] = 0;
      }
    }
    __syncthreads();
    const int e0 = A.off[a], e1 = A.off[a + 1];
    for (int eb = e0 + wid * 32; eb < e1; eb += kCtaWarps * 32) {
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
          if (len > 0) w = arc_weight<V>(A.measure, t.z, A.fixbits);
        }
      }
      if (is_dense) {
        flat_scan<V>(s, len, w, A.idx, [&](int c, V wc) {
          if (MODE == 1 && c == a) return;
          atomicAdd(&dense[c - lo], wc);
        });
      } else {
        flat_scan<V>(s, len, w, A.idx, [&](int c, V wc) {
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
      if (threadIdx.x == 0) {
        const u64 f = atomicAdd(&A.ctr->nsplit, 1ull);
        if (f < A.split_cap) A.split[f] = rec;
        else A.ctr->error = 2u;
      }
      __syncthreads();
      continue;
    }
    // drop first-order neighbours inside [lo, hi)
    for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
      const int b = __ldg(A.idx + e);
      if (b < lo || b >= hi || (MODE == 0 && b <= a)) continue;
      if (is_dense) dense[b - lo] = 0;
      else hash_kill<V>(keys, vals, logcap, b);
    }
    __syncthreads();
    // score and select
    const u64 da = (u64)(e1 - e0);
    const int nscan = is_dense ? span : nslots;
    const int nscan32 = (nscan + 31) & ~31;
    bool fail = false;
    TopEnt* top = tops + wid * (MODE ? A.k : 0);
    int tcnt = 0;
    for (int i = threadIdx.x; i < nscan32; i += blockDim.x) {  // warp-uniform trip count
      int c = kEmpty;
      V v = 0;
      if (i < nscan) {
        if (is_dense) {
          v = dense[i];
          c = lo + i;
        } else {
          c = keys[i];
          v = vals[i];
        }
      }
      const bool live = (c != kEmpty) && (v != 0);
      u64 num = 0, den = 1;
      bool pass = false;
      if (live) {
        ++n_cand;
        const u64 dc = dc_needed ? (u64)__ldg(A.deg + c) : 0;
        make_key(A.measure, (u64)v, da, dc, num, den);
        pass = !A.thr_check || key_value(A.measure, num, den, (u64)v, A.fixbits) > A.threshold;
        if (MODE == 0 && pass && T.valid) pass = before(num, den, a, c, T.num, T.den, T.u, T.v);
      }
      if (MODE == 0) {
        fail |= admit_global(A, pass, num, den, a, c);
      } else {
        TopEnt x;
        x.num = num;
        x.den = den;
        x.c = c;
        x.cn = V64 ? 0 : (int)v;
        top_offer(top, tcnt, A.k, pass, x);
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
        for (int w2 = 1; w2 < kCtaWarps; ++w2) {
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
          if (lane == 0) p = atomicAdd(&A.ctr->npartial, 1ull);
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
  if (j >= cnt[r]) return;
  const TopEnt x = top[i];
  u64 cn = (u64)x.cn;
  out[i] = make_link(measure, sources[r], x.c, x.num, x.den, cn, fixbits);
}

// Common neighbours b of (u, v) with |Gamma_b| <= cap, one warp per link
// (AA / RA lists, whose tables hold weight sums rather than counts).
__global__ void k_pair_cn(lp_link* __restrict__ links, const int* __restrict__ cnt_rows, int k,
                          u64 n, const int* __restrict__ off, const int* __restrict__ idx,
                          const int* __restrict__ deg, int cap) {
  const u64 gw = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = lane_id();
  if (gw >= n) return;
  if (cnt_rows && (int)(gw % k) >= cnt_rows[gw / k]) return;
  lp_link L = links[gw];
  int x = L.u, y = L.v;
  if (off[x + 1] - off[x] > off[y + 1] - off[y]) {
    const int t = x;
    x = y;
    y = t;
  }
  const int ys = off[y], ye = off[y + 1];
  int c = 0;
  for (int e = off[x] + lane; e < off[x + 1]; e += 32) {
    const int b = __ldg(idx + e);
    if (__ldg(deg + b) > cap) continue;
    const int p = lower_bound_g(idx, ys, ye, b);
    if (p < ye && __ldg(idx + p) == b) ++c;
  }
  c = __reduce_add_sync(FULLMASK, (u32)c);
  if (lane == 0) links[gw].cn = c;
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

cudaError_t launch_estimate(const ScanArgs& A, int n_rec, int4* warpq, int4* itemq, u64 itemq_cap,
                            int2* grp, cudaStream_t st) {
  if (n_rec <= 0) return cudaSuccess;
  const int threads = 256;
  const int blocks = (int)min((u64)num_sms() * 8, ((u64)n_rec * 32 + threads - 1) / threads);
  const bool v64 = A.measure == LP_AA || A.measure == LP_RA;
  if (A.mode == 0) {
    if (v64) k_estimate<0, true><<<blocks, threads, 0, st>>>(A, n_rec, warpq, itemq, itemq_cap, grp);
    else k_estimate<0, false><<<blocks, threads, 0, st>>>(A, n_rec, warpq, itemq, itemq_cap, grp);
  } else {
    if (v64) k_estimate<1, true><<<blocks, threads, 0, st>>>(A, n_rec, warpq, itemq, itemq_cap, grp);
    else k_estimate<1, false><<<blocks, threads, 0, st>>>(A, n_rec, warpq, itemq, itemq_cap, grp);
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
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
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

template <bool V64, int MODE>
static cudaError_t launch_cta_t(const ScanArgs& A, const int4* q, u64 nq, cudaStream_t st) {
  const size_t smem = (size_t)kCtaSmem + (MODE ? (size_t)kCtaWarps * A.k * sizeof(TopEnt) : 0);
  auto kern = k_scan_cta<V64, MODE>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int blocks = (int)max((u64)1, min((u64)num_sms(), nq));
  kern<<<blocks, kCtaThreads, smem, st>>>(A, q, nq);
  return cudaGetLastError();
}

cudaError_t launch_scan_cta(const ScanArgs& A, const int4* q, u64 nq, cudaStream_t st) {
  if (nq == 0) return cudaSuccess;
  const bool v64 = A.measure == LP_AA || A.measure == LP_RA;
  if (A.mode == 0) return v64 ? launch_cta_t<true, 0>(A, q, nq, st) : launch_cta_t<false, 0>(A, q, nq, st);
  return v64 ? launch_cta_t<true, 1>(A, q, nq, st) : launch_cta_t<false, 1>(A, q, nq, st);
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

cudaError_t launch_pair_cn(lp_link* links, const int* cnt_rows, int k, u64 n, const int* off,
                           const int* idx, const int* deg, int cap, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const u64 threads = 256;
  k_pair_cn<<<(unsigned)((n * 32 + threads - 1) / threads), (unsigned)threads, 0, st>>>(
      links, cnt_rows, k, n, off, idx, deg, cap);
  return cudaGetLastError();
}

}  // namespace lp
