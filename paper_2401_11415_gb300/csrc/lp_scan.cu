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
#include "lp_scan_dev.cuh"

namespace lp {

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

// --------------------------------------------------------------- estimate --

struct TierStats {
  u64 w[4], a[4], k[4];
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
  for (int i = 0; i < 4; ++i) ts.w[i] = ts.a[i] = ts.k[i] = 0;
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
    // global mode: a large source that would be cut into several items is
    // expanded and counted by bucket instead (wedge offsets are 32-bit)
    if (MODE == 0 && tier == 2 && A.expand && W > (u64)A.x_min && W < (1ull << 31)) tier = 3;
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
    // expand-and-count tier: one unit record per source
    if (MODE == 0) {
      const u32 m = __ballot_sync(FULLMASK, tier == 3);
      if (m) {
        const int leader = __ffs(m) - 1;
        u64 q = 0;
        if (lane == leader) q = atomicAdd(&A.ctr->nexp, (u64)__popc(m));
        q = __shfl_sync(FULLMASK, q, leader);
        const u64 pos = q + __popc(m & lt);
        if (tier == 3 && pos < A.xq_cap) {  // else the host re-runs with a larger queue
          A.xq[pos] = make_int4(r, lo, hi, (int)kept);
          A.xw[pos] = W;
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
  for (int i = 0; i < 4; ++i) {
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
    for (int i = 0; i < 4; ++i) {
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
          if (hash_add<V>(keys, vals, logcap, c, wc, fill_probes(logcap)) == 2) s_overflow = 1;
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
  __shared__ int s_overflow, s_fail, s_qnl, s_qns;
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
          if (hash_add<V>(keys, vals, logcap, c, wc, fill_probes(logcap)) == 2) s_overflow = 1;
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
        // A warp takes pieces p = wid, wid + NW, ...: the loads of its next
        // piece are issued before the inserts of the current one.
        int jl = 0;   // long segment of the warp's last piece
        int jsh = H;  // short segment of the lane's last wedge
        auto fetch = [&](int p, int (&c8)[kPerLane], int (&j8)[kPerLane]) {
          if (p < npl) {
            // c_p rises strictly over the long segments and the last piece,
            // p - NW, lay in segment jl: p lies in one of jl .. jl + NW, and
            // one ballot over the next 32 starts finds it
            const int cand = jl + 1 + lane;
            jl += __popc(__ballot_sync(FULLMASK, cand < nl && c_p[cand] <= p));
            const int off = (p - c_p[jl]) * kPiece;
            const int plen = min(kPiece, c_l[jl] - off);
            const int* src = A.idx + c_s[jl] + off;
#pragma unroll
            for (int u = 0; u < kPerLane; ++u) {
              c8[u] = lane + 32 * u < plen ? __ldg(src + lane + 32 * u) : -1;
              j8[u] = jl;
            }
          } else {
            const int i0 = (p - npl) * kPiece + lane;
            // the lane's wedges rise from piece to piece
            if (i0 < tsw) jsh = last_le(c_p, jsh, H + ns, i0);
#pragma unroll
            for (int u = 0; u < kPerLane; ++u) {
              const int i = i0 + 32 * u;
              c8[u] = -1;
              if (i < tsw) {
                // i - 32 lay in segment jsh and segments are not empty, so i
                // lies in one of the segments jsh .. jsh + 32
                if (jsh + 1 < H + ns && c_p[jsh + 1] <= i)
                  jsh = last_le(c_p, jsh + 1, min(H + ns, jsh + 33), i);
                c8[u] = __ldg(A.idx + c_s[jsh] + i);
              }
              j8[u] = jsh;
            }
          }
        };
        int c8[kPerLane], j8[kPerLane];
        if (wid < npieces) fetch(wid, c8, j8);
        for (int p = wid; p < npieces; p += NW) {  // warp-uniform trips
          int n8[kPerLane], m8[kPerLane];
#pragma unroll
          for (int u = 0; u < kPerLane; ++u) n8[u] = m8[u] = -1;
          if (p + NW < npieces) fetch(p + NW, n8, m8);
#pragma unroll
          for (int u = 0; u < kPerLane; ++u)
            if (c8[u] >= 0) insert(c8[u], V64 ? (V)c_w[j8[u]] : (V)1);
          if (!is_dense && __any_sync(FULLMASK, *(volatile int*)&s_overflow != 0)) break;
#pragma unroll
          for (int u = 0; u < kPerLane; ++u) {
            c8[u] = n8[u];
            j8[u] = m8[u];
          }
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
