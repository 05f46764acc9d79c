// lp_expand.cu -- the expand-and-count large tier of the global mode.
//
// Algorithm 1 counts, for a source a, the paths a -> b -> c (c > a) through
// intermediaries b with |Gamma_b| <= L_H into a table indexed by c
// (scanEdges; Sections 4.1.2-4.1.3, 4.2.1).  For a source whose second-order
// vertices spread over more ids than one shared-memory table covers, the
// window sweeps of the large tier revisit every arc of the source once per
// id window; when the index array does not stay in the L2 cache those visits
// are DRAM round trips and cost far more than the wedges themselves.  This
// tier reads every wedge once instead:
//
//  * arc pass (k_exp_arcs, one CTA per source): the kept arcs' c > a
//    suffixes, compacted, with their running wedge offsets;
//  * expand pass (k_exp_tiles, one CTA per tile of consecutive arcs): every
//    wedge's c (with |Gamma_b| for AA / RA) is read once, streamed by the
//    warp-cooperative wedge loop, histogrammed by bucket (an id range of
//    2^wlog) in shared memory, and written back grouped by bucket within the
//    tile, with the tile's bucket starts;
//  * count pass (k_exp_count, one CTA per bucket): the bucket's records from
//    every tile of the source are counted in shared memory -- dense counters
//    when the source's wedges are dense in its id range, else a hash table
//    -- then the first-order neighbours are dropped (Section 4.1.4) and the
//    counters scored and admitted exactly as in the other tiers (Eq. 1-9,
//    count floor, admission threshold; Sections 4.1.5-4.1.6).
//
// Records are the only extra traffic: 4 bytes per wedge written and read
// back (8 for AA / RA), against the per-arc round trips of every window.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "lp_internal.cuh"
#include "lp_scan_dev.cuh"

namespace lp {

constexpr int kExpThreads = 256;    // arc and expand passes
constexpr int kSub = kExpThreads / 32;  // a tile's sub-tiles: one per warp of the expand CTA
constexpr int kCountThreads = 256;  // count pass (three CTAs per SM)

// Exclusive CTA-wide prefix sums of two ints per thread (ex, ey) and their
// totals.  wsum: 2 * (threads / 32) ints of shared memory; one barrier, and
// wsum must not be written again before the caller's next barrier.
template <int THREADS>
__device__ __forceinline__ void exp_scan2(int x, int y, int& ex, int& ey, int& tx, int& ty,
                                          int* wsum) {
  constexpr int NW = THREADS / 32;
  const int lane = lane_id(), wid = threadIdx.x >> 5;
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
  if (lane == 31) {
    wsum[wid] = ix;
    wsum[NW + wid] = iy;
  }
  __syncthreads();
  int bx = 0, by = 0;
  tx = ty = 0;
#pragma unroll
  for (int w = 0; w < NW; ++w) {
    const int vx = wsum[w], vy = wsum[NW + w];
    if (w < wid) {
      bx += vx;
      by += vy;
    }
    tx += vx;
    ty += vy;
  }
  ex = bx + ix - x;
  ey = by + iy - y;
}

// ------------------------------------------------------------- arc pass --

// One CTA per unit: the kept arcs (|Gamma_b| <= L_H) with a nonempty c > a
// suffix of Gamma_b, compacted: aseg = first index of the suffix in idx, aoff
// = wedges of the unit before it (aoff[K] = W), adeg = |Gamma_b| (AA / RA).
// Then the first segment of every sub-tile (tiles of tile_w wedges, cut into
// kSub sub-tiles of tile_w / kSub, take the segments that start in them)
// and, for every bucket, the first entry of
// Gamma_a at or above the bucket's start (c > a) -- the count pass's
// first-order exclusion range -- so that neither pass searches.
__global__ void __launch_bounds__(kExpThreads) k_exp_arcs(ScanArgs A, ExpUnit* __restrict__ units,
                                                           int nunits, int* __restrict__ aseg,
                                                           int* __restrict__ aoff,
                                                           int* __restrict__ adeg,
                                                           int* __restrict__ tfirst,
                                                           int* __restrict__ excl) {
  __shared__ int wsum[2 * (kExpThreads / 32)];
  for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
    const ExpUnit U = units[u];
    const int a = U.a;
    const long long base = U.arc_base;
    const int e0 = A.off[a], e1 = A.off[a + 1];
    int carry = 0, cnt = 0;
    for (int eb = e0; eb < e1; eb += kExpThreads) {  // CTA-uniform trips
      const int e = eb + threadIdx.x;
      int s0 = 0, len = 0, db = 0;
      if (e < e1) {
        const Arc t = A.arc[e];
        if (t.z <= A.cap) {
          s0 = t.x + 1;
          len = t.y - s0;
          db = t.z;
        }
      }
      if (len < 0) len = 0;
      const int nz = len > 0 ? 1 : 0;
      int elen, enz, tlen, tnz;
      exp_scan2<kExpThreads>(len, nz, elen, enz, tlen, tnz, wsum);
      if (nz) {
        const long long k = base + cnt + enz;
        aseg[k] = s0;
        aoff[k] = carry + elen;
        if (adeg) adeg[k] = db;
      }
      carry += tlen;
      cnt += tnz;
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      aoff[base + cnt] = carry;
      units[u].K = cnt;
      if ((long long)carry != U.W) atomicExch(&A.ctr->error, 4u);
    }
    __syncthreads();  // this CTA's segment offsets are visible to it
    // sub-tile t starts at the first segment j with aoff[j] >= t * sw:
    // segment j is the first of the sub-tiles in (aoff[j-1] / sw, aoff[j] / sw]
    const long long tw = U.tile_w / kSub;
    const long long nsub = (long long)U.T * kSub;
    int* tf = tfirst + U.tfirst_base;
    for (int j = threadIdx.x; j <= cnt; j += kExpThreads) {
      long long t0, t1;
      if (j == 0) {
        t0 = 0;
        t1 = 0;
      } else if (j < cnt) {
        t0 = (long long)aoff[base + j - 1] / tw + 1;
        t1 = (long long)aoff[base + j] / tw;
      } else {  // sub-tiles past the last segment's start: no segment
        t0 = cnt > 0 ? (long long)aoff[base + cnt - 1] / tw + 1 : 0;
        t1 = nsub;
      }
      for (long long t = t0; t <= t1 && t <= nsub; ++t) tf[t] = j;
    }
    // exclusion table: entry b = first index of Gamma_a with value >= the
    // bucket's start lo + b 2^wlog (entry nb: >= hi); lo > a, so these are
    // first-order neighbours above a.  With g(x) the number of starts <= x,
    // entry e of Gamma_a begins the entries b in [g(Gamma_a[e-1]), g(Gamma_a[e])):
    // one pass over Gamma_a, no search.
    int* ex = excl + U.excl_base;
    const int lo = U.lo, hi = U.hi, nb = U.nb, wlog = U.wlog;
    auto starts_le = [&](int x) {
      return x < lo ? 0 : (x >= hi ? nb + 1 : ((x - lo) >> wlog) + 1);
    };
    for (int e = e0 + threadIdx.x; e <= e1; e += kExpThreads) {
      const int gp = e > e0 ? starts_le(__ldg(A.idx + e - 1)) : 0;
      const int gc = e < e1 ? starts_le(__ldg(A.idx + e)) : nb + 1;
      for (int b = gp; b < gc; ++b) ex[b] = e;
    }
    __syncthreads();
  }
}

// ----------------------------------------------------------- expand pass --

// One CTA per tile: the segments of the unit that start in
// [tl * tile_w, (tl + 1) * tile_w), each warp those of one sub-tile (about
// tile_w / kSub wedges, so the warps reach the barriers together).  Two
// passes over their wedges (the second from the cache): a bucket histogram,
// then every record written to its bucket's slot within the tile.
template <bool V64>
__global__ void __launch_bounds__(kExpThreads) k_exp_tiles(ScanArgs A, const ExpUnit* __restrict__ units,
                                                           const int* __restrict__ tile_unit,
                                                           int ntiles, const int* __restrict__ aseg,
                                                           const int* __restrict__ aoff,
                                                           const int* __restrict__ adeg,
                                                           const int* __restrict__ tfirst,
                                                           void* __restrict__ rec,
                                                           u64* __restrict__ tile_rec,
                                                           int* __restrict__ pre) {
  constexpr int NW = kExpThreads / 32;
  __shared__ int hist[kExpMaxBuckets];
  __shared__ int wsum[2 * NW];
  const int lane = lane_id(), wid = threadIdx.x >> 5;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int u = tile_unit[t];
    const ExpUnit U = units[u];
    const long long tl = t - U.tile_base;
    const int* off_u = aoff + U.arc_base;
    const int* tf = tfirst + U.tfirst_base + tl * kSub;
    const int j0 = tf[0];                    // the tile's first segment
    const int jw0 = tf[wid], jw1 = tf[wid + 1];  // this warp's sub-tile
    for (int b = threadIdx.x; b < U.nb; b += kExpThreads) hist[b] = 0;
    __syncthreads();
    const int lo = U.lo, wlog = U.wlog;
    // pass 1: bucket histogram
    for (int jb = jw0; jb < jw1; jb += 32) {  // warp-uniform trips
      const int j = jb + lane;
      int s = 0, len = 0;
      if (j < jw1) {
        s = aseg[U.arc_base + j];
        len = off_u[j + 1] - off_u[j];
      }
      scan_arcs<int>(s, len, 0, A.idx, [&](int c, int) { atomicAdd(&hist[(c - lo) >> wlog], 1); });
    }
    __syncthreads();
    // exclusive prefix of the histogram (each thread a run of buckets); the
    // starts become the write cursors and the tile's bucket-start table
    const int per = (U.nb + kExpThreads - 1) / kExpThreads;
    const int b0 = min(U.nb, (int)threadIdx.x * per), b1 = min(U.nb, b0 + per);
    int run = 0;
    for (int b = b0; b < b1; ++b) run += hist[b];
    int ex, ey, tot, tot2;
    exp_scan2<kExpThreads>(run, 0, ex, ey, tot, tot2, wsum);
    int* pt = pre + U.pre_base + tl * (U.nb + 1);
    for (int b = b0; b < b1; ++b) {
      const int h = hist[b];
      hist[b] = ex;
      pt[b] = ex;
      ex += h;
    }
    const u64 rb = (u64)(U.rec_base + off_u[j0]);
    if (threadIdx.x == 0) {
      pt[U.nb] = tot;
      tile_rec[t] = rb;
    }
    __syncthreads();
    // pass 2: every record to its bucket's next slot
    for (int jb = jw0; jb < jw1; jb += 32) {  // warp-uniform trips
      const int j = jb + lane;
      int s = 0, len = 0, db = 0;
      if (j < jw1) {
        s = aseg[U.arc_base + j];
        len = off_u[j + 1] - off_u[j];
        if (V64) db = adeg[U.arc_base + j];
      }
      scan_arcs<int>(s, len, db, A.idx, [&](int c, int w) {
        const int pos = atomicAdd(&hist[(c - lo) >> wlog], 1);
        if (V64) reinterpret_cast<int2*>(rec)[rb + pos] = make_int2(c, w);
        else reinterpret_cast<int*>(rec)[rb + pos] = c;
      });
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------ count pass --

// One CTA per count item {a, clo, chi, batch bucket | kExpItem}; three CTAs
// of kCountThreads per SM (a 64 KB table each).  Per item: the run table (the
// bucket's first and last record in every tile of the unit) and the slice of
// Gamma_a in the bucket are loaded at once; the records with clo <= c < chi
// are counted in shared memory, each warp taking an equal share of them in
// the order of the runs; the first-order neighbours are dropped; and the
// counters are scored and admitted.  The next item's record and unit are
// fetched by thread 0 while the current one is counted, so its chain of
// dependent loads overlaps the work.  A hash item whose table fills is handed
// back for splitting; a dense item cannot overflow.
template <bool V64>
__global__ void __launch_bounds__(kCountThreads, 3) k_exp_count(ScanArgs A, const int4* __restrict__ q,
                                                                u64 nq, u64* __restrict__ claim) {
  typedef typename std::conditional<V64, u64, u32>::type V;
  constexpr int NW = kCountThreads / 32;
  constexpr int kSlotsMax = kExpTableBytes / (4 + sizeof(V)) >= 8192 ? 8192 : 4096;
  const int logcap = A.x_logcap;
  extern __shared__ __align__(16) unsigned char smem[];  // kExpTableBytes
  int* keys = reinterpret_cast<int*>(smem);
  V* vals = reinterpret_cast<V*>(smem + (size_t)kSlotsMax * 4);
  u32* words = reinterpret_cast<u32*>(smem);
  __shared__ int s_p0[kExpMaxTiles];       // run start within its tile
  __shared__ int s_pre[kExpMaxTiles + 1];  // records before the run (flattened order)
  __shared__ u64 s_rb[kExpMaxTiles];       // the tile's first record
  __shared__ int2 s_wsum[NW];
  __shared__ int4 s_rec, s_rec_next;
  __shared__ ExpUnit s_unit, s_unit_next;
  __shared__ int s_p0n[kExpMaxTiles], s_lenn[kExpMaxTiles];  // the next item's runs
  __shared__ u64 s_rbn[kExpMaxTiles];
  __shared__ u64 s_next;
  __shared__ int s_overflow, s_fail, s_e0, s_e1, s_e0n, s_e1n;
  const int lane = lane_id(), wid = threadIdx.x >> 5;
  for (int i = threadIdx.x * 16; i < kExpTableBytes; i += kCountThreads * 16)
    *reinterpret_cast<int4*>(smem + i) = make_int4(0, 0, 0, 0);
  const Thresh T = *A.thresh;
  u64 n_cand = 0;
  // warp 0: claim the next item and load its record, unit, run of every tile
  // and slice of Gamma_a, so that none of these chains of dependent loads
  // lies on the path of the item after it
  auto prefetch = [&]() {
    if (lane == 0) {
      const u64 nx = *(volatile u32*)&A.ctr->full ? ~0ull : atomicAdd(claim, 1ull);
      s_next = nx;
      if (nx < nq) {
        s_rec_next = q[nx];
        s_unit_next = A.xunit[A.xbucket_unit[s_rec_next.w & kExpGbMask]];
      }
    }
    __syncwarp();
    if (s_next >= nq) return;  // warp-uniform
    const int4 r = s_rec_next;
    const ExpUnit& U = s_unit_next;
    const int bb = (int)((r.w & kExpGbMask) - U.bucket_base);
    for (int tt = lane; tt < U.T; tt += 32) {
      const int* pt = A.xpre + U.pre_base + (long long)tt * (U.nb + 1) + bb;
      const int p0 = pt[0];
      s_p0n[tt] = p0;
      s_lenn[tt] = pt[1] - p0;
      s_rbn[tt] = A.xtile_rec[U.tile_base + tt];
    }
    if (lane == 0) {
      const int* ex = A.xexcl + U.excl_base + bb;
      int e0 = ex[0], e1 = ex[1];
      if (r.w & kExpSplit) {  // a part of the bucket: narrow the slice
        e0 = lower_bound_g(A.idx, e0, e1, max(r.y, r.x + 1));
        e1 = lower_bound_g(A.idx, e0, e1, r.z);
      }
      s_e0n = e0;
      s_e1n = e1;
    }
  };
  if (wid == 0) prefetch();
  __syncthreads();
  for (;;) {
    const u64 qi = s_next;
    if (qi >= nq) break;
    if (threadIdx.x == 0) {
      s_rec = s_rec_next;
      s_unit = s_unit_next;
      s_e0 = s_e0n;
      s_e1 = s_e1n;
      s_fail = 0;
      s_overflow = 0;
    }
    __syncthreads();
    const int4 rec = s_rec;
    const ExpUnit& U = s_unit;
    const int a = rec.x, clo = rec.y, chi = rec.z;
    const int gb = rec.w & kExpGbMask;
    const int b = (int)(gb - U.bucket_base);
    const bool dense = (U.flags & kExpDense) != 0;
    const int cw = U.flags & 3;
    const int wlog = U.wlog, nt = U.T;
    const int lg = clo, hg = chi;
    const int nslots = 1 << logcap;
    const int limit = (nslots * 3) / 4;
    u32* dlo = words;
    u32* dhi = words + (1 << wlog);
    (void)b;
    // the bucket's run in every tile (one per thread; loaded ahead) and
    // their prefix
    {
      int len = 0;
      const int tt = threadIdx.x;
      if (tt < nt) {
        len = s_lenn[tt];
        s_p0[tt] = s_p0n[tt];
        s_rb[tt] = s_rbn[tt];
      }
      int incl = len;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(FULLMASK, incl, o);
        if (lane >= o) incl += t;
      }
      if (lane == 31) s_wsum[wid] = make_int2(incl, 0);
      __syncthreads();
      int before = 0, total = 0;
#pragma unroll
      for (int w = 0; w < NW; ++w) {
        const int v = s_wsum[w].x;
        if (w < wid) before += v;
        total += v;
      }
      if (tt < nt) s_pre[tt] = before + incl - len;
      if (threadIdx.x == 0) s_pre[nt] = total;
    }
    __syncthreads();
    if (wid == 0) prefetch();  // the next item, while this one is counted
    // a table that receives at most `limit` records stays at most three
    // quarters full: then it is probed to the end and never overflows
    const int R = s_pre[nt];
    const bool guard = !dense && R > limit;
    auto insert = [&](int c, V wc) {
      if (dense) {
        const int p = swz(c - lg);
        if (cw == kExpC8) {
          atomicAdd(words + (p >> 2), 1u << ((p & 3) << 3));
        } else if (cw == kExpC16) {
          atomicAdd(words + (p >> 1), 1u << ((p & 1) << 4));
        } else if (cw == kExpC32) {
          atomicAdd(words + p, (u32)wc);
        } else {  // split halves: low word, then high word plus carry
          const u32 l = (u32)wc, h = (u32)((u64)wc >> 32);
          const u32 old = atomicAdd(dlo + p, l);
          const u32 hc = h + ((old + l < old) ? 1u : 0u);
          if (hc) atomicAdd(dhi + p, hc);
        }
      } else if (!guard) {
        // the bucket cannot fill: claim or find the key with one compare-and-swap
        // per probe (most keys of a hash bucket are new)
        const u32 mask = (1u << logcap) - 1u;
        u32 h = hash_slot(c + 1, logcap);
        for (u32 probe = 0;; ++probe) {
          if (probe > mask) {  // cannot happen: at most 3/4 of the slots are taken
            A.ctr->error = 5u;
            return;
          }
          const int old = atomicCAS(&keys[h], kEmpty, c + 1);
          if (old == kEmpty || old == c + 1) break;
          h = (h + 1u) & mask;
        }
        shared_add<V>(&vals[h], wc);
      } else {
        if (*(volatile int*)&s_overflow) return;
        if (hash_add<V>(keys, vals, logcap, c, wc, fill_probes(logcap)) == 2) s_overflow = 1;
      }
    };
    // insert the bucket's records: warp w > 0 takes the flattened records
    // [(w - 1) R / (NW - 1), w R / (NW - 1)); warp 0 fetches the next item
    // meanwhile (its chain of dependent loads stays off the barrier's path)
    if (wid > 0) {
      const int r0 = (int)(((long long)R * (wid - 1)) / (NW - 1));
      const int r1 = (int)(((long long)R * wid) / (NW - 1));
      int tt = 0;
      {  // the run holding r0 (last tt with s_pre[tt] <= r0)
        int l = 0, h = nt;
        while (h - l > 1) {
          const int m = (l + h) >> 1;
          if (s_pre[m] <= r0) l = m; else h = m;
        }
        tt = l;
      }
      // 256 records per step, eight loads in flight per lane before any insert
      for (int rb0 = r0; rb0 < r1; rb0 += 256) {  // warp-uniform trips
        int cc[8], dd[8];
        int t = tt;  // the lane's run, carried from record to record (they rise)
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int r = rb0 + 32 * k + lane;
          cc[k] = -1;
          dd[k] = 0;
          if (r < r1) {
            while (s_pre[t + 1] <= r) ++t;
            const u64 at = s_rb[t] + (u64)(s_p0[t] + (r - s_pre[t]));
            if (V64) {
              const int2 x = reinterpret_cast<const int2*>(A.xrec)[at];
              cc[k] = x.x;
              dd[k] = x.y;  // |Gamma_b|, for the weight lookup below
            } else {
              cc[k] = reinterpret_cast<const int*>(A.xrec)[at];
            }
          }
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int c = cc[k];
          if (c >= clo && c < chi) insert(c, V64 ? (V)__ldg(A.wt + dd[k]) : (V)1);
        }
        // the run of the warp's next first record
        const int rn = min(rb0 + 256, r1 - 1);
        while (tt + 1 < nt && s_pre[tt + 1] <= rn) ++tt;
        if (guard && *(volatile int*)&s_overflow) break;
      }
    }
    __syncthreads();
    if (guard && s_overflow) {
      // hand the item back for splitting; leave the table empty
      for (int i = threadIdx.x * 4; i < nslots; i += kCountThreads * 4) {
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
    // drop the first-order neighbours c in [max(clo, a + 1), chi)
    for (int e = s_e0 + threadIdx.x; e < s_e1; e += kCountThreads) {
      const int c = __ldg(A.idx + e);
      if (dense) {
        const int p = swz(c - lg);
        if (cw == kExpC8) atomicAnd(words + (p >> 2), ~(0xffu << ((p & 3) << 3)));
        else if (cw == kExpC16) atomicAnd(words + (p >> 1), ~(0xffffu << ((p & 1) << 4)));
        else if (cw == kExpC32) words[p] = 0;
        else {
          dlo[p] = 0;
          dhi[p] = 0;
        }
      } else {
        hash_kill<V>(keys, vals, logcap, c);
      }
    }
    __syncthreads();
    // score: every counter or slot once; the ones below the count floor of
    // the source's degree are only counted
    const u64 da = (u64)(A.off[a + 1] - A.off[a]);
    const u64 vmin = T.valid ? __ldg(A.vfloor + da) : 1;
    bool fail = false;
    int qn = 0, qc = 0, qd = 0;
    V qv = 0;
    const int npos = (hg - lg + 31) & ~31;
    if (dense && cw == kExpC8) {
      u32 q8 = (u32)qv;
      for (int base0 = wid * 256; base0 < npos; base0 += kCountThreads * 8)  // warp-uniform
        fail |= score_dense8_linear(A, T, a, da, words, base0, npos, lg, vmin, n_cand, qn, qc, q8,
                                    qd);
      qv = (V)q8;
    } else if (dense && cw == kExpC16) {
      u32 q16 = (u32)qv;
      for (int base0 = wid * 256; base0 < npos; base0 += kCountThreads * 8)  // warp-uniform
        fail |= score_dense16_linear(A, T, a, da, words, base0, npos, lg, vmin, n_cand, qn, qc,
                                     q16, qd);
      qv = (V)q16;
    } else if (dense && cw == kExpC32) {
      u32 q32 = (u32)qv;
      for (int base0 = wid * 128; base0 < npos; base0 += kCountThreads * 4)  // warp-uniform
        fail |= score_dense_linear<u32>(A, T, a, da, words, base0, npos, lg, vmin, n_cand, qn, qc,
                                        q32, qd);
      qv = (V)q32;
    } else if (dense) {
      u64 q64 = (u64)qv;
      for (int base0 = wid * 128; base0 < npos; base0 += kCountThreads * 4)  // warp-uniform
        fail |= score_dense64_linear(A, T, a, da, dlo, dhi, base0, npos, lg, vmin, n_cand, qn, qc,
                                     q64, qd);
      qv = (V)q64;
    } else if (T.valid) {
      for (int base0 = wid * 128; base0 < nslots; base0 += kCountThreads * 4)
        fail |= score_hash_linear<V>(A, T, a, da, keys, vals, base0, nslots, vmin, n_cand, qn, qc,
                                     qv, qd);
    } else {
      int tcnt = 0;
      for (int base0 = wid * 128; base0 < nslots; base0 += kCountThreads * 4)
        fail |= score_hash_chunk<V, 0>(A, T, a, da, keys, vals, base0, nslots, nullptr, tcnt,
                                       n_cand);
    }
    if (qn > 0) fail |= survivors_flush<V>(A, T, a, da, qn, qc, qv, qd);
    if (fail && lane == 0) s_fail = 1;
    __syncthreads();
    if (threadIdx.x == 0 && s_fail) {
      A.ctr->full = 1u;
      const u64 f = atomicAdd(&A.ctr->nfailed, 1ull);
      if (f < A.failed_cap) A.failed[f] = rec;
      else A.ctr->error = 1u;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) n_cand += __shfl_xor_sync(FULLMASK, n_cand, o);
  if (lane == 0 && n_cand) atomicAdd(&A.ctr->candidates, n_cand);
}

// ------------------------------------------------------------- launchers --

static int exp_num_sms() {
  int dev = 0, nsm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  return nsm > 0 ? nsm : 1;
}

cudaError_t launch_exp_arcs(const ScanArgs& A, ExpUnit* units, int nunits, int* aseg, int* aoff,
                            int* adeg, int* tfirst, int* excl, cudaStream_t st) {
  if (nunits <= 0) return cudaSuccess;
  const int blocks = std::min(nunits, exp_num_sms() * 8);
  k_exp_arcs<<<blocks, kExpThreads, 0, st>>>(A, units, nunits, aseg, aoff, adeg, tfirst, excl);
  return cudaGetLastError();
}

cudaError_t launch_exp_tiles(const ScanArgs& A, const ExpUnit* units, const int* tile_unit,
                             int ntiles, const int* aseg, const int* aoff, const int* adeg,
                             const int* tfirst, void* rec, u64* tile_rec, int* pre,
                             cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  const int blocks = std::min(ntiles, exp_num_sms() * 8);
  if (A.measure == LP_AA || A.measure == LP_RA)
    k_exp_tiles<true><<<blocks, kExpThreads, 0, st>>>(A, units, tile_unit, ntiles, aseg, aoff,
                                                       adeg, tfirst, rec, tile_rec, pre);
  else
    k_exp_tiles<false><<<blocks, kExpThreads, 0, st>>>(A, units, tile_unit, ntiles, aseg, aoff,
                                                        adeg, tfirst, rec, tile_rec, pre);
  return cudaGetLastError();
}

cudaError_t launch_exp_count(const ScanArgs& A, const int4* q, u64 nq, cudaStream_t st) {
  if (nq == 0) return cudaSuccess;
  const int blocks = (int)std::max<u64>(1, std::min<u64>((u64)exp_num_sms() * 3, nq));
  const bool v64 = A.measure == LP_AA || A.measure == LP_RA;
  auto kern = v64 ? k_exp_count<true> : k_exp_count<false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kExpTableBytes);
  if (e != cudaSuccess) return e;
  kern<<<blocks, kCountThreads, kExpTableBytes, st>>>(A, q, nq, &A.ctr->claim_x);
  return cudaGetLastError();
}

}  // namespace lp

// ------------------------------------------------------------ host plan --

namespace lp {

namespace {

constexpr double kDenseMinRecords = 4096;  // expected records per window for dense counting
// expected records per hash bucket: half the table's slots

int floor_log2(double x) {
  int l = 0;
  while (l < 62 && std::ldexp(1.0, l + 1) <= x) ++l;
  return l;
}

#define XCU(x)                                             \
  do {                                                     \
    cudaError_t e_ = (x);                                  \
    if (e_ != cudaSuccess) return report_cuda(e_, #x);     \
  } while (0)

}  // namespace

lp_status exp_setup(Graph& g, ScanArgs& A, u64 nexp, long long batch_wedges, bool timing,
                    ExpState& S) {
  S = ExpState();
  if (nexp == 0) return LP_OK;
  cudaStream_t st = g.stream;
  std::vector<int4> q(nexp);
  std::vector<u64> w(nexp);
  XCU(cudaMemcpyAsync(q.data(), g.s_xq.p, sizeof(int4) * nexp, cudaMemcpyDeviceToHost, st));
  XCU(cudaMemcpyAsync(w.data(), g.s_xw.p, sizeof(u64) * nexp, cudaMemcpyDeviceToHost, st));
  XCU(cudaStreamSynchronize(st));
  const bool v64 = A.measure == LP_AA || A.measure == LP_RA;
  S.units.resize(nexp);
  long long arcs = 0, tfirsts = 0, excls = 0;
  u64 wmax = 0;
  for (u64 i = 0; i < nexp; ++i) {
    ExpUnit U;
    memset(&U, 0, sizeof(U));
    U.a = q[i].x;
    U.lo = q[i].y;
    U.hi = q[i].z;
    U.kept = q[i].w;
    U.W = (long long)w[i];
    const double span = (double)std::max(1, U.hi - U.lo);
    // counter width of a dense window: a count never exceeds the kept arcs
    // (windows fill the count pass's 64 KB table)
    int cw, wd;
    if (v64) {
      cw = kExpC64;
      wd = 13;
    } else if (U.kept <= 255) {
      cw = kExpC8;
      wd = 16;
    } else if (U.kept <= 65535) {
      cw = kExpC16;
      wd = 15;
    } else {
      cw = kExpC32;
      wd = 14;
    }
    const double nb_dense = std::ceil(span / std::ldexp(1.0, wd));
    const double per_window = (double)U.W * std::ldexp(1.0, wd) / span;
    if (per_window >= kDenseMinRecords && nb_dense <= kExpMaxBuckets) {
      U.flags = kExpDense | cw;
      U.wlog = wd;
    } else {
      U.flags = cw;
      const double per_bucket = std::ldexp(1.0, A.x_logcap - 1);  // half the table
      U.wlog = std::max(0, floor_log2(per_bucket * span / (double)std::max<long long>(1, U.W)));
      while (std::ceil(span / std::ldexp(1.0, U.wlog)) > kExpMaxBuckets) ++U.wlog;
    }
    U.nb = (int)std::ceil(span / std::ldexp(1.0, U.wlog));
    // tiles of at least 4K wedges, at most kExpMaxTiles per unit (the count
    // pass loads a bucket's runs of every tile at once)
    U.tile_w = (int)std::max<long long>(4096, (U.W + kExpMaxTiles - 1) / kExpMaxTiles);
    U.tile_w = (U.tile_w + kSub - 1) / kSub * kSub;
    U.T = (int)((U.W + U.tile_w - 1) / U.tile_w);
    U.arc_base = arcs;
    arcs += (long long)U.kept + 1;
    U.tfirst_base = tfirsts;
    tfirsts += (long long)U.T * kSub + 1;
    U.excl_base = excls;
    excls += (long long)U.nb + 1;
    wmax = std::max<u64>(wmax, (u64)U.W);
    S.units[i] = U;
  }
  // batches: consecutive units, at most batch_wedges wedges (a larger unit alone)
  const u64 cap = std::max<u64>((u64)batch_wedges, wmax);
  for (size_t i = 0; i < S.units.size();) {
    ExpBatch B{i, i, 0, 0, 0, 0};
    while (B.u1 < S.units.size() && (B.u1 == B.u0 || B.wedges + S.units[B.u1].W <= cap)) {
      ExpUnit& U = S.units[B.u1];
      U.rec_base = (long long)B.wedges;
      U.tile_base = (long long)B.tiles;
      U.pre_base = (long long)B.pre;
      U.bucket_base = (long long)B.buckets;
      B.wedges += (u64)U.W;
      B.tiles += (u64)U.T;
      B.pre += (u64)U.T * (U.nb + 1);
      B.buckets += (u64)U.nb;
      ++B.u1;
    }
    S.batches.push_back(B);
    i = B.u1;
  }
  XCU(ensure(g, g.s_xunit, sizeof(ExpUnit) * nexp));
  XCU(ensure(g, g.s_xaseg, sizeof(int) * (size_t)arcs));
  XCU(ensure(g, g.s_xaoff, sizeof(int) * (size_t)arcs));
  if (v64) XCU(ensure(g, g.s_xadeg, sizeof(int) * (size_t)arcs));
  XCU(ensure(g, g.s_xtfirst, sizeof(int) * (size_t)tfirsts));
  XCU(ensure(g, g.s_xexcl, sizeof(int) * (size_t)excls));
  XCU(cudaMemcpyAsync(g.s_xunit.p, S.units.data(), sizeof(ExpUnit) * nexp, cudaMemcpyHostToDevice,
                      st));
  if (timing) cudaEventRecord(g.xev[0], st);
  XCU(launch_exp_arcs(A, sp<ExpUnit>(g.s_xunit), (int)nexp, sp<int>(g.s_xaseg),
                      sp<int>(g.s_xaoff), v64 ? sp<int>(g.s_xadeg) : nullptr,
                      sp<int>(g.s_xtfirst), sp<int>(g.s_xexcl), st));
  if (timing) cudaEventRecord(g.xev[1], st);
  S.launches++;
  // the arc pass checks every unit's wedge count against the estimate
  u32 err = 0;
  XCU(cudaMemcpyAsync(&err, &A.ctr->error, sizeof(u32), cudaMemcpyDeviceToHost, st));
  XCU(cudaStreamSynchronize(st));
  if (err) return report_error(LP_EINTERNAL, "expand tier: arc pass check failed");
  if (timing) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, g.xev[0], g.xev[1]) == cudaSuccess) S.ms_expand += ms;
  }
  A.xunit = sp<ExpUnit>(g.s_xunit);
  A.xexcl = sp<int>(g.s_xexcl);
  return LP_OK;
}

lp_status exp_next_batch(Graph& g, ScanArgs& A, ExpState& S, bool timing,
                         std::vector<int4>& items) {
  items.clear();
  if (S.next >= S.batches.size()) return LP_OK;
  const ExpBatch B = S.batches[S.next++];
  cudaStream_t st = g.stream;
  const bool v64 = A.measure == LP_AA || A.measure == LP_RA;
  XCU(ensure(g, g.s_xrec, (v64 ? sizeof(int2) : sizeof(int)) * (size_t)B.wedges));
  XCU(ensure(g, g.s_xtile, sizeof(u64) * (size_t)B.tiles));
  XCU(ensure(g, g.s_xtunit, sizeof(int) * (size_t)B.tiles));
  XCU(ensure(g, g.s_xpre, sizeof(int) * (size_t)B.pre));
  XCU(ensure(g, g.s_xbunit, sizeof(int) * (size_t)B.buckets));
  std::vector<int> tile_unit(B.tiles), bucket_unit(B.buckets);
  items.reserve(B.buckets);
  for (size_t u = B.u0; u < B.u1; ++u) {
    const ExpUnit& U = S.units[u];
    for (int t = 0; t < U.T; ++t) tile_unit[U.tile_base + t] = (int)u;
    for (int b = 0; b < U.nb; ++b) {
      bucket_unit[U.bucket_base + b] = (int)u;
      const long long clo = (long long)U.lo + ((long long)b << U.wlog);
      const long long chi = std::min<long long>(U.hi, clo + (1ll << U.wlog));
      items.push_back(make_int4(U.a, (int)clo, (int)chi, (int)(U.bucket_base + b) | kExpItem));
    }
  }
  XCU(cudaMemcpyAsync(g.s_xtunit.p, tile_unit.data(), sizeof(int) * B.tiles,
                      cudaMemcpyHostToDevice, st));
  XCU(cudaMemcpyAsync(g.s_xbunit.p, bucket_unit.data(), sizeof(int) * B.buckets,
                      cudaMemcpyHostToDevice, st));
  if (timing) cudaEventRecord(g.xev[0], st);
  XCU(launch_exp_tiles(A, sp<ExpUnit>(g.s_xunit), sp<int>(g.s_xtunit), (int)B.tiles,
                       sp<int>(g.s_xaseg), sp<int>(g.s_xaoff), v64 ? sp<int>(g.s_xadeg) : nullptr,
                       sp<int>(g.s_xtfirst), g.s_xrec.p, sp<u64>(g.s_xtile), sp<int>(g.s_xpre),
                       st));
  if (timing) cudaEventRecord(g.xev[1], st);
  S.launches++;
  // the host vectors must outlive the asynchronous copies
  XCU(cudaStreamSynchronize(st));
  if (timing) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, g.xev[0], g.xev[1]) == cudaSuccess) S.ms_expand += ms;
  }
  A.xunit = sp<ExpUnit>(g.s_xunit);
  A.xbucket_unit = sp<int>(g.s_xbunit);
  A.xrec = g.s_xrec.p;
  A.xtile_rec = sp<u64>(g.s_xtile);
  A.xpre = sp<int>(g.s_xpre);
  A.xexcl = sp<int>(g.s_xexcl);
  return LP_OK;
}

#undef XCU

}  // namespace lp
