// lp_pair.cu -- common-neighbour counts of the predicted pairs (AA and RA).
//
// The AA and RA scans accumulate fixed-point weight sums, not counts, so the
// count |Gamma_u ∩ Gamma_v| over intermediaries b with |Gamma_b| <= L_H that
// every predicted link reports (Section 4.1.5) is recomputed for the links the
// selection kept.  Their top pairs join high-degree vertices, and a vertex
// takes part in many of them, so the links are grouped by their endpoint of
// larger degree, u.  A small group (short Gamma_u, few links) is one warp's:
// a hash set of Gamma_u in the warp's slice of shared memory, then each link
// (u, v) counts the entries of Gamma_v found in it.  For the others one CTA
// marks Gamma_u (hub test applied) in shared memory
// (a bitmap over the vertex ids, in windows of ids when they do not all fit,
// or a hash set when Gamma_u is short and the ids need several windows), and
// its warps count, for every link (u, v) of the group, the marked entries of
// the shorter Gamma_v.  Building the groups is a counting sort by u
// (histogram, scan, scatter) in a handful of small kernels.  Under a hub
// limit both sides read a kept copy of the lists (the entries b with
// |Gamma_b| <= L_H, in order), built per call: a hub's list keeps about a
// third of its entries on the power-law graphs, and the walks shrink with it.
#include "lp_internal.cuh"

namespace lp {

#define FULLMASK 0xffffffffu

constexpr int kScanThreads = 1024;
constexpr int kScanChunk = kScanThreads * 4;  // int2 entries per block

// A link is grouped under its endpoint with the longer (kept) list (u on a
// tie), so the list streamed per link is the shorter one.
__device__ __forceinline__ int pair_owner(const lp_link& L, const int* __restrict__ off) {
  const int du = off[L.u + 1] - off[L.u], dv = off[L.v + 1] - off[L.v];
  return du >= dv ? L.u : L.v;
}

__global__ void k_pair_hist(const lp_link* __restrict__ links, u64 n, const int* __restrict__ off,
                            int* __restrict__ cnt) {
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x)
    atomicAdd(&cnt[pair_owner(links[i], off)], 1);
}

// Exclusive scan of the pairs v[i] (i < n) of one chunk of kScanChunk entries
// starting at `base` (four per thread): out[i] gets the sums before i within
// the chunk; returns the chunk total (every thread).
__device__ __forceinline__ int2 scan_chunk(const int2 (&v)[4], int base, int n, int2* out) {
  __shared__ int2 wsum[kScanThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int2 t = make_int2(0, 0);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    t.x += v[j].x;
    t.y += v[j].y;
  }
  int2 inc = t;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int x = __shfl_up_sync(FULLMASK, inc.x, o), y = __shfl_up_sync(FULLMASK, inc.y, o);
    if (lane >= o) {
      inc.x += x;
      inc.y += y;
    }
  }
  if (lane == 31) wsum[wid] = inc;
  __syncthreads();
  const int2 w = wsum[lane];
  int2 wi = w;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int x = __shfl_up_sync(FULLMASK, wi.x, o), y = __shfl_up_sync(FULLMASK, wi.y, o);
    if (lane >= o) {
      wi.x += x;
      wi.y += y;
    }
  }
  const int2 total = make_int2(__shfl_sync(FULLMASK, wi.x, 31), __shfl_sync(FULLMASK, wi.y, 31));
  int2 run = make_int2(__shfl_sync(FULLMASK, wi.x - w.x, wid) + inc.x - t.x,
                       __shfl_sync(FULLMASK, wi.y - w.y, wid) + inc.y - t.y);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int i = base + threadIdx.x * 4 + j;
    if (i < n) out[i] = run;
    run.x += v[j].x;
    run.y += v[j].y;
  }
  return total;
}

// sc[i] = (links before vertex i, vertices before i with a link), chunk-local;
// sums[chunk] = the chunk's totals.
__global__ void __launch_bounds__(kScanThreads) k_scan_counts(const int* __restrict__ cnt, int n,
                                                              int2* __restrict__ sc,
                                                              int2* __restrict__ sums) {
  const int base = blockIdx.x * kScanChunk;
  int2 v[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int i = base + threadIdx.x * 4 + j;
    const int c = i < n ? cnt[i] : 0;
    v[j] = make_int2(c, c > 0 ? 1 : 0);
  }
  const int2 total = scan_chunk(v, base, n, sc);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// Exclusive scan of the nb chunk totals, in place (one block, kScanChunk at a
// time with a running carry).
__global__ void __launch_bounds__(kScanThreads) k_scan_sums(int2* __restrict__ sums, int nb) {
  int2 carry = make_int2(0, 0);
  for (int base = 0; base < nb; base += kScanChunk) {  // block-uniform trips
    int2 v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int i = base + threadIdx.x * 4 + j;
      v[j] = i < nb ? sums[i] : make_int2(0, 0);
    }
    __syncthreads();  // every value read before any is overwritten
    const int2 tot = scan_chunk(v, base, nb, sums);
#pragma unroll
    for (int j = 0; j < 4; ++j) {  // the entries this thread wrote
      const int i = base + threadIdx.x * 4 + j;
      if (i < nb) {
        sums[i].x += carry.x;
        sums[i].y += carry.y;
      }
    }
    carry.x += tot.x;
    carry.y += tot.y;
    __syncthreads();  // scan_chunk's staging is reused by the next chunk
  }
}

__global__ void k_scan_add(int2* __restrict__ sc, int n, const int2* __restrict__ sums) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const int2 s = sums[i / kScanChunk];
    sc[i].x += s.x;
    sc[i].y += s.y;
  }
}

// Kept lists under a hub limit: kcnt[v] = |{b in Gamma_v : |Gamma_b| <= cap}|,
// and after the scan of kcnt into koff the entries themselves, in their order
// in Gamma_v.  A thread takes a vertex of degree at most kKeptThread (most
// of them, so many short lists are read at once), a warp one of larger
// degree; each kernel runs both passes and skips the other's vertices.
constexpr int kKeptThread = 64;

__global__ void k_kept_count(const int* __restrict__ off, const int* __restrict__ idx,
                             const int* __restrict__ deg, int n, int cap, int* __restrict__ kcnt) {
  const int lane = threadIdx.x & 31;
  const int nthreads = gridDim.x * blockDim.x;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += nthreads) {
    const int e0 = off[v], e1 = off[v + 1];
    if (e1 - e0 > kKeptThread) continue;
    int c = 0, e = e0;
    for (; e + 4 <= e1; e += 4) {  // four list entries, then their degrees, in flight
      const int b0 = __ldg(idx + e), b1 = __ldg(idx + e + 1), b2 = __ldg(idx + e + 2),
                b3 = __ldg(idx + e + 3);
      c += (__ldg(deg + b0) <= cap) + (__ldg(deg + b1) <= cap) + (__ldg(deg + b2) <= cap) +
           (__ldg(deg + b3) <= cap);
    }
    for (; e < e1; ++e) c += __ldg(deg + __ldg(idx + e)) <= cap ? 1 : 0;
    kcnt[v] = c;
  }
  const int nwarps = nthreads >> 5;
  for (int v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += nwarps) {
    const int e0 = off[v], e1 = off[v + 1];
    if (e1 - e0 <= kKeptThread) continue;  // warp-uniform
    int c = 0;
    for (int e = e0 + lane; e < e1; e += 32) c += __ldg(deg + __ldg(idx + e)) <= cap ? 1 : 0;
    c = (int)__reduce_add_sync(FULLMASK, (u32)c);
    if (lane == 0) kcnt[v] = c;
  }
}

__global__ void k_kept_scatter(const int* __restrict__ off, const int* __restrict__ idx,
                               const int* __restrict__ deg, int n, int cap,
                               const int2* __restrict__ koff, int* __restrict__ kidx) {
  const int lane = threadIdx.x & 31;
  const int nthreads = gridDim.x * blockDim.x;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += nthreads) {
    const int e0 = off[v], e1 = off[v + 1];
    if (e1 - e0 > kKeptThread) continue;
    int o = koff[v].x, e = e0;
    for (; e + 4 <= e1; e += 4) {
      const int b[4] = {__ldg(idx + e), __ldg(idx + e + 1), __ldg(idx + e + 2), __ldg(idx + e + 3)};
      const bool k[4] = {__ldg(deg + b[0]) <= cap, __ldg(deg + b[1]) <= cap,
                         __ldg(deg + b[2]) <= cap, __ldg(deg + b[3]) <= cap};
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (k[j]) kidx[o++] = b[j];
    }
    for (; e < e1; ++e) {
      const int b = __ldg(idx + e);
      if (__ldg(deg + b) <= cap) kidx[o++] = b;
    }
  }
  const int nwarps = nthreads >> 5;
  for (int v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += nwarps) {
    const int e0 = off[v], e1 = off[v + 1];
    if (e1 - e0 <= kKeptThread) continue;  // warp-uniform
    int o = koff[v].x;
    for (int eb = e0; eb < e1; eb += 32) {  // warp-uniform trips
      const int e = eb + lane;
      const int b = e < e1 ? __ldg(idx + e) : 0;
      const bool keep = e < e1 && __ldg(deg + b) <= cap;
      const u32 m = __ballot_sync(FULLMASK, keep);
      if (keep) kidx[o + __popc(m & ((1u << lane) - 1u))] = b;
      o += __popc(m);
    }
  }
}

// koff[i] = koff2[i].x for i <= n (the scan leaves (prefix, flags) pairs).
__global__ void k_kept_offsets(const int2* __restrict__ koff2, int n1, int* __restrict__ koff) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n1) koff[i] = koff2[i].x;
}

// A group whose owner list has at most kSmallDeg entries and which has at
// most kSmallLinks links is counted by one warp with a hash set of its own
// (kSmallLog slots: at most a quarter taken); the others by a whole CTA.
constexpr int kSmallDeg = 256;
constexpr int kSmallLinks = 64;
constexpr int kSmallLog = 10;
constexpr int kSmallWarps = 8;  // per 256-thread CTA: 32 KB of tables

// A CTA group of more links is cut into parts of kGroupLinks links, each a
// CTA's (it marks the owner's list again), so that a hub with a hundred
// thousand links is not one CTA's long tail.
constexpr int kGroupLinks = 4096;

// Entries of groups (gcap of them): n + links / kGroupLinks + 1 bound the
// warp groups and CTA group parts together.
static inline size_t pair_group_cap(int n, u64 nlinks) {
  return (size_t)n + nlinks / kGroupLinks + 1;
}

// groups[g] = (u, first position in perm, links), warp groups from the front
// (count nsg[0]), CTA group parts from the back (count nsg[1]); cnt: the
// histogram (kept apart from the scanned array sc).
__global__ void k_pair_groups(const int* __restrict__ cnt, const int2* __restrict__ sc,
                              const int* __restrict__ off, int n, int4* __restrict__ groups,
                              long long gcap, u32* __restrict__ nsg) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u < n && cnt[u] > 0) {
    const int c = cnt[u], first = sc[u].x;
    if (off[u + 1] - off[u] <= kSmallDeg && c <= kSmallLinks) {
      groups[atomicAdd(&nsg[0], 1u)] = make_int4(u, first, c, 0);
    } else {
      const int parts = (c + kGroupLinks - 1) / kGroupLinks;
      const long long at = (long long)atomicAdd(&nsg[1], (u32)parts);
      for (int j = 0; j < parts; ++j)
        groups[gcap - 1 - (at + j)] =
            make_int4(u, first + j * kGroupLinks, min(kGroupLinks, c - j * kGroupLinks), 0);
    }
  }
}

__device__ __forceinline__ u32 small_hash(int b) {
  return ((u32)b * 0x9E3779B1u) >> (32 - kSmallLog);
}

// 1 if b is in the warp's set (keys b + 1, 0 = empty; an empty slot always
// comes, as at most a quarter are taken).
__device__ __forceinline__ u32 small_has(const u32* t, int b) {
  const u32 key = (u32)b + 1u;
  u32 h = small_hash(b);
  for (;;) {
    const u32 k2 = t[h];
    if (k2 == key) return 1u;
    if (k2 == 0u) return 0u;
    h = (h + 1) & ((1u << kSmallLog) - 1);
  }
}

// The warp groups: a warp claims a group, puts the owner's list in its set,
// counts every link's other list against it (four loads in flight per lane)
// and clears the slots it took.
__global__ void __launch_bounds__(kSmallWarps * 32) k_pair_cn_small(lp_link* __restrict__ links,
                                                                   const int* __restrict__ perm,
                                                                   const int4* __restrict__ groups,
                                                                   const u32* __restrict__ nsg,
                                                                   const int* __restrict__ off,
                                                                   const int* __restrict__ idx,
                                                                   u32* __restrict__ claim) {
  __shared__ u32 tab[kSmallWarps][1 << kSmallLog];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  u32* t = tab[wid];
  for (int i = lane; i < (1 << kSmallLog); i += 32) t[i] = 0;
  __syncwarp();
  const u32 ng = nsg[0];
  for (;;) {
    u32 gi = 0;
    if (lane == 0) gi = atomicAdd(claim, 1u);
    gi = __shfl_sync(FULLMASK, gi, 0);
    if (gi >= ng) break;
    const int4 G = groups[gi];
    const int u = G.x, e0 = off[u], e1 = off[u + 1];
    int slot[kSmallDeg / 32];
#pragma unroll
    for (int q = 0; q < kSmallDeg / 32; ++q) {
      slot[q] = -1;
      const int e = e0 + q * 32 + lane;
      if (e < e1) {
        const int b = __ldg(idx + e);
        u32 h = small_hash(b);
        while (atomicCAS(&t[h], 0u, (u32)b + 1u) != 0u)  // keys are distinct
          h = (h + 1) & ((1u << kSmallLog) - 1);
        slot[q] = (int)h;
      }
    }
    __syncwarp();
    for (int j = 0; j < G.z; ++j) {
      const int li = perm[G.y + j];
      const int lu = links[li].u, lv = links[li].v;
      const int v = lu == u ? lv : lu;
      const int vs = off[v], ve = off[v + 1];
      u32 c = 0;
      int e = vs + lane;
      for (; e + 96 < ve; e += 128) {
        const int b0 = __ldg(idx + e), b1 = __ldg(idx + e + 32), b2 = __ldg(idx + e + 64),
                  b3 = __ldg(idx + e + 96);
        c += small_has(t, b0) + small_has(t, b1) + small_has(t, b2) + small_has(t, b3);
      }
      for (; e < ve; e += 32) c += small_has(t, __ldg(idx + e));
      c = __reduce_add_sync(FULLMASK, c);
      if (lane == 0) links[li].cn = (int)c;
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < kSmallDeg / 32; ++q)
      if (slot[q] >= 0) t[slot[q]] = 0u;
    __syncwarp();
  }
}

// perm: link indices grouped by u (the group starts in sc[u].x serve as
// cursors; the groups were recorded before).
__global__ void k_pair_scatter(const lp_link* __restrict__ links, u64 n,
                               const int* __restrict__ off, int2* __restrict__ sc,
                               int* __restrict__ perm) {
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x)
    perm[atomicAdd(&sc[pair_owner(links[i], off)].x, 1)] = (int)i;
}

constexpr int kPairHashLog = 14;                    // hash-set slots (64 KB of keys)
constexpr int kPairHashMaxDeg = 1 << (kPairHashLog - 1);

__device__ __forceinline__ u32 pair_hash(int b) {
  return ((u32)b * 0x9E3779B1u) >> (32 - kPairHashLog);
}

// One group at a time per CTA (claimed from *claim): the marked set is the
// kept list of u (off / idx: the kept lists, or the whole lists without a hub
// limit); every link (u, v) of the group counts the marked entries of v's
// list (a warp per link).  The set is a bitmap over the ids
// [w0, w0 + 32 * nwords): over all vertices when they fit, else one window of
// ids at a time; a group whose Gamma_u is short uses a hash set of its
// entries (keys b + 1, 0 = empty) in the same shared memory instead.
// Its groups are the CTA groups, counted from the back of groups (nsg[1]).
__global__ void __launch_bounds__(1024, 1) k_pair_cn_groups(lp_link* __restrict__ links,
                                                            const int* __restrict__ perm,
                                                            const int4* __restrict__ groups,
                                                            const u32* __restrict__ nsg,
                                                            const int* __restrict__ off,
                                                            const int* __restrict__ idx,
                                                            const int* __restrict__ foff,
                                                            const int* __restrict__ fidx,
                                                            const int* __restrict__ deg,
                                                            int nwords, int n, long long gcap,
                                                            u32* __restrict__ claim,
                                                            int* __restrict__ cur) {
  extern __shared__ u32 bits[];
  __shared__ u32 s_g;
  __shared__ unsigned long long s_cost[2];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const u32 ngroups = nsg[1];
  const int width = nwords * 32;
  const bool one_window = n <= width;
  // the table of the wedge form: slots keys then slots counts, half the slots
  // taken at most (a chunk of the group's links at a time)
  const int slog = 31 - __clz(nwords / 2);
  const int slots = 1 << slog, chunk = slots / 2;
  u32* tkey = bits;
  u32* tcnt = bits + slots;
  for (int i = threadIdx.x; i < nwords; i += blockDim.x) bits[i] = 0;
  for (;;) {
    if (threadIdx.x == 0) {
      s_g = atomicAdd(claim, 1u);
      s_cost[0] = s_cost[1] = 0ull;
    }
    __syncthreads();
    const u32 gi = s_g;
    if (gi >= ngroups) break;
    const int4 G = groups[gcap - 1 - (long long)gi];
    const int u = G.x, e0 = off[u], e1 = off[u + 1];
    // Two ways to count: walk every link's list (the sum of their lengths),
    // or expand the wedges of u once per chunk of links (the kept b of u,
    // each with its whole list Gamma_b) and look every second-order vertex up
    // in a table of the chunk's other endpoints.  The cheaper one is taken.
    {
      unsigned long long wk = 0, wg = 0;
      for (int j = threadIdx.x; j < G.z; j += blockDim.x) {
        const int li = perm[G.y + j];
        const int lu = links[li].u, lv = links[li].v;
        const int v = lu == u ? lv : lu;
        wk += (unsigned long long)(off[v + 1] - off[v]);
      }
      for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x)
        wg += (unsigned long long)__ldg(deg + __ldg(idx + e));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        wk += __shfl_xor_sync(FULLMASK, wk, o);
        wg += __shfl_xor_sync(FULLMASK, wg, o);
      }
      if (lane == 0) {
        atomicAdd(&s_cost[0], wk);
        atomicAdd(&s_cost[1], wg);
      }
    }
    __syncthreads();
    const unsigned long long nchunks = ((unsigned long long)G.z + chunk - 1) / chunk;
    if (s_cost[1] * nchunks < s_cost[0]) {  // CTA-uniform
      for (int c0 = 0; c0 < G.z; c0 += chunk) {
        const int c1 = min(G.z, c0 + chunk);
        for (int j = c0 + threadIdx.x; j < c1; j += blockDim.x) {
          const int li = perm[G.y + j];
          const int lu = links[li].u, lv = links[li].v;
          const int v = lu == u ? lv : lu;
          u32 h = ((u32)v * 0x9E3779B1u) >> (32 - slog);
          while (atomicCAS(&tkey[h], 0u, (u32)v + 1u) != 0u)  // the endpoints are distinct
            h = (h + 1) & (slots - 1);
        }
        __syncthreads();
        for (int e = e0 + wid; e < e1; e += nw) {  // a warp per kept b of u
          const int b = __ldg(idx + e);
          const int fe = __ldg(foff + b + 1);
          for (int f = __ldg(foff + b) + lane; f < fe; f += 32) {
            const int c = __ldg(fidx + f);
            const u32 key = (u32)c + 1u;
            u32 h = ((u32)c * 0x9E3779B1u) >> (32 - slog);
            for (;;) {  // at most half the slots are taken, so an empty one comes
              const u32 k2 = tkey[h];
              if (k2 == key) {
                atomicAdd(&tcnt[h], 1u);
                break;
              }
              if (k2 == 0u) break;
              h = (h + 1) & (slots - 1);
            }
          }
        }
        __syncthreads();
        for (int j = c0 + threadIdx.x; j < c1; j += blockDim.x) {
          const int li = perm[G.y + j];
          const int lu = links[li].u, lv = links[li].v;
          const int v = lu == u ? lv : lu;
          u32 h = ((u32)v * 0x9E3779B1u) >> (32 - slog);
          while (tkey[h] != (u32)v + 1u) h = (h + 1) & (slots - 1);  // it is there
          links[li].cn = (int)tcnt[h];
        }
        __syncthreads();
        for (int i = threadIdx.x; i < 2 * slots; i += blockDim.x) bits[i] = 0;
        __syncthreads();
      }
      continue;
    }
    if (!one_window && e1 - e0 <= kPairHashMaxDeg) {
      for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const int b = __ldg(idx + e);
        u32 h = pair_hash(b);
        while (atomicCAS(&bits[h], 0u, (u32)b + 1u) != 0u)  // keys are distinct
          h = (h + 1) & ((1u << kPairHashLog) - 1);
      }
      __syncthreads();
      for (int j = wid; j < G.z; j += nw) {  // warp-uniform trips
        const int li = perm[G.y + j];
        const lp_link L = links[li];
        const int v = L.u == u ? L.v : L.u;
        // at most half the slots are taken, so an empty one comes
        auto has = [&](int b) -> u32 {
          const u32 key = (u32)b + 1u;
          u32 h = pair_hash(b);
          for (;;) {
            const u32 k2 = bits[h];
            if (k2 == key) return 1u;
            if (k2 == 0u) return 0u;
            h = (h + 1) & ((1u << kPairHashLog) - 1);
          }
        };
        u32 c = 0;
        const int ve = off[v + 1];
        int e = off[v] + lane;
        for (; e + 96 < ve; e += 128) {  // four loads in flight per lane
          const int b0 = __ldg(idx + e), b1 = __ldg(idx + e + 32), b2 = __ldg(idx + e + 64),
                    b3 = __ldg(idx + e + 96);
          c += has(b0) + has(b1) + has(b2) + has(b3);
        }
        for (; e < ve; e += 32) c += has(__ldg(idx + e));
        c = __reduce_add_sync(FULLMASK, c);
        if (lane == 0) links[li].cn = c;
      }
      __syncthreads();
      for (int i = threadIdx.x; i < (1 << kPairHashLog); i += blockDim.x) bits[i] = 0;
      __syncthreads();
      continue;
    }
    for (int w0 = 0; w0 < n; w0 += width) {  // one pass when the bitmap covers every id
      const int w1 = min(n, w0 + width);
      for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const int b = __ldg(idx + e);
        if (b < w0 || b >= w1) continue;
        atomicOr(&bits[(b - w0) >> 5], 1u << ((b - w0) & 31));
      }
      __syncthreads();
      for (int j = wid; j < G.z; j += nw) {  // warp-uniform trips
        const int li = perm[G.y + j];
        const lp_link L = links[li];
        const int v = L.u == u ? L.v : L.u;
        int c = 0;
        const int vs = off[v], ve = off[v + 1];
        // Gamma_v is sorted and the windows ascend: this window's entries
        // start where the previous window's ended (a cursor per link), and
        // end at the first entry >= w1, found by the walk itself
        if (one_window) {  // every id in the bitmap: the whole list, no bound
          int e = vs + lane;
          for (; e + 96 < ve; e += 128) {  // four loads in flight per lane
            const int b0 = __ldg(idx + e), b1 = __ldg(idx + e + 32), b2 = __ldg(idx + e + 64),
                      b3 = __ldg(idx + e + 96);
            c += ((bits[b0 >> 5] >> (b0 & 31)) & 1u) + ((bits[b1 >> 5] >> (b1 & 31)) & 1u) +
                 ((bits[b2 >> 5] >> (b2 & 31)) & 1u) + ((bits[b3 >> 5] >> (b3 & 31)) & 1u);
          }
          for (; e < ve; e += 32) {
            const int b = __ldg(idx + e);
            c += (bits[b >> 5] >> (b & 31)) & 1u;
          }
          c = __reduce_add_sync(FULLMASK, (u32)c);
          if (lane == 0) links[li].cn = c;
          continue;
        }
        int e0 = w0 == 0 ? vs : cur[G.y + j];
        int next = ve;
        for (;;) {  // warp-uniform trips; four loads in flight per lane
          int bb[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int e = e0 + 32 * k + lane;
            bb[k] = e < ve ? __ldg(idx + e) : INT_MAX;
          }
          bool stop = false;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const bool in = bb[k] < w1;
            const int b = bb[k] - w0;
            c += in ? ((bits[b >> 5] >> (b & 31)) & 1u) : 0u;
            const u32 m = __ballot_sync(FULLMASK, !in);
            if (m) {  // warp-uniform
              next = e0 + 32 * k + __ffs(m) - 1;
              stop = true;
              break;
            }
          }
          if (stop) break;
          e0 += 128;
        }
        c = __reduce_add_sync(FULLMASK, (u32)c);
        if (lane == 0) {
          cur[G.y + j] = min(next, ve);
          if (w0 == 0) links[li].cn = c;
          else links[li].cn += c;
        }
      }
      __syncthreads();
      for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const int b = __ldg(idx + e);
        if (b >= w0 && b < w1) bits[(b - w0) >> 5] = 0;
      }
      __syncthreads();
    }
  }
}

// Scratch layout: sc int2[n + 1], cnt int[n + 1], perm int[links], groups
// int4[n + links / kGroupLinks + 1], sums int2[chunks], claim u32, window
// cursors int[links]; under a hub limit also the kept lists: koff int[n + 1]
// and kidx int[arcs]; every part 256-byte aligned (groups are int4).
static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t pair_groups_scratch(int n, u64 nlinks, long long kept_arcs) {
  const size_t n1 = (size_t)n + 1;
  size_t b = align256(n1 * sizeof(int2)) + align256(n1 * sizeof(int)) +
             align256(nlinks * sizeof(int)) + align256(pair_group_cap(n, nlinks) * sizeof(int4)) +
             align256(((n1 + kScanChunk - 1) / kScanChunk) * sizeof(int2)) + 256 +
             align256(nlinks * sizeof(int));
  if (kept_arcs > 0) b += align256(n1 * sizeof(int)) + align256((size_t)kept_arcs * sizeof(int));
  return b;
}

// Counts of links[0, n), grouped by the endpoint of larger degree; scratch of pair_groups_scratch bytes.
cudaError_t launch_pair_cn_groups(lp_link* links, u64 n, int nv, const int* off, const int* idx,
                                  const int* deg, long long arcs, int dmax, int cap, void* scratch,
                                  cudaStream_t st, int* launches) {
  if (n == 0) return cudaSuccess;
  const int n1 = nv + 1;
  const bool kept = cap < dmax;  // else every list is kept whole
  const int* foff = off;  // the whole lists (second-order vertices of the wedge form)
  const int* fidx = idx;
  char* p = static_cast<char*>(scratch);
  int2* sc = reinterpret_cast<int2*>(p);
  p += align256((size_t)n1 * sizeof(int2));
  int* cnt = reinterpret_cast<int*>(p);
  p += align256((size_t)n1 * sizeof(int));
  int* perm = reinterpret_cast<int*>(p);
  p += align256(n * sizeof(int));
  int4* groups = reinterpret_cast<int4*>(p);
  const long long gcap = (long long)pair_group_cap(nv, n);
  p += align256((size_t)gcap * sizeof(int4));
  const int nb = (n1 + kScanChunk - 1) / kScanChunk;
  int2* sums = reinterpret_cast<int2*>(p);
  p += align256((size_t)nb * sizeof(int2));
  u32* claim = reinterpret_cast<u32*>(p);
  p += 256;
  int* cur = reinterpret_cast<int*>(p);
  p += align256(n * sizeof(int));
  int dev = 0, nsm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaSuccess;
  if (kept) {
    // the kept lists: counts (in cnt), their scan (in sc, as the groups'
    // scan below does), offsets, entries; sc and cnt are reset afterwards
    int* koff = reinterpret_cast<int*>(p);
    p += align256((size_t)n1 * sizeof(int));
    int* kidx = reinterpret_cast<int*>(p);
    const int wb = nsm * 8;  // 256-thread blocks
    k_kept_count<<<wb, 256, 0, st>>>(off, idx, deg, nv, cap, cnt);
    e = cudaMemsetAsync(cnt + nv, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    k_scan_counts<<<nb, kScanThreads, 0, st>>>(cnt, n1, sc, sums);
    k_scan_sums<<<1, kScanThreads, 0, st>>>(sums, nb);
    k_scan_add<<<(n1 + 255) / 256, 256, 0, st>>>(sc, n1, sums);
    k_kept_offsets<<<(n1 + 255) / 256, 256, 0, st>>>(sc, n1, koff);
    k_kept_scatter<<<wb, 256, 0, st>>>(off, idx, deg, nv, cap, sc, kidx);
    if (launches) *launches += 6;
    off = koff;
    idx = kidx;
  }
  (void)arcs;
  e = cudaMemsetAsync(cnt, 0, (size_t)n1 * sizeof(int), st);
  // claim: [0] CTA groups claimed, [1] warp groups claimed, [2] / [3] warp /
  // CTA groups written
  if (e == cudaSuccess) e = cudaMemsetAsync(claim, 0, 4 * sizeof(u32), st);
  if (e != cudaSuccess) return e;
  const int gb = (int)std::min<u64>((n + 255) / 256, 152 * 8);
  k_pair_hist<<<gb, 256, 0, st>>>(links, n, off, cnt);
  k_scan_counts<<<nb, kScanThreads, 0, st>>>(cnt, n1, sc, sums);
  k_scan_sums<<<1, kScanThreads, 0, st>>>(sums, nb);
  k_scan_add<<<(n1 + 255) / 256, 256, 0, st>>>(sc, n1, sums);
  k_pair_groups<<<(nv + 255) / 256, 256, 0, st>>>(cnt, sc, off, nv, groups, gcap, claim + 2);
  k_pair_scatter<<<gb, 256, 0, st>>>(links, n, off, sc, perm);
  // a bitmap over every vertex when it fits in 224 KB, else windows of that
  // size (and room for the hash set)
  const int nwords = std::max(1 << kPairHashLog, std::min((nv + 31) / 32, 224 * 1024 / 4));
  const size_t smem = (size_t)nwords * 4;
  e = cudaFuncSetAttribute(k_pair_cn_groups, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           224 * 1024);
  if (e != cudaSuccess) return e;
  k_pair_cn_small<<<nsm * 7, kSmallWarps * 32, 0, st>>>(links, perm, groups, claim + 2, off, idx,
                                                        claim + 1);
  k_pair_cn_groups<<<nsm, 1024, smem, st>>>(links, perm, groups, claim + 2, off, idx, foff, fidx,
                                            deg, nwords, nv, gcap, claim, cur);
  if (launches) *launches += 8;
  return cudaGetLastError();
}

}  // namespace lp
