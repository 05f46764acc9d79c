// lp_serve_dev.cu -- the resident kernel of the serving loop (lp_serve_*).
//
// One kernel stays on the GPU while requests arrive.  The host writes each
// admitted request's parameters, sources and a work item per source into
// host memory that the GPU reads directly (mapped, pinned), then advances a
// published-item counter.  Every CTA of the kernel claims work items one at a
// time, computes that source's k best partners (the per-vertex form of the
// ranked top-k list of Section 3, with the scan of Algorithm 1: the hub test
// of Section 4.2.1, the first-order exclusion of Section 4.1.4, Eq. 1-9 and
// the library's total order) and writes the row straight into the request's
// host result buffer.  The CTA that finishes a request's last source raises
// the request's completion word.  No host round trip lies between requests,
// and requests that arrive while others run are claimed by whichever CTA is
// free, so their work overlaps on the device.
//
// Waits are bounded: a CTA that finds no work for idle_polls polls (a short
// sleep each) leaves, and the host launches the kernel again when work is
// published while it is not running.
//
// A source is counted in a shared-memory hash table.  Sources whose wedges
// could hold more distinct partners than half the table are counted over
// consecutive vertex-id ranges (a binary search of each intermediary list per
// range), and a range whose table fills is split in two; the per-warp k-best
// lists run across the ranges.  Results equal lp_predict_sources byte for byte
// (the same keys, order, fixed-point sums and common-neighbour counts).
#include "lp_internal.cuh"
#include "lp_scan_dev.cuh"

namespace lp {

constexpr int kSrvThreads = 512;
constexpr int kSrvWarps = kSrvThreads / 32;
constexpr int kSrvLogcap = 13;  // 8192 slots: 96 KB with 64-bit values
constexpr int kSrvSlots = 1 << kSrvLogcap;
constexpr int kSrvStack = 48;   // pending split ranges of one source

__device__ __forceinline__ unsigned long long ld_acquire_sys(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_sys(unsigned* p, unsigned v) {
  asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// One source: its k best partners into row[0, k) (fillers after the count).
// Returns false, writing nothing, for a source with more than defer_wedges
// wedges (the host counts it with the tiered pipeline).
template <typename V>
__device__ bool serve_source(const SrvArgs& S, const SrvReq& R, int a, lp_link* row,
                             unsigned char* smem, TopEnt* tops) {
  int* keys = reinterpret_cast<int*>(smem);
  V* vals = reinterpret_cast<V*>(smem + (size_t)kSrvSlots * 4);
  __shared__ unsigned long long s_w;
  __shared__ int s_overflow, s_nstack, s_err, s_tcnt[kSrvWarps];
  __shared__ int2 s_stack[kSrvStack];
  const int lane = lane_id(), wid = threadIdx.x >> 5;
  const int cap = R.cap < 0 ? INT32_MAX : R.cap;
  // the per-source scan's arguments (the scoring helpers read these fields)
  ScanArgs A;
  A.off = S.off;
  A.idx = S.idx;
  A.deg = S.deg;
  A.arc = S.arc;
  A.wt = R.measure == LP_AA ? S.wt : (R.measure == LP_RA ? S.wt + (size_t)S.dmax + 1 : nullptr);
  A.n = S.n;
  A.cap = cap;
  A.measure = R.measure;
  A.mode = 1;
  A.fixbits = S.fixbits;
  A.thr_check = 0;
  A.threshold = 0.0;
  A.k = R.k;
  Thresh T;
  T.valid = 0;
  const int e0 = S.off[a], e1 = S.off[a + 1];
  const u64 da = (u64)(e1 - e0);
  // wedges through the kept intermediaries (c != a): a bound on the partners
  u64 w = 0;
  for (int e = e0 + threadIdx.x; e < e1; e += kSrvThreads) {
    const Arc t = S.arc[e];
    if (t.z <= cap) w += (u64)(t.z - 1);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(FULLMASK, w, o);
  if (threadIdx.x == 0) {
    s_w = 0;
    s_err = 0;
  }
  __syncthreads();
  if (lane == 0 && w) atomicAdd(&s_w, w);
  __syncthreads();
  const u64 W = s_w;
  if (W > S.defer_wedges) return false;  // CTA-uniform
  TopEnt* top = tops + wid * R.k;
  int tcnt = 0;
  u64 n_cand = 0;
  if (W > 0) {
    // consecutive id ranges, each expected to fill at most half the table
    const u64 half = kSrvSlots / 2;
    const int nr = (int)min((u64)S.n, (W + half - 1) / half);
    for (int r = 0; r < nr; ++r) {
      if (threadIdx.x == 0) {
        s_stack[0] = make_int2((int)(((long long)S.n * r) / nr), (int)(((long long)S.n * (r + 1)) / nr));
        s_nstack = 1;
      }
      __syncthreads();
      while (s_nstack > 0) {  // CTA-uniform
        const int2 rg = s_stack[s_nstack - 1];
        const int lo = rg.x, hi = rg.y;
        const bool whole = lo == 0 && hi == S.n;
        __syncthreads();
        if (threadIdx.x == 0) {
          s_nstack -= 1;
          s_overflow = 0;
        }
        __syncthreads();
        // insert the wedges with lo <= c < hi, c != a
        for (int eb = e0 + wid * 32; eb < e1; eb += kSrvThreads) {  // warp-uniform trips
          const int e = eb + lane;
          int s = 0, len = 0;
          V wb = 0;
          if (e < e1) {
            const Arc t = S.arc[e];
            if (t.z <= cap) {
              int s0 = t.y - t.z, s1 = t.y;
              if (!whole) {
                s0 = lower_bound_interp(S.idx, s0, s1, lo);
                s1 = lower_bound_interp(S.idx, s0, s1, hi);
              }
              s = s0;
              len = s1 - s0;
              if (len > 0) wb = arc_weight<V>(A, t.z);
            }
          }
          scan_arcs<V>(s, len, wb, S.idx, [&](int c, V wc) {
            if (c == a || *(volatile int*)&s_overflow) return;
            if (hash_add<V>(keys, vals, kSrvLogcap, c, wc, fill_probes(kSrvLogcap)) == 2) s_overflow = 1;
          });
          if (__any_sync(FULLMASK, *(volatile int*)&s_overflow != 0)) break;
        }
        __syncthreads();
        if (s_overflow) {  // CTA-uniform: clear, and count the range in halves
          for (int i = threadIdx.x * 4; i < kSrvSlots; i += kSrvThreads * 4) {
            *reinterpret_cast<int4*>(keys + i) = make_int4(0, 0, 0, 0);
            zero4<V>(vals + i);
          }
          if (threadIdx.x == 0) {
            if (hi - lo < 2 || s_nstack + 2 > kSrvStack) {
              // cannot happen: one id never overflows, and each split halves
              *(volatile unsigned*)S.status = 1u;
              s_err = 1;
              s_nstack = 0;
            } else {
              const int mid = lo + (hi - lo) / 2;
              s_stack[s_nstack] = make_int2(mid, hi);
              s_stack[s_nstack + 1] = make_int2(lo, mid);
              s_nstack += 2;
            }
          }
          __syncthreads();
          if (s_err) break;
          continue;
        }
        // drop the first-order neighbours in [lo, hi)
        for (int e = e0 + threadIdx.x; e < e1; e += kSrvThreads) {
          const int b = __ldg(S.idx + e);
          if (b >= lo && b < hi) hash_kill<V>(keys, vals, kSrvLogcap, b);
        }
        __syncthreads();
        for (int base0 = wid * 128; base0 < kSrvSlots; base0 += kSrvThreads * 4)  // warp-uniform
          score_hash_chunk<V, 1>(A, T, a, da, keys, vals, base0, kSrvSlots, top, tcnt, n_cand);
        __syncthreads();
      }
    }
  }
  // merge the warps' lists into warp 0's
  if (lane == 0) s_tcnt[wid] = tcnt;
  __syncthreads();
  if (wid == 0) {
    int cnt = s_tcnt[0];
    for (int w2 = 1; w2 < kSrvWarps; ++w2) {
      const TopEnt* other = tops + w2 * R.k;
      const int oc = s_tcnt[w2];
      for (int j = 0; j < oc; ++j) {
        const TopEnt x = other[j];
        if (cnt >= R.k && !ent_before(x, top[R.k - 1])) break;  // sorted: the rest is worse
        top_insert(top, cnt, R.k, x);
      }
    }
    if (lane == 0) s_tcnt[0] = cnt;
  }
  __syncthreads();
  const int cnt = s_tcnt[0];
  // the row: links in order, then fillers; AA / RA count their common
  // neighbours (one warp per link)
  const bool v64 = R.measure == LP_AA || R.measure == LP_RA;
  for (int j = wid; j < R.k; j += kSrvWarps) {  // warp-uniform trips
    lp_link L;
    if (j < cnt) {
      const TopEnt x = tops[j];
      u64 cn = (u64)x.cn;
      if (v64) cn = pair_common(a, x.c, S.off, S.idx, S.deg, S.arc, cap, nullptr);
      L.u = a;
      L.v = x.c;
      L.score = (float)key_value(R.measure, x.num, x.den, cn, S.fixbits);
      L.cn = (int)cn;
    } else {
      L.u = -1;
      L.v = -1;
      L.score = 0.f;
      L.cn = 0;
    }
    if (lane == 0) row[j] = L;
  }
  __syncthreads();
  return true;
}

// The resident kernel: claim work items {request slot, source index} until
// none comes for idle_polls polls.
__global__ void __launch_bounds__(kSrvThreads, 2) k_serve(SrvArgs S) {
  extern __shared__ __align__(16) unsigned char smem[];
  TopEnt* tops = reinterpret_cast<TopEnt*>(smem + (size_t)kSrvSlots * (4 + 8));
  __shared__ int2 s_item;
  __shared__ int s_have, s_stop;
  __shared__ SrvReq s_req;
  for (int i = threadIdx.x * 16; i < kSrvSlots * (4 + 8); i += kSrvThreads * 16)
    *reinterpret_cast<int4*>(smem + i) = make_int4(0, 0, 0, 0);
  // Idle polls back off from 1 us to 128 us: every poll reads host memory
  // over the chip-to-chip link.  The kernel leaves when the host sets the
  // stop word (it does so once no work has been outstanding for idle_polls x
  // 4 us); a CTA also leaves on its own after 100 times that without work,
  // so that no wait is unbounded.  CTAs do not leave one by one between
  // bursts of requests: a thinned-out grid would serve the next burst with
  // a few CTAs.  The request record is re-read only when the claimed item
  // belongs to another request than the CTA's last one.
  unsigned long long idle_ns = 0;
  unsigned nap = 1000;
  int last_req = -1;
  unsigned long long last_seq = 0;
  for (;;) {
    if (threadIdx.x == 0) {
      s_have = 0;
      s_stop = *(const volatile unsigned*)S.stop;
      for (int tries = 0; tries < 64; ++tries) {  // bounded: claim races with other CTAs
        const unsigned long long t = ld_acquire_sys(S.tail);
        const unsigned long long h = *(volatile unsigned long long*)S.head;
        if (h >= t) break;
        if (atomicCAS(S.head, h, h + 1) == h) {
          const volatile int* ip = reinterpret_cast<const volatile int*>(S.ring + h % S.ring_cap);
          const int2 it = make_int2(ip[0], ip[1]);
          s_item = it;
          const volatile SrvReq* rq = S.reqs + it.x;
          // a slot is reused by later requests: its sequence number tells
          const unsigned long long seq = rq->seq;
          if (it.x != last_req || seq != last_seq) {
            SrvReq r;
            r.measure = rq->measure;
            r.cap = rq->cap;
            r.k = rq->k;
            r.n_src = rq->n_src;
            r.src_off = rq->src_off;
            r.out_off = rq->out_off;
            r.target = rq->target;
            r.seq = seq;
            s_req = r;
            last_req = it.x;
            last_seq = seq;
          }
          s_have = 1;
          break;
        }
      }
    }
    __syncthreads();
    if (!s_have) {  // CTA-uniform
      idle_ns += nap;
      if (idle_ns > (unsigned long long)S.idle_polls * 400000ull || s_stop) break;
      if (threadIdx.x == 0) __nanosleep(nap);
      nap = min(2u * nap, 128000u);
      __syncthreads();
      continue;
    }
    idle_ns = 0;
    nap = 1000;
    const int2 it = s_item;
    const SrvReq R = s_req;
    const int a = *(const volatile int*)(S.src_pool + R.src_off + it.y);
    lp_link* row = S.out_pool + R.out_off + (long long)it.y * R.k;
    const bool ok = (R.measure == LP_AA || R.measure == LP_RA)
                        ? serve_source<u64>(S, R, a, row, smem, tops)
                        : serve_source<u32>(S, R, a, row, smem, tops);
    if (threadIdx.x == 0) {
      if (!ok) *(volatile unsigned char*)(S.defer + R.src_off + it.y) = 1;
      __threadfence_system();  // the row is visible before the count and the flag
      const unsigned long long old = atomicAdd(S.finished + it.x, 1ull);
      if ((long long)old + 1 == R.target) st_release_sys(S.done + it.x, R.seq);
    }
    __syncthreads();
  }
}

size_t serve_smem_bytes(int max_k) {
  return (size_t)kSrvSlots * (4 + 8) + (size_t)kSrvWarps * max_k * sizeof(TopEnt);
}

cudaError_t launch_serve(const SrvArgs& S, int max_k, cudaStream_t st) {
  const size_t smem = serve_smem_bytes(max_k);
  cudaError_t e = cudaFuncSetAttribute(k_serve, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0, dev = 0, nsm = 1;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_serve, kSrvThreads, smem);
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  k_serve<<<nsm * per_sm, kSrvThreads, smem, st>>>(S);
  return cudaGetLastError();
}

cudaError_t preload_serve_kernel() {
  cudaFuncAttributes fa;
  return cudaFuncGetAttributes(&fa, k_serve);
}

}  // namespace lp
