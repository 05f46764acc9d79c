// lp_sort.cu -- exact sort of selection candidates, and buffer compaction.
//
// The paper merges per-thread top-N_P lists with a sequential max-heap
// (Algorithm 1, merging phase; Section 4.1.7), the part that does not scale
// (Section 5.4).  Here the candidates of all sources sit in one device buffer
// and are ordered by a parallel merge sort whose comparator is the exact
// total order: the rational score num/den by 128-bit cross-multiplication,
// then u, then v.  Blocks sort 2048-element tiles with a bitonic network in
// shared memory; merge-path passes then double the run length.
#include "lp_internal.cuh"

namespace lp {

constexpr int kTile = 2048;          // elements per block-sorted tile
constexpr int kTileThreads = 1024;
constexpr int kMergeThreads = 256;
constexpr int kMergeVT = 8;
constexpr int kMergeNB = kMergeThreads * kMergeVT;  // outputs per merge block (= kTile)

__device__ __forceinline__ Cand worst_cand() {
  Cand c;
  c.num = 0;
  c.den = 1;
  c.u = 0x7fffffff;
  c.v = 0x7fffffff;
  return c;
}

// Sort each kTile-element tile in place (bitonic network, padded with the
// worst possible candidate).
__global__ void __launch_bounds__(kTileThreads) k_tile_sort(Cand* __restrict__ a, u64 n) {
  __shared__ Cand s[kTile];
  const u64 base = (u64)blockIdx.x * kTile;
  for (int i = threadIdx.x; i < kTile; i += blockDim.x)
    s[i] = (base + i < n) ? a[base + i] : worst_cand();
  __syncthreads();
  for (int size = 2; size <= kTile; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = threadIdx.x; t < kTile / 2; t += blockDim.x) {
        const int i = 2 * t - (t & (stride - 1));
        const int j = i + stride;
        const bool up = ((i & size) == 0);  // ascending in "before" order
        Cand x = s[i], y = s[j];
        const bool swap = up ? cand_before(y, x) : cand_before(x, y);
        if (swap) {
          s[i] = y;
          s[j] = x;
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < kTile; i += blockDim.x)
    if (base + i < n) a[base + i] = s[i];
}

// Merge path: number of elements taken from A among the first `diag` outputs
// of merge(A, B), A first on ties.
template <typename GetA, typename GetB>
__device__ __forceinline__ int merge_path(GetA ga, int na, GetB gb, int nb, int diag) {
  int lo = diag > nb ? diag - nb : 0;
  int hi = diag < na ? diag : na;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    const Cand b = gb(diag - 1 - mid);
    const Cand x = ga(mid);
    if (!cand_before(b, x)) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Split points of every merge block of one pass (runs of length `width`).
__global__ void k_merge_partition(const Cand* __restrict__ src, u64 n, u64 width,
                                  int* __restrict__ splits, u64 nblocks) {
  const u64 bi = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (bi >= nblocks) return;
  const u64 k0 = bi * kMergeNB;
  const u64 pair0 = (k0 / (2 * width)) * (2 * width);
  const u64 a0 = pair0;
  const int na = (int)min(width, n - a0);
  const u64 b0 = a0 + na;
  const int nb = (int)(b0 < n ? min(width, n - b0) : 0);
  const int diag = (int)(k0 - pair0);
  splits[bi] = merge_path([&](int i) { return src[a0 + i]; }, na,
                          [&](int i) { return src[b0 + i]; }, nb, diag);
}

__global__ void __launch_bounds__(kMergeThreads) k_merge(const Cand* __restrict__ src,
                                                         Cand* __restrict__ dst, u64 n, u64 width,
                                                         const int* __restrict__ splits) {
  __shared__ Cand s[kMergeNB];
  const u64 bi = blockIdx.x;
  const u64 k0 = bi * kMergeNB;
  const u64 pair0 = (k0 / (2 * width)) * (2 * width);
  const u64 a0 = pair0;
  const int na = (int)min(width, n - a0);
  const u64 b0 = a0 + na;
  const int nb = (int)(b0 < n ? min(width, n - b0) : 0);
  const int d0 = (int)(k0 - pair0);
  const int d1 = (int)min((u64)(d0 + kMergeNB), (u64)(na + nb));
  const int as = splits[bi];
  const int ae = (d1 == na + nb) ? na : splits[bi + 1];
  const int bs = d0 - as, be = d1 - ae;
  const int la = ae - as, lb = be - bs;
  for (int i = threadIdx.x; i < la; i += blockDim.x) s[i] = src[a0 + as + i];
  for (int i = threadIdx.x; i < lb; i += blockDim.x) s[la + i] = src[b0 + bs + i];
  __syncthreads();
  const int total = la + lb;
  const int diag = min((int)threadIdx.x * kMergeVT, total);
  int ai = merge_path([&](int i) { return s[i]; }, la, [&](int i) { return s[la + i]; }, lb, diag);
  int bj = diag - ai;
  Cand out[kMergeVT];
  int cnt = 0;
#pragma unroll
  for (int t = 0; t < kMergeVT; ++t) {
    if (diag + t < total) {
      bool takeA;
      if (ai >= la) takeA = false;
      else if (bj >= lb) takeA = true;
      else takeA = !cand_before(s[la + bj], s[ai]);
      out[t] = takeA ? s[ai] : s[la + bj];
      if (takeA) ++ai; else ++bj;
      cnt = t + 1;
    }
  }
  __syncthreads();
#pragma unroll
  for (int t = 0; t < kMergeVT; ++t)
    if (t < cnt) dst[k0 + diag + t] = out[t];
}

// Sort d_a[0, n).  The result ends in *result (d_a or d_tmp).  splits must
// hold sort_splits_needed(n) ints.
cudaError_t launch_sort_cands(Cand* d_a, Cand* d_tmp, int* splits, u64 n, cudaStream_t st,
                              Cand** result, int* launches) {
  *result = d_a;
  if (n <= 1) return cudaSuccess;
  const u64 tiles = (n + kTile - 1) / kTile;
  k_tile_sort<<<(unsigned)tiles, kTileThreads, 0, st>>>(d_a, n);
  if (launches) ++*launches;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  Cand* src = d_a;
  Cand* dst = d_tmp;
  const u64 nblocks = (n + kMergeNB - 1) / kMergeNB;
  for (u64 width = kTile; width < n; width *= 2) {
    k_merge_partition<<<(unsigned)((nblocks + 255) / 256), 256, 0, st>>>(src, n, width, splits,
                                                                         nblocks);
    k_merge<<<(unsigned)nblocks, kMergeThreads, 0, st>>>(src, dst, n, width, splits);
    if (launches) *launches += 2;
    e = cudaGetLastError();
    if (e != cudaSuccess) break;
    Cand* t = src;
    src = dst;
    dst = t;
  }
  *result = src;
  return e;
}

// Drop entries that belong to failed records: flagged source u with v inside
// one of the failed ranges of u (failed sorted by (a, lo)).  Appends the kept
// entries to d_out[*d_count ...).
__global__ void k_filter_failed(const Cand* __restrict__ buf, u64 n,
                                const unsigned char* __restrict__ flag,
                                const int4* __restrict__ failed, int nfailed,
                                Cand* __restrict__ out, u64* __restrict__ count) {
  const u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  bool keep = false;
  Cand x;
  if (i < n) {
    x = buf[i];
    keep = true;
    if (flag[x.u]) {
      int lo = 0, hi = nfailed;  // first record with a >= x.u
      while (lo < hi) {
        const int m = (lo + hi) >> 1;
        if (failed[m].x < x.u) lo = m + 1; else hi = m;
      }
      for (int j = lo; j < nfailed && failed[j].x == x.u; ++j)
        if (x.v >= failed[j].y && x.v < failed[j].z) keep = false;
    }
  }
  const unsigned mask = __ballot_sync(0xffffffffu, keep);
  if (mask == 0) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(mask) - 1;
  u64 base = 0;
  if (lane == leader) base = atomicAdd(count, (u64)__popc(mask));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (keep) out[base + __popc(mask & ((1u << lane) - 1u))] = x;
}

cudaError_t launch_filter_failed(Cand* d_buf, u64 n, const unsigned char* d_flag,
                                 const int4* d_failed_sorted, int nfailed, Cand* d_out,
                                 Counters* d_ctr, u64* d_count, cudaStream_t st) {
  (void)d_ctr;
  if (n == 0) return cudaSuccess;
  k_filter_failed<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(d_buf, n, d_flag, d_failed_sorted,
                                                               nfailed, d_out, d_count);
  return cudaGetLastError();
}

// Threshold := element k-1 of the sorted candidates.
__global__ void k_set_thresh(const Cand* __restrict__ sorted, u64 k, Thresh* __restrict__ t) {
  const Cand c = sorted[k - 1];
  t->num = c.num;
  t->den = c.den;
  t->u = c.u;
  t->v = c.v;
  t->valid = 1;
}

cudaError_t launch_set_thresh(const Cand* sorted, u64 k, Thresh* t, cudaStream_t st) {
  k_set_thresh<<<1, 1, 0, st>>>(sorted, k, t);
  return cudaGetLastError();
}

}  // namespace lp
