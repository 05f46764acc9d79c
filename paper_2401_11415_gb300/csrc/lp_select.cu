// lp_select.cu -- exact top-k selection of candidates by radix digits.
//
// The selection keeps the N_P best pairs under the total order (score desc,
// u asc, v asc); the paper does this with per-thread min-heaps and a
// sequential heap merge (Section 4.1.6-4.1.7, Algorithm 1).  Here each
// candidate gets a 128-bit rank key K:~u:~v whose order is the total order,
// and the k largest keys are found by most-significant-digit radix
// selection: one histogram per digit over the still-undecided candidates,
// the bins above the cut are taken whole, the bin at the cut is refined by
// the next digit.  Only the k survivors are then sorted exactly.
//
// K is exact for CN (the count), AA and RA (the fixed-point sum) and for JC,
// SI, HP and HD, whose values p/q lie in [0, 1] with q < 2^32:
// K = floor(p * 2^64 / q) (2^64 - 1 for p = q) separates any two distinct
// such fractions, because they differ by at least 1 / (q q') > 2^-64.  For
// Salton (through its square) and LHN the denominators reach 2^62, so K is
// the bit pattern of the FP64 value: monotone but not strict.  For those the
// selection stops once K is resolved and keeps the whole group that ties on
// K at the cut; the exact sort then orders it and the caller cuts to k.
#include <algorithm>
#include <vector>

#include "lp_internal.cuh"

namespace lp {

constexpr int kRadixBins = 2048;

// Digit schedule over the 128-bit key (bit 127 first): widths per pass.
__host__ __device__ __forceinline__ void digit_at(int pass, int& shift, int& width) {
  // K: 11 11 11 11 10 10 | ~u: 11 11 10 | ~v: 11 11 10
  const int widths[12] = {11, 11, 11, 11, 10, 10, 11, 11, 10, 11, 11, 10};
  int top = 128;
  for (int i = 0; i < pass; ++i) top -= widths[i];
  width = widths[pass];
  shift = top - width;
}

__device__ __forceinline__ u64 frac64(u64 p, u64 q) {
  if (p >= q) return ~0ull;
  const u64 hi = (p << 32) / q;
  const u64 r = (p << 32) % q;
  const u64 lo = (r << 32) / q;
  return (hi << 32) | lo;
}

__device__ __forceinline__ u64 rank_k(int measure, const Cand& c) {
  switch (measure) {
    case LP_JC:
    case LP_SI:
    case LP_HP:
    case LP_HD:
      return frac64(c.num, c.den);
    case LP_SC:
    case LP_LHN:
      return (u64)__double_as_longlong(__ddiv_rn(__ull2double_rn(c.num), __ull2double_rn(c.den)));
    default:
      return c.num;  // CN count, AA / RA fixed-point sum (den = 1)
  }
}

__device__ __forceinline__ u32 digit_of(int measure, const Cand& c, int shift, int width) {
  const u64 hi = rank_k(measure, c);
  const u64 lo = ((u64)(~(u32)c.u) << 32) | (u64)(~(u32)c.v);
  u64 d;
  if (shift >= 64) d = hi >> (shift - 64);
  else if (shift + width <= 64) d = lo >> shift;
  else d = (hi << (64 - shift)) | (lo >> shift);  // straddles the halves
  return (u32)(d & ((1u << width) - 1u));
}

__global__ void k_radix_hist(const Cand* __restrict__ a, u64 n, int measure, int shift, int width,
                             u32* __restrict__ hist) {
  __shared__ u32 h[kRadixBins];
  for (int i = threadIdx.x; i < kRadixBins; i += blockDim.x) h[i] = 0;
  __syncthreads();
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x) {
    const u32 d = digit_of(measure, a[i], shift, width);
    // aggregate equal digits within the warp (scores often concentrate)
    const u32 peers = __match_any_sync(__activemask(), d);
    if ((threadIdx.x & 31) == (u32)(__ffs(peers) - 1)) atomicAdd(&h[d], (u32)__popc(peers));
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kRadixBins; i += blockDim.x)
    if (h[i]) atomicAdd(&hist[i], h[i]);
}

// digit > cut -> sel[*sel_n ...]; digit == cut -> act[*act_n ...] (take_cut:
// the cut bin goes to sel as well).
__global__ void k_radix_split(const Cand* __restrict__ a, u64 n, int measure, int shift, int width,
                              u32 cut, int take_cut, Cand* __restrict__ sel, u64* __restrict__ sel_n,
                              Cand* __restrict__ act, u64* __restrict__ act_n) {
  const int lane = threadIdx.x & 31;
  const u64 stride = (u64)gridDim.x * blockDim.x;
  const u64 n_round = ((n + stride - 1) / stride) * stride;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n_round; i += stride) {
    Cand c;
    int dest = -1;  // 0 sel, 1 act
    if (i < n) {
      c = a[i];
      const u32 d = digit_of(measure, c, shift, width);
      if (d > cut || (take_cut && d == cut)) dest = 0;
      else if (d == cut) dest = 1;
    }
    const u32 ms = __ballot_sync(0xffffffffu, dest == 0);
    const u32 ma = __ballot_sync(0xffffffffu, dest == 1);
    u64 bs = 0, ba = 0;
    if (lane == 0) {
      if (ms) bs = atomicAdd(sel_n, (u64)__popc(ms));
      if (ma) ba = atomicAdd(act_n, (u64)__popc(ma));
    }
    bs = __shfl_sync(0xffffffffu, bs, 0);
    ba = __shfl_sync(0xffffffffu, ba, 0);
    const u32 lt = (1u << lane) - 1u;
    if (dest == 0) sel[bs + __popc(ms & lt)] = c;
    if (dest == 1) act[ba + __popc(ma & lt)] = c;
  }
}

static int grid_for(u64 n) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const u64 want = (n + 255) / 256;
  return (int)std::max<u64>(1, std::min<u64>(want, (u64)nsm * 8));
}

// Select the k best of src[0, n) into sel.  actA / actB: scratch of n
// entries each (actB may be src itself: src is read only by the first pass).  d_hist: kRadixBins u32; d_cnt: 2 u64.  *out_n = k for the
// exact measures; for SC / LHN it can be larger (the whole tie group on K at
// the cut is kept).  Host-synchronous.
cudaError_t radix_select(const Cand* src, u64 n, u64 k, int measure, Cand* sel, Cand* actA,
                         Cand* actB, u32* d_hist, u64* d_cnt, cudaStream_t st, u64* out_n,
                         int* launches) {
  // (the last pass of the exact schedule leaves at most one key per bin, and
  // the last pass of the K-only schedule keeps the tie group on K at the cut)
  const bool exact = !(measure == LP_SC || measure == LP_LHN);
  const int npass = exact ? 12 : 6;
  *out_n = 0;
  if (k == 0 || n == 0) return cudaSuccess;
  if (k >= n) {
    *out_n = n;
    return cudaMemcpyAsync(sel, src, sizeof(Cand) * n, cudaMemcpyDeviceToDevice, st);
  }
  u64 sel_n = 0;
  u64 need = k;
  const Cand* act = src;
  u64 act_n = n;
  Cand* bufs[2] = {actA, actB};
  int which = 0;
  std::vector<u32> h(kRadixBins);
  cudaError_t e = cudaSuccess;
  for (int pass = 0; pass < npass && need > 0; ++pass) {
    int shift, width;
    digit_at(pass, shift, width);
    const int bins = 1 << width;
    e = cudaMemsetAsync(d_hist, 0, sizeof(u32) * kRadixBins, st);
    if (e != cudaSuccess) return e;
    k_radix_hist<<<grid_for(act_n), 256, 0, st>>>(act, act_n, measure, shift, width, d_hist);
    if (launches) ++*launches;
    e = cudaMemcpyAsync(h.data(), d_hist, sizeof(u32) * kRadixBins, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    // cut bin: count strictly above < need <= above + h[cut]
    u64 above = 0;
    int cut = bins - 1;
    for (; cut >= 0; --cut) {
      if (above + h[cut] >= need) break;
      above += h[cut];
    }
    if (cut < 0) cut = 0;  // cannot happen: need <= act_n
    const bool take_all = (above + h[cut] == need) || (pass == npass - 1);
    u64 cnt_host[2] = {sel_n, 0};
    e = cudaMemcpyAsync(d_cnt, cnt_host, sizeof(cnt_host), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    Cand* next = bufs[which];
    k_radix_split<<<grid_for(act_n), 256, 0, st>>>(act, act_n, measure, shift, width, (u32)cut,
                                                   take_all ? 1 : 0, sel, d_cnt, next, d_cnt + 1);
    if (launches) ++*launches;
    e = cudaMemcpyAsync(cnt_host, d_cnt, sizeof(cnt_host), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    sel_n = cnt_host[0];
    if (take_all) {
      need = 0;
      break;
    }
    need -= above;
    act = next;
    act_n = cnt_host[1];
    which ^= 1;
  }
  *out_n = sel_n;
  return e;
}

// The worst candidate of a[0, n) under the total order (for the threshold
// after a compaction): block minima, then one block over the partials.
__global__ void k_worst(const Cand* __restrict__ a, u64 n, Cand* __restrict__ out) {
  __shared__ Cand s[256];
  Cand w;
  bool have = false;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x) {
    const Cand c = a[i];
    if (!have || cand_before(w, c)) w = c;
    have = true;
  }
  if (!have) {
    w.num = ~0ull;  // neutral: ranks before everything
    w.den = 1;
    w.u = -1;
    w.v = -1;
  }
  s[threadIdx.x] = w;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < (unsigned)o && cand_before(s[threadIdx.x], s[threadIdx.x + o]))
      s[threadIdx.x] = s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = s[0];
}

__global__ void k_thresh_from(const Cand* __restrict__ c, Thresh* __restrict__ t) {
  t->num = c->num;
  t->den = c->den;
  t->u = c->u;
  t->v = c->v;
  t->valid = 1;
}

// Threshold := the worst of a[0, n) (n >= 1).  tmp: >= 257 Cand.
cudaError_t launch_thresh_worst(const Cand* a, u64 n, Cand* tmp, Thresh* t, cudaStream_t st,
                                int* launches) {
  const int blocks = (int)std::min<u64>(256, (n + 255) / 256);
  k_worst<<<blocks, 256, 0, st>>>(a, n, tmp);
  k_worst<<<1, 256, 0, st>>>(tmp, (u64)blocks, tmp + 256);
  k_thresh_from<<<1, 1, 0, st>>>(tmp + 256, t);
  if (launches) *launches += 3;
  return cudaGetLastError();
}

}  // namespace lp
