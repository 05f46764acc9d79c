// lp_noalloc.cu -- per-source prediction without any allocation.
//
// Some callers cannot allocate device memory at call time: code that runs
// under a memory pool it does not own, inside a runtime that forbids
// cudaMalloc on its request path, or where an allocation could trigger a
// device-wide synchronisation at an unwanted moment.  For them
// lp_predict_sources_static runs the same per-source scan as
// lp_predict_sources_dev, but every piece of working memory comes from one
// fixed array in device global memory that the library declares at file
// scope (kStaticScratchBytes).  The caller passes inputs and outputs as
// device pointers; nothing is allocated, neither on the device nor on the
// host heap.
//
// The array is a host-side symbol: its device address is looked up with
// cudaGetSymbolAddress once per device, with that device current, and the
// address is what the kernels receive.  The lookup is what makes the array
// (and the code of its module) resident on the device, so it is done when a
// graph is created on that device (prepare_static, called by
// lp_graph_create), together with loading every kernel the per-source path
// launches: a query never performs it.  Every call uses the same array, so
// calls that overlap on the GPU race on it; the per-call counters are
// cleared at the start of each call.
#include <mutex>

#include "lp_internal.cuh"

namespace lp {

constexpr size_t kStaticScratchBytes = 32u << 20;  // 32 MiB per device
constexpr int kStaticMaxDevices = 64;
constexpr int kStaticMaxSplits = 4096;      // split records handled per round
constexpr int kStaticMaxPartials = 65536;   // partial lists merged per call

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

static std::mutex g_static_mu;
static void* g_static_ptr[kStaticMaxDevices];
static std::mutex g_call_mu;  // host-side serialisation of the shared array

// Host-side fixed buffers (no heap use at call time).
static int4 h_splits[kStaticMaxSplits];
static int4 h_heads[2 * kStaticMaxSplits];
static int2 h_hdr[kStaticMaxPartials];
static int h_order[kStaticMaxPartials];
static int4 h_grp[kStaticMaxPartials];
constexpr int kStaticMaxSources = 1 << 20;
static int h_cnt[kStaticMaxSources];   // zero between calls
static int h_pos[kStaticMaxSources];

__global__ void k_static_check_sources(const int* __restrict__ s, int n_src, int n,
                                       u32* __restrict__ bad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_src && (s[i] < 0 || s[i] >= n)) atomicExch(bad, 1u);
}

// Device address of the array on device dev (current), looked up once.
cudaError_t prepare_static(int dev) {
  if (dev < 0 || dev >= kStaticMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (g_static_ptr[dev]) return cudaSuccess;
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, k_static_check_sources);
  if (e == cudaSuccess) e = preload_sources_kernels();
  if (e != cudaSuccess) return e;
  g_static_ptr[dev] = p;
  return cudaSuccess;
}

// The address prepared for device dev, or null if no graph was created there.
static void* static_scratch(int dev) {
  if (dev < 0 || dev >= kStaticMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lock(g_static_mu);
  return g_static_ptr[dev];
}

// Bump allocator over the static array.
struct Arena {
  unsigned char* base;
  size_t used, cap;
  template <typename T>
  T* take(size_t count) {
    const size_t off = (used + 255) & ~size_t(255);
    const size_t bytes = count * sizeof(T);
    if (off + bytes > cap) return nullptr;
    used = off + bytes;
    return reinterpret_cast<T*>(base + off);
  }
  size_t left() const { return cap > used + 256 ? cap - used - 256 : 0; }
};

static lp_status run_static(Graph& g, int measure, int cap, const int* d_src, int n_src, int k,
                            double threshold, lp_link* d_out, int* d_counts) {
  cudaStream_t st = g.stream;
  {
    const lp_status s = accuracy_guard(g, measure, cap, "lp_predict_sources_static");
    if (s != LP_OK) return s;
  }
  void* base = static_scratch(g.device);
  if (!base)
    return report_error(LP_EINTERNAL,
                        "lp_predict_sources_static: static scratch not prepared on this device");
  cudaError_t e = cudaSuccess;
  Arena ar{reinterpret_cast<unsigned char*>(base), 0, kStaticScratchBytes};
  Counters* d_ctr = ar.take<Counters>(1);
  int4* warpq = ar.take<int4>((size_t)n_src + 1);
  int4* medq = ar.take<int4>((size_t)n_src + 1);
  int2* grp = ar.take<int2>((size_t)n_src + 1);
  TopEnt* top = ar.take<TopEnt>((size_t)n_src * k);
  int4* split = ar.take<int4>(kStaticMaxSplits);
  int4* qa = ar.take<int4>(2 * kStaticMaxSplits);
  if (!d_ctr || !warpq || !medq || !grp || !top || !split || !qa)
    return report_error(LP_EINVAL,
                        "lp_predict_sources_static: n_src * k does not fit the static scratch "
                        "(32 MiB: about n_src * (40 + 24 k) bytes plus item space)");
  // the rest: per large item one queue record, one partial list and its index
  const size_t per_item = sizeof(int4) + (size_t)k * sizeof(TopEnt) + sizeof(int2) + sizeof(int4) +
                          sizeof(int);
  const u64 item_cap = (u64)(ar.left() / (per_item + 64));
  int4* itemq = ar.take<int4>(item_cap + 1);
  TopEnt* partial = ar.take<TopEnt>(item_cap * k + 1);
  int2* phdr = ar.take<int2>(item_cap + 1);
  int4* d_grp = ar.take<int4>(item_cap + 1);
  int* d_order = ar.take<int>(item_cap + 1);
  if (!itemq || !partial || !phdr || !d_grp || !d_order || item_cap == 0)
    return report_error(LP_EINVAL, "lp_predict_sources_static: no room left for items");

  // reject out-of-range sources before any kernel reads them
  e = cudaMemsetAsync(d_ctr, 0, sizeof(Counters), st);
  if (e != cudaSuccess) return report_cuda(e, "lp_predict_sources_static: clear");
  k_static_check_sources<<<(n_src + 255) / 256, 256, 0, st>>>(d_src, n_src, g.n, &d_ctr->error);
  u32 bad = 0;
  e = cudaMemcpyAsync(&bad, &d_ctr->error, sizeof(u32), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return report_cuda(e, "lp_predict_sources_static: source check");
  if (bad) return report_error(LP_EINVAL, "lp_predict_sources_static: source id out of range");
  e = cudaMemsetAsync(d_counts, 0, sizeof(int) * (size_t)n_src, st);
  if (e != cudaSuccess) return report_cuda(e, "lp_predict_sources_static: clear counts");
  if (cap == 0 || g.n == 0) {  // nothing to predict: rows of fillers
    e = launch_emit_sources(nullptr, d_counts, d_src, n_src, k, measure, g.fixbits, d_out, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? LP_OK : report_cuda(e, "lp_predict_sources_static");
  }

  ScanArgs A = scan_args(g, measure, cap, threshold, 1, k);
  A.sources = d_src;
  A.out_top = top;
  A.out_cnt = d_counts;
  A.ctr = d_ctr;
  Counters h{};
  e = cudaMemsetAsync(d_ctr, 0, sizeof(Counters), st);
  if (e == cudaSuccess) e = launch_estimate2(A, n_src, warpq, medq, itemq, item_cap, grp, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d_ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return report_cuda(e, "lp_predict_sources_static: estimate");
  if (h.nitem > item_cap)
    return report_error(LP_EINVAL,
                        "lp_predict_sources_static: the sources need more work items than the "
                        "static scratch holds; use fewer sources per call");
  stats_estimate(h);
  int launches = 1;
  u64 nw = h.nwarp, nm = h.nmed, nc = h.nitem;
  int4* cq = itemq;
  u64 npartial = 0;
  for (int round = 0; nw + nm + nc > 0; ++round) {
    if (round > 10000) return report_error(LP_EINTERNAL, "lp_predict_sources_static: no progress");
    Counters z{};
    z.npartial = npartial;
    e = cudaMemcpyAsync(d_ctr, &z, sizeof(Counters), cudaMemcpyHostToDevice, st);
    A.split = split;
    A.split_cap = kStaticMaxSplits;
    A.partial = partial;
    A.partial_hdr = phdr;
    A.partial_cap = item_cap;
    if (e == cudaSuccess && nc) e = launch_scan_cta(A, cq, nc, st);
    if (e == cudaSuccess && nm) e = launch_scan_med(A, medq, nm, st);
    if (e == cudaSuccess && nw) e = launch_scan_warp(A, warpq, nw, st);
    launches += (nc > 0) + (nm > 0) + (nw > 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d_ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return report_cuda(e, "lp_predict_sources_static: scan");
    if (h.error == 2u)  // more overflowed items than the split records hold
      return report_error(LP_EINVAL,
                          "lp_predict_sources_static: the sources overflow more work items than "
                          "the static scratch can re-split in one round; use fewer sources per call");
    if (h.error == 3u)  // more partial lists than the static scratch holds
      return report_error(LP_EINVAL,
                          "lp_predict_sources_static: the sources need more partial lists than the "
                          "static scratch holds; use fewer sources per call");
    if (h.error) return report_error(LP_EINTERNAL, "lp_predict_sources_static: device check failed");
    stats_add((int64_t)h.candidates, (int32_t)h.nsplit, 0);
    npartial = h.npartial;
    if (npartial > (u64)kStaticMaxPartials)
      return report_error(LP_EINVAL,
                          "lp_predict_sources_static: the sources need more partial lists than "
                          "can be merged in one call (65536); use fewer sources per call");
    nw = nm = nc = 0;
    if (h.nsplit == 0) break;
    // overflowed hash items: run again as two halves (dense when narrow)
    if (h.nsplit > (u64)kStaticMaxSplits)
      return report_error(LP_EINVAL,
                          "lp_predict_sources_static: too many overflowed items to re-split; use "
                          "fewer sources per call");
    e = cudaMemcpy(h_splits, split, sizeof(int4) * h.nsplit, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return report_cuda(e, "lp_predict_sources_static: splits");
    u64 nh = 0;
    for (u64 i = 0; i < h.nsplit; ++i) {
      const int4 r = h_splits[i];
      const int logcap = (r.w >> 8) & 0xff;
      if (r.z - r.y <= A.big_span) {
        h_heads[nh++] = make_int4(r.x, r.y, r.z, kItemDense | (logcap << 8));
      } else {
        const int mid = r.y + (r.z - r.y) / 2;
        h_heads[nh++] = make_int4(r.x, r.y, mid, logcap << 8);
        h_heads[nh++] = make_int4(r.x, mid, r.z, logcap << 8);
      }
    }
    if (npartial + nh > item_cap)
      return report_error(LP_EINVAL, "lp_predict_sources_static: partial lists exceed the scratch");
    e = cudaMemcpyAsync(qa, h_heads, sizeof(int4) * nh, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return report_cuda(e, "lp_predict_sources_static: requeue");
    cq = qa;
    nc = nh;
  }
  if (npartial) {
    e = cudaMemcpy(h_hdr, phdr, sizeof(int2) * npartial, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return report_cuda(e, "lp_predict_sources_static: partials");
    // group the partial lists by record: counting sort over the records
    // that occur (fixed host arrays, left zero afterwards)
    for (u64 i = 0; i < npartial; ++i) h_cnt[h_hdr[i].x]++;
    int ng = 0, run = 0;
    for (u64 i = 0; i < npartial; ++i) {
      const int r = h_hdr[i].x;
      if (h_cnt[r] > 0) {
        h_grp[ng++] = make_int4(r, run, h_cnt[r], 0);
        h_pos[r] = run;
        run += h_cnt[r];
        h_cnt[r] = -1;  // placed
      }
    }
    for (u64 i = 0; i < npartial; ++i) h_order[h_pos[h_hdr[i].x]++] = (int)i;
    for (u64 i = 0; i < npartial; ++i) h_cnt[h_hdr[i].x] = 0;
    e = cudaMemcpyAsync(d_grp, h_grp, sizeof(int4) * ng, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_order, h_order, sizeof(int) * npartial, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = launch_merge_partials(d_grp, ng, d_order, partial, phdr, k, top, d_counts, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return report_cuda(e, "lp_predict_sources_static: merge");
    ++launches;
  }
  e = launch_emit_sources(top, d_counts, d_src, n_src, k, measure, g.fixbits, d_out, st);
  ++launches;
  if (e == cudaSuccess && (measure == LP_AA || measure == LP_RA)) {
    e = launch_pair_cn(d_out, d_counts, k, (u64)n_src * k, g.d_off, g.d_idx, g.d_deg, g.d_arc,
                       A.cap, st);
    ++launches;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return report_cuda(e, "lp_predict_sources_static: emit");
  stats_add(0, 0, launches);
  return LP_OK;
}

}  // namespace lp

extern "C" lp_status lp_predict_sources_static(const lp_graph* g, lp_measure measure,
                                               int32_t degree_cap, const int32_t* d_sources,
                                               int32_t n_src, int32_t k, double threshold,
                                               lp_link* d_out, int32_t* d_counts) {
  lp::stats_begin();
  lp_status s = lp::sources_args_ok(g, (int)measure, d_sources, n_src, k, d_out, d_counts);
  if (s != LP_OK) return s;
  if (n_src == 0) return LP_OK;
  if (n_src > lp::kStaticMaxSources)
    return lp::report_error(LP_EINVAL, "lp_predict_sources_static: n_src above 2^20");
  lp::Graph& gg = lp::graph_of(g);
  std::lock_guard<std::mutex> lock_graph(gg.mu);
  std::lock_guard<std::mutex> lock_static(lp::g_call_mu);
  const cudaError_t e = cudaSetDevice(gg.device);
  if (e != cudaSuccess) return lp::report_cuda(e, "cudaSetDevice");
  return lp::run_static(gg, (int)measure, degree_cap, d_sources, n_src, k, threshold, d_out,
                        d_counts);
}
