// lp_api.cu -- the C ABI of liblp: graph residency and the predict calls.
//
// Graph residency: the CSR is validated on the host, uploaded once, and a
// per-arc table is built on the device (for arc a -> b: the position of a in
// the sorted list of b, the end of that list and |Gamma_b|), so that the scan
// finds the c > a suffix of Gamma_b without searching and tests the hub limit
// without touching Gamma_b (Algorithm 1; Sections 4.1.2 and 4.2.1).
//
// Global mode (Algorithm 1 end to end): estimate and bin the sources, scan
// them, and select the N_P best pairs.  The paper keeps a top-N_P heap per
// thread and merges the heaps sequentially (Section 4.1.7).  Here every
// scored pair that ranks before a running threshold T is appended to one
// device buffer; when the buffer fills, it is sorted exactly, cut to N_P,
// and T becomes its N_P-th entry, so later pairs must beat it.  Work that
// was in flight when the buffer filled is re-queued and its partial output
// removed, which keeps the result exact and deterministic.
#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "lp_internal.cuh"

#ifdef _OPENMP
#include <omp.h>
#endif

using namespace lp;

struct lp_graph : public lp::Graph {};

namespace lp {

static thread_local std::string t_err;
static thread_local lp_stats t_stats;
static std::atomic<int> g_timing{0};
static std::mutex g_opt_mu;
static Options g_opt;

Options options_snapshot() {
  std::lock_guard<std::mutex> l(g_opt_mu);
  return g_opt;
}

static lp_status fail(lp_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  t_err = buf;
  return s;
}

static lp_status cuda_fail(cudaError_t e, const char* what) {
  cudaGetLastError();  // clear a sticky-free error
  return fail(e == cudaErrorMemoryAllocation ? LP_ENOMEM : LP_ECUDA, "%s: %s", what,
              cudaGetErrorString(e));
}

#define CU(x)                                   \
  do {                                          \
    cudaError_t e_ = (x);                       \
    if (e_ != cudaSuccess) return cuda_fail(e_, #x); \
  } while (0)

// Grow a scratch allocation to at least `bytes` (contents are not kept).
cudaError_t ensure(Graph& g, Graph::Scratch& s, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (s.bytes >= bytes) return cudaSuccess;
  if (s.p) {
    cudaStreamSynchronize(g.stream);
    cudaFree(s.p);
    s.p = nullptr;
    s.bytes = 0;
  }
  size_t want = bytes + bytes / 4;
  cudaError_t e = cudaMalloc(&s.p, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    e = cudaMalloc(&s.p, bytes);
    if (e != cudaSuccess) return e;
    want = bytes;
  }
  s.bytes = want;
  return cudaSuccess;
}


// ------------------------------------------------------ graph residency --

// One warp per vertex a: deg[a] and the arc table of a's arcs; sets *err if
// some reverse arc is missing.
__global__ void k_build_arcs(const int* __restrict__ off, const int* __restrict__ idx, int n,
                             int* __restrict__ deg, Arc* __restrict__ arc, int* __restrict__ err) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int a = warp; a < n; a += nwarps) {
    const int e0 = off[a], e1 = off[a + 1];
    if (lane == 0) deg[a] = e1 - e0;
    for (int e = e0 + lane; e < e1; e += 32) {
      const int b = idx[e];
      int l = off[b], r = off[b + 1];
      const int end = r;
      while (l < r) {
        const int m = (l + r) >> 1;
        if (idx[m] < a) l = m + 1; else r = m;
      }
      if (l >= end || idx[l] != a) {
        atomicExch(err, 1);
        l = end - 1;
      }
      arc[e] = make_int4(l, end, end - off[b], b);
    }
  }
}

static void free_graph(Graph* g) {
  if (!g) return;
  if (g->stream) cudaStreamSynchronize(g->stream);
  Graph::Scratch* all[] = {&g->s_ctr, &g->s_w, &g->s_warpq, &g->s_itemq, &g->s_warpq2,
                           &g->s_itemq2, &g->s_medq, &g->s_medq2, &g->s_buf, &g->s_buf2,
                           &g->s_buf3, &g->s_misc, &g->s_failed, &g->s_split,
                           &g->s_thresh, &g->s_vfloor, &g->s_pair, &g->s_gcur, &g->s_flags,
                           &g->s_partial,
                           &g->s_phdr, &g->s_top,
                           &g->s_cnt, &g->s_links, &g->s_src, &g->s_grp, &g->s_xq, &g->s_xw,
                           &g->s_xunit, &g->s_xaseg, &g->s_xaoff, &g->s_xadeg, &g->s_xrec,
                           &g->s_xtile, &g->s_xtunit, &g->s_xpre, &g->s_xbunit, &g->s_countq,
                           &g->s_countq2, &g->s_xtfirst, &g->s_xexcl};
  for (auto* s : all)
    if (s->p) cudaFree(s->p);
  if (g->owns_arrays) {
    cudaFree(g->d_off);
    cudaFree(g->d_idx);
    cudaFree(g->d_deg);
    cudaFree(g->d_arc);
    cudaFree(g->d_wt);
  }
  for (auto& e : g->ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : g->kev)
    if (e) cudaEventDestroy(e);
  for (auto& e : g->xev)
    if (e) cudaEventDestroy(e);
  if (g->stream) cudaStreamDestroy(g->stream);
  delete static_cast<lp_graph*>(g);
}

}  // namespace lp

extern "C" {

const char* lp_last_error(void) { return lp::t_err.c_str(); }

const char* lp_version(void) { return "liblp 0.1 (sm_103a)"; }

void lp_set_timing(int enable) { lp::g_timing.store(enable ? 1 : 0); }

lp_status lp_set_option(lp_option option, int64_t value) {
  std::lock_guard<std::mutex> l(lp::g_opt_mu);
  switch (option) {
    case LP_OPT_SELECT_BUFFER:
      if (value < 16 || value > (1ll << 34)) break;
      lp::g_opt.select_buffer = value;
      return LP_OK;
    case LP_OPT_WARP_MAX_WEDGES:
      if (value < 1 || value > lp::kWarpMaxWedges) break;
      lp::g_opt.warp_max = (int)value;
      return LP_OK;
    case LP_OPT_MED_MAX_WEDGES:
      if (value < 1 || value > lp::kMedMaxWedges) break;
      lp::g_opt.med_max = (int)value;
      return LP_OK;
    case LP_OPT_ITEM_WEDGES:
      if (value < 1024 || value > (1ll << 30)) break;
      lp::g_opt.item_wedges = value;
      return LP_OK;
    case LP_OPT_PHASE_PROFILE:
      if (value < 0 || value > 1) break;
      lp::g_opt.phase_profile = (int)value;
      return LP_OK;
    case LP_OPT_BIG_CTA_THREADS:
      if (value != 512 && value != 1024) break;
      lp::g_opt.big_threads = (int)value;
      return LP_OK;
    case LP_OPT_EXPAND:
      if (value < 0 || value > 2) break;
      lp::g_opt.expand = (int)value;
      return LP_OK;
    case LP_OPT_EXPAND_BATCH:
      if (value < (1 << 16) || value > (1ll << 34)) break;
      lp::g_opt.expand_batch = value;
      return LP_OK;
    case LP_OPT_EXPAND_HASH_LOGCAP:
      if (value < 6 || value > 14) break;
      lp::g_opt.expand_logcap = (int)value;
      return LP_OK;
    case LP_OPT_EXPAND_MIN_WEDGES:
      if (value < 257 || value > (1ll << 30)) break;
      lp::g_opt.expand_min = (int)value;
      return LP_OK;
    case LP_OPT_CTA_MAX_WEDGES:
      if (value < 257 || value > lp::kCtaMaxWedges) break;
      lp::g_opt.cta_max = (int)value;
      return LP_OK;
    case LP_OPT_SPLIT_TARGET:
      if (value < 256 || value > 32768) break;
      lp::g_opt.split_target = (int)value;
      return LP_OK;
    case LP_OPT_SPLIT_LOGCAP:
      if (value < 6 || value > 14) break;
      lp::g_opt.split_logcap = (int)value;
      return LP_OK;
    default:
      break;
  }
  return fail(LP_EINVAL, "lp_set_option: option %d value %lld out of range", (int)option,
              (long long)value);
}

int64_t lp_get_option(lp_option option) {
  const lp::Options o = lp::options_snapshot();
  switch (option) {
    case LP_OPT_SELECT_BUFFER: return o.select_buffer;
    case LP_OPT_WARP_MAX_WEDGES: return o.warp_max;
    case LP_OPT_CTA_MAX_WEDGES: return o.cta_max;
    case LP_OPT_SPLIT_TARGET: return o.split_target;
    case LP_OPT_SPLIT_LOGCAP: return o.split_logcap;
    case LP_OPT_MED_MAX_WEDGES: return o.med_max;
    case LP_OPT_ITEM_WEDGES: return o.item_wedges;
    case LP_OPT_PHASE_PROFILE: return o.phase_profile;
    case LP_OPT_BIG_CTA_THREADS: return o.big_threads;
    case LP_OPT_EXPAND: return o.expand;
    case LP_OPT_EXPAND_BATCH: return o.expand_batch;
    case LP_OPT_EXPAND_HASH_LOGCAP: return o.expand_logcap;
    case LP_OPT_EXPAND_MIN_WEDGES: return o.expand_min;
    default: return -1;
  }
}

lp_status lp_last_stats(lp_stats* out) {
  if (!out) return fail(LP_EINVAL, "lp_last_stats: null output");
  *out = lp::t_stats;
  return LP_OK;
}

void* lp_graph_stream(const lp_graph* g) { return g ? (void*)g->stream : nullptr; }

lp_status lp_graph_info(const lp_graph* g, int32_t* n, int64_t* arcs, int32_t* max_degree) {
  if (!g) return fail(LP_EINVAL, "lp_graph_info: null graph");
  if (n) *n = g->n;
  if (arcs) *arcs = g->arcs;
  if (max_degree) *max_degree = g->dmax;
  return LP_OK;
}

lp_status lp_graph_destroy(lp_graph* g) {
  lp::free_graph(g);
  return LP_OK;
}

lp_status lp_graph_create(int32_t n, const int32_t* offsets, const int32_t* indices,
                          uint32_t flags, lp_graph** out) {
  if (!out) return fail(LP_EINVAL, "lp_graph_create: null output handle");
  *out = nullptr;
  if (n < 0) return fail(LP_EINVAL, "lp_graph_create: n < 0");
  if (!offsets) return fail(LP_EINVAL, "lp_graph_create: null offsets");
  if (offsets[0] != 0) return fail(LP_EINVAL, "lp_graph_create: offsets[0] != 0");
  for (int32_t v = 0; v < n; ++v)
    if (offsets[v + 1] < offsets[v])
      return fail(LP_EINVAL, "lp_graph_create: offsets decrease at vertex %d", v);
  const int64_t A = offsets[n];
  if (A < 0 || A >= INT32_MAX) return fail(LP_EINVAL, "lp_graph_create: too many arcs");
  if (A > 0 && !indices) return fail(LP_EINVAL, "lp_graph_create: null indices");
  // range, self-loops, order
  int bad_range = 0, bad_loop = 0, unsorted = 0, dup = 0;
  int32_t dmax = 0;
#pragma omp parallel for schedule(dynamic, 4096) reduction(| : bad_range, bad_loop, unsorted, dup) reduction(max : dmax)
  for (int32_t v = 0; v < n; ++v) {
    const int32_t d = offsets[v + 1] - offsets[v];
    if (d > dmax) dmax = d;
    for (int32_t e = offsets[v]; e < offsets[v + 1]; ++e) {
      const int32_t x = indices[e];
      if (x < 0 || x >= n) bad_range = 1;
      if (x == v) bad_loop = 1;
      if (e > offsets[v]) {
        if (indices[e - 1] > x) unsorted = 1;
        else if (indices[e - 1] == x) dup = 1;
      }
    }
  }
  if (bad_range) return fail(LP_EINVAL, "lp_graph_create: neighbour index out of range");
  if (bad_loop) return fail(LP_EINVAL, "lp_graph_create: self-loop");
  std::vector<int32_t> sorted;
  const int32_t* idx = indices;
  if (unsorted) {
    sorted.assign(indices, indices + A);
    dup = 0;
#pragma omp parallel for schedule(dynamic, 1024) reduction(| : dup)
    for (int32_t v = 0; v < n; ++v) {
      std::sort(sorted.begin() + offsets[v], sorted.begin() + offsets[v + 1]);
      for (int32_t e = offsets[v] + 1; e < offsets[v + 1]; ++e)
        if (sorted[e] == sorted[e - 1]) dup = 1;
    }
    idx = sorted.data();
  }
  if (dup) return fail(LP_EINVAL, "lp_graph_create: duplicate arc");
  if (flags & LP_VALIDATE_FULL) {
    int asym = 0;
#pragma omp parallel for schedule(dynamic, 1024) reduction(| : asym)
    for (int32_t v = 0; v < n; ++v)
      for (int32_t e = offsets[v]; e < offsets[v + 1]; ++e) {
        const int32_t b = idx[e];
        if (!std::binary_search(idx + offsets[b], idx + offsets[b + 1], v)) asym = 1;
      }
    if (asym) return fail(LP_EINVAL, "lp_graph_create: missing reverse arc");
  }

  lp_graph* g = new (std::nothrow) lp_graph();
  if (!g) return fail(LP_ENOMEM, "lp_graph_create: host allocation");
  g->n = n;
  g->arcs = A;
  g->dmax = dmax;
  {
    int lg = 0;
    while ((1ll << lg) < (int64_t)dmax + 1) ++lg;
    int f = 62 - lg;
    g->fixbits = f > 50 ? 50 : (f < 8 ? 8 : f);
  }
  cudaError_t e = cudaGetDevice(&g->device);
  int* d_err = nullptr;
  int h_err = 0;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc(&g->d_off, sizeof(int) * ((size_t)n + 1));
  if (e == cudaSuccess) e = cudaMalloc(&g->d_idx, sizeof(int) * (size_t)(A > 0 ? A : 1));
  if (e == cudaSuccess) e = cudaMalloc(&g->d_deg, sizeof(int) * (size_t)(n > 0 ? n : 1));
  if (e == cudaSuccess) e = cudaMalloc(&g->d_arc, sizeof(Arc) * (size_t)(A > 0 ? A : 1));
  if (e == cudaSuccess) e = cudaMalloc(&g->d_wt, sizeof(u64) * 2 * ((size_t)dmax + 1));
  if (e == cudaSuccess) e = cudaMalloc(&d_err, sizeof(int));
  for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaEventCreate(&g->ev[i]);
  for (int i = 0; i < 8 && e == cudaSuccess; ++i) e = cudaEventCreate(&g->kev[i]);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaEventCreate(&g->xev[i]);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(g->d_off, offsets, sizeof(int) * ((size_t)n + 1), cudaMemcpyHostToDevice,
                        g->stream);
  if (e == cudaSuccess && A > 0)
    e = cudaMemcpyAsync(g->d_idx, idx, sizeof(int) * (size_t)A, cudaMemcpyHostToDevice, g->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_err, 0, sizeof(int), g->stream);
  if (e == cudaSuccess && n > 0) {
    const int threads = 256;
    const int blocks = (int)std::min<int64_t>(((int64_t)n * 32 + threads - 1) / threads, 152 * 16);
    k_build_arcs<<<blocks, threads, 0, g->stream>>>(g->d_off, g->d_idx, n, g->d_deg, g->d_arc,
                                                    d_err);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = launch_build_weights(dmax, g->fixbits, g->d_wt, g->stream);
  // the allocation-free per-source query: its static scratch array and its
  // kernels become resident here, so that no query loads them
  if (e == cudaSuccess) e = prepare_static(g->device);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, g->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
  if (d_err) cudaFree(d_err);
  if (e != cudaSuccess) {
    lp_status s = cuda_fail(e, "lp_graph_create");
    free_graph(g);
    return s;
  }
  if (h_err) {
    free_graph(g);
    return fail(LP_EINVAL, "lp_graph_create: missing reverse arc (graph is not undirected)");
  }
  *out = g;
  return LP_OK;
}

}  // extern "C"

namespace lp {

// ------------------------------------------------------------ utilities --

static void begin_stats() {
  memset(&t_stats, 0, sizeof(t_stats));
  t_err.clear();
}

struct Timer {
  Graph& g;
  bool on;
  explicit Timer(Graph& gg) : g(gg), on(g_timing.load() != 0) {}
  void mark(int i) {
    if (on) cudaEventRecord(g.ev[i], g.stream);
  }
  float ms(int i, int j) {
    if (!on) return 0.f;
    float t = 0.f;
    cudaEventSynchronize(g.ev[j]);
    cudaEventElapsedTime(&t, g.ev[i], g.ev[j]);
    return t;
  }
};

// The three work queues (warp tier, medium tier, large tier).  cur[t] holds
// the records of the next launch, alt[t] receives the rebuilt queue.
struct Queues {
  Graph::Scratch* cur[4];
  Graph::Scratch* alt[4];
  u64 n[4];
};

// Launch the scan kernels; with timing on, time each on the graph's stream.
// Launch the scan of every tier, smallest sources first; of the large tier
// only the first large_limit items (the rest stay queued).
static cudaError_t scan_launches(Graph& g, const ScanArgs& A, const Queues& Q, bool timing,
                                 u64 large_limit = ~0ull) {
  cudaStream_t st = g.stream;
  for (int t = 0; t < 4; ++t) {
    const u64 n = t == 2 ? std::min(Q.n[t], large_limit) : Q.n[t];
    if (!n) continue;
    if (timing) cudaEventRecord(g.kev[2 * t], st);
    const int4* q = sp<int4>(*Q.cur[t]);
    cudaError_t e = t == 0   ? launch_scan_warp(A, q, n, st)
                    : t == 1 ? launch_scan_med(A, q, n, st)
                    : t == 2 ? launch_scan_cta(A, q, n, st)
                             : launch_exp_count(A, q, n, st);
    if (e != cudaSuccess) return e;
    if (timing) cudaEventRecord(g.kev[2 * t + 1], st);
    t_stats.tier_launches[t]++;
    t_stats.launches++;
  }
  return cudaSuccess;
}

// After the stream synchronised: add the kernels' event times to the stats.
static void scan_times(Graph& g, const Queues& Q, bool timing) {
  if (!timing) return;
  for (int t = 0; t < 4; ++t) {
    float ms = 0.f;
    if (Q.n[t] && cudaEventElapsedTime(&ms, g.kev[2 * t], g.kev[2 * t + 1]) == cudaSuccess)
      t_stats.tier_ms[t] += ms;
  }
}

static void estimate_stats(const Counters& h) {
  t_stats.wedges = (int64_t)h.wedges;
  t_stats.kept_arcs = (int64_t)h.kept_arcs;
  t_stats.scanned_arcs = (int64_t)h.scanned_arcs;
  t_stats.warp_sources = (int32_t)h.nwarp;
  t_stats.cta_items = (int32_t)(h.nmed + h.nitem);
  t_stats.dense_items = (int32_t)h.dense_items;
  for (int i = 0; i < 4; ++i) {
    t_stats.tier_wedges[i] = (int64_t)h.tier_wedges[i];
    t_stats.tier_arcs[i] = (int64_t)h.tier_arcs[i];
    t_stats.tier_kept[i] = (int64_t)h.tier_kept[i];
  }
}

cudaError_t attach_cursors(Graph& g, ScanArgs& A) {
  int dev = 0, nsm = 1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int ctas = 2 * nsm;  // the large tier runs at most two CTAs per SM
  const size_t stride = (size_t)g.dmax + 1;
  const size_t bytes = sizeof(int) * stride * (size_t)ctas;
  // a graph with a vertex of enormous degree does without (the sweeps then
  // search each range's boundaries), and so does a device without room
  if (bytes > (size_t)4 << 30) return cudaSuccess;
  if (ensure(g, g.s_gcur, bytes) != cudaSuccess) {
    cudaGetLastError();
    return cudaSuccess;
  }
  A.gcur = sp<int>(g.s_gcur);
  A.gcur_stride = (int)stride;
  A.gcur_ctas = ctas;
  return cudaSuccess;
}

static ScanArgs base_args(Graph& g, int measure, int cap, double threshold, int mode, int k) {
  return base_args_opts(g, measure, cap, threshold, mode, k, options_snapshot());
}

ScanArgs base_args_opts(Graph& g, int measure, int cap, double threshold, int mode, int k,
                        const Options& o) {
  ScanArgs A;
  memset(&A, 0, sizeof(A));
  const bool v64 = measure == LP_AA || measure == LP_RA;
  const int vbytes = v64 ? 8 : 4;
  const int bt = o.big_threads;
  const int tops = mode == 1 ? (bt / 32) * k * (int)sizeof(TopEnt) : 0;
  int big_bytes = kCtaSmem;
  if (bt == 1024) {
    if (mode == 1) {
      const int avail = 227 * 1024 - 2048 - big_extra_smem(1024) - tops;
      if (avail < big_bytes) big_bytes = avail & ~1023;
    }
  } else {  // two CTAs per SM: half the SM's shared memory each (1 KB for statics)
    big_bytes = (kSmemPerSm / 2 - kSmemPerCtaReserved - 1024 - big_extra_smem(bt) - tops) & ~1023;
  }
  A.big_threads = bt;
  int big_logcap = 0;
  while ((2ll << big_logcap) * (4 + vbytes) <= big_bytes) ++big_logcap;
  A.big_bytes = big_bytes;
  A.big_logcap = big_logcap;
  // dense window (128-aligned): in the global mode counters only (scored by
  // a linear scan; 16-bit for the count measures while every count, at most
  // the source degree, stays below 2^16), in the per-source mode counters
  // plus one touched bit each
  A.dense16 = mode == 0 && !v64 && g.dmax < 65536;
  const int cbytes = A.dense16 ? 2 : vbytes;
  A.big_span = mode == 0 ? (int)(((long long)big_bytes / cbytes) & ~127ll)
                         : (int)(((long long)big_bytes * 8 / (8 * vbytes + 1)) & ~127ll);
  A.warp_max = std::min(o.warp_max, kWarpMaxWedges);
  A.med_max = std::max(A.warp_max, std::min(o.med_max, kMedMaxWedges));
  A.cta_max = std::max(A.med_max, std::min(o.cta_max, 1 << (big_logcap - 1)));
  A.item_wedges = (int)o.item_wedges;
  A.split_logcap = std::min(o.split_logcap, big_logcap);
  // a smaller split table than asked for takes proportionally fewer wedges;
  // per-source items also keep k-best lists beside the table: half as many
  A.split_target = std::max(256, o.split_target >> (o.split_logcap - A.split_logcap + mode));
  A.off = g.d_off;
  A.idx = g.d_idx;
  A.deg = g.d_deg;
  A.wt = measure == LP_AA ? g.d_wt : (measure == LP_RA ? g.d_wt + (size_t)g.dmax + 1 : nullptr);
  A.arc = g.d_arc;
  A.n = g.n;
  A.cap = cap < 0 ? INT32_MAX : cap;
  A.measure = measure;
  A.mode = mode;
  A.fixbits = g.fixbits;
  A.thr_check = (threshold <= 0.0) ? 0 : 1;  // scores are > 0; NaN keeps the test
  A.threshold = threshold;
  A.k = k;
  A.prof = nullptr;
  return A;
}

// RA weights 1/|Gamma_b| are rounded to 2^-F, a relative error of at most
// |Gamma_b| 2^-(F+1) per weight and so per sum (Eq. 9).  With the largest
// degree an intermediary can have, min(L_H, dmax), that bound must stay
// within the 1e-6 contract; beyond it (intermediaries of degree above about
// 2.2M) the call is refused instead of returning less accurate scores.  AA
// weights 1/ln|Gamma_b| (Eq. 8) are large enough that the bound is
// ln|Gamma_b| 2^-(F+1), far below 1e-6 at any degree.
lp_status accuracy_guard(const Graph& g, int measure, int cap, const char* who) {
  if (measure != LP_RA) return LP_OK;
  const long long dbmax = cap < 0 ? (long long)g.dmax : std::min<long long>(cap, g.dmax);
  const double bound = (double)dbmax * ldexp(1.0, -(g.fixbits + 1));
  if (bound > 1e-6)
    return fail(LP_EINVAL,
                "%s: RA with intermediaries of degree up to %lld would exceed the 1e-6 accuracy "
                "bound (%.3g); use a hub limit below %lld",
                who, dbmax, bound, (long long)(1e-6 * ldexp(1.0, g.fixbits + 1)));
  return LP_OK;
}

// Split an overflowed hash item into two halves (dense when narrow enough).
static void split_item(const int4& r, int dense_span, std::vector<int4>& out) {
  int lo = r.y;
  const int hi = r.z;
  const int logcap = (r.w >> 8) & 0xff;
  const int keep = r.w & kItemSingle;
  const int G = ((r.w >> 16) & 0xfff) + 1;
  if (G > 1) {
    // a sweep that overflowed in its first remaining range: that range is
    // split below, the ranges after it stay one sweep
    const int first_end = lo + (int)(((long long)(hi - lo)) / G);
    out.push_back(make_int4(r.x, first_end, hi, (logcap << 8) | ((G - 2) << 16)));
    split_item(make_int4(r.x, lo, first_end, logcap << 8), dense_span, out);
    return;
  }
  if (hi - lo <= dense_span) {
    out.push_back(make_int4(r.x, lo, hi, kItemDense | (logcap << 8)));
    return;
  }
  const int mid = lo + (hi - lo) / 2;
  (void)keep;
  out.push_back(make_int4(r.x, lo, mid, (logcap << 8)));
  out.push_back(make_int4(r.x, mid, hi, (logcap << 8)));
}

// Queue = host records followed by a device remainder [src + from, src + to).
static cudaError_t build_queue(Graph& g, Graph::Scratch& dst, const std::vector<int4>& head,
                               const int4* src, u64 from, u64 to, u64* len) {
  const u64 rem = to > from ? to - from : 0;
  const u64 total = head.size() + rem;
  *len = total;
  cudaError_t e = ensure(g, dst, sizeof(int4) * (total + 1));
  if (e != cudaSuccess) return e;
  if (!head.empty())
    e = cudaMemcpyAsync(dst.p, head.data(), sizeof(int4) * head.size(), cudaMemcpyHostToDevice,
                        g.stream);
  if (e == cudaSuccess && rem)
    e = cudaMemcpyAsync(sp<int4>(dst) + head.size(), src + from, sizeof(int4) * rem,
                        cudaMemcpyDeviceToDevice, g.stream);
  if (e == cudaSuccess && !head.empty()) e = cudaStreamSynchronize(g.stream);
  return e;
}

// Rebuild the four queues: re-queued records first, then the unclaimed
// remainder of each queue.
static cudaError_t rebuild_queues(Graph& g, Queues& Q, const std::vector<int4>* heads,
                                  const u64* done) {
  for (int t = 0; t < 4; ++t) {
    if (Q.n[t] == 0 && heads[t].empty()) continue;  // stays empty
    u64 n2 = 0;
    cudaError_t e = build_queue(g, *Q.alt[t], heads[t], sp<int4>(*Q.cur[t]), done[t], Q.n[t], &n2);
    if (e != cudaSuccess) return e;
    std::swap(Q.cur[t], Q.alt[t]);
    Q.n[t] = n2;
  }
  return cudaSuccess;
}

static int record_tier(const int4& r) {
  if (r.w & (1 << 30)) return 0;
  if (r.w & (1 << 29)) return 1;
  if (r.w & kExpItem) return 3;
  return 2;
}

// An overflowed count item of the expand-and-count tier: its id range in
// halves (a range narrower than the table's fill limit cannot overflow).
static void split_count_item(const int4& r, std::vector<int4>& out) {
  const int mid = r.y + (r.z - r.y) / 2;
  out.push_back(make_int4(r.x, r.y, mid, r.w | kExpSplit));
  out.push_back(make_int4(r.x, mid, r.z, r.w | kExpSplit));
}

__global__ void k_set_flags(const int4* __restrict__ rec, int n, unsigned char* __restrict__ flag,
                            unsigned char v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) flag[rec[i].x] = v;
}

__global__ void k_check_sources(const int* __restrict__ s, int n_src, int n, int* __restrict__ bad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_src && (s[i] < 0 || s[i] >= n)) atomicExch(bad, 1);
}

// Estimate and bin; re-run once with a larger item queue if it overflowed.
static lp_status run_estimate(Graph& g, ScanArgs& A, int n_rec, int2* grp, Counters& h) {
  cudaStream_t st = g.stream;
  Counters* d_ctr = sp<Counters>(g.s_ctr);
  CU(ensure(g, g.s_warpq, sizeof(int4) * ((size_t)n_rec + 1)));
  CU(ensure(g, g.s_medq, sizeof(int4) * ((size_t)n_rec + 1)));
  u64 itemq_cap = std::max<u64>(1024, g.s_itemq.bytes / sizeof(int4));
  CU(ensure(g, g.s_itemq, sizeof(int4) * itemq_cap));
  u64 xq_cap = 0;
  if (A.expand) {
    xq_cap = std::max<u64>(1024, g.s_xq.bytes / sizeof(int4));
    CU(ensure(g, g.s_xq, sizeof(int4) * xq_cap));
    CU(ensure(g, g.s_xw, sizeof(u64) * xq_cap));
    A.xq = sp<int4>(g.s_xq);
    A.xw = sp<u64>(g.s_xw);
    A.xq_cap = xq_cap;
  }
  for (int attempt = 0; attempt < 3; ++attempt) {
    CU(cudaMemsetAsync(d_ctr, 0, sizeof(Counters), st));
    A.ctr = d_ctr;
    CU(launch_estimate2(A, n_rec, sp<int4>(g.s_warpq), sp<int4>(g.s_medq), sp<int4>(g.s_itemq),
                        itemq_cap, grp, st));
    t_stats.launches++;
    CU(cudaMemcpyAsync(&h, d_ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    if (h.nitem <= itemq_cap && h.nexp <= xq_cap) break;
    if (h.nitem > itemq_cap) {
      itemq_cap = h.nitem + 1024;
      CU(ensure(g, g.s_itemq, sizeof(int4) * itemq_cap));
    }
    if (h.nexp > xq_cap) {
      xq_cap = h.nexp + 1024;
      CU(ensure(g, g.s_xq, sizeof(int4) * xq_cap));
      CU(ensure(g, g.s_xw, sizeof(u64) * xq_cap));
      A.xq = sp<int4>(g.s_xq);
      A.xw = sp<u64>(g.s_xw);
      A.xq_cap = xq_cap;
    }
  }
  if (h.nitem > itemq_cap || h.nexp > xq_cap) return fail(LP_EINTERNAL, "item queue sizing");
  estimate_stats(h);
  return LP_OK;
}

// ---------------------------------------------------------- global mode --

constexpr size_t kMiscBytes = sizeof(u32) * 2048 + 2 * sizeof(u64) + 512 * sizeof(Cand);

static u32* misc_hist(Graph& g) { return sp<u32>(g.s_misc); }
static u64* misc_cnt(Graph& g) { return reinterpret_cast<u64*>(sp<u32>(g.s_misc) + 2048); }
static Cand* misc_worst(Graph& g) { return reinterpret_cast<Cand*>(misc_cnt(g) + 2); }

// The best k of s_buf[0, m) by radix selection; on return s_buf holds them
// (sorted = true: in order, first k of *n_out entries valid).  SC and LHN
// keep their tie group on the FP64 key and are always sorted here.
static cudaError_t select_best(Graph& g, int measure, u64 m, u64 k, u64* n_out, bool sorted) {
  cudaStream_t st = g.stream;
  u64 ns = 0;
  cudaError_t e = radix_select(sp<Cand>(g.s_buf), m, k, measure, sp<Cand>(g.s_buf2),
                               sp<Cand>(g.s_buf3), sp<Cand>(g.s_buf), misc_hist(g), misc_cnt(g), st,
                               &ns, &t_stats.launches);
  if (e != cudaSuccess) return e;
  std::swap(g.s_buf, g.s_buf2);  // s_buf = the selected entries
  const bool inexact = measure == LP_SC || measure == LP_LHN;
  if (sorted || inexact) {
    Cand* res = nullptr;
    e = launch_sort_cands(sp<Cand>(g.s_buf), sp<Cand>(g.s_buf2), sp<int>(g.s_grp), ns, st, &res,
                          &t_stats.launches);
    if (e != cudaSuccess) return e;
    if (res != sp<Cand>(g.s_buf)) std::swap(g.s_buf, g.s_buf2);
  }
  *n_out = ns;
  return cudaSuccess;
}

static lp_status predict_global(Graph& g, int measure, int cap, int64_t k, double threshold,
                                lp_link* out, bool out_dev, int64_t out_cap, int64_t* out_n,
                                int src_begin, int src_end) {
  begin_stats();
  *out_n = 0;
  if (measure < 0 || measure > LP_RA) return fail(LP_EINVAL, "lp_predict: bad measure");
  if (k < 0) return fail(LP_EINVAL, "lp_predict: k < 0");
  if (out_cap < 0 || (out_cap > 0 && !out)) return fail(LP_EINVAL, "lp_predict: bad output buffer");
  if (src_begin < 0 || src_end < src_begin || src_end > g.n)
    return fail(LP_EINVAL, "lp_predict: source range [%d, %d) outside [0, %d)", src_begin, src_end,
                g.n);
  {
    const lp_status s = accuracy_guard(g, measure, cap, "lp_predict");
    if (s != LP_OK) return s;
  }
  if (src_end == src_begin || cap == 0) return LP_OK;
  std::lock_guard<std::mutex> lock(g.mu);
  CU(cudaSetDevice(g.device));
  cudaStream_t st = g.stream;
  Timer tm(g);
  tm.mark(0);
  ScanArgs A = base_args(g, measure, cap, threshold, 0, 0);
  A.rec_base = src_begin;
  CU(attach_cursors(g, A));
  const Options opt = options_snapshot();
  // the expand-and-count tier pays off where the index array does not stay
  // in the L2 cache (window sweeps then pay DRAM round trips per arc)
  A.expand = opt.expand == 1 || (opt.expand == 2 && g.arcs * (int64_t)sizeof(int) > (128ll << 20));
  // the count pass's 64 KB table holds 8192 slots of 32-bit values, 4096 of 64-bit
  A.x_logcap = std::min(opt.expand_logcap, (measure == LP_AA || measure == LP_RA) ? 12 : 13);
  A.x_min = std::max(opt.expand_min, A.med_max);
  // selection buffer
  const u64 minbuf = (u64)std::max<long long>(16, options_snapshot().select_buffer);
  u64 C = k > 0 ? std::max<u64>(minbuf, 2ull * (u64)k + std::min<u64>(minbuf, 1ull << 20)) : minbuf;
  const u64 failed_cap = 1 << 20, split_cap = 1 << 20;
  CU(ensure(g, g.s_ctr, sizeof(Counters)));
  CU(ensure(g, g.s_thresh, sizeof(Thresh)));
  CU(ensure(g, g.s_vfloor, sizeof(u64) * ((size_t)g.dmax + 1)));
  CU(ensure(g, g.s_buf, sizeof(Cand) * C));
  CU(ensure(g, g.s_buf2, sizeof(Cand) * C));
  CU(ensure(g, g.s_buf3, sizeof(Cand) * C));
  CU(ensure(g, g.s_misc, kMiscBytes));
  CU(ensure(g, g.s_failed, sizeof(int4) * failed_cap));
  CU(ensure(g, g.s_split, sizeof(int4) * split_cap));
  CU(ensure(g, g.s_flags, (size_t)g.n + 1));
  CU(ensure(g, g.s_grp, sizeof(int) * sort_splits_needed(C)));
  Counters* d_ctr = sp<Counters>(g.s_ctr);
  Thresh* d_th = sp<Thresh>(g.s_thresh);
  CU(cudaMemsetAsync(d_th, 0, sizeof(Thresh), st));
  CU(cudaMemsetAsync(g.s_flags.p, 0, (size_t)g.n + 1, st));
  Counters h{};
  lp_status s = run_estimate(g, A, src_end - src_begin, nullptr, h);
  if (s != LP_OK) return s;
  ExpState X;
  if (h.nexp) {
    s = exp_setup(g, A, h.nexp, opt.expand_batch, tm.on, X);
    if (s != LP_OK) return s;
    t_stats.launches += X.launches;
    X.launches = 0;
  }
  tm.mark(1);

  Queues Q = {{&g.s_warpq, &g.s_medq, &g.s_itemq, &g.s_countq},
              {&g.s_warpq2, &g.s_medq2, &g.s_itemq2, &g.s_countq2},
              {h.nwarp, h.nmed, h.nitem, 0}};
  u64 kept = 0;  // valid entries at the start of the buffer
  std::vector<int4> failed, splits, xitems;
  std::vector<int4> heads[4];
  for (int round = 0; Q.n[0] + Q.n[1] + Q.n[2] + Q.n[3] > 0 || X.next < X.batches.size();
       ++round) {
    if (round > 100000) return fail(LP_EINTERNAL, "lp_predict: no progress");
    // first round: the small tiers and an eighth of the large tier (items
    // in source order, a sample of the sources), so that the threshold they
    // set (a compaction below) already filters the rest of the large tier
    // and every batch of the expand-and-count tier
    const bool seed = round == 0 && k > 0 && (Q.n[2] >= 64 || !X.batches.empty());
    const u64 large_n = seed && Q.n[2] >= 64 ? Q.n[2] / 8 : Q.n[2];
    if (!seed && Q.n[3] == 0 && X.next < X.batches.size()) {
      // the previous batch's items are all done: expand the next one
      s = exp_next_batch(g, A, X, tm.on, xitems);
      if (s != LP_OK) return s;
      t_stats.launches += X.launches;
      X.launches = 0;
      CU(build_queue(g, *Q.cur[3], xitems, nullptr, 0, 0, &Q.n[3]));
    }
    Counters z{};
    z.cand_cnt = kept;
    CU(cudaMemcpyAsync(d_ctr, &z, sizeof(Counters), cudaMemcpyHostToDevice, st));
    A.ctr = d_ctr;
    A.buf = sp<Cand>(g.s_buf);
    A.buf_cap = C;
    A.thresh = d_th;
    A.vfloor = sp<u64>(g.s_vfloor);
    A.failed = sp<int4>(g.s_failed);
    A.failed_cap = failed_cap;
    A.split = sp<int4>(g.s_split);
    A.split_cap = split_cap;
    A.prof = opt.phase_profile ? d_ctr->prof : nullptr;
    CU(scan_launches(g, A, Q, tm.on, large_n));
    CU(cudaMemcpyAsync(&h, d_ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    scan_times(g, Q, tm.on);
    for (int i = 0; i < 6; ++i) t_stats.phase_cycles[i] += (int64_t)h.prof[i];
    if (h.error) return fail(LP_EINTERNAL, "lp_predict: device check %u", h.error);
    t_stats.candidates += (int64_t)h.candidates;
    failed.resize(h.nfailed);
    splits.resize(h.nsplit);
    if (h.nfailed)
      CU(cudaMemcpy(failed.data(), g.s_failed.p, sizeof(int4) * h.nfailed, cudaMemcpyDeviceToHost));
    if (h.nsplit)
      CU(cudaMemcpy(splits.data(), g.s_split.p, sizeof(int4) * h.nsplit, cudaMemcpyDeviceToHost));
    const u64 done[4] = {std::min<u64>(h.claim_w, Q.n[0]), std::min<u64>(h.claim_m, Q.n[1]),
                         std::min<u64>(h.claim_c, large_n), std::min<u64>(h.claim_x, Q.n[3])};
    t_stats.exp_items += (int64_t)done[3];
    const u64 valid = std::min<u64>(h.cand_cnt, C);
    t_stats.splits += (int32_t)h.nsplit;
    if (h.full || (seed && valid >= (u64)k)) {
      // compaction: drop failed output, then sort and cut to k
      t_stats.compactions++;
      Cand* src = sp<Cand>(g.s_buf);
      u64 m = valid;
      if (!failed.empty()) {
        std::vector<int4> fs(failed);
        std::sort(fs.begin(), fs.end(), [](const int4& x, const int4& y) {
          return x.x != y.x ? x.x < y.x : x.y < y.y;
        });
        CU(cudaMemcpyAsync(g.s_split.p, fs.data(), sizeof(int4) * fs.size(), cudaMemcpyHostToDevice,
                           st));
        const int nf = (int)fs.size();
        k_set_flags<<<(nf + 255) / 256, 256, 0, st>>>(sp<int4>(g.s_split), nf,
                                                      sp<unsigned char>(g.s_flags), 1);
        u64* d_cnt = &d_ctr->pad[0];
        CU(cudaMemsetAsync(d_cnt, 0, sizeof(u64), st));
        CU(launch_filter_failed(src, valid, sp<unsigned char>(g.s_flags), sp<int4>(g.s_split), nf,
                                sp<Cand>(g.s_buf2), d_ctr, d_cnt, st));
        k_set_flags<<<(nf + 255) / 256, 256, 0, st>>>(sp<int4>(g.s_split), nf,
                                                      sp<unsigned char>(g.s_flags), 0);
        t_stats.launches += 3;
        CU(cudaMemcpyAsync(&m, d_cnt, sizeof(u64), cudaMemcpyDeviceToHost, st));
        CU(cudaStreamSynchronize(st));
        std::swap(g.s_buf, g.s_buf2);
        src = sp<Cand>(g.s_buf);
      }
      if (k > 0 && m >= (u64)k) {
        u64 kk = 0;
        CU(select_best(g, measure, m, (u64)k, &kk, /*sorted=*/false));
        // s_buf now holds the best k (exact measures: unordered, the worst of
        // them is the threshold; SC / LHN: sorted, entry k-1 is)
        if (measure == LP_SC || measure == LP_LHN) CU(launch_set_thresh(sp<Cand>(g.s_buf), (u64)k, d_th, st));
        else CU(launch_thresh_worst(sp<Cand>(g.s_buf), (u64)k, misc_worst(g), d_th, st, &t_stats.launches));
        CU(launch_count_floor(measure, g.dmax, d_th, sp<u64>(g.s_vfloor), st));
        t_stats.launches += 1;
        kept = (u64)k;
      } else {
        kept = m;
      }
      // guarantee room for progress
      const bool progress = (done[0] + done[1] + done[2] + done[3]) > h.nfailed;
      if (k == 0 || !progress || C - kept < (C >> 2)) {
        const u64 C2 = C * 2;
        CU(ensure(g, g.s_buf2, sizeof(Cand) * C2));
        CU(cudaMemcpyAsync(g.s_buf2.p, g.s_buf.p, sizeof(Cand) * kept, cudaMemcpyDeviceToDevice, st));
        CU(cudaStreamSynchronize(st));
        std::swap(g.s_buf, g.s_buf2);
        CU(ensure(g, g.s_buf2, sizeof(Cand) * C2));
        CU(ensure(g, g.s_buf3, sizeof(Cand) * C2));
        CU(ensure(g, g.s_grp, sizeof(int) * sort_splits_needed(C2)));
        C = C2;
      }
    } else {
      kept = valid;
    }
    for (auto& hd : heads) hd.clear();
    for (const int4& r : failed) heads[record_tier(r)].push_back(r);
    for (const int4& r : splits) {
      if (r.w & kExpItem) split_count_item(r, heads[3]);
      else split_item(r, A.big_span, heads[2]);
    }
    CU(rebuild_queues(g, Q, heads, done));
  }
  t_stats.tier_ms[3] += X.ms_expand;
  t_stats.ms_expand = X.ms_expand;
  t_stats.exp_units = (int32_t)X.units.size();
  t_stats.exp_batches = (int32_t)X.batches.size();
  for (const ExpUnit& U : X.units) t_stats.exp_dense_units += (U.flags & kExpDense) ? 1 : 0;
  tm.mark(2);
  // final selection: the best k, sorted
  u64 nsorted = kept;
  if (k > 0 && kept > (u64)k) CU(select_best(g, measure, kept, (u64)k, &nsorted, /*sorted=*/true));
  Cand* res = sp<Cand>(g.s_buf);
  if (!(k > 0 && kept > (u64)k)) {
    CU(launch_sort_cands(res, sp<Cand>(g.s_buf2), sp<int>(g.s_grp), kept, st, &res,
                         &t_stats.launches));
  }
  const u64 found = k > 0 ? std::min<u64>(kept, (u64)k) : kept;
  *out_n = (int64_t)found;
  t_stats.admitted = (int64_t)kept;
  const u64 nwrite = std::min<u64>(found, (u64)out_cap);
  lp_link* d_links = nullptr;
  if (out_dev) {
    d_links = out;
  } else {
    CU(ensure(g, g.s_links, sizeof(lp_link) * (nwrite + 1)));
    d_links = sp<lp_link>(g.s_links);
  }
  if (nwrite) {
    CU(launch_emit_global(res, nwrite, measure, g.fixbits, d_links, st));
    t_stats.launches++;
    if (measure == LP_AA || measure == LP_RA) {
      // grouped by the endpoint of larger degree: the top pairs share
      // high-degree endpoints, whose lists are then read once per group
      CU(ensure(g, g.s_pair, pair_groups_scratch(g.n, nwrite, A.cap < g.dmax ? g.arcs : 0)));
      CU(launch_pair_cn_groups(d_links, nwrite, g.n, g.d_off, g.d_idx, g.d_deg, g.arcs, g.dmax,
                               A.cap, g.s_pair.p, st, &t_stats.launches));
    }
    if (!out_dev)
      CU(cudaMemcpyAsync(out, d_links, sizeof(lp_link) * nwrite, cudaMemcpyDeviceToHost, st));
  }
  tm.mark(3);
  CU(cudaStreamSynchronize(st));
  t_stats.ms_estimate = tm.ms(0, 1);
  t_stats.ms_scan = tm.ms(1, 2);
  t_stats.ms_select = tm.ms(2, 3);
  t_stats.ms_total = tm.ms(0, 3);
  if (found > (u64)out_cap)
    return fail(LP_ETRUNC, "lp_predict: %lld links found, room for %lld", (long long)found,
                (long long)out_cap);
  return LP_OK;
}

// ------------------------------------------------------------- merging --

// The best k of a set of global-mode links under the total order, with the
// exact keys of the selection (Section 4.1.7: the merge of lists that
// independent groups of sources produced).  Count measures take the key from
// each link's common-neighbour count and the degrees; AA and RA rebuild their
// fixed-point sums from the graph, so the result equals, bit for bit, what
// one lp_predict call over all the sources returns.
static lp_status merge_links(Graph& g, int measure, int cap, const lp_link* links, int64_t n_links,
                             int64_t k, lp_link* out, int64_t out_cap, int64_t* out_n) {
  begin_stats();
  *out_n = 0;
  if (measure < 0 || measure > LP_RA) return fail(LP_EINVAL, "lp_merge_links: bad measure");
  if (k < 0 || n_links < 0) return fail(LP_EINVAL, "lp_merge_links: negative k or link count");
  if (n_links > 0 && !links) return fail(LP_EINVAL, "lp_merge_links: null links");
  if (out_cap < 0 || (out_cap > 0 && !out))
    return fail(LP_EINVAL, "lp_merge_links: bad output buffer");
  for (int64_t i = 0; i < n_links; ++i)
    if (links[i].u < 0 || links[i].u >= links[i].v || links[i].v >= g.n || links[i].cn < 0)
      return fail(LP_EINVAL, "lp_merge_links: link %lld is not a pair u < v of the graph",
                  (long long)i);
  {
    const lp_status s = accuracy_guard(g, measure, cap, "lp_merge_links");
    if (s != LP_OK) return s;
  }
  if (n_links == 0) return LP_OK;
  std::lock_guard<std::mutex> lock(g.mu);
  CU(cudaSetDevice(g.device));
  cudaStream_t st = g.stream;
  const ScanArgs A = base_args(g, measure, cap, 0.0, 0, 0);
  const u64 n = (u64)n_links;
  CU(ensure(g, g.s_links, sizeof(lp_link) * n));
  CU(ensure(g, g.s_buf, sizeof(Cand) * n));
  CU(ensure(g, g.s_buf2, sizeof(Cand) * n));
  CU(ensure(g, g.s_buf3, sizeof(Cand) * n));
  CU(ensure(g, g.s_misc, kMiscBytes));
  CU(ensure(g, g.s_grp, sizeof(int) * sort_splits_needed(n)));
  CU(cudaMemcpyAsync(g.s_links.p, links, sizeof(lp_link) * n, cudaMemcpyHostToDevice, st));
  CU(launch_link_keys(sp<lp_link>(g.s_links), n, measure, g.d_off, g.d_idx, g.d_deg, g.d_arc,
                      A.cap, A.wt, sp<Cand>(g.s_buf), st));
  t_stats.launches++;
  u64 nsorted = n;
  Cand* res = sp<Cand>(g.s_buf);
  if (k > 0 && n > (u64)k) {
    CU(select_best(g, measure, n, (u64)k, &nsorted, /*sorted=*/true));
    res = sp<Cand>(g.s_buf);
  } else {
    CU(launch_sort_cands(res, sp<Cand>(g.s_buf2), sp<int>(g.s_grp), n, st, &res,
                         &t_stats.launches));
  }
  const u64 found = k > 0 ? std::min<u64>(n, (u64)k) : n;
  *out_n = (int64_t)found;
  const u64 nwrite = std::min<u64>(found, (u64)out_cap);
  if (nwrite) {
    lp_link* d_links = sp<lp_link>(g.s_links);  // the input copy is no longer needed
    CU(launch_emit_global(res, nwrite, measure, g.fixbits, d_links, st));
    t_stats.launches++;
    if (measure == LP_AA || measure == LP_RA) {
      CU(ensure(g, g.s_pair, pair_groups_scratch(g.n, nwrite, A.cap < g.dmax ? g.arcs : 0)));
      CU(launch_pair_cn_groups(d_links, nwrite, g.n, g.d_off, g.d_idx, g.d_deg, g.arcs, g.dmax,
                               A.cap, g.s_pair.p, st, &t_stats.launches));
    }
    CU(cudaMemcpyAsync(out, d_links, sizeof(lp_link) * nwrite, cudaMemcpyDeviceToHost, st));
  }
  CU(cudaStreamSynchronize(st));
  if (found > (u64)out_cap)
    return fail(LP_ETRUNC, "lp_merge_links: %lld links found, room for %lld", (long long)found,
                (long long)out_cap);
  return LP_OK;
}

// ------------------------------------------------------- per-source mode --

static lp_status predict_sources(Graph& g, int measure, int cap, const int* d_src, int n_src, int k,
                                 double threshold, lp_link* d_out, int* d_counts) {
  if (n_src == 0) return LP_OK;
  {
    const lp_status s = accuracy_guard(g, measure, cap, "lp_predict_sources");
    if (s != LP_OK) return s;
  }
  cudaStream_t st = g.stream;
  Timer tm(g);
  tm.mark(0);
  // reject out-of-range sources before any kernel reads them
  CU(ensure(g, g.s_ctr, sizeof(Counters)));
  Counters* d_ctr = sp<Counters>(g.s_ctr);
  {
    int* d_bad = reinterpret_cast<int*>(&d_ctr->error);
    int bad = 0;
    CU(cudaMemsetAsync(d_bad, 0, sizeof(int), st));
    k_check_sources<<<(n_src + 255) / 256, 256, 0, st>>>(d_src, n_src, g.n, d_bad);
    CU(cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    if (bad) return fail(LP_EINVAL, "lp_predict_sources: source id out of range");
  }
  CU(cudaMemsetAsync(d_counts, 0, sizeof(int) * (size_t)n_src, st));
  if (cap == 0 || g.n == 0) {  // nothing to predict: rows of fillers
    CU(launch_emit_sources(nullptr, d_counts, d_src, n_src, k, measure, g.fixbits, d_out, st));
    CU(cudaStreamSynchronize(st));
    return LP_OK;
  }
  ScanArgs A = base_args(g, measure, cap, threshold, 1, k);
  A.sources = d_src;
  CU(attach_cursors(g, A));
  CU(ensure(g, g.s_top, sizeof(TopEnt) * (size_t)n_src * k));
  CU(ensure(g, g.s_grp, sizeof(int2) * ((size_t)n_src + 1)));
  CU(ensure(g, g.s_split, sizeof(int4) * (1 << 20)));
  A.out_top = sp<TopEnt>(g.s_top);
  A.out_cnt = d_counts;
  Counters h{};
  lp_status s = run_estimate(g, A, n_src, sp<int2>(g.s_grp), h);
  if (s != LP_OK) return s;
  tm.mark(1);
  // partial lists: one per non-single item, including split halves
  u64 partial_cap = h.nitem + 16;
  CU(ensure(g, g.s_partial, sizeof(TopEnt) * partial_cap * k));
  CU(ensure(g, g.s_phdr, sizeof(int2) * partial_cap));
  // (the expand-and-count tier is global-mode only: its queue stays empty)
  Queues Q = {{&g.s_warpq, &g.s_medq, &g.s_itemq, &g.s_countq},
              {&g.s_warpq2, &g.s_medq2, &g.s_itemq2, &g.s_countq2},
              {h.nwarp, h.nmed, h.nitem, 0}};
  u64 npartial = 0;
  std::vector<int4> splits;
  std::vector<int4> heads[4];
  for (int round = 0; Q.n[0] + Q.n[1] + Q.n[2] > 0; ++round) {
    if (round > 10000) return fail(LP_EINTERNAL, "lp_predict_sources: no progress");
    Counters z{};
    z.npartial = npartial;
    CU(cudaMemcpyAsync(d_ctr, &z, sizeof(Counters), cudaMemcpyHostToDevice, st));
    A.ctr = d_ctr;
    A.split = sp<int4>(g.s_split);
    A.split_cap = 1 << 20;
    A.partial = sp<TopEnt>(g.s_partial);
    A.partial_hdr = sp<int2>(g.s_phdr);
    A.partial_cap = partial_cap;
    A.prof = options_snapshot().phase_profile ? d_ctr->prof : nullptr;
    CU(scan_launches(g, A, Q, tm.on));
    CU(cudaMemcpyAsync(&h, d_ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    scan_times(g, Q, tm.on);
    for (int i = 0; i < 6; ++i) t_stats.phase_cycles[i] += (int64_t)h.prof[i];
    if (h.error) return fail(LP_EINTERNAL, "lp_predict_sources: device check %u", h.error);
    t_stats.candidates += (int64_t)h.candidates;
    t_stats.splits += (int32_t)h.nsplit;
    npartial = h.npartial;
    splits.resize(h.nsplit);
    if (h.nsplit)
      CU(cudaMemcpy(splits.data(), g.s_split.p, sizeof(int4) * h.nsplit, cudaMemcpyDeviceToHost));
    for (auto& hd : heads) hd.clear();
    for (const int4& r : splits) split_item(r, A.big_span, heads[2]);
    for (int4& r : heads[2]) r.w &= ~kItemSingle;
    const u64 done[4] = {Q.n[0], Q.n[1], Q.n[2], 0};  // no buffer: everything claimed ran
    CU(rebuild_queues(g, Q, heads, done));
    if (npartial + Q.n[2] + 16 > partial_cap) {
      // grow the partial store, keeping what is there
      const u64 cap2 = (npartial + Q.n[2]) * 2 + 16;
      Graph::Scratch np, nh;
      CU(cudaMalloc(&np.p, sizeof(TopEnt) * cap2 * k));
      np.bytes = sizeof(TopEnt) * cap2 * k;
      CU(cudaMalloc(&nh.p, sizeof(int2) * cap2));
      nh.bytes = sizeof(int2) * cap2;
      CU(cudaMemcpyAsync(np.p, g.s_partial.p, sizeof(TopEnt) * npartial * k,
                         cudaMemcpyDeviceToDevice, st));
      CU(cudaMemcpyAsync(nh.p, g.s_phdr.p, sizeof(int2) * npartial, cudaMemcpyDeviceToDevice, st));
      CU(cudaStreamSynchronize(st));
      cudaFree(g.s_partial.p);
      cudaFree(g.s_phdr.p);
      g.s_partial = np;
      g.s_phdr = nh;
      partial_cap = cap2;
    }
  }
  tm.mark(2);
  // merge the partial lists of split sources
  if (npartial) {
    std::vector<int2> hdr(npartial);
    CU(cudaMemcpy(hdr.data(), g.s_phdr.p, sizeof(int2) * npartial, cudaMemcpyDeviceToHost));
    std::vector<int> order(npartial);
    for (u64 i = 0; i < npartial; ++i) order[i] = (int)i;
    std::sort(order.begin(), order.end(),
              [&](int x, int y) { return hdr[x].x != hdr[y].x ? hdr[x].x < hdr[y].x : x < y; });
    std::vector<int4> grp;
    for (u64 i = 0; i < npartial;) {
      u64 j = i;
      while (j < npartial && hdr[order[j]].x == hdr[order[i]].x) ++j;
      grp.push_back(make_int4(hdr[order[i]].x, (int)i, (int)(j - i), 0));
      i = j;
    }
    Graph::Scratch& tmp = g.s_failed;
    const size_t need = sizeof(int4) * grp.size() + sizeof(int) * order.size() + 64;
    CU(ensure(g, tmp, need));
    int4* d_grp = sp<int4>(tmp);
    int* d_order = reinterpret_cast<int*>(d_grp + grp.size());
    CU(cudaMemcpyAsync(d_grp, grp.data(), sizeof(int4) * grp.size(), cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(d_order, order.data(), sizeof(int) * order.size(), cudaMemcpyHostToDevice, st));
    CU(launch_merge_partials(d_grp, (int)grp.size(), d_order, sp<TopEnt>(g.s_partial),
                             sp<int2>(g.s_phdr), k, sp<TopEnt>(g.s_top), d_counts, st));
    t_stats.launches++;
    CU(cudaStreamSynchronize(st));
  }
  CU(launch_emit_sources(sp<TopEnt>(g.s_top), d_counts, d_src, n_src, k, measure, g.fixbits, d_out,
                         st));
  t_stats.launches++;
  if (measure == LP_AA || measure == LP_RA) {
    CU(launch_pair_cn(d_out, d_counts, k, (u64)n_src * k, g.d_off, g.d_idx, g.d_deg, g.d_arc, A.cap, st));
    t_stats.launches++;
  }
  tm.mark(3);
  CU(cudaStreamSynchronize(st));
  t_stats.ms_estimate = tm.ms(0, 1);
  t_stats.ms_scan = tm.ms(1, 2);
  t_stats.ms_select = tm.ms(2, 3);
  t_stats.ms_total = tm.ms(0, 3);
  return LP_OK;
}

static lp_status check_sources_args(const lp_graph* g, int measure, const void* sources, int n_src,
                                    int k, const void* out, const void* counts) {
  if (!g) return fail(LP_EINVAL, "lp_predict_sources: null graph");
  if (measure < 0 || measure > LP_RA) return fail(LP_EINVAL, "lp_predict_sources: bad measure");
  if (n_src < 0) return fail(LP_EINVAL, "lp_predict_sources: n_src < 0");
  if (k < 1 || k > LP_MAX_TOPK_PER_SOURCE)
    return fail(LP_EINVAL, "lp_predict_sources: k must be in [1, %d]", LP_MAX_TOPK_PER_SOURCE);
  if (n_src > 0 && (!sources || !out || !counts))
    return fail(LP_EINVAL, "lp_predict_sources: null buffer");
  return LP_OK;
}

// Entry points for other translation units of the library (thin wrappers).
lp_status report_error(lp_status s, const char* msg) { return fail(s, "%s", msg); }
lp_status report_cuda(cudaError_t e, const char* what) { return cuda_fail(e, what); }
void stats_begin() { begin_stats(); }
void stats_estimate(const Counters& h) { estimate_stats(h); }
void stats_add(int64_t candidates, int32_t splits, int32_t launches) {
  t_stats.candidates += candidates;
  t_stats.splits += splits;
  t_stats.launches += launches;
}
ScanArgs scan_args(Graph& g, int measure, int cap, double threshold, int mode, int k) {
  return base_args(g, measure, cap, threshold, mode, k);
}
lp_status sources_args_ok(const lp_graph* g, int measure, const void* sources, int n_src, int k,
                          const void* out, const void* counts) {
  return check_sources_args(g, measure, sources, n_src, k, out, counts);
}
Graph& graph_of(const lp_graph* g) { return *const_cast<lp_graph*>(g); }

lp_status make_shadow(const Graph& g, Graph** out) {
  lp_graph* s = new (std::nothrow) lp_graph();
  if (!s) return fail(LP_ENOMEM, "shadow graph: host allocation");
  s->owns_arrays = false;
  s->device = g.device;
  s->n = g.n;
  s->arcs = g.arcs;
  s->dmax = g.dmax;
  s->fixbits = g.fixbits;
  s->d_off = g.d_off;
  s->d_idx = g.d_idx;
  s->d_deg = g.d_deg;
  s->d_arc = g.d_arc;
  s->d_wt = g.d_wt;
  cudaError_t e = cudaSetDevice(g.device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
  for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaEventCreate(&s->ev[i]);
  for (int i = 0; i < 8 && e == cudaSuccess; ++i) e = cudaEventCreate(&s->kev[i]);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaEventCreate(&s->xev[i]);
  if (e != cudaSuccess) {
    free_graph(s);
    return cuda_fail(e, "shadow graph");
  }
  *out = s;
  return LP_OK;
}

void destroy_shadow(Graph* s) { free_graph(s); }

lp_status run_sources_dev(Graph& g, int measure, int cap, const int* d_src, int n_src, int k,
                          double threshold, lp_link* d_out, int* d_counts) {
  std::lock_guard<std::mutex> lock(g.mu);
  cudaError_t e = cudaSetDevice(g.device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  return predict_sources(g, measure, cap, d_src, n_src, k, threshold, d_out, d_counts);
}

}  // namespace lp

extern "C" {

lp_status lp_predict(const lp_graph* g, lp_measure measure, int32_t degree_cap, int64_t k,
                     double threshold, lp_link* out, int64_t out_cap, int64_t* out_n) {
  if (!g || !out_n) return lp::fail(LP_EINVAL, "lp_predict: null argument");
  return lp::predict_global(*const_cast<lp_graph*>(g), (int)measure, degree_cap, k, threshold, out,
                            false, out_cap, out_n, 0, g->n);
}

lp_status lp_predict_range(const lp_graph* g, lp_measure measure, int32_t degree_cap, int64_t k,
                           double threshold, int32_t src_begin, int32_t src_end, lp_link* out,
                           int64_t out_cap, int64_t* out_n) {
  if (!g || !out_n) return lp::fail(LP_EINVAL, "lp_predict_range: null argument");
  return lp::predict_global(*const_cast<lp_graph*>(g), (int)measure, degree_cap, k, threshold, out,
                            false, out_cap, out_n, src_begin, src_end);
}

lp_status lp_merge_links(const lp_graph* g, lp_measure measure, int32_t degree_cap,
                         const lp_link* links, int64_t n_links, int64_t k, lp_link* out,
                         int64_t out_cap, int64_t* out_n) {
  if (!g || !out_n) return lp::fail(LP_EINVAL, "lp_merge_links: null argument");
  return lp::merge_links(*const_cast<lp_graph*>(g), (int)measure, degree_cap, links, n_links, k,
                         out, out_cap, out_n);
}

lp_status lp_predict_dev(const lp_graph* g, lp_measure measure, int32_t degree_cap, int64_t k,
                         double threshold, lp_link* d_out, int64_t out_cap, int64_t* out_n) {
  if (!g || !out_n) return lp::fail(LP_EINVAL, "lp_predict_dev: null argument");
  return lp::predict_global(*const_cast<lp_graph*>(g), (int)measure, degree_cap, k, threshold,
                            d_out, true, out_cap, out_n, 0, g->n);
}

lp_status lp_predict_sources_dev(const lp_graph* g, lp_measure measure, int32_t degree_cap,
                                 const int32_t* d_sources, int32_t n_src, int32_t k,
                                 double threshold, lp_link* d_out, int32_t* d_counts) {
  lp::begin_stats();
  lp_status s = lp::check_sources_args(g, (int)measure, d_sources, n_src, k, d_out, d_counts);
  if (s != LP_OK) return s;
  lp::Graph& gg = *const_cast<lp_graph*>(g);
  std::lock_guard<std::mutex> lock(gg.mu);
  cudaError_t e = cudaSetDevice(gg.device);
  if (e != cudaSuccess) return lp::cuda_fail(e, "cudaSetDevice");
  return lp::predict_sources(gg, (int)measure, degree_cap, d_sources, n_src, k, threshold, d_out,
                             d_counts);
}

lp_status lp_predict_sources(const lp_graph* g, lp_measure measure, int32_t degree_cap,
                             const int32_t* sources, int32_t n_src, int32_t k, double threshold,
                             lp_link* out, int32_t* counts) {
  lp::begin_stats();
  lp_status s = lp::check_sources_args(g, (int)measure, sources, n_src, k, out, counts);
  if (s != LP_OK) return s;
  if (n_src == 0) return LP_OK;
  for (int32_t i = 0; i < n_src; ++i)
    if (sources[i] < 0 || sources[i] >= g->n)
      return lp::fail(LP_EINVAL, "lp_predict_sources: source %d out of range", sources[i]);
  lp::Graph& gg = *const_cast<lp_graph*>(g);
  std::lock_guard<std::mutex> lock(gg.mu);
  cudaError_t e = cudaSetDevice(gg.device);
  if (e != cudaSuccess) return lp::cuda_fail(e, "cudaSetDevice");
  const size_t nl = (size_t)n_src * k;
  e = lp::ensure(gg, gg.s_src, sizeof(int) * n_src);
  if (e == cudaSuccess) e = lp::ensure(gg, gg.s_links, sizeof(lp_link) * nl);
  if (e == cudaSuccess) e = lp::ensure(gg, gg.s_cnt, sizeof(int) * n_src);
  if (e != cudaSuccess) return lp::cuda_fail(e, "lp_predict_sources: scratch");
  e = cudaMemcpyAsync(gg.s_src.p, sources, sizeof(int) * n_src, cudaMemcpyHostToDevice, gg.stream);
  if (e != cudaSuccess) return lp::cuda_fail(e, "lp_predict_sources: upload");
  s = lp::predict_sources(gg, (int)measure, degree_cap, lp::sp<int>(gg.s_src), n_src, k, threshold,
                          lp::sp<lp_link>(gg.s_links), lp::sp<int>(gg.s_cnt));
  if (s != LP_OK) return s;
  e = cudaMemcpyAsync(out, gg.s_links.p, sizeof(lp_link) * nl, cudaMemcpyDeviceToHost, gg.stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(counts, gg.s_cnt.p, sizeof(int) * n_src, cudaMemcpyDeviceToHost, gg.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(gg.stream);
  if (e != cudaSuccess) return lp::cuda_fail(e, "lp_predict_sources: download");
  return LP_OK;
}

}  // extern "C"
