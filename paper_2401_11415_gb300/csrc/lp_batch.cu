// lp_batch.cu -- batched multi-graph mode: many graphs, one recorded launch
// sequence, autotuned binning.
//
// The graphs of a batch are packed into one block-diagonal graph: graph i's
// vertex v becomes bases[i] + v.  Two-hop neighbourhoods never cross blocks,
// so the per-source top-k of every packed vertex is the per-source top-k of
// every vertex of every graph (Section 4.1.7: sources are independent), and
// one set of scan launches serves all graphs of uneven sizes at once.
//
// A query (measure, hub limit, k) is planned once: the work estimate bins
// every source, large sources become dense items (they cannot overflow, so no
// host round trip is needed), items of a split source write their partial
// lists to a slot fixed by their queue position, and the merge of those lists
// is set up from the estimate.  The scan, merge and emit launches are then
// recorded in a CUDA graph and every later call replays it.  The autotuner
// times replays of plans built with other binning options (tier limits, item
// size, large-tier CTA shape) and keeps the fastest.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "lp_internal.cuh"

namespace lp {

namespace {

__global__ void k_iota(int* __restrict__ a, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) a[i] = i;
}

struct AllPlan {
  bool ready = false;
  bool dense_only = false;  // set after a replay saw a split hash item overflow
  int measure = -1, cap = 0, k = 0;
  Options opt;
  lp_link* d_out = nullptr;
  int* d_counts = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  Graph::Scratch src, warpq, medq, itemq, grp, ctr, top, partial, phdr, mgrp, morder, split;
  u64 nwarp = 0, nmed = 0, nitem = 0;
  int nmulti = 0;

  void drop_graph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
    ready = false;
  }
  void release() {
    drop_graph();
    Graph::Scratch* all[] = {&src, &warpq, &medq, &itemq, &grp, &ctr, &top,
                             &partial, &phdr, &mgrp, &morder, &split};
    for (auto* s : all) {
      if (s->p) cudaFree(s->p);
      s->p = nullptr;
      s->bytes = 0;
    }
  }
};

bool same_options(const Options& a, const Options& b) {
  return a.warp_max == b.warp_max && a.med_max == b.med_max && a.cta_max == b.cta_max &&
         a.split_target == b.split_target && a.split_logcap == b.split_logcap &&
         a.item_wedges == b.item_wedges && a.big_threads == b.big_threads;
}

#define BU(x)                                                \
  do {                                                       \
    cudaError_t e_ = (x);                                    \
    if (e_ != cudaSuccess) return lp::report_cuda(e_, #x);   \
  } while (0)

// Estimate, bin and record the per-source query of every vertex of g.
lp_status build_plan(Graph& g, AllPlan& P, int measure, int cap, int k, const Options& opt,
                     lp_link* d_out, int* d_counts) {
  {
    const lp_status s = accuracy_guard(g, measure, cap, "batched query");
    if (s != LP_OK) return s;
  }
  P.drop_graph();
  cudaStream_t st = g.stream;
  const int n = g.n;
  ScanArgs A = base_args_opts(g, measure, cap, 0.0, 1, k, opt);
  BU(attach_cursors(g, A));
  A.no_split = P.dense_only ? 1 : 0;
  A.partial_by_item = 1;
  BU(ensure(g, P.src, sizeof(int) * ((size_t)n + 1)));
  BU(ensure(g, P.warpq, sizeof(int4) * ((size_t)n + 1)));
  BU(ensure(g, P.medq, sizeof(int4) * ((size_t)n + 1)));
  BU(ensure(g, P.grp, sizeof(int2) * ((size_t)n + 1)));
  BU(ensure(g, P.ctr, sizeof(Counters)));
  BU(ensure(g, P.top, sizeof(TopEnt) * ((size_t)n * k + 1)));
  BU(ensure(g, P.split, sizeof(int4) * 1024));
  if (n > 0) {
    k_iota<<<std::min(1024, (n + 255) / 256), 256, 0, st>>>(sp<int>(P.src), n);
    BU(cudaGetLastError());
  }
  A.sources = sp<int>(P.src);
  A.out_top = sp<TopEnt>(P.top);
  A.out_cnt = d_counts;
  A.ctr = sp<Counters>(P.ctr);
  A.split = sp<int4>(P.split);
  A.split_cap = 1024;
  u64 itemq_cap = std::max<u64>(1024, P.itemq.bytes / sizeof(int4));
  BU(ensure(g, P.itemq, sizeof(int4) * itemq_cap));
  Counters h{};
  for (int attempt = 0; attempt < 3; ++attempt) {
    BU(cudaMemsetAsync(P.ctr.p, 0, sizeof(Counters), st));
    BU(launch_estimate2(A, n, sp<int4>(P.warpq), sp<int4>(P.medq), sp<int4>(P.itemq), itemq_cap,
                        sp<int2>(P.grp), st));
    BU(cudaMemcpyAsync(&h, P.ctr.p, sizeof(Counters), cudaMemcpyDeviceToHost, st));
    BU(cudaStreamSynchronize(st));
    if (h.nitem <= itemq_cap) break;
    itemq_cap = h.nitem + 1024;
    BU(ensure(g, P.itemq, sizeof(int4) * itemq_cap));
  }
  if (h.nitem > itemq_cap) return report_error(LP_EINTERNAL, "batched plan: item queue sizing");
  P.nwarp = h.nwarp;
  P.nmed = h.nmed;
  P.nitem = h.nitem;
  // the merge of split sources: (source, first partial slot, partial count)
  std::vector<int2> grp((size_t)n);
  if (n > 0)
    BU(cudaMemcpy(grp.data(), P.grp.p, sizeof(int2) * (size_t)n, cudaMemcpyDeviceToHost));
  std::vector<int4> multi;
  for (int r = 0; r < n; ++r)
    if (grp[r].y > 1) multi.push_back(make_int4(r, grp[r].x, grp[r].y, 0));
  P.nmulti = (int)multi.size();
  std::vector<int> order((size_t)P.nitem);
  for (u64 i = 0; i < P.nitem; ++i) order[i] = (int)i;
  BU(ensure(g, P.mgrp, sizeof(int4) * (multi.size() + 1)));
  BU(ensure(g, P.morder, sizeof(int) * (order.size() + 1)));
  BU(ensure(g, P.partial, sizeof(TopEnt) * ((size_t)P.nitem * k + 1)));
  BU(ensure(g, P.phdr, sizeof(int2) * ((size_t)P.nitem + 1)));
  if (!multi.empty())
    BU(cudaMemcpy(P.mgrp.p, multi.data(), sizeof(int4) * multi.size(), cudaMemcpyHostToDevice));
  if (!order.empty())
    BU(cudaMemcpy(P.morder.p, order.data(), sizeof(int) * order.size(), cudaMemcpyHostToDevice));
  A.partial = sp<TopEnt>(P.partial);
  A.partial_hdr = sp<int2>(P.phdr);
  A.partial_cap = P.nitem;
  // record: reset counters and counts, scan the three tiers, merge, emit
  BU(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaMemsetAsync(P.ctr.p, 0, sizeof(Counters), st);
  if (e == cudaSuccess && n > 0) e = cudaMemsetAsync(d_counts, 0, sizeof(int) * (size_t)n, st);
  if (e == cudaSuccess) e = launch_scan_warp(A, sp<int4>(P.warpq), P.nwarp, st);
  if (e == cudaSuccess) e = launch_scan_med(A, sp<int4>(P.medq), P.nmed, st);
  if (e == cudaSuccess) e = launch_scan_cta(A, sp<int4>(P.itemq), P.nitem, st);
  if (e == cudaSuccess)
    e = launch_merge_partials(sp<int4>(P.mgrp), P.nmulti, sp<int>(P.morder), sp<TopEnt>(P.partial),
                              sp<int2>(P.phdr), k, sp<TopEnt>(P.top), d_counts, st);
  if (e == cudaSuccess)
    e = launch_emit_sources(sp<TopEnt>(P.top), d_counts, sp<int>(P.src), n, k, measure,
                            g.fixbits, d_out, st);
  if (e == cudaSuccess && (measure == LP_AA || measure == LP_RA))
    e = launch_pair_cn(d_out, d_counts, k, (u64)n * k, g.d_off, g.d_idx, g.d_deg, g.d_arc, A.cap,
                       st);
  cudaGraph_t graph = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(st, &graph);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return report_cuda(e != cudaSuccess ? e : e2, "batched plan: recording");
  }
  P.graph = graph;
  BU(cudaGraphInstantiate(&P.exec, P.graph, 0));
  P.measure = measure;
  P.cap = cap;
  P.k = k;
  P.opt = opt;
  P.d_out = d_out;
  P.d_counts = d_counts;
  P.ready = true;
  return LP_OK;
}

// Replay the recorded query; ms (if not null) receives its device time.
// *split_seen: a split hash item overflowed (its source is incomplete; the
// plan must be recorded again with dense items only).
lp_status replay(Graph& g, AllPlan& P, float* ms, bool* split_seen) {
  cudaStream_t st = g.stream;
  cudaEvent_t e0 = g.ev[0], e1 = g.ev[1];
  if (ms) BU(cudaEventRecord(e0, st));
  BU(cudaGraphLaunch(P.exec, st));
  if (ms) BU(cudaEventRecord(e1, st));
  Counters h{};
  BU(cudaMemcpyAsync(&h, P.ctr.p, sizeof(Counters), cudaMemcpyDeviceToHost, st));
  BU(cudaStreamSynchronize(st));
  if (ms) BU(cudaEventElapsedTime(ms, e0, e1));
  // overflowed split items (their records may also exceed the split list,
  // device check 2) are redone by a dense plan; any other check is an error
  *split_seen = h.nsplit > 0;
  if (h.error && !(h.error == 2u && *split_seen))
    return report_error(LP_EINTERNAL, "batched query: device consistency check failed");
  return LP_OK;
}

// Replay; after an overflow of a split hash item, record the plan again with
// dense items only (they cannot overflow) and replay that.
lp_status replay_checked(Graph& g, AllPlan& P, float* ms) {
  bool split = false;
  lp_status s = replay(g, P, ms, &split);
  if (s != LP_OK || !split) return s;
  if (P.dense_only) return report_error(LP_EINTERNAL, "batched query: overflow in a dense plan");
  P.dense_only = true;
  s = build_plan(g, P, P.measure, P.cap, P.k, P.opt, P.d_out, P.d_counts);
  if (s != LP_OK) return s;
  return replay(g, P, ms, &split);
}

}  // namespace
}  // namespace lp

struct lp_batch {
  lp_graph* g = nullptr;
  std::vector<int32_t> bases;
  lp::Options opt;
  lp::AllPlan plan;
  std::mutex mu;
};

lp_status lp_batch_create(int32_t n_graphs, const int32_t* n_vertices,
                          const int32_t* const* offsets, const int32_t* const* indices,
                          uint32_t flags, lp_batch** out) {
  if (!out || n_graphs < 1 || !n_vertices || !offsets || !indices)
    return lp::report_error(LP_EINVAL, "lp_batch_create: bad arguments");
  *out = nullptr;
  int64_t nt = 0, at = 0;
  for (int i = 0; i < n_graphs; ++i) {
    if (n_vertices[i] < 0 || !offsets[i])
      return lp::report_error(LP_EINVAL, "lp_batch_create: bad graph");
    if (offsets[i][0] != 0 || offsets[i][n_vertices[i]] < 0)
      return lp::report_error(LP_EINVAL, "lp_batch_create: offsets must start at 0");
    nt += n_vertices[i];
    at += offsets[i][n_vertices[i]];
  }
  if (nt > INT32_MAX - 1 || at > INT32_MAX)
    return lp::report_error(LP_EINVAL, "lp_batch_create: packed graph exceeds int32 ids");
  lp_batch* b = new (std::nothrow) lp_batch();
  if (!b) return lp::report_error(LP_ENOMEM, "lp_batch_create: host allocation");
  std::vector<int32_t> off((size_t)nt + 1), idx((size_t)std::max<int64_t>(at, 1));
  b->bases.resize((size_t)n_graphs + 1);
  int64_t vb = 0, ab = 0;
  for (int i = 0; i < n_graphs; ++i) {
    b->bases[i] = (int32_t)vb;
    const int32_t ni = n_vertices[i];
    const int32_t ai = offsets[i][ni];
    for (int32_t v = 0; v < ni; ++v) off[(size_t)(vb + v)] = (int32_t)(ab + offsets[i][v]);
    for (int32_t e = 0; e < ai; ++e) {
      const int32_t c = indices[i][e];
      // an out-of-range id is kept out of range so that validation rejects it
      idx[(size_t)(ab + e)] = (c >= 0 && c < ni) ? (int32_t)(vb + c) : (int32_t)-1;
    }
    vb += ni;
    ab += ai;
  }
  off[(size_t)nt] = (int32_t)ab;
  b->bases[n_graphs] = (int32_t)vb;
  const lp_status s = lp_graph_create((int32_t)nt, off.data(), idx.data(), flags, &b->g);
  if (s != LP_OK) {
    delete b;
    return s;
  }
  b->opt = lp::options_snapshot();
  *out = b;
  return LP_OK;
}

lp_status lp_batch_destroy(lp_batch* b) {
  if (!b) return LP_OK;
  {
    std::lock_guard<std::mutex> l(b->mu);
    if (b->g) cudaStreamSynchronize(lp::graph_of(b->g).stream);
    b->plan.release();
  }
  lp_graph_destroy(b->g);
  delete b;
  return LP_OK;
}

lp_status lp_batch_info(const lp_batch* b, int32_t* n_graphs, int32_t* n_total, int32_t* bases) {
  if (!b) return lp::report_error(LP_EINVAL, "lp_batch_info: null batch");
  const int32_t ng = (int32_t)b->bases.size() - 1;
  if (n_graphs) *n_graphs = ng;
  if (n_total) *n_total = b->bases[(size_t)ng];
  if (bases) std::memcpy(bases, b->bases.data(), sizeof(int32_t) * b->bases.size());
  return LP_OK;
}

const lp_graph* lp_batch_graph(const lp_batch* b) { return b ? b->g : nullptr; }

static lp_status batch_args_ok(lp_batch* b, int measure, int32_t k, lp_link* d_out,
                               int32_t* d_counts) {
  if (!b || !b->g) return lp::report_error(LP_EINVAL, "batched query: null batch");
  const int n = lp::graph_of(b->g).n;
  if (measure < 0 || measure > LP_RA) return lp::report_error(LP_EINVAL, "batched query: bad measure");
  if (k < 1 || k > LP_MAX_TOPK_PER_SOURCE)
    return lp::report_error(LP_EINVAL, "batched query: k out of range");
  if ((!d_out || !d_counts) && n > 0)
    return lp::report_error(LP_EINVAL, "batched query: null output");
  return LP_OK;
}

lp_status lp_batch_predict_all(lp_batch* b, lp_measure measure, int32_t degree_cap, int32_t k,
                               lp_link* d_out, int32_t* d_counts) {
  lp_status s = batch_args_ok(b, (int)measure, k, d_out, d_counts);
  if (s != LP_OK) return s;
  std::lock_guard<std::mutex> l(b->mu);
  lp::Graph& g = lp::graph_of(b->g);
  std::lock_guard<std::mutex> lg(g.mu);
  BU(cudaSetDevice(g.device));
  const int cap = degree_cap < 0 ? -1 : degree_cap;
  lp::AllPlan& P = b->plan;
  if (!P.ready || P.measure != (int)measure || P.cap != cap || P.k != k || P.d_out != d_out ||
      P.d_counts != d_counts || !lp::same_options(P.opt, b->opt)) {
    if (!P.ready || P.measure != (int)measure || P.cap != cap || P.k != k) P.dense_only = false;
    s = lp::build_plan(g, P, (int)measure, cap, k, b->opt, d_out, d_counts);
    if (s != LP_OK) return s;
  }
  return lp::replay_checked(g, P, nullptr);
}

lp_status lp_batch_autotune(lp_batch* b, lp_measure measure, int32_t degree_cap, int32_t k,
                            int32_t repeats, lp_link* d_out, int32_t* d_counts, float* default_ms,
                            float* best_ms) {
  lp_status s = batch_args_ok(b, (int)measure, k, d_out, d_counts);
  if (s != LP_OK) return s;
  if (repeats < 1) repeats = 1;
  std::lock_guard<std::mutex> l(b->mu);
  lp::Graph& g = lp::graph_of(b->g);
  std::lock_guard<std::mutex> lg(g.mu);
  BU(cudaSetDevice(g.device));
  const int cap = degree_cap < 0 ? -1 : degree_cap;
  auto trial = [&](const lp::Options& o, float* out_ms) -> lp_status {
    b->plan.dense_only = false;
    lp_status r = lp::build_plan(g, b->plan, (int)measure, cap, k, o, d_out, d_counts);
    if (r != LP_OK) return r;
    float best = 0.f;
    for (int i = 0; i < repeats + 1; ++i) {  // the first replay warms up
      float ms = 0.f;
      r = lp::replay_checked(g, b->plan, &ms);
      if (r != LP_OK) return r;
      if (i == 1 || (i > 1 && ms < best)) best = ms;
    }
    *out_ms = repeats >= 1 ? best : 0.f;
    return LP_OK;
  };
  lp::Options cur = b->opt;
  float cur_ms = 0.f;
  s = trial(cur, &cur_ms);
  if (s != LP_OK) return s;
  if (default_ms) *default_ms = cur_ms;
  // coordinate descent over the binning options, each from a few values
  const int warp_v[] = {64, 128, 256};
  const int med_v[] = {512, 1024};
  const int cta_v[] = {2048, 4096, 8192};
  const long long item_v[] = {1ll << 16, 1ll << 18, 1ll << 20};
  const int thr_v[] = {1024, 512};
  for (int pass = 0; pass < 2; ++pass) {
    auto try_set = [&](auto apply) -> lp_status {
      lp::Options o = cur;
      apply(o);
      if (lp::same_options(o, cur)) return LP_OK;
      float ms = 0.f;
      const lp_status r = trial(o, &ms);
      if (r != LP_OK) return r;
      if (ms < cur_ms) {
        cur = o;
        cur_ms = ms;
      }
      return LP_OK;
    };
    for (int v : warp_v) if ((s = try_set([&](lp::Options& o) { o.warp_max = v; })) != LP_OK) return s;
    for (int v : med_v) if ((s = try_set([&](lp::Options& o) { o.med_max = v; })) != LP_OK) return s;
    for (int v : cta_v) if ((s = try_set([&](lp::Options& o) { o.cta_max = v; })) != LP_OK) return s;
    for (long long v : item_v)
      if ((s = try_set([&](lp::Options& o) { o.item_wedges = v; })) != LP_OK) return s;
    for (int v : thr_v) if ((s = try_set([&](lp::Options& o) { o.big_threads = v; })) != LP_OK) return s;
  }
  b->opt = cur;
  if (best_ms) *best_ms = cur_ms;
  // leave the plan of the chosen options recorded
  b->plan.dense_only = false;
  return lp::build_plan(g, b->plan, (int)measure, cap, k, cur, d_out, d_counts);
}

int64_t lp_batch_get_option(const lp_batch* b, lp_option option) {
  if (!b) return -1;
  const lp::Options& o = b->opt;
  switch (option) {
    case LP_OPT_WARP_MAX_WEDGES: return o.warp_max;
    case LP_OPT_MED_MAX_WEDGES: return o.med_max;
    case LP_OPT_CTA_MAX_WEDGES: return o.cta_max;
    case LP_OPT_SPLIT_TARGET: return o.split_target;
    case LP_OPT_SPLIT_LOGCAP: return o.split_logcap;
    case LP_OPT_ITEM_WEDGES: return o.item_wedges;
    case LP_OPT_BIG_CTA_THREADS: return o.big_threads;
    default: return -1;
  }
}
