// lp_internal.cuh -- shared declarations of the liblp CUDA implementation.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <vector>

#include "lp.h"

namespace lp {

typedef unsigned long long u64;
typedef unsigned int u32;

constexpr int kEmpty = 0;                // empty hash key (keys are stored as c + 1)
constexpr int kWarpSlots = 512;          // per-warp hash table (warp tier)
constexpr int kWarpMaxWedges = 256;      // warp tier: W(a) <= this
constexpr int kWarpTierThreads = 256;
constexpr int kMedThreads = 128;         // medium tier: one 4-warp CTA per source
constexpr int kMedSlots = 2048;
constexpr int kMedMaxWedges = 1024;
constexpr int kCtaThreads = 1024;        // large tier: one 32-warp CTA per item
constexpr int kCtaWarps = kCtaThreads / 32;
constexpr int kCtaSlots = 16384;         // largest CTA hash table
constexpr int kCtaMaxWedges = 8192;      // single-item hash: W <= this
constexpr int kSplitTarget = 12288;      // wedges per split hash item
constexpr int kCtaSmem = 192 * 1024;     // table bytes of a 1024-thread large-tier CTA
// shared memory of a large-tier CTA of `threads` threads beyond its table:
// 3 * threads window boundaries (or arc cursors) and a queue of `threads`
// segments (prefix, start, length, weight)
constexpr int big_extra_smem(int threads) { return threads * 3 * 4 + threads * (4 + 4 + 4 + 8); }
// shared memory the large tier may use per SM (two 512-thread CTAs share it)
constexpr int kSmemPerSm = 228 * 1024;
constexpr int kSmemPerCtaReserved = 1024;

// Item kinds (int4.w of a CTA work record).
constexpr int kItemDense = 1;    // dense counters over [lo, hi)
constexpr int kItemSingle = 2;   // the only item of its source (per-source mode)
constexpr int kItemWhole = 4;    // one item covers the source's whole second-order id range
constexpr int kItemD8 = 8;       // dense, 8-bit counters (global mode, source degree <= 255)
constexpr int kMaxSweep = 4096;  // windows or ranges of one item (a 12-bit field of the record)
// Count items of the expand-and-count tier carry this flag in int4.w (the
// other item kinds leave bit 28 clear) and their batch bucket below it.
constexpr int kExpItem = 1 << 28;
constexpr int kExpSplit = 1 << 27;      // a re-split part of a hash bucket
constexpr int kExpGbMask = kExpSplit - 1;
constexpr int kExpMaxBuckets = 4096;    // buckets of one unit
constexpr int kExpMaxTiles = 256;       // tiles of one unit
constexpr int kExpTableBytes = 64 * 1024;  // count pass: table of one CTA (three per SM)
// ExpUnit.flags
constexpr int kExpDense = 4;            // dense counter windows (else a hash table per bucket)
constexpr int kExpC8 = 0, kExpC16 = 1, kExpC32 = 2, kExpC64 = 3;  // counter width (flags & 3)

// One source of the expand-and-count large tier (global mode): its wedges
// are expanded once into records grouped by bucket (an id range of 2^wlog),
// then each bucket is counted in shared memory.
struct ExpUnit {
  int a, lo, hi, kept;   // source, second-order id range [lo, hi), arcs passing the hub test
  int wlog, nb, flags, tile_w;  // bucket width 2^wlog, buckets, kind, wedges per tile
  int K, T, pad0, pad1;  // nonempty arc segments (arc pass), tiles (at most kExpMaxTiles)
  long long W;           // wedges
  long long arc_base;    // first entry of the unit in the segment lists (K + 1 entries)
  long long tfirst_base; // first entry of the unit's tile table (T + 1: first segment of each tile)
  long long excl_base;   // first entry of the unit's exclusion table (nb + 1: first index of
                         // Gamma_a at or above each bucket start)
  long long rec_base;    // first record of the unit in its batch
  long long tile_base;   // first tile of the unit in its batch
  long long pre_base;    // first bucket-start entry of the unit in its batch
  long long bucket_base; // first batch bucket of the unit
};

// Arc table entry for arc e = (a -> b): x = position of a in Gamma_b
// (absolute index into idx), y = off[b + 1], z = |Gamma_b|, w = b.
typedef int4 Arc;

// Selection candidate: exact key num/den, pair (u, v).
struct __align__(8) Cand {
  u64 num, den;
  int u, v;
};

// Per-source top-k entry.
struct __align__(8) TopEnt {
  u64 num, den;
  int c, cn;
};

// Admission threshold: candidates must rank strictly before it.
struct Thresh {
  u64 num, den;
  int u, v;
  int valid;
  int pad;
};

// Device-side counters of one predict call (one allocation, read back whole).
struct Counters {
  u64 wedges;        // estimate: wedges of scanned sources
  u64 kept_arcs;
  u64 scanned_arcs;
  u64 nwarp;         // warp queue length written by the estimate kernel
  u64 nitem;         // large-tier item queue length written by the estimate kernel
  u64 nmed;          // medium queue length
  u64 claim_m;
  u64 claim_w;       // dynamic claim counters
  u64 claim_c;
  u64 cand_cnt;      // selection buffer fill (may exceed capacity)
  u64 candidates;    // distinct candidates scored
  u64 nfailed;       // failed records (buffer overflow)
  u64 nsplit;        // overflowed hash items
  u64 npartial;      // per-source partial lists written
  u64 dense_items;
  u64 tier_wedges[4]; // [3]: the expand-and-count tier
  u64 tier_arcs[4];
  u64 tier_kept[4];
  u64 prof[6];
  u64 nexp;          // expand-and-count units written by the estimate kernel
  u64 claim_x;       // count-item claims
  u32 full;          // selection buffer full
  u32 error;         // device consistency error code
  u64 pad[2];
};

// Everything a scan kernel needs (passed by value).
struct ScanArgs {
  const int* off;
  const int* idx;
  const int* deg;
  const Arc* arc;
  const u64* wt;      // AA / RA: fixed-point weight by intermediary degree
  int n;
  int cap;            // hub limit; INT32_MAX for none
  int measure;
  int mode;           // 0 global (c > a), 1 per-source (c != a)
  int fixbits;        // AA/RA fixed-point fraction bits
  int thr_check;      // 1 if the S_th test is needed (threshold > 0)
  double threshold;
  const int* sources; // per-source mode: source vertex of record index
  Counters* ctr;
  // global mode selection buffer
  Cand* buf;
  u64 buf_cap;
  const Thresh* thresh;
  const u64* vfloor;   // [dmax + 1]: count floor of a source degree under *thresh
  int* gcur;           // large tier: per-arc cursors of sweeps over sources with more arcs
                       // than the shared boundary table (gcur_stride ints per CTA), or null
  int gcur_stride;
  int gcur_ctas;
  // failure / split records
  int4* failed;
  u64 failed_cap;
  int4* split;
  u64 split_cap;
  // per-source mode outputs
  int k;
  TopEnt* out_top;     // [n_src * k] final lists (single items / warp tier)
  int* out_cnt;        // [n_src]
  TopEnt* partial;     // [partial_cap * k] lists of split items
  int2* partial_hdr;   // [partial_cap] (record index, count)
  u64 partial_cap;
  // binning parameters
  int warp_max;        // warp tier: W <= warp_max (<= kWarpMaxWedges)
  int med_max;         // medium tier: W <= med_max (<= kMedMaxWedges)
  int cta_max;         // single large item: W <= cta_max (<= 2^(big_logcap-1))
  int split_target;    // wedges per split hash item
  int split_logcap;    // log2 slots of split hash items (<= big_logcap)
  int big_logcap;      // log2 hash slots that fit the large-tier table bytes
  int big_span;        // dense window of a large-tier item (vertices)
  int big_bytes;       // table bytes of a large-tier CTA
  int dense16;         // global mode, count measures, degrees < 2^16: 16-bit dense counters
  int rec_base;        // global mode: record r is source rec_base + r (a source range)
  int no_split;        // per-source mode: large sources become dense items (no hash overflow)
  int partial_by_item; // per-source mode: an item's partial list goes to slot = its queue index
  int item_wedges;     // target wedges of one dense sweep item
  int big_threads;     // threads of a large-tier CTA: 1024 (one per SM) or 512 (two)
  u64* prof;           // optional: large-tier phase cycles (6 entries) or null
  // expand-and-count tier (global mode)
  int expand;          // 1: large sources with W > cta_max become units (when W < 2^31)
  int x_logcap;        // log2 slots of a hash bucket's table
  int x_min;           // large sources with more wedges than this are units
  int4* xq;            // estimate output: unit records {a, lo, hi, kept}
  u64* xw;             // and their wedge counts
  u64 xq_cap;
  const ExpUnit* xunit;        // units
  const int* xbucket_unit;     // batch bucket -> unit
  const void* xrec;            // batch records: int c (count measures) or int2 {c, |Gamma_b|}
  const u64* xtile_rec;        // batch tile -> first record
  const int* xpre;             // per tile and bucket: first record within the tile (nb + 1 each)
  const int* xexcl;            // per unit and bucket: first index of Gamma_a in the bucket
};

// Process-wide tuning options (lp_set_option).
struct Options {
  long long select_buffer = 8ll << 20;
  int warp_max = kWarpMaxWedges;
  int med_max = kMedMaxWedges;
  int cta_max = kCtaMaxWedges;
  int split_target = kSplitTarget;
  int split_logcap = 14;
  long long item_wedges = 1 << 18;
  int phase_profile = 0;
  int big_threads = 1024;
  int expand = 2;                  // 0 off, 1 on, 2 when the index array exceeds 128 MB
  long long expand_batch = 1ll << 29;  // wedges expanded per batch
  int expand_logcap = 14;          // log2 slots of the count pass's hash tables
  int expand_min = 8192;           // smallest units (wedges, exclusive)
};
Options options_snapshot();

// Host-side graph object.
struct Graph {
  bool owns_arrays = true;  // false for a shadow that shares another graph's arrays
  int device = 0;
  int32_t n = 0;
  int64_t arcs = 0;
  int32_t dmax = 0;
  int fixbits = 40;
  cudaStream_t stream = nullptr;
  int* d_off = nullptr;
  int* d_idx = nullptr;
  int* d_deg = nullptr;
  Arc* d_arc = nullptr;
  u64* d_wt = nullptr;     // [2 * (dmax + 1)]: AA then RA weight by degree
  std::mutex mu;
  // scratch, grown on demand
  struct Scratch {
    void* p = nullptr;
    size_t bytes = 0;
  };
  Scratch s_ctr, s_w, s_warpq, s_itemq, s_warpq2, s_itemq2, s_medq, s_medq2, s_buf, s_buf2,
      s_failed, s_split, s_thresh, s_flags, s_partial, s_phdr, s_top, s_cnt, s_links, s_src, s_grp,
      s_buf3, s_misc, s_vfloor, s_pair, s_gcur, s_xq, s_xw, s_xunit, s_xaseg, s_xaoff, s_xadeg,
      s_xrec, s_xtile, s_xtunit, s_xpre, s_xbunit, s_countq, s_countq2, s_xtfirst, s_xexcl;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t kev[8] = {nullptr, nullptr, nullptr, nullptr,
                        nullptr, nullptr, nullptr, nullptr};  // per scan kernel (start, end)
  cudaEvent_t xev[2] = {nullptr, nullptr};  // expand-and-count passes
};

// ---------------------------------------------------------------- device --

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// Exact total order: x strictly before y (score desc, u asc, v asc).
__device__ __forceinline__ bool before(u64 xn, u64 xd, int xu, int xv, u64 yn, u64 yd, int yu,
                                       int yv) {
  u64 lh = __umul64hi(xn, yd), ll = xn * yd;
  u64 rh = __umul64hi(yn, xd), rl = yn * xd;
  if (lh != rh) return lh > rh;
  if (ll != rl) return ll > rl;
  if (xu != yu) return xu < yu;
  return xv < yv;
}

__device__ __forceinline__ bool cand_before(const Cand& x, const Cand& y) {
  return before(x.num, x.den, x.u, x.v, y.num, y.den, y.u, y.v);
}

}  // namespace lp

// Host-side launchers implemented in the .cu files.
namespace lp {
inline u64 sort_splits_needed(u64 n) { return n / 2048 + 2; }
cudaError_t launch_sort_cands(Cand* d_a, Cand* d_tmp, int* splits, u64 n, cudaStream_t st,
                              Cand** result, int* launches);
cudaError_t launch_set_thresh(const Cand* sorted, u64 k, Thresh* t, cudaStream_t st);
cudaError_t launch_count_floor(int measure, int dmax, const Thresh* thresh, u64* floor,
                               cudaStream_t st);
cudaError_t launch_scan_warp(const ScanArgs& A, const int4* q, u64 nq, cudaStream_t st);
cudaError_t launch_scan_cta(const ScanArgs& A, const int4* q, u64 nq, cudaStream_t st);
cudaError_t launch_scan_med(const ScanArgs& A, const int4* q, u64 nq, cudaStream_t st);
// Expand-and-count tier (lp_expand.cu).
cudaError_t launch_exp_arcs(const ScanArgs& A, ExpUnit* units, int nunits, int* aseg, int* aoff,
                            int* adeg, int* tfirst, int* excl, cudaStream_t st);
cudaError_t launch_exp_tiles(const ScanArgs& A, const ExpUnit* units, const int* tile_unit,
                             int ntiles, const int* aseg, const int* aoff, const int* adeg,
                             const int* tfirst, void* rec, u64* tile_rec, int* pre,
                             cudaStream_t st);
cudaError_t launch_exp_count(const ScanArgs& A, const int4* q, u64 nq, cudaStream_t st);
// Resident serving kernel (lp_serve_dev.cu).  A request slot's parameters,
// written by the host before its work items are published.
struct SrvReq {
  int measure, cap, k, n_src;
  long long src_off;  // first source in the source pool
  long long out_off;  // first link of row 0 in the output pool (rows of k links)
  long long target;   // value of finished[slot] once the request is complete
  unsigned seq;       // written to done[slot] on completion
  int pad;
};
struct SrvArgs {
  const int* off;
  const int* idx;
  const int* deg;
  const Arc* arc;
  const u64* wt;                      // AA then RA weights by degree
  int n, dmax, fixbits, idle_polls;
  const int2* ring;                   // work items {slot, source index} (host memory)
  unsigned long long ring_cap;
  const unsigned long long* tail;     // items published (host memory)
  unsigned long long* head;           // items claimed (device)
  const SrvReq* reqs;                 // request slots (host memory)
  const int* src_pool;                // sources (host memory)
  lp_link* out_pool;                  // result rows (host memory)
  unsigned long long* finished;       // sources finished per slot (device)
  unsigned* done;                     // completion word per slot (host memory)
  unsigned* status;                   // device error word (host memory)
  const unsigned* stop;               // 1: leave at once when idle (host memory)
  unsigned char* defer;               // per pool source: 1 = left to the host (host memory)
  unsigned long long defer_wedges;    // sources with more wedges are deferred
};
size_t serve_smem_bytes(int max_k);
cudaError_t launch_serve(const SrvArgs& S, int max_k, cudaStream_t st);
cudaError_t preload_serve_kernel();

// Host plan of the expand-and-count tier for one global call: the units in
// batches of at most expand_batch wedges (a larger unit alone).
struct ExpBatch {
  size_t u0, u1;               // units [u0, u1)
  u64 wedges, tiles, pre, buckets;
};
struct ExpState {
  std::vector<ExpUnit> units;
  std::vector<ExpBatch> batches;
  size_t next = 0;             // next batch
  float ms_expand = 0.f;       // device time of the arc and expand passes (timing on)
  int launches = 0;
};
// Read the units the estimate wrote, lay them out and run the arc pass.
lp_status exp_setup(Graph& g, ScanArgs& A, u64 nexp, long long batch_wedges, bool timing,
                    ExpState& S);
// Expand the next batch into A's record buffers; items receives its count
// items (one per bucket).
lp_status exp_next_batch(Graph& g, ScanArgs& A, ExpState& S, bool timing,
                         std::vector<int4>& items);
cudaError_t launch_build_weights(int dmax, int fixbits, u64* wt, cudaStream_t st);
cudaError_t launch_estimate2(const ScanArgs& A, int n_rec, int4* warpq, int4* medq, int4* itemq,
                             u64 itemq_cap, int2* grp, cudaStream_t st);
cudaError_t launch_merge_partials(const int4* grp_list, int ngrp, const int* order,
                                  const TopEnt* partial, const int2* hdr, int k, TopEnt* out_top,
                                  int* out_cnt, cudaStream_t st);
cudaError_t launch_emit_global(const Cand* c, u64 n, int measure, int fixbits, lp_link* out,
                               cudaStream_t st);
cudaError_t launch_emit_sources(const TopEnt* top, const int* cnt, const int* sources, int n_src,
                                int k, int measure, int fixbits, lp_link* out, cudaStream_t st);
// Common-neighbour counts of global-mode links grouped by their endpoint of
// larger degree (lp_pair.cu); pair_groups_scratch(n, links, kept_arcs) bytes
// of device scratch, kept_arcs = the arc count when cap < dmax (the kept
// lists are built), else 0.
size_t pair_groups_scratch(int n, u64 nlinks, long long kept_arcs);
cudaError_t launch_pair_cn_groups(lp_link* links, u64 n, int nv, const int* off, const int* idx,
                                  const int* deg, long long arcs, int dmax, int cap, void* scratch,
                                  cudaStream_t st, int* launches);
cudaError_t launch_pair_cn(lp_link* links, const int* cnt_rows, int k, u64 n, const int* off,
                           const int* idx, const int* deg, const Arc* arc, int cap,
                           cudaStream_t st);
// Exact selection keys of global-mode links: count measures from the link's
// cn and the degrees, AA / RA by rebuilding the fixed-point sum (wt: the
// measure's weight table).
cudaError_t launch_link_keys(const lp_link* links, u64 n, int measure, const int* off,
                             const int* idx, const int* deg, const Arc* arc, int cap,
                             const u64* wt, Cand* out, cudaStream_t st);
constexpr int kRadixBinsHost = 2048;
cudaError_t radix_select(const Cand* src, u64 n, u64 k, int measure, Cand* sel, Cand* actA,
                         Cand* actB, u32* d_hist, u64* d_cnt, cudaStream_t st, u64* out_n,
                         int* launches);
cudaError_t launch_thresh_worst(const Cand* a, u64 n, Cand* tmp, Thresh* t, cudaStream_t st,
                                int* launches);
cudaError_t launch_filter_failed(Cand* d_buf, u64 n, const unsigned char* d_flag,
                                 const int4* d_failed_sorted, int nfailed, Cand* d_out,
                                 Counters* d_ctr, u64* d_count, cudaStream_t st);
// Helpers of lp_api.cu used by other translation units.
lp_status report_error(lp_status s, const char* msg);
lp_status report_cuda(cudaError_t e, const char* what);
void stats_begin();
void stats_estimate(const Counters& h);
void stats_add(int64_t candidates, int32_t splits, int32_t launches);
ScanArgs scan_args(Graph& g, int measure, int cap, double threshold, int mode, int k);
// scan_args with explicit options instead of the process-wide ones
// Give the large tier its per-arc cursor scratch (allocates; not for the
// allocation-free path, which leaves A.gcur null).
cudaError_t attach_cursors(Graph& g, ScanArgs& A);
ScanArgs base_args_opts(Graph& g, int measure, int cap, double threshold, int mode, int k,
                        const Options& o);
// Grow a scratch allocation to at least `bytes` (contents are not kept).
cudaError_t ensure(Graph& g, Graph::Scratch& s, size_t bytes);
template <typename T>
inline T* sp(Graph::Scratch& s) {
  return reinterpret_cast<T*>(s.p);
}
lp_status sources_args_ok(const lp_graph* g, int measure, const void* sources, int n_src, int k,
                          const void* out, const void* counts);
Graph& graph_of(const lp_graph* g);
// LP_EINVAL (with a message naming `who`) when RA scores of the hub limit cap
// could exceed the 1e-6 relative accuracy of the fixed-point sums.
lp_status accuracy_guard(const Graph& g, int measure, int cap, const char* who);
// A graph view sharing g's device arrays with its own stream, events and
// scratch (for concurrent workers); freed with destroy_shadow.
lp_status make_shadow(const Graph& g, Graph** out);
void destroy_shadow(Graph* s);
// Load every kernel of the per-source mode (no launch).
cudaError_t preload_sources_kernels();
// Make the allocation-free per-source query ready on the current device dev:
// look up the device address of its static scratch array (which loads the
// array's module) and load the kernels it launches.  Called by
// lp_graph_create, so that no query has to.
cudaError_t prepare_static(int dev);
lp_status run_sources_dev(Graph& g, int measure, int cap, const int* d_src, int n_src, int k,
                          double threshold, lp_link* d_out, int* d_counts);
}  // namespace lp
