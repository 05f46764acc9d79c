/*
 * lp.h -- C ABI of liblp, GPU (sm_103a) neighbourhood-based link prediction.
 *
 * The library implements the scoring and selection of "A Fast Parallel
 * Approach for Neighborhood-based Link Prediction by Disregarding Large Hubs"
 * (Sahu, arXiv 2401.11415):
 *   - IBase (Section 4.1): for every source vertex a, the second-order
 *     vertices c reachable as a -> b -> c are scored; first-order neighbours
 *     and c = a are never predicted (Sections 4.1.1, 4.1.2, 4.1.4).
 *   - DLH (Section 4.2, Algorithm 1): the same, but an intermediary b is
 *     used only when |Gamma_b| <= L_H (the hub limit, inclusive).
 *   - Scores: the nine measures of Section 3.1 (Eq. 1-9).  AA and RA sum over
 *     the common neighbours b (as Algorithm 1 accumulates them) with the
 *     natural logarithm.  The normalisations use full degrees; under DLH, CN
 *     counts only the intermediaries that pass the hub limit.
 *   - Selection: the N_P best pairs with a score strictly above S_th
 *     (Section 4.3 and Algorithm 1), or the k best partners of each requested
 *     source (a per-vertex form of the ranked top-k list of Section 3).
 *
 * Conventions for every call:
 *   - All pointers are HOST pointers unless the name says "_dev"/"d_" (a
 *     CUDA device pointer on the graph's device).  Inputs are copied; the
 *     caller keeps ownership of everything it passes in.  Outputs go into
 *     caller-owned buffers.
 *   - Calls are synchronous and thread-safe: a graph is immutable after
 *     creation and may be shared by threads; calls on one graph serialise
 *     on that graph's CUDA stream.  No call aborts the process: each returns
 *     an lp_status and sets a thread-local message (lp_last_error).
 *   - Results are deterministic: ties are broken by one total order, higher
 *     score first, then smaller u, then smaller v (per-source: smaller v).
 *     The seven count measures are ordered by their exact rational value
 *     (Salton through CN^2 / (|Gamma_a| |Gamma_c|)); AA and RA by their
 *     fixed-point sums (each weight rounded to 2^-F with
 *     F = min(50, 62 - ceil(log2(dmax + 1))), then summed exactly), which
 *     agree with FP64 sums to within |Gamma_b|max * 2^-(F+1) relative for RA
 *     and ln|Gamma_b|max * 2^-(F+1) for AA, |Gamma_b|max = min(L_H, dmax):
 *     below 1e-9 for dmax < 2^16.  An RA call whose bound would exceed 1e-6
 *     (intermediaries of degree above about 2.2M: dmax >= 2^21 without a
 *     hub limit below that) is refused with LP_EINVAL and a message naming
 *     the largest hub limit that keeps it.
 */
#ifndef LP_H
#define LP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Opaque device-resident graph (CSR, sorted adjacency, per-arc table). */
typedef struct lp_graph lp_graph;
/* Opaque request server (continuous batching of per-source queries). */
typedef struct lp_server lp_server;

/* Similarity measures, Eq. 1-9 of Section 3.1. */
typedef enum {
  LP_CN = 0,  /* common neighbours |Ga n Gc|                         (Eq. 1) */
  LP_JC = 1,  /* Jaccard CN / (|Ga| + |Gc| - CN)                      (Eq. 2) */
  LP_SI = 2,  /* Sorensen CN / (|Ga| + |Gc|)                          (Eq. 3) */
  LP_SC = 3,  /* Salton CN / sqrt(|Ga| |Gc|)                          (Eq. 4) */
  LP_HP = 4,  /* hub promoted CN / min(|Ga|, |Gc|)                    (Eq. 5) */
  LP_HD = 5,  /* hub depressed CN / max(|Ga|, |Gc|)                   (Eq. 6) */
  LP_LHN = 6, /* Leicht-Holme-Newman CN / (|Ga| |Gc|)                 (Eq. 7) */
  LP_AA = 7,  /* Adamic-Adar sum over common b of 1 / ln |Gb|         (Eq. 8) */
  LP_RA = 8   /* resource allocation sum over common b of 1 / |Gb|    (Eq. 9) */
} lp_measure;

typedef enum {
  LP_OK = 0,
  LP_EINVAL = 1,    /* bad argument or malformed graph */
  LP_ENOMEM = 2,    /* device or host allocation failed */
  LP_ECUDA = 3,     /* a CUDA call failed */
  LP_ETRUNC = 4,    /* output buffer too small: first out_cap links written */
  LP_ETIMEOUT = 5,  /* a bounded wait ran out */
  LP_EBUSY = 6,     /* queue full or object in use */
  LP_EINTERNAL = 7  /* a device-side consistency check failed */
} lp_status;

/* One predicted link.  Global mode: u < v.  Per-source mode: u = source.
 * score: the FP32 value of the measure; cn: common neighbours b of (u, v)
 * with |Gamma_b| <= degree_cap. */
typedef struct {
  int32_t u, v;
  float score;
  int32_t cn;
} lp_link;

#define LP_CAP_NONE (-1)          /* degree_cap for IBase (no hub limit) */
#define LP_MAX_TOPK_PER_SOURCE 64
#define LP_VALIDATE_FULL 1u       /* lp_graph_create: also check on the host */

/* Statistics of the last lp_predict / lp_predict_sources call on this thread. */
typedef struct {
  int64_t wedges;          /* (a, b, c) triples scanned: b passes the hub test,
                              c > a (global) or c != a (per-source)            */
  int64_t kept_arcs;       /* (a, b) arcs of scanned sources passing the hub test */
  int64_t scanned_arcs;    /* (a, b) arcs read (hub test included)            */
  int64_t candidates;      /* distinct (a, c) scored                          */
  int64_t admitted;        /* candidates written to the selection buffer      */
  int32_t warp_sources;    /* sources scanned by one warp                     */
  int32_t cta_items;       /* (source, vertex range) items scanned by one CTA */
  int32_t dense_items;     /* of which dense-counter items                    */
  int32_t splits;          /* items re-split after a hash overflow            */
  int32_t compactions;     /* selection-buffer compactions                    */
  int32_t launches;        /* kernels launched                                */
  float ms_estimate;       /* device time per phase (0 unless timing enabled) */
  float ms_scan;
  float ms_select;
  float ms_total;
  /* per scan kernel: [0] warp tier, [1] medium tier, [2] large tier,
     [3] expand-and-count tier (global mode; its time includes the arc and
     expand passes, its launches count the count-pass launches) */
  int64_t tier_wedges[4];  /* wedges of the sources binned to the tier       */
  int64_t tier_arcs[4];    /* arc-table entries read by the tier             */
  int64_t tier_kept[4];    /* of which pass the hub test                     */
  int32_t tier_launches[4];/* launches of the tier's scan kernel             */
  float tier_ms[4];        /* summed device time of those launches (timing on) */
  int64_t phase_cycles[6]; /* LP_OPT_PHASE_PROFILE: SM cycles of the large tier
                              (summed over CTAs) in [0] item setup, [1] arc
                              segments and short walks, [3] long-segment
                              pieces, [4] exclusion and scoring, [5] item end;
                              [2] is the whole time of dense items (also in
                              the others)                                     */
  float ms_expand;         /* device time of the expand-and-count tier's arc and
                              expand passes (timing on; also in tier_ms[3])   */
  int32_t exp_units;       /* sources of the expand-and-count tier            */
  int32_t exp_batches;     /* their expand batches                            */
  int64_t exp_items;       /* count items (buckets) run, re-queued ones included */
  int64_t exp_dense_units; /* units counted in dense windows (the rest: hash)   */
} lp_stats;

/*
 * Upload an undirected graph and make it resident on the current CUDA device.
 *   n        number of vertices (>= 0)
 *   offsets  host int32[n + 1], offsets[0] = 0, non-decreasing,
 *            offsets[n] = number of arcs A < 2^31
 *   indices  host int32[A]: neighbours of v are indices[offsets[v] ..
 *            offsets[v+1]); every edge must appear in both directions
 *   flags    LP_VALIDATE_FULL or 0 (the device always checks symmetry)
 *   out      receives the graph handle
 * Lists need not be sorted (the library sorts copies).  Rejected with
 * LP_EINVAL: non-monotone offsets, out-of-range indices, self-loops,
 * duplicate arcs, a missing reverse arc.  The input model is the paper's
 * undirected 32-bit-id graph (Section 5.1.2, Table 1).
 */
lp_status lp_graph_create(int32_t n, const int32_t* offsets, const int32_t* indices,
                          uint32_t flags, lp_graph** out);

/* Free a graph.  NULL is accepted. */
lp_status lp_graph_destroy(lp_graph* g);

/* Vertex count, arc count and largest degree of a graph. */
lp_status lp_graph_info(const lp_graph* g, int32_t* n, int64_t* arcs, int32_t* max_degree);

/*
 * Global mode (Algorithm 1, predictLinksDLH): the k best pairs (u < v, not
 * adjacent, at least one common neighbour through the hub limit) whose score
 * is strictly above `threshold` (S_th), sorted by the total order.
 *   degree_cap  L_H, or LP_CAP_NONE (any negative value) for IBase;
 *               0 gives an empty result
 *   k           N_P, the maximum number of links; 0 = all of them
 *   out         host lp_link[out_cap]
 *   out_n       receives the number of links found (<= k when k > 0)
 * If out_cap < found, the first out_cap links are written, *out_n = found,
 * and LP_ETRUNC is returned.
 */
lp_status lp_predict(const lp_graph* g, lp_measure measure, int32_t degree_cap, int64_t k,
                     double threshold, lp_link* out, int64_t out_cap, int64_t* out_n);

/* As lp_predict, but `d_out` is a device pointer (lp_link[out_cap]) on the
 * graph's device; nothing is copied to the host except *out_n. */
lp_status lp_predict_dev(const lp_graph* g, lp_measure measure, int32_t degree_cap, int64_t k,
                         double threshold, lp_link* d_out, int64_t out_cap, int64_t* out_n);

/*
 * Global mode over a source range: as lp_predict, restricted to the pairs
 * (u, v) with src_begin <= u < src_end (still u < v).  Sources are independent
 * (Section 4.1.7), so the ranges of a partition of [0, n) can run on separate
 * GPUs: the best k of the union of their lists, under the same total order,
 * is the lp_predict result.  0 <= src_begin <= src_end <= n, else LP_EINVAL.
 * Host output, as lp_predict.  Not in the paper (the sharding of Section 4.1.7
 * across devices).
 */
lp_status lp_predict_range(const lp_graph* g, lp_measure measure, int32_t degree_cap, int64_t k,
                           double threshold, int32_t src_begin, int32_t src_end, lp_link* out,
                           int64_t out_cap, int64_t* out_n);

/*
 * Merge of global-mode results (the merging phase of Algorithm 1, Section
 * 4.1.7, across devices): the k best of n_links distinct links (u < v) of
 * graph g under the total order, sorted.  The intended input is the
 * concatenation of lp_predict_range results of one measure and degree_cap
 * over a partition of [0, n): the result is then, bit for bit, what one
 * lp_predict call returns.  Count measures take each link's exact key from
 * its cn and the two degrees; AA and RA rebuild their fixed-point sums from
 * the graph (the score field of the input is not read), so near-equal FP32
 * scores are ordered exactly as the library's selection orders them.
 *   links  host lp_link[n_links], any order; k = 0 keeps them all
 *   out    host lp_link[out_cap]; *out_n receives the number of links kept
 * LP_EINVAL if a link is not a pair 0 <= u < v < n with cn >= 0, or for the
 * RA accuracy limit above; LP_ETRUNC as in lp_predict.  Not in the paper's
 * single-machine design (its merge is sequential over per-thread lists).
 */
lp_status lp_merge_links(const lp_graph* g, lp_measure measure, int32_t degree_cap,
                         const lp_link* links, int64_t n_links, int64_t k, lp_link* out,
                         int64_t out_cap, int64_t* out_n);

/*
 * Per-source mode: for each sources[i], its k best partners c != sources[i]
 * that are not adjacent to it and score strictly above `threshold`, sorted by
 * (score desc, c asc).  out holds n_src * k links (row i for sources[i]);
 * counts[i] receives the number of links in row i (<= k); the rest of the
 * row is filled with {u = -1, v = -1, score = 0, cn = 0}.  1 <= k <=
 * LP_MAX_TOPK_PER_SOURCE.  Sources may repeat.  Host pointers.
 */
lp_status lp_predict_sources(const lp_graph* g, lp_measure measure, int32_t degree_cap,
                             const int32_t* sources, int32_t n_src, int32_t k,
                             double threshold, lp_link* out, int32_t* counts);

/* As lp_predict_sources with device pointers for sources, out and counts. */
lp_status lp_predict_sources_dev(const lp_graph* g, lp_measure measure, int32_t degree_cap,
                                 const int32_t* d_sources, int32_t n_src, int32_t k,
                                 double threshold, lp_link* d_out, int32_t* d_counts);

/* Tuning options (process-wide; each applies to calls that start after it is
 * set).  They change speed and memory use, never results. */
typedef enum {
  LP_OPT_SELECT_BUFFER = 1,   /* minimum selection-buffer capacity in candidates
                                 (default 8388608; 24 bytes each, twice)       */
  LP_OPT_WARP_MAX_WEDGES = 2, /* warp tier: sources with W <= this (1..256, 256) */
  LP_OPT_CTA_MAX_WEDGES = 3,  /* one large item per source up to W (257..8192, 8192) */
  LP_OPT_SPLIT_TARGET = 4,    /* wedges per split hash item (256..32768, 12288),
                                 halved per log2 step the table is below LOGCAP,
                                 and halved in the per-source calls            */
  LP_OPT_SPLIT_LOGCAP = 5,    /* log2 slots of a split hash item (6..14, 14)     */
  LP_OPT_MED_MAX_WEDGES = 6,  /* medium tier: W <= this (1..1024, 1024); the
                                 warp tier takes precedence                     */
  LP_OPT_ITEM_WEDGES = 7,     /* target wedges of one dense sweep item
                                 (1024..2^30, 262144)                           */
  LP_OPT_PHASE_PROFILE = 8,   /* 1: record per-phase clock cycles of the large
                                 tier in lp_stats.phase_cycles (0..1, 0)        */
  LP_OPT_BIG_CTA_THREADS = 9, /* threads of a large-tier CTA: 1024 (one per SM,
                                 192 KB table) or 512 (two per SM, 98 KB each;
                                 split targets shrink with the table) (1024)   */
  LP_OPT_EXPAND = 10,         /* global mode: large sources with more wedges
                                 than LP_OPT_EXPAND_MIN_WEDGES are instead
                                 expanded once into per-bucket records and
                                 counted bucket by bucket: 0 never, 1 always,
                                 2 when the index array exceeds 128 MB (2)     */
  LP_OPT_EXPAND_BATCH = 11,   /* wedges expanded per batch of that tier
                                 (2^16..2^34, 2^29; 4 bytes each, 8 for AA/RA) */
  LP_OPT_EXPAND_HASH_LOGCAP = 12, /* log2 slots of that tier's hash tables (6..14,
                                 14); a bucket whose table fills is re-split */
  LP_OPT_EXPAND_MIN_WEDGES = 13, /* that tier takes the large sources with more
                                 wedges than this (257..2^30; at least the
                                 medium-tier limit) (8192)                     */
} lp_option;

/*
 * Batched multi-graph mode (not in the paper).  n_graphs independent CSR
 * graphs (each as for lp_graph_create; host arrays, copied) are packed into
 * one block-diagonal graph: vertex v of graph i becomes bases[i] + v, and no
 * two-hop path crosses graphs.  lp_batch_predict_all gives the per-source
 * top-k (as lp_predict_sources) of every packed vertex: d_out lp_link[n_total
 * * k] and d_counts int32[n_total] on the device, pairs in packed ids (subtract
 * bases[i] for graph i's own ids).  The first call for a (measure, degree_cap,
 * k, output buffers, options) records the launches in a CUDA graph after one
 * work estimate; later calls replay it.  lp_batch_autotune times replays of
 * plans built with other binning options (tier limits, item size, large-tier
 * CTA size), keeps the fastest for the batch (lp_batch_get_option) and
 * reports the default and best device times of one query (ms).
 * Errors: LP_EINVAL for bad arguments or graphs, LP_ENOMEM, LP_ECUDA,
 * LP_EINTERNAL if a device check fails.
 */
typedef struct lp_batch lp_batch;
lp_status lp_batch_create(int32_t n_graphs, const int32_t* n_vertices,
                          const int32_t* const* offsets, const int32_t* const* indices,
                          uint32_t flags, lp_batch** out);
lp_status lp_batch_destroy(lp_batch* b);
/* n_graphs, n_total and bases (int32[n_graphs + 1]) of a batch; any may be null. */
lp_status lp_batch_info(const lp_batch* b, int32_t* n_graphs, int32_t* n_total, int32_t* bases);
/* The packed graph (for lp_graph_info, lp_predict_sources, ...); owned by the batch. */
const lp_graph* lp_batch_graph(const lp_batch* b);
lp_status lp_batch_predict_all(lp_batch* b, lp_measure measure, int32_t degree_cap, int32_t k,
                               lp_link* d_out, int32_t* d_counts);
lp_status lp_batch_autotune(lp_batch* b, lp_measure measure, int32_t degree_cap, int32_t k,
                            int32_t repeats, lp_link* d_out, int32_t* d_counts, float* default_ms,
                            float* best_ms);
/* The batch's value of a binning option (-1 for others). */
int64_t lp_batch_get_option(const lp_batch* b, lp_option option);

/* Set a tuning option; LP_EINVAL if the option or value is out of range. */
lp_status lp_set_option(lp_option option, int64_t value);

/* Current value of a tuning option (-1 if unknown). */
int64_t lp_get_option(lp_option option);

/*
 * As lp_predict_sources_dev, but allocates nothing: no cudaMalloc or
 * cudaFree, no allocating library routine, no host heap use.  This is for
 * callers that cannot allocate at call time, for example code running under
 * a memory pool it does not own or on a request path where an allocation
 * (and the device synchronisation it can cause) is not allowed.  The paper
 * has no counterpart; it is an integration feature of this library.
 *   Inputs and outputs are device pointers supplied by the caller, as in
 *   lp_predict_sources_dev.  All working memory comes from one fixed 32 MiB
 *   array in device global memory that the library declares statically; each
 *   device that loads the library holds it until the process exits.
 *   Limits: n_src <= 2^20 and n_src * (40 + 24 k) bytes plus the work items
 *   of the sources must fit in the 32 MiB; larger requests are rejected with
 *   LP_EINVAL and a message (split them into several calls).
 *   The array and the code of the kernels this call launches become
 *   resident on a device when the first graph is created there:
 *   lp_graph_create looks up the array's device address
 *   (cudaGetSymbolAddress, with that device current) and loads those
 *   kernels, so no call of this function loads or allocates anything, the
 *   first one included.  Calls are serialised on the host, but every call
 *   shares the one array: work that overlaps on the GPU from other
 *   threads or processes using the same library copy must not run at the
 *   same time (it would race on the array).  Per-call state is cleared at
 *   the start of each call.  A request whose overflowed or partial work
 *   items exceed what the array holds also fails with LP_EINVAL and a
 *   message (use fewer sources per call).
 */
lp_status lp_predict_sources_static(const lp_graph* g, lp_measure measure, int32_t degree_cap,
                                    const int32_t* d_sources, int32_t n_src, int32_t k,
                                    double threshold, lp_link* d_out, int32_t* d_counts);

/* ------------------------------------------------------------ serving --
 * Continuous batching of per-source top-k queries (lp_predict_sources
 * semantics, threshold 0) on one resident graph.  Requests of uneven sizes
 * arrive at any time from any thread; `slots` worker threads each take the
 * oldest pending request together with every other pending request of the
 * same (measure, degree_cap, k), up to max_batch_sources sources, and run
 * them as one device batch on their own CUDA stream, so batches of different
 * slots overlap on the GPU and requests that arrive while others run join the
 * next batch.  Each request's result is exactly what lp_predict_sources
 * returns for it alone.  Not in the paper (a per-vertex serving form of the
 * ranked top-k list of Section 3).
 */
typedef struct {
  int32_t slots;             /* concurrent device batches, 1..8 (0: 2)           */
  int32_t max_batch_sources; /* sources per batch and per request (0: 65536)    */
  int32_t max_pending;       /* queued requests before LP_EBUSY (0: 65536)      */
  int32_t max_k;             /* largest k accepted, <= LP_MAX_TOPK_PER_SOURCE (0: 16) */
  int32_t paused;            /* 1: queue requests but start no batch until
                                lp_serve_resume                                   */
  int32_t mode;              /* 0: host worker threads run batches (the default);
                                1: a resident kernel serves the requests (it can
                                defer sources above defer_wedges to a host
                                thread running the tiered pipeline)            */
  int32_t idle_polls;        /* mode 1: the kernel is asked to leave once no work
                                has been outstanding for idle_polls x 4 us, and
                                a CTA leaves on its own after 100 times that
                                without work (0: 2500)                           */
  int32_t defer_wedges;      /* mode 1: a source with more wedges than this (its
                                hub-limited two-hop work) is not counted by the
                                resident kernel but by the tiered per-source
                                pipeline when its request is collected; the
                                kernel leaves the GPU to that pipeline until
                                those rows are in (0: 65536)                    */
} lp_serve_opts;

typedef struct {
  int64_t submitted;         /* requests accepted                                 */
  int64_t completed;         /* requests finished (result ready or failed)        */
  int64_t batches;           /* device batches run                                */
  int64_t batched_sources;   /* sources over all batches                          */
  int64_t max_batch_requests;/* most requests merged into one batch (mode 1: most
                                requests in flight on the device at once)        */
  int64_t kernel_launches;   /* mode 1: launches of the resident kernel (it leaves
                                after idle_polls polls without work and is
                                launched again when work arrives)                */
  int64_t deferred_sources;  /* mode 1: sources counted by the tiered pipeline
                                (more than defer_wedges wedges)                   */
} lp_serve_stats;

/* Start a server on graph g (which must outlive it).  opts may be NULL.
 * Device memory for the batches is allocated here, not per request. */
lp_status lp_serve_open(const lp_graph* g, const lp_serve_opts* opts, lp_server** out);

/* Queue a request: host array sources[n_src] (copied; ids checked against
 * the graph), 1 <= n_src <= max_batch_sources, 1 <= k <= max_k.  Returns at
 * once with *req_id.  LP_EBUSY if max_pending requests are queued,
 * LP_EINVAL on bad arguments or after lp_serve_close started. */
lp_status lp_serve_submit(lp_server* s, const int32_t* sources, int32_t n_src, lp_measure measure,
                          int32_t degree_cap, int32_t k, uint64_t* req_id);

/* Wait at most timeout_us microseconds (< 0: no limit) for request req_id.
 * When it is done its result is copied to host out[n_src * k] (row i for
 * sources[i]) and counts[n_src], the request is released, and its status is
 * returned.  LP_ETIMEOUT if it is not done in time (the request stays and can
 * be waited for again); LP_EINVAL for an unknown or already released id. */
lp_status lp_serve_wait(lp_server* s, uint64_t req_id, int64_t timeout_us, lp_link* out,
                        int32_t* counts);

/* Let the workers start batches (after lp_serve_open with paused = 1). */
lp_status lp_serve_resume(lp_server* s);

/* *done = 1 if request req_id has finished, else 0 (LP_EINVAL: unknown id). */
lp_status lp_serve_poll(lp_server* s, uint64_t req_id, int32_t* done);

/* Counters of the server since lp_serve_open. */
lp_status lp_serve_get_stats(lp_server* s, lp_serve_stats* out);

/* Finish every queued request (a paused server is resumed), stop the
 * workers and free the server.  Results not collected with lp_serve_wait are
 * discarded.  No other call on the server may run concurrently with it or
 * after it.  NULL accepted. */
lp_status lp_serve_close(lp_server* s);

/* Statistics of this thread's last predict call. */
lp_status lp_last_stats(lp_stats* out);

/* Enable (1) or disable (0) device timing of the phases in lp_stats (CUDA
 * events on the graph's stream).  Process-wide; off by default. */
void lp_set_timing(int enable);

/* The CUDA stream (cudaStream_t) the graph's calls run on. */
void* lp_graph_stream(const lp_graph* g);

/* Thread-local message for the last failing call ("" if none). */
const char* lp_last_error(void);

/* Library version string. */
const char* lp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LP_H */
