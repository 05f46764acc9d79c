/*
 * lp_oracle.c -- CPU oracle for neighbourhood-based link prediction.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this file; the product path never
 * does.  It shares no code, header, table or helper with the CUDA library.
 *
 * It follows the paper's Algorithm 1 (predictLinksDLH with scanEdges) step by
 * step, in plain C with FP64 arithmetic:
 *   - for every source a, a distance-2 traversal a -> b -> c that skips
 *     intermediaries b with |Gamma_b| > L_H (Section 4.2.1, the DLH rule; no
 *     limit gives IBase, Section 4.1.1),
 *   - counting paths per second-order vertex c into a dense per-thread table
 *     with a touched-key list (the collision-free hashtable of Section 4.1.3),
 *     skipping c <= a in the global mode (Section 4.1.2),
 *   - dropping the first-order neighbours of a (Section 4.1.4),
 *   - scoring with Eq. 1-9 (Section 3.1) and the union identity
 *     |Gamma_a u Gamma_c| = |Gamma_a| + |Gamma_c| - CN (Section 4.1.2),
 *   - keeping scores strictly above S_th and the top N_P per thread in a
 *     min-heap (Section 4.1.6), then merging the per-thread lists (4.1.7).
 *
 * Readings where the paper is silent or inconsistent:
 *   - AA and RA sum over the common neighbours (the wedge midpoints b), as
 *     Algorithm 1 and Section 4.1.2 accumulate them; Eq. 8-9 print a union.
 *   - AA uses the natural logarithm.
 *   - Under DLH the normalisations use the full degrees |Gamma_a|, |Gamma_c|
 *     and CN counts only the intermediaries that pass the hub limit.
 *   - The hub test is inclusive: an intermediary is used when
 *     |Gamma_b| <= L_H.
 *   - Scores must be strictly greater than S_th; adjacent pairs are dropped
 *     explicitly, whatever S_th is.
 *   - Ties (Section 4.2.3 leaves their order open) are resolved by one total
 *     order: higher score first, then smaller u, then smaller v.  The seven
 *     count measures compare their exact rational value num/den by 128-bit
 *     cross-multiplication (Salton through its square CN^2/(da*dc)); AA and
 *     RA compare their FP64 sums.
 *   - The per-source mode (a top-k list for each requested vertex) is not in
 *     the paper; it scores every c != a and orders by (score desc, c asc).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { LPO_CN, LPO_JC, LPO_SI, LPO_SC, LPO_HP, LPO_HD, LPO_LHN, LPO_AA, LPO_RA, LPO_NMEASURES };

typedef struct {
  int32_t u, v;      /* source a and second-order vertex c */
  int64_t cn;        /* common neighbours through non-hub intermediaries */
  uint64_t num, den; /* exact score num/den (count measures); den = 0 for AA/RA */
  double value;      /* FP64 score */
} lpo_link;

/* ------------------------------------------------------------ scoring --- */

/* Eq. 1-9 for one pair: fills num/den (count measures) and the FP64 value. */
static void score_pair(int measure, int64_t cn, double acc, int64_t da, int64_t dc,
                       lpo_link* o) {
  uint64_t c = (uint64_t)cn, a = (uint64_t)da, d = (uint64_t)dc;
  o->cn = cn;
  o->num = c;
  o->den = 1;
  switch (measure) {
    case LPO_CN: /* Eq. 1 */
      o->value = (double)c;
      break;
    case LPO_JC: /* Eq. 2 with |Ga u Gc| = |Ga| + |Gc| - CN */
      o->den = a + d - c;
      o->value = (double)c / (double)o->den;
      break;
    case LPO_SI: /* Eq. 3 */
      o->den = a + d;
      o->value = (double)c / (double)o->den;
      break;
    case LPO_SC: /* Eq. 4; ordered through its square CN^2 / (da dc) */
      o->num = c * c;
      o->den = a * d;
      o->value = (double)c / sqrt((double)(a * d));
      break;
    case LPO_HP: /* Eq. 5 */
      o->den = a < d ? a : d;
      o->value = (double)c / (double)o->den;
      break;
    case LPO_HD: /* Eq. 6 */
      o->den = a > d ? a : d;
      o->value = (double)c / (double)o->den;
      break;
    case LPO_LHN: /* Eq. 7 */
      o->den = a * d;
      o->value = (double)c / (double)o->den;
      break;
    default: /* AA (Eq. 8), RA (Eq. 9): the accumulated FP64 sum */
      o->num = 0;
      o->den = 0;
      o->value = acc;
      break;
  }
}

/* Weight that one intermediary b of degree db adds (Algorithm 1, scanEdges). */
static double wedge_weight(int measure, int64_t db) {
  if (measure == LPO_AA) return 1.0 / log((double)db);
  if (measure == LPO_RA) return 1.0 / (double)db;
  return 0.0;
}

/* > 0 if x ranks before y in the total order (score desc, u asc, v asc). */
static int better(const lpo_link* x, const lpo_link* y) {
  if (x->den != 0 && y->den != 0) {
    unsigned __int128 l = (unsigned __int128)x->num * y->den;
    unsigned __int128 r = (unsigned __int128)y->num * x->den;
    if (l != r) return l > r;
  } else if (x->value != y->value) {
    return x->value > y->value;
  }
  if (x->u != y->u) return x->u < y->u;
  return x->v < y->v;
}

static int cmp_links(const void* p, const void* q) {
  const lpo_link* x = (const lpo_link*)p;
  const lpo_link* y = (const lpo_link*)q;
  if (better(x, y)) return -1;
  if (better(y, x)) return 1;
  return 0;
}

/* ---------------------------------------------- per-thread prediction list -- */

/* Prediction list P_t (Section 4.1.6): appended until it holds k entries,
 * then kept as a heap whose root is the worst entry.  k = 0: unbounded. */
typedef struct {
  lpo_link* a;
  int64_t n, cap, k;
  int heap;
  int oom;
} plist;

static void sift_down(lpo_link* h, int64_t n, int64_t i) {
  for (;;) {
    int64_t l = 2 * i + 1, r = l + 1, w = i;
    if (l < n && better(&h[w], &h[l])) w = l;   /* w: the worse of the three */
    if (r < n && better(&h[w], &h[r])) w = r;
    if (w == i) return;
    lpo_link t = h[i]; h[i] = h[w]; h[w] = t;
    i = w;
  }
}

static void plist_push(plist* p, const lpo_link* x) {
  if (p->k == 0 || p->n < p->k) {
    if (p->n == p->cap) {
      int64_t nc = p->cap ? 2 * p->cap : 1024;
      if (p->k && nc > p->k) nc = p->k;
      lpo_link* na = (lpo_link*)realloc(p->a, sizeof(lpo_link) * (size_t)nc);
      if (!na) { p->oom = 1; return; }
      p->a = na;
      p->cap = nc;
    }
    p->a[p->n++] = *x;
    if (p->k && p->n == p->k) {           /* make the heap once it is full */
      for (int64_t i = p->n / 2 - 1; i >= 0; --i) sift_down(p->a, p->n, i);
      p->heap = 1;
    }
  } else if (better(x, &p->a[0])) {       /* replace the worst kept entry */
    p->a[0] = *x;
    sift_down(p->a, p->n, 0);
  }
}

/* ------------------------------------------------------ one source's scan -- */

typedef struct {
  int64_t* cnt;      /* dense path counts, indexed by vertex */
  double* acc;       /* dense AA/RA sums */
  int32_t* touched;  /* keys in insertion order */
  int64_t ntouched;
} table;

/*
 * Scan the second-order neighbourhood of a (Algorithm 1: the loop over
 * G.out(a) with the hub test, then scanEdges for each kept b).  mode 0: global
 * (skip c <= a); mode 1: per-source (skip only c == a).
 */
static void scan_source(int32_t a, const int32_t* off, const int32_t* idx, int measure,
                        int64_t cap, int mode, table* t) {
  t->ntouched = 0;
  for (int32_t j = off[a]; j < off[a + 1]; ++j) {
    int32_t b = idx[j];
    int64_t db = (int64_t)off[b + 1] - off[b];
    if (cap >= 0 && db > cap) continue;          /* disregard the large hub */
    for (int32_t q = off[b]; q < off[b + 1]; ++q) {
      int32_t c = idx[q];
      if (mode == 0 ? (c <= a) : (c == a)) continue;
      if (t->cnt[c] == 0) t->touched[t->ntouched++] = c;
      t->cnt[c] += 1;
      t->acc[c] += wedge_weight(measure, db);
    }
  }
  /* drop first-order neighbours (Section 4.1.4) */
  for (int32_t j = off[a]; j < off[a + 1]; ++j) t->cnt[idx[j]] = -1;
}

static void clear_source(int32_t a, const int32_t* off, const int32_t* idx, table* t) {
  for (int64_t i = 0; i < t->ntouched; ++i) {
    t->cnt[t->touched[i]] = 0;
    t->acc[t->touched[i]] = 0.0;
  }
  for (int32_t j = off[a]; j < off[a + 1]; ++j) t->cnt[idx[j]] = 0;
  t->ntouched = 0;
}

static int table_init(table* t, int32_t n) {
  t->cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  t->acc = (double*)calloc((size_t)n + 1, sizeof(double));
  t->touched = (int32_t*)malloc(sizeof(int32_t) * ((size_t)n + 1));
  t->ntouched = 0;
  return t->cnt && t->acc && t->touched;
}

static void table_free(table* t) {
  free(t->cnt); free(t->acc); free(t->touched);
}

/* --------------------------------------------------------- public calls -- */

/*
 * Global mode (Algorithm 1): the top k (k = 0: all) pairs u < v with a score
 * strictly above `threshold`, ordered by the total order.  cap < 0: IBase.
 * Writes min(out_cap, found) links and sets *out_n to the number found
 * (<= k).  Returns 0, -1 on bad arguments, -2 on allocation failure.
 */
int lpo_predict(int32_t n, const int32_t* off, const int32_t* idx, int measure, int64_t cap,
                int64_t k, double threshold, int nthreads, lpo_link* out, int64_t out_cap,
                int64_t* out_n) {
  if (n < 0 || measure < 0 || measure >= LPO_NMEASURES || k < 0 || !out_n) return -1;
  *out_n = 0;
  if (n == 0) return 0;
  int nt = 1;
#ifdef _OPENMP
  nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#endif
  plist* lists = (plist*)calloc((size_t)nt, sizeof(plist));
  if (!lists) return -2;
  int fail = 0;
#pragma omp parallel num_threads(nt)
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    plist* p = &lists[tid];
    p->k = k;
    table t;
    int ok = table_init(&t, n);
    if (!ok) {
#pragma omp atomic write
      fail = 1;
    }
#pragma omp for schedule(dynamic, 64)
    for (int32_t a = 0; a < n; ++a) {
      if (!ok) continue;
      scan_source(a, off, idx, measure, cap, 0, &t);
      int64_t da = (int64_t)off[a + 1] - off[a];
      for (int64_t i = 0; i < t.ntouched; ++i) {
        int32_t c = t.touched[i];
        if (t.cnt[c] <= 0) continue;               /* excluded neighbour */
        lpo_link x;
        x.u = a;
        x.v = c;
        score_pair(measure, t.cnt[c], t.acc[c], da, (int64_t)off[c + 1] - off[c], &x);
        if (!(x.value > threshold)) continue;      /* keep scores above S_th */
        plist_push(p, &x);
      }
      clear_source(a, off, idx, &t);
    }
    if (ok) table_free(&t);
    if (p->oom) {
#pragma omp atomic write
      fail = 1;
    }
  }
  int rc = 0;
  if (fail) {
    rc = -2;
  } else {
    /* merge: all per-thread lists, sorted by the total order, first k */
    int64_t tot = 0;
    for (int i = 0; i < nt; ++i) tot += lists[i].n;
    lpo_link* all = (lpo_link*)malloc(sizeof(lpo_link) * (size_t)(tot > 0 ? tot : 1));
    if (!all) {
      rc = -2;
    } else {
      int64_t w = 0;
      for (int i = 0; i < nt; ++i) {
        memcpy(all + w, lists[i].a, sizeof(lpo_link) * (size_t)lists[i].n);
        w += lists[i].n;
      }
      qsort(all, (size_t)tot, sizeof(lpo_link), cmp_links);
      int64_t keep = (k > 0 && tot > k) ? k : tot;
      int64_t wr = keep < out_cap ? keep : out_cap;
      if (wr > 0) memcpy(out, all, sizeof(lpo_link) * (size_t)wr);
      *out_n = keep;
      free(all);
    }
  }
  for (int i = 0; i < nt; ++i) free(lists[i].a);
  free(lists);
  return rc;
}

/*
 * Per-source mode: for each sources[i], its k best partners c != a that are
 * not adjacent to a, with score strictly above threshold, ordered by
 * (score desc, c asc).  out holds n_src * k links; counts[i] = links for
 * sources[i].  Returns 0, -1 on bad arguments, -2 on allocation failure.
 */
int lpo_predict_sources(int32_t n, const int32_t* off, const int32_t* idx, int measure,
                        int64_t cap, const int32_t* sources, int32_t n_src, int32_t k,
                        double threshold, int nthreads, lpo_link* out, int32_t* counts) {
  if (n < 0 || measure < 0 || measure >= LPO_NMEASURES || k < 0 || n_src < 0) return -1;
  for (int32_t i = 0; i < n_src; ++i)
    if (sources[i] < 0 || sources[i] >= n) return -1;
  int nt = 1;
#ifdef _OPENMP
  nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#endif
  int fail = 0;
#pragma omp parallel num_threads(nt)
  {
    table t;
    int ok = table_init(&t, n);
    lpo_link* cand = (lpo_link*)malloc(sizeof(lpo_link) * ((size_t)n + 1));
    if (!ok || !cand) {
#pragma omp atomic write
      fail = 1;
    }
#pragma omp for schedule(dynamic, 16)
    for (int32_t i = 0; i < n_src; ++i) {
      if (!ok || !cand) continue;
      int32_t a = sources[i];
      scan_source(a, off, idx, measure, cap, 1, &t);
      int64_t da = (int64_t)off[a + 1] - off[a];
      int64_t nc = 0;
      for (int64_t q = 0; q < t.ntouched; ++q) {
        int32_t c = t.touched[q];
        if (t.cnt[c] <= 0) continue;
        lpo_link x;
        x.u = a;
        x.v = c;
        score_pair(measure, t.cnt[c], t.acc[c], da, (int64_t)off[c + 1] - off[c], &x);
        if (!(x.value > threshold)) continue;
        cand[nc++] = x;
      }
      qsort(cand, (size_t)nc, sizeof(lpo_link), cmp_links);
      int32_t keep = nc < k ? (int32_t)nc : k;
      memcpy(out + (int64_t)i * k, cand, sizeof(lpo_link) * (size_t)keep);
      counts[i] = keep;
      clear_source(a, off, idx, &t);
    }
    if (ok) table_free(&t);
    free(cand);
  }
  return fail ? -2 : 0;
}

/*
 * Score of one pair (u, v) straight from the definitions (Eq. 1-9): a merge
 * of the two sorted adjacency lists, counting the common neighbours b with
 * |Gamma_b| <= cap (cap < 0: all).  Independent of the traversal above;
 * used for sampled checks at sizes where the full oracle is too slow.
 * Returns 0, or -1 on bad arguments.  adjacent is set when v is in Gamma_u.
 */
int lpo_pair(int32_t n, const int32_t* off, const int32_t* idx, int measure, int64_t cap,
             int32_t u, int32_t v, lpo_link* out, int32_t* adjacent) {
  if (u < 0 || v < 0 || u >= n || v >= n || measure < 0 || measure >= LPO_NMEASURES) return -1;
  int32_t i = off[u], j = off[v];
  int64_t cn = 0;
  double acc = 0.0;
  *adjacent = 0;
  for (int32_t q = off[u]; q < off[u + 1]; ++q) if (idx[q] == v) *adjacent = 1;
  while (i < off[u + 1] && j < off[v + 1]) {
    if (idx[i] < idx[j]) { ++i; continue; }
    if (idx[i] > idx[j]) { ++j; continue; }
    int32_t b = idx[i];
    int64_t db = (int64_t)off[b + 1] - off[b];
    if (cap < 0 || db <= cap) { cn += 1; acc += wedge_weight(measure, db); }
    ++i; ++j;
  }
  out->u = u;
  out->v = v;
  score_pair(measure, cn, acc, (int64_t)off[u + 1] - off[u], (int64_t)off[v + 1] - off[v], out);
  return 0;
}

/*
 * Work counts: total wedges (a, b, c) with b in Gamma_a, |Gamma_b| <= cap and
 * c in Gamma_b, c > a (mode 0) or c != a (mode 1), and the number of
 * (a, b) arcs that pass the hub test.
 */
void lpo_work(int32_t n, const int32_t* off, const int32_t* idx, int64_t cap, int mode,
              int64_t* wedges, int64_t* kept_arcs) {
  int64_t w = 0, ka = 0;
#pragma omp parallel for reduction(+ : w, ka) schedule(dynamic, 256)
  for (int32_t a = 0; a < n; ++a) {
    for (int32_t j = off[a]; j < off[a + 1]; ++j) {
      int32_t b = idx[j];
      int64_t db = (int64_t)off[b + 1] - off[b];
      if (cap >= 0 && db > cap) continue;
      ++ka;
      for (int32_t q = off[b]; q < off[b + 1]; ++q) {
        int32_t c = idx[q];
        if (mode == 0 ? (c > a) : (c != a)) ++w;
      }
    }
  }
  *wedges = w;
  *kept_arcs = ka;
}

/* Ordering used by both modes, exposed for the selection tests:
 * returns 1 if x ranks strictly before y. */
int lpo_better(const lpo_link* x, const lpo_link* y) { return better(x, y); }

int lpo_sizeof_link(void) { return (int)sizeof(lpo_link); }
