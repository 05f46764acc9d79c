/*
 * Seeded synthetic graph generators and the hold-out split.
 *
 * Test and benchmark infrastructure shared by the CPU oracle side and the
 * CUDA side: it produces inputs only and contains none of the link
 * prediction arithmetic.  Every random draw comes from one counter-based
 * generator (SplitMix64 applied to seed, stream and index), so the graphs are
 * identical for any thread count and on any host architecture.
 *
 * Graph classes stand in for the paper's web, social and road inputs
 * (Section 5.1.3, Table 1): R-MAT (web-like), Chung-Lu power law
 * (social-like) and a 4-neighbour grid (road-like).  Every graph is made
 * undirected, loses its self-loops and duplicate edges, and is stored as a CSR
 * with int32 offsets and indices and sorted adjacency lists (Section 5.1.3).
 * The hold-out split removes a uniform sample of undirected edges, without
 * replacement (Section 5.1.4).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- RNG --- */

/* SplitMix64 finaliser (Steele, Lea and Flood, 2014). */
static inline uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* The i-th draw of stream `stream` under `seed`. */
static inline uint64_t rng_u64(uint64_t seed, uint64_t stream, uint64_t i) {
  return mix64(mix64(seed ^ (stream * 0xD1B54A32D192ED03ull)) + i);
}

/* Uniform double in [0, 1) with 53 random bits. */
static inline double rng_unit(uint64_t seed, uint64_t stream, uint64_t i) {
  return (double)(rng_u64(seed, stream, i) >> 11) * (1.0 / 9007199254740992.0);
}

uint64_t lpi_rng_u64(uint64_t seed, uint64_t stream, uint64_t i) {
  return rng_u64(seed, stream, i);
}

/* ----------------------------------------------------- edge generators --- */

/*
 * R-MAT edge samples: each of the `m` samples descends `scale` levels of the
 * adjacency matrix, picking a quadrant with probabilities (a, b, c, 1-a-b-c).
 * Level l of sample i uses draw (i * scale + l) of stream 1.
 */
void lpi_rmat_edges(int32_t scale, int64_t m, double a, double b, double c,
                    uint64_t seed, int32_t* u, int32_t* v) {
  const double ab = a + b, abc = a + b + c;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < m; ++i) {
    uint32_t uu = 0, vv = 0;
    for (int32_t l = 0; l < scale; ++l) {
      double r = rng_unit(seed, 1, (uint64_t)i * (uint64_t)scale + (uint64_t)l);
      uint32_t bu, bv;
      if (r < a) { bu = 0; bv = 0; }
      else if (r < ab) { bu = 0; bv = 1; }
      else if (r < abc) { bu = 1; bv = 0; }
      else { bu = 1; bv = 1; }
      uu = (uu << 1) | bu;
      vv = (vv << 1) | bv;
    }
    u[i] = (int32_t)uu;
    v[i] = (int32_t)vv;
  }
}

/*
 * Chung-Lu expected-degree weights w_i = C (i + i0)^(-1/(gamma-1)), scaled
 * so that sum w_i = n * mean_deg.  If dmax > 0, i0 is chosen by bisection so
 * that the largest weight w_0 equals dmax (when that is reachable); else
 * i0 = 1.  Writes the cumulative distribution cdf[0..n) (last entry 1).
 */
static double chung_lu_w0(int32_t n, double alpha, double mean_deg, double i0) {
  double s = 0.0;
  for (int32_t i = 0; i < n; ++i) s += pow((double)i + i0, -alpha);
  return (double)n * mean_deg * pow(i0, -alpha) / s;
}

double lpi_chung_lu_i0(int32_t n, double gamma, double mean_deg, double dmax) {
  const double alpha = 1.0 / (gamma - 1.0);
  if (dmax <= 0.0) return 1.0;
  double lo = 1e-3, hi = (double)n;
  if (chung_lu_w0(n, alpha, mean_deg, lo) <= dmax) return lo;
  for (int it = 0; it < 200; ++it) {
    double mid = sqrt(lo * hi);
    if (chung_lu_w0(n, alpha, mean_deg, mid) > dmax) lo = mid; else hi = mid;
  }
  return hi;
}

static void chung_lu_cdf(int32_t n, double gamma, double i0, double* cdf) {
  const double alpha = 1.0 / (gamma - 1.0);
  double s = 0.0;
  for (int32_t i = 0; i < n; ++i) { s += pow((double)i + i0, -alpha); cdf[i] = s; }
  for (int32_t i = 0; i < n; ++i) cdf[i] /= s;
  cdf[n - 1] = 1.0;
}

static inline int32_t cdf_pick(const double* cdf, int32_t n, double r) {
  int32_t lo = 0, hi = n - 1;            /* first index with cdf > r */
  while (lo < hi) {
    int32_t mid = lo + (hi - lo) / 2;
    if (cdf[mid] > r) hi = mid; else lo = mid + 1;
  }
  return lo;
}

static int cmp_u64(const void* x, const void* y) {
  uint64_t a = *(const uint64_t*)x, b = *(const uint64_t*)y;
  return (a > b) - (a < b);
}

/* Sort + unique of packed (min<<32 | max) undirected keys; returns the count. */
static int64_t sort_unique(uint64_t* k, int64_t m) {
  qsort(k, (size_t)m, sizeof(uint64_t), cmp_u64);
  int64_t w = 0;
  for (int64_t i = 0; i < m; ++i)
    if (w == 0 || k[w - 1] != k[i]) k[w++] = k[i];
  return w;
}

/*
 * Chung-Lu graph with exactly `m_target` distinct undirected edges (unless
 * 64 top-up rounds do not reach it): both endpoints of each sample are drawn
 * from the weight distribution, self-loops and duplicates are dropped, and the
 * deficit is re-sampled from fresh counters.  Writes the edges as u < v pairs
 * (sorted) and returns their count.  `u`, `v` must hold m_target entries.
 */
int64_t lpi_chung_lu_edges(int32_t n, double gamma, double i0, int64_t m_target,
                           uint64_t seed, int32_t* u, int32_t* v) {
  double* cdf = (double*)malloc(sizeof(double) * (size_t)n);
  uint64_t* keys = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(2 * m_target + 64));
  if (!cdf || !keys) { free(cdf); free(keys); return -1; }
  chung_lu_cdf(n, gamma, i0, cdf);
  int64_t have = 0;
  uint64_t counter = 0;
  for (int round = 0; round < 64 && have < m_target; ++round) {
    int64_t need = m_target - have;
    int64_t draw = need;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < draw; ++i) {
      uint64_t id = counter + (uint64_t)i;
      int32_t x = cdf_pick(cdf, n, rng_unit(seed, 2, 2 * id));
      int32_t y = cdf_pick(cdf, n, rng_unit(seed, 2, 2 * id + 1));
      uint64_t lo = (uint64_t)(x < y ? x : y), hi = (uint64_t)(x < y ? y : x);
      keys[have + i] = (x == y) ? ~0ull : ((lo << 32) | hi);
    }
    counter += (uint64_t)draw;
    int64_t tot = sort_unique(keys, have + draw);
    if (tot > 0 && keys[tot - 1] == ~0ull) --tot;   /* drop the self-loop marker */
    have = tot;
  }
  if (have > m_target) have = m_target;
  for (int64_t i = 0; i < have; ++i) {
    u[i] = (int32_t)(keys[i] >> 32);
    v[i] = (int32_t)(keys[i] & 0xffffffffu);
  }
  free(cdf);
  free(keys);
  return have;
}

/* rows x cols 4-neighbour grid, vertex id r * cols + c; writes u < v pairs. */
int64_t lpi_grid_edges(int32_t rows, int32_t cols, int32_t* u, int32_t* v) {
  int64_t w = 0;
  for (int32_t r = 0; r < rows; ++r)
    for (int32_t c = 0; c < cols; ++c) {
      int32_t id = r * cols + c;
      if (c + 1 < cols) { u[w] = id; v[w] = id + 1; ++w; }
      if (r + 1 < rows) { u[w] = id; v[w] = id + cols; ++w; }
    }
  return w;
}

/* Seeded Fisher-Yates permutation of 0..n-1 (stream 3). */
void lpi_permutation(int32_t n, uint64_t seed, int32_t* perm) {
  for (int32_t i = 0; i < n; ++i) perm[i] = i;
  for (int32_t i = n - 1; i > 0; --i) {
    int32_t j = (int32_t)(rng_u64(seed, 3, (uint64_t)i) % (uint64_t)(i + 1));
    int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
  }
}

/* ------------------------------------------------------------ CSR build --- */

static int cmp_i32(const void* x, const void* y) {
  int32_t a = *(const int32_t*)x, b = *(const int32_t*)y;
  return (a > b) - (a < b);
}

static void sort_list(int32_t* p, int64_t len) {
  if (len <= 24) {
    for (int64_t i = 1; i < len; ++i) {
      int32_t x = p[i];
      int64_t j = i - 1;
      while (j >= 0 && p[j] > x) { p[j + 1] = p[j]; --j; }
      p[j + 1] = x;
    }
  } else {
    qsort(p, (size_t)len, sizeof(int32_t), cmp_i32);
  }
}

/*
 * Symmetric CSR from m edge samples (u[i], v[i]): both directions are
 * inserted, self-loops dropped, each adjacency list sorted and deduplicated.
 * If perm != NULL every endpoint x is renamed perm[x] first.
 * Pass 1 (idx == NULL): writes the deduplicated degrees into off[1..n] and
 * returns the arc count A.  The caller allocates idx[A] and calls again with
 * the same arguments (pass 2), which fills off[0..n] and idx.
 * scratch must hold 2*m int32 (used only in pass 2); returns -1 on overflow.
 */
int64_t lpi_build_csr(int32_t n, int64_t m, const int32_t* u, const int32_t* v,
                      const int32_t* perm, int32_t* off, int32_t* idx,
                      int32_t* scratch) {
  int64_t* cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  if (!cnt) return -1;
  for (int64_t i = 0; i < m; ++i) {
    int32_t x = perm ? perm[u[i]] : u[i], y = perm ? perm[v[i]] : v[i];
    if (x == y) continue;
    cnt[x + 1]++; cnt[y + 1]++;
  }
  for (int32_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
  int64_t raw = cnt[n];
  int32_t* buf = scratch;
  int64_t* cur = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  int32_t* dd = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  if (!cur || !dd) { free(cnt); free(cur); free(dd); return -1; }
  int local_buf = 0;
  if (!buf) {
    buf = (int32_t*)malloc(sizeof(int32_t) * (size_t)(raw > 0 ? raw : 1));
    if (!buf) { free(cnt); free(cur); free(dd); return -1; }
    local_buf = 1;
  }
  for (int32_t i = 0; i < n; ++i) cur[i] = cnt[i];
  for (int64_t i = 0; i < m; ++i) {
    int32_t x = perm ? perm[u[i]] : u[i], y = perm ? perm[v[i]] : v[i];
    if (x == y) continue;
    buf[cur[x]++] = y;
    buf[cur[y]++] = x;
  }
#pragma omp parallel for schedule(dynamic, 1024)
  for (int32_t i = 0; i < n; ++i) {
    int32_t* p = buf + cnt[i];
    int64_t len = cnt[i + 1] - cnt[i];
    sort_list(p, len);
    int64_t w = 0;
    for (int64_t j = 0; j < len; ++j)
      if (w == 0 || p[w - 1] != p[j]) p[w++] = p[j];
    dd[i] = (int32_t)w;
  }
  int64_t total = 0;
  for (int32_t i = 0; i < n; ++i) total += dd[i];
  if (total >= 2147483647ll) total = -1;
  if (total >= 0) {
    off[0] = 0;
    for (int32_t i = 0; i < n; ++i) off[i + 1] = off[i] + dd[i];
    if (idx) {
#pragma omp parallel for schedule(dynamic, 1024)
      for (int32_t i = 0; i < n; ++i)
        memcpy(idx + off[i], buf + cnt[i], sizeof(int32_t) * (size_t)dd[i]);
    }
  }
  if (local_buf) free(buf);
  free(cnt); free(cur); free(dd);
  return total;
}

/* ------------------------------------------------------------- hold-out --- */

typedef struct { uint64_t key; int64_t e; int32_t x, j; } keyed_t;

static int cmp_keyed(const void* x, const void* y) {
  const keyed_t* a = (const keyed_t*)x;
  const keyed_t* b = (const keyed_t*)y;
  if (a->key != b->key) return (a->key > b->key) - (a->key < b->key);
  return (a->e > b->e) - (a->e < b->e);
}

/*
 * Uniform sample of k of the undirected edges (u < v) of a symmetric CSR,
 * without replacement: the e-th (u < v) arc in CSR order gets key
 * rng(seed, 4, e) and the k smallest (key, e) are taken.  Marks the chosen
 * arcs in held[A] (both directions) and writes the pairs to hu/hv in
 * increasing key order.  Returns k, or -1 on allocation failure.
 */
int64_t lpi_holdout(int32_t n, const int32_t* off, const int32_t* idx, int64_t k,
                    uint64_t seed, uint8_t* held, int32_t* hu, int32_t* hv) {
  int64_t A = off[n];
  memset(held, 0, (size_t)A);
  int64_t* ue = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1));
  if (!ue) return -1;
  /* ue[x] = number of (x < y) arcs before vertex x */
  int64_t m = 0;
  for (int32_t x = 0; x < n; ++x) {
    ue[x] = m;
    for (int32_t j = off[x]; j < off[x + 1]; ++j) if (idx[j] > x) ++m;
  }
  ue[n] = m;
  if (k > m) k = m;
  if (k <= 0) { free(ue); return 0; }
  /* Threshold pre-filter: keys are uniform, so the k smallest lie below
   * t = (k/m)(1+slack) * 2^64 with overwhelming probability; retry wider. */
  double slack = 0.05 + 8.0 / sqrt((double)k);
  keyed_t* sel = NULL;
  int64_t ns = 0;
  for (int attempt = 0; attempt < 64; ++attempt) {
    double frac = (double)k / (double)m * (1.0 + slack);
    uint64_t t = frac >= 1.0 ? ~0ull : (uint64_t)(frac * 18446744073709551616.0);
    ns = 0;
#pragma omp parallel for reduction(+ : ns) schedule(static)
    for (int64_t e = 0; e < m; ++e) if (rng_u64(seed, 4, (uint64_t)e) <= t) ++ns;
    if (ns >= k || frac >= 1.0) {
      sel = (keyed_t*)malloc(sizeof(keyed_t) * (size_t)(ns > 0 ? ns : 1));
      if (!sel) { free(ue); return -1; }
      int64_t w = 0;
      for (int32_t x = 0; x < n; ++x) {
        int64_t e = ue[x];
        for (int32_t j = off[x]; j < off[x + 1]; ++j) {
          if (idx[j] <= x) continue;
          uint64_t key = rng_u64(seed, 4, (uint64_t)e);
          if (key <= t) { sel[w].key = key; sel[w].e = e; sel[w].x = x; sel[w].j = j; ++w; }
          ++e;
        }
      }
      break;
    }
    slack *= 2.0;
  }
  if (!sel) { free(ue); return -1; }
  qsort(sel, (size_t)ns, sizeof(keyed_t), cmp_keyed);
  for (int64_t i = 0; i < k; ++i) {
    int32_t x = sel[i].x, jx = sel[i].j, y = idx[jx];
    held[jx] = 1;
    /* reverse arc: x in the sorted list of y */
    int32_t l2 = off[y], h2 = off[y + 1] - 1;
    while (l2 < h2) {
      int32_t mid = l2 + (h2 - l2) / 2;
      if (idx[mid] < x) l2 = mid + 1; else h2 = mid;
    }
    held[l2] = 1;
    hu[i] = x;
    hv[i] = y;
  }
  free(sel);
  free(ue);
  return k;
}

/* Observed CSR: the input CSR without the arcs marked in held[]. */
int64_t lpi_filter_csr(int32_t n, const int32_t* off, const int32_t* idx,
                       const uint8_t* held, int32_t* off_out, int32_t* idx_out) {
  int64_t w = 0;
  off_out[0] = 0;
  for (int32_t x = 0; x < n; ++x) {
    for (int32_t j = off[x]; j < off[x + 1]; ++j)
      if (!held[j]) idx_out[w++] = idx[j];
    off_out[x + 1] = (int32_t)w;
  }
  return w;
}
