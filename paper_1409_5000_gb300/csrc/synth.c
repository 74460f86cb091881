/*
 * Seeded synthetic graph generators (host C, no CUDA).
 *
 * These produce the inputs that BOTH the CUDA path and the FP64 oracle
 * consume.  They contain none of the method's arithmetic: only random
 * background graphs (Erdos-Renyi, Barabasi-Albert, Watts-Strogatz), the
 * embedded target (random tree plus extra edges, or a clique) and a
 * symmetric CSR builder.
 *
 * Paper context: the backgrounds and the embedded target follow the
 * paper's experimental set-up ("Multiple backgrounds scenario" and
 * "Single background scenario", Tables 1-3): ER/SW/BA backgrounds with a
 * target sub-graph OR-ed into every realisation, target nodes placed
 * uniformly at random.  Generator conventions the paper leaves open
 * (p = dbar/(n-1) for ER, BA seeded with m0 isolated nodes, WS with k/2
 * neighbours per side) are the readings stated in the design notes.
 *
 * RNG: SplitMix64 (Steele, Lea, Flood 2014), one stream per generator
 * call, seeded by the caller.  Uniform doubles use the top 53 bits.
 *
 * Usage protocol (two calls, so that Python owns the output memory):
 *   h = cbs_*_begin(...)        -> builds an undirected edge list
 *   cbs_add_edges(h, ...)       -> optional: OR-in target edges
 *   nnz = cbs_finish_count(h)   -> dedupes, returns directed entry count
 *   cbs_finish_fill(h, row_ptr, col) -> writes CSR, frees h
 * Errors: *_begin returns NULL on bad arguments or allocation failure;
 * cbs_finish_count returns -1 on allocation failure.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static inline uint64_t sm64_next(uint64_t *s) {
  uint64_t z = (*s += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
static inline double sm64_unit(uint64_t *s) { /* [0,1) */
  return (double)(sm64_next(s) >> 11) * (1.0 / 9007199254740992.0);
}
static inline uint64_t sm64_below(uint64_t *s, uint64_t bound) { /* [0,bound) */
  /* Lemire-style multiply-high would need 128-bit; use rejection. */
  uint64_t lim = UINT64_MAX - (UINT64_MAX % bound);
  uint64_t x;
  do { x = sm64_next(s); } while (x >= lim);
  return x % bound;
}

/* Exposed so Python can derive per-realisation seeds from one base. */
/* `count` consecutive SplitMix64 outputs from state `seed` (the sequential
 * form of the generator; the counter form used for on-device generation is
 * output(c) = mix(seed + (c + 1) * golden)). */
int cbs_sm64_stream(uint64_t seed, uint64_t count, uint64_t *out) {
  uint64_t s = seed;
  for (uint64_t i = 0; i < count; ++i) out[i] = sm64_next(&s);
  return 0;
}

uint64_t cbs_mix(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t s = a;
  uint64_t x = sm64_next(&s);
  s = x ^ (b * 0xD1B54A32D192ED03ULL);
  x = sm64_next(&s);
  s = x ^ (c * 0x8CB92BA72F3D8DD7ULL);
  return sm64_next(&s);
}

typedef struct {
  uint32_t n;
  uint64_t ne, cap; /* undirected edges (u,v), u != v */
  uint32_t *eu, *ev;
  /* filled by finish_count */
  uint32_t *deg;     /* n entries, deduplicated degree */
  uint32_t *tmp_col; /* raw directed adjacency before dedupe */
  uint64_t *tmp_ptr; /* n+1 */
  uint64_t nnz;
} cbs_graph;

static int push_edge(cbs_graph *g, uint32_t u, uint32_t v) {
  if (g->ne == g->cap) {
    uint64_t nc = g->cap ? g->cap * 2 : 1024;
    uint32_t *a = (uint32_t *)realloc(g->eu, nc * sizeof(uint32_t));
    if (!a) return -1;
    g->eu = a;
    uint32_t *b = (uint32_t *)realloc(g->ev, nc * sizeof(uint32_t));
    if (!b) return -1;
    g->ev = b;
    g->cap = nc;
  }
  g->eu[g->ne] = u;
  g->ev[g->ne] = v;
  g->ne++;
  return 0;
}

static cbs_graph *new_graph(uint32_t n, uint64_t cap_hint) {
  cbs_graph *g = (cbs_graph *)calloc(1, sizeof(cbs_graph));
  if (!g) return NULL;
  g->n = n;
  if (cap_hint) {
    g->eu = (uint32_t *)malloc(cap_hint * sizeof(uint32_t));
    g->ev = (uint32_t *)malloc(cap_hint * sizeof(uint32_t));
    if (!g->eu || !g->ev) { free(g->eu); free(g->ev); free(g); return NULL; }
    g->cap = cap_hint;
  }
  return g;
}

uint32_t cbs_n(const cbs_graph *g) { return g->n; }

void cbs_free(cbs_graph *g) {
  if (!g) return;
  free(g->eu); free(g->ev); free(g->deg); free(g->tmp_col); free(g->tmp_ptr);
  free(g);
}

cbs_graph *cbs_empty_begin(uint32_t n) { return new_graph(n, 0); }

/* Erdos-Renyi G(n,p) by geometric skipping over the lower triangle
 * (Batagelj & Brandes, Phys. Rev. E 71, 036113, 2005). */
cbs_graph *cbs_er_begin(uint32_t n, double p, uint64_t seed) {
  if (n == 0 || !(p >= 0.0) || p > 1.0) return NULL;
  double mean = p * 0.5 * (double)n * (double)(n - 1);
  uint64_t hint = (uint64_t)(mean + 6.0 * sqrt(mean + 1.0)) + 16;
  cbs_graph *g = new_graph(n, hint);
  if (!g) return NULL;
  if (p <= 0.0 || n < 2) return g;
  uint64_t s = seed;
  if (p >= 1.0) {
    for (uint32_t v = 1; v < n; ++v)
      for (uint32_t w = 0; w < v; ++w)
        if (push_edge(g, v, w)) { cbs_free(g); return NULL; }
    return g;
  }
  double lq = log1p(-p);
  int64_t v = 1, w = -1;
  while (v < (int64_t)n) {
    double r = sm64_unit(&s);
    w += 1 + (int64_t)floor(log1p(-r) / lq);
    while (w >= v && v < (int64_t)n) { w -= v; v += 1; }
    if (v < (int64_t)n)
      if (push_edge(g, (uint32_t)v, (uint32_t)w)) { cbs_free(g); return NULL; }
  }
  return g;
}

/* Barabasi-Albert: m0 = m isolated seed nodes; node t >= m attaches to m
 * distinct earlier nodes chosen with probability proportional to degree
 * (repeated-endpoint list); the first new node links to all m seeds. */
cbs_graph *cbs_ba_begin(uint32_t n, uint32_t m, uint64_t seed) {
  if (m == 0 || n <= m) return NULL;
  uint64_t ne = (uint64_t)(n - m) * m;
  cbs_graph *g = new_graph(n, ne);
  if (!g) return NULL;
  uint32_t *ends = (uint32_t *)malloc(2 * ne * sizeof(uint32_t));
  uint32_t *pick = (uint32_t *)malloc(m * sizeof(uint32_t));
  if (!ends || !pick) { free(ends); free(pick); cbs_free(g); return NULL; }
  uint64_t nends = 0, s = seed;
  for (uint32_t t = m; t < n; ++t) {
    uint32_t k = 0;
    if (t == m) {
      for (uint32_t i = 0; i < m; ++i) pick[k++] = i;
    } else {
      while (k < m) {
        uint32_t c = ends[sm64_below(&s, nends)];
        int dup = 0;
        for (uint32_t i = 0; i < k; ++i) dup |= (pick[i] == c);
        if (!dup) pick[k++] = c;
      }
    }
    for (uint32_t i = 0; i < m; ++i) {
      g->eu[g->ne] = t; g->ev[g->ne] = pick[i]; g->ne++;
      ends[nends++] = t; ends[nends++] = pick[i];
    }
  }
  free(ends); free(pick);
  return g;
}

/* open-addressing set of undirected edge keys, used by WS rewiring */
typedef struct { uint64_t *k; uint64_t mask; } eset;
static inline uint64_t ekey(uint32_t a, uint32_t b) {
  return a < b ? ((uint64_t)a << 32) | b : ((uint64_t)b << 32) | a;
}
static inline uint64_t hmix(uint64_t x) {
  x ^= x >> 33; x *= 0xff51afd7ed558ccdULL; x ^= x >> 33; return x;
}
static int eset_has(const eset *s, uint64_t key) {
  uint64_t i = hmix(key) & s->mask;
  while (s->k[i] != UINT64_MAX) { if (s->k[i] == key) return 1; i = (i + 1) & s->mask; }
  return 0;
}
static void eset_put(eset *s, uint64_t key) {
  uint64_t i = hmix(key) & s->mask;
  while (s->k[i] != UINT64_MAX) { if (s->k[i] == key) return; i = (i + 1) & s->mask; }
  s->k[i] = key;
}
static void eset_del(eset *s, uint64_t key) { /* backward-shift deletion */
  uint64_t i = hmix(key) & s->mask;
  while (s->k[i] != key) { if (s->k[i] == UINT64_MAX) return; i = (i + 1) & s->mask; }
  uint64_t j = i;
  for (;;) {
    j = (j + 1) & s->mask;
    if (s->k[j] == UINT64_MAX) break;
    uint64_t h = hmix(s->k[j]) & s->mask;
    /* can k[j] move to i? only if h is not cyclically in (i, j] */
    int in = (i <= j) ? (h > i && h <= j) : (h > i || h <= j);
    if (!in) { s->k[i] = s->k[j]; i = j; }
  }
  s->k[i] = UINT64_MAX;
}

/* Watts-Strogatz: ring lattice, k/2 neighbours per side; each lattice
 * edge (i, i+j) is rewired with probability p to (i, w), w uniform among
 * nodes that are neither i nor current neighbours of i. */
cbs_graph *cbs_ws_begin(uint32_t n, uint32_t k, double p, uint64_t seed) {
  if (k < 2 || (k & 1) || k >= n || !(p >= 0.0) || p > 1.0) return NULL;
  uint32_t h = k / 2;
  uint64_t ne = (uint64_t)n * h;
  cbs_graph *g = new_graph(n, ne);
  if (!g) return NULL;
  uint64_t cap = 1; while (cap < 4 * ne) cap <<= 1;
  eset S; S.k = (uint64_t *)malloc(cap * sizeof(uint64_t)); S.mask = cap - 1;
  uint32_t *cur = (uint32_t *)malloc(ne * sizeof(uint32_t)); /* edge e = (src[e], cur[e]) */
  uint32_t *deg = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
  if (!S.k || !cur || !deg) { free(S.k); free(cur); free(deg); cbs_free(g); return NULL; }
  memset(S.k, 0xff, cap * sizeof(uint64_t));
  for (uint32_t i = 0; i < n; ++i) deg[i] = k;
  for (uint32_t j = 1; j <= h; ++j)
    for (uint32_t i = 0; i < n; ++i) {
      uint32_t t = (uint32_t)(((uint64_t)i + j) % n);
      cur[(uint64_t)(j - 1) * n + i] = t;
      eset_put(&S, ekey(i, t));
    }
  uint64_t s = seed;
  for (uint32_t j = 1; j <= h; ++j)
    for (uint32_t i = 0; i < n; ++i) {
      uint64_t e = (uint64_t)(j - 1) * n + i;
      if (sm64_unit(&s) >= p) continue;
      if (deg[i] >= n - 1) continue; /* no free target */
      uint32_t w;
      for (;;) {
        w = (uint32_t)sm64_below(&s, n);
        if (w != i && !eset_has(&S, ekey(i, w))) break;
      }
      uint32_t old = cur[e];
      eset_del(&S, ekey(i, old));
      eset_put(&S, ekey(i, w));
      deg[old]--; deg[w]++;
      cur[e] = w;
    }
  for (uint32_t j = 1; j <= h; ++j)
    for (uint32_t i = 0; i < n; ++i) {
      g->eu[g->ne] = i; g->ev[g->ne] = cur[(uint64_t)(j - 1) * n + i]; g->ne++;
    }
  free(S.k); free(cur); free(deg);
  return g;
}

/* OR extra undirected edges into the graph (duplicates collapse later). */
int cbs_add_edges(cbs_graph *g, const uint32_t *u, const uint32_t *v, uint64_t cnt) {
  for (uint64_t i = 0; i < cnt; ++i) {
    if (u[i] >= g->n || v[i] >= g->n || u[i] == v[i]) return -2;
    if (push_edge(g, u[i], v[i])) return -1;
  }
  return 0;
}

/* Target sub-graph on a node set: a random recursive tree over a seeded
 * permutation of the nodes plus `extra` edges drawn uniformly among the
 * non-edges of the set; or, if clique != 0, all pairs.  Writes up to
 * cap edges into (eu, ev) and returns their count (or -1). */
int64_t cbs_target_edges(const uint32_t *nodes, uint32_t k, uint32_t extra,
                         int clique, uint64_t seed, uint32_t *eu, uint32_t *ev,
                         uint64_t cap) {
  uint64_t cnt = 0;
  if (k < 2) return 0;
  if (clique) {
    if ((uint64_t)k * (k - 1) / 2 > cap) return -1;
    for (uint32_t a = 0; a < k; ++a)
      for (uint32_t b = a + 1; b < k; ++b) { eu[cnt] = nodes[a]; ev[cnt] = nodes[b]; cnt++; }
    return (int64_t)cnt;
  }
  uint64_t maxe = (uint64_t)k * (k - 1) / 2;
  if (extra > maxe - (k - 1)) extra = (uint32_t)(maxe - (k - 1));
  if ((uint64_t)(k - 1) + extra > cap) return -1;
  uint32_t *perm = (uint32_t *)malloc(k * sizeof(uint32_t));
  unsigned char *adj = (unsigned char *)calloc((size_t)k * k, 1);
  if (!perm || !adj) { free(perm); free(adj); return -1; }
  uint64_t s = seed;
  for (uint32_t i = 0; i < k; ++i) perm[i] = i;
  for (uint32_t i = k - 1; i > 0; --i) {
    uint32_t j = (uint32_t)sm64_below(&s, (uint64_t)i + 1);
    uint32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
  }
  for (uint32_t i = 1; i < k; ++i) {
    uint32_t par = perm[sm64_below(&s, i)];
    uint32_t ch = perm[i];
    adj[(size_t)par * k + ch] = adj[(size_t)ch * k + par] = 1;
    eu[cnt] = nodes[par]; ev[cnt] = nodes[ch]; cnt++;
  }
  for (uint32_t x = 0; x < extra; ++x) {
    uint32_t a, b;
    do {
      a = (uint32_t)sm64_below(&s, k);
      b = (uint32_t)sm64_below(&s, k);
    } while (a == b || adj[(size_t)a * k + b]);
    adj[(size_t)a * k + b] = adj[(size_t)b * k + a] = 1;
    eu[cnt] = nodes[a]; ev[cnt] = nodes[b]; cnt++;
  }
  free(perm); free(adj);
  return (int64_t)cnt;
}

/* k distinct node indices drawn uniformly from [0, range), sorted. */
int cbs_sample_nodes(uint32_t range, uint32_t k, uint64_t seed, uint32_t *out) {
  if (k > range) return -1;
  uint64_t s = seed;
  uint32_t cnt = 0;
  while (cnt < k) {
    uint32_t c = (uint32_t)sm64_below(&s, range);
    int dup = 0;
    for (uint32_t i = 0; i < cnt; ++i) dup |= (out[i] == c);
    if (!dup) out[cnt++] = c;
  }
  for (uint32_t i = 1; i < k; ++i) { /* insertion sort */
    uint32_t x = out[i]; int32_t j = (int32_t)i - 1;
    while (j >= 0 && out[j] > x) { out[j + 1] = out[j]; --j; }
    out[j + 1] = x;
  }
  return 0;
}

static int cmp_u32(const void *x, const void *y) {
  uint32_t a = *(const uint32_t *)x, b = *(const uint32_t *)y;
  return (a > b) - (a < b);
}
static void sort_u32(uint32_t *a, uint64_t n) {
  if (n > 48) { qsort(a, (size_t)n, sizeof(uint32_t), cmp_u32); return; }
  for (uint64_t i = 1; i < n; ++i) {
    uint32_t x = a[i]; int64_t j = (int64_t)i - 1;
    while (j >= 0 && a[j] > x) { a[j + 1] = a[j]; --j; }
    a[j + 1] = x;
  }
}

/* Build the deduplicated symmetric adjacency; returns the number of
 * directed CSR entries (2|E| after collapsing duplicates). */
int64_t cbs_finish_count(cbs_graph *g) {
  uint32_t n = g->n;
  g->tmp_ptr = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
  g->deg = (uint32_t *)calloc((size_t)n, sizeof(uint32_t));
  if (!g->tmp_ptr || !g->deg) return -1;
  for (uint64_t e = 0; e < g->ne; ++e) { g->tmp_ptr[g->eu[e] + 1]++; g->tmp_ptr[g->ev[e] + 1]++; }
  for (uint32_t i = 0; i < n; ++i) g->tmp_ptr[i + 1] += g->tmp_ptr[i];
  g->tmp_col = (uint32_t *)malloc((g->tmp_ptr[n] ? g->tmp_ptr[n] : 1) * sizeof(uint32_t));
  uint64_t *fillp = (uint64_t *)malloc(((size_t)n + 1) * sizeof(uint64_t));
  if (!g->tmp_col || !fillp) { free(fillp); return -1; }
  memcpy(fillp, g->tmp_ptr, ((size_t)n + 1) * sizeof(uint64_t));
  for (uint64_t e = 0; e < g->ne; ++e) {
    g->tmp_col[fillp[g->eu[e]]++] = g->ev[e];
    g->tmp_col[fillp[g->ev[e]]++] = g->eu[e];
  }
  free(fillp);
  free(g->eu); free(g->ev); g->eu = g->ev = NULL;
  uint64_t tot = 0;
  for (uint32_t i = 0; i < n; ++i) {
    uint32_t *r = g->tmp_col + g->tmp_ptr[i];
    uint64_t len = g->tmp_ptr[i + 1] - g->tmp_ptr[i];
    sort_u32(r, len);
    uint32_t d = 0;
    for (uint64_t t = 0; t < len; ++t)
      if (t == 0 || r[t] != r[t - 1]) r[d++] = r[t];
    g->deg[i] = d;
    tot += d;
  }
  g->nnz = tot;
  return (int64_t)tot;
}

/* Write CSR (row_ptr: n+1 u32 when nnz < 2^32, col: nnz u32) and free g. */
int cbs_finish_fill(cbs_graph *g, uint32_t *row_ptr, uint32_t *col) {
  if (g->nnz >= 0xffffffffULL) { cbs_free(g); return -1; }
  uint64_t off = 0;
  for (uint32_t i = 0; i < g->n; ++i) {
    row_ptr[i] = (uint32_t)off;
    memcpy(col + off, g->tmp_col + g->tmp_ptr[i], (size_t)g->deg[i] * sizeof(uint32_t));
    off += g->deg[i];
  }
  row_ptr[g->n] = (uint32_t)off;
  cbs_free(g);
  return 0;
}
