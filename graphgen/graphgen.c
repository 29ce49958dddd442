/*
 * graphgen.c -- seeded synthetic graph generators shared by the CPU oracle tests and the GPU
 * path's tests and benchmark.  This file holds NO arithmetic of the Louvain method: it only
 * draws graphs and lays them out as symmetric CSR.
 *
 * Randomness is counter based: every draw is gg_hash3(seed, stream, index), built from the
 * SplitMix64 output function (Steele, Lea and Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014: add the golden gamma 0x9e3779b97f4a7c15, then the two
 * xor-shift-multiply rounds with 0xbf58476d1ce4e5b9 / 0x94d049bb133111eb and shifts 30, 27, 31).
 * Nothing depends on the platform's libm: the one logarithm needed (geometric skipping) is
 * computed below from IEEE + - * / only, and the file must be compiled with
 * -ffp-contract=off, so x86-64 and aarch64 hosts produce bit-identical graphs.
 *
 * Graph convention (the paper's, Section 3): undirected, every edge stored as two arcs, rows
 * sorted by target, no duplicate arcs, no self-loops in generated inputs.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GG_GAMMA 0x9e3779b97f4a7c15ULL

static inline uint64_t gg_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

/* i-th output of a SplitMix64 stream seeded with s: mix(s + (i+1)*gamma). */
uint64_t gg_splitmix64_nth(uint64_t seed, uint64_t i) { return gg_mix(seed + (i + 1) * GG_GAMMA); }

/* Three-word counter hash: x = mix(a + g); x = mix(x + b + 2g); return mix(x + c + 3g). */
uint64_t gg_hash3(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t x = gg_mix(a + GG_GAMMA);
  x = gg_mix(x + b + 2 * GG_GAMMA);
  return gg_mix(x + c + 3 * GG_GAMMA);
}

/* Uniform in (0, 1]: ((h >> 11) + 1) * 2^-53. */
static inline double gg_u01(uint64_t h) { return (double)((h >> 11) + 1) * (1.0 / 9007199254740992.0); }

/* Natural log from basic IEEE operations only: x = m * 2^e with m in [sqrt(1/2), sqrt(2)),
 * ln x = e ln 2 + 2 atanh((m-1)/(m+1)), atanh by its odd power series (|s| <= 0.1716, 12 terms
 * leave < 1e-19).  Only its determinism matters here, not its last-bit accuracy. */
double gg_log(double x) {
  if (!(x > 0.0)) return -1.0e308;
  int e = 0;
  while (x >= 1.4142135623730951) { x *= 0.5; e++; }
  while (x < 0.7071067811865476) { x *= 2.0; e--; }
  double s = (x - 1.0) / (x + 1.0), s2 = s * s, term = s, sum = 0.0;
  for (int k = 1; k <= 23; k += 2) { sum += term / (double)k; term *= s2; }
  return (double)e * 0.6931471805599453 + 2.0 * sum;
}

/* exp from basic operations: x = k ln2 + r, |r| <= ln2/2, Taylor series to r^20. */
double gg_exp(double x) {
  if (x > 700.0) x = 700.0;
  if (x < -700.0) return 0.0;
  double kf = x / 0.6931471805599453;
  long k = (long)(kf < 0 ? kf - 0.5 : kf + 0.5);
  double r = x - (double)k * 0.6931471805599453;
  double term = 1.0, sum = 1.0;
  for (int i = 1; i <= 20; i++) { term *= r / (double)i; sum += term; }
  while (k > 0) { sum *= 2.0; k--; }
  while (k < 0) { sum *= 0.5; k++; }
  return sum;
}

/* ------------------------------------------------------------------------------------------
 * Growable edge list of undirected pairs, stored as 64-bit keys (u << 32) | v with u < v.
 * ---------------------------------------------------------------------------------------- */
typedef struct { uint64_t* k; int64_t len, cap; int oom; } gg_keys;

static void keys_push(gg_keys* e, uint64_t key) {
  if (e->oom) return;
  if (e->len == e->cap) {
    int64_t nc = e->cap ? e->cap * 2 : 1 << 16;
    uint64_t* p = (uint64_t*)realloc(e->k, (size_t)nc * sizeof(uint64_t));
    if (!p) { e->oom = 1; return; }
    e->k = p; e->cap = nc;
  }
  e->k[e->len++] = key;
}

static inline void push_edge(gg_keys* e, int64_t u, int64_t v) {
  if (u == v) return;
  if (u > v) { int64_t t = u; u = v; v = t; }
  keys_push(e, ((uint64_t)u << 32) | (uint64_t)v);
}

/* LSD radix sort of 64-bit keys, 16 bits per pass (4 passes). */
static int radix_sort_u64(uint64_t* a, int64_t n) {
  if (n < 2) return 0;
  uint64_t* tmp = (uint64_t*)malloc((size_t)n * sizeof(uint64_t));
  if (!tmp) return -1;
  int64_t* cnt = (int64_t*)malloc(65536 * sizeof(int64_t));
  if (!cnt) { free(tmp); return -1; }
  uint64_t *src = a, *dst = tmp;
  for (int pass = 0; pass < 4; pass++) {
    int sh = 16 * pass;
    memset(cnt, 0, 65536 * sizeof(int64_t));
    for (int64_t i = 0; i < n; i++) cnt[(src[i] >> sh) & 0xFFFF]++;
    int64_t s = 0;
    for (int b = 0; b < 65536; b++) { int64_t c = cnt[b]; cnt[b] = s; s += c; }
    for (int64_t i = 0; i < n; i++) dst[cnt[(src[i] >> sh) & 0xFFFF]++] = src[i];
    uint64_t* t = src; src = dst; dst = t;
  }
  /* 4 passes: result is back in a */
  free(tmp); free(cnt);
  return 0;
}

/* ------------------------------------------------------------------------------------------
 * CSR result
 * ---------------------------------------------------------------------------------------- */
typedef struct {
  int64_t n, n_arcs;
  int64_t* offsets;  /* n + 1 */
  int32_t* targets;  /* n_arcs */
  int32_t* wi;       /* int32 weights (weight_kind 0 or 1), else NULL */
  float* wf;         /* fp32 weights (weight_kind 2), else NULL */
  int64_t n_edges_drawn;
} gg_csr;

void gg_free(gg_csr* g) {
  if (!g) return;
  free(g->offsets); free(g->targets); free(g->wi); free(g->wf); free(g);
}

/* weight_kind: 0 = unit int32, 1 = int32 uniform in 1..8 from gg_hash3(wseed, u, v) (u < v),
 *              2 = fp32 ((h >> 40) + 1) * 2^-24 in (0, 1] from the same hash. */
static gg_csr* csr_from_keys(gg_keys* e, int64_t n, int weight_kind, uint64_t wseed) {
  if (e->oom) return NULL;
  if (radix_sort_u64(e->k, e->len) != 0) return NULL;
  int64_t m = 0;
  for (int64_t i = 0; i < e->len; i++)
    if (m == 0 || e->k[i] != e->k[m - 1]) e->k[m++] = e->k[i];
  gg_csr* g = (gg_csr*)calloc(1, sizeof(gg_csr));
  if (!g) return NULL;
  g->n = n; g->n_arcs = 2 * m;
  g->offsets = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  g->targets = (int32_t*)malloc((size_t)(2 * m > 0 ? 2 * m : 1) * sizeof(int32_t));
  if (weight_kind == 2) g->wf = (float*)malloc((size_t)(2 * m > 0 ? 2 * m : 1) * sizeof(float));
  else g->wi = (int32_t*)malloc((size_t)(2 * m > 0 ? 2 * m : 1) * sizeof(int32_t));
  int64_t* cur = (int64_t*)malloc(((size_t)n + 1) * sizeof(int64_t));
  if (!g->offsets || !g->targets || (!g->wf && !g->wi) || !cur) { free(cur); gg_free(g); return NULL; }
  for (int64_t i = 0; i < m; i++) {
    int64_t u = (int64_t)(e->k[i] >> 32), v = (int64_t)(e->k[i] & 0xFFFFFFFFULL);
    g->offsets[u + 1]++; g->offsets[v + 1]++;
  }
  for (int64_t i = 0; i < n; i++) g->offsets[i + 1] += g->offsets[i];
  memcpy(cur, g->offsets, ((size_t)n + 1) * sizeof(int64_t));
  /* Two sweeps keep every row sorted: first the arcs to smaller ids (v -> u, u < v, keys in
   * increasing u for fixed v), then the arcs to larger ids (u -> v, increasing v). */
  for (int sweep = 0; sweep < 2; sweep++) {
    for (int64_t i = 0; i < m; i++) {
      int64_t u = (int64_t)(e->k[i] >> 32), v = (int64_t)(e->k[i] & 0xFFFFFFFFULL);
      int64_t row = sweep == 0 ? v : u, col = sweep == 0 ? u : v;
      int64_t p = cur[row]++;
      g->targets[p] = (int32_t)col;
      uint64_t h = weight_kind == 0 ? 0 : gg_hash3(wseed, (uint64_t)u, (uint64_t)v);
      if (weight_kind == 0) g->wi[p] = 1;
      else if (weight_kind == 1) g->wi[p] = 1 + (int32_t)(h & 7ULL);
      else g->wf[p] = (float)((double)((h >> 40) + 1) * (1.0 / 16777216.0));
    }
  }
  free(cur);
  return g;
}

/* Index t in the strict upper triangle of an s x s matrix, row-major over (u, v), u < v:
 * row u holds s-1-u entries and starts at u(2s-u-1)/2. */
static inline void tri_pair(int64_t s, int64_t t, int64_t* pu, int64_t* pv) {
  /* start(u) <= t; binary search on u in [0, s-1) */
  int64_t lo = 0, hi = s - 2;
  while (lo < hi) {
    int64_t mid = (lo + hi + 1) / 2;
    int64_t st = mid * (2 * s - mid - 1) / 2;
    if (st <= t) lo = mid; else hi = mid - 1;
  }
  int64_t st = lo * (2 * s - lo - 1) / 2;
  *pu = lo; *pv = lo + 1 + (t - st);
}

/* Geometric skipping (Batagelj and Brandes, Phys. Rev. E 71, 036113, 2005) over the strict
 * upper triangle of a block of s vertices starting at vertex `base`: each pair is an edge
 * independently with probability p.  Draws come from gg_hash3(seed, stream, k). */
static void skip_triangle(gg_keys* e, int64_t base, int64_t s, double p, uint64_t seed, uint64_t stream) {
  if (s < 2 || !(p > 0.0)) return;
  int64_t total = s * (s - 1) / 2;
  if (p >= 1.0) {
    for (int64_t t = 0; t < total; t++) { int64_t u, v; tri_pair(s, t, &u, &v); push_edge(e, base + u, base + v); }
    return;
  }
  double lq = gg_log(1.0 - p);
  int64_t t = -1;
  for (uint64_t k = 0;; k++) {
    double r = gg_u01(gg_hash3(seed, stream, k));
    double sk = gg_log(r) / lq;  /* >= 0 */
    if (sk > 9.0e18) break;
    t += 1 + (int64_t)sk;
    if (t >= total) break;
    int64_t u, v;
    tri_pair(s, t, &u, &v);
    push_edge(e, base + u, base + v);
  }
}

/* Planted-partition SBM: n vertices in k near-equal blocks (block b = [floor(bn/k),
 * floor((b+1)n/k))), in-block pair probability p_in, cross-block p_out.  Realised as the union
 * of an all-pairs p_out graph and, per block, an in-block graph with
 * p' = (p_in - p_out) / (1 - p_out), so an in-block pair is present with probability
 * p_out + (1 - p_out) p' = p_in.  Unit weights (weight_kind 0) or 1..8 (weight_kind 1). */
gg_csr* gg_sbm(int64_t n, int64_t k, double p_in, double p_out, uint64_t seed, int weight_kind) {
  if (n < 0 || n > 0x7fffffffLL || k < 1 || k > (n > 0 ? n : 1)) return NULL;
  gg_keys e = {0};
  skip_triangle(&e, 0, n, p_out, seed, 0);
  double pp = p_out < 1.0 ? (p_in - p_out) / (1.0 - p_out) : 0.0;
  for (int64_t b = 0; b < k; b++) {
    int64_t lo = b * n / k, hi = (b + 1) * n / k;
    skip_triangle(&e, lo, hi - lo, pp, seed, 1 + (uint64_t)b);
  }
  int64_t drawn = e.len;
  gg_csr* g = csr_from_keys(&e, n, weight_kind, seed ^ 0x5bd1e995ULL);
  free(e.k);
  if (g) g->n_edges_drawn = drawn;
  return g;
}

/* R-MAT (Chakrabarti, Zhan and Faloutsos, SDM 2004) without noise and without vertex
 * scrambling: edge_factor * 2^scale draws; draw d takes `scale` levels, level l choosing the
 * quadrant from 16 bits of gg_hash3(seed, d, l / 4) (bits 16 (l % 4) .. +15) against the
 * cumulative thresholds floor(65536 a), floor(65536 (a+b)), floor(65536 (a+b+c)).  Level 0 sets
 * the most significant bit.  Self-loops dropped, symmetrised, deduplicated. */
gg_csr* gg_rmat(int scale, int64_t edge_factor, double a, double b, double c, uint64_t seed, int weight_kind) {
  if (scale < 1 || scale > 30 || edge_factor < 1) return NULL;
  int64_t n = (int64_t)1 << scale, draws = edge_factor * n;
  uint32_t t1 = (uint32_t)(65536.0 * a), t2 = (uint32_t)(65536.0 * (a + b)), t3 = (uint32_t)(65536.0 * (a + b + c));
  gg_keys e = {0};
  e.cap = draws; e.k = (uint64_t*)malloc((size_t)draws * sizeof(uint64_t));
  if (!e.k) return NULL;
  for (int64_t d = 0; d < draws; d++) {
    int64_t u = 0, v = 0;
    uint64_t h = 0;
    for (int l = 0; l < scale; l++) {
      if ((l & 3) == 0) h = gg_hash3(seed, (uint64_t)d, (uint64_t)(l >> 2));
      uint32_t r = (uint32_t)((h >> (16 * (l & 3))) & 0xFFFF);
      int ub = 0, vb = 0;
      if (r < t1) { }
      else if (r < t2) vb = 1;
      else if (r < t3) ub = 1;
      else { ub = 1; vb = 1; }
      u |= (int64_t)ub << (scale - 1 - l);
      v |= (int64_t)vb << (scale - 1 - l);
    }
    push_edge(&e, u, v);
  }
  gg_csr* g = csr_from_keys(&e, n, weight_kind, seed ^ 0x5bd1e995ULL);
  free(e.k);
  if (g) g->n_edges_drawn = draws;
  return g;
}

/* Road-like grid: rows x cols lattice with 4-neighbour edges, each edge deleted independently
 * with probability p_del (kept iff hash < (1 - p_del) 2^64), then floor(p_long * kept) random
 * long links between uniform endpoints (dropped if a loop, deduplicated).  Unit weights. */
gg_csr* gg_grid(int64_t rows, int64_t cols, double p_del, double p_long, uint64_t seed) {
  if (rows < 1 || cols < 1 || rows * cols > 0x7fffffffLL) return NULL;
  int64_t n = rows * cols;
  double keep = 1.0 - p_del;
  uint64_t thr = keep >= 1.0 ? UINT64_MAX : (uint64_t)(keep * 18446744073709551616.0);
  gg_keys e = {0};
  for (int64_t r = 0; r < rows; r++)
    for (int64_t c = 0; c < cols; c++) {
      int64_t v = r * cols + c;
      if (c + 1 < cols && gg_hash3(seed, (uint64_t)v, 0) < thr) push_edge(&e, v, v + 1);
      if (r + 1 < rows && gg_hash3(seed, (uint64_t)v, 1) < thr) push_edge(&e, v, v + cols);
    }
  int64_t kept = e.len;
  int64_t nl = (int64_t)(p_long * (double)kept);
  for (int64_t i = 0; i < nl; i++) {
    uint64_t h1 = gg_hash3(seed, (uint64_t)n + (uint64_t)i, 2), h2 = gg_hash3(seed, (uint64_t)n + (uint64_t)i, 3);
    push_edge(&e, (int64_t)(h1 % (uint64_t)n), (int64_t)(h2 % (uint64_t)n));
  }
  gg_csr* g = csr_from_keys(&e, n, 0, 0);
  free(e.k);
  if (g) g->n_edges_drawn = kept + nl;
  return g;
}

/* Parameters of graph g of the batched SBM workload: n log-uniform in [n_lo, n_hi], k uniform
 * integer in [k_lo, k_hi] (capped at n), average degree log-uniform in [d_lo, d_hi],
 * p_in = d / ((s - 1) + ratio (n - s)) with s = n / k, p_out = ratio * p_in; seed of the graph
 * = gg_hash3(base_seed, g, 0).  Written to out[0..3] = n, k, p_in, p_out and *seed_out. */
void gg_batch_params(uint64_t base_seed, int64_t g, double n_lo, double n_hi, int64_t k_lo, int64_t k_hi,
                     double d_lo, double d_hi, double ratio, double* out, uint64_t* seed_out) {
  uint64_t h0 = gg_hash3(base_seed, (uint64_t)g, 1), h1 = gg_hash3(base_seed, (uint64_t)g, 2),
           h2 = gg_hash3(base_seed, (uint64_t)g, 3);
  double un = gg_u01(h0), ud = gg_u01(h2);
  int64_t n = (int64_t)gg_exp(gg_log(n_lo) + un * (gg_log(n_hi) - gg_log(n_lo)));
  if (n < 2) n = 2;
  int64_t k = k_lo + (int64_t)(h1 % (uint64_t)(k_hi - k_lo + 1));
  if (k > n) k = n;
  double d = gg_exp(gg_log(d_lo) + ud * (gg_log(d_hi) - gg_log(d_lo)));
  double s = (double)n / (double)k;
  double p_in = d / ((s - 1.0) + ratio * ((double)n - s));
  if (p_in > 1.0) p_in = 1.0;
  out[0] = (double)n; out[1] = (double)k; out[2] = p_in; out[3] = ratio * p_in;
  *seed_out = gg_hash3(base_seed, (uint64_t)g, 0);
}
