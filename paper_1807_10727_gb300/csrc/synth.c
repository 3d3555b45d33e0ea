/*
 * Seeded synthetic graph generators (host C, multithreaded, deterministic).
 *
 * These build the input edge lists only: Erdos-Renyi G(n,m) with replacement,
 * R-MAT (Chakrabarti, Zhan, Faloutsos 2004) with a random id permutation, a
 * 4-neighbour 2D grid, and a mix of power-law-sized ER components.  They hold
 * none of the connected-components arithmetic and none of the vertex-ranking
 * hash: their random stream is the MurmurHash3 64-bit finaliser (Appleby,
 * public domain) applied to a counter, so every output element depends only on
 * (seed, element index) and the result is identical for any thread count.
 *
 * The same bytes feed the CPU oracle and the GPU path.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <pthread.h>
#include <unistd.h>

/* ---------------------------------------------------------------- random */

static inline uint64_t fmix64(uint64_t k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdULL;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ULL;
  k ^= k >> 33;
  return k;
}

/* j-th 64-bit draw of stream `s` */
static inline uint64_t draw(uint64_t s, uint64_t j) {
  return fmix64(fmix64(s ^ 0x5851f42d4c957f2dULL) + j * 0x9fb21c651e98df25ULL);
}

/* uniform integer in [0, n) from the high 32 bits (multiply-shift) */
static inline uint32_t bounded32(uint64_t x, uint64_t n) {
  return (uint32_t)(((x >> 32) * n) >> 32);
}

/* ------------------------------------------------------------ threading */

typedef void (*range_fn)(void* ctx, uint64_t lo, uint64_t hi);
typedef struct { range_fn fn; void* ctx; uint64_t lo, hi; } job_t;

static void* job_main(void* p) {
  job_t* j = (job_t*)p;
  j->fn(j->ctx, j->lo, j->hi);
  return NULL;
}

static int pick_threads(int nthreads, uint64_t work) {
  if (nthreads <= 0) {
    long c = sysconf(_SC_NPROCESSORS_ONLN);
    nthreads = c > 0 ? (int)c : 1;
  }
  if (nthreads > 256) nthreads = 256;
  if (work < (1u << 16)) nthreads = 1;
  return nthreads;
}

static void parallel_for(uint64_t total, int nthreads, range_fn fn, void* ctx) {
  int t = pick_threads(nthreads, total);
  if (t == 1) { fn(ctx, 0, total); return; }
  pthread_t th[256];
  job_t jobs[256];
  for (int i = 0; i < t; ++i) {
    jobs[i].fn = fn; jobs[i].ctx = ctx;
    jobs[i].lo = total * (uint64_t)i / (uint64_t)t;
    jobs[i].hi = total * (uint64_t)(i + 1) / (uint64_t)t;
    pthread_create(&th[i], NULL, job_main, &jobs[i]);
  }
  for (int i = 0; i < t; ++i) pthread_join(th[i], NULL);
}

/* ---------------------------------------------- bijective id permutation */
/* Unbalanced Feistel network over [0, 2^k) with cycle walking into [0, n). */

typedef struct { uint64_t n; int k; uint64_t seed; } perm_t;

static perm_t perm_make(uint64_t n, uint64_t seed) {
  perm_t p; p.n = n; p.seed = seed; p.k = 2;
  while (p.k < 64 && (1ULL << p.k) < n) ++p.k;
  return p;
}

static inline uint64_t perm_once(const perm_t* p, uint64_t x) {
  int a = p->k - p->k / 2, b = p->k / 2;  /* left a bits, right b bits */
  for (int r = 0; r < 6; ++r) {
    uint64_t L = x >> b, R = x & ((1ULL << b) - 1);
    uint64_t F = fmix64(R ^ draw(p->seed, (uint64_t)r)) & ((1ULL << a) - 1);
    x = (R << a) | (L ^ F);
    int t = a; a = b; b = t;
  }
  return x;
}

static inline uint32_t perm_apply(const perm_t* p, uint32_t v) {
  uint64_t x = v;
  do { x = perm_once(p, x); } while (x >= p->n);
  return (uint32_t)x;
}

/* ----------------------------------------------------------------- ER */

typedef struct { uint64_t n, seed; uint32_t *src, *dst; } er_ctx;

static void er_range(void* c, uint64_t lo, uint64_t hi) {
  er_ctx* e = (er_ctx*)c;
  for (uint64_t j = lo; j < hi; ++j) {
    e->src[j] = bounded32(draw(e->seed, 2 * j), e->n);
    e->dst[j] = bounded32(draw(e->seed, 2 * j + 1), e->n);
  }
}

/* G(n, m): m pairs, each endpoint uniform in [0, n), with replacement. */
int synth_er(uint64_t n, uint64_t m, uint64_t seed, uint32_t* src, uint32_t* dst,
             int nthreads) {
  if (n == 0 || n > 0xFFFFFFFFULL) return 1;
  er_ctx c = {n, seed, src, dst};
  parallel_for(m, nthreads, er_range, &c);
  return 0;
}

/* ---------------------------------------------------------------- RMAT */

typedef struct {
  int scale; uint64_t n_keep, seed; uint32_t ta, tab, tabc;
  uint32_t *src, *dst; int permute; perm_t perm;
} rmat_ctx;

static inline void rmat_edge(const rmat_ctx* r, uint64_t j, uint64_t attempt,
                             uint32_t* pu, uint32_t* pv) {
  uint64_t u = 0, v = 0, w = 0;
  uint64_t base = (j * 1024 + attempt) * 16;
  for (int k = 0; k < r->scale; ++k) {
    if ((k & 1) == 0) w = draw(r->seed, base + (uint64_t)(k >> 1));
    uint32_t x = (k & 1) ? (uint32_t)w : (uint32_t)(w >> 32);
    uint64_t bu = 0, bv = 0;
    if (x < r->ta) { bu = 0; bv = 0; }
    else if (x < r->tab) { bu = 0; bv = 1; }
    else if (x < r->tabc) { bu = 1; bv = 0; }
    else { bu = 1; bv = 1; }
    u = (u << 1) | bu;
    v = (v << 1) | bv;
  }
  *pu = (uint32_t)u; *pv = (uint32_t)v;
}

static void rmat_range(void* c, uint64_t lo, uint64_t hi) {
  rmat_ctx* r = (rmat_ctx*)c;
  for (uint64_t j = lo; j < hi; ++j) {
    uint32_t u = 0, v = 0;
    uint64_t t = 0;
    for (;;) {
      rmat_edge(r, j, t, &u, &v);
      if (((uint64_t)u < r->n_keep && (uint64_t)v < r->n_keep) || t == 1023) break;
      ++t;
    }
    if ((uint64_t)u >= r->n_keep) u = (uint32_t)(u % r->n_keep);
    if ((uint64_t)v >= r->n_keep) v = (uint32_t)(v % r->n_keep);
    if (r->permute) { u = perm_apply(&r->perm, u); v = perm_apply(&r->perm, v); }
    r->src[j] = u; r->dst[j] = v;
  }
}

static uint32_t prob_threshold(double p) {
  double t = p * 4294967296.0;
  if (t <= 0) return 0;
  if (t >= 4294967295.0) return 0xFFFFFFFFu;
  return (uint32_t)t;
}

/* R-MAT: `scale` levels of quadrant choice with probabilities (a, b, c, 1-a-b-c)
 * and no noise.  Ids >= n_keep (n_keep <= 2^scale) are rejected and the edge is
 * redrawn.  With perm_seed != 0 a random bijection of [0, n_keep) is applied to
 * both endpoints. */
int synth_rmat(int scale, uint64_t n_keep, uint64_t m, double a, double b, double c,
               uint64_t seed, uint64_t perm_seed, uint32_t* src, uint32_t* dst,
               int nthreads) {
  if (scale < 1 || scale > 32) return 1;
  if (n_keep == 0 || n_keep > (1ULL << scale)) return 1;
  rmat_ctx r;
  r.scale = scale; r.n_keep = n_keep; r.seed = seed;
  r.ta = prob_threshold(a);
  r.tab = prob_threshold(a + b);
  r.tabc = prob_threshold(a + b + c);
  r.src = src; r.dst = dst;
  r.permute = perm_seed != 0;
  r.perm = perm_make(n_keep, perm_seed);
  parallel_for(m, nthreads, rmat_range, &r);
  return 0;
}

/* -------------------------------------------------------- permutations */

typedef struct { perm_t p; uint32_t* x; } pa_ctx;

static void pa_range(void* c, uint64_t lo, uint64_t hi) {
  pa_ctx* q = (pa_ctx*)c;
  for (uint64_t j = lo; j < hi; ++j) q->x[j] = perm_apply(&q->p, q->x[j]);
}

/* x[j] <- pi(x[j]) for a seeded bijection pi of [0, n). */
int synth_permute_ids(uint64_t n, uint64_t perm_seed, uint32_t* x, uint64_t len,
                      int nthreads) {
  if (n == 0 || n > 0xFFFFFFFFULL) return 1;
  pa_ctx c; c.p = perm_make(n, perm_seed); c.x = x;
  parallel_for(len, nthreads, pa_range, &c);
  return 0;
}

/* pi(v) for one id (used by tests to check bijectivity). */
uint32_t synth_perm_one(uint64_t n, uint64_t perm_seed, uint32_t v) {
  perm_t p = perm_make(n, perm_seed);
  return perm_apply(&p, v);
}

/* ----------------------------------------------------------------- grid */

typedef struct { uint64_t w, h, off; uint32_t *src, *dst; } grid_ctx;

static void grid_range(void* c, uint64_t lo, uint64_t hi) {
  grid_ctx* g = (grid_ctx*)c;
  uint64_t nh = g->h * (g->w - 1);
  for (uint64_t j = lo; j < hi; ++j) {
    uint64_t a, b;
    if (j < nh) {
      uint64_t y = j / (g->w - 1), x = j % (g->w - 1);
      a = y * g->w + x; b = a + 1;
    } else {
      uint64_t k = j - nh;
      uint64_t y = k / g->w, x = k % g->w;
      a = y * g->w + x; b = a + g->w;
    }
    g->src[j] = (uint32_t)(a + g->off);
    g->dst[j] = (uint32_t)(b + g->off);
  }
}

uint64_t synth_grid_edges(uint64_t w, uint64_t h) {
  if (w == 0 || h == 0) return 0;
  return h * (w - 1) + w * (h - 1);
}

/* w x h 4-neighbour grid, vertex (x, y) = off + y*w + x; all horizontal edges
 * first, then all vertical ones. */
int synth_grid(uint64_t w, uint64_t h, uint64_t off, uint32_t* src, uint32_t* dst,
               int nthreads) {
  if (w == 0 || h == 0) return 0;
  if (off + w * h > 0x100000000ULL) return 1;
  grid_ctx g = {w, h, off, src, dst};
  parallel_for(synth_grid_edges(w, h), nthreads, grid_range, &g);
  return 0;
}

/* ------------------------------------------------ power-law ER mixture */

/* Component sizes s in [smin, smax] with P(s) proportional to s^-alpha, by
 * inverse CDF over the discrete distribution (cumulative weights quantised to
 * integers so that 1-ulp libm differences do not move a sample). */
int synth_powerlaw_sizes(uint64_t count, uint32_t smin, uint32_t smax, double alpha,
                         uint64_t seed, uint32_t* sizes) {
  if (smin < 1 || smax < smin) return 1;
  uint64_t span = (uint64_t)smax - smin + 1;
  uint64_t* cdf = (uint64_t*)malloc(span * sizeof(uint64_t));
  if (!cdf) return 2;
  double tot = 0.0;
  for (uint64_t i = 0; i < span; ++i) tot += pow((double)(smin + i), -alpha);
  double acc = 0.0;
  for (uint64_t i = 0; i < span; ++i) {
    acc += pow((double)(smin + i), -alpha);
    double q = acc / tot * 9007199254740992.0; /* 2^53 */
    uint64_t qi = (uint64_t)q;
    cdf[i] = (qi >> 12) << 12;
  }
  cdf[span - 1] = 9007199254740992ULL;
  for (uint64_t j = 0; j < count; ++j) {
    uint64_t u = draw(seed, j) >> 11; /* uniform in [0, 2^53) */
    uint64_t lo = 0, hi = span - 1;
    while (lo < hi) {
      uint64_t mid = (lo + hi) / 2;
      if (u < cdf[mid]) hi = mid; else lo = mid + 1;
    }
    sizes[j] = (uint32_t)(smin + lo);
  }
  free(cdf);
  return 0;
}

typedef struct {
  const uint64_t* voff; const uint64_t* eoff; const uint32_t* sizes;
  uint64_t seed, base_v; uint32_t *src, *dst;
} mix_ctx;

static void mix_range(void* c, uint64_t lo, uint64_t hi) {
  mix_ctx* q = (mix_ctx*)c;
  for (uint64_t g = lo; g < hi; ++g) {
    uint64_t s = q->sizes[g];
    uint64_t vb = q->base_v + q->voff[g];
    for (uint64_t e = q->eoff[g]; e < q->eoff[g + 1]; ++e) {
      q->src[e] = (uint32_t)(vb + bounded32(draw(q->seed, 2 * e), s));
      q->dst[e] = (uint32_t)(vb + bounded32(draw(q->seed, 2 * e + 1), s));
    }
  }
}

/* Component g has sizes[g] vertices starting at base_v + voff[g] and edges
 * [eoff[g], eoff[g+1]) drawn uniformly inside it with replacement. */
int synth_components(uint64_t count, const uint32_t* sizes, const uint64_t* voff,
                     const uint64_t* eoff, uint64_t base_v, uint64_t seed,
                     uint32_t* src, uint32_t* dst, int nthreads) {
  mix_ctx c = {voff, eoff, sizes, seed, base_v, src, dst};
  parallel_for(count, nthreads, mix_range, &c);
  return 0;
}

/* --------------------------------------------------------- misc draws */

/* out[j] = j-th 64-bit draw of stream `seed` (used for batch / request shapes). */
void synth_draws(uint64_t seed, uint64_t count, uint64_t* out) {
  for (uint64_t j = 0; j < count; ++j) out[j] = draw(seed, j);
}
