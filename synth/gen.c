/*
 * Seeded synthetic columns for the relational hot path (fused filter +
 * group-by, equi-join build + probe).
 *
 * This module produces INPUTS only.  It holds none of the arithmetic of the
 * operators themselves (no hashing of keys into tables, no aggregation, no
 * matching); both the CPU oracle and the GPU path read the bytes it writes.
 *
 * Every value is a pure function of (seed, column tag, row index): the
 * counter-based generator is the splitmix64 output function of Steele, Lea &
 * Flood (2014) applied to  stream_key(seed, tag) + i.  Work is split across
 * threads by row ranges, which cannot change any value.
 *
 * Uniform integers in [lo, hi] (inclusive) use the multiply-high mapping of
 * Lemire (2019) without rejection: bias <= span / 2^64.
 *
 * The only floating point is the Zipf inverse-CDF table (pow and a running
 * sum in double); its rounding may differ between C libraries, so Zipf
 * columns are consumed within one run and never stored as expected values.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define GAMMA 0x9E3779B97F4A7C15ull

static inline uint64_t fin64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* One splitmix64 step from state x: a bijection on 64-bit words. */
uint64_t syn_mix64(uint64_t x) { return fin64(x + GAMMA); }

static inline uint64_t stream_key(uint64_t seed, uint64_t tag) {
  return syn_mix64(syn_mix64(seed) ^ tag);
}

static inline uint64_t draw(uint64_t key, uint64_t i) { return syn_mix64(key + i); }

/* lo + floor(r * span / 2^64), span = hi - lo + 1 (span 0 means 2^64). */
static inline int64_t uniform_in(uint64_t r, int64_t lo, int64_t hi) {
  uint64_t span = (uint64_t)hi - (uint64_t)lo + 1u;
  if (span == 0) return (int64_t)((uint64_t)lo + r);
  uint64_t off = (uint64_t)(((unsigned __int128)r * span) >> 64);
  return (int64_t)((uint64_t)lo + off);
}

uint64_t syn_draw(uint64_t seed, uint64_t tag, uint64_t i) {
  return draw(stream_key(seed, tag), i);
}

int64_t syn_uniform_at(uint64_t seed, uint64_t tag, uint64_t i, int64_t lo, int64_t hi) {
  return uniform_in(syn_draw(seed, tag, i), lo, hi);
}

/* ---------------------------------------------------------------- threads */

typedef void (*range_fn)(void* ctx, int64_t b, int64_t e);
typedef struct { range_fn fn; void* ctx; int64_t b, e; } range_job;

static void* run_job(void* p) {
  range_job* j = (range_job*)p;
  j->fn(j->ctx, j->b, j->e);
  return NULL;
}

static void parallel_rows(int64_t n, range_fn fn, void* ctx) {
  long nt = sysconf(_SC_NPROCESSORS_ONLN);
  if (nt < 1) nt = 1;
  if (nt > 64) nt = 64;
  if (n < (1 << 18)) nt = 1;
  if (nt == 1) { fn(ctx, 0, n); return; }
  pthread_t th[64];
  range_job jobs[64];
  int live[64] = {0};
  int64_t chunk = (n + nt - 1) / nt;
  for (long t = 0; t < nt; t++) {
    int64_t b = t * chunk, e = b + chunk < n ? b + chunk : n;
    if (b >= e) break;
    jobs[t] = (range_job){fn, ctx, b, e};
    if (pthread_create(&th[t], NULL, run_job, &jobs[t]) == 0)
      live[t] = 1;
    else
      fn(ctx, b, e);
  }
  for (long t = 0; t < nt; t++)
    if (live[t]) pthread_join(th[t], NULL);
}

/* ------------------------------------------------------- uniform integers */

typedef struct { void* out; int elem; int64_t lo, hi; uint64_t key; int mix; } uni_ctx;

static void uni_body(void* p, int64_t b, int64_t e) {
  uni_ctx* c = (uni_ctx*)p;
  for (int64_t i = b; i < e; i++) {
    int64_t v = uniform_in(draw(c->key, (uint64_t)i), c->lo, c->hi);
    if (c->mix) v = (int64_t)syn_mix64((uint64_t)v);
    switch (c->elem) {
      case 1: ((uint8_t*)c->out)[i] = (uint8_t)v; break;
      case 4: ((int32_t*)c->out)[i] = (int32_t)v; break;
      default: ((int64_t*)c->out)[i] = v; break;
    }
  }
}

/* out[i] = U[lo, hi] narrowed to elem bytes (1, 4 or 8). */
void syn_uniform(void* out, int64_t n, int elem, int64_t lo, int64_t hi, uint64_t seed,
                 uint64_t tag) {
  uni_ctx c = {out, elem, lo, hi, stream_key(seed, tag), 0};
  parallel_rows(n, uni_body, &c);
}

/* out[i] = mix64(U[lo, hi]): a few (or many) distinct keys scattered over
 * the whole int64 domain, negatives included. */
void syn_uniform_mixed(int64_t* out, int64_t n, int64_t lo, int64_t hi, uint64_t seed,
                       uint64_t tag) {
  uni_ctx c = {out, 8, lo, hi, stream_key(seed, tag), 1};
  parallel_rows(n, uni_body, &c);
}

/* ------------------------------------------- 40-bit Feistel permutation */

/* A bijection on [0, 2^40): four Feistel rounds over two 20-bit halves,
 * round function = low 20 bits of splitmix64 of (round key ^ half). */
static inline uint64_t perm40(uint64_t x, uint64_t pkey) {
  const uint64_t M = (1ull << 20) - 1;
  uint64_t L = (x >> 20) & M, R = x & M;
  for (uint64_t k = 0; k < 4; k++) {
    uint64_t rk = syn_mix64(pkey ^ (k + 1));
    uint64_t F = syn_mix64(rk ^ R) & M;
    uint64_t nL = R, nR = L ^ F;
    L = nL;
    R = nR;
  }
  return (L << 20) | R;
}

uint64_t syn_perm40(uint64_t x, uint64_t seed) { return perm40(x, stream_key(seed, 0x50)); }

enum { TAG_PERM = 0x50, TAG_PAYLOAD = 0x51, TAG_HIT = 0x52, TAG_PICK = 0x53, TAG_MISS = 0x54 };

typedef struct { int64_t* keys; int64_t* pay; uint64_t pk, payk; } jb_ctx;

static void jb_body(void* p, int64_t b, int64_t e) {
  jb_ctx* c = (jb_ctx*)p;
  for (int64_t j = b; j < e; j++) {
    c->keys[j] = (int64_t)perm40((uint64_t)j, c->pk);
    if (c->pay) c->pay[j] = uniform_in(draw(c->payk, (uint64_t)j), 0, INT64_MAX);
  }
}

/* Build side: key[j] = pi(j) for j < n_b (distinct, since pi is a bijection),
 * payload[j] = U[0, 2^63). */
void syn_join_build(int64_t* keys, int64_t* payload, int64_t n_b, uint64_t seed) {
  jb_ctx c = {keys, payload, stream_key(seed, TAG_PERM), stream_key(seed, TAG_PAYLOAD)};
  parallel_rows(n_b, jb_body, &c);
}

typedef struct {
  int64_t* keys; uint8_t* present; int64_t n_b; uint64_t thr;
  uint64_t pk, hk, ck, mk; int64_t* counts;  /* per-thread present counts */
} jp_ctx;

static void jp_body(void* p, int64_t b, int64_t e) {
  jp_ctx* c = (jp_ctx*)p;
  for (int64_t i = b; i < e; i++) {
    int hit = draw(c->hk, (uint64_t)i) < c->thr;
    uint64_t src;
    if (hit)
      src = (uint64_t)uniform_in(draw(c->ck, (uint64_t)i), 0, c->n_b - 1);
    else
      src = (uint64_t)uniform_in(draw(c->mk, (uint64_t)i), c->n_b, (int64_t)(1ull << 40) - 1);
    c->keys[i] = (int64_t)perm40(src, c->pk);
    if (c->present) c->present[i] = (uint8_t)hit;
  }
}

/* Probe side: row i is "present" when its draw is below hit_threshold
 * (hit rate = threshold / 2^64).  A present row takes the key of a uniform
 * build row; an absent row takes pi(n_b + U[0, 2^40 - n_b)), which no build
 * row holds.  Requires 1 <= n_b < 2^40. */
void syn_join_probe(int64_t* keys, uint8_t* present, int64_t n_p, int64_t n_b,
                    uint64_t hit_threshold, uint64_t seed) {
  jp_ctx c = {keys, present, n_b, hit_threshold, stream_key(seed, TAG_PERM),
              stream_key(seed, TAG_HIT), stream_key(seed, TAG_PICK), stream_key(seed, TAG_MISS),
              NULL};
  parallel_rows(n_p, jp_body, &c);
}

/* ------------------------------------------------------------------ Zipf */

typedef struct {
  int64_t n;       /* ranks 1..n */
  double* cdf;     /* cdf[k-1] = P(rank <= k) */
  int64_t* guide;  /* guide[g] = smallest k-1 with cdf[k-1] > g / n_guide */
  int64_t n_guide;
} zipf_table;

void* syn_zipf_new(int64_t n, double s) {
  if (n < 1) return NULL;
  zipf_table* t = (zipf_table*)calloc(1, sizeof(zipf_table));
  if (!t) return NULL;
  t->n = n;
  t->cdf = (double*)malloc(sizeof(double) * (size_t)n);
  t->n_guide = n;
  t->guide = (int64_t*)malloc(sizeof(int64_t) * (size_t)t->n_guide);
  if (!t->cdf || !t->guide) { free(t->cdf); free(t->guide); free(t); return NULL; }
  double acc = 0.0;
  for (int64_t k = 1; k <= n; k++) {
    acc += pow((double)k, -s);
    t->cdf[k - 1] = acc;
  }
  for (int64_t k = 0; k < n; k++) t->cdf[k] /= acc;
  t->cdf[n - 1] = 1.0;
  int64_t k = 0;
  for (int64_t g = 0; g < t->n_guide; g++) {
    double u = (double)g / (double)t->n_guide;
    while (t->cdf[k] <= u) k++;
    t->guide[g] = k;
  }
  return t;
}

void syn_zipf_free(void* h) {
  zipf_table* t = (zipf_table*)h;
  if (!t) return;
  free(t->cdf);
  free(t->guide);
  free(t);
}

/* Smallest rank k with cdf(k) > u, for u in [0, 1). */
static inline int64_t zipf_rank(const zipf_table* t, double u) {
  int64_t g = (int64_t)(u * (double)t->n_guide);
  if (g >= t->n_guide) g = t->n_guide - 1;
  int64_t k = t->guide[g];
  while (t->cdf[k] <= u) k++;
  return k + 1;
}

int64_t syn_zipf_rank_of(void* h, double u) { return zipf_rank((const zipf_table*)h, u); }

typedef struct { const zipf_table* t; int64_t* out; uint64_t key; int mix; } zk_ctx;

static void zk_body(void* p, int64_t b, int64_t e) {
  zk_ctx* c = (zk_ctx*)p;
  for (int64_t i = b; i < e; i++) {
    double u = (double)(draw(c->key, (uint64_t)i) >> 11) * 0x1.0p-53;
    int64_t r = zipf_rank(c->t, u);
    c->out[i] = c->mix ? (int64_t)syn_mix64((uint64_t)r) : r;
  }
}

/* out[i] = mix64(rank) (mix != 0) or rank, rank ~ Zipf(s) over 1..n. */
void syn_zipf_keys(void* h, int64_t* out, int64_t n, uint64_t seed, uint64_t tag, int mix) {
  zk_ctx c = {(const zipf_table*)h, out, stream_key(seed, tag), mix};
  parallel_rows(n, zk_body, &c);
}
