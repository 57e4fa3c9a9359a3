/*
 * Seeded synthetic transaction databases (input generation only).
 *
 * This file holds no frequent-itemset arithmetic: it only writes horizontal
 * databases in CSR form (tx_offsets[D+1], tx_items[nnz], items ascending and
 * distinct inside a transaction).  Both the CPU oracle and the GPU path read
 * the same arrays.
 *
 * Random numbers come from SplitMix64 (G. Steele, D. Lea, C. Flood, "Fast
 * splittable pseudorandom number generators", OOPSLA 2014), used as a
 * sequential stream per purpose; each stream is seeded from (seed, purpose).
 * The only transcendental functions (exp, log) are computed here from IEEE
 * additions, multiplications and divisions, and the file is compiled without
 * floating-point contraction, so a seed gives the same database bit for bit on
 * every IEEE-754 machine (x86-64 and aarch64 alike).
 *
 * Generators:
 *  - pattern-embedded ("Quest-like") databases: npat seed patterns with
 *    Poisson(PL) lengths (minimum 1), distinct items drawn by a popularity law
 *    (uniform, or Zipf(s) over a seeded permutation of the item ids), Exp(1)
 *    pattern weights.  Each transaction draws a target length L ~ Poisson(TL)
 *    (zero allowed) and is filled by at most 100 attempts: with probability q
 *    one noise item (same popularity law), otherwise one weighted pattern whose
 *    items are each kept with probability keep_p; filling stops as soon as the
 *    transaction holds L distinct items.
 *  - dense Bernoulli databases: item i present independently with probability
 *    p_lo + (p_hi - p_lo) * i / (N - 1).
 *  - dense fixed-length databases: exactly k distinct items per transaction,
 *    drawn without replacement with weights p_i as above.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GAMMA64 0x9E3779B97F4A7C15ULL

/* exp and log from basic IEEE operations only (no libm: its last-bit results
 * differ between platforms).  ln 2 is split in a high part exact in 32 bits
 * and a low part, as in Cody-Waite range reduction. */
static const double LN2_HI = 6.93147180369123816490e-01;
static const double LN2_LO = 1.90821492927058770002e-10;
static double scale2(double x, int k) {
  /* x * 2^k for |k| < 1000 by repeated exact scaling */
  while (k > 60) { x *= 1152921504606846976.0; k -= 60; }
  while (k < -60) { x *= 8.67361737988403547206e-19; k += 60; }
  if (k >= 0) return x * (double)(1ULL << k);
  return x / (double)(1ULL << (-k));
}
static double my_exp(double x) {
  if (x < -700.0) return 0.0;
  if (x > 700.0) x = 700.0;
  double kd = x / (LN2_HI + LN2_LO);
  int k = (int)(kd < 0 ? kd - 0.5 : kd + 0.5);
  double r = (x - (double)k * LN2_HI) - (double)k * LN2_LO;   /* |r| <= ln2/2 */
  double term = 1.0, sum = 1.0;
  for (int n = 1; n < 30; ++n) { term = term * r / (double)n; sum += term; }
  return scale2(sum, k);
}
static double my_log(double x) {
  /* x > 0: x = m * 2^k with m in [1, 2); log m = 2 atanh((m-1)/(m+1)) */
  int k = 0;
  while (x >= 2.0) { x *= 0.5; ++k; }
  while (x < 1.0) { x *= 2.0; --k; }
  double z = (x - 1.0) / (x + 1.0), z2 = z * z, term = z, sum = 0.0;
  for (int n = 1; n < 80; n += 2) { sum += term / (double)n; term *= z2; }
  return 2.0 * sum + (double)k * LN2_HI + (double)k * LN2_LO;
}
static double my_pow(double b, double e) { return my_exp(e * my_log(b)); }

typedef struct { uint64_t s; } rng_t;

static uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
static rng_t rng_make(uint64_t seed, uint64_t purpose) {
  rng_t r;
  r.s = mix64(seed * 0x2545F4914F6CDD1DULL + purpose * GAMMA64 + 0x1234567ULL);
  return r;
}
static uint64_t rng_next(rng_t* r) {
  r->s += GAMMA64;
  return mix64(r->s);
}
/* uniform double in (0, 1] */
static double rng_unit(rng_t* r) { return ((double)(rng_next(r) >> 11) + 1.0) * (1.0 / 9007199254740992.0); }
/* uniform integer in [0, n) by multiply-shift */
static uint32_t rng_below(rng_t* r, uint32_t n) {
  return (uint32_t)(((rng_next(r) >> 32) * (uint64_t)n) >> 32);
}
static uint32_t rng_poisson(rng_t* r, double lam) {
  /* sequential inversion; lam here is at most a few tens */
  double u = rng_unit(r), p = my_exp(-lam), f = p;
  uint32_t k = 0;
  while (u > f && k < 10000) {
    ++k;
    p *= lam / (double)k;
    f += p;
    if (p < 1e-300 && f < u) break;
  }
  return k;
}

typedef struct {
  uint32_t n;
  int zipf;
  double* cdf;     /* n entries, zipf only */
  uint32_t* perm;  /* rank -> item id, zipf only */
} popularity_t;

static int pop_init(popularity_t* p, uint32_t n, int zipf, double s, uint64_t seed) {
  p->n = n; p->zipf = zipf; p->cdf = NULL; p->perm = NULL;
  if (!zipf) return 0;
  p->cdf = (double*)malloc(sizeof(double) * n);
  p->perm = (uint32_t*)malloc(sizeof(uint32_t) * n);
  if (!p->cdf || !p->perm) return -1;
  double acc = 0.0;
  for (uint32_t k = 0; k < n; ++k) { acc += my_pow((double)(k + 1), -s); p->cdf[k] = acc; }
  for (uint32_t k = 0; k < n; ++k) p->cdf[k] /= acc;
  p->cdf[n - 1] = 1.0;
  for (uint32_t k = 0; k < n; ++k) p->perm[k] = k;
  rng_t r = rng_make(seed, 7);
  for (uint32_t k = n - 1; k > 0; --k) {  /* Fisher-Yates */
    uint32_t j = rng_below(&r, k + 1);
    uint32_t t = p->perm[k]; p->perm[k] = p->perm[j]; p->perm[j] = t;
  }
  return 0;
}
static void pop_free(popularity_t* p) { free(p->cdf); free(p->perm); }
static uint32_t pop_draw(const popularity_t* p, rng_t* r) {
  if (!p->zipf) return rng_below(r, p->n);
  double u = rng_unit(r);
  uint32_t lo = 0, hi = p->n - 1;
  while (lo < hi) { uint32_t mid = (lo + hi) / 2; if (p->cdf[mid] >= u) hi = mid; else lo = mid + 1; }
  return p->perm[lo];
}

typedef struct {
  uint32_t* offsets;
  uint32_t* items;
  uint32_t D;
  uint64_t nnz;
  uint64_t cap;
} synth_db;

static int db_init(synth_db* db, uint32_t D, uint64_t cap) {
  db->D = D; db->nnz = 0; db->cap = cap ? cap : 16;
  db->offsets = (uint32_t*)malloc(sizeof(uint32_t) * ((size_t)D + 1));
  db->items = (uint32_t*)malloc(sizeof(uint32_t) * db->cap);
  if (!db->offsets || !db->items) return -1;
  db->offsets[0] = 0;
  return 0;
}
static int db_push(synth_db* db, uint32_t v) {
  if (db->nnz == db->cap) {
    uint64_t nc = db->cap * 2;
    uint32_t* ni = (uint32_t*)realloc(db->items, sizeof(uint32_t) * nc);
    if (!ni) return -1;
    db->items = ni; db->cap = nc;
  }
  db->items[db->nnz++] = v;
  return 0;
}
static int cmp_u32(const void* a, const void* b) {
  uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
  return (x > y) - (x < y);
}

void synth_free(synth_db* db) {
  if (!db) return;
  free(db->offsets); free(db->items); free(db);
}
uint32_t synth_num_tx(const synth_db* db) { return db->D; }
uint64_t synth_nnz(const synth_db* db) { return db->nnz; }
void synth_copy(const synth_db* db, uint32_t* offsets_out, uint32_t* items_out) {
  memcpy(offsets_out, db->offsets, sizeof(uint32_t) * ((size_t)db->D + 1));
  if (db->nnz) memcpy(items_out, db->items, sizeof(uint32_t) * db->nnz);
}

/* Pattern-embedded database; see the header comment for the recipe. */
synth_db* synth_pattern_db(uint64_t seed, uint32_t D, uint32_t N, double TL, double PL, uint32_t npat,
                           int zipf, double zipf_s, double q_noise, double keep_p) {
  if (N == 0) return NULL;
  popularity_t pop;
  if (pop_init(&pop, N, zipf, zipf_s, seed) != 0) { pop_free(&pop); return NULL; }
  if (npat == 0) npat = 1;
  uint32_t* pat_off = (uint32_t*)malloc(sizeof(uint32_t) * ((size_t)npat + 1));
  double* pat_cdf = (double*)malloc(sizeof(double) * npat);
  uint32_t pat_cap = 1024, pat_n = 0;
  uint32_t* pat_items = (uint32_t*)malloc(sizeof(uint32_t) * pat_cap);
  synth_db* db = (synth_db*)calloc(1, sizeof(synth_db));
  uint8_t* mark = (uint8_t*)calloc(N, 1);
  uint32_t* cur = NULL;
  if (!pat_off || !pat_cdf || !pat_items || !db || !mark) goto fail;

  {
    rng_t rp = rng_make(seed, 1);
    double wsum = 0.0;
    pat_off[0] = 0;
    for (uint32_t p = 0; p < npat; ++p) {
      uint32_t len = rng_poisson(&rp, PL);
      if (len < 1) len = 1;
      if (len > N) len = N;
      uint32_t got = 0, tries = 0;
      while (got < len && tries < 1000u * len) {
        ++tries;
        uint32_t it = pop_draw(&pop, &rp);
        if (mark[it]) continue;
        mark[it] = 1;
        if (pat_n == pat_cap) {
          pat_cap *= 2;
          uint32_t* np_ = (uint32_t*)realloc(pat_items, sizeof(uint32_t) * pat_cap);
          if (!np_) goto fail;
          pat_items = np_;
        }
        pat_items[pat_n++] = it;
        ++got;
      }
      for (uint32_t k = pat_off[p]; k < pat_n; ++k) mark[pat_items[k]] = 0;
      pat_off[p + 1] = pat_n;
      wsum += -my_log(rng_unit(&rp));
      pat_cdf[p] = wsum;
    }
    for (uint32_t p = 0; p < npat; ++p) pat_cdf[p] /= wsum;
    pat_cdf[npat - 1] = 1.0;
  }

  if (db_init(db, D, (uint64_t)((double)D * (TL + 1.0)) + 16) != 0) goto fail;
  cur = (uint32_t*)malloc(sizeof(uint32_t) * ((size_t)N + 1));
  if (!cur) goto fail;
  {
    rng_t rl = rng_make(seed, 2);  /* transaction lengths */
    rng_t rt = rng_make(seed, 3);  /* filling */
    for (uint32_t t = 0; t < D; ++t) {
      uint32_t L = rng_poisson(&rl, TL);
      if (L > N) L = N;
      uint32_t n = 0;
      for (uint32_t att = 0; att < 100 && n < L; ++att) {
        if (rng_unit(&rt) <= q_noise) {
          uint32_t it = pop_draw(&pop, &rt);
          if (!mark[it]) { mark[it] = 1; cur[n++] = it; }
        } else {
          double u = rng_unit(&rt);
          uint32_t lo = 0, hi = npat - 1;
          while (lo < hi) { uint32_t mid = (lo + hi) / 2; if (pat_cdf[mid] >= u) hi = mid; else lo = mid + 1; }
          for (uint32_t k = pat_off[lo]; k < pat_off[lo + 1] && n < L; ++k) {
            if (rng_unit(&rt) > keep_p) continue;
            uint32_t it = pat_items[k];
            if (!mark[it]) { mark[it] = 1; cur[n++] = it; }
          }
        }
      }
      qsort(cur, n, sizeof(uint32_t), cmp_u32);
      for (uint32_t k = 0; k < n; ++k) { mark[cur[k]] = 0; if (db_push(db, cur[k]) != 0) goto fail; }
      db->offsets[t + 1] = (uint32_t)db->nnz;
    }
  }
  free(cur); free(mark); free(pat_off); free(pat_cdf); free(pat_items); pop_free(&pop);
  return db;
fail:
  free(cur); free(mark); free(pat_off); free(pat_cdf); free(pat_items); pop_free(&pop);
  if (db) { free(db->offsets); free(db->items); free(db); }
  return NULL;
}

/* Dense Bernoulli database: item i in a transaction with p_i = p_lo + (p_hi-p_lo)*i/(N-1). */
synth_db* synth_dense_bernoulli(uint64_t seed, uint32_t D, uint32_t N, double p_lo, double p_hi) {
  synth_db* db = (synth_db*)calloc(1, sizeof(synth_db));
  if (!db || db_init(db, D, (uint64_t)D * N / 2 + 16) != 0) { synth_free(db); return NULL; }
  rng_t r = rng_make(seed, 4);
  for (uint32_t t = 0; t < D; ++t) {
    for (uint32_t i = 0; i < N; ++i) {
      double p = N > 1 ? p_lo + (p_hi - p_lo) * (double)i / (double)(N - 1) : p_lo;
      if (rng_unit(&r) <= p) { if (db_push(db, i) != 0) { synth_free(db); return NULL; } }
    }
    db->offsets[t + 1] = (uint32_t)db->nnz;
  }
  return db;
}

/* Dense fixed-length database: exactly k distinct items per transaction, drawn one
 * at a time without replacement with weights p_i (as in synth_dense_bernoulli). */
synth_db* synth_dense_fixed(uint64_t seed, uint32_t D, uint32_t N, uint32_t k, double p_lo, double p_hi) {
  if (k > N) k = N;
  synth_db* db = (synth_db*)calloc(1, sizeof(synth_db));
  double* w = (double*)malloc(sizeof(double) * N);
  uint8_t* taken = (uint8_t*)malloc(N);
  uint32_t* cur = (uint32_t*)malloc(sizeof(uint32_t) * ((size_t)k + 1));
  if (!db || !w || !taken || !cur || db_init(db, D, (uint64_t)D * k + 16) != 0) {
    free(w); free(taken); free(cur); synth_free(db); return NULL;
  }
  for (uint32_t i = 0; i < N; ++i) w[i] = N > 1 ? p_lo + (p_hi - p_lo) * (double)i / (double)(N - 1) : p_lo;
  rng_t r = rng_make(seed, 5);
  for (uint32_t t = 0; t < D; ++t) {
    memset(taken, 0, N);
    double total = 0.0;
    for (uint32_t i = 0; i < N; ++i) total += w[i];
    for (uint32_t c = 0; c < k; ++c) {
      double u = rng_unit(&r) * total, acc = 0.0;
      uint32_t pick = N;
      for (uint32_t i = 0; i < N; ++i) {
        if (taken[i]) continue;
        acc += w[i];
        pick = i;
        if (acc >= u) break;
      }
      taken[pick] = 1; total -= w[pick]; cur[c] = pick;
    }
    qsort(cur, k, sizeof(uint32_t), cmp_u32);
    for (uint32_t c = 0; c < k; ++c) db_push(db, cur[c]);
    db->offsets[t + 1] = (uint32_t)db->nnz;
  }
  free(w); free(taken); free(cur);
  return db;
}

/* Raw SplitMix64 stream values, exposed so tests can pin this file's generator
 * against the published reference sequence. */
double synth_exp(double x) { return my_exp(x); }
double synth_log(double x) { return my_log(x); }

uint64_t synth_splitmix64_next(uint64_t* state) {
  *state += GAMMA64;
  return mix64(*state);
}
