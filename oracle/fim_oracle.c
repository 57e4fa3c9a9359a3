/*
 * CPU oracle for frequent-itemset mining -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load this file's library.  It shares no code, header, table or helper with
 * the GPU path (paper_2108_05038_gb300/csrc); both sides only read the same
 * CSR arrays written by the seeded input generator.
 *
 * Source of every definition: R. Kessl, "Parallel algorithms for mining of
 * frequent itemsets" (thesis, 2011; arXiv 2108.05038).
 *
 *  O1 oracle_eclat       -- Eclat-DFS / Eclat-DFS-Computation (App. B.3.2) over
 *                           sorted tidlists (Def. "Transaction id list", Ch. 2),
 *                           support of a union = size of the intersection of the
 *                           tidlists of two generating subsets (App. B.3.1 and
 *                           the Lemma/Corollary of Sec. 2.4).  Reading of the
 *                           garbled listing: an atom carries t(P u {a}); the step
 *                           for a_i < a_j forms t(P u {a_i,a_j}) =
 *                           t(P u {a_i}) n t(P u {a_j}), outputs P u {a_i,a_j} when
 *                           its support is >= minsupp, and recurses with the new
 *                           atoms and prefix P u {a_i}; frequent singletons are
 *                           output at the top; the empty set is never output.
 *  O1 oracle_eclat_mt    -- the same recursion with the one-item classes [a_i | later
 *                           atoms] handed to threads (the classes are independent,
 *                           Sec. 2.4); each thread keeps its own output, the outputs are
 *                           concatenated.  Used to time the oracle on every host core.
 *  O2 oracle_bruteforce  -- the definition itself (Def. "Frequent itemset",
 *                           Ch. 2): every non-empty subset of the item base,
 *                           support counted by scanning all transactions.
 *  O3 oracle_apriori     -- level-wise Apriori (App. B.1): candidates C_k from
 *                           pairs of frequent (k-1)-itemsets sharing their first
 *                           k-2 items, pruned when a (k-1)-subset is infrequent
 *                           (monotonicity, Thm. 2.1), counted by scanning the
 *                           transactions.
 *  O4 oracle_check       -- certificate from an output alone: exact recount by
 *                           tidlist intersection, singletons = item counts,
 *                           anti-monotone supports along prefixes (Thm. 2.1),
 *                           and completeness by downward closure (every
 *                           one-item extension X u {b}, b > max X, missing from
 *                           the output has support < minsupp).
 *  oracle_class_costs    -- the sample-based PBEC size estimate (Sec. 6.2 and
 *                           Phase 2, Sec. 8.2): a database sample D_s drawn with
 *                           replacement (Sec. 6.1), mined at the relative
 *                           minimum support, and the relative size
 *                           |[U] n F_s| / |F_s| of each class [U|E] with a
 *                           one-item prefix (Def. "Relative size of a PBEC").
 *
 * Relation >= : an itemset is frequent iff supp >= minsupp (Def. "Frequent
 * itemset"); Phase-4-Eclat prints ">" but the definition governs.
 * Precision: counts are exact integers; relative sizes are one IEEE double
 * division count / total.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* output container                                                          */

typedef struct {
  uint64_t n_sets;
  uint64_t cap_sets;
  uint64_t n_items;
  uint64_t cap_items;
  uint64_t* set_offsets; /* n_sets + 1 */
  uint32_t* set_items;   /* items ascending inside each set (original ids) */
  uint32_t* supports;
} or_result;

static or_result* res_new(void) {
  or_result* r = (or_result*)calloc(1, sizeof(or_result));
  if (!r) return NULL;
  r->cap_sets = 64; r->cap_items = 256;
  r->set_offsets = (uint64_t*)malloc(sizeof(uint64_t) * (r->cap_sets + 1));
  r->set_items = (uint32_t*)malloc(sizeof(uint32_t) * r->cap_items);
  r->supports = (uint32_t*)malloc(sizeof(uint32_t) * r->cap_sets);
  if (!r->set_offsets || !r->set_items || !r->supports) return NULL;
  r->set_offsets[0] = 0;
  return r;
}

void oracle_result_free(or_result* r) {
  if (!r) return;
  free(r->set_offsets); free(r->set_items); free(r->supports); free(r);
}

static int cmp_u32(const void* a, const void* b) {
  uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
  return (x > y) - (x < y);
}

/* append one itemset (items in any order; stored ascending) */
static int res_add(or_result* r, const uint32_t* items, uint32_t k, uint32_t supp) {
  if (r->n_sets == r->cap_sets) {
    uint64_t nc = r->cap_sets * 2;
    uint64_t* no = (uint64_t*)realloc(r->set_offsets, sizeof(uint64_t) * (nc + 1));
    if (!no) return -1;
    r->set_offsets = no;
    uint32_t* ns = (uint32_t*)realloc(r->supports, sizeof(uint32_t) * nc);
    if (!ns) return -1;
    r->supports = ns;
    r->cap_sets = nc;
  }
  while (r->n_items + k > r->cap_items) {
    uint64_t nc = r->cap_items * 2;
    uint32_t* ni = (uint32_t*)realloc(r->set_items, sizeof(uint32_t) * nc);
    if (!ni) return -1;
    r->set_items = ni; r->cap_items = nc;
  }
  uint32_t* dst = r->set_items + r->n_items;
  memcpy(dst, items, sizeof(uint32_t) * k);
  qsort(dst, k, sizeof(uint32_t), cmp_u32);
  r->n_items += k;
  r->supports[r->n_sets] = supp;
  r->n_sets += 1;
  r->set_offsets[r->n_sets] = r->n_items;
  return 0;
}

uint64_t oracle_result_n_sets(const or_result* r) { return r->n_sets; }
uint64_t oracle_result_n_items(const or_result* r) { return r->n_items; }
void oracle_result_copy(const or_result* r, uint64_t* offsets, uint32_t* items, uint32_t* supports) {
  memcpy(offsets, r->set_offsets, sizeof(uint64_t) * (r->n_sets + 1));
  if (r->n_items) memcpy(items, r->set_items, sizeof(uint32_t) * r->n_items);
  if (r->n_sets) memcpy(supports, r->supports, sizeof(uint32_t) * r->n_sets);
}

/* Lexicographic order of itemsets (Def. in Ch. 9): compare item by item; a
 * proper prefix comes first. */
static const or_result* g_sort_res;
static int cmp_sets(const void* a, const void* b) {
  uint64_t i = *(const uint64_t*)a, j = *(const uint64_t*)b;
  const uint32_t* x = g_sort_res->set_items + g_sort_res->set_offsets[i];
  const uint32_t* y = g_sort_res->set_items + g_sort_res->set_offsets[j];
  uint64_t nx = g_sort_res->set_offsets[i + 1] - g_sort_res->set_offsets[i];
  uint64_t ny = g_sort_res->set_offsets[j + 1] - g_sort_res->set_offsets[j];
  uint64_t n = nx < ny ? nx : ny;
  for (uint64_t k = 0; k < n; ++k) {
    if (x[k] != y[k]) return x[k] < y[k] ? -1 : 1;
  }
  return (nx > ny) - (nx < ny);
}

/* Sort the result canonically (not thread safe; the oracle is single threaded). */
int oracle_result_sort(or_result* r) {
  uint64_t n = r->n_sets;
  uint64_t* idx = (uint64_t*)malloc(sizeof(uint64_t) * (n ? n : 1));
  uint64_t* no = (uint64_t*)malloc(sizeof(uint64_t) * (n + 1));
  uint32_t* ni = (uint32_t*)malloc(sizeof(uint32_t) * (r->n_items ? r->n_items : 1));
  uint32_t* ns = (uint32_t*)malloc(sizeof(uint32_t) * (n ? n : 1));
  if (!idx || !no || !ni || !ns) { free(idx); free(no); free(ni); free(ns); return -1; }
  for (uint64_t i = 0; i < n; ++i) idx[i] = i;
  g_sort_res = r;
  qsort(idx, n, sizeof(uint64_t), cmp_sets);
  uint64_t pos = 0;
  no[0] = 0;
  for (uint64_t i = 0; i < n; ++i) {
    uint64_t s = idx[i];
    uint64_t k = r->set_offsets[s + 1] - r->set_offsets[s];
    memcpy(ni + pos, r->set_items + r->set_offsets[s], sizeof(uint32_t) * k);
    pos += k;
    no[i + 1] = pos;
    ns[i] = r->supports[s];
  }
  free(idx); free(r->set_offsets); free(r->set_items); free(r->supports);
  r->set_offsets = no; r->set_items = ni; r->supports = ns;
  r->cap_sets = n; r->cap_items = r->n_items ? r->n_items : 1;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* vertical representation: tidlist of every item (Def. tidlist, Ch. 2).     */
/* Set semantics: a duplicate item inside one transaction counts once.       */

typedef struct {
  uint32_t N;
  uint64_t* off;   /* N + 1 */
  uint32_t* tids;  /* ascending per item */
} tidlists;

static void tl_free(tidlists* t) { free(t->off); free(t->tids); }

static int tl_build(tidlists* t, const uint32_t* off, const uint32_t* items, uint32_t D, uint32_t N) {
  t->N = N;
  t->tids = NULL;
  t->off = (uint64_t*)calloc((size_t)N + 1, sizeof(uint64_t));
  uint32_t* last = (uint32_t*)malloc(sizeof(uint32_t) * (N ? N : 1));
  if (!t->off || !last) { free(last); return -1; }
  for (uint32_t i = 0; i < N; ++i) last[i] = UINT32_MAX;
  for (uint32_t tx = 0; tx < D; ++tx)
    for (uint32_t k = off[tx]; k < off[tx + 1]; ++k) {
      uint32_t it = items[k];
      if (it >= N) { free(last); return -2; }
      if (last[it] != tx) { last[it] = tx; t->off[it + 1]++; }
    }
  for (uint32_t i = 0; i < N; ++i) t->off[i + 1] += t->off[i];
  t->tids = (uint32_t*)malloc(sizeof(uint32_t) * (t->off[N] ? t->off[N] : 1));
  uint64_t* pos = (uint64_t*)malloc(sizeof(uint64_t) * (N ? N : 1));
  if (!t->tids || !pos) { free(last); free(pos); return -1; }
  for (uint32_t i = 0; i < N; ++i) { pos[i] = t->off[i]; last[i] = UINT32_MAX; }
  for (uint32_t tx = 0; tx < D; ++tx)
    for (uint32_t k = off[tx]; k < off[tx + 1]; ++k) {
      uint32_t it = items[k];
      if (last[it] != tx) { last[it] = tx; t->tids[pos[it]++] = tx; }
    }
  free(pos); free(last);
  return 0;
}

/* |a n b| written to out (may be NULL: count only); both ascending */
static uint32_t intersect(const uint32_t* a, uint32_t na, const uint32_t* b, uint32_t nb, uint32_t* out) {
  uint32_t i = 0, j = 0, n = 0;
  while (i < na && j < nb) {
    if (a[i] < b[j]) ++i;
    else if (a[i] > b[j]) ++j;
    else { if (out) out[n] = a[i]; ++n; ++i; ++j; }
  }
  return n;
}

/* ------------------------------------------------------------------------ */
/* O1: Eclat-DFS over tidlists                                               */

typedef struct {
  uint32_t item;
  uint32_t n;
  uint32_t* tids; /* owned */
} atom;

typedef struct {
  uint32_t minsup;
  uint32_t* prefix; /* current P, up to depth */
  or_result* out;
  int err;          /* -1 allocation failure, 1 more than `limit` itemsets */
  uint64_t limit;   /* 0 = none */
} eclat_ctx;

static void eclat_rec(eclat_ctx* c, atom* A, uint32_t nA, uint32_t depth);

/* One step of Eclat-DFS-Computation(A, P): the class of atom i, i.e. every
 * P u {a_i, a_j} (j > i) from t(P u {a_i}) n t(P u {a_j}), output when frequent,
 * then the recursion on the new atoms with prefix P u {a_i}. */
static void eclat_class(eclat_ctx* c, atom* A, uint32_t nA, uint32_t i, uint32_t depth) {
  atom* Ai = (atom*)malloc(sizeof(atom) * (nA - i > 1 ? nA - i - 1 : 1));
  uint32_t nAi = 0;
  if (!Ai) { c->err = -1; return; }
  c->prefix[depth] = A[i].item;
  for (uint32_t j = i + 1; j < nA; ++j) {
    uint32_t cap = A[i].n < A[j].n ? A[i].n : A[j].n;
    uint32_t* buf = (uint32_t*)malloc(sizeof(uint32_t) * (cap ? cap : 1));
    if (!buf) { c->err = -1; break; }
    uint32_t n = intersect(A[i].tids, A[i].n, A[j].tids, A[j].n, buf);
    if (n >= c->minsup) {
      Ai[nAi].item = A[j].item; Ai[nAi].n = n; Ai[nAi].tids = buf; ++nAi;
      c->prefix[depth + 1] = A[j].item;
      if (res_add(c->out, c->prefix, depth + 2, n) != 0) { c->err = -1; break; }
      if (c->limit && c->out->n_sets > c->limit) { c->err = 1; break; }
    } else {
      free(buf);
    }
  }
  if (!c->err) eclat_rec(c, Ai, nAi, depth + 1);
  for (uint32_t k = 0; k < nAi; ++k) free(Ai[k].tids);
  free(Ai);
}

/* Eclat-DFS-Computation(A, P): A holds atoms a with t(P u {a}); every atom is
 * itself already frequent and already output by the caller. */
static void eclat_rec(eclat_ctx* c, atom* A, uint32_t nA, uint32_t depth) {
  for (uint32_t i = 0; i < nA && !c->err; ++i) eclat_class(c, A, nA, i, depth);
}

/* Eclat-DFS(D, minsupp, F) that gives up once F holds more than `limit`
 * itemsets (limit 0: never): returns 0 on success, 1 when |F| > limit, -2 on an
 * item id >= N, -3 on minsup == 0, -1 on allocation failure. Items are visited
 * in id order. */
static int eclat_limited(const uint32_t* off, const uint32_t* items, uint32_t D, uint32_t N, uint32_t minsup,
                         uint64_t limit, or_result** out) {
  *out = NULL;
  if (minsup == 0) return -3;
  tidlists t;
  int rc = tl_build(&t, off, items, D, N);
  if (rc != 0) { tl_free(&t); return rc; }
  or_result* r = res_new();
  atom* A = (atom*)malloc(sizeof(atom) * (N ? N : 1));
  uint32_t* prefix = (uint32_t*)malloc(sizeof(uint32_t) * ((size_t)N + 2));
  if (!r || !A || !prefix) { tl_free(&t); oracle_result_free(r); free(A); free(prefix); return -1; }
  uint32_t nA = 0;
  for (uint32_t it = 0; it < N; ++it) {
    uint32_t n = (uint32_t)(t.off[it + 1] - t.off[it]);
    if (n >= minsup) {
      A[nA].item = it; A[nA].n = n; A[nA].tids = t.tids + t.off[it]; ++nA;
      if (res_add(r, &it, 1, n) != 0) { rc = -1; break; }
      if (limit && r->n_sets > limit) { rc = 1; break; }
    }
  }
  eclat_ctx c = {minsup, prefix, r, 0, limit};
  if (rc == 0) {
    /* top-level atoms point into the tidlist table, which eclat_rec never frees */
    eclat_rec(&c, A, nA, 0);
    rc = c.err;
  }
  free(A); free(prefix); tl_free(&t);
  if (rc != 0) { oracle_result_free(r); return rc; }
  *out = r;
  return 0;
}

int oracle_eclat(const uint32_t* off, const uint32_t* items, uint32_t D, uint32_t N, uint32_t minsup,
                 or_result** out) {
  return eclat_limited(off, items, D, N, minsup, 0, out);
}

/* O1 on several threads: the top-level classes are claimed one at a time
 * (lowest unclaimed atom first) under a mutex; every thread runs the same
 * eclat_class on its own output and prefix buffer. */
typedef struct {
  atom* A;
  uint32_t nA, minsup, N;
  uint32_t next;
  pthread_mutex_t mu;
  int err;
} mt_shared;

typedef struct {
  mt_shared* sh;
  or_result* out;
  int err;
} mt_worker;

static void* mt_main(void* arg) {
  mt_worker* w = (mt_worker*)arg;
  mt_shared* sh = w->sh;
  uint32_t* prefix = (uint32_t*)malloc(sizeof(uint32_t) * ((size_t)sh->N + 2));
  w->out = res_new();
  if (!prefix || !w->out) { free(prefix); w->err = -1; return NULL; }
  eclat_ctx c = {sh->minsup, prefix, w->out, 0, 0};
  for (;;) {
    pthread_mutex_lock(&sh->mu);
    const uint32_t i = sh->err ? sh->nA : sh->next++;
    pthread_mutex_unlock(&sh->mu);
    if (i >= sh->nA) break;
    eclat_class(&c, sh->A, sh->nA, i, 0);
    if (c.err) {
      pthread_mutex_lock(&sh->mu);
      sh->err = c.err;
      pthread_mutex_unlock(&sh->mu);
      break;
    }
  }
  w->err = c.err;
  free(prefix);
  return NULL;
}

int oracle_eclat_mt(const uint32_t* off, const uint32_t* items, uint32_t D, uint32_t N, uint32_t minsup,
                    uint32_t n_threads, or_result** out) {
  *out = NULL;
  if (minsup == 0) return -3;
  if (n_threads == 0) n_threads = 1;
  tidlists t;
  int rc = tl_build(&t, off, items, D, N);
  if (rc != 0) { tl_free(&t); return rc; }
  or_result* r = res_new();
  atom* A = (atom*)malloc(sizeof(atom) * (N ? N : 1));
  mt_worker* ws = (mt_worker*)calloc(n_threads, sizeof(mt_worker));
  pthread_t* th = (pthread_t*)calloc(n_threads, sizeof(pthread_t));
  if (!r || !A || !ws || !th) { tl_free(&t); oracle_result_free(r); free(A); free(ws); free(th); return -1; }
  uint32_t nA = 0;
  for (uint32_t it = 0; it < N && rc == 0; ++it) {
    uint32_t n = (uint32_t)(t.off[it + 1] - t.off[it]);
    if (n >= minsup) {
      A[nA].item = it; A[nA].n = n; A[nA].tids = t.tids + t.off[it]; ++nA;
      if (res_add(r, &it, 1, n) != 0) rc = -1;
    }
  }
  mt_shared sh;
  sh.A = A; sh.nA = nA; sh.minsup = minsup; sh.N = N; sh.next = 0; sh.err = 0;
  pthread_mutex_init(&sh.mu, NULL);
  uint32_t started = 0;
  if (rc == 0)
    for (; started < n_threads; ++started) {
      ws[started].sh = &sh;
      if (pthread_create(&th[started], NULL, mt_main, &ws[started]) != 0) break;
    }
  if (rc == 0 && started == 0) rc = -1;
  for (uint32_t k = 0; k < started; ++k) pthread_join(th[k], NULL);
  for (uint32_t k = 0; k < started && rc == 0; ++k) {
    if (ws[k].err) { rc = ws[k].err; break; }
    const or_result* o = ws[k].out;
    for (uint64_t s = 0; s < o->n_sets && rc == 0; ++s)
      if (res_add(r, o->set_items + o->set_offsets[s], (uint32_t)(o->set_offsets[s + 1] - o->set_offsets[s]),
                  o->supports[s]) != 0)
        rc = -1;
  }
  for (uint32_t k = 0; k < n_threads; ++k) oracle_result_free(ws[k].out);
  pthread_mutex_destroy(&sh.mu);
  free(A); free(ws); free(th); tl_free(&t);
  if (rc != 0) { oracle_result_free(r); return rc; }
  *out = r;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* O2: brute force over all non-empty subsets (N <= 20)                      */

int oracle_bruteforce(const uint32_t* off, const uint32_t* items, uint32_t D, uint32_t N, uint32_t minsup,
                      or_result** out) {
  *out = NULL;
  if (minsup == 0) return -3;
  if (N > 20) return -4;
  uint32_t* mask = (uint32_t*)calloc(D ? D : 1, sizeof(uint32_t));
  or_result* r = res_new();
  if (!mask || !r) { free(mask); oracle_result_free(r); return -1; }
  for (uint32_t tx = 0; tx < D; ++tx)
    for (uint32_t k = off[tx]; k < off[tx + 1]; ++k) {
      if (items[k] >= N) { free(mask); oracle_result_free(r); return -2; }
      mask[tx] |= 1u << items[k];
    }
  uint32_t buf[32];
  for (uint32_t s = 1; s < (1u << N); ++s) {
    uint32_t cnt = 0;
    for (uint32_t tx = 0; tx < D; ++tx) cnt += (mask[tx] & s) == s;
    if (cnt >= minsup) {
      uint32_t k = 0;
      for (uint32_t b = 0; b < N; ++b) if (s & (1u << b)) buf[k++] = b;
      if (res_add(r, buf, k, cnt) != 0) { free(mask); oracle_result_free(r); return -1; }
    }
  }
  free(mask);
  *out = r;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* O3: level-wise Apriori                                                    */

typedef struct {
  uint32_t k;       /* itemset size */
  uint64_t n;       /* number of itemsets */
  uint32_t* items;  /* n * k, each ascending, whole list lexicographically sorted */
  uint32_t* supp;
} level_t;

static uint32_t g_cmp_k;
static int cmp_kset(const void* a, const void* b) {
  const uint32_t* x = (const uint32_t*)a; const uint32_t* y = (const uint32_t*)b;
  for (uint32_t i = 0; i < g_cmp_k; ++i) if (x[i] != y[i]) return x[i] < y[i] ? -1 : 1;
  return 0;
}
static int level_contains(const level_t* L, const uint32_t* s) {
  uint64_t lo = 0, hi = L->n;
  while (lo < hi) {
    uint64_t mid = (lo + hi) / 2;
    const uint32_t* m = L->items + mid * L->k;
    int c = 0;
    for (uint32_t i = 0; i < L->k && !c; ++i) if (m[i] != s[i]) c = m[i] < s[i] ? -1 : 1;
    if (c == 0) return 1;
    if (c < 0) lo = mid + 1; else hi = mid;
  }
  return 0;
}

int oracle_apriori(const uint32_t* off, const uint32_t* items, uint32_t D, uint32_t N, uint32_t minsup,
                   or_result** out) {
  *out = NULL;
  if (minsup == 0) return -3;
  or_result* r = res_new();
  uint8_t* mark = (uint8_t*)calloc(N ? N : 1, 1);
  uint32_t* cnt1 = (uint32_t*)calloc(N ? N : 1, sizeof(uint32_t));
  if (!r || !mark || !cnt1) { oracle_result_free(r); free(mark); free(cnt1); return -1; }
  /* pass 1: item counts (set semantics) */
  for (uint32_t tx = 0; tx < D; ++tx) {
    for (uint32_t k = off[tx]; k < off[tx + 1]; ++k) {
      uint32_t it = items[k];
      if (it >= N) { oracle_result_free(r); free(mark); free(cnt1); return -2; }
      if (!mark[it]) { mark[it] = 1; cnt1[it]++; }
    }
    for (uint32_t k = off[tx]; k < off[tx + 1]; ++k) mark[items[k]] = 0;
  }
  level_t L;
  L.k = 1; L.n = 0;
  L.items = (uint32_t*)malloc(sizeof(uint32_t) * (N ? N : 1));
  L.supp = (uint32_t*)malloc(sizeof(uint32_t) * (N ? N : 1));
  if (!L.items || !L.supp) { free(L.items); free(L.supp); oracle_result_free(r); free(mark); free(cnt1); return -1; }
  for (uint32_t it = 0; it < N; ++it)
    if (cnt1[it] >= minsup) { L.items[L.n] = it; L.supp[L.n] = cnt1[it]; L.n++; res_add(r, &it, 1, cnt1[it]); }
  free(cnt1);
  int rc = 0;
  uint32_t* sub = (uint32_t*)malloc(sizeof(uint32_t) * ((size_t)N + 2));
  while (L.n > 1 && rc == 0) {
    uint32_t k = L.k + 1;
    /* Generate-Candidates: join sets sharing the first k-2 items, prune by subsets */
    uint64_t cap = 1024, nc = 0;
    uint32_t* C = (uint32_t*)malloc(sizeof(uint32_t) * cap * k);
    if (!C || !sub) { free(C); rc = -1; break; }
    for (uint64_t a = 0; a < L.n && rc == 0; ++a) {
      const uint32_t* x = L.items + a * L.k;
      for (uint64_t b = a + 1; b < L.n; ++b) {
        const uint32_t* y = L.items + b * L.k;
        if (L.k > 1 && memcmp(x, y, sizeof(uint32_t) * (L.k - 1)) != 0) break; /* sorted: no later match */
        uint32_t* c = (uint32_t*)malloc(sizeof(uint32_t) * k);
        memcpy(c, x, sizeof(uint32_t) * L.k);
        c[L.k] = y[L.k - 1];
        int ok = 1;
        for (uint32_t drop = 0; drop + 2 < k && ok; ++drop) { /* the two generators are frequent */
          uint32_t m = 0;
          for (uint32_t i = 0; i < k; ++i) if (i != drop) sub[m++] = c[i];
          ok = level_contains(&L, sub);
        }
        if (ok) {
          if (nc == cap) { cap *= 2; uint32_t* nC = (uint32_t*)realloc(C, sizeof(uint32_t) * cap * k); if (!nC) { free(c); rc = -1; break; } C = nC; }
          memcpy(C + nc * k, c, sizeof(uint32_t) * k);
          ++nc;
        }
        free(c);
      }
    }
    if (rc != 0) { free(C); break; }
    /* Compute-Support: scan the transactions */
    uint32_t* sc = (uint32_t*)calloc(nc ? nc : 1, sizeof(uint32_t));
    if (!sc) { free(C); rc = -1; break; }
    for (uint32_t tx = 0; tx < D; ++tx) {
      uint32_t len = off[tx + 1] - off[tx];
      if (len < k) continue;
      for (uint32_t q = off[tx]; q < off[tx + 1]; ++q) mark[items[q]] = 1;
      for (uint64_t ci = 0; ci < nc; ++ci) {
        const uint32_t* c = C + ci * k;
        uint32_t i = 0;
        while (i < k && mark[c[i]]) ++i;
        sc[ci] += (i == k);
      }
      for (uint32_t q = off[tx]; q < off[tx + 1]; ++q) mark[items[q]] = 0;
    }
    level_t NL;
    NL.k = k; NL.n = 0;
    NL.items = (uint32_t*)malloc(sizeof(uint32_t) * (nc ? nc : 1) * k);
    NL.supp = (uint32_t*)malloc(sizeof(uint32_t) * (nc ? nc : 1));
    if (!NL.items || !NL.supp) { free(NL.items); free(NL.supp); free(C); free(sc); rc = -1; break; }
    for (uint64_t ci = 0; ci < nc; ++ci)
      if (sc[ci] >= minsup) {
        memcpy(NL.items + NL.n * k, C + ci * k, sizeof(uint32_t) * k);
        NL.supp[NL.n] = sc[ci];
        NL.n++;
        if (res_add(r, C + ci * k, k, sc[ci]) != 0) rc = -1;
      }
    free(C); free(sc);
    g_cmp_k = k;
    /* keep L_k sorted lexicographically for the next join (joined lists stay sorted,
       the sort only guards the invariant) */
    {
      uint32_t* tmp = (uint32_t*)malloc(sizeof(uint32_t) * (NL.n ? NL.n : 1) * (k + 1));
      for (uint64_t i = 0; i < NL.n; ++i) { memcpy(tmp + i * (k + 1), NL.items + i * k, sizeof(uint32_t) * k); tmp[i * (k + 1) + k] = NL.supp[i]; }
      g_cmp_k = k + 1;
      qsort(tmp, NL.n, sizeof(uint32_t) * (k + 1), cmp_kset);
      for (uint64_t i = 0; i < NL.n; ++i) { memcpy(NL.items + i * k, tmp + i * (k + 1), sizeof(uint32_t) * k); NL.supp[i] = tmp[i * (k + 1) + k]; }
      free(tmp);
    }
    free(L.items); free(L.supp);
    L = NL;
  }
  free(L.items); free(L.supp); free(mark); free(sub);
  if (rc != 0) { oracle_result_free(r); return rc; }
  *out = r;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* O4: certificate check of an output (no mining)                            */
/*                                                                           */
/* Input sets must be ascending inside each set.  Returns 0 when every check  */
/* passes, else a positive code naming the first failure, with *bad_index the */
/* offending set (or item for code 5):                                       */
/*   1 support differs from the tidlist recount                              */
/*   2 support below minsup                                                  */
/*   3 parent (set minus its last item) missing or with smaller support      */
/*   4 a missing one-item extension is frequent (incompleteness)             */
/*   5 a frequent singleton is missing / singleton support != item count     */
/*   6 duplicate set / malformed input                                       */
/* check_stride > 1 checks only every check_stride-th set for 1, 3 and 4.    */

static const uint32_t* g_ck_items;
static const uint64_t* g_ck_off;
static int cmp_idx_sets(const void* a, const void* b) {
  uint64_t i = *(const uint64_t*)a, j = *(const uint64_t*)b;
  const uint32_t* x = g_ck_items + g_ck_off[i]; const uint32_t* y = g_ck_items + g_ck_off[j];
  uint64_t nx = g_ck_off[i + 1] - g_ck_off[i], ny = g_ck_off[j + 1] - g_ck_off[j];
  uint64_t n = nx < ny ? nx : ny;
  for (uint64_t k = 0; k < n; ++k) if (x[k] != y[k]) return x[k] < y[k] ? -1 : 1;
  return (nx > ny) - (nx < ny);
}
/* index of set equal to s[0..k) in the sorted index, or -1 */
static int64_t find_set(const uint64_t* idx, uint64_t n, const uint32_t* s, uint64_t k) {
  uint64_t lo = 0, hi = n;
  while (lo < hi) {
    uint64_t mid = (lo + hi) / 2;
    uint64_t m = idx[mid];
    const uint32_t* x = g_ck_items + g_ck_off[m];
    uint64_t nx = g_ck_off[m + 1] - g_ck_off[m];
    uint64_t nn = nx < k ? nx : k;
    int c = 0;
    for (uint64_t q = 0; q < nn && !c; ++q) if (x[q] != s[q]) c = x[q] < s[q] ? -1 : 1;
    if (!c) c = (nx > k) - (nx < k);
    if (c == 0) return (int64_t)m;
    if (c < 0) lo = mid + 1; else hi = mid;
  }
  return -1;
}

int oracle_check(const uint32_t* off, const uint32_t* items, uint32_t D, uint32_t N, uint32_t minsup,
                 uint64_t n_sets, const uint64_t* set_offsets, const uint32_t* set_items, const uint32_t* supports,
                 uint64_t check_stride, uint64_t* bad_index) {
  *bad_index = 0;
  if (check_stride == 0) check_stride = 1;
  tidlists t;
  int rc = tl_build(&t, off, items, D, N);
  if (rc != 0) { tl_free(&t); return -1; }
  uint64_t* idx = (uint64_t*)malloc(sizeof(uint64_t) * (n_sets ? n_sets : 1));
  uint32_t* cur = (uint32_t*)malloc(sizeof(uint32_t) * (D ? D : 1));
  uint32_t* tmp = (uint32_t*)malloc(sizeof(uint32_t) * (D ? D : 1));
  uint32_t* ext = (uint32_t*)malloc(sizeof(uint32_t) * ((size_t)N + 2));
  if (!idx || !cur || !tmp || !ext) { rc = -1; goto done; }
  for (uint64_t i = 0; i < n_sets; ++i) {
    for (uint64_t k = set_offsets[i]; k + 1 < set_offsets[i + 1]; ++k)
      if (set_items[k] >= set_items[k + 1]) { rc = 6; *bad_index = i; goto done; }
    if (set_offsets[i + 1] == set_offsets[i]) { rc = 6; *bad_index = i; goto done; }
    for (uint64_t k = set_offsets[i]; k < set_offsets[i + 1]; ++k)
      if (set_items[k] >= N) { rc = 6; *bad_index = i; goto done; }
    idx[i] = i;
  }
  g_ck_items = set_items; g_ck_off = set_offsets;
  qsort(idx, n_sets, sizeof(uint64_t), cmp_idx_sets);
  for (uint64_t i = 0; i + 1 < n_sets; ++i)
    if (cmp_idx_sets(&idx[i], &idx[i + 1]) == 0) { rc = 6; *bad_index = idx[i + 1]; goto done; }
  /* singletons: present iff frequent, support = item count */
  for (uint32_t it = 0; it < N; ++it) {
    uint32_t c = (uint32_t)(t.off[it + 1] - t.off[it]);
    int64_t f = find_set(idx, n_sets, &it, 1);
    if ((c >= minsup) != (f >= 0) || (f >= 0 && supports[f] != c)) { rc = 5; *bad_index = it; goto done; }
  }
  /* completeness at the empty set is the singleton check above */
  for (uint64_t i = 0; i < n_sets; i += check_stride) {
    const uint32_t* s = set_items + set_offsets[i];
    uint64_t k = set_offsets[i + 1] - set_offsets[i];
    if (supports[i] < minsup) { rc = 2; *bad_index = i; goto done; }
    /* recount by tidlist intersection of the singletons */
    uint32_t n = (uint32_t)(t.off[s[0] + 1] - t.off[s[0]]);
    memcpy(cur, t.tids + t.off[s[0]], sizeof(uint32_t) * n);
    for (uint64_t q = 1; q < k; ++q) {
      n = intersect(cur, n, t.tids + t.off[s[q]], (uint32_t)(t.off[s[q] + 1] - t.off[s[q]]), tmp);
      memcpy(cur, tmp, sizeof(uint32_t) * n);
    }
    if (n != supports[i]) { rc = 1; *bad_index = i; goto done; }
    if (k > 1) {
      int64_t p = find_set(idx, n_sets, s, k - 1);
      if (p < 0 || supports[p] < supports[i]) { rc = 3; *bad_index = i; goto done; }
    }
    /* every extension by a larger item that is absent must be infrequent */
    memcpy(ext, s, sizeof(uint32_t) * k);
    for (uint32_t b = s[k - 1] + 1; b < N; ++b) {
      uint32_t nb = (uint32_t)(t.off[b + 1] - t.off[b]);
      if (nb < minsup) continue;
      ext[k] = b;
      if (find_set(idx, n_sets, ext, k + 1) >= 0) continue;
      uint32_t c = intersect(cur, n, t.tids + t.off[b], nb, NULL);
      if (c >= minsup) { rc = 4; *bad_index = i; goto done; }
    }
  }
  rc = 0;
done:
  free(idx); free(cur); free(tmp); free(ext); tl_free(&t);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Sample-based class-cost estimate                                          */
/*                                                                           */
/* Item order of the classes: the kept items (support >= prefilter_minsup in  */
/* the whole database; prefilter 0 keeps every item) sorted by ascending      */
/* support, ties by ascending id -- the ascending-support order of Sec. B.4.2.*/
/* Sample: m = max(ceil(rate * D), min(D, 738)) transactions drawn with      */
/* replacement (Sec. 6.1; 738 = the Theorem 6.1 size for eps = delta = 0.05); */
/* draw k uses the SplitMix64 output x_k = mix(seed + (k + 1) * gamma) (the   */
/* k-th output of the stream started at state seed; Steele et al. 2014) and   */
/* the transaction index ((x_k >> 32) * D) >> 32.  The sample keeps only the   */
/* kept items and is mined at minsup_s = max(1, ceil(rel_minsup * m)); while   */
/* the sample then has more than `limit` frequent itemsets (limit 0: never),  */
/* minsup_s doubles (a reading: the thesis does not treat a sample whose      */
/* itemsets explode; a coarser threshold keeps the estimate's cost bounded).  */
/* cost[r] = #{X in F_s : the first item of X in the class order is rank r}   */
/*           / |F_s|  (0 when F_s is empty);  order = ranks by cost desc,     */
/* ties by rank asc (LPT order, Sec. 8.2).                                    */

static uint64_t sm64_at(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

static const uint32_t* g_rank_supp;
static int cmp_by_supp(const void* a, const void* b) {
  uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
  if (g_rank_supp[x] != g_rank_supp[y]) return g_rank_supp[x] < g_rank_supp[y] ? -1 : 1;
  return (x > y) - (x < y);
}
static const double* g_cost;
static int cmp_by_cost(const void* a, const void* b) {
  uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
  if (g_cost[x] != g_cost[y]) return g_cost[x] > g_cost[y] ? -1 : 1;
  return (x > y) - (x < y);
}

/* rank order of the kept items; rank_item[r] = original id; returns N_f */
int oracle_item_order(const uint32_t* off, const uint32_t* items, uint32_t D, uint32_t N, uint32_t prefilter_minsup,
                      uint32_t* rank_item, uint32_t* n_kept) {
  tidlists t;
  if (tl_build(&t, off, items, D, N) != 0) { tl_free(&t); return -1; }
  uint32_t* supp = (uint32_t*)malloc(sizeof(uint32_t) * (N ? N : 1));
  if (!supp) { tl_free(&t); return -1; }
  uint32_t nk = 0;
  for (uint32_t it = 0; it < N; ++it) {
    supp[it] = (uint32_t)(t.off[it + 1] - t.off[it]);
    if (supp[it] >= prefilter_minsup) rank_item[nk++] = it;
  }
  g_rank_supp = supp;
  qsort(rank_item, nk, sizeof(uint32_t), cmp_by_supp);
  *n_kept = nk;
  free(supp); tl_free(&t);
  return 0;
}

/* the sample's itemsets sorted by (length, rank sequence): sets P u {e} with the
 * same prefix P are then contiguous */
static const uint32_t* g_rs_items;
static const uint64_t* g_rs_off;
static int cmp_len_seq(const void* a, const void* b) {
  uint64_t i = *(const uint64_t*)a, j = *(const uint64_t*)b;
  uint64_t ni = g_rs_off[i + 1] - g_rs_off[i], nj = g_rs_off[j + 1] - g_rs_off[j];
  if (ni != nj) return ni < nj ? -1 : 1;
  const uint32_t* x = g_rs_items + g_rs_off[i];
  const uint32_t* y = g_rs_items + g_rs_off[j];
  for (uint64_t k = 0; k < ni; ++k) if (x[k] != y[k]) return x[k] < y[k] ? -1 : 1;
  return 0;
}

/* kind 0: cost = #sample FIs of the class (the thesis's measure, Sec. 8.2).
 * kind 1: cost = #AND+popcount intersections the bitmap Eclat performs for the
 * class on the sample, in the class order: the class of row r counts its
 * level-2 candidates (the sample-frequent rows after r) plus, for every
 * sample FI P whose first row is r, k_P (k_P - 1) / 2 where k_P is the number
 * of sample FIs P u {e} with e after P's last row (each child P u {e_k} of P
 * is intersected with the later survivors of P). */
int oracle_class_costs_limit(const uint32_t* off, const uint32_t* items, uint32_t D, uint32_t N,
                             uint32_t prefilter_minsup, double sample_rate, double rel_minsup, uint64_t seed, int kind,
                             uint64_t limit, double* cost_out, uint32_t* order_out, uint32_t* n_kept_out,
                             uint64_t* n_sample_fis, uint32_t* minsup_used) {
  if (!(sample_rate > 0.0 && sample_rate <= 1.0) || !(rel_minsup >= 0.0 && rel_minsup <= 1.0) || D == 0) return -3;
  uint32_t* rank_item = (uint32_t*)malloc(sizeof(uint32_t) * (N ? N : 1));
  int32_t* rank_of = (int32_t*)malloc(sizeof(int32_t) * (N ? N : 1));
  if (!rank_item || !rank_of) { free(rank_item); free(rank_of); return -1; }
  uint32_t nk = 0;
  if (oracle_item_order(off, items, D, N, prefilter_minsup, rank_item, &nk) != 0) { free(rank_item); free(rank_of); return -1; }
  for (uint32_t it = 0; it < N; ++it) rank_of[it] = -1;
  for (uint32_t r = 0; r < nk; ++r) rank_of[rank_item[r]] = (int32_t)r;
  /* m = max(ceil(rate D), min(D, m0)), m0 = the Theorem 6.1 size for eps = delta = 0.05 */
  double m0 = ceil(log(2.0 / 0.05) / (2.0 * 0.05 * 0.05));
  double md = ceil(sample_rate * (double)D);
  if (md < m0) md = m0 < (double)D ? m0 : (double)D;
  uint64_t m = (uint64_t)md;
  if (m < 1) m = 1;
  double ms = ceil(rel_minsup * (double)m);
  uint32_t minsup_s = ms < 1.0 ? 1u : (uint32_t)ms;
  /* sample database over kept items only */
  uint32_t* soff = (uint32_t*)malloc(sizeof(uint32_t) * (m + 1));
  uint64_t cap = 1024, nnz = 0;
  uint32_t* sit = (uint32_t*)malloc(sizeof(uint32_t) * cap);
  if (!soff || !sit) { free(rank_item); free(rank_of); free(soff); free(sit); return -1; }
  soff[0] = 0;
  for (uint64_t k = 0; k < m; ++k) {
    uint64_t x = sm64_at(seed, k);
    uint32_t tx = (uint32_t)(((x >> 32) * (uint64_t)D) >> 32);
    for (uint32_t q = off[tx]; q < off[tx + 1]; ++q) {
      if (items[q] >= N) { free(rank_item); free(rank_of); free(soff); free(sit); return -2; }
      if (rank_of[items[q]] < 0) continue;
      if (nnz == cap) { cap *= 2; uint32_t* ns = (uint32_t*)realloc(sit, sizeof(uint32_t) * cap); if (!ns) { free(rank_item); free(rank_of); free(soff); free(sit); return -1; } sit = ns; }
      sit[nnz++] = items[q];
    }
    soff[k + 1] = (uint32_t)nnz;
  }
  or_result* fs = NULL;
  int rc;
  for (;;) {
    rc = eclat_limited(soff, sit, (uint32_t)m, N, minsup_s, limit, &fs);
    if (rc != 1) break;
    minsup_s = minsup_s > UINT32_MAX / 2 ? UINT32_MAX : 2 * minsup_s;
  }
  free(soff); free(sit);
  if (minsup_used) *minsup_used = minsup_s;
  if (rc != 0) { free(rank_item); free(rank_of); return rc; }
  uint64_t* cnt = (uint64_t*)calloc(nk ? nk : 1, sizeof(uint64_t));
  uint32_t* ord = (uint32_t*)malloc(sizeof(uint32_t) * (nk ? nk : 1));
  if (!cnt || !ord) { free(cnt); free(ord); free(rank_item); free(rank_of); oracle_result_free(fs); return -1; }
  uint64_t total = 0;
  if (kind == 0) {
    for (uint64_t i = 0; i < fs->n_sets; ++i) {
      int32_t best = INT32_MAX;
      for (uint64_t q = fs->set_offsets[i]; q < fs->set_offsets[i + 1]; ++q) {
        int32_t rr = rank_of[fs->set_items[q]];
        if (rr < best) best = rr;
      }
      cnt[best]++;
    }
    total = fs->n_sets;
  } else {
    /* rewrite every set as its ascending rank sequence */
    uint32_t* rs = (uint32_t*)malloc(sizeof(uint32_t) * (fs->n_items ? fs->n_items : 1));
    uint64_t* idx = (uint64_t*)malloc(sizeof(uint64_t) * (fs->n_sets ? fs->n_sets : 1));
    if (!rs || !idx) { free(rs); free(idx); free(cnt); free(ord); free(rank_item); free(rank_of); oracle_result_free(fs); return -1; }
    for (uint64_t q = 0; q < fs->n_items; ++q) rs[q] = (uint32_t)rank_of[fs->set_items[q]];
    for (uint64_t i = 0; i < fs->n_sets; ++i) {
      qsort(rs + fs->set_offsets[i], fs->set_offsets[i + 1] - fs->set_offsets[i], sizeof(uint32_t), cmp_u32);
      idx[i] = i;
    }
    g_rs_items = rs; g_rs_off = fs->set_offsets;
    qsort(idx, fs->n_sets, sizeof(uint64_t), cmp_len_seq);
    /* level 2: the singletons of the sample in rank order, each with the later ones as candidates */
    uint64_t n1s = 0;
    for (uint64_t i = 0; i < fs->n_sets; ++i) n1s += (fs->set_offsets[i + 1] - fs->set_offsets[i]) == 1;
    uint64_t pos = 0;
    for (uint64_t k = 0; k < fs->n_sets; ++k) {
      uint64_t i = idx[k];
      if (fs->set_offsets[i + 1] - fs->set_offsets[i] != 1) break;
      cnt[rs[fs->set_offsets[i]]] += n1s - 1 - pos;
      ++pos;
    }
    /* deeper: runs of sets (same length >= 2) sharing all but their last row */
    uint64_t k = 0;
    while (k < fs->n_sets) {
      uint64_t i = idx[k];
      uint64_t len = fs->set_offsets[i + 1] - fs->set_offsets[i];
      if (len < 2) { ++k; continue; }
      uint64_t run = 1;
      while (k + run < fs->n_sets) {
        uint64_t j = idx[k + run];
        if (fs->set_offsets[j + 1] - fs->set_offsets[j] != len) break;
        if (memcmp(rs + fs->set_offsets[i], rs + fs->set_offsets[j], sizeof(uint32_t) * (len - 1)) != 0) break;
        ++run;
      }
      cnt[rs[fs->set_offsets[i]]] += run * (run - 1) / 2;
      k += run;
    }
    for (uint32_t r = 0; r < nk; ++r) total += cnt[r];
    free(rs); free(idx);
  }
  for (uint32_t r = 0; r < nk; ++r) cost_out[r] = total ? (double)cnt[r] / (double)total : 0.0;
  for (uint32_t r = 0; r < nk; ++r) ord[r] = r;
  g_cost = cost_out;
  qsort(ord, nk, sizeof(uint32_t), cmp_by_cost);
  memcpy(order_out, ord, sizeof(uint32_t) * nk);
  *n_kept_out = nk;
  *n_sample_fis = fs->n_sets;
  free(cnt); free(ord); free(rank_item); free(rank_of); oracle_result_free(fs);
  return 0;
}

int oracle_class_costs_kind(const uint32_t* off, const uint32_t* items, uint32_t D, uint32_t N, uint32_t prefilter_minsup,
                            double sample_rate, double rel_minsup, uint64_t seed, int kind, double* cost_out,
                            uint32_t* order_out, uint32_t* n_kept_out, uint64_t* n_sample_fis) {
  return oracle_class_costs_limit(off, items, D, N, prefilter_minsup, sample_rate, rel_minsup, seed, kind,
                                  (uint64_t)1 << 20, cost_out, order_out, n_kept_out, n_sample_fis, NULL);
}

int oracle_class_costs(const uint32_t* off, const uint32_t* items, uint32_t D, uint32_t N, uint32_t prefilter_minsup,
                       double sample_rate, double rel_minsup, uint64_t seed, double* cost_out, uint32_t* order_out,
                       uint32_t* n_kept_out, uint64_t* n_sample_fis) {
  return oracle_class_costs_kind(off, items, D, N, prefilter_minsup, sample_rate, rel_minsup, seed, 0, cost_out,
                                 order_out, n_kept_out, n_sample_fis);
}

/* SplitMix64 at a counter, exposed for pinning against the published stream. */
uint64_t oracle_splitmix64_at(uint64_t seed, uint64_t k) { return sm64_at(seed, k); }
