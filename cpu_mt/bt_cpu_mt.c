/*
 * bt_cpu_mt.c -- a straightforward multithreaded CPU block-tree builder
 * (OpenMP), reported as a baseline beside the GPU build.  It builds the same
 * tree as the plain builder of the tests (the exported bit vectors, pointers
 * and leaf text), following the paper's construction:
 *
 *   - Karp-Rabin prefix fingerprints H(p) mod 2^61-1 (section 2), computed in
 *     parallel: per-thread chunk hashes, a sequential combine, a parallel
 *     expansion;
 *   - per level (section 3.1): block and pair fingerprints in hash tables;
 *     the window scan over the runs of consecutive blocks split over the
 *     threads, each window probing the tables and lowering a shared per-slot
 *     minimum with a compare-and-swap; every minimum that differs from the
 *     key's own start is verified byte by byte, and a mismatch (a
 *     fingerprint collision) falls back to an exact scan for that key;
 *   - marks, pointers and children as in section 3; the optional pruning
 *     pass and the leaf text, sequentially.
 *
 * The rank/select counters are not built: they are not part of the exported
 * tree.  Readings where the paper is silent are the same as the library's:
 * a block in no pair is marked, the last level is marked, windows are
 * restricted to runs, pruning conditions (i)-(iv) with the static (iii).
 */
#include "bt_cpu_mt.h"

#include <stdlib.h>
#include <string.h>

#include <omp.h>

#define Q61 ((1ull << 61) - 1)
#define NONE (~0ull)

typedef unsigned __int128 u128;

static inline uint64_t mulq(uint64_t a, uint64_t b) {
  u128 p = (u128)a * b;
  uint64_t r = (uint64_t)(p & Q61) + (uint64_t)(p >> 61);
  r = (r & Q61) + (r >> 61);
  return r >= Q61 ? r - Q61 : r;
}
static inline uint64_t addq(uint64_t a, uint64_t b) {
  uint64_t s = a + b;
  return s >= Q61 ? s - Q61 : s;
}
static inline uint64_t subq(uint64_t a, uint64_t b) { return a >= b ? a - b : a + Q61 - b; }
static uint64_t powq(uint64_t a, uint64_t e) {
  uint64_t r = 1;
  while (e) {
    if (e & 1) r = mulq(r, a);
    a = mulq(a, a);
    e >>= 1;
  }
  return r;
}
static uint64_t mix(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

/* Base B from the seed (the same published map the library uses). */
static uint64_t base_of(uint64_t seed) { return mix(seed) % (Q61 - 256) + 256; }

/* Lower *a to v if v is smaller (lock-free). */
static inline void atomic_min_u64(uint64_t* a, uint64_t v) {
  uint64_t cur = __atomic_load_n(a, __ATOMIC_RELAXED);
  while (v < cur && !__atomic_compare_exchange_n(a, &cur, v, 1, __ATOMIC_RELAXED, __ATOMIC_RELAXED)) {
  }
}

/* Open addressing: key -> slot (keys != NONE). */
typedef struct {
  uint64_t* key;
  uint64_t mask;
} table;

static int table_init(table* t, uint64_t n) {
  uint64_t cap = 16;
  while (cap < 2 * n) cap <<= 1;
  t->key = (uint64_t*)malloc(cap * sizeof(uint64_t));
  if (!t->key) return BTMT_ENOMEM;
  memset(t->key, 0xFF, cap * sizeof(uint64_t));
  t->mask = cap - 1;
  return BTMT_OK;
}
static uint64_t table_insert(table* t, uint64_t key) {
  uint64_t h = mix(key) & t->mask;
  while (t->key[h] != NONE && t->key[h] != key) h = (h + 1) & t->mask;
  t->key[h] = key;
  return h;
}
static inline uint64_t table_find(const table* t, uint64_t key) {
  uint64_t h = mix(key) & t->mask;
  for (;;) {
    const uint64_t k = t->key[h];
    if (k == key) return h;
    if (k == NONE) return NONE;
    h = (h + 1) & t->mask;
  }
}

typedef struct {
  uint64_t b, c;
  uint64_t *st, *len, *ptr, *off, *lo;
  uint8_t* mark;
} level;

static void level_free(level* v) {
  free(v->st);
  free(v->len);
  free(v->ptr);
  free(v->off);
  free(v->lo);
  free(v->mark);
  memset(v, 0, sizeof(*v));
}
static int level_alloc(level* v, uint64_t c) {
  const uint64_t m = c ? c : 1;
  v->c = c;
  v->st = (uint64_t*)malloc(m * 8);
  v->len = (uint64_t*)malloc(m * 8);
  v->ptr = (uint64_t*)calloc(m, 8);
  v->off = (uint64_t*)calloc(m, 8);
  v->lo = (uint64_t*)malloc(m * 8);
  v->mark = (uint8_t*)calloc(m, 1);
  return (v->st && v->len && v->ptr && v->off && v->lo && v->mark) ? BTMT_OK : BTMT_ENOMEM;
}

/* Block of level v holding position p (NONE if p is in no block). */
static uint64_t block_at(const level* v, uint64_t p) {
  uint64_t a = 0, z = v->c;
  while (a < z) {
    const uint64_t mid = (a + z) / 2;
    if (v->st[mid] <= p) a = mid + 1;
    else z = mid;
  }
  if (a == 0) return NONE;
  return p < v->st[a - 1] + v->len[a - 1] ? a - 1 : NONE;
}

/* End of the run of consecutive blocks that contains block k. */
static uint64_t run_end(const level* v, uint64_t k) {
  uint64_t e = v->st[k] + v->len[k];
  while (k + 1 < v->c && v->st[k + 1] == e) {
    k++;
    e += v->len[k];
  }
  return e;
}

typedef struct {
  const uint8_t* T;
  uint64_t n, B;
  uint64_t* H; /* H[p], p in [0, n] */
} text;

static inline uint64_t window(const text* x, uint64_t p, uint64_t L, uint64_t BL) {
  return subq(x->H[p + L], mulq(x->H[p], BL));
}

/* H[p] for every p, in parallel. */
static int prefix(text* x) {
  const uint64_t n = x->n, B = x->B;
  x->H = (uint64_t*)malloc((n + 1) * 8);
  if (!x->H) return BTMT_ENOMEM;
  const int P = omp_get_max_threads();
  uint64_t* part = (uint64_t*)calloc((size_t)P + 1, 8);
  if (!part) return BTMT_ENOMEM;
  const uint64_t step = (n + P - 1) / P;
#pragma omp parallel num_threads(P)
  {
    const int i = omp_get_thread_num();
    const uint64_t a = (uint64_t)i * step, e = a + step < n ? a + step : n;
    uint64_t h = 0;
    for (uint64_t p = a; p < e; p++) h = addq(mulq(h, B), (uint64_t)x->T[p] + 1);
    part[i + 1] = h;
  }
  /* part[i] becomes H(i * step). */
  uint64_t acc = 0;
  for (int i = 0; i < P; i++) {
    const uint64_t a = (uint64_t)i * step, e = a + step < n ? a + step : n;
    const uint64_t h = part[i + 1];
    part[i] = acc;
    if (e > a) acc = addq(mulq(acc, powq(B, e - a)), h);
  }
  part[P] = acc;
#pragma omp parallel num_threads(P)
  {
    const int i = omp_get_thread_num();
    const uint64_t a = (uint64_t)i * step, e = a + step < n ? a + step : n;
    uint64_t h = part[i];
    for (uint64_t p = a; p < e; p++) {
      x->H[p] = h;
      h = addq(mulq(h, B), (uint64_t)x->T[p] + 1);
    }
  }
  x->H[n] = part[P];
  free(part);
  return BTMT_OK;
}

/* The smallest p inside a run of level v with T[p, p+L) == T[s, s+L),
 * by direct comparison (the fallback after a fingerprint collision). */
static uint64_t exact_leftmost(const text* x, const level* v, uint64_t s, uint64_t L) {
  for (uint64_t k = 0; k < v->c; k++) {
    const uint64_t e = run_end(v, k);
    for (uint64_t p = v->st[k]; p < v->st[k] + v->len[k] && p + L <= e; p++) {
      if (p > s) return s;
      if (memcmp(x->T + p, x->T + s, L) == 0) return p;
    }
  }
  return s;
}

/* One level: leftmost occurrences of pairs and blocks, marks, pointers. */
static int build_level(const text* x, level* v, uint64_t* verify_bytes) {
  const uint64_t c = v->c, b = v->b;
  if (c == 0) return BTMT_OK;
  const uint64_t r = v->len[c - 1] < b ? v->len[c - 1] : 0;
  const uint64_t Bb = powq(x->B, b), Br = r ? powq(x->B, r) : 0;
  int rc = BTMT_OK;
  uint64_t* fp = (uint64_t*)malloc(c * 8);
  uint64_t* slot = (uint64_t*)malloc(c * 8);
  uint64_t* pslot = (uint64_t*)malloc(c * 8);
  uint64_t* run = (uint64_t*)malloc(c * 8);
  table bt = {0, 0}, pt = {0, 0};
  uint64_t *bmin = NULL, *pmin = NULL;
  if (!fp || !slot || !pslot || !run) {
    rc = BTMT_ENOMEM;
    goto out;
  }
#pragma omp parallel for schedule(static)
  for (uint64_t k = 0; k < c; k++) fp[k] = window(x, v->st[k], v->len[k], v->len[k] == b ? Bb : Br);
  for (uint64_t k = c; k-- > 0;) run[k] = (k + 1 < c && v->st[k + 1] == v->st[k] + v->len[k]) ? run[k + 1] : v->st[k] + v->len[k];
  /* Tables: blocks by fingerprint; pairs by their two block slots. */
  if (table_init(&bt, c) != BTMT_OK || table_init(&pt, c) != BTMT_OK) {
    rc = BTMT_ENOMEM;
    goto out;
  }
  uint64_t fp_tail = NONE, pretail = NONE;
  for (uint64_t k = 0; k < c; k++) {
    if (v->len[k] == b) slot[k] = table_insert(&bt, fp[k]);
    else {
      slot[k] = NONE;
      fp_tail = fp[k];
    }
  }
  for (uint64_t k = 0; k + 1 < c; k++) {
    pslot[k] = NONE;
    if (v->st[k + 1] != v->st[k] + b) continue;
    if (slot[k + 1] == NONE) pretail = slot[k];
    else pslot[k] = table_insert(&pt, (slot[k] << 32) | slot[k + 1]);
  }
  bmin = (uint64_t*)malloc((bt.mask + 1) * 8);
  pmin = (uint64_t*)malloc((pt.mask + 1) * 8);
  if (!bmin || !pmin) {
    rc = BTMT_ENOMEM;
    goto out;
  }
  memset(bmin, 0xFF, (bt.mask + 1) * 8);
  memset(pmin, 0xFF, (pt.mask + 1) * 8);
  uint64_t tail_min = NONE, tailpair_min = NONE;
  /* The window scan: every start p in block k whose window lies inside the
   * run; units of at most 4096 starts per block, spread over the threads. */
  const uint64_t per = (b + 4095) / 4096;
#pragma omp parallel for schedule(dynamic, 64) reduction(min : tail_min, tailpair_min)
  for (uint64_t unit = 0; unit < c * per; unit++) {
    const uint64_t k = unit / per, p0 = v->st[k] + (unit % per) * 4096;
    const uint64_t pe = v->st[k] + v->len[k] < p0 + 4096 ? v->st[k] + v->len[k] : p0 + 4096;
    const uint64_t av = run[k];
    for (uint64_t p = p0; p < pe; p++) {
      if (p + b <= av) {
        const uint64_t s1 = table_find(&bt, window(x, p, b, Bb));
        if (s1 != NONE) {
          atomic_min_u64(&bmin[s1], p);
          if (p + 2 * b <= av) {
            const uint64_t s2 = table_find(&bt, window(x, p + b, b, Bb));
            if (s2 != NONE) {
              const uint64_t ps = table_find(&pt, (s1 << 32) | s2);
              if (ps != NONE) atomic_min_u64(&pmin[ps], p);
            }
          }
          if (r && s1 == pretail && p + b + r <= av && window(x, p + b, r, Br) == fp_tail && p < tailpair_min)
            tailpair_min = p;
        }
      }
      if (r && p + r <= av && window(x, p, r, Br) == fp_tail && p < tail_min) tail_min = p;
    }
  }
  /* Pairs: verify the minimum; leftmost iff it is the pair's own start. */
  uint8_t* pairmark = (uint8_t*)calloc(c, 1);
  uint8_t* haspair = (uint8_t*)calloc(c, 1);
  if (!pairmark || !haspair) {
    free(pairmark);
    free(haspair);
    rc = BTMT_ENOMEM;
    goto out;
  }
  uint64_t vb = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : vb)
  for (uint64_t k = 0; k < c - 1; k++) {
    if (v->st[k + 1] != v->st[k] + v->len[k]) continue;
    haspair[k] = 1;
    const uint64_t s = v->st[k], L = v->len[k] + v->len[k + 1];
    uint64_t lo = pslot[k] != NONE ? pmin[pslot[k]] : (v->len[k + 1] < b ? tailpair_min : NONE);
    if (lo > s) lo = s;
    if (lo < s) {
      vb += 2 * L;
      if (memcmp(x->T + lo, x->T + s, L) != 0) lo = exact_leftmost(x, v, s, L);
    }
    pairmark[k] = lo == s;
  }
  for (uint64_t k = 0; k < c; k++) {
    const int left = k > 0 && haspair[k - 1], right = haspair[k];
    v->mark[k] = (uint8_t)((k > 0 && pairmark[k - 1]) || pairmark[k] || (!left && !right));
  }
  free(pairmark);
  free(haspair);
  /* Blocks: verified leftmost occurrence of every block, pointers of the
   * unmarked ones. */
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : vb)
  for (uint64_t k = 0; k < c; k++) {
    const uint64_t s = v->st[k], L = v->len[k];
    uint64_t lo = slot[k] != NONE ? bmin[slot[k]] : tail_min;
    if (lo > s) lo = s;
    if (lo < s) {
      vb += 2 * L;
      if (memcmp(x->T + lo, x->T + s, L) != 0) lo = exact_leftmost(x, v, s, L);
    }
    v->lo[k] = lo;
    if (!v->mark[k]) {
      const uint64_t j = block_at(v, lo);
      v->ptr[k] = j;
      v->off[k] = lo - v->st[j];
    }
  }
  *verify_bytes += vb;
out:
  free(fp);
  free(slot);
  free(pslot);
  free(run);
  free(bt.key);
  free(pt.key);
  free(bmin);
  free(pmin);
  return rc;
}

/* Children of the marked blocks (ceil(len / b_next) each, in text order). */
static int children(const level* v, level* w) {
  uint64_t cnt = 0;
  for (uint64_t k = 0; k < v->c; k++)
    if (v->mark[k]) cnt += (v->len[k] + w->b - 1) / w->b;
  if (level_alloc(w, cnt) != BTMT_OK) return BTMT_ENOMEM;
  uint64_t i = 0;
  for (uint64_t k = 0; k < v->c; k++) {
    if (!v->mark[k]) continue;
    const uint64_t e = v->st[k] + v->len[k];
    for (uint64_t s = v->st[k]; s < e; s += w->b, i++) {
      w->st[i] = s;
      w->len[i] = s + w->b <= e ? w->b : e - s;
    }
  }
  return BTMT_OK;
}

static void flag_range(const level* v, uint8_t* flag, uint64_t p, uint64_t L) {
  for (uint64_t j = block_at(v, p); j != NONE && j < v->c && v->st[j] < p + L; j++) flag[j] = 1;
}

/* The pruning pass, bottom-up and right to left (section 3.1): a marked
 * block becomes a pointer when (i) none of its children has children, (ii) no
 * pointer of its level targets it, (iii) no pointer of the level below (as
 * the pass over the level starts) targets a child, (iv) its leftmost
 * occurrence ends at or before its start. */
static int prune(level* lv, uint32_t L) {
  for (int l = (int)L - 2; l >= 0; l--) {
    level* v = &lv[l];
    level* w = &lv[l + 1];
    const int w_last = l + 1 == (int)L - 1;
    uint64_t* fc = (uint64_t*)calloc(v->c ? v->c : 1, 8);
    uint8_t* hit = (uint8_t*)calloc(v->c ? v->c : 1, 1);
    uint8_t* hitw = (uint8_t*)calloc(w->c ? w->c : 1, 1);
    uint8_t* gone = (uint8_t*)calloc(w->c ? w->c : 1, 1);
    uint64_t* nidx = (uint64_t*)malloc((w->c ? w->c : 1) * 8);
    if (!fc || !hit || !hitw || !gone || !nidx) {
      free(fc);
      free(hit);
      free(hitw);
      free(gone);
      free(nidx);
      return BTMT_ENOMEM;
    }
    for (uint64_t k = 0, i = 0; k < v->c; k++)
      if (v->mark[k]) {
        fc[k] = i;
        i += (v->len[k] + w->b - 1) / w->b;
      }
    for (uint64_t u = 0; u < v->c; u++)
      if (!v->mark[u]) flag_range(v, hit, v->st[v->ptr[u]] + v->off[u], v->len[u]);
    for (uint64_t u = 0; u < w->c; u++)
      if (!w->mark[u]) flag_range(w, hitw, w->st[w->ptr[u]] + w->off[u], w->len[u]);
    for (uint64_t k = v->c; k-- > 0;) {
      if (!v->mark[k]) continue;
      const uint64_t nch = (v->len[k] + w->b - 1) / w->b;
      int ok = !hit[k] && v->lo[k] + v->len[k] <= v->st[k];
      for (uint64_t i = 0; i < nch && ok; i++) {
        if (!w_last && w->mark[fc[k] + i]) ok = 0;
        if (hitw[fc[k] + i]) ok = 0;
      }
      if (!ok) continue;
      const uint64_t j = block_at(v, v->lo[k]);
      v->mark[k] = 0;
      v->ptr[k] = j;
      v->off[k] = v->lo[k] - v->st[j];
      flag_range(v, hit, v->lo[k], v->len[k]);
      for (uint64_t i = 0; i < nch; i++) gone[fc[k] + i] = 1;
    }
    uint64_t m = 0;
    for (uint64_t k = 0; k < w->c; k++) nidx[k] = gone[k] ? NONE : m++;
    for (uint64_t k = 0, i = 0; k < w->c; k++) {
      if (gone[k]) continue;
      w->st[i] = w->st[k];
      w->len[i] = w->len[k];
      w->mark[i] = w->mark[k];
      w->ptr[i] = w->mark[k] ? 0 : nidx[w->ptr[k]];
      w->off[i] = w->off[k];
      w->lo[i] = w->lo[k];
      i++;
    }
    w->c = m;
    free(fc);
    free(hit);
    free(hitw);
    free(gone);
    free(nidx);
  }
  return BTMT_OK;
}

typedef struct {
  uint8_t* buf;
  uint64_t len, cap;
  int failed; /* an allocation failed: the output is incomplete */
} out_buf;

static void put(out_buf* o, uint64_t x) {
  if (o->failed) return;
  if (o->len + 8 > o->cap) {
    uint64_t cap = o->cap ? 2 * o->cap : 4096;
    uint8_t* nb = (uint8_t*)realloc(o->buf, cap);
    if (!nb) {
      o->failed = 1;
      return;
    }
    o->buf = nb;
    o->cap = cap;
  }
  memcpy(o->buf + o->len, &x, 8);
  o->len += 8;
}

int btmt_build(const uint8_t* T, uint64_t n, uint32_t tau, uint32_t leaf, int do_prune, uint64_t seed,
               int threads, uint8_t** blob, uint64_t* blob_len) {
  if (!T || !blob || !blob_len || n == 0 || tau < 2 || leaf == 0) return BTMT_EINVAL;
  *blob = NULL;
  *blob_len = 0;
  if (threads > 0) omp_set_num_threads(threads);
  /* Level sizes: b_L = leaf, b_l = tau b_{l+1}, the smallest height with
   * tau * leaf * tau^h >= n. */
  uint32_t L = 1;
  u128 size = (u128)tau * leaf;
  while (size < n) {
    size *= tau;
    L++;
    if (L > 63) return BTMT_EINVAL;
  }
  level* lv = (level*)calloc(L, sizeof(level));
  if (!lv) return BTMT_ENOMEM;
  uint64_t b = leaf;
  for (int l = (int)L - 1; l >= 0; l--, b *= tau) lv[l].b = b;
  text x = {T, n, base_of(seed), NULL};
  int rc = prefix(&x);
  uint64_t vb = 0;
  if (rc == BTMT_OK) {
    const uint64_t c = (n + lv[0].b - 1) / lv[0].b;
    rc = level_alloc(&lv[0], c);
    for (uint64_t k = 0; k < c && rc == BTMT_OK; k++) {
      lv[0].st[k] = k * lv[0].b;
      lv[0].len[k] = (k + 1) * lv[0].b <= n ? lv[0].b : n - k * lv[0].b;
    }
  }
  for (uint32_t l = 0; l < L && rc == BTMT_OK; l++) {
    rc = build_level(&x, &lv[l], &vb);
    if (rc == BTMT_OK && l + 1 < L) rc = children(&lv[l], &lv[l + 1]);
  }
  if (rc == BTMT_OK && do_prune) rc = prune(lv, L);
  out_buf o = {NULL, 0, 0, 0};
  if (rc == BTMT_OK) {
    put(&o, 0x31454552544B4C42ull);
    put(&o, n);
    put(&o, tau);
    put(&o, leaf);
    put(&o, L);
    put(&o, (uint64_t)(do_prune != 0));
    for (uint32_t l = 0; l < L; l++) {
      const level* v = &lv[l];
      put(&o, v->c);
      put(&o, v->b);
      for (uint64_t k0 = 0; k0 < v->c; k0 += 64) {
        uint64_t word = 0;
        for (uint64_t k = k0; k < v->c && k < k0 + 64; k++)
          if (v->mark[k]) word |= 1ull << (k - k0);
        put(&o, word);
      }
      uint64_t np = 0;
      for (uint64_t k = 0; k < v->c; k++) np += !v->mark[k];
      put(&o, np);
      for (uint64_t k = 0; k < v->c; k++)
        if (!v->mark[k]) {
          put(&o, v->ptr[k]);
          put(&o, v->off[k]);
        }
    }
    /* Leaf text: the marked last-level blocks in order. */
    const level* z = &lv[L - 1];
    uint64_t nl = 0;
    for (uint64_t k = 0; k < z->c; k++)
      if (z->mark[k]) nl += z->len[k];
    put(&o, nl);
    uint64_t word = 0, fill = 0;
    for (uint64_t k = 0; k < z->c; k++) {
      if (!z->mark[k]) continue;
      for (uint64_t i = 0; i < z->len[k]; i++) {
        word |= (uint64_t)T[z->st[k] + i] << (8 * fill);
        if (++fill == 8) {
          put(&o, word);
          word = 0;
          fill = 0;
        }
      }
    }
    if (fill) put(&o, word);
    if (o.failed || !o.buf) rc = BTMT_ENOMEM;
  }
  for (uint32_t l = 0; l < L; l++) level_free(&lv[l]);
  free(lv);
  free(x.H);
  if (rc != BTMT_OK) {
    free(o.buf);
    return rc;
  }
  *blob = o.buf;
  *blob_len = o.len;
  return BTMT_OK;
}

void btmt_free(uint8_t* blob) { free(blob); }

int btmt_threads(void) { return omp_get_max_threads(); }
