/*
 * bt_oracle.c -- plain, single-threaded CPU block-tree builder.
 *
 * TEST INFRASTRUCTURE ONLY (see bt_oracle.h).  Written for a reader who checks
 * it against the paper by eye: no blocking, no fusion, no reordering beyond
 * what the definitions state.  Every function names the passage it follows.
 *
 * Readings of the paper that this file takes where the paper is silent:
 *  - sizing: b_L = leaf_len, b_l = tau*b_{l+1}; the height is the smallest h
 *    with s0*leaf_len*tau^h >= n (s0 = root arity, default tau); the root has
 *    s = ceil(n/b_1) children and only the globally last block may be short
 *    (section 3 assumes n = s*tau^h; the caption of Figure 1 allows the
 *    irregular case);
 *  - a block in no pair of consecutive blocks is marked (it has no pair that
 *    could be leftmost and must keep its content);
 *  - the last level is marked like the others; its marked blocks store text;
 *  - leftmost occurrence LO(x) is the minimum start over ALL of T;
 *  - pruning (section 3.1, "Optional Pruning") runs after construction, from
 *    the second-to-last level up, right to left over each level, and turns a
 *    marked block k into a pointer when (i) none of its children has
 *    children, (ii) no pointer of its own level has a target window
 *    overlapping k, (iii) no pointer of the next level targets one of k's
 *    children, and (iv) LO(S(k)) + |k| <= start(k).  In (ii) the pointers
 *    created earlier in the same pass count; in (iii) the next level's
 *    pointers are taken as they stand when the pass over the level starts.
 */
#include "bt_oracle.h"

#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

#define UNSET UINT64_MAX
#define MERSENNE61 ((1ull << 61) - 1)

/* ------------------------------------------------------------------ */
/* Karp-Rabin fingerprints (section 2, definition of phi)             */
/* ------------------------------------------------------------------ */

static uint64_t mulmod(uint64_t a, uint64_t b, uint64_t q) {
  return (uint64_t)(((u128)a * b) % q);
}

static uint64_t powmod(uint64_t a, uint64_t e, uint64_t q) {
  uint64_t r = 1 % q;
  a %= q;
  while (e) {
    if (e & 1) r = mulmod(r, a, q);
    a = mulmod(a, a, q);
    e >>= 1;
  }
  return r;
}

/* splitmix64 (Steele, Lea, Flood 2014) -- used only to turn a seed into a base. */
static uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

uint64_t bto_base(uint64_t seed, uint64_t q) {
  if (q == 0) q = MERSENNE61;
  return splitmix64(seed) % (q - 256) + 256;
}

/* Symbols enter the fingerprint as byte+1, so that the alphabet is [1, 256]
 * as in the paper's T in [1, sigma]^n. */
uint64_t bto_fingerprint(const uint8_t* T, uint64_t s, uint64_t len, uint64_t B, uint64_t q) {
  if (q == 0) q = MERSENNE61;
  uint64_t h = 0;
  for (uint64_t i = s; i < s + len; i++) h = (mulmod(h, B, q) + (uint64_t)T[i] + 1) % q;
  return h;
}

/* ------------------------------------------------------------------ */
/* Leftmost occurrences (section 3.1, first and second phase)         */
/* ------------------------------------------------------------------ */

typedef struct {
  uint64_t verify_bytes;
  uint64_t collisions;
} scan_stats;

typedef struct {
  uint64_t* fp;
  int64_t* head;
  uint64_t mask;
} fp_map;

static int map_init(fp_map* m, uint64_t nkeys) {
  uint64_t cap = 16;
  while (cap < 2 * nkeys) cap <<= 1;
  m->fp = (uint64_t*)malloc(cap * sizeof(uint64_t));
  m->head = (int64_t*)malloc(cap * sizeof(int64_t));
  if (!m->fp || !m->head) return BTO_ENOMEM;
  for (uint64_t i = 0; i < cap; i++) m->head[i] = -1;
  m->mask = cap - 1;
  return BTO_OK;
}

static void map_free(fp_map* m) {
  free(m->fp);
  free(m->head);
}

static uint64_t map_slot(const fp_map* m, uint64_t fp) {
  uint64_t i = splitmix64(fp) & m->mask;
  while (m->head[i] != -1 && m->fp[i] != fp) i = (i + 1) & m->mask;
  return i;
}

typedef struct {
  const uint64_t* st;
  const uint64_t* len;
} keyref;

static const uint64_t* g_sort_len;
static int by_len(const void* a, const void* b) {
  uint64_t x = g_sort_len[*(const uint64_t*)a], y = g_sort_len[*(const uint64_t*)b];
  return x < y ? -1 : x > y;
}

/*
 * For every key string x_k = T[st[k], st[k]+len[k]) find LO(x_k), the
 * smallest p with T[p, p+len[k]) = x_k.  The keys' fingerprints go into a
 * hash table; one rolling pass over all windows of T in increasing position
 * probes it; a probe hit is accepted only after a byte comparison, so the
 * first accepted window of a key is its leftmost occurrence.  The rolling
 * step is the relation phi(s..e) = phi(s-1..e-1)*r - T[s-1]*r^(e-s+1) + T[e]
 * (section 4.3).
 */
static int leftmost_all(const uint8_t* T, uint64_t n, uint64_t B, uint64_t q, const uint64_t* st,
                        const uint64_t* len, uint64_t m, uint64_t* lo, scan_stats* ss) {
  if (m == 0) return BTO_OK;
  uint64_t* order = (uint64_t*)malloc(m * sizeof(uint64_t));
  int64_t* next = (int64_t*)malloc(m * sizeof(int64_t));
  if (!order || !next) {
    free(order);
    free(next);
    return BTO_ENOMEM;
  }
  for (uint64_t k = 0; k < m; k++) {
    order[k] = k;
    lo[k] = UNSET;
  }
  g_sort_len = len;
  qsort(order, m, sizeof(uint64_t), by_len);

  int rc = BTO_OK;
  for (uint64_t g0 = 0; g0 < m && rc == BTO_OK;) {
    uint64_t L = len[order[g0]], g1 = g0;
    while (g1 < m && len[order[g1]] == L) g1++;
    fp_map map;
    rc = map_init(&map, g1 - g0);
    if (rc != BTO_OK) break;
    uint64_t maxst = 0;
    for (uint64_t t = g0; t < g1; t++) {
      uint64_t k = order[t];
      uint64_t fp = bto_fingerprint(T, st[k], L, B, q);
      uint64_t s = map_slot(&map, fp);
      map.fp[s] = fp;
      next[k] = map.head[s];
      map.head[s] = (int64_t)k;
      if (st[k] > maxst) maxst = st[k];
    }
    uint64_t unresolved = g1 - g0;
    uint64_t BL = powmod(B, L, q);
    uint64_t fp = bto_fingerprint(T, 0, L, B, q);
    for (uint64_t p = 0; p + L <= n && p <= maxst && unresolved; p++) {
      if (p > 0) {
        uint64_t out = mulmod((uint64_t)T[p - 1] + 1, BL, q);
        fp = (mulmod(fp, B, q) + q - out + (uint64_t)T[p + L - 1] + 1) % q;
      }
      uint64_t s = map_slot(&map, fp);
      if (map.head[s] == -1) continue;
      for (int64_t k = map.head[s]; k != -1; k = next[k]) {
        if (lo[k] != UNSET) continue;
        int equal;
        if (st[k] == p) {
          equal = 1;
        } else {
          ss->verify_bytes += 2 * L;
          equal = memcmp(T + p, T + st[k], L) == 0;
        }
        if (equal) {
          lo[k] = p;
          unresolved--;
        } else {
          ss->collisions++;
        }
      }
    }
    map_free(&map);
    if (unresolved) rc = BTO_EINTERNAL; /* every key occurs at its own start */
    g0 = g1;
  }
  free(order);
  free(next);
  return rc;
}

/* ------------------------------------------------------------------ */
/* Tree                                                               */
/* ------------------------------------------------------------------ */

typedef struct {
  uint64_t b;       /* nominal block length of the level                */
  uint64_t c;       /* number of blocks                                 */
  uint64_t* st;     /* block starts, increasing                         */
  uint64_t* len;    /* block lengths (only the last block of T is short) */
  uint8_t* mark;    /* 1 = marked (inner node, or leaf text on level L)  */
  uint64_t* ptr;    /* unmarked: index of the block holding LO            */
  uint64_t* off;    /* unmarked: LO - st[ptr]                             */
  uint64_t* lo;     /* LO of the block's string (unpruned construction)   */
  uint64_t* fc;     /* marked, not last level: index of the first child   */
  uint64_t* cnt;    /* nsym counts per block                              */
  uint64_t* pc;     /* unmarked: nsym counts of T[st[ptr], st[ptr]+off)   */
} olvl;

struct bto_tree {
  uint64_t n, tau, leaf;
  int prune;
  uint32_t L;
  olvl* lv;
  uint64_t stats[64 * BTO_ST_FIELDS];
  uint8_t* leaftext;
  uint64_t leafn;
  uint64_t* leafpos; /* per last-level block: offset of its text in leaftext */
  int sym[256];      /* byte -> dense symbol index, -1 if absent            */
  uint32_t nsym;
  uint64_t* pre;     /* level 1: nsym counts of T[0, st[k])                 */
};

static void lvl_free(olvl* v) {
  free(v->st);
  free(v->len);
  free(v->mark);
  free(v->ptr);
  free(v->off);
  free(v->lo);
  free(v->fc);
  free(v->cnt);
  free(v->pc);
  memset(v, 0, sizeof(*v));
}

static int lvl_alloc(olvl* v, uint64_t c) {
  v->c = c;
  uint64_t k = c ? c : 1;
  v->st = (uint64_t*)calloc(k, sizeof(uint64_t));
  v->len = (uint64_t*)calloc(k, sizeof(uint64_t));
  v->mark = (uint8_t*)calloc(k, 1);
  v->ptr = (uint64_t*)calloc(k, sizeof(uint64_t));
  v->off = (uint64_t*)calloc(k, sizeof(uint64_t));
  v->lo = (uint64_t*)calloc(k, sizeof(uint64_t));
  if (!v->st || !v->len || !v->mark || !v->ptr || !v->off || !v->lo) return BTO_ENOMEM;
  return BTO_OK;
}

void bto_free(bto_tree* t) {
  if (!t) return;
  if (t->lv)
    for (uint32_t l = 0; l < t->L; l++) lvl_free(&t->lv[l]);
  free(t->lv);
  free(t->leaftext);
  free(t->leafpos);
  free(t->pre);
  free(t);
}

/* Index of the block of level v that contains position p, or UNSET. */
static uint64_t block_of(const olvl* v, uint64_t p) {
  uint64_t lo = 0, hi = v->c;
  while (lo < hi) {
    uint64_t mid = (lo + hi) / 2;
    if (v->st[mid] <= p) lo = mid + 1;
    else hi = mid;
  }
  if (lo == 0) return UNSET;
  uint64_t k = lo - 1;
  return p < v->st[k] + v->len[k] ? k : UNSET;
}

/* Does [p, p+L) lie inside consecutive blocks of level v? */
static int inside_run(const olvl* v, uint64_t p, uint64_t L) {
  uint64_t k = block_of(v, p);
  if (k == UNSET) return 0;
  uint64_t end = v->st[k] + v->len[k];
  while (end < p + L) {
    k++;
    if (k >= v->c || v->st[k] != end) return 0;
    end += v->len[k];
  }
  return 1;
}

/* Block sizes per level (section 3 and the sizing reading above). */
static int plan_sizes(uint64_t n, uint32_t tau, uint32_t leaf, const bto_opts* o, uint64_t** bout,
                      uint32_t* Lout) {
  if (o && o->level_sizes) {
    uint32_t L = o->nlevels;
    if (L == 0 || L > 64) return BTO_EINVAL;
    for (uint32_t l = 0; l < L; l++) {
      if (o->level_sizes[l] == 0) return BTO_EINVAL;
      if (l + 1 < L && (o->level_sizes[l] < 2 * o->level_sizes[l + 1] ||
                        o->level_sizes[l] % o->level_sizes[l + 1] != 0))
        return BTO_EINVAL;
    }
    uint64_t* b = (uint64_t*)malloc(L * sizeof(uint64_t));
    if (!b) return BTO_ENOMEM;
    memcpy(b, o->level_sizes, L * sizeof(uint64_t));
    *bout = b;
    *Lout = L;
    return BTO_OK;
  }
  uint64_t s0 = (o && o->root_arity) ? o->root_arity : tau;
  uint32_t h = 0;
  u128 size = (u128)s0 * leaf; /* s0 * leaf * tau^h */
  while (size < n) {
    size *= tau;
    h++;
    if (h > 62) return BTO_EINVAL;
  }
  uint32_t L = h + 1;
  uint64_t* b = (uint64_t*)malloc(L * sizeof(uint64_t));
  if (!b) return BTO_ENOMEM;
  b[L - 1] = leaf;
  for (int l = (int)L - 2; l >= 0; l--) b[l] = b[l + 1] * tau;
  *bout = b;
  *Lout = L;
  return BTO_OK;
}

/*
 * One level of the construction (section 3, marking rule; section 3.1, first
 * and second phase): pairs of consecutive blocks, their leftmost occurrences,
 * marks, then the leftmost occurrence of every block and the pointers of the
 * unmarked ones.
 */
static int build_level(bto_tree* t, const uint8_t* T, uint32_t l, uint64_t B, uint64_t q) {
  olvl* v = &t->lv[l];
  uint64_t c = v->c;
  uint64_t* S = &t->stats[l * BTO_ST_FIELDS];
  scan_stats ss = {0, 0};
  int rc = BTO_OK;

  uint64_t* pst = (uint64_t*)malloc((c ? c : 1) * sizeof(uint64_t));
  uint64_t* plen = (uint64_t*)malloc((c ? c : 1) * sizeof(uint64_t));
  uint64_t* pidx = (uint64_t*)malloc((c ? c : 1) * sizeof(uint64_t));
  uint64_t* plo = (uint64_t*)malloc((c ? c : 1) * sizeof(uint64_t));
  uint8_t* pairmark = (uint8_t*)calloc(c ? c : 1, 1);
  uint8_t* haspair = (uint8_t*)calloc(c ? c : 1, 1);
  if (!pst || !plen || !pidx || !plo || !pairmark || !haspair) {
    rc = BTO_ENOMEM;
    goto done;
  }

  /* Pairs B_k B_{k+1} of blocks consecutive in T (section 3). */
  uint64_t np = 0;
  for (uint64_t k = 0; k + 1 < c; k++) {
    if (v->st[k + 1] == v->st[k] + v->len[k]) {
      haspair[k] = 1;
      pst[np] = v->st[k];
      plen[np] = v->len[k] + v->len[k + 1];
      pidx[np] = k;
      np++;
    }
  }
  rc = leftmost_all(T, t->n, B, q, pst, plen, np, plo, &ss);
  if (rc != BTO_OK) goto done;
  for (uint64_t i = 0; i < np; i++) {
    if (plo[i] == pst[i]) pairmark[pidx[i]] = 1;
    /* The leftmost occurrence of a pair lies inside consecutive blocks of
     * this level (it lies inside a marked pair or block of the level above). */
    if (!inside_run(v, plo[i], plen[i])) {
      rc = BTO_EINTERNAL;
      goto done;
    }
  }
  /* Mark both blocks of a leftmost pair; keep blocks that belong to no pair. */
  uint64_t nmarked = 0;
  for (uint64_t k = 0; k < c; k++) {
    int left = k > 0 && haspair[k - 1], right = haspair[k];
    int m = (k > 0 && pairmark[k - 1]) || pairmark[k] || (!left && !right);
    v->mark[k] = (uint8_t)m;
    nmarked += m;
  }

  /* Leftmost occurrence of every block string (second phase; the marked
   * blocks' values are kept for pruning). */
  rc = leftmost_all(T, t->n, B, q, v->st, v->len, c, v->lo, &ss);
  if (rc != BTO_OK) goto done;
  for (uint64_t u = 0; u < c; u++) {
    if (v->mark[u]) continue;
    uint64_t p = v->lo[u], L = v->len[u];
    uint64_t j = block_of(v, p);
    if (j == UNSET || !v->mark[j] || p + L > v->st[u]) {
      rc = BTO_EINTERNAL;
      goto done;
    }
    if (p + L > v->st[j] + v->len[j]) {
      if (j + 1 >= c || v->st[j + 1] != v->st[j] + v->len[j] || !v->mark[j + 1] ||
          p + L > v->st[j + 1] + v->len[j + 1]) {
        rc = BTO_EINTERNAL;
        goto done;
      }
    }
    v->ptr[u] = j;
    v->off[u] = p - v->st[j];
  }

  uint64_t cov = 0;
  for (uint64_t k = 0; k < c; k++) cov += v->len[k];
  S[BTO_ST_NBLOCKS] = c;
  S[BTO_ST_B] = v->b;
  S[BTO_ST_COV] = cov;
  S[BTO_ST_NMARKED] = nmarked;
  S[BTO_ST_NPAIRS] = np;
  S[BTO_ST_VERIFY_BYTES] = ss.verify_bytes;
  S[BTO_ST_COLLISIONS] = ss.collisions;

done:
  free(pst);
  free(plen);
  free(pidx);
  free(plo);
  free(pairmark);
  free(haspair);
  return rc;
}

/* Children of the marked blocks of level l (section 3: marked blocks are
 * inner nodes; a block of length len has ceil(len / b_{l+1}) children). */
static int make_children(bto_tree* t, uint32_t l) {
  olvl* v = &t->lv[l];
  olvl* w = &t->lv[l + 1];
  uint64_t bn = w->b, cnt = 0;
  for (uint64_t k = 0; k < v->c; k++)
    if (v->mark[k]) cnt += (v->len[k] + bn - 1) / bn;
  int rc = lvl_alloc(w, cnt);
  if (rc != BTO_OK) return rc;
  uint64_t i = 0;
  for (uint64_t k = 0; k < v->c; k++) {
    if (!v->mark[k]) continue;
    for (uint64_t s = v->st[k]; s < v->st[k] + v->len[k]; s += bn) {
      w->st[i] = s;
      uint64_t e = v->st[k] + v->len[k];
      w->len[i] = (s + bn <= e) ? bn : e - s;
      i++;
    }
  }
  return BTO_OK;
}

/* First child index of every marked block of level l (children are stored
 * in the order of their parents). */
static void link_children(bto_tree* t, uint32_t l) {
  olvl* v = &t->lv[l];
  free(v->fc);
  v->fc = (uint64_t*)calloc(v->c ? v->c : 1, sizeof(uint64_t));
  uint64_t bn = t->lv[l + 1].b, i = 0;
  for (uint64_t k = 0; k < v->c; k++) {
    if (!v->mark[k]) continue;
    v->fc[k] = i;
    i += (v->len[k] + bn - 1) / bn;
  }
}

/* Set flag[j] for every block j of level v that [p, p+L) overlaps. */
static void flag_window(const olvl* v, uint8_t* flag, uint64_t p, uint64_t L) {
  uint64_t j = block_of(v, p);
  while (j != UNSET && j < v->c && v->st[j] < p + L) {
    flag[j] = 1;
    j++;
  }
}

/* Optional pruning (section 3.1), under the reading in the file header. */
static int prune_tree(bto_tree* t) {
  for (int l = (int)t->L - 2; l >= 0; l--) {
    olvl* v = &t->lv[l];
    olvl* w = &t->lv[l + 1];
    int w_last = (l + 1 == (int)t->L - 1);
    link_children(t, (uint32_t)l);
    uint8_t* hit = (uint8_t*)calloc(v->c ? v->c : 1, 1);      /* level l targets  */
    uint8_t* hitw = (uint8_t*)calloc(w->c ? w->c : 1, 1);     /* level l+1 targets */
    uint8_t* gone = (uint8_t*)calloc(w->c ? w->c : 1, 1);     /* deleted children */
    if (!hit || !hitw || !gone) {
      free(hit);
      free(hitw);
      free(gone);
      return BTO_ENOMEM;
    }
    for (uint64_t u = 0; u < v->c; u++)
      if (!v->mark[u]) flag_window(v, hit, v->st[v->ptr[u]] + v->off[u], v->len[u]);
    for (uint64_t u = 0; u < w->c; u++)
      if (!w->mark[u]) flag_window(w, hitw, w->st[w->ptr[u]] + w->off[u], w->len[u]);
    uint64_t bn = w->b;
    for (uint64_t kk = v->c; kk-- > 0;) {
      if (!v->mark[kk]) continue;
      uint64_t f = v->fc[kk], nch = (v->len[kk] + bn - 1) / bn;
      int ok = !hit[kk] && v->lo[kk] + v->len[kk] <= v->st[kk];
      for (uint64_t i = 0; i < nch && ok; i++) {
        uint64_t ch = f + i;
        if (!w_last && w->mark[ch]) ok = 0; /* (i) a child has children    */
        if (hitw[ch]) ok = 0;               /* (iii) a child is a target   */
      }
      if (!ok) continue;
      uint64_t p = v->lo[kk];
      uint64_t j = block_of(v, p);
      if (j == UNSET || !v->mark[j]) {
        free(hit);
        free(hitw);
        free(gone);
        return BTO_EINTERNAL;
      }
      v->mark[kk] = 0;
      v->ptr[kk] = j;
      v->off[kk] = p - v->st[j];
      flag_window(v, hit, p, v->len[kk]); /* (ii) for blocks further left */
      for (uint64_t i = 0; i < nch; i++) gone[f + i] = 1;
    }
    /* Renumber level l+1 without the deleted children. */
    uint64_t* nidx = (uint64_t*)malloc((w->c ? w->c : 1) * sizeof(uint64_t));
    if (!nidx) {
      free(hit);
      free(hitw);
      free(gone);
      return BTO_ENOMEM;
    }
    uint64_t m = 0;
    for (uint64_t k = 0; k < w->c; k++) nidx[k] = gone[k] ? UNSET : m++;
    for (uint64_t k = 0, i = 0; k < w->c; k++) {
      if (gone[k]) continue;
      w->st[i] = w->st[k];
      w->len[i] = w->len[k];
      w->mark[i] = w->mark[k];
      w->ptr[i] = w->mark[k] ? 0 : nidx[w->ptr[k]];
      w->off[i] = w->off[k];
      w->lo[i] = w->lo[k];
      if (!w->mark[k] && w->ptr[i] == UNSET) {
        free(nidx);
        free(hit);
        free(hitw);
        free(gone);
        return BTO_EINTERNAL;
      }
      i++;
    }
    w->c = m;
    free(nidx);
    free(hit);
    free(hitw);
    free(gone);
  }
  return BTO_OK;
}

/* Leaf text of the marked last-level blocks and the per-block symbol counts
 * used by rank and select (counted directly from T). */
static int finalize(bto_tree* t, const uint8_t* T) {
  for (uint32_t l = 0; l + 1 < t->L; l++) link_children(t, l);
  olvl* z = &t->lv[t->L - 1];
  t->leafpos = (uint64_t*)calloc(z->c ? z->c : 1, sizeof(uint64_t));
  uint64_t tot = 0;
  for (uint64_t k = 0; k < z->c; k++)
    if (z->mark[k]) tot += z->len[k];
  t->leaftext = (uint8_t*)malloc(tot ? tot : 1);
  if (!t->leafpos || !t->leaftext) return BTO_ENOMEM;
  t->leafn = 0;
  for (uint64_t k = 0; k < z->c; k++) {
    if (!z->mark[k]) continue;
    t->leafpos[k] = t->leafn;
    memcpy(t->leaftext + t->leafn, T + z->st[k], z->len[k]);
    t->leafn += z->len[k];
  }

  for (int i = 0; i < 256; i++) t->sym[i] = -1;
  t->nsym = 0;
  for (uint64_t i = 0; i < t->n; i++)
    if (t->sym[T[i]] < 0) t->sym[T[i]] = 0;
  for (int i = 0; i < 256; i++)
    if (t->sym[i] == 0) t->sym[i] = (int)t->nsym++;
  uint32_t S = t->nsym;
  for (uint32_t l = 0; l < t->L; l++) {
    olvl* v = &t->lv[l];
    v->cnt = (uint64_t*)calloc((v->c ? v->c : 1) * S, sizeof(uint64_t));
    v->pc = (uint64_t*)calloc((v->c ? v->c : 1) * S, sizeof(uint64_t));
    if (!v->cnt || !v->pc) return BTO_ENOMEM;
    for (uint64_t k = 0; k < v->c; k++) {
      for (uint64_t i = v->st[k]; i < v->st[k] + v->len[k]; i++) v->cnt[k * S + t->sym[T[i]]]++;
      if (!v->mark[k]) {
        uint64_t s = v->st[v->ptr[k]];
        for (uint64_t i = s; i < s + v->off[k]; i++) v->pc[k * S + t->sym[T[i]]]++;
      }
    }
  }
  olvl* r = &t->lv[0];
  t->pre = (uint64_t*)calloc((r->c + 1) * S, sizeof(uint64_t));
  if (!t->pre) return BTO_ENOMEM;
  for (uint64_t k = 0; k < r->c; k++)
    for (uint32_t s = 0; s < S; s++) t->pre[(k + 1) * S + s] = t->pre[k * S + s] + r->cnt[k * S + s];
  return BTO_OK;
}

int bto_build(const uint8_t* T, uint64_t n, uint32_t tau, uint32_t leaf, const bto_opts* o,
              bto_tree** out) {
  if (!out) return BTO_EINVAL;
  *out = NULL;
  if (!T || n == 0 || tau < 2 || leaf == 0) return BTO_EINVAL;
  uint64_t q = (o && o->modulus) ? o->modulus : MERSENNE61;
  if (q < 300 || q >= (1ull << 62)) return BTO_EINVAL;
  uint64_t B = bto_base(o ? o->seed : 0, q);

  bto_tree* t = (bto_tree*)calloc(1, sizeof(bto_tree));
  if (!t) return BTO_ENOMEM;
  t->n = n;
  t->tau = tau;
  t->leaf = leaf;
  t->prune = o ? o->prune : 0;
  uint64_t* b = NULL;
  int rc = plan_sizes(n, tau, leaf, o, &b, &t->L);
  if (rc != BTO_OK) {
    free(t);
    return rc;
  }
  t->lv = (olvl*)calloc(t->L, sizeof(olvl));
  if (!t->lv) {
    free(b);
    free(t);
    return BTO_ENOMEM;
  }
  for (uint32_t l = 0; l < t->L; l++) t->lv[l].b = b[l];
  free(b);

  /* Level 1: consecutive blocks of length b_1; the last may be short. */
  olvl* r = &t->lv[0];
  uint64_t s = (n + r->b - 1) / r->b;
  rc = lvl_alloc(r, s);
  for (uint64_t k = 0; k < s && rc == BTO_OK; k++) {
    r->st[k] = k * r->b;
    r->len[k] = (k + 1) * r->b <= n ? r->b : n - k * r->b;
  }
  for (uint32_t l = 0; l < t->L && rc == BTO_OK; l++) {
    rc = build_level(t, T, l, B, q);
    if (rc == BTO_OK && l + 1 < t->L) rc = make_children(t, l);
  }
  if (rc == BTO_OK && t->prune) rc = prune_tree(t);
  if (rc == BTO_OK) rc = finalize(t, T);
  if (rc != BTO_OK) {
    bto_free(t);
    return rc;
  }
  *out = t;
  return BTO_OK;
}

uint32_t bto_levels(const bto_tree* t) { return t ? t->L : 0; }

int bto_stats(const bto_tree* t, uint64_t* out, uint64_t cap) {
  if (!t || !out || cap < (uint64_t)t->L * BTO_ST_FIELDS) return BTO_EINVAL;
  memcpy(out, t->stats, (uint64_t)t->L * BTO_ST_FIELDS * sizeof(uint64_t));
  return BTO_OK;
}

/* ------------------------------------------------------------------ */
/* Canonical serialization                                            */
/* ------------------------------------------------------------------ */

typedef struct {
  uint8_t* buf;
  uint64_t cap, len;
} wbuf;

static void put64(wbuf* w, uint64_t x) {
  if (w->buf && w->len + 8 <= w->cap) memcpy(w->buf + w->len, &x, 8);
  w->len += 8;
}

/*
 * Layout (all u64 little-endian):
 *   magic "BLKTREE1", n, tau, leaf_len, L, prune
 *   per level: nblocks, b, ceil(nblocks/64) words of marks (LSB first),
 *              nptr, then (ptr, off) of every unmarked block in order
 *   leaf_bytes, leaf text (marked last-level blocks in order), zero pad to 8.
 */
int bto_export(const bto_tree* t, uint8_t* buf, uint64_t cap, uint64_t* len) {
  if (!t || !len) return BTO_EINVAL;
  wbuf w = {buf, cap, 0};
  put64(&w, 0x31454552544B4C42ull);
  put64(&w, t->n);
  put64(&w, t->tau);
  put64(&w, t->leaf);
  put64(&w, t->L);
  put64(&w, (uint64_t)t->prune);
  for (uint32_t l = 0; l < t->L; l++) {
    const olvl* v = &t->lv[l];
    put64(&w, v->c);
    put64(&w, v->b);
    for (uint64_t k0 = 0; k0 < v->c; k0 += 64) {
      uint64_t word = 0;
      for (uint64_t k = k0; k < v->c && k < k0 + 64; k++)
        if (v->mark[k]) word |= 1ull << (k - k0);
      put64(&w, word);
    }
    uint64_t nptr = 0;
    for (uint64_t k = 0; k < v->c; k++) nptr += !v->mark[k];
    put64(&w, nptr);
    for (uint64_t k = 0; k < v->c; k++) {
      if (v->mark[k]) continue;
      put64(&w, v->ptr[k]);
      put64(&w, v->off[k]);
    }
  }
  put64(&w, t->leafn);
  for (uint64_t i = 0; i < t->leafn; i += 8) {
    uint64_t word = 0;
    for (uint64_t j = 0; j < 8 && i + j < t->leafn; j++) word |= (uint64_t)t->leaftext[i + j] << (8 * j);
    put64(&w, word);
  }
  *len = w.len;
  return (buf && w.len > cap) ? BTO_ERANGE : BTO_OK;
}

/* ------------------------------------------------------------------ */
/* Queries (section 1): access, rank, select on the tree              */
/* ------------------------------------------------------------------ */

int bto_access(const bto_tree* t, uint64_t i, uint8_t* out) {
  if (!t || !out) return BTO_EINVAL;
  if (i >= t->n) return BTO_ERANGE;
  uint32_t l = 0;
  uint64_t k = i / t->lv[0].b, x = i;
  for (uint64_t step = 0; step < 4ull * t->L + 4; step++) {
    const olvl* v = &t->lv[l];
    if (v->mark[k]) {
      if (l + 1 == t->L) {
        *out = t->leaftext[t->leafpos[k] + (x - v->st[k])];
        return BTO_OK;
      }
      k = v->fc[k] + (x - v->st[k]) / t->lv[l + 1].b;
      l++;
    } else {
      uint64_t P = v->ptr[k];
      x = v->st[P] + v->off[k] + (x - v->st[k]);
      k = x < v->st[P] + v->len[P] ? P : P + 1;
    }
  }
  return BTO_EINTERNAL;
}

/* Count of symbol s in T[st[k], st[k]+o) for block k of level l. */
static int rank_in(const bto_tree* t, uint32_t l, uint64_t k, uint32_t s, uint64_t o, uint64_t* out) {
  const uint32_t S = t->nsym;
  int64_t acc = 0;
  for (uint64_t step = 0; step < 4ull * t->L + 4; step++) {
    const olvl* v = &t->lv[l];
    if (o == 0) {
      *out = (uint64_t)acc;
      return BTO_OK;
    }
    if (o == v->len[k]) {
      *out = (uint64_t)(acc + (int64_t)v->cnt[k * S + s]);
      return BTO_OK;
    }
    if (v->mark[k]) {
      if (l + 1 == t->L) {
        const uint8_t* p = t->leaftext + t->leafpos[k];
        for (uint64_t i = 0; i < o; i++) acc += t->sym[p[i]] == (int)s;
        *out = (uint64_t)acc;
        return BTO_OK;
      }
      const olvl* w = &t->lv[l + 1];
      uint64_t j = o / w->b, f = v->fc[k];
      for (uint64_t i = 0; i < j; i++) acc += (int64_t)w->cnt[(f + i) * S + s];
      o -= j * w->b;
      k = f + j;
      l++;
    } else {
      uint64_t P = v->ptr[k], x = v->off[k] + o;
      acc -= (int64_t)v->pc[k * S + s];
      if (x <= v->len[P]) {
        k = P;
        o = x;
      } else {
        acc += (int64_t)v->cnt[P * S + s];
        k = P + 1;
        o = x - v->len[P];
      }
    }
  }
  return BTO_EINTERNAL;
}

int bto_rank(const bto_tree* t, uint8_t c, uint64_t i, uint64_t* out) {
  if (!t || !out) return BTO_EINVAL;
  if (i > t->n) return BTO_ERANGE;
  if (t->sym[c] < 0) {
    *out = 0;
    return BTO_OK;
  }
  const uint32_t S = t->nsym, s = (uint32_t)t->sym[c];
  const olvl* r = &t->lv[0];
  if (i == t->n) {
    *out = t->pre[r->c * S + s];
    return BTO_OK;
  }
  uint64_t k = i / r->b, in = 0;
  int rc = rank_in(t, 0, k, s, i - r->st[k], &in);
  *out = t->pre[k * S + s] + in;
  return rc;
}

int bto_select(const bto_tree* t, uint8_t c, uint64_t j, uint64_t* out) {
  if (!t || !out) return BTO_EINVAL;
  if (t->sym[c] < 0 || j == 0) return BTO_ERANGE;
  const uint32_t S = t->nsym, s = (uint32_t)t->sym[c];
  const olvl* r = &t->lv[0];
  if (j > t->pre[r->c * S + s]) return BTO_ERANGE;
  uint64_t k = 0;
  while (t->pre[(k + 1) * S + s] < j) k++;
  j -= t->pre[k * S + s];
  int64_t res = (int64_t)r->st[k];
  uint32_t l = 0;
  for (uint64_t step = 0; step < 4ull * t->L + 4; step++) {
    const olvl* v = &t->lv[l];
    if (v->mark[k]) {
      if (l + 1 == t->L) {
        const uint8_t* p = t->leaftext + t->leafpos[k];
        for (uint64_t i = 0; i < v->len[k]; i++) {
          if (t->sym[p[i]] == (int)s && --j == 0) {
            *out = (uint64_t)(res + (int64_t)i);
            return BTO_OK;
          }
        }
        return BTO_EINTERNAL;
      }
      const olvl* w = &t->lv[l + 1];
      uint64_t f = v->fc[k], i = 0;
      while (w->cnt[(f + i) * S + s] < j) {
        j -= w->cnt[(f + i) * S + s];
        i++;
      }
      res += (int64_t)(i * w->b);
      k = f + i;
      l++;
    } else {
      uint64_t P = v->ptr[k], jj = j + v->pc[k * S + s];
      if (jj <= v->cnt[P * S + s]) {
        res -= (int64_t)v->off[k];
        k = P;
        j = jj;
      } else {
        res += (int64_t)(v->len[P] - v->off[k]);
        j = jj - v->cnt[P * S + s];
        k = P + 1;
      }
    }
  }
  return BTO_EINTERNAL;
}
