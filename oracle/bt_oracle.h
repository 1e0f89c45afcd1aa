/*
 * bt_oracle.h -- plain, single-threaded CPU block-tree builder.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant with the CUDA library, and the CUDA library never
 * calls it.
 *
 * What it computes (paper section 3, "Block Trees", and section 3.1):
 *  - block sizes b_1 > b_2 > ... > b_L, b_L = leaf_len, b_l = tau * b_{l+1};
 *  - level 1: consecutive blocks of length b_1 (the last one may be short);
 *  - a pair of consecutive blocks (consecutive in T) is "leftmost" when the
 *    leftmost occurrence of its string in T starts at the pair's own start;
 *    both blocks of a leftmost pair are marked; a block in no pair is marked;
 *  - marked blocks of a non-last level have children on the next level;
 *    unmarked blocks store (ptr, off): the level block holding the leftmost
 *    occurrence of their string, and the offset into it;
 *  - the optional pruning post-pass of section 3.1 ("Optional Pruning");
 *  - access / rank / select of section 1 on the finished tree.
 * Leftmost occurrences are found as in section 3.1: Karp-Rabin fingerprints
 * (section 2) of all keys go into a hash table, a rolling scan over every
 * window of T probes it, and every fingerprint match is verified byte by byte
 * before it is accepted, so the result is exact for any base and modulus.
 *
 * Positions are 0-based.  rank(c, i) counts c in T[0, i); select(c, j)
 * returns the 0-based position of the j-th c (j >= 1).
 */
#ifndef BT_ORACLE_H
#define BT_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { BTO_OK = 0, BTO_EINVAL = 1, BTO_ERANGE = 2, BTO_ENOMEM = 3, BTO_EINTERNAL = 4 };

typedef struct bto_tree bto_tree;

typedef struct {
  int prune;                   /* 1: apply the pruning post-pass                  */
  uint32_t root_arity;         /* 0: smallest height with leaf*tau^(h+1) >= n     */
  uint64_t seed;               /* selects the fingerprint base                    */
  uint64_t modulus;            /* 0: 2^61-1; else any q in [300, 2^62)            */
  const uint64_t* level_sizes; /* explicit block size per level, or NULL          */
  uint32_t nlevels;            /* entries in level_sizes                          */
} bto_opts;

/* Per-level statistics of the unpruned construction (7 u64 per level). */
enum { BTO_ST_NBLOCKS = 0, BTO_ST_B, BTO_ST_COV, BTO_ST_NMARKED, BTO_ST_NPAIRS,
       BTO_ST_VERIFY_BYTES, BTO_ST_COLLISIONS, BTO_ST_FIELDS };

int bto_build(const uint8_t* text, uint64_t n, uint32_t tau, uint32_t leaf_len,
              const bto_opts* opts, bto_tree** out);
int bto_export(const bto_tree* t, uint8_t* buf, uint64_t cap, uint64_t* len);
int bto_access(const bto_tree* t, uint64_t i, uint8_t* out);
int bto_rank(const bto_tree* t, uint8_t c, uint64_t i, uint64_t* out);
int bto_select(const bto_tree* t, uint8_t c, uint64_t j, uint64_t* out);
uint32_t bto_levels(const bto_tree* t);
int bto_stats(const bto_tree* t, uint64_t* out, uint64_t cap);
void bto_free(bto_tree* t);

/* Fingerprint base for a seed and modulus (0 = 2^61-1). */
uint64_t bto_base(uint64_t seed, uint64_t modulus);
/* phi(s, s+len) = sum_i (T[i]+1) * base^(s+len-1-i) mod q, by Horner. */
uint64_t bto_fingerprint(const uint8_t* text, uint64_t s, uint64_t len,
                         uint64_t base, uint64_t modulus);

#ifdef __cplusplus
}
#endif
#endif
