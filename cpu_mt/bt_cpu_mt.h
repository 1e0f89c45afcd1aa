/*
 * bt_cpu_mt.h -- a straightforward multithreaded CPU block-tree builder
 * (OpenMP), the multicore CPU baseline reported beside the GPU build.
 *
 * btmt_build builds the block tree of T[0, n) (section 3, with the per-level
 * Karp-Rabin pass of section 3.1; level sizes b_L = leaf, b_l = tau b_{l+1},
 * root arity tau) and returns its canonical serialization (the byte layout of
 * bt_export in include/bt.h) in a buffer the caller releases with btmt_free.
 * threads <= 0 uses the OpenMP default (every host core).  seed selects the
 * Karp-Rabin base; the tree does not depend on it.
 *
 * Errors: BTMT_EINVAL for n = 0, tau < 2, leaf = 0 or a null pointer;
 * BTMT_ENOMEM when an allocation fails.  The text stays the caller's.
 */
#ifndef BT_CPU_MT_H
#define BT_CPU_MT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { BTMT_OK = 0, BTMT_EINVAL = 1, BTMT_ENOMEM = 3 };

int btmt_build(const uint8_t* text, uint64_t n, uint32_t tau, uint32_t leaf_len, int prune, uint64_t seed,
               int threads, uint8_t** blob, uint64_t* blob_len);
void btmt_free(uint8_t* blob);
int btmt_threads(void);

#ifdef __cplusplus
}
#endif

#endif
