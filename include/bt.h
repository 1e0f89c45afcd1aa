/*
 * bt.h -- C ABI of the GB300 block-tree library (libbt.so).
 *
 * A block tree (Belazzougui et al.; the paper's section 3, "Block Trees") is a
 * compressed index of a text T[0, n) that answers access, rank and select
 * (the paper's section 1).  bt_build runs the per-level Karp-Rabin pass of
 * sections 3.1 and 4 on the GPU: fingerprints of every block and of every
 * pair of consecutive blocks, a scan of every window of the level against
 * them to find leftmost occurrences, byte verification of every accepted
 * fingerprint match, marking, back-pointers with offsets, the optional
 * pruning pass, and the split of surviving blocks into the next level.
 *
 * Conventions for every entry point:
 *  - Positions are 0-based.  The paper's access(i), rank_c(i) (inclusive,
 *    1-based) and select_c(j) (1-based) map to bt_access(i-1),
 *    bt_rank(c, i) and bt_select(c, j) + 1.
 *  - Return value: 0 (BT_OK) or a positive bt_status code; outputs are
 *    written only on BT_OK.  bt_strerror names a code.
 *  - Pointers named d_* are device pointers (cudaMalloc'd memory of the
 *    current device); `text` may be a host or a device pointer (detected with
 *    cudaPointerGetAttributes).  The caller keeps ownership of every buffer
 *    it passes; the library owns a bt_tree until bt_free.
 *  - `stream` is a cudaStream_t passed as void*; NULL means the per-thread
 *    default stream.  Entry points that return host values synchronize it.
 *  - A built tree is immutable: queries on one tree may run concurrently
 *    from several host threads.  bt_free must not race with queries.
 *  - Limits: 1 <= n < 2^32, 2 <= tau <= 64, leaf_len >= 1.
 *  - There is no CPU fallback: without a usable CUDA device every entry
 *    point that computes returns BT_ECUDA.
 */
#ifndef BT_H
#define BT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  BT_OK = 0,
  BT_EINVAL = 1,    /* bad argument: n = 0, tau < 2, leaf_len = 0, more distinct
                       byte values than sigma, bad opts or level sizes       */
  BT_ERANGE = 2,    /* query out of range; export buffer too small            */
  BT_ENOMEM = 3,    /* device or host allocation failed                       */
  BT_ECUDA = 4,     /* a CUDA call failed (no device, launch error, ...)      */
  BT_ETIMEOUT = 5,  /* reserved: no entry point returns it today (the library's
                       kernels wait on nothing that another launch, stream or
                       device sets, so no device-side wait can run out)       */
  BT_EINTERNAL = 6  /* a device-side invariant check failed                   */
} bt_status;

typedef struct bt_tree bt_tree;

/* Build options.  Initialise with bt_opts_default. */
typedef struct {
  int prune;                   /* 1 (default): run the pruning post-pass of
                                  section 3.1 ("Optional Pruning")            */
  uint32_t root_arity;         /* 0 (default): the height h is the smallest
                                  with tau*leaf_len*tau^h >= n; otherwise the
                                  smallest with root_arity*leaf_len*tau^h >= n */
  uint64_t seed;               /* selects the Karp-Rabin base B (section 2)   */
  uint64_t modulus;            /* 0 (default): q = 2^61-1.  Test hook: any q in
                                  [300, 2^32) makes fingerprint collisions
                                  frequent; the result must not change.       */
  const uint64_t* level_sizes; /* host array of explicit block sizes, level 1
                                  first, each >= 2x and a multiple of the
                                  next; NULL (default) derives them.          */
  uint32_t nlevels;            /* entries of level_sizes                      */
  uint64_t max_rounds;         /* pruning: parallel frontier rounds before a
                                  single-thread right-to-left finish of the
                                  rest; 0 = default 4096.                     */
  uint32_t flags;              /* BT_FLAG_* (0 by default)                    */
  uint32_t batch_ctas;         /* bt_build_batch: CTAs of the batched kernel's
                                  launch; 0 (default) = the autotuned shape
                                  over every SM.  A smaller grid leaves SMs to
                                  other work, e.g. a second batch on another
                                  host thread.                                 */
  uint32_t partitions;         /* with BT_FLAG_SORT_SCAN: the number K of parts
                                  of the domain decomposition (section 4.2);
                                  0 or 1 (default): one part.  Ignored by the
                                  other passes.                                */
} bt_opts;

/* flags: BT_FLAG_DENSE_SCAN probes the table at every window position instead
 * of the anchored scan (a diagnostic; both give the same tree).
 * BT_FLAG_TINY_QUEUE caps the anchored scan's queue of proposed windows at 64
 * entries, so that nearly every level takes the overflow path, a second scan
 * that tests the windows in place (a test hook; the same tree again). */
/* BT_FLAG_GRAM_LIST builds the selected-gram list (the gram positions and
 * hashes the anchored scan shares between levels) whatever the text length;
 * by default only texts of 8 MiB or more use it (a test hook; same tree). */
/* BT_FLAG_TWO_PHASE tests the proposed windows of every anchored level in two
 * phases: the windows of the gram hits in the first 1/16 of the text, then
 * the rest, against per-gram bounds lowered to the leftmost positions found so
 * far (a window after every such position of the keys on its gram is not
 * proposed).  The same tree.  It pays where the keys on a gram mostly have
 * their leftmost occurrence early (DNA copies with sparse point mutations:
 * about a third fewer windows); where most grams also carry a key first seen
 * late (edits in every copy of a versioned text) few windows are saved and the
 * two extra kernels and the second hit pass cost more, hence off by default. */
/* BT_FLAG_BATCH_WORKERS makes bt_build_batch build every document with
 * bt_build_ex on host worker threads instead of the persistent batched kernel
 * (the comparison arm of the batched build; the same trees). */
/* BT_FLAG_LEAF_COUNTS: space-efficient rank/select support (the paper's
 * section 6 names the auxiliary space of rank and select as future work).
 * The last level, which holds most blocks, stores no per-block symbol
 * counters: a query that needs one counts it in the leaf text (the block's
 * own text when marked, the at most two marked blocks its pointer copies
 * from otherwise; at most 2 leaf_len bytes).  Same tree and same answers,
 * fewer device bytes, slower rank and select at the last level.  Single-text
 * builds only (bt_build_batch ignores it). */
/* BT_FLAG_ANCHOR_ALL (a test hook of bt_build_batch): the batched kernel
 * scans every level with blocks of 32 bytes or more by anchors (by default
 * only levels with blocks of 1024 bytes or more), so that its anchored scan
 * and the 8-byte prefix filter of blocks without an anchor run on short
 * blocks too.  The same trees. */
/* BT_FLAG_SORT_SCAN: the sort-based level pass of the paper's section 4.1
 * instead of the table probes: every window of length b (then 2b) inside a
 * run becomes a (fingerprint, position) tuple, the tuples are radix-sorted
 * stably, and each block (pair) takes the first position of its
 * fingerprint's group as its leftmost candidate.  Verification and the rest of
 * the level are shared with the default path; the same tree.  It moves about
 * 24 bytes per covered position and sort pass (slower; a second algorithm to
 * compare with).  Single-text builds only; c_l * b_l < 2^32 per level.
 * With opts.partitions = K > 1 the windows are taken in K parts of
 * consecutive windows (the domain decomposition of section 4.2): a part keeps
 * only its windows whose fingerprint is a key's, sorts them and keeps the
 * first of each fingerprint; the kept tuples of all parts (at most K per key)
 * are sorted once more and give the same minima.  Working memory per level:
 * about 44 bytes per window of a part plus 12 bytes per kept tuple (at most
 * one per key and part), instead of about 24 bytes per window; two host
 * synchronisations per part.  The same tree; n < 2^32. */
enum { BT_FLAG_DENSE_SCAN = 1, BT_FLAG_TINY_QUEUE = 2, BT_FLAG_GRAM_LIST = 4, BT_FLAG_TWO_PHASE = 8,
       BT_FLAG_BATCH_WORKERS = 16, BT_FLAG_LEAF_COUNTS = 32, BT_FLAG_SORT_SCAN = 64,
       BT_FLAG_ANCHOR_ALL = 128 };

void bt_opts_default(bt_opts* opts);

/*
 * Build the block tree of text[0, n) (section 3; per-level pass of sections
 * 3.1 and 4).  sigma is the alphabet size: the text may hold at most sigma
 * distinct byte values (any values; they need not be < sigma).  tau is the
 * arity of inner nodes, leaf_len the block length of the last level.
 * Equivalent to bt_build_ex with bt_opts_default and a NULL stream.
 * On success *out holds a new tree; on failure *out is NULL.
 */
int bt_build(const uint8_t* text, uint64_t n, uint32_t sigma, uint32_t tau,
             uint32_t leaf_len, bt_tree** out);

int bt_build_ex(const uint8_t* text, uint64_t n, uint32_t sigma, uint32_t tau,
                uint32_t leaf_len, const bt_opts* opts, void* stream, bt_tree** out);

/*
 * Build the trees of ndocs independent texts in one call.  Document d is
 * texts[d][0, ns[d]) with sigmas[d], taus[d], leaf_lens[d]; every document
 * uses *opts (NULL: defaults).  Texts may be host or device pointers.
 *
 * Documents of at most 2^30 bytes and 40 levels are built by one persistent
 * kernel launch per size class (the paper's section 3 levels and section 3.1
 * pass, per document): each CTA takes the next document from a device work
 * queue (longest first) and builds its whole tree -- alphabet, prefix
 * fingerprints, every level's scan, verification, marks, pointers and split,
 * pruning and counters -- level by level with barriers of the CTA, without
 * any host round trip.  The trees of one call share one device allocation,
 * released when the last of them is freed.  Larger documents, and every
 * document when opts->flags has BT_FLAG_BATCH_WORKERS, are built with
 * bt_build_ex on `nworkers` host threads (0: 8), one CUDA stream each.
 *
 * Each tree is identical to the one bt_build_ex makes for that document
 * alone.  On success outs[d] holds document d's tree; if any build fails,
 * every tree of the batch is freed, outs[] is set to NULL and the first
 * failure's status is returned (BT_EINVAL for bad arguments, including a
 * document with more distinct bytes than its sigma; BT_ENOMEM when device
 * memory or a host worker thread is not available).
 */
int bt_build_batch(const uint8_t* const* texts, const uint64_t* ns, const uint32_t* sigmas,
                   const uint32_t* taus, const uint32_t* leaf_lens, uint64_t ndocs,
                   const bt_opts* opts, uint32_t nworkers, bt_tree** outs);

/* Measurement hooks of the batched build (not part of the paper's method).
 * bt_batch_report: what the last bt_build_batch call of the process did, 13
 * u64: documents built by the batched kernel, documents built by host
 * workers, kernel launches, documents built a second time because the output
 * pool ran out, threads per CTA, CTAs per SM, output pool bytes, CTA scratch
 * bytes, the largest grid, the scan's window run (consecutive positions per
 * lane), the autotuner's trial builds in this call, the microseconds the
 * host spent issuing the texts' copies to the device (the copies themselves
 * when the texts are in pageable memory) and the microseconds of device time
 * of the batched kernel's launches.  The launch shape (threads, CTAs per SM,
 * run) of a batch of 1024 or more documents is chosen the first time a batch
 * of its size class is built, and cached for the process: each candidate
 * builds a seeded sample of the batch, and the one whose measured cycles per
 * byte and level give the shortest simulated batch wins.  bt_batch_cycles: for a tree from the batched
 * kernel, the SM clock cycles its CTA spent per phase (6 u64: set-up,
 * tables, window scan, verification/marks/pointers/split, pruning, output
 * and counters); zeros for other trees.  BT_EINVAL for null pointers or cap
 * too small. */
int bt_batch_report(uint64_t* out, uint32_t cap);
int bt_batch_cycles(const bt_tree* t, uint64_t* out, uint32_t cap);

/* access(i) = T[i], 0 <= i < n (section 1).  BT_ERANGE if i >= n. */
int bt_access(const bt_tree* t, uint64_t i, uint8_t* out);

/* rank_c(i) = number of j < i with T[j] = c, 0 <= i <= n (section 1).
 * A byte absent from T has rank 0.  BT_ERANGE if i > n. */
int bt_rank(const bt_tree* t, uint8_t c, uint64_t i, uint64_t* out);

/* select_c(j) = 0-based position of the j-th occurrence of c, j >= 1
 * (section 1).  BT_ERANGE if j = 0 or j > rank_c(n). */
int bt_select(const bt_tree* t, uint8_t c, uint64_t j, uint64_t* out);

/* Batched queries on device arrays, asynchronous on `stream`.
 *   kind BT_Q_ACCESS: d_args[q] = i;                 d_out[q] = T[i]
 *   kind BT_Q_RANK:   d_args[2q] = c, d_args[2q+1] = i; d_out[q] = rank_c(i)
 *   kind BT_Q_SELECT: d_args[2q] = c, d_args[2q+1] = j; d_out[q] = select_c(j)
 * A query out of range writes UINT64_MAX to d_out[q].  Returns BT_EINVAL for a
 * bad kind, BT_ECUDA if the launch fails. */
enum { BT_Q_ACCESS = 0, BT_Q_RANK = 1, BT_Q_SELECT = 2 };
int bt_query_batch(const bt_tree* t, int kind, const uint64_t* d_args, uint64_t m,
                   uint64_t* d_out, void* stream);

/*
 * Canonical serialization of the tree (all u64, little-endian):
 *   "BLKTREE1", n, tau, leaf_len, L, prune;
 *   per level: nblocks, b, ceil(nblocks/64) words of marks (bit k of word
 *   k/64 = block k is marked), nptr, then (ptr, off) of every unmarked block
 *   in block order;
 *   leaf_bytes, the text of the marked last-level blocks in order, zero
 *   padded to a multiple of 8.
 * With buf == NULL (or cap too small) *len receives the size needed; a too
 * small buffer returns BT_ERANGE.
 */
int bt_export(const bt_tree* t, uint8_t* buf, uint64_t cap, uint64_t* len);

/* Device memory held by a built tree, in bytes (levels, counters, leaf text). */
uint64_t bt_device_bytes(const bt_tree* t);

/* Number of levels of a built tree. */
uint32_t bt_levels(const bt_tree* t);

/* Per-level statistics of the construction, BT_ST_FIELDS u64 per level:
 * blocks, block size, covered bytes (sum of block lengths), marked blocks,
 * pairs, bytes read by verification, fingerprint collisions found by
 * verification, blocks after pruning, windows the anchored scan proposed,
 * proposed windows whose fingerprint belongs to a key.  cap is in u64 units. */
enum { BT_ST_NBLOCKS = 0, BT_ST_B, BT_ST_COV, BT_ST_NMARKED, BT_ST_NPAIRS,
       BT_ST_VERIFY_BYTES, BT_ST_COLLISIONS, BT_ST_FINAL_BLOCKS, BT_ST_CANDIDATES,
       BT_ST_HITS, BT_ST_FIELDS };
int bt_stats(const bt_tree* t, uint64_t* out, uint64_t cap);

/*
 * Karp-Rabin prefix fingerprints (section 2; the data-parallel form of
 * section 4.1): d_out[j] = H(j*stride) for j = 0 .. n/stride, where
 * H(0) = 0 and H(p+1) = H(p)*B + T[p] + 1 mod q, with the base B that
 * bt_build uses for `seed` and q = 2^61-1 (modulus 0) or the given test
 * modulus.  d_text and d_out are device pointers; d_out holds n/stride + 1
 * entries.  stride must be 32.  Asynchronous on `stream`.
 */
int bt_prefix_fingerprints(const uint8_t* d_text, uint64_t n, uint64_t seed, uint64_t modulus,
                           uint32_t stride, uint64_t* d_out, void* stream);

/*
 * bt_prefix_fingerprints without allocating device memory.  The paper has no
 * counterpart; this entry point exists for callers that cannot allocate.
 * Examples: a host runtime that hands all device memory to its own allocator
 * up front and forbids libraries it loads to call cudaMalloc, or code on a
 * latency-critical path that cannot risk an allocation's implicit
 * synchronisation or its failure.
 *
 * Same arguments, results and stream semantics as bt_prefix_fingerprints.
 * The caller still provides d_text and d_out.  The scratch (power tables and
 * per-CTA aggregates) is a fixed 528 KiB array in device memory, which every
 * GPU that loads the library holds until the process exits.  The entry point
 * calls no cudaMalloc, cudaFree or allocating library routine.
 *  - n may be at most 2^31 (2 GiB); larger texts return BT_ERANGE before any
 *    other check and before any work is queued.
 *  - The first call on a device looks up the array's device address (with
 *    that device current) and caches it; make that first call before any
 *    stream capture.  The cache is per device ordinal and is not refreshed
 *    when the device's primary context is reset (cudaDeviceReset); do not
 *    call this entry point again in a process after such a reset.
 *  - Every call shares the one array: calls whose work overlaps on the GPU
 *    (for example on two streams) race and give wrong results; serialise
 *    them.  No scratch entry needs to start at zero: each call writes every
 *    entry it reads before reading it.
 */
int bt_prefix_fingerprints_noalloc(const uint8_t* d_text, uint64_t n, uint64_t seed,
                                   uint64_t modulus, uint32_t stride, uint64_t* d_out,
                                   void* stream);

/* The base B selected by seed for modulus (0 = 2^61-1). */
uint64_t bt_fingerprint_base(uint64_t seed, uint64_t modulus);

void bt_free(bt_tree* t);

const char* bt_strerror(int status);

/*
 * Measurement hooks (not part of the paper's method).  When enabled, the
 * library records a pair of CUDA events on the launching stream around the
 * window-scan, prefix-fingerprint, verification and counter kernels of every
 * build.  bt_profile_read aggregates, per kernel name: launches, total
 * milliseconds between the events, and the algorithmic bytes those launches
 * process (the covered bytes of the level for the window scan, n for the
 * prefix fingerprints, the compared bytes for verification).  It waits for
 * the recorded events.  Profiling state is process-wide; reads and resets
 * must not race with builds that record.
 */
typedef struct {
  char name[32];
  uint64_t launches;
  double ms;
  uint64_t bytes;
} bt_profile_entry;
void bt_profile_enable(int on);
void bt_profile_reset(void);
int bt_profile_read(bt_profile_entry* out, uint32_t cap, uint32_t* count);

/* Test hooks for allocation failures (not part of the paper's method).
 * bt_test_alloc_limit(bytes): from now on, any single device allocation a
 * build makes (text copy, prefix fingerprints, level scratch, the batched
 * build's buffers and output pool) that is larger than `bytes` fails as if
 * the device were out of memory, so the build returns BT_ENOMEM; 0 removes
 * the limit.  Process-wide; not for concurrent use with real builds.
 * bt_device_pool_used: bytes currently allocated from the current device's
 * stream-ordered memory pool (the library's builds allocate there), for
 * checking that a failed build gave everything back.
 * bt_device_pool_peak: the high-water mark of those bytes since the last
 * reset; reset != 0 then sets the mark to the bytes in use now (a working
 * memory measurement: reset, build, read). */
void bt_test_alloc_limit(uint64_t bytes);
int bt_device_pool_used(uint64_t* out);
int bt_device_pool_peak(uint64_t* out, int reset);

/* Number of kernels this library has launched in the process so far. */
uint64_t bt_launch_count(void);

/* Integer-pipe microbenchmark for the roofline of the fingerprint arithmetic
 * (section 2: one 61-bit modular multiply per window and length).  Launches,
 * on `stream` (NULL: the per-thread default stream), `blocks` CTAs of 256
 * threads that each run 8 independent chains of `iters` multiplies mod
 * 2^61-1 by the base of `seed`, and store one word per thread in d_out
 * (device memory, blocks * 256 u64, owned by the caller).  *mulmods receives
 * the number of multiplies launched; the caller times the launch (CUDA events
 * on the same stream).  BT_EINVAL for null pointers or zero sizes, BT_ECUDA
 * when the launch fails.  Returns without waiting. */
int bt_mulmod_bench(uint32_t blocks, uint32_t iters, uint64_t seed, uint64_t* d_out, void* stream,
                    uint64_t* mulmods);

#ifdef __cplusplus
}
#endif
#endif
