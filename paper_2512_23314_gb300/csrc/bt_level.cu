// bt_level.cu -- one level of block-tree construction on the GPU.
//
// Section 3 defines the level: blocks B_k (consecutive in T), pairs
// B_k B_{k+1} of blocks that are consecutive in T, both blocks of a pair
// marked when the pair's string occurs leftmost at the pair's own start, a
// block in no pair kept marked, and every unmarked block turned into a
// pointer (ptr, off) to the leftmost occurrence of its string.  Section 3.1
// finds leftmost occurrences with Karp-Rabin fingerprints in a hash table and
// a scan of the level, verifying each accepted match once; section 4.2 lets
// every processing element filter locally before a global minimum.  On the
// GPU the global minimum is an atomicMin per hash-table slot:
//
//   1. k_block_fp     fingerprint of every block (prefix form of section 4.1)
//                     and insertion of the full-length ones into the block
//                     table (one slot per distinct fingerprint);
//   2. k_pair_insert  one pair-table slot per distinct (slot_k, slot_k+1);
//   3. k_scan         every window of length b that lies inside a run of
//                     consecutive blocks: rolling fingerprint, table probe,
//                     atomicMin of the position into the slot; at a hit the
//                     fingerprint of the next b bytes finds the pair slot.  The
//                     short last block of T (length r < b) and the pair that
//                     ends in it are matched by a second rolling hash;
//   4. verification   every slot minimum that differs from the key's own start
//                     is compared byte by byte (k_verify, warp-cooperative, in
//                     fixed-size pieces); a mismatch is a fingerprint
//                     collision, and the key is resolved exactly by
//                     k_exact_scan (fingerprint filter + byte compare of every
//                     window), so collisions cannot change the result;
//   5. k_mark         marks from the pair results (warp ballot -> bit words),
//                     popcount prefix for rank;
//   6. k_pointers     unmarked blocks -> (ptr, off) by binary search;
//   7. k_children     the tau-way split of marked blocks into the next level.
#include <atomic>
#include <cmath>
#include <chrono>
#include <cstdio>
#include <cstdlib>

#include "bt_internal.cuh"

namespace bt {

namespace {

constexpr uint32_t kTailPair = 0xFFFFFFFEu;  // slotP of the pair ending in the short tail
constexpr uint32_t kScanQ = 64;              // window starts per scan thread
constexpr uint64_t kPiece = 4096;            // bytes per verification piece

struct Job {
  uint64_t a, b, len;   // compare T[a, a+len) with T[b, b+len)
  uint64_t idx;         // key index (block or pair)
};

// Per-level device scalars.
struct LevelDev {
  unsigned long long fp_tail;       // fingerprint of the short tail block
  unsigned long long lo_tail;       // min window position matching fp_tail
  unsigned long long lo_tailpair;   // min position matching the pair ending in the tail
  unsigned int pretail_slot;        // block slot of the block before the tail
  unsigned int npairs;
  unsigned long long njobs;
  unsigned long long nsusp;
  unsigned int anchorless;          // some full-length key has no anchor
  unsigned int tail_anchorless;     // tail key: 1 shorter than a gram, 2 no anchor
  unsigned int tail_gram;           // anchor gram of the tail key (remapped)
  unsigned int tail_a;              // its anchor offset
  unsigned int far_end;             // 1 + the largest far anchor offset of a full-length key
  unsigned long long cands;         // windows proposed by anchors and filters
  unsigned long long hits;          // proposed windows whose fingerprint is a key's
  unsigned int qover;               // some CTA's queue segment overflowed
  unsigned int nfar;                // FarNodes taken
};

struct Geo {
  const uint8_t* T;
  uint64_t n;
  const uint64_t* H;        // prefix fingerprints at every position
  uint64_t B, Bb, Br, Bbr;  // B, B^b, B^r, B^(b+r)
  uint64_t c, b, r;         // blocks, block length, tail length (0: no short tail)
  const uint64_t* st;
};

__device__ __forceinline__ uint64_t blen(const Geo& g, uint64_t k) {
  uint64_t s = g.st[k];
  return g.n - s < g.b ? g.n - s : g.b;
}

// End of the text covered by block k and up to two following blocks that are
// consecutive in T; a window of length <= 2b starting in block k lies inside
// a run iff it ends at or before this position.
__device__ __forceinline__ uint64_t avail_end(const Geo& g, uint64_t k) {
  uint64_t e = g.st[k] + blen(g, k);
  if (k + 1 < g.c && g.st[k + 1] == e) {
    e += blen(g, k + 1);
    if (k + 2 < g.c && g.st[k + 2] == e) e += blen(g, k + 2);
  }
  return e;
}

// One block-table slot, one 32-byte sector: the key (a block fingerprint),
// the leftmost window seen with that fingerprint, and the last start of a
// pair whose first block has this slot.  A probe, its minimum update and the
// pair bound touch the same sector.
struct __align__(32) BSlot {
  unsigned long long key;
  unsigned long long lo;
  unsigned long long maxpst;
  unsigned long long pad;
};
// One pair-table slot: the key (the two block slots) and the leftmost window.
struct __align__(16) PSlot {
  unsigned long long key;
  unsigned long long lo;
};

// Open addressing with linear probing on the slots' keys.
// A plain read comes first: repeated keys (the same block content in many
// versions) find their slot without an atomic on a contended address.
template <class S>
__device__ __forceinline__ uint32_t tbl_insert(S* t, uint64_t mask, uint64_t key) {
  uint64_t h = mix64(key) & mask;
  for (uint64_t it = 0; it <= mask; it++) {
    unsigned long long old = *(volatile unsigned long long*)&t[h].key;
    if (old == kNone) old = atomicCAS(&t[h].key, (unsigned long long)kNone, (unsigned long long)key);
    if (old == kNone || old == key) return (uint32_t)h;
    h = (h + 1) & mask;
  }
  return kNoSlot;
}

template <class S>
__device__ __forceinline__ uint32_t tbl_find(const S* __restrict__ t, uint64_t mask, uint64_t key) {
  uint64_t h = mix64(key) & mask;
  for (uint64_t it = 0; it <= mask; it++) {
    uint64_t k = t[h].key;
    if (k == key) return (uint32_t)h;
    if (k == kNone) return kNoSlot;
    h = (h + 1) & mask;
  }
  return kNoSlot;
}

__device__ __forceinline__ void min_pos(unsigned long long* a, uint64_t p) {
  if (*(volatile unsigned long long*)a > p) atomicMin(a, (unsigned long long)p);
}

// Warp-aggregated slot claim: one atomicAdd per warp.  Every lane of the
// warp must call it (the loops above keep warps uniform).
__device__ __forceinline__ uint64_t warp_claim(unsigned long long* ctr, bool want) {
  const unsigned lane = threadIdx.x & 31;
  const unsigned m = __ballot_sync(0xFFFFFFFFu, want);
  unsigned long long base = 0;
  if (m) {
    const int leader = __ffs(m) - 1;
    if ((int)lane == leader) base = atomicAdd(ctr, (unsigned long long)__popc(m));
    base = __shfl_sync(0xFFFFFFFFu, base, leader);
  }
  return want ? base + __popc(m & ((1u << lane) - 1u)) : kNone;
}

__device__ __forceinline__ uint64_t warp_sum(uint64_t v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  return v;
}

// 1. Block fingerprints and block-table insertion.
template <class M>
__global__ void k_block_fp(M m, Geo g, uint64_t* __restrict__ fpB, uint32_t* __restrict__ slotB,
                           BSlot* bt, uint64_t bmask, LevelDev* ld, Status* status) {
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < g.c;
       k += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t s = g.st[k], len = blen(g, k);
    uint64_t fp = window_fast(m, g.H, len == g.b ? g.Bb : g.Br, s, len);
    fpB[k] = fp;
    if (len == g.b) {
      uint32_t slot = tbl_insert(bt, bmask, fp);
      if (slot == kNoSlot) {
        atomicExch(&status->error, 1ull);
        slotB[k] = kNoSlot;
        continue;
      }
      slotB[k] = slot;
      // A block's own start is an occurrence: the slot minimum starts there
      // (the scan need not propose own windows).
      if (*(volatile unsigned long long*)&bt[slot].lo > s) atomicMin(&bt[slot].lo, (unsigned long long)s);
    } else {
      slotB[k] = kNoSlot;
      ld->fp_tail = fp;
      atomicMin(&ld->lo_tail, (unsigned long long)s);
    }
  }
}

// 2. Pair-table insertion: key (slot_k, slot_k+1) for pairs of full blocks.
__global__ void k_pair_insert(Geo g, const uint32_t* __restrict__ slotB, uint32_t* __restrict__ slotP,
                              PSlot* pt, uint64_t pmask, BSlot* bt, LevelDev* ld, Status* status) {
  // Warp-uniform loop: the pair count is summed per warp (one atomic each).
  const unsigned lane = threadIdx.x & 31;
  for (uint64_t base = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) & ~31ull; base + 1 < g.c;
       base += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t k = base + lane;
    const bool pair = k + 1 < g.c && g.st[k + 1] == g.st[k] + g.b;
    const uint32_t np = __popc(__ballot_sync(0xFFFFFFFFu, pair));
    if (lane == 0 && np) atomicAdd(&ld->npairs, np);
    if (k + 1 >= g.c) continue;
    uint32_t sp = kNoSlot;
    if (pair) {
      // The last pair start per first-block slot: a window after it cannot
      // be the leftmost occurrence of any pair that starts with that slot.
      if (slotB[k] != kNoSlot && *(volatile unsigned long long*)&bt[slotB[k]].maxpst < g.st[k])
        atomicMax(&bt[slotB[k]].maxpst, (unsigned long long)g.st[k]);
      if (slotB[k + 1] == kNoSlot) {
        sp = kTailPair;
        ld->pretail_slot = slotB[k];
        atomicMin(&ld->lo_tailpair, (unsigned long long)g.st[k]);  // its own start
      } else {
        sp = tbl_insert(pt, pmask, ((uint64_t)slotB[k] << 32) | slotB[k + 1]);
        if (sp == kNoSlot) atomicExch(&status->error, 2ull);
        else if (*(volatile unsigned long long*)&pt[sp].lo > g.st[k])
          atomicMin(&pt[sp].lo, (unsigned long long)g.st[k]);  // its own start
      }
    }
    slotP[k] = sp;
  }
}

// 3. The window scan.
// `tail_only`: only the short-tail windows, and only when the anchored scan
// could not cover the tail key (it has no anchor).
template <class M>
__global__ void __launch_bounds__(256) k_scan(M m, Geo g, uint64_t cpb,
                                             BSlot* bt, uint64_t bmask, PSlot* pt, uint64_t pmask,
                                             LevelDev* ld, int tail_only) {
  if (tail_only && ld->tail_anchorless != 1u) return;  // 1: the tail is shorter than a gram
  const uint64_t total = g.c * cpb;
  const uint32_t pretail = ld->pretail_slot;
  const uint64_t fp_tail = ld->fp_tail;
  for (uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; w < total;
       w += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t k = w / cpb, j = w - k * cpb;
    const uint64_t s = g.st[k], len = blen(g, k);
    const uint64_t p0 = s + j * kScanQ;
    if (p0 >= s + len) continue;
    const uint64_t pend = (p0 + kScanQ < s + len) ? p0 + kScanQ : s + len;
    const uint64_t av = avail_end(g, k);
    if (!tail_only && p0 + g.b <= av) {
      uint64_t fp = window_fast(m, g.H, g.Bb, p0, g.b);
      for (uint64_t p = p0; p < pend && p + g.b <= av; p++) {
        if (p > p0) {
          uint64_t out = (uint64_t)g.T[p - 1] + 1, in = (uint64_t)g.T[p + g.b - 1] + 1;
          fp = m.add(m.sub(m.mul(fp, g.B), m.mul(out, g.Bb)), in);
        }
        uint32_t sl = tbl_find(bt, bmask, fp);
        if (sl == kNoSlot) continue;
        min_pos(&bt[sl].lo, p);
        if (p + 2 * g.b <= av) {
          uint64_t fp2 = window_fast(m, g.H, g.Bb, p + g.b, g.b);
          uint32_t s2 = tbl_find(bt, bmask, fp2);
          if (s2 != kNoSlot) {
            uint32_t ps = tbl_find(pt, pmask, ((uint64_t)sl << 32) | s2);
            if (ps != kNoSlot) min_pos(&pt[ps].lo, p);
          }
        }
        if (g.r && sl == pretail && p + g.b + g.r <= av &&
            window_fast(m, g.H, g.Br, p + g.b, g.r) == fp_tail)
          min_pos(&ld->lo_tailpair, p);
      }
    }
    if (g.r && p0 + g.r <= av) {
      uint64_t fp = window_fast(m, g.H, g.Br, p0, g.r);
      for (uint64_t p = p0; p < pend && p + g.r <= av; p++) {
        if (p > p0) {
          uint64_t out = (uint64_t)g.T[p - 1] + 1, in = (uint64_t)g.T[p + g.r - 1] + 1;
          fp = m.add(m.sub(m.mul(fp, g.B), m.mul(out, g.Br)), in);
        }
        if (fp == fp_tail) min_pos(&ld->lo_tail, p);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// 3''. The sort-based window pass (BT_FLAG_SORT_SCAN; section 4.1).  Instead
// of probing the key table with every window, the fingerprints of all windows
// of a length are written as (fingerprint, position) tuples in text order and
// sorted stably: equal fingerprints become consecutive, in position order, so
// the first tuple of a key's group is the leftmost window with the key's
// fingerprint.  Each key finds its group by binary search.  The minima go to
// the same table fields the scan fills, and verification, marks, pointers and
// the split follow unchanged.
// ---------------------------------------------------------------------------
template <class M>
__global__ void k_sort_windows(M m, Geo g, uint64_t L, uint64_t BL, uint32_t bshift, uint64_t* __restrict__ keys,
                               uint32_t* __restrict__ vals) {
  const uint64_t total = g.c * g.b;
  for (uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; w < total;
       w += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t k = bshift != 0xFFu ? w >> bshift : w / g.b, j = w - k * g.b;
    uint64_t key = kNone;
    const uint64_t p = g.st[k] + j;
    if (j < blen(g, k) && p + L <= avail_end(g, k)) key = window_fast(m, g.H, BL, p, L);
    keys[w] = key;
    vals[w] = (uint32_t)p;
  }
}

__device__ __forceinline__ uint64_t lower_bound_u64(const uint64_t* __restrict__ a, uint64_t n, uint64_t x) {
  uint64_t lo = 0, hi = n;
  while (lo < hi) {
    const uint64_t mid = (lo + hi) / 2;
    if (a[mid] < x) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// pair = 0: every full-length block's slot minimum from the sorted windows of
// length b; pair = 1: every pair's slot minimum from those of length 2b.
template <class M>
__global__ void k_sort_minima(M m, Geo g, int pair, const uint64_t* __restrict__ fpB,
                              const uint32_t* __restrict__ slotB, const uint32_t* __restrict__ slotP, BSlot* bt,
                              PSlot* pt, const uint64_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                              uint64_t nkeys) {
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < g.c;
       k += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t F;
    unsigned long long* lo;
    if (!pair) {
      if (slotB[k] == kNoSlot) continue;
      F = fpB[k];
      lo = &bt[slotB[k]].lo;
    } else {
      if (k + 1 >= g.c || slotP[k] == kNoSlot || slotP[k] == kTailPair) continue;
      F = m.add(m.mul(fpB[k], g.Bb), fpB[k + 1]);
      lo = &pt[slotP[k]].lo;
    }
    const uint64_t h = lower_bound_u64(keys, nkeys, F);
    if (h < nkeys && keys[h] == F) min_pos(lo, vals[h]);
  }
}

// The short tail (length r) and the pair ending in it (length b + r): the
// leftmost window with each fingerprint, a minimum per CTA then one atomic.
template <class M>
__global__ void __launch_bounds__(256) k_sort_tail(M m, Geo g, uint32_t bshift, const uint64_t* __restrict__ fpB,
                                                   const uint32_t* __restrict__ slotP, LevelDev* ld) {
  __shared__ unsigned long long s_min[2];
  if (threadIdx.x == 0) s_min[0] = s_min[1] = kNone;
  __syncthreads();
  const uint64_t fp_tail = ld->fp_tail;
  const bool tp = g.c >= 2 && slotP[g.c - 2] == kTailPair;
  const uint64_t fp_tp = tp ? m.add(m.mul(fpB[g.c - 2], g.Br), fp_tail) : 0;
  uint64_t m0 = kNone, m1 = kNone;
  const uint64_t total = g.c * g.b;
  for (uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; w < total;
       w += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t k = bshift != 0xFFu ? w >> bshift : w / g.b, j = w - k * g.b;
    if (j >= blen(g, k)) continue;
    const uint64_t p = g.st[k] + j, av = avail_end(g, k);
    if (p < m0 && p + g.r <= av && window_fast(m, g.H, g.Br, p, g.r) == fp_tail) m0 = p;
    if (tp && p < m1 && p + g.b + g.r <= av && window_fast(m, g.H, g.Bbr, p, g.b + g.r) == fp_tp) m1 = p;
  }
  if (m0 != kNone) atomicMin(&s_min[0], (unsigned long long)m0);
  if (m1 != kNone) atomicMin(&s_min[1], (unsigned long long)m1);
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s_min[0] != kNone) atomicMin(&ld->lo_tail, s_min[0]);
    if (s_min[1] != kNone) atomicMin(&ld->lo_tailpair, s_min[1]);
  }
}

// ---------------------------------------------------------------------------
// 3'''. Domain decomposition of the sort-based pass (section 4.2): the
// windows of a level are taken in K parts of consecutive windows.  In each
// part only the windows whose fingerprint is a key's pass the filter (a bit
// map of the keys' fingerprints, then a binary search in their sorted list),
// those are sorted, and the first of each fingerprint -- the part's leftmost
// occurrence -- is kept.  The kept tuples of all parts, at most K per key, are
// sorted once more; as the parts are in text order and the sort is stable,
// the first tuple of a key's group is again its leftmost window.  The working
// memory is a part's tuples plus K tuples per key instead of a tuple per
// window.
// ---------------------------------------------------------------------------

// Fingerprints of the keys of one length: a block's (pair = 0) or a pair's
// (pair = 1), kNone where block k has no such key; each key's bit is set in
// kbits.
template <class M>
__global__ void k_key_list(M m, Geo g, int pair, const uint64_t* __restrict__ fpB,
                           const uint32_t* __restrict__ slotB, const uint32_t* __restrict__ slotP,
                           uint64_t* __restrict__ out, uint32_t* __restrict__ kbits, uint64_t kbmask) {
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < g.c;
       k += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t F = kNone;
    if (!pair) {
      if (slotB[k] != kNoSlot) F = fpB[k];
    } else if (k + 1 < g.c && slotP[k] != kNoSlot && slotP[k] != kTailPair) {
      F = m.add(m.mul(fpB[k], g.Bb), fpB[k + 1]);
    }
    out[k] = F;
    if (F != kNone) {
      const uint64_t bit = mix64(F) & kbmask;
      atomicOr(&kbits[bit >> 5], 1u << (bit & 31));
    }
  }
}

// Windows [w0, w0 + nw) of length L: the tuple of each, and flag = 1 where
// its fingerprint is a key's.
template <class M>
__global__ void k_part_windows(M m, Geo g, uint64_t L, uint64_t BL, uint32_t bshift, uint64_t w0, uint64_t nw,
                               const uint32_t* __restrict__ kbits, uint64_t kbmask,
                               const uint64_t* __restrict__ skeys, uint64_t nk, uint64_t* __restrict__ keys,
                               uint32_t* __restrict__ vals, uint32_t* __restrict__ flag) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < nw;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t w = w0 + i;
    const uint64_t k = bshift != 0xFFu ? w >> bshift : w / g.b, j = w - k * g.b;
    const uint64_t p = g.st[k] + j;
    uint64_t key = kNone;
    uint32_t f = 0;
    if (j < blen(g, k) && p + L <= avail_end(g, k)) {
      key = window_fast(m, g.H, BL, p, L);
      const uint64_t bit = mix64(key) & kbmask;
      if ((kbits[bit >> 5] >> (bit & 31)) & 1u) {
        const uint64_t h = lower_bound_u64(skeys, nk, key);
        f = h < nk && skeys[h] == key;
      }
    }
    keys[i] = key;
    vals[i] = (uint32_t)p;
    flag[i] = f;
  }
}

// The tuples i < n with flag[i] = 1 to out[offs[i]] (offs: exclusive prefix
// sums of flag); *count = their number.
__global__ void k_compact_tuples(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                                 const uint32_t* __restrict__ flag, const uint32_t* __restrict__ offs, uint64_t n,
                                 uint64_t* __restrict__ okeys, uint32_t* __restrict__ ovals,
                                 unsigned long long* count) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    if (flag[i]) {
      okeys[offs[i]] = keys[i];
      ovals[offs[i]] = vals[i];
    }
    if (i + 1 == n) *count = (unsigned long long)offs[i] + flag[i];
  }
}

// flag[i] = 1 for the first tuple of each fingerprint of a sorted list.
__global__ void k_first_of_key(const uint64_t* __restrict__ keys, uint64_t n, uint32_t* __restrict__ flag) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    flag[i] = i == 0 || keys[i] != keys[i - 1];
}

// ---------------------------------------------------------------------------
// 3'. The anchored window scan.
//
// Probing the table at every window position costs a random memory access
// per text byte.  Instead every window gets an anchor that depends only on its
// content: the first position of a w-gram whose mixed 32-bit gram hash is
// "selected" (at most 2^(32-sbits) - 1, density 2^-sbits).  Every key is
// registered under its anchor gram: the anchor table maps a gram to the set of
// offsets (a 64-bit mask for offsets below W, plus one far offset) at which
// keys anchor on it.  The scan rolls the 32-bit gram hash over the level (no
// 61-bit arithmetic per byte) and only records the selected grams; a second
// pass tests those against a bitmap filter, reads the anchor table for the
// few that pass, and each offset a proposes the window at x - a, whose 61-bit
// fingerprint is then looked up in the block table.  A window equal to a key
// has the key's anchor (same gram, same offset), so it is always proposed: the
// slot minima are the same as when probing every window.  A key without any
// selected gram (or whose far offset clashes with another key's on the same
// gram) is registered by its first gram in a small shared-memory filter that
// is checked at every position only when such keys exist.
// ---------------------------------------------------------------------------
constexpr uint32_t kAnchorQ = 128;        // gram positions per thread
constexpr uint32_t kAnchorWmax = 64;      // near anchor range (bits of the offset mask)
constexpr uint32_t kFarMax = 4096;        // far anchors are searched up to this offset
constexpr uint32_t kNoFar = 0xFFFFFFFFu;
constexpr uint32_t kEmptyGram = 0xFFFFFFFFu;
constexpr uint32_t kFibMul = 0x9E3779B1u;
constexpr uint32_t kScanThreads = 256;
constexpr uint32_t kSlotWords = 37;       // staging words per thread (37 is odd: no bank conflicts)
constexpr uint32_t kRing = 32;            // selected grams remembered per thread
constexpr uint32_t kSecBits = 4096;       // first-gram filter of keys without an anchor
constexpr uint32_t kSmemBitmapWords = 8192;  // anchor bitmap kept in shared memory up to 32 KiB

struct GramP {
  uint32_t w;        // gram length
  uint32_t W;        // near anchor range for full-length windows
  uint32_t Wr;       // near anchor range for the short tail (0: no gram fits)
  uint32_t sbits;    // selection density 2^-sbits
  uint32_t sel_max;  // a mixed gram hash is selected iff it is <= sel_max
  uint32_t fbits;    // bitmap index bits
  uint32_t rb;       // gram base (odd)
  uint32_t rw;       // rb^w mod 2^32
};

// gram -> offsets at which keys anchor on it.
struct __align__(32) AnchorSet {
  uint32_t gram;             // remapped mixed gram hash (kEmptyGram: empty slot)
  uint32_t far;              // one anchor offset >= W (kNoFar: none)
  unsigned long long offs;   // bit a: some key has its anchor at offset a < W
  unsigned long long maxst;  // largest start of a key anchored on this gram
  uint32_t more;             // further anchor offsets >= W: a list of FarNodes (kNoFar: none)
  uint32_t pad;
};

// A further far anchor offset of a gram (keys whose first selected gram lies
// beyond the offset mask are rare; two of them on one gram rarer still).
struct FarNode {
  uint32_t off;
  uint32_t next;
};

// The gram hash is a polynomial in rb over the symbols; its mixed value
// (times an odd constant, a bijection) decides selection, the bitmap bit and
// the table key.
__device__ __forceinline__ uint32_t gram_mix(uint32_t gh) { return gh * kFibMul; }
__device__ __forceinline__ uint32_t gram_bit(const GramP& gp, uint32_t mx) {
  return (mx << gp.sbits) >> (32 - gp.fbits);
}
// Mixed hashes are remapped away from 0xFFFFFFFF, the empty marker.
__device__ __forceinline__ uint32_t gram_key(uint32_t mx) { return mx == kEmptyGram ? kEmptyGram - 1 : mx; }
__device__ __forceinline__ uint32_t gram_slot(uint32_t g, uint32_t mask) {
  g ^= g >> 16;
  g *= 0x7FEB352Du;
  g ^= g >> 15;
  g *= 0x846CA68Bu;
  g ^= g >> 16;
  return g & mask;
}
__device__ __forceinline__ uint32_t sec_bit(uint32_t mx) { return (mx * 0x2545F491u) >> 20; }  // 12 bits

// Register the anchor of every key (every block and the tail).
__global__ void k_anchor_keys(Geo g, GramP gp, const uint32_t* __restrict__ slotB, AnchorSet* atab,
                              uint32_t amask, FarNode* fnode, uint32_t fcap, uint32_t* bitmap,
                              uint32_t* secbits, uint32_t* __restrict__ aidx, LevelDev* ld, Status* status) {
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < g.c;
       k += (uint64_t)gridDim.x * blockDim.x) {
    aidx[k] = kNoSlot;
    const uint64_t s = g.st[k], len = blen(g, k);
    const bool tail = len != g.b;
    uint32_t Wk;
    if (!tail) {
      if (slotB[k] == kNoSlot) continue;
      Wk = gp.W;
    } else {
      Wk = gp.Wr;
      if (Wk == 0) {  // shorter than a gram: the dense tail scan covers it
        ld->tail_anchorless = 1u;
        continue;
      }
    }
    // Gram positions of the key: [0, len - w]; the far search stops at kFarMax.
    const uint64_t npos = len - gp.w + 1;
    const uint32_t lim = (uint32_t)(npos < kFarMax ? npos : kFarMax);
    uint32_t gh = 0;
    for (uint32_t i = 0; i < gp.w; i++) gh = gh * gp.rb + g.T[s + i];
    const uint32_t mx0 = gram_mix(gh);
    uint32_t a = kNoSlot, mx = mx0;
    for (uint32_t o = 0; o < lim; o++) {
      if (o > 0) gh = gh * gp.rb - (uint32_t)g.T[s + o - 1] * gp.rw + g.T[s + o + gp.w - 1];
      mx = gram_mix(gh);
      if (mx <= gp.sel_max) {
        a = o;
        break;
      }
    }
    const uint32_t gk = gram_key(mx);
    bool sec = a == kNoSlot;
    if (!sec && !tail) {
      uint32_t h = gram_slot(gk, amask), hp = kNoSlot;
      bool placed = false;
      for (uint32_t it = 0; it <= amask && !placed; it++) {
        const uint32_t cur = atomicCAS(&atab[h].gram, kEmptyGram, gk);
        if (cur == kEmptyGram || cur == gk) {
          placed = true;
          hp = h;
          if (a < Wk) {
            atomicOr(&atab[h].offs, 1ull << a);
          } else {
            const uint32_t f = atomicCAS(&atab[h].far, kNoFar, a);
            if (f != kNoFar && f != a) {  // another far offset holds the entry: a list node
              const uint32_t id = atomicAdd(&ld->nfar, 1u);
              if (id < fcap) {
                fnode[id].off = a;
                fnode[id].next = atomicExch(&atab[h].more, id);
              } else {
                sec = true;
              }
            }
            if (!sec) atomicMax(&ld->far_end, a + 1);
          }
          atomicMax(&atab[h].maxst, (unsigned long long)s);
        } else {
          h = (h + 1) & amask;
        }
      }
      if (!placed) atomicExch(&status->error, 7ull);
      if (placed && !sec) aidx[k] = hp;
    }
    if (sec) {  // no usable anchor: registered by its first gram
      const uint32_t sb = sec_bit(mx0);
      atomicOr(&secbits[sb >> 5], 1u << (sb & 31));
      if (tail) ld->tail_anchorless = 2u;
      else ld->anchorless = 1u;
      continue;
    }
    const uint32_t bit = gram_bit(gp, mx);
    atomicOr(&bitmap[bit >> 5], 1u << (bit & 31));
    if (tail) {
      ld->tail_gram = gk;
      ld->tail_a = a;
    }
  }
}

template <class M>
struct ScanCtx {
  M m;
  Geo g;
  BSlot* bt;
  uint64_t bmask;
  PSlot* pt;
  uint64_t pmask;
  LevelDev* ld;
  uint32_t pretail;
  uint64_t fp_tail;
  struct Hit* q;                     // gram hits: one segment of `seg` entries per scan CTA
  uint32_t* segn;                    // hits recorded by each scan CTA (may exceed seg)
  uint32_t seg;
  unsigned long long* qn;            // hits recorded in all
  struct Cand* cq;                   // proposed windows: one segment of `cseg` entries per CTA
  uint32_t* csegn;                   // windows proposed by each k_hits CTA (may exceed cseg)
  uint32_t cseg;
  Status* status;                    // device-side invariant checks
  const FarNode* fnode;              // further far anchor offsets of the anchor table
  const uint32_t* slotB;             // block slot of every block
};

// A gram position x found by the scan in (a chunk of) block k: a selected
// gram that passed the bitmap filter, with its mixed hash mx; or, with the
// top bit of x set, a position whose first gram hit the filter of keys
// without an anchor.
struct Hit {
  uint64_t x;
  uint32_t k;
  uint32_t mx;
};
constexpr uint64_t kHitSec = 1ull << 63;

// A proposed window: start p and the end of the run span it lies in; the top
// bit of `av` marks the short tail key (else a full-length key).
struct Cand {
  uint64_t p;
  uint64_t av;
};
constexpr uint64_t kCandTail = 1ull << 63;

// A full-length window at p (inside a run ending at av) matches slot sl;
// Hb = H[p + b].  Updates the slot minimum and joins the pair starting here.
template <class M>
__device__ __forceinline__ void on_block_hit(const ScanCtx<M>& C, uint32_t sl, uint64_t p, uint64_t av,
                                             uint64_t Hb) {
  const Geo& g = C.g;
  min_pos(&C.bt[sl].lo, p);
  if (p > C.bt[sl].maxpst) return;  // no pair starting with this slot can begin here or later
  if (p + 2 * g.b <= av) {
    const uint64_t fp2 = C.m.sub(__ldcs(g.H + p + 2 * g.b), C.m.mul(Hb, g.Bb));
    const uint32_t s2 = tbl_find(C.bt, C.bmask, fp2);
    if (s2 != kNoSlot) {
      const uint32_t ps = tbl_find(C.pt, C.pmask, ((uint64_t)sl << 32) | s2);
      if (ps != kNoSlot) min_pos(&C.pt[ps].lo, p);
    }
  }
  if (g.r && sl == C.pretail && p + g.b + g.r <= av &&
      window_fast(C.m, g.H, g.Br, p + g.b, g.r) == C.fp_tail)
    min_pos(&C.ld->lo_tailpair, p);
}

// Does the window [p, p+L) lie inside a run?  p lies in block k or, when k-1 is
// consecutive with k, in block k-1.  *avp receives the end of its run span.
__device__ __forceinline__ bool window_in_run(const Geo& g, uint64_t k, uint64_t s, uint64_t av,
                                              uint64_t p, uint64_t L, uint64_t* avp) {
  if (p >= s) {
    *avp = av;
  } else if (k > 0 && g.st[k - 1] + g.b == s && p >= g.st[k - 1]) {
    *avp = avail_end(g, k - 1);
  } else {
    return false;
  }
  return p + L <= *avp;
}

// Test one candidate window.
template <class M>
__device__ __forceinline__ void test_candidate(const ScanCtx<M>& C, uint64_t p, uint64_t avp, uint32_t kind,
                                               uint32_t& ncand, uint32_t& nhit) {
  const Geo& g = C.g;
  if (kind) {
    if (window_fast(C.m, g.H, g.Br, p, g.r) == C.fp_tail) min_pos(&C.ld->lo_tail, p);
    return;
  }
  ncand++;
  const uint64_t Hb = __ldcs(g.H + p + g.b);
  const uint64_t fp = C.m.sub(Hb, C.m.mul(__ldcs(g.H + p), g.Bb));
  const uint32_t sl = tbl_find(C.bt, C.bmask, fp);
  if (sl != kNoSlot) {
    nhit++;
    on_block_hit(C, sl, p, avp, Hb);
  }
}

// A proposed window that starts at p (kind 0: a full-length key, 1: the
// short tail), if it lies inside a run: queued in this CTA's candidate
// segment (sq: its shared-memory counter), or tested here when sq is null.
template <class M>
__device__ __forceinline__ void propose(const ScanCtx<M>& C, unsigned int* sq, uint64_t k, uint64_t s,
                                        uint64_t av, uint64_t p, uint32_t kind, uint32_t& ncand,
                                        uint32_t& nhit) {
  uint64_t avp;
  if (!window_in_run(C.g, k, s, av, p, kind ? C.g.r : C.g.b, &avp)) return;
  // Own windows (a full block at its start, the tail at its start) are
  // occurrences the tables start with; so are the pairs starting there.  A
  // full block with the slot of the block before the tail is still tested:
  // the pair ending in the tail may occur at its start.
  if (kind == 0) {
    const uint64_t own = (p == s && C.g.n - s >= C.g.b) ? k : (p + C.g.b == s ? k - 1 : kNone);
    if (own != kNone && !(C.g.r && C.slotB[own] == C.pretail)) return;
  } else if (p == s && C.g.n - s < C.g.b) {
    return;
  }
  if (!sq) {
    test_candidate(C, p, avp, kind, ncand, nhit);
    return;
  }
  const uint32_t idx = atomicAdd(sq, 1u);
  if (idx < C.cseg) C.cq[blockIdx.x * (uint64_t)C.cseg + idx] = Cand{p, avp | (kind ? kCandTail : 0)};
}

// Record a hit in this CTA's segment (a shared-memory counter claims the
// slot; past the segment's end only the count grows).
template <class M>
__device__ __forceinline__ void record_hit(const ScanCtx<M>& C, unsigned int* sq, uint64_t x, uint64_t k,
                                           uint32_t mx) {
  const uint32_t idx = atomicAdd(sq, 1u);
  if (idx < C.seg) C.q[blockIdx.x * (uint64_t)C.seg + idx] = Hit{x, (uint32_t)k, mx};
}

// The anchor-table lookup of a hit at x (mixed gram mx) in block k and the
// test of every window its anchors propose.
template <class M>
__device__ __forceinline__ void anchor_hit(const ScanCtx<M>& C, unsigned int* sq, const AnchorSet* __restrict__ atab,
                                           uint32_t amask, uint32_t tail_gram, uint32_t tail_a, uint64_t k,
                                           uint64_t s, uint64_t av, uint64_t x, uint32_t mx, uint32_t& ncand,
                                           uint32_t& nhit) {
  const uint32_t gk = gram_key(mx);
  unsigned long long offs = 0, maxst = 0;
  uint32_t far = kNoFar, node = kNoFar;
  for (uint32_t h = gram_slot(gk, amask), it = 0; it <= amask; h = (h + 1) & amask, it++) {
    const uint32_t eg = atab[h].gram;
    if (eg == gk) {
      offs = atab[h].offs;
      far = atab[h].far;
      maxst = atab[h].maxst;
      node = atab[h].more;
      break;
    }
    if (eg == kEmptyGram) break;
  }
  // A window that starts after every key anchored on this gram cannot be
  // the leftmost occurrence of any of them, nor of a pair that starts with
  // one of them (both are at or before the key's start).
  bool pt = gk == tail_gram && x >= tail_a;
  bool pf = far != kNoFar;
  while (offs || pf || pt || node != kNoFar) {
    uint32_t a = 0, kind = 0;
    if (pt) {
      pt = false;
      a = tail_a;
      kind = 1;
    } else if (offs) {
      a = __ffsll(offs) - 1;
      offs &= offs - 1;
    } else if (pf) {
      pf = false;
      a = far;
    } else {
      const FarNode fn = C.fnode[node];
      node = fn.next;
      a = fn.off;
    }
    if (a <= x && (kind || x - a <= maxst)) propose(C, sq, k, s, av, x - a, kind, ncand, nhit);
  }
}

// Copy T[a, a+cnt) (cnt <= 144) into a thread's shared-memory slot.  When a
// is 16-byte aligned (block starts are multiples of 16 at the usual leaf
// lengths) the whole 16-byte units covering it are loaded at once, all in
// flight together; otherwise 16-byte loads for the aligned body and bytes
// for the rest.
__device__ __forceinline__ void stage(uint8_t* slot, const uint8_t* __restrict__ T, uint64_t n,
                                      uint64_t a, uint32_t cnt, bool aligned16) {
  const uint32_t units = (cnt + 15) / 16;
  if (aligned16 && (a & 15) == 0 && a + 16ull * units <= n) {
    const uint4* src = (const uint4*)(T + a);
    uint32_t* d = (uint32_t*)slot;
#pragma unroll
    for (uint32_t h = 0; h < 9; h += 5) {  // two batches of loads in flight
      uint4 v[5];
#pragma unroll
      for (uint32_t u = 0; u < 5; u++)
        if (h + u < units) v[u] = src[h + u];
#pragma unroll
      for (uint32_t u = 0; u < 5; u++)
        if (h + u < units) {
          d[4 * (h + u)] = v[u].x;
          d[4 * (h + u) + 1] = v[u].y;
          d[4 * (h + u) + 2] = v[u].z;
          d[4 * (h + u) + 3] = v[u].w;
        }
    }
    return;
  }
  uint32_t i = 0;
  if (aligned16) {
    const uint64_t a16 = (a + 15) & ~15ull;
    const uint32_t head = (uint32_t)(a16 - a) < cnt ? (uint32_t)(a16 - a) : cnt;
    for (; i < head; i++) slot[i] = T[a + i];
    for (; i + 16 <= cnt && a + i + 16 <= n; i += 16) {
      const uint4 q = *(const uint4*)(T + a + i);
      uint32_t* d = (uint32_t*)(slot + i);
      if ((((uintptr_t)d) & 3) == 0) {
        d[0] = q.x;
        d[1] = q.y;
        d[2] = q.z;
        d[3] = q.w;
      } else {
        const uint32_t v[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int t = 0; t < 16; t++) slot[i + t] = (uint8_t)(v[t >> 2] >> (8 * (t & 3)));
      }
    }
  }
  for (; i < cnt; i++) slot[i] = T[a + i];
}

// Mixed gram hash at slot position i, from the staged bytes.
__device__ __forceinline__ uint32_t gram_at(const uint8_t* slot, uint32_t i, uint32_t w, uint32_t rb) {
  uint32_t h = 0;
  for (uint32_t t = 0; t < w; t++) h = h * rb + slot[i + t];
  return gram_mix(h);
}

__device__ __forceinline__ uint32_t pick4(uint32_t G, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  return G == 0 ? a : G == 1 ? b : G == 2 ? c : d;
}

// Record a position's mixed gram: selected ones set bit BIT of V and enter
// the ring at rp (the ring pointer advances and saturates at rlim; entries
// past kRing - 1 are recomputed when needed).
#define BT_RECORD(MX, V, BIT)                      \
  {                                                \
    const bool sel_ = (MX) <= sel_max;             \
    *rp = (MX);                                    \
    rp += sel_ ? kScanThreads : 0u;                \
    rp = rp < rlim ? rp : rlim;                    \
    if (sel_) V |= 1u << (BIT);                    \
  }

// INLINE = false: the scan, which queues proposed windows.  INLINE = true:
// runs only when the queue overflowed, and tests every proposed window here.
template <class M, bool INLINE>
__global__ void __launch_bounds__(kScanThreads, 3) k_scan_anchor(ScanCtx<M> C0, GramP gp, uint64_t cpb,
                                                             const AnchorSet* __restrict__ atab,
                                                             uint32_t amask,
                                                             const uint32_t* __restrict__ bitmap_g,
                                                             uint32_t bm_smem_words,
                                                             const uint32_t* __restrict__ secbits_g,
                                                             int sec_only) {
  if (INLINE && C0.ld->qover == 0) return;
  // sec_only: k_scan_list covers this level unless it has keys without an anchor.
  if (!INLINE && sec_only && C0.ld->anchorless != 1u && C0.ld->tail_anchorless != 2u) return;
  extern __shared__ uint32_t smem[];
  __shared__ unsigned int s_qn;  // hits this CTA recorded
  uint32_t* sec = smem;                                      // kSecBits / 32 words
  uint32_t* ring = sec + kSecBits / 32 + threadIdx.x;        // kRing x kScanThreads, this thread's column
  uint32_t* bms = smem + kSecBits / 32 + kRing * kScanThreads;  // bm_smem_words words
  uint32_t* slotw = bms + bm_smem_words + threadIdx.x * kSlotWords;
  uint8_t* slot = (uint8_t*)slotw;
  ScanCtx<M> C = C0;
  C.pretail = C.ld->pretail_slot;
  C.fp_tail = C.ld->fp_tail;
  const Geo& g = C.g;
  const bool anchorless = C.ld->anchorless == 1u;
  const bool tail_sec = C.ld->tail_anchorless == 2u;
  const uint32_t tail_gram = C.ld->tail_gram, tail_a = C.ld->tail_a;
  // Anchors lie below a window's start + Wx (+ Wt for the tail window).
  const uint32_t far_end = C.ld->far_end;
  const uint32_t Wx = gp.W > far_end ? gp.W : far_end;
  const uint32_t Wt0 = gp.Wr ? gp.Wr : 1;
  const uint32_t Wt = tail_a != 0xFFFFFFFFu && tail_a + 1 > Wt0 ? tail_a + 1 : Wt0;
  for (uint32_t i = threadIdx.x; i < kSecBits / 32; i += blockDim.x) sec[i] = secbits_g[i];
  for (uint32_t i = threadIdx.x; i < bm_smem_words; i += blockDim.x) bms[i] = bitmap_g[i];
  if (threadIdx.x == 0) s_qn = 0;
  __syncthreads();
  const uint32_t* bitmap = bm_smem_words ? bms : bitmap_g;
  const bool check_sec = anchorless || tail_sec;
  const bool aligned16 = (((uintptr_t)g.T) & 15) == 0;
  const uint32_t w = gp.w, rb = gp.rb, rw = gp.rw, sel_max = gp.sel_max;
  uint32_t* const rlim = ring + (kRing - 1) * kScanThreads;
  const uint64_t total = g.c * cpb;
  uint32_t ncand = 0, nhit = 0;
  // Warp-uniform trip count and a single-exit body, so that the lanes of a
  // warp meet again after every chunk.
  const unsigned lane = threadIdx.x & 31;
  for (uint64_t base = blockIdx.x * (uint64_t)blockDim.x + (threadIdx.x & ~31u); base < total;
       base += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t wi = base + lane;
    do {
      if (wi >= total) break;
      const uint64_t k = cpb == 1 ? wi : wi / cpb, j = wi - k * cpb;
      const uint64_t s = g.st[k], len = blen(g, k);
      const uint64_t p0 = s + j * kAnchorQ;
      if (p0 >= s + len) break;
      const uint64_t av = avail_end(g, k);
      // Gram positions x in [p0, xe): owned by this thread and able to anchor a
      // window that fits in the run (windows without an anchor start at their
      // first gram).
      uint64_t xe = p0 + kAnchorQ < s + len ? p0 + kAnchorQ : s + len;
      uint64_t xm = av >= g.b ? av - g.b + Wx : 0;
      if (g.r && av >= g.r) {
        const uint64_t xr = av - g.r + Wt;
        if (xr > xm) xm = xr;
      }
      const uint64_t gram_end = av + 1 >= w ? av + 1 - w : 0;  // grams must fit in the run
      if (xm > gram_end) xm = gram_end;
      if (xe > xm) xe = xm;
      if (xe <= p0) break;
      const uint32_t nx = (uint32_t)(xe - p0);
      if (p0 + nx + w - 1 > g.n || av > g.n) {  // invariant: grams lie inside the text
        atomicExch(&C.status->error, 8ull);
        break;
      }
      stage(slot, g.T, g.n, p0, nx + w - 1, aligned16);
      // Pass 1: roll the gram hash; selected grams set a bit of (m0, m1, m2, m3)
      // (positions 0-31, 32-63, ...) and enter the ring.  Positions past nx
      // are masked off afterwards (their ring entries follow the valid ones).
      uint32_t m0 = 0, m1 = 0, m2 = 0, m3 = 0;
      uint32_t* rp = ring;
      if (w == 16) {
        // The transition to position i removes byte i-1 and adds byte i+15, so
        // positions 4q+1 .. 4q+4 take the bytes of words q and q+4.
        uint32_t gh = 0;
#pragma unroll
        for (int t = 0; t < 4; t++) {
          const uint32_t v = slotw[t];
#pragma unroll
          for (int u = 0; u < 4; u++) gh = gh * rb + __byte_perm(v, 0, 0x4440 + u);
        }
        uint32_t cur = 0;
        {
          const uint32_t mx = gram_mix(gh);
          BT_RECORD(mx, cur, 0);
        }
        const uint32_t ngroups = (nx + 31) / 32;
#pragma unroll 1
        for (uint32_t G = 0; G < 4; G++) {
          uint32_t carry = 0;
          if (G < ngroups) {
#pragma unroll
            for (uint32_t qq = 0; qq < 8; qq++) {
              const uint32_t wo = slotw[8 * G + qq], wn = slotw[8 * G + qq + 4];
#pragma unroll
              for (uint32_t u = 0; u < 4; u++) {
                gh = gh * rb + __byte_perm(wn, 0, 0x4440 + u) - __byte_perm(wo, 0, 0x4440 + u) * rw;
                const uint32_t mx = gram_mix(gh);
                if (4 * qq + u + 1 < 32) {
                  BT_RECORD(mx, cur, (4 * qq + u + 1) & 31);
                } else {
                  BT_RECORD(mx, carry, 0);
                }
              }
            }
          }
          m3 = m2;
          m2 = m1;
          m1 = m0;
          m0 = cur;
          cur = carry;
        }
        // After four shifts m3 holds positions 0-31, ..., m0 positions 96-127.
        const uint32_t t0 = m3, t1 = m2;
        m3 = m0;
        m2 = m1;
        m0 = t0;
        m1 = t1;
      } else {
        uint32_t gh = 0;
        for (uint32_t i = 0; i < w; i++) gh = gh * rb + slot[i];
        for (uint32_t i = 0; i < nx; i++) {
          if (i) gh = gh * rb - (uint32_t)slot[i - 1] * rw + slot[i + w - 1];
          const uint32_t mx = gram_mix(gh);
          uint32_t bv = 0;
          BT_RECORD(mx, bv, 0);
          const uint32_t sh = bv << (i & 31);
          if (i < 32) m0 |= sh;
          else if (i < 64) m1 |= sh;
          else if (i < 96) m2 |= sh;
          else m3 |= sh;
        }
      }
      // Keep positions below nx.
      if (nx < 128) {
        m3 &= nx > 96 ? 0xFFFFFFFFu >> (128 - nx) : 0u;
        m2 &= nx >= 96 ? 0xFFFFFFFFu : nx > 64 ? 0xFFFFFFFFu >> (96 - nx) : 0u;
        m1 &= nx >= 64 ? 0xFFFFFFFFu : nx > 32 ? 0xFFFFFFFFu >> (64 - nx) : 0u;
        m0 &= nx >= 32 ? 0xFFFFFFFFu : 0xFFFFFFFFu >> (32 - nx);
      }
      const uint32_t c0 = __popc(m0), c1 = __popc(m1), c2 = __popc(m2);
      const uint32_t nsel = c0 + c1 + c2 + __popc(m3);
      const uint32_t exact = nsel < kRing ? nsel : kRing - 1;  // ring entries [0, exact) hold their gram
      // Pass 2a: bitmap filter of the selected grams, four loads in flight.
      uint32_t h0 = 0, h1 = 0, h2 = 0, h3 = 0;
      {
        uint32_t jr = 0;
#pragma unroll 1
        for (uint32_t G = 0; G < 4; G++) {
          uint32_t mm = pick4(G, m0, m1, m2, m3);
          uint32_t hit = 0;
          while (mm) {
            uint32_t pos[4], wv[4], bt[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
              pos[u] = 32;
              wv[u] = 0;
              bt[u] = 0;
              if (mm) {
                const uint32_t bpos = __ffs(mm) - 1;
                mm &= mm - 1;
                const uint32_t mx = jr < exact ? ring[jr * kScanThreads] : gram_at(slot, 32 * G + bpos, w, rb);
                jr++;
                const uint32_t bit = gram_bit(gp, mx);
                pos[u] = bpos;
                bt[u] = bit & 31;
                wv[u] = bitmap[bit >> 5];
              }
            }
#pragma unroll
            for (int u = 0; u < 4; u++)
              if (pos[u] < 32 && ((wv[u] >> bt[u]) & 1u)) hit |= 1u << pos[u];
          }
          if (G == 0) h0 = hit;
          else if (G == 1) h1 = hit;
          else if (G == 2) h2 = hit;
          else h3 = hit;
        }
      }
      // Pass 2b: the grams that passed the filter go to k_hits (INLINE: their
      // anchor-table lookup and window tests happen here).
#pragma unroll 1
      for (uint32_t G = 0; G < 4; G++) {
        uint32_t hm = pick4(G, h0, h1, h2, h3);
        const uint32_t below = pick4(G, 0, c0, c0 + c1, c0 + c1 + c2);
        const uint32_t mg = pick4(G, m0, m1, m2, m3);
        while (hm) {
          const uint32_t bpos = __ffs(hm) - 1;
          hm &= hm - 1;
          const uint32_t i = 32 * G + bpos;
          const uint32_t jr = below + __popc(mg & ((1u << bpos) - 1u));
          const uint32_t mx = jr < exact ? ring[jr * kScanThreads] : gram_at(slot, i, w, rb);
          if (INLINE) anchor_hit(C, nullptr, atab, amask, tail_gram, tail_a, k, s, av, p0 + i, mx, ncand, nhit);
          else record_hit(C, &s_qn, p0 + i, k, mx);
        }
      }
      // Pass 2c: windows of keys without an anchor start at a gram in the
      // first-gram filter (only when such keys exist).
      if (check_sec) {
        uint32_t gh = 0;
        for (uint32_t i = 0; i < w; i++) gh = gh * rb + slot[i];
        for (uint32_t i = 0; i < nx; i++) {
          if (i) gh = gh * rb - (uint32_t)slot[i - 1] * rw + slot[i + w - 1];
          const uint32_t sb = sec_bit(gram_mix(gh));
          if ((sec[sb >> 5] >> (sb & 31)) & 1u) {
            if (!INLINE) {
              record_hit(C, &s_qn, (p0 + i) | kHitSec, k, 0);
            } else {
#pragma unroll 1
              for (uint32_t kind = 0; kind < 2; kind++)
                if (kind ? tail_sec : anchorless) propose(C, nullptr, k, s, av, p0 + i, kind, ncand, nhit);
            }
          }
        }
      }
    } while (0);
  }
  if (ncand) atomicAdd(&C.ld->cands, (unsigned long long)ncand);
  if (nhit) atomicAdd(&C.ld->hits, (unsigned long long)nhit);
  if (!INLINE) {
    __syncthreads();
    if (threadIdx.x == 0) {
      C.segn[blockIdx.x] = s_qn;
      atomicAdd(C.qn, (unsigned long long)s_qn);
      if (s_qn > C.seg) C.ld->qover = 1u;
    }
  }
}
#undef BT_RECORD

// ---------------------------------------------------------------------------
// The selected-gram list.  On the levels whose block length is a multiple of
// 128 and whose selection is the default (w = 16, density 1/8), the selected
// grams of a chunk are the same at every level: their positions and mixed
// hashes are computed once per build, in 128-byte text chunks (the grams of
// chunk j at gl_chunk[j] .. gl_chunk[j+1] of gl_mx / gl_x, positions absolute),
// and those levels read the list instead of rolling the hash again.
// ---------------------------------------------------------------------------
constexpr uint32_t kGlSbits = 3;
constexpr uint64_t kGlMinText = 8ull << 20;  // smaller texts roll the hash at every level

// One 128-byte chunk per thread: count the selected grams starting in it
// into cnt[j] (WRITE = false), or write them from offset cnt[j] on (WRITE =
// true, cnt holding the exclusive prefix sums of the counts).
template <bool WRITE>
__global__ void __launch_bounds__(256) k_gl_pass(const uint8_t* __restrict__ T, uint64_t n, uint64_t nchunks,
                                                 uint32_t rb, uint32_t rw, uint32_t sel_max,
                                                 uint32_t* __restrict__ cnt, uint32_t* __restrict__ out_mx,
                                                 uint32_t* __restrict__ out_x) {
  __shared__ uint32_t slots[256 * kSlotWords];
  uint32_t* slotw = slots + threadIdx.x * kSlotWords;
  const bool aligned16 = (((uintptr_t)T) & 15) == 0;
  const uint64_t xlim = n - 15;  // grams start below n - 15
  for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < nchunks;
       j += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t p0 = j * kAnchorQ;
    const uint32_t nx = (uint32_t)(xlim - p0 < kAnchorQ ? xlim - p0 : kAnchorQ);
    stage((uint8_t*)slotw, T, n, p0, nx + 15, aligned16);
    const uint64_t o = WRITE ? cnt[j] : 0;
    uint32_t c = 0;
    uint32_t gh = 0;
#pragma unroll
    for (int t = 0; t < 4; t++) {
      const uint32_t v = slotw[t];
#pragma unroll
      for (int u = 0; u < 4; u++) gh = gh * rb + __byte_perm(v, 0, 0x4440 + u);
    }
    {
      const uint32_t mx = gram_mix(gh);
      if (mx <= sel_max) {
        if (WRITE) {
          out_mx[o] = mx;
          out_x[o] = (uint32_t)p0;
        }
        c++;
      }
    }
#pragma unroll 1
    for (uint32_t G = 0; G < 4 && 32 * G + 1 < nx; G++) {
#pragma unroll
      for (uint32_t qq = 0; qq < 8; qq++) {
        const uint32_t wo = slotw[8 * G + qq], wn = slotw[8 * G + qq + 4];
#pragma unroll
        for (uint32_t u = 0; u < 4; u++) {
          const uint32_t i = 32 * G + 4 * qq + u + 1;
          gh = gh * rb + __byte_perm(wn, 0, 0x4440 + u) - __byte_perm(wo, 0, 0x4440 + u) * rw;
          const uint32_t mx = gram_mix(gh);
          if (mx <= sel_max && i < nx) {
            if (WRITE) {
              out_mx[o + c] = mx;
              out_x[o + c] = (uint32_t)(p0 + i);
            }
            c++;
          }
        }
      }
    }
    if (!WRITE) cnt[j] = c;
  }
}

// The anchored scan of a level from the selected-gram list: per chunk, the
// listed grams below the chunk's end pass the bitmap filter (four loads in
// flight) and go to the hit queue.  Levels with keys without an anchor are
// left to k_scan_anchor (it needs every position's gram).
template <class M>
__global__ void __launch_bounds__(256) k_scan_list(ScanCtx<M> C0, GramP gp, uint64_t cpb,
                                                   const uint32_t* __restrict__ bitmap_g, uint32_t bm_smem_words,
                                                   const uint32_t* __restrict__ gl_chunk,
                                                   const uint32_t* __restrict__ gl_mx,
                                                   const uint32_t* __restrict__ gl_x) {
  if (C0.ld->anchorless == 1u || C0.ld->tail_anchorless == 2u) return;
  extern __shared__ uint32_t bms[];
  __shared__ unsigned int s_qn;
  const ScanCtx<M>& C = C0;
  const Geo& g = C.g;
  const uint32_t tail_a = C.ld->tail_a;
  const uint32_t far_end = C.ld->far_end;
  const uint32_t Wx = gp.W > far_end ? gp.W : far_end;
  const uint32_t Wt0 = gp.Wr ? gp.Wr : 1;
  const uint32_t Wt = tail_a != 0xFFFFFFFFu && tail_a + 1 > Wt0 ? tail_a + 1 : Wt0;
  for (uint32_t i = threadIdx.x; i < bm_smem_words; i += blockDim.x) bms[i] = bitmap_g[i];
  if (threadIdx.x == 0) s_qn = 0;
  __syncthreads();
  const uint32_t* bitmap = bm_smem_words ? bms : bitmap_g;
  const uint32_t w = gp.w;
  const uint64_t total = g.c * cpb;
  const unsigned lane = threadIdx.x & 31;
  for (uint64_t base = blockIdx.x * (uint64_t)blockDim.x + (threadIdx.x & ~31u); base < total;
       base += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t wi = base + lane;
    do {
      if (wi >= total) break;
      const uint64_t k = cpb == 1 ? wi : wi / cpb, j = wi - k * cpb;
      const uint64_t s = g.st[k], len = blen(g, k);
      const uint64_t p0 = s + j * kAnchorQ;
      if (p0 >= s + len) break;
      const uint64_t av = avail_end(g, k);
      uint64_t xe = p0 + kAnchorQ < s + len ? p0 + kAnchorQ : s + len;
      uint64_t xm = av >= g.b ? av - g.b + Wx : 0;
      if (g.r && av >= g.r) {
        const uint64_t xr = av - g.r + Wt;
        if (xr > xm) xm = xr;
      }
      const uint64_t gram_end = av + 1 >= w ? av + 1 - w : 0;
      if (xm > gram_end) xm = gram_end;
      if (xe > xm) xe = xm;
      if (xe <= p0) break;
      const uint32_t nx = (uint32_t)(xe - p0);
      const uint64_t cj = p0 / kAnchorQ;
      const uint32_t e1 = gl_chunk[cj + 1];
      for (uint32_t e = gl_chunk[cj]; e < e1; e += 4) {
        uint32_t pos[4], mx[4], wv[4], bt[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
          pos[u] = kAnchorQ;
          wv[u] = 0;
          bt[u] = 0;
          mx[u] = 0;
          if (e + u < e1) {
            pos[u] = (uint32_t)(gl_x[e + u] - p0);
            mx[u] = gl_mx[e + u];
            const uint32_t bit = gram_bit(gp, mx[u]);
            bt[u] = bit & 31;
            wv[u] = bitmap[bit >> 5];
          }
        }
#pragma unroll
        for (int u = 0; u < 4; u++)
          if (pos[u] < nx && ((wv[u] >> bt[u]) & 1u)) record_hit(C, &s_qn, p0 + pos[u], k, mx[u]);
      }
    } while (0);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    C.segn[blockIdx.x] = s_qn;
    atomicAdd(C.qn, (unsigned long long)s_qn);
    if (s_qn > C.seg) C.ld->qover = 1u;
  }
}

// The list scan of a level whose blocks are all present ([k b, (k+1) b),
// consecutive): the block of a gram and the end of its run follow from its
// position, so the whole list is read in order, coalesced, 16 entries per
// thread and step (16-byte loads), their bitmap loads in flight together.
// bshift: log2 b when b is a power of two, else 0.
template <class M>
__global__ void __launch_bounds__(256) k_scan_stream(ScanCtx<M> C0, GramP gp, uint32_t total, uint32_t bshift,
                                                     const uint32_t* __restrict__ bitmap_g, uint32_t bm_smem_words,
                                                     const uint32_t* __restrict__ gl_mx,
                                                     const uint32_t* __restrict__ gl_x) {
  if (C0.ld->anchorless == 1u || C0.ld->tail_anchorless == 2u) return;
  extern __shared__ uint32_t bms[];
  __shared__ unsigned int s_qn;
  const ScanCtx<M>& C = C0;
  const Geo& g = C.g;
  const uint32_t tail_a = C.ld->tail_a;
  const uint32_t far_end = C.ld->far_end;
  const uint32_t Wx = gp.W > far_end ? gp.W : far_end;
  const uint32_t Wt0 = gp.Wr ? gp.Wr : 1;
  const uint32_t Wt = tail_a != 0xFFFFFFFFu && tail_a + 1 > Wt0 ? tail_a + 1 : Wt0;
  for (uint32_t i = threadIdx.x; i < bm_smem_words; i += blockDim.x) bms[i] = bitmap_g[i];
  if (threadIdx.x == 0) s_qn = 0;
  __syncthreads();
  const uint32_t* bitmap = bm_smem_words ? bms : bitmap_g;
  const uint64_t b = g.b, w = gp.w;
  constexpr uint32_t U = 16;  // entries per thread and step (four 16-byte loads per array)
  const uint32_t totalU = (total + U - 1) / U;
  for (uint64_t eu = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; eu < totalU;
       eu += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t xs[U], mxs[U], wv[U], bt[U];
    if (U * eu + U <= total) {
#pragma unroll
      for (uint32_t q = 0; q < U / 4; q++) {
        const uint4 X = ((const uint4*)gl_x)[eu * (U / 4) + q], Y = ((const uint4*)gl_mx)[eu * (U / 4) + q];
        xs[4 * q] = X.x, xs[4 * q + 1] = X.y, xs[4 * q + 2] = X.z, xs[4 * q + 3] = X.w;
        mxs[4 * q] = Y.x, mxs[4 * q + 1] = Y.y, mxs[4 * q + 2] = Y.z, mxs[4 * q + 3] = Y.w;
      }
    } else {
#pragma unroll
      for (uint32_t u = 0; u < U; u++) {
        xs[u] = U * eu + u < total ? gl_x[U * eu + u] : 0xFFFFFFFFu;
        mxs[u] = U * eu + u < total ? gl_mx[U * eu + u] : 0;
      }
    }
#pragma unroll
    for (uint32_t u = 0; u < U; u++) {
      wv[u] = 0;
      bt[u] = 32;  // 32: no test
      const uint64_t x = xs[u];
      if (x >= g.n) continue;
      const uint64_t k = bshift ? x >> bshift : x / b;
      // End of block k and up to two following blocks.
      const uint64_t av = (k + 3) * b < g.n ? (k + 3) * b : g.n;
      uint64_t xm = av >= b ? av - b + Wx : 0;
      if (g.r && av >= g.r) {
        const uint64_t xr = av - g.r + Wt;
        if (xr > xm) xm = xr;
      }
      const uint64_t gram_end = av + 1 >= w ? av + 1 - w : 0;
      if (xm > gram_end) xm = gram_end;
      if (x >= xm) continue;
      const uint32_t bit = gram_bit(gp, mxs[u]);
      bt[u] = bit & 31;
      wv[u] = bitmap[bit >> 5];
    }
#pragma unroll
    for (uint32_t u = 0; u < U; u++)
      if (bt[u] < 32 && ((wv[u] >> bt[u]) & 1u))
        record_hit(C, &s_qn, xs[u], bshift ? (uint64_t)xs[u] >> bshift : xs[u] / b, mxs[u]);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    C.segn[blockIdx.x] = s_qn;
    atomicAdd(C.qn, (unsigned long long)s_qn);
    if (s_qn > C.seg) C.ld->qover = 1u;
  }
}

// The hits of scan CTA j's segment, one per thread: anchor-table lookup; the
// windows the anchors propose go to this CTA's candidate segment.
// With BT_FLAG_TWO_PHASE the windows of a level are tested in two phases:
// first those of the hits in the first 1/16 of the text, then the rest.
__device__ __forceinline__ uint64_t hit_split(const Geo& g) { return g.n >> 4; }

template <class M>
__global__ void __launch_bounds__(512) k_hits(ScanCtx<M> C0, const AnchorSet* __restrict__ atab,
                                              uint32_t amask, uint32_t phase) {
  __shared__ unsigned int s_cn;
  if (threadIdx.x == 0) s_cn = 0;
  __syncthreads();
  ScanCtx<M> C = C0;
  C.pretail = C.ld->pretail_slot;
  const Geo& g = C.g;
  const bool anchorless = C.ld->anchorless == 1u;
  const bool tail_sec = C.ld->tail_anchorless == 2u;
  const uint32_t tail_gram = C.ld->tail_gram, tail_a = C.ld->tail_a;
  const uint32_t sn = C.segn[blockIdx.x];
  const uint32_t n = sn < C.seg ? sn : C.seg;
  const Hit* q = C.q + blockIdx.x * (uint64_t)C.seg;
  // phase 0: every hit; 1: hits before the split; 2: hits from the split on.
  uint64_t x_lo = 0, x_hi = ~0ull;
  if (phase == 1) x_hi = hit_split(g);
  if (phase == 2) x_lo = hit_split(g);
  uint32_t ncand = 0, nhit = 0;
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
    const Hit e = q[i];
    const uint64_t x = e.x & ~kHitSec;
    if (e.k >= g.c || x >= g.n) {  // invariant check
      atomicExch(&C.status->error, 9ull);
      continue;
    }
    if (x < x_lo || x >= x_hi) continue;
    const uint64_t k = e.k, s = g.st[k], av = avail_end(g, k);
    if (e.x & kHitSec) {
      if (anchorless) propose(C, &s_cn, k, s, av, x, 0, ncand, nhit);
      if (tail_sec) propose(C, &s_cn, k, s, av, x, 1, ncand, nhit);
    } else {
      anchor_hit(C, &s_cn, atab, amask, tail_gram, tail_a, k, s, av, x, e.mx, ncand, nhit);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    C.csegn[blockIdx.x] = s_cn;
    if (s_cn > C.cseg) C.ld->qover = 1u;
  }
}

// Between the two phases of a level: each gram's bound on useful window
// starts (AnchorSet::maxst, first the largest start of a key anchored on it)
// drops to the largest current leftmost position among its keys, counting the
// pairs that start with them and the pair ending in the tail.  A window that
// starts after all of these cannot lower any of them, so the second phase
// proposes fewer windows and finds the same minima.  step 0 clears the bound
// of every gram that holds an anchored key, step 1 raises it again.
__global__ void k_anchor_bound(Geo g, const uint32_t* __restrict__ aidx, const uint32_t* __restrict__ slotB,
                               const uint32_t* __restrict__ slotP, const BSlot* __restrict__ bt,
                               const PSlot* __restrict__ pt, AnchorSet* atab, const LevelDev* ld, int step) {
  const uint32_t pretail = ld->pretail_slot;
  const unsigned long long ltp = ld->lo_tailpair;
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < g.c;
       k += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t h = aidx[k];
    if (h == kNoSlot) continue;
    if (step == 0) {
      atab[h].maxst = 0;
      continue;
    }
    const uint32_t sb = slotB[k];
    unsigned long long hi = bt[sb].lo;
    if (k + 1 < g.c) {
      const uint32_t sp = slotP[k];
      if (sp != kNoSlot && sp != kTailPair && pt[sp].lo > hi) hi = pt[sp].lo;
    }
    if (g.r && sb == pretail && ltp > hi) hi = ltp;
    atomicMax(&atab[h].maxst, hi);
  }
}

// Test the proposed windows of k_hits CTA j's segment, four per thread, in
// phases whose loads are all in flight together: the prefix fingerprints at
// p and p+b, the block-table probe; for the windows that match a block, the
// slot minimum (an atomic without return), the last pair start of the slot
// and the prefix fingerprint at p+2b; then the probe of the block at p+b and
// of the pair table.  Prefix fingerprints are read with the streaming
// (evict-first) hint: random and used once, they should not push the tables
// out of L2.
template <class M>
__global__ void __launch_bounds__(256, 3) k_candidates(ScanCtx<M> C0) {
  constexpr int U = 4;
  ScanCtx<M> C = C0;
  C.pretail = C.ld->pretail_slot;
  C.fp_tail = C.ld->fp_tail;
  const Geo& g = C.g;
  const uint32_t sn = C.csegn[blockIdx.x];
  const uint64_t n = sn < C.cseg ? sn : C.cseg;
  const Cand* q = C.cq + blockIdx.x * (uint64_t)C.cseg;
  uint32_t ncand = 0, nhit = 0;
  const unsigned lane = threadIdx.x & 31;
  for (uint64_t base = (threadIdx.x & ~31u) * (uint64_t)U; base < n; base += (uint64_t)blockDim.x * U) {
    const uint64_t i0 = base + lane * U;
    uint64_t p[U], av[U], H1[U], x[U], y[U];
    uint32_t sl[U];
    bool live[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      live[u] = false;
      sl[u] = kNoSlot;
      if (i0 + u < n) {
        const Cand e = q[i0 + u];
        p[u] = e.p;
        av[u] = e.av & ~kCandTail;
        if (av[u] > g.n || e.p + ((e.av & kCandTail) ? g.r : g.b) > av[u]) {  // invariant check
          atomicExch(&C.status->error, 9ull);
          continue;
        }
        if (e.av & kCandTail) {
          if (window_fast(C.m, g.H, g.Br, e.p, g.r) == C.fp_tail) min_pos(&C.ld->lo_tail, e.p);
        } else {
          live[u] = true;
        }
      }
    }
    // Window fingerprints and the first block-table probe.
#pragma unroll
    for (int u = 0; u < U; u++)
      if (live[u]) {
        x[u] = __ldcs(g.H + p[u]);
        H1[u] = __ldcs(g.H + p[u] + g.b);
      }
#pragma unroll
    for (int u = 0; u < U; u++)
      if (live[u]) {
        ncand++;
        x[u] = C.m.sub(H1[u], C.m.mul(x[u], g.Bb));  // x: the window's fingerprint
        y[u] = mix64(x[u]) & C.bmask;                  // y: its first slot
        sl[u] = (uint32_t)y[u];
        y[u] = C.bt[y[u]].key;                         // y: the key there
      }
#pragma unroll
    for (int u = 0; u < U; u++)
      if (live[u]) {
        if (y[u] != x[u]) sl[u] = y[u] == kNone ? kNoSlot : tbl_find(C.bt, C.bmask, x[u]);
        live[u] = sl[u] != kNoSlot;
      }
    // Block hits: slot minimum, pair start bound, prefix fingerprint at p+2b.
#pragma unroll
    for (int u = 0; u < U; u++)
      if (live[u]) {
        nhit++;
        atomicMin(&C.bt[sl[u]].lo, (unsigned long long)p[u]);
        x[u] = C.bt[sl[u]].maxpst;
        y[u] = p[u] + 2 * g.b <= av[u] ? __ldcs(g.H + p[u] + 2 * g.b) : kNone;
      }
#pragma unroll
    for (int u = 0; u < U; u++)
      if (live[u]) {
        // The short tail pair (rare: only the block before the tail).
        if (g.r && sl[u] == C.pretail && p[u] + g.b + g.r <= av[u] &&
            window_fast(C.m, g.H, g.Br, p[u] + g.b, g.r) == C.fp_tail)
          min_pos(&C.ld->lo_tailpair, p[u]);
        live[u] = p[u] <= x[u] && y[u] != kNone;  // a pair starting with this slot can begin here
        if (live[u]) {
          x[u] = C.m.sub(y[u], C.m.mul(H1[u], g.Bb));  // fingerprint of the block at p+b
          y[u] = mix64(x[u]) & C.bmask;
          H1[u] = C.bt[y[u]].key;
        }
      }
#pragma unroll
    for (int u = 0; u < U; u++)
      if (live[u]) {
        uint32_t s2 = (uint32_t)y[u];
        if (H1[u] != x[u]) s2 = H1[u] == kNone ? kNoSlot : tbl_find(C.bt, C.bmask, x[u]);
        live[u] = s2 != kNoSlot;
        if (live[u]) {
          x[u] = ((uint64_t)sl[u] << 32) | s2;  // the pair key
          y[u] = mix64(x[u]) & C.pmask;
          H1[u] = C.pt[y[u]].key;
        }
      }
#pragma unroll
    for (int u = 0; u < U; u++)
      if (live[u]) {
        uint32_t ps = (uint32_t)y[u];
        if (H1[u] != x[u]) ps = H1[u] == kNone ? kNoSlot : tbl_find(C.pt, C.pmask, x[u]);
        if (ps != kNoSlot) atomicMin(&C.pt[ps].lo, (unsigned long long)p[u]);
      }
  }
  if (ncand) atomicAdd(&C.ld->cands, (unsigned long long)ncand);
  if (nhit) atomicAdd(&C.ld->hits, (unsigned long long)nhit);
}

// 4a. Pair results: leftmost when the slot minimum is the pair's own start;
// otherwise queue a verification of the earlier occurrence.
__global__ void k_pair_jobs(Geo g, const uint32_t* __restrict__ slotP,
                            const PSlot* __restrict__ pt, uint64_t* __restrict__ plo_k,
                            uint8_t* __restrict__ pm, Job* jobs, uint64_t* job_of, LevelDev* ld,
                            Status* status) {
  const uint64_t np = g.c ? g.c - 1 : 0;
  const unsigned lane = threadIdx.x & 31;
  for (uint64_t base = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) & ~31ull; base < np;
       base += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t k = base + lane;
    bool want = false;
    uint64_t lo = 0, s = 0, len = 0;
    if (k < np) {
      const uint32_t sp = slotP[k];
      pm[k] = 0;
      job_of[k] = kNone;
      if (sp != kNoSlot) {
        lo = sp == kTailPair ? ld->lo_tailpair : pt[sp].lo;
        s = g.st[k];
        plo_k[k] = lo;
        if (lo == s) {
          pm[k] = 1;
        } else if (lo < s) {
          want = true;
          len = g.b + blen(g, k + 1);
        } else {
          atomicExch(&status->error, 3ull);  // the pair's own window was not seen
        }
      }
    }
    const uint64_t id = warp_claim(&ld->njobs, want);
    if (want) {
      jobs[id] = Job{lo, s, len, k};
      job_of[k] = id;
    }
    const uint64_t vb = warp_sum(want ? 2 * len : 0);
    if (lane == 0 && vb) atomicAdd(&status->verify_bytes, (unsigned long long)vb);
  }
}

// 4b. Byte verification of the queued jobs, in pieces of kPiece bytes, one
// warp per piece.
// The 16 bytes T[A, A+16) from the aligned units at A & ~15 (u0, u1).
__device__ __forceinline__ uint4 unaligned16(uint4 u0, uint4 u1, uint32_t d) {
  const uint32_t q = d >> 2, sh = 8 * (d & 3);
  const uint32_t w0 = q == 0 ? u0.x : q == 1 ? u0.y : q == 2 ? u0.z : u0.w;
  const uint32_t w1 = q == 0 ? u0.y : q == 1 ? u0.z : q == 2 ? u0.w : u1.x;
  const uint32_t w2 = q == 0 ? u0.z : q == 1 ? u0.w : q == 2 ? u1.x : u1.y;
  const uint32_t w3 = q == 0 ? u0.w : q == 1 ? u1.x : q == 2 ? u1.y : u1.z;
  const uint32_t w4 = q == 0 ? u1.x : q == 1 ? u1.y : q == 2 ? u1.z : u1.w;
  return make_uint4(__funnelshift_r(w0, w1, sh), __funnelshift_r(w1, w2, sh), __funnelshift_r(w2, w3, sh),
                    __funnelshift_r(w3, w4, sh));
}

// Compare T[J.a + x] and T[J.b + x] for x in [off, end): 16 bytes per lane
// and step when the own side J.b + off is 16-byte aligned (block starts are
// multiples of 16 at the usual leaf lengths), the other side realigned from
// two aligned loads; bytes otherwise and for the ragged end.
__device__ __forceinline__ bool differs(const uint8_t* __restrict__ T, uint64_t n, bool aligned16, uint64_t a,
                                        uint64_t b, uint64_t off, uint64_t end, unsigned lane, unsigned L) {
  bool diff = false;
  uint64_t x = off;
  if (aligned16 && ((b + off) & 15) == 0) {
    const uint64_t full = off + ((end - off) & ~15ull);
    for (uint64_t y = off + 16ull * lane; y < full; y += 16ull * L) {
      const uint4 vb = *(const uint4*)(T + b + y);
      const uint64_t A = a + y, A0 = A & ~15ull;
      const uint32_t d = (uint32_t)(A & 15);
      const uint4 u0 = *(const uint4*)(T + A0);
      uint4 va;
      if (d == 0) {
        va = u0;
      } else if (A0 + 32 <= n) {
        va = unaligned16(u0, *(const uint4*)(T + A0 + 16), d);
      } else {  // the unit past the text's end is not read
        uint32_t v[4] = {0, 0, 0, 0};
        for (uint32_t t = 0; t < 16; t++) v[t >> 2] |= (uint32_t)T[A + t] << (8 * (t & 3));
        va = make_uint4(v[0], v[1], v[2], v[3]);
      }
      diff |= va.x != vb.x || va.y != vb.y || va.z != vb.z || va.w != vb.w;
    }
    x = full;
  }
  for (x += lane; x < end; x += L) diff |= T[a + x] != T[b + x];
  return diff;
}

// One group of L lanes (a power of two up to 32, about b/16 so that short
// jobs do not leave most of a warp idle) per (job, piece of 4 KiB).
__global__ void __launch_bounds__(256) k_verify(const uint8_t* __restrict__ T, uint64_t n,
                                                const Job* __restrict__ jobs, const LevelDev* ld,
                                                uint64_t ppj, unsigned int* mismatch, unsigned L) {
  const uint64_t total = ld->njobs * ppj;
  const unsigned lane = threadIdx.x & 31, grp = lane / L, gl = lane % L, gpw = 32 / L;
  const unsigned gmask = (L == 32 ? 0xFFFFFFFFu : ((1u << L) - 1u)) << (grp * L);
  const bool aligned16 = (((uintptr_t)T) & 15) == 0;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x / 32);
  // Warp-uniform loop: every lane reaches the ballot of every iteration.
  for (uint64_t base = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) / 32 * gpw; base < total;
       base += warps * gpw) {
    const uint64_t u = base + grp;
    bool diff = false, active = false;
    uint64_t jb = 0;
    if (u < total) {
      jb = u / ppj;
      const uint64_t piece = u - jb * ppj;
      const Job J = jobs[jb];
      const uint64_t off = piece * kPiece;
      if (off < J.len && *(volatile unsigned int*)&mismatch[jb] == 0) {
        active = true;
        const uint64_t end = off + kPiece < J.len ? off + kPiece : J.len;
        diff = differs(T, n, aligned16, J.a, J.b, off, end, gl, L);
      }
    }
    const unsigned bal = __ballot_sync(0xFFFFFFFFu, diff);
    if (active && gl == 0 && (bal & gmask)) atomicOr(&mismatch[jb], 1u);
  }
}

// 4c. Apply the pair verifications: a mismatch makes the pair a suspect key.
__global__ void k_pair_apply(Geo g, const uint64_t* __restrict__ job_of,
                             const unsigned int* __restrict__ mismatch, uint64_t* susp,
                             unsigned long long* exlo, LevelDev* ld, Status* status) {
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k + 1 < g.c;
       k += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t id = job_of[k];
    if (id == kNone || !mismatch[id]) continue;
    atomicAdd(&status->collisions, 1ull);
    const unsigned long long i = atomicAdd(&ld->nsusp, 1ull);
    susp[i] = k;
    exlo[i] = g.st[k];  // the key's own start is an occurrence
  }
}

// 4d. Exact leftmost occurrence of every suspect key: each window before
// the key's start whose fingerprint equals the key's is compared byte by
// byte.  `pair` selects whether the suspects are pairs (k, k+1) or blocks.
template <class M>
__global__ void __launch_bounds__(256) k_exact_scan(M m, Geo g, uint64_t cpb, int pair,
                                                   const uint64_t* __restrict__ fpB,
                                                   const uint64_t* __restrict__ susp,
                                                   unsigned long long* exlo, const LevelDev* ld) {
  const uint64_t ns = ld->nsusp;
  const uint64_t per = g.c * cpb;
  for (uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; w < ns * per;
       w += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i = w / per, rest = w - i * per;
    const uint64_t key = susp[i];
    const uint64_t ks = g.st[key];
    uint64_t klen = blen(g, key), kfp = fpB[key], BL;
    if (pair) {
      uint64_t l2 = blen(g, key + 1);
      kfp = m.add(m.mul(kfp, l2 == g.b ? g.Bb : g.Br), fpB[key + 1]);
      klen += l2;
      BL = l2 == g.b ? m.mul(g.Bb, g.Bb) : g.Bbr;
    } else {
      BL = klen == g.b ? g.Bb : g.Br;
    }
    const uint64_t k = rest / cpb, j = rest - k * cpb;
    const uint64_t s = g.st[k], len = blen(g, k);
    const uint64_t p0 = s + j * kScanQ;
    if (p0 >= s + len || p0 >= ks) continue;
    const uint64_t pend = (p0 + kScanQ < s + len) ? p0 + kScanQ : s + len;
    const uint64_t av = avail_end(g, k);
    if (p0 + klen > av) continue;
    uint64_t fp = window_fast(m, g.H, BL, p0, klen);
    for (uint64_t p = p0; p < pend && p < ks && p + klen <= av; p++) {
      if (p > p0) {
        uint64_t out = (uint64_t)g.T[p - 1] + 1, in = (uint64_t)g.T[p + klen - 1] + 1;
        fp = m.add(m.sub(m.mul(fp, g.B), m.mul(out, BL)), in);
      }
      if (fp != kfp) continue;
      bool eq = true;
      for (uint64_t x = 0; x < klen && eq; x++) eq = g.T[p + x] == g.T[ks + x];
      if (eq) min_pos(&exlo[i], p);
    }
  }
}

__global__ void k_pair_exact_apply(Geo g, const uint64_t* __restrict__ susp,
                                   const unsigned long long* __restrict__ exlo, uint8_t* pm,
                                   uint64_t* plo_k, const LevelDev* ld) {
  const uint64_t ns = ld->nsusp;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < ns;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t k = susp[i];
    plo_k[k] = exlo[i];
    pm[k] = exlo[i] == g.st[k];
  }
}

// 5. Marks: a block is marked when a pair it belongs to is leftmost, or when
// it belongs to no pair.  One warp covers one 32-bit word of the bit vector.
__global__ void k_mark(Geo g, const uint32_t* __restrict__ slotP, const uint8_t* __restrict__ pm,
                       uint32_t* __restrict__ mw, uint32_t* __restrict__ wpop) {
  const uint64_t words = (g.c + 31) / 32;
  for (uint64_t base = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) & ~31ull; base < words * 32;
       base += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t k = base + (threadIdx.x & 31);
    bool mk = false;
    if (k < g.c) {
      bool left = k > 0 && slotP[k - 1] != kNoSlot;
      bool right = k + 1 < g.c && slotP[k] != kNoSlot;
      mk = (left && pm[k - 1]) || (right && pm[k]) || (!left && !right);
    }
    uint32_t bits = __ballot_sync(0xFFFFFFFFu, mk);
    if ((threadIdx.x & 31) == 0) {
      mw[base / 32] = bits;
      wpop[base / 32] = __popc(bits);
    }
  }
}

__device__ __forceinline__ bool is_marked(const uint32_t* mw, uint64_t k) {
  return (mw[k >> 5] >> (k & 31)) & 1u;
}

// 6a. Block leftmost occurrences: unmarked blocks always (they become
// pointers), marked blocks too when pruning needs them.
__global__ void k_block_jobs(Geo g, const uint32_t* __restrict__ slotB,
                             const BSlot* __restrict__ bt, const uint32_t* __restrict__ mw,
                             int all, uint64_t* __restrict__ lo, Job* jobs, uint64_t* job_of,
                             LevelDev* ld, Status* status) {
  const unsigned lane = threadIdx.x & 31;
  for (uint64_t base = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) & ~31ull; base < g.c;
       base += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t k = base + lane;
    bool want = false;
    uint64_t p = 0, s = 0, len = 0;
    if (k < g.c) {
      job_of[k] = kNone;
      lo[k] = kNone;
      if (all || !is_marked(mw, k)) {
        s = g.st[k];
        len = blen(g, k);
        p = slotB[k] == kNoSlot ? ld->lo_tail : bt[slotB[k]].lo;
        lo[k] = p;
        if (p < s) want = true;
        else if (p > s) atomicExch(&status->error, 4ull);
      }
    }
    const uint64_t id = warp_claim(&ld->njobs, want);
    if (want) {
      jobs[id] = Job{p, s, len, k};
      job_of[k] = id;
    }
    const uint64_t vb = warp_sum(want ? 2 * len : 0);
    if (lane == 0 && vb) atomicAdd(&status->verify_bytes, (unsigned long long)vb);
  }
}

__global__ void k_block_apply(Geo g, const uint64_t* __restrict__ job_of,
                              const unsigned int* __restrict__ mismatch, uint64_t* susp,
                              unsigned long long* exlo, LevelDev* ld, Status* status) {
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < g.c;
       k += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t id = job_of[k];
    if (id == kNone || !mismatch[id]) continue;
    atomicAdd(&status->collisions, 1ull);
    const unsigned long long i = atomicAdd(&ld->nsusp, 1ull);
    susp[i] = k;
    exlo[i] = g.st[k];  // the key's own start is an occurrence
  }
}

__global__ void k_block_exact_apply(const uint64_t* __restrict__ susp,
                                    const unsigned long long* __restrict__ exlo, uint64_t* lo,
                                    const LevelDev* ld) {
  const uint64_t ns = ld->nsusp;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < ns;
       i += (uint64_t)gridDim.x * blockDim.x)
    lo[susp[i]] = exlo[i];
}

// 6b. Pointers of unmarked blocks: the block holding the leftmost occurrence
// (binary search over the sorted starts) and the offset into it.  The
// target, and its right neighbour when the occurrence crosses into it, must
// be marked; the occurrence must end before the block starts.
__global__ void k_pointers(Geo g, const uint32_t* __restrict__ mw, const uint64_t* __restrict__ lo,
                           uint32_t* __restrict__ ptr, uint64_t* __restrict__ off, Status* status) {
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < g.c;
       k += (uint64_t)gridDim.x * blockDim.x) {
    if (is_marked(mw, k)) {
      ptr[k] = 0;
      off[k] = 0;
      continue;
    }
    uint64_t p = lo[k], len = blen(g, k);
    uint64_t a = 0, z = g.c;  // first index with st > p
    while (a < z) {
      uint64_t mid = (a + z) / 2;
      if (g.st[mid] <= p) a = mid + 1;
      else z = mid;
    }
    bool ok = a > 0;
    uint64_t j = a - 1;
    if (ok) ok = p < g.st[j] + blen(g, j) && is_marked(mw, j) && p + len <= g.st[k];
    if (ok && p + len > g.st[j] + blen(g, j))
      ok = j + 1 < g.c && g.st[j + 1] == g.st[j] + blen(g, j) && is_marked(mw, j + 1);
    if (!ok) {
      atomicExch(&status->error, 5ull);
      continue;
    }
    ptr[k] = (uint32_t)j;
    off[k] = p - g.st[j];
  }
}

// 7. Children of marked blocks: the block with mark rank r puts its children
// at r*arity + i, each starting i*bn after it.
__global__ void k_children(Geo g, const uint32_t* __restrict__ mw, const uint32_t* __restrict__ mr,
                           uint32_t arity, uint64_t bn, uint64_t* __restrict__ next_st) {
  const uint64_t total = g.c * arity;
  for (uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; w < total;
       w += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t k = w / arity, i = w - k * arity;
    if (!is_marked(mw, k)) continue;
    uint64_t s = g.st[k] + i * bn;
    if (s >= g.st[k] + blen(g, k)) continue;
    uint64_t r = mr[k >> 5] + __popc(mw[k >> 5] & ((1u << (k & 31)) - 1u));
    next_st[r * arity + i] = s;
  }
}

// Size of the next level and the start of its last block.
__global__ void k_level_finish(Geo g, const uint32_t* __restrict__ mw, const uint32_t* __restrict__ mr,
                               uint32_t arity, uint64_t bn, Status* status) {
  const uint64_t words = (g.c + 31) / 32;
  uint64_t nmarked = mr[words];
  uint64_t last = kNone;
  for (uint64_t w = words; w-- > 0;) {
    if (mw[w]) {
      last = w * 32 + 31 - __clz(mw[w]);
      break;
    }
  }
  if (last == kNone || arity == 0) {
    status->next_c = 0;
    status->last_start = 0;
    return;
  }
  uint64_t len = blen(g, last), nch = (len + bn - 1) / bn;
  status->next_c = (nmarked - 1) * arity + nch;
  status->last_start = g.st[last] + (nch - 1) * bn;
}

__global__ void k_level_start(uint64_t c, uint64_t b, uint64_t* st) {
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < c;
       k += (uint64_t)gridDim.x * blockDim.x)
    st[k] = k * b;
}

struct InitArgs {
  BSlot* bt;
  uint64_t bcap;
  PSlot* pt;
  uint64_t pcap;
  unsigned int* mismatch;
  uint64_t c;
  AnchorSet* atab;
  uint64_t acap;
  uint32_t* bitmap;
  uint64_t bwords;
  uint32_t* secbits;
  unsigned long long* qn;
  LevelDev* ld;
};

// All per-level tables and flags in one launch: keys and minima to "empty",
// counters and filters to zero.
__global__ void k_level_init(InitArgs a) {
  uint64_t top = a.bcap > a.pcap ? a.bcap : a.pcap;
  if (a.c > top) top = a.c;
  if (a.acap > top) top = a.acap;
  if (a.bwords > top) top = a.bwords;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < top;
       i += (uint64_t)gridDim.x * blockDim.x) {
    if (i < a.bcap) a.bt[i] = BSlot{kNone, kNone, 0, 0};
    if (i < a.pcap) a.pt[i] = PSlot{kNone, kNone};
    if (i < a.c) a.mismatch[i] = 0;
    if (a.atab && i < a.acap) {
      a.atab[i].gram = kEmptyGram;
      a.atab[i].far = kNoFar;
      a.atab[i].more = kNoFar;
      a.atab[i].offs = 0;
      a.atab[i].maxst = 0;
    }
    if (a.bitmap && i < a.bwords) a.bitmap[i] = 0;
    if (a.secbits && i < kSecBits / 32) a.secbits[i] = 0;
    if (i == 0) {
      LevelDev d;
      d.fp_tail = kNone;
      d.lo_tail = kNone;
      d.lo_tailpair = kNone;
      d.pretail_slot = 0xFFFFFFFFu;
      d.npairs = 0;
      d.njobs = 0;
      d.nsusp = 0;
      d.anchorless = 0;
      d.tail_anchorless = 0;
      d.tail_gram = 0xFFFFFFFFu;
      d.tail_a = 0xFFFFFFFFu;
      d.far_end = 0;
      d.qover = 0;
      d.nfar = 0;
      d.cands = 0;
      d.hits = 0;
      *a.ld = d;
      if (a.qn) *a.qn = 0;
    }
  }
}

// Between the pair and the block verification: empty the job list again.
__global__ void k_reset_jobs(unsigned int* mismatch, uint64_t c, LevelDev* ld) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < c;
       i += (uint64_t)gridDim.x * blockDim.x) {
    mismatch[i] = 0;
    if (i == 0) {
      ld->njobs = 0;
      ld->nsusp = 0;
    }
  }
}

// Gram length 16 (at most half a block): long enough that a gram is rare
// even over small or skewed alphabets, so few keys share an anchor gram;
// anchor range W <= 64; selection density 2^-sbits chosen so that
// W / 2^sbits >= 8 (a window without an anchor is then rare).
// Gram length w = 16 (half the block when shorter), near range W <= 64.
// Each gram is selected with probability 2^-sbits, so a key has no selected
// gram among its first npos positions with probability (1 - 2^-sbits)^npos;
// sbits is the largest value in 0..3 that leaves well under one such key per
// level (c keys), since those keys are found by a per-position filter.
GramP choose_gram(uint64_t b, uint64_t r, uint64_t c) {
  uint32_t w = 16;
  if (w > b / 2) w = (uint32_t)(b / 2 > 0 ? b / 2 : 1);
  GramP gp;
  gp.w = w;
  gp.W = (uint32_t)(b - w + 1 < kAnchorWmax ? b - w + 1 : kAnchorWmax);
  const double npos = (double)(b - w + 1 < kFarMax ? b - w + 1 : kFarMax);
  gp.sbits = 0;
  for (uint32_t sb = 3; sb >= 1; sb--) {
    if ((double)c * std::pow(1.0 - std::ldexp(1.0, -(int)sb), npos) <= 0.02) {
      gp.sbits = sb;
      break;
    }
  }
  gp.sel_max = gp.sbits ? (1u << (32 - gp.sbits)) - 1u : 0xFFFFFFFFu;
  gp.Wr = (r && r >= w) ? (uint32_t)(r - w + 1 < kAnchorWmax ? r - w + 1 : kAnchorWmax) : 0;
  gp.fbits = 12;
  gp.rb = 0x01000193u;
  uint32_t rw = 1;
  for (uint32_t i = 0; i < w; i++) rw *= gp.rb;
  gp.rw = rw;
  return gp;
}

// Streaming multiprocessors of the current device (cached per device).
unsigned sm_count() {
  static std::atomic<unsigned> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  unsigned v = cache[dev].load(std::memory_order_relaxed);
  if (v) return v;
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
  cache[dev].store((unsigned)n, std::memory_order_relaxed);
  return (unsigned)n;
}

// CTAs of a kernel that fit on one SM at once (at least 1).
template <class F>
unsigned resident_ctas(F* fn, int threads, size_t smem) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, smem) != cudaSuccess || n < 1) {
    cudaGetLastError();
    n = 1;
  }
  return (unsigned)n;
}

// Opt a kernel in to more than 48 KiB of dynamic shared memory, once per
// device (the attribute is a property of the function on each device; the
// template parameter gives every kernel its own flags).
template <auto FN>
int allow_scan_smem(int bytes) {
  static std::atomic<uint64_t> done{0};
  int dev = 0;
  BT_CUDA(cudaGetDevice(&dev));
  const uint64_t bit = 1ull << (dev & 63);
  if (done.load(std::memory_order_acquire) & bit) return BT_OK;
  BT_CUDA(cudaFuncSetAttribute(FN, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  done.fetch_or(bit, std::memory_order_acq_rel);
  return BT_OK;
}

uint64_t pow2_at_least(uint64_t x) {
  uint64_t p = 16;
  while (p < x) p <<= 1;
  return p;
}

struct LevelWork {
  uint64_t *fpB, *plo_k, *job_of, *susp;
  BSlot* bt;
  PSlot* pt;
  uint32_t *slotB, *slotP, *wpop;
  unsigned long long* exlo;
  uint8_t* pm;
  Job* jobs;
  unsigned int* mismatch;
  LevelDev* ld;
};

// Resolve suspects by the exact scan; `pair` selects the key kind.
template <class M>
int exact_pass(const M& m, const Geo& g, uint64_t cpb, int pair, LevelWork& W, cudaStream_t s) {
  const unsigned T = 256;
  BT_LAUNCH(k_exact_scan<M><<<grid_for(g.c * cpb, T), T, 0, s>>>(m, g, cpb, pair, W.fpB, W.susp, W.exlo, W.ld));
  BT_CUDA(cudaGetLastError());
  return BT_OK;
}

// The sort-based pass of a level: sorted windows of length b give the block
// minima, sorted windows of length 2b the pair minima, a dense pass the two
// tail keys.  With parts > 1 the windows are taken in that many parts
// (domain decomposition, above).
template <class M>
int sort_minima(const M& m, const Geo& g, LevelWork& W, uint64_t c, uint64_t b, uint64_t r, uint32_t parts,
                cudaStream_t s) {
  const uint64_t npos = c * b;
  const uint32_t bshift = (b & (b - 1)) == 0 ? (uint32_t)__builtin_ctzll(b) : 0xFFu;
  const unsigned T = 256;
  Scratch sc(s);
  if (parts <= 1) {
    if (npos >= (1ull << 32)) return BT_EINVAL;
    uint64_t *keys, *tk;
    uint32_t *vals, *tv, *scr;
    BT_TRY(sc.alloc(&keys, npos));
    BT_TRY(sc.alloc(&tk, npos));
    BT_TRY(sc.alloc(&vals, npos));
    BT_TRY(sc.alloc(&tv, npos));
    BT_TRY(sc.alloc(&scr, radix_sort_scratch_words(npos)));
    for (int pair = 0; pair < 2; pair++) {
      const uint64_t L = pair ? 2 * b : b;
      const uint64_t BL = pair ? m.mul(g.Bb, g.Bb) : g.Bb;
      BT_LAUNCH(k_sort_windows<M><<<grid_for(npos, T), T, 0, s>>>(m, g, L, BL, bshift, keys, vals));
      BT_TRY(radix_sort_u64_u32(keys, vals, tk, tv, npos, 64, scr, s));
      BT_LAUNCH(k_sort_minima<M><<<grid_for(c, T), T, 0, s>>>(m, g, pair, W.fpB, W.slotB, W.slotP, W.bt, W.pt,
                                                              keys, vals, npos));
    }
  } else {
    if (g.n >= (1ull << 32)) return BT_EINVAL;
    const uint64_t part = (npos + parts - 1) / parts;  // windows per part
    uint64_t kbits_n = 4096;
    while (kbits_n < 32 * c) kbits_n <<= 1;
    const uint64_t big = std::max<uint64_t>(part, c);
    uint64_t *skeys, *keys, *ck, *tk;
    uint32_t *sv, *vals, *cv, *tv, *flag, *offs, *scr, *sagg, *kbits;
    unsigned long long* d_count;
    BT_TRY(sc.alloc(&skeys, c));
    BT_TRY(sc.alloc(&sv, c));
    BT_TRY(sc.alloc(&kbits, kbits_n / 32));
    BT_TRY(sc.alloc(&keys, part));
    BT_TRY(sc.alloc(&vals, part));
    BT_TRY(sc.alloc(&flag, part));
    BT_TRY(sc.alloc(&offs, part + 1));  // the scan also writes the total at [n]
    BT_TRY(sc.alloc(&ck, part));
    BT_TRY(sc.alloc(&cv, part));
    BT_TRY(sc.alloc(&tk, big));
    BT_TRY(sc.alloc(&tv, big));
    BT_TRY(sc.alloc(&scr, radix_sort_scratch_words(big)));
    BT_TRY(sc.alloc(&sagg, scan_scratch_words(part)));
    BT_TRY(sc.alloc(&d_count, 1));
    // The kept tuples: a list that grows by doubling (at most one tuple per
    // key fingerprint and part), so that it holds what the parts keep.
    struct Grown {
      cudaStream_t s;
      void* p = nullptr;
      ~Grown() {
        if (p) cudaFreeAsync(p, s);
      }
    };
    Grown gk{s}, gv{s};
    uint64_t kcap = 0;
    auto reserve_kept = [&](uint64_t need, uint64_t kept) -> int {
      if (need <= kcap) return BT_OK;
      const uint64_t cap = std::max<uint64_t>(need, 2 * kcap);
      void *nk = nullptr, *nv = nullptr;
      if (!alloc_allowed(cap * sizeof(uint64_t))) return BT_ENOMEM;
      cudaError_t e1 = cudaMallocAsync(&nk, cap * sizeof(uint64_t), s);
      cudaError_t e2 = e1 == cudaSuccess ? cudaMallocAsync(&nv, cap * sizeof(uint32_t), s) : e1;
      if (e2 != cudaSuccess) {
        if (nk) cudaFreeAsync(nk, s);
        cudaGetLastError();
        return e2 == cudaErrorMemoryAllocation ? BT_ENOMEM : BT_ECUDA;
      }
      if (kept) {
        BT_CUDA(cudaMemcpyAsync(nk, gk.p, kept * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
        BT_CUDA(cudaMemcpyAsync(nv, gv.p, kept * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
      }
      if (gk.p) cudaFreeAsync(gk.p, s);
      if (gv.p) cudaFreeAsync(gv.p, s);
      gk.p = nk;
      gv.p = nv;
      kcap = cap;
      return BT_OK;
    };
    unsigned long long h_count = 0;
    auto read_count = [&](uint64_t* out) -> int {
      BT_CUDA(cudaMemcpyAsync(&h_count, d_count, sizeof(h_count), cudaMemcpyDeviceToHost, s));
      BT_CUDA(cudaStreamSynchronize(s));
      *out = h_count;
      return BT_OK;
    };
    for (int pair = 0; pair < 2; pair++) {
      const uint64_t L = pair ? 2 * b : b;
      const uint64_t BL = pair ? m.mul(g.Bb, g.Bb) : g.Bb;
      // The keys of this length: a bit map and the sorted list.
      BT_CUDA(cudaMemsetAsync(kbits, 0, kbits_n / 8, s));
      BT_LAUNCH(k_key_list<M><<<grid_for(c, T), T, 0, s>>>(m, g, pair, W.fpB, W.slotB, W.slotP, skeys, kbits,
                                                           kbits_n - 1));
      BT_TRY(radix_sort_u64_u32(skeys, sv, tk, tv, c, 64, scr, s));
      uint64_t kept = 0;
      for (uint64_t w0 = 0; w0 < npos; w0 += part) {
        const uint64_t nw = std::min(part, npos - w0);
        BT_LAUNCH(k_part_windows<M><<<grid_for(nw, T), T, 0, s>>>(m, g, L, BL, bshift, w0, nw, kbits, kbits_n - 1,
                                                                  skeys, c, keys, vals, flag));
        BT_TRY(scan_u32(flag, offs, nw, s, sagg));
        BT_LAUNCH(k_compact_tuples<<<grid_for(nw, T), T, 0, s>>>(keys, vals, flag, offs, nw, ck, cv, d_count));
        uint64_t nm = 0;
        BT_TRY(read_count(&nm));
        if (nm == 0) continue;
        BT_TRY(radix_sort_u64_u32(ck, cv, tk, tv, nm, 64, scr, s));
        BT_LAUNCH(k_first_of_key<<<grid_for(nm, T), T, 0, s>>>(ck, nm, flag));
        BT_TRY(scan_u32(flag, offs, nm, s, sagg));
        // The part keeps at most one tuple per key fingerprint.
        BT_TRY(reserve_kept(kept + std::min<uint64_t>(nm, c), kept));
        BT_LAUNCH(k_compact_tuples<<<grid_for(nm, T), T, 0, s>>>(ck, cv, flag, offs, nm, (uint64_t*)gk.p + kept,
                                                                 (uint32_t*)gv.p + kept, d_count));
        uint64_t nu = 0;
        BT_TRY(read_count(&nu));
        kept += nu;
      }
      if (kept) {
        uint64_t* kk = (uint64_t*)gk.p;
        uint32_t* kv = (uint32_t*)gv.p;
        if (kept <= big) {
          BT_TRY(radix_sort_u64_u32(kk, kv, tk, tv, kept, 64, scr, s));
        } else {
          Scratch sc2(s);
          uint64_t* tkk;
          uint32_t *tkv, *scr2;
          BT_TRY(sc2.alloc(&tkk, kept));
          BT_TRY(sc2.alloc(&tkv, kept));
          BT_TRY(sc2.alloc(&scr2, radix_sort_scratch_words(kept)));
          BT_TRY(radix_sort_u64_u32(kk, kv, tkk, tkv, kept, 64, scr2, s));
        }
        BT_LAUNCH(k_sort_minima<M><<<grid_for(c, T), T, 0, s>>>(m, g, pair, W.fpB, W.slotB, W.slotP, W.bt, W.pt,
                                                                kk, kv, kept));
      }
    }
  }
  if (r) BT_LAUNCH(k_sort_tail<M><<<grid_for(npos, T), T, 0, s>>>(m, g, bshift, W.fpB, W.slotP, W.ld));
  BT_CUDA(cudaGetLastError());
  return BT_OK;
}

template <class M>
int level_pass(const M& m, BuildCtx& ctx, uint32_t l, uint64_t last_start) {
  bt_tree* t = ctx.t;
  Level& v = t->lv[l];
  cudaStream_t s = ctx.s;
  const uint64_t c = v.c, b = v.b, n = t->n;
  const bool last_level = l + 1 == t->L;
  const uint64_t bn = last_level ? 0 : t->lv[l + 1].b;
  const uint64_t len_last = n - last_start;
  const uint64_t r = len_last < b ? len_last : 0;

  Geo g;
  g.T = ctx.T;
  g.n = n;
  g.H = ctx.H;
  g.B = t->B;
  g.Bb = pow_mod(m, t->B, b);
  g.Br = r ? pow_mod(m, t->B, r) : 0;
  g.Bbr = r ? pow_mod(m, t->B, b + r) : 0;
  g.c = c;
  g.b = b;
  g.r = r;
  g.st = v.st;
  const uint64_t cpb = (b + kScanQ - 1) / kScanQ;
  const uint64_t bcap = pow2_at_least(2 * c), pcap = pow2_at_least(2 * c);

  const unsigned T = 256;
  const unsigned gc = grid_for(c, T);
  const uint64_t words = (c + 31) / 32;
  const bool anchored = !ctx.dense_scan && !ctx.sort_scan;
  const GramP gp = choose_gram(b, r, c);
  const uint64_t acap = anchored ? pow2_at_least(2 * (c + 2)) : 0;
  GramP gq = gp;
  uint64_t bwords = 0;
  if (anchored) {
    uint64_t fb = pow2_at_least(16 * (c + 2));
    uint32_t fbits = 0;
    while ((1ull << fbits) < fb) fbits++;
    if (fbits < 12) fbits = 12;
    if (fbits + gp.sbits > 32) fbits = 32 - gp.sbits;
    gq.fbits = fbits;
    bwords = (1ull << fbits) / 32;
  }
  // Anchored scan launch: one wave of resident CTAs (shared memory allows 3
  // per SM, 2 with the bitmap in shared memory); threads stride over chunks.
  const uint64_t cpa = (b + kAnchorQ - 1) / kAnchorQ;
  const uint32_t bm_smem = bwords <= kSmemBitmapWords ? (uint32_t)bwords : 0;
  const unsigned scan_grid = anchored ? grid_for(c * cpa, kScanThreads, sm_count() * (bm_smem ? 2u : 3u)) : 0;
  // Queues of gram hits and of proposed windows, one segment per scan CTA:
  // one entry per two covered bytes, at most 64 Mi, is plenty for most texts;
  // if a segment overflows, a second scan tests windows in place.  Highly
  // repetitive texts (copies of a genome) hit a key's gram at most selected
  // grams of their lowest levels and propose a window every few bytes, and
  // the rerun would cost more than the build.  So the gram hits get room for
  // 1.25 times the level's expected selected grams (cov / 2^sbits), and the
  // proposed windows for up to 16 times the previous level's, at most a
  // quarter of the covered bytes.
  const uint64_t cov_l = (c - 1) * b + (len_last < b ? len_last : b);
  uint64_t qcap = cov_l / 2 + 4096;
  if (qcap > (64ull << 20)) qcap = 64ull << 20;
  uint64_t hcap = qcap, ccap = qcap;
  const uint64_t sel = (cov_l >> gp.sbits) + (cov_l >> (gp.sbits + 2)) + 4096;
  if (sel > hcap) hcap = std::min<uint64_t>(sel, cov_l + 4096);
  const uint64_t grow = std::min<uint64_t>(cov_l / 4 + 4096, 16 * ctx.prev_cands + 4096);
  if (grow > ccap) ccap = grow;
  if (ctx.tiny_queue) hcap = ccap = 64;
  const uint32_t seg = anchored ? (uint32_t)(hcap / scan_grid) : 0;
  const uint32_t cseg = anchored ? (uint32_t)(ccap / scan_grid) : 0;

  // Scratch: carved from the build's arena (a dry carving sizes it).
  Arena& A = ctx.arena;
  LevelWork W;
  AnchorSet* atab = nullptr;
  FarNode* fnode = nullptr;
  const uint32_t fcap = (uint32_t)(c / 16 + 1024);
  uint32_t *bitmap = nullptr, *secbits = nullptr, *sagg = nullptr;
  Hit* q = nullptr;
  uint32_t* segn = nullptr;
  Cand* cq = nullptr;
  uint32_t* csegn = nullptr;
  unsigned long long* qn = nullptr;
  uint32_t* aidx = nullptr;
  auto carve = [&]() {
    W.fpB = A.take<uint64_t>(c);
    W.slotB = A.take<uint32_t>(c);
    W.slotP = A.take<uint32_t>(c);
    W.pm = A.take<uint8_t>(c);
    W.plo_k = A.take<uint64_t>(c);
    W.job_of = A.take<uint64_t>(c);
    W.susp = A.take<uint64_t>(c);
    W.exlo = A.take<unsigned long long>(c);
    W.jobs = A.take<Job>(c);
    W.mismatch = A.take<unsigned int>(c);
    W.bt = A.take<BSlot>(bcap);
    W.pt = A.take<PSlot>(pcap);
    W.ld = A.take<LevelDev>(1);
    W.wpop = A.take<uint32_t>(words);
    sagg = A.take<uint32_t>(scan_scratch_words(words));
    if (anchored) {
      atab = A.take<AnchorSet>(acap);
      fnode = A.take<FarNode>(fcap);
      bitmap = A.take<uint32_t>(bwords);
      secbits = A.take<uint32_t>(kSecBits / 32);
      q = A.take<Hit>((uint64_t)seg * scan_grid);
      segn = A.take<uint32_t>(scan_grid);
      cq = A.take<Cand>((uint64_t)cseg * scan_grid);
      csegn = A.take<uint32_t>(scan_grid);
      qn = A.take<unsigned long long>(1);
      aidx = A.take<uint32_t>(c);
    }
  };
  A.begin_dry();
  carve();
  BT_TRY(A.reserve());
  carve();

  // Persistent level arrays: one allocation, owned by the level.
  {
    auto al = [](uint64_t x) { return (x + 255) & ~255ull; };
    const uint64_t o_mw = 0, o_mr = o_mw + al(words * 4 + 4), o_ptr = o_mr + al((words + 1) * 4),
                   o_off = o_ptr + al(c * 4 + 4), o_lo = o_off + al(c * 8 + 8), total = o_lo + al(c * 8 + 8);
    char* mem;
    BT_CUDA(cudaMallocAsync((void**)&mem, total, s));
    v.owned.push_back(mem);
    v.mw = (uint32_t*)(mem + o_mw);
    v.mr = (uint32_t*)(mem + o_mr);
    v.ptr = (uint32_t*)(mem + o_ptr);
    v.off = (uint64_t*)(mem + o_off);
    v.lo = (uint64_t*)(mem + o_lo);
  }

  InitArgs ia{W.bt, bcap, W.pt, pcap, W.mismatch, c,
              atab, acap, bitmap, bwords, secbits, qn, W.ld};
  {
    uint64_t top = bcap > acap ? bcap : acap;
    if (bwords > top) top = bwords;
    BT_LAUNCH(k_level_init<<<grid_for(top, T), T, 0, s>>>(ia));
  }
  BT_LAUNCH(k_block_fp<M><<<gc, T, 0, s>>>(m, g, W.fpB, W.slotB, W.bt, bcap - 1, W.ld, ctx.st));
  BT_LAUNCH(k_pair_insert<<<gc, T, 0, s>>>(g, W.slotB, W.slotP, W.pt, pcap - 1, W.bt, W.ld,
                                           ctx.st));
  if (ctx.sort_scan) {
    ProfScope ps("window_scan", s, cov_l);
    BT_TRY(sort_minima(m, g, W, c, b, r, ctx.partitions, s));
  } else if (!anchored) {
    ProfScope ps("window_scan", s, cov_l);
    BT_LAUNCH(k_scan<M><<<grid_for(c * cpb, T), T, 0, s>>>(m, g, cpb, W.bt, bcap - 1, W.pt, pcap - 1,
                                                            W.ld, 0));
  } else {
    BT_LAUNCH(k_anchor_keys<<<gc, T, 0, s>>>(g, gq, W.slotB, atab, (uint32_t)(acap - 1), fnode, fcap, bitmap, secbits,
                                             aidx, W.ld, ctx.st));
    ScanCtx<M> C{m, g, W.bt, bcap - 1, W.pt, pcap - 1, W.ld, 0, 0,
                 q, segn, seg, qn, cq, csegn, cseg, ctx.st, fnode, W.slotB};
    const size_t smem_base = ((size_t)kSecBits / 32 + (size_t)kRing * kScanThreads +
                              (size_t)kScanThreads * kSlotWords) * 4;
    const size_t smem = smem_base + (size_t)bm_smem * 4;
    const int smem_max = (int)(smem_base + (size_t)kSmemBitmapWords * 4);
    int rc_a = allow_scan_smem<k_scan_anchor<M, false>>(smem_max);
    if (rc_a == BT_OK) rc_a = allow_scan_smem<k_scan_anchor<M, true>>(smem_max);
    if (rc_a != BT_OK) return rc_a;
    ProfScope ps("window_scan", s, cov_l);
    // The selected-gram list serves levels with the default selection whose
    // chunks are the list's chunks; k_scan_anchor then runs only when the
    // level has keys without an anchor.
    const bool use_list = ctx.gl_chunk && gq.w == 16 && gq.sbits == kGlSbits && b % kAnchorQ == 0;
    // Every block present: blocks k b .. (k+1) b (the level covers the text).
    const bool all_present = c == (n + b - 1) / b;
    if (use_list && all_present)
      BT_LAUNCH(k_scan_stream<M><<<scan_grid, kScanThreads, (size_t)bm_smem * 4, s>>>(
          C, gq, ctx.gl_total, (b & (b - 1)) == 0 ? (uint32_t)__builtin_ctzll(b) : 0u, bitmap, bm_smem,
          ctx.gl_mx, ctx.gl_x));
    else if (use_list)
      BT_LAUNCH(k_scan_list<M><<<scan_grid, kScanThreads, (size_t)bm_smem * 4, s>>>(
          C, gq, cpa, bitmap, bm_smem, ctx.gl_chunk, ctx.gl_mx, ctx.gl_x));
    BT_LAUNCH(k_scan_anchor<M, false><<<scan_grid, kScanThreads, smem, s>>>(
        C, gq, cpa, atab, (uint32_t)(acap - 1), bitmap, bm_smem, secbits, use_list ? 1 : 0));
    if (ctx.two_phase) {
      // Two phases: the hits in the first 1/16 of the text, then the rest
      // against the bounds the first phase tightened.
      BT_LAUNCH(k_hits<M><<<scan_grid, 512, 0, s>>>(C, atab, (uint32_t)(acap - 1), 1u));
      BT_LAUNCH(k_candidates<M><<<scan_grid, 256, 0, s>>>(C));
      for (int step = 0; step < 2; step++)
        BT_LAUNCH(k_anchor_bound<<<gc, T, 0, s>>>(g, aidx, W.slotB, W.slotP, W.bt, W.pt, atab, W.ld, step));
      BT_LAUNCH(k_hits<M><<<scan_grid, 512, 0, s>>>(C, atab, (uint32_t)(acap - 1), 2u));
    } else {
      BT_LAUNCH(k_hits<M><<<scan_grid, 512, 0, s>>>(C, atab, (uint32_t)(acap - 1), 0u));
    }
    BT_LAUNCH(k_candidates<M><<<scan_grid, 256, 0, s>>>(C));
    // Only when the queue overflowed: the scan again, testing windows inline.
    BT_LAUNCH(k_scan_anchor<M, true><<<scan_grid, kScanThreads, smem, s>>>(
        C, gq, cpa, atab, (uint32_t)(acap - 1), bitmap, bm_smem, secbits, 0));
    if (r)
      BT_LAUNCH(k_scan<M><<<grid_for(c * cpb, T), T, 0, s>>>(m, g, cpb, W.bt, bcap - 1, W.pt, pcap - 1,
                                                              W.ld, 1));
  }
  BT_CUDA(cudaGetLastError());

  // Pairs: verify, resolve collisions exactly, mark.
  const uint64_t ppj_pair = (2 * b + kPiece - 1) / kPiece;
  BT_LAUNCH(k_pair_jobs<<<gc, T, 0, s>>>(g, W.slotP, W.pt, W.plo_k, W.pm, W.jobs, W.job_of, W.ld, ctx.st));
  const unsigned vl = b >= 512 ? 32u : b >= 256 ? 16u : b >= 128 ? 8u : b >= 64 ? 4u : 2u;  // lanes per job
  BT_LAUNCH(k_verify<<<grid_for(c * ppj_pair * vl, T), T, 0, s>>>(ctx.T, n, W.jobs, W.ld, ppj_pair, W.mismatch,
                                                                  vl));
  BT_LAUNCH(k_pair_apply<<<gc, T, 0, s>>>(g, W.job_of, W.mismatch, W.susp, W.exlo, W.ld, ctx.st));
  BT_TRY(exact_pass(m, g, cpb, 1, W, s));
  BT_LAUNCH(k_pair_exact_apply<<<gc, T, 0, s>>>(g, W.susp, W.exlo, W.pm, W.plo_k, W.ld));
  BT_LAUNCH(k_mark<<<grid_for(words * 32, T), T, 0, s>>>(g, W.slotP, W.pm, v.mw, W.wpop));
  BT_CUDA(cudaGetLastError());
  BT_TRY(scan_u32(W.wpop, v.mr, words, s, sagg));

  // Blocks: leftmost occurrences, verified; pointers.
  BT_LAUNCH(k_reset_jobs<<<gc, T, 0, s>>>(W.mismatch, c, W.ld));
  const uint64_t ppj_blk = (b + kPiece - 1) / kPiece;
  BT_LAUNCH(k_block_jobs<<<gc, T, 0, s>>>(g, W.slotB, W.bt, v.mw, t->prune, v.lo, W.jobs, W.job_of, W.ld,
                                ctx.st));
  BT_LAUNCH(k_verify<<<grid_for(c * ppj_blk * vl, T), T, 0, s>>>(ctx.T, n, W.jobs, W.ld, ppj_blk, W.mismatch,
                                                                 vl));
  BT_LAUNCH(k_block_apply<<<gc, T, 0, s>>>(g, W.job_of, W.mismatch, W.susp, W.exlo, W.ld, ctx.st));
  BT_TRY(exact_pass(m, g, cpb, 0, W, s));
  BT_LAUNCH(k_block_exact_apply<<<gc, T, 0, s>>>(W.susp, W.exlo, v.lo, W.ld));
  BT_LAUNCH(k_pointers<<<gc, T, 0, s>>>(g, v.mw, v.lo, v.ptr, v.off, ctx.st));
  BT_CUDA(cudaGetLastError());

  // Statistics of the level.
  LevelDev ldh;
  BT_CUDA(cudaMemcpyAsync(&ldh, W.ld, sizeof(LevelDev), cudaMemcpyDeviceToHost, s));
  uint32_t nmarked = 0;
  BT_CUDA(cudaMemcpyAsync(&nmarked, v.mr + words, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));

  if (!last_level) {
    const Level& w = t->lv[l + 1];
    v.arity = (uint32_t)(b / w.b);
    BT_LAUNCH(k_level_finish<<<1, 1, 0, s>>>(g, v.mw, v.mr, v.arity, bn, ctx.st));
    BT_TRY(sync_status(ctx));
    Level& nx = t->lv[l + 1];
    nx.c = ctx.st_host->next_c;
    if (nx.c == 0) return BT_EINTERNAL;
    BT_CUDA(cudaMallocAsync(&nx.st, nx.c * sizeof(uint64_t), s));
    nx.owned.push_back(nx.st);
    BT_LAUNCH(k_children<<<grid_for(c * v.arity, T), T, 0, s>>>(g, v.mw, v.mr, v.arity, bn, nx.st));
    BT_CUDA(cudaGetLastError());
  } else {
    v.arity = 0;
    BT_TRY(sync_status(ctx));
  }
  v.nmarked = nmarked;
  v.stats[BT_ST_NBLOCKS] = c;
  v.stats[BT_ST_B] = b;
  v.stats[BT_ST_COV] = (c - 1) * b + (n - last_start < b ? n - last_start : b);
  v.stats[BT_ST_NMARKED] = nmarked;
  v.stats[BT_ST_NPAIRS] = ldh.npairs;
  v.stats[BT_ST_VERIFY_BYTES] = ctx.st_host->verify_bytes - ctx.verify_bytes;
  v.stats[BT_ST_COLLISIONS] = ctx.st_host->collisions - ctx.collisions;
  v.stats[BT_ST_CANDIDATES] = ldh.cands;
  ctx.prev_cands = ldh.cands;
  v.stats[BT_ST_HITS] = ldh.hits;
  ctx.verify_bytes = ctx.st_host->verify_bytes;
  ctx.collisions = ctx.st_host->collisions;
  if (ctx.st_host->error) {
    if (getenv("BT_VERBOSE"))
      fprintf(stderr, "bt: level %u (b=%llu, c=%llu): device check %llu failed\n", l,
              (unsigned long long)b, (unsigned long long)c, (unsigned long long)ctx.st_host->error);
    return BT_EINTERNAL;
  }
  return BT_OK;
}

template <class M>
int all_levels(const M& m, BuildCtx& ctx) {
  bt_tree* t = ctx.t;
  Level& r = t->lv[0];
  r.c = (t->n + r.b - 1) / r.b;
  BT_CUDA(cudaMallocAsync(&r.st, r.c * sizeof(uint64_t), ctx.s));
  r.owned.push_back(r.st);
  BT_LAUNCH(k_level_start<<<grid_for(r.c, 256), 256, 0, ctx.s>>>(r.c, r.b, r.st));
  uint64_t last_start = (r.c - 1) * r.b;
  const bool trace = getenv("BT_TRACE") != nullptr;
  // The selected-gram list pays off when several levels cover large texts.
  struct ListMem {
    cudaStream_t s;
    std::vector<void*> p;
    ~ListMem() {
      for (void* q : p) cudaFreeAsync(q, s);
    }
  } lm{ctx.s, {}};
  if (!ctx.dense_scan && t->n >= 16 && (t->n >= kGlMinText || ctx.force_list)) {
    const uint64_t n = t->n, nchunks = (n - 15 + kAnchorQ - 1) / kAnchorQ;
    uint32_t* chunk;
    BT_CUDA(cudaMallocAsync((void**)&chunk, (nchunks + 1) * sizeof(uint32_t), ctx.s));
    lm.p.push_back(chunk);
    uint32_t *agg, *cnt;
    BT_CUDA(cudaMallocAsync((void**)&agg, scan_scratch_words(nchunks) * sizeof(uint32_t), ctx.s));
    lm.p.push_back(agg);
    BT_CUDA(cudaMallocAsync((void**)&cnt, nchunks * sizeof(uint32_t), ctx.s));
    lm.p.push_back(cnt);
    const uint32_t rb = 0x01000193u;
    uint32_t rw = 1;
    for (int i = 0; i < 16; i++) rw *= rb;
    const uint32_t sel_max = (1u << (32 - kGlSbits)) - 1u;
    const unsigned grid = grid_for(nchunks, 256);
    {
      ProfScope ps("gram_list", ctx.s, n);
      BT_LAUNCH(k_gl_pass<false><<<grid, 256, 0, ctx.s>>>(ctx.T, n, nchunks, rb, rw, sel_max, cnt, nullptr,
                                                          nullptr));
      BT_TRY(scan_u32(cnt, chunk, nchunks, ctx.s, agg));
      uint32_t total = 0;
      BT_CUDA(cudaMemcpyAsync(&total, chunk + nchunks, sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx.s));
      BT_CUDA(cudaStreamSynchronize(ctx.s));
      uint32_t *mx, *xs;
      BT_CUDA(cudaMallocAsync((void**)&mx, (uint64_t)(total ? total : 1) * sizeof(uint32_t), ctx.s));
      lm.p.push_back(mx);
      BT_CUDA(cudaMallocAsync((void**)&xs, (uint64_t)(total ? total : 1) * sizeof(uint32_t), ctx.s));
      lm.p.push_back(xs);
      BT_LAUNCH(k_gl_pass<true><<<grid, 256, 0, ctx.s>>>(ctx.T, n, nchunks, rb, rw, sel_max, chunk, mx, xs));
      ctx.gl_chunk = chunk;
      ctx.gl_mx = mx;
      ctx.gl_x = xs;
      ctx.gl_total = total;
    }
  }
  for (uint32_t l = 0; l < t->L; l++) {
    auto h0 = std::chrono::steady_clock::now();
    BT_TRY(level_pass(m, ctx, l, last_start));
    last_start = ctx.st_host->last_start;
    if (trace) {
      auto h1 = std::chrono::steady_clock::now();
      fprintf(stderr, "bt-trace level %u c=%llu host %.3f ms\n", l, (unsigned long long)t->lv[l].c,
              std::chrono::duration<double, std::milli>(h1 - h0).count());
    }
  }
  ctx.gl_chunk = nullptr;
  ctx.gl_mx = nullptr;
  ctx.gl_x = nullptr;
  ctx.gl_total = 0;
  return BT_OK;
}

}  // namespace

int build_levels(BuildCtx& ctx) {
  if (ctx.t->q == Mersenne61::Q) return all_levels(Mersenne61{}, ctx);
  return all_levels(SmallMod{ctx.t->q}, ctx);
}

}  // namespace bt
