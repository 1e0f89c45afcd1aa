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
  unsigned long long cands;         // windows proposed by anchors and filters
  unsigned long long hits;          // proposed windows whose fingerprint is a key's
};

struct Geo {
  const uint8_t* T;
  uint64_t n;
  const uint64_t* Hs;
  const uint64_t* PB;       // B^k, k <= 32
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

__device__ __forceinline__ uint32_t tbl_insert(uint64_t* keys, uint64_t mask, uint64_t key) {
  uint64_t h = mix64(key) & mask;
  for (uint64_t it = 0; it <= mask; it++) {
    unsigned long long old = atomicCAS((unsigned long long*)&keys[h], (unsigned long long)kNone,
                                       (unsigned long long)key);
    if (old == kNone || old == key) return (uint32_t)h;
    h = (h + 1) & mask;
  }
  return kNoSlot;
}

__device__ __forceinline__ uint32_t tbl_find(const uint64_t* __restrict__ keys, uint64_t mask,
                                             uint64_t key) {
  uint64_t h = mix64(key) & mask;
  for (uint64_t it = 0; it <= mask; it++) {
    uint64_t k = keys[h];
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
                           uint64_t* bkey, uint64_t bmask, uint32_t* brep, LevelDev* ld,
                           Status* status) {
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < g.c;
       k += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t s = g.st[k], len = blen(g, k);
    uint64_t fp = window_fast(m, g.T, g.Hs, g.PB, len == g.b ? g.Bb : g.Br, s, len);
    fpB[k] = fp;
    if (len == g.b) {
      uint32_t slot = tbl_insert(bkey, bmask, fp);
      if (slot == kNoSlot) {
        atomicExch(&status->error, 1ull);
        slotB[k] = kNoSlot;
        continue;
      }
      slotB[k] = slot;
      atomicMin(&brep[slot], (uint32_t)k);
    } else {
      slotB[k] = kNoSlot;
      ld->fp_tail = fp;
    }
  }
}

// 2. Pair-table insertion: key (slot_k, slot_k+1) for pairs of full blocks.
__global__ void k_pair_insert(Geo g, const uint32_t* __restrict__ slotB, uint32_t* __restrict__ slotP,
                              uint64_t* pkey, uint64_t pmask, unsigned long long* maxpst, LevelDev* ld,
                              Status* status) {
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k + 1 < g.c;
       k += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t sp = kNoSlot;
    if (g.st[k + 1] == g.st[k] + g.b) {
      atomicAdd(&ld->npairs, 1u);
      // The last pair start per first-block slot: a window after it cannot
      // be the leftmost occurrence of any pair that starts with that slot.
      if (slotB[k] != kNoSlot) atomicMax(&maxpst[slotB[k]], (unsigned long long)g.st[k]);
      if (slotB[k + 1] == kNoSlot) {
        sp = kTailPair;
        ld->pretail_slot = slotB[k];
      } else {
        sp = tbl_insert(pkey, pmask, ((uint64_t)slotB[k] << 32) | slotB[k + 1]);
        if (sp == kNoSlot) atomicExch(&status->error, 2ull);
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
                                             const uint64_t* __restrict__ bkey, uint64_t bmask,
                                             unsigned long long* blo,
                                             const uint64_t* __restrict__ pkey, uint64_t pmask,
                                             unsigned long long* plo, LevelDev* ld, int tail_only) {
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
      uint64_t fp = window_fast(m, g.T, g.Hs, g.PB, g.Bb, p0, g.b);
      for (uint64_t p = p0; p < pend && p + g.b <= av; p++) {
        if (p > p0) {
          uint64_t out = (uint64_t)g.T[p - 1] + 1, in = (uint64_t)g.T[p + g.b - 1] + 1;
          fp = m.add(m.sub(m.mul(fp, g.B), m.mul(out, g.Bb)), in);
        }
        uint32_t sl = tbl_find(bkey, bmask, fp);
        if (sl == kNoSlot) continue;
        min_pos(&blo[sl], p);
        if (p + 2 * g.b <= av) {
          uint64_t fp2 = window_fast(m, g.T, g.Hs, g.PB, g.Bb, p + g.b, g.b);
          uint32_t s2 = tbl_find(bkey, bmask, fp2);
          if (s2 != kNoSlot) {
            uint32_t ps = tbl_find(pkey, pmask, ((uint64_t)sl << 32) | s2);
            if (ps != kNoSlot) min_pos(&plo[ps], p);
          }
        }
        if (g.r && sl == pretail && p + g.b + g.r <= av &&
            window_fast(m, g.T, g.Hs, g.PB, g.Br, p + g.b, g.r) == fp_tail)
          min_pos(&ld->lo_tailpair, p);
      }
    }
    if (g.r && p0 + g.r <= av) {
      uint64_t fp = window_fast(m, g.T, g.Hs, g.PB, g.Br, p0, g.r);
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
// 3'. The anchored window scan.
//
// Probing the table at every window position costs a random memory access
// per text byte.  Instead every window gets an anchor that depends only on its
// content: the first position, among its first W, of a w-gram whose 32-bit
// gram hash is "selected" (top sbits of a multiplicative mix are zero, density
// 2^-sbits).  Every key is registered under its anchor gram: the anchor table
// maps a gram to the set of offsets (a 64-bit mask) at which keys anchor on
// it.  The scan rolls a 32-bit gram hash over the level (no 61-bit arithmetic
// per byte); only at a selected gram that passes a bitmap filter does it read
// the anchor table, and each offset a in the gram's mask proposes the window
// at x - a, whose 61-bit fingerprint is looked up in the block table.  A
// window equal to a key has the key's anchor (same gram, same offset), so it
// is always proposed: the slot minima are the same as when probing every
// window.  A key without an anchor in its first W grams can only be equal to a
// window without one; such keys are registered by their first gram in a small
// shared-memory filter, checked at every position only when such keys exist.
// ---------------------------------------------------------------------------
constexpr uint32_t kAnchorQ = 128;        // window starts per thread
constexpr uint32_t kAnchorWmax = 64;      // anchor search range
constexpr uint32_t kEmptyGram = 0xFFFFFFFFu;
constexpr uint32_t kFibMul = 0x9E3779B1u;
constexpr uint32_t kScanThreads = 256;
constexpr uint32_t kSlotBytes = 180;      // staging bytes per thread (45 words: 45 = 13 mod 32)
constexpr uint32_t kSecBits = 4096;       // first-gram filter of keys without an anchor
constexpr uint32_t kSmemBitmapWords = 8192;  // anchor bitmap kept in shared memory up to 32 KiB

struct GramP {
  uint32_t w;      // gram length
  uint32_t W;      // anchor search range for full-length windows
  uint32_t Wr;     // anchor search range for the short tail (0: none)
  uint32_t sbits;  // selection: top sbits of the mixed gram are zero
  uint32_t fbits;  // bitmap index bits
  uint32_t rb;     // gram base (odd)
  uint32_t rw;     // rb^w mod 2^32
};

// gram -> offsets at which keys anchor on it.
struct AnchorSet {
  uint32_t gram;             // remapped gram hash (kEmptyGram: empty slot)
  uint32_t pad;
  unsigned long long offs;   // bit a: some key has its anchor at offset a
  unsigned long long maxst;  // largest start of a key anchored on this gram
};

__device__ __forceinline__ uint32_t gram_hash(const uint8_t* __restrict__ T, uint64_t x, uint32_t w,
                                              uint32_t rb) {
  uint32_t h = 0;
  for (uint32_t i = 0; i < w; i++) h = h * rb + T[x + i];
  return h;
}
__device__ __forceinline__ bool gram_selected(const GramP& gp, uint32_t g) {
  return gp.sbits == 0 || ((g * kFibMul) >> (32 - gp.sbits)) == 0;
}
__device__ __forceinline__ uint32_t gram_bit(const GramP& gp, uint32_t g) {
  return ((g * kFibMul) << gp.sbits) >> (32 - gp.fbits);
}
// Gram hashes are remapped away from 0xFFFFFFFF, the empty marker.
__device__ __forceinline__ uint32_t gram_key(uint32_t g) { return g == kEmptyGram ? kEmptyGram - 1 : g; }
__device__ __forceinline__ uint32_t gram_slot(uint32_t g, uint32_t mask) {
  g ^= g >> 16;
  g *= 0x7FEB352Du;
  g ^= g >> 15;
  g *= 0x846CA68Bu;
  g ^= g >> 16;
  return g & mask;
}
__device__ __forceinline__ uint32_t sec_bit(uint32_t g) { return (g * 0x2545F491u) >> 20; }  // 12 bits

__global__ void k_clear_offs(AnchorSet* atab, uint64_t cap) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < cap;
       i += (uint64_t)gridDim.x * blockDim.x) {
    atab[i].offs = 0;
    atab[i].maxst = 0;
  }
}

// Register the anchor of every key (every block and the tail).
__global__ void k_anchor_keys(Geo g, GramP gp, const uint32_t* __restrict__ slotB, AnchorSet* atab,
                              uint32_t amask, uint32_t* bitmap, uint32_t* secbits, LevelDev* ld,
                              Status* status) {
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < g.c;
       k += (uint64_t)gridDim.x * blockDim.x) {
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
    const uint32_t g0 = gram_hash(g.T, s, gp.w, gp.rb);
    uint32_t gh = g0, a = kNoSlot;
    for (uint32_t o = 0; o < Wk; o++) {
      if (o > 0) gh = gh * gp.rb - (uint32_t)g.T[s + o - 1] * gp.rw + g.T[s + o + gp.w - 1];
      if (gram_selected(gp, gh)) {
        a = o;
        break;
      }
    }
    if (a == kNoSlot) {  // no anchor: registered by its first gram
      const uint32_t sb = sec_bit(g0);
      atomicOr(&secbits[sb >> 5], 1u << (sb & 31));
      if (tail) ld->tail_anchorless = 2u;
      else ld->anchorless = 1u;
      continue;
    }
    const uint32_t gk = gram_key(gh);
    const uint32_t bit = gram_bit(gp, gh);
    atomicOr(&bitmap[bit >> 5], 1u << (bit & 31));
    if (tail) {
      ld->tail_gram = gk;
      ld->tail_a = a;
      continue;
    }
    uint32_t h = gram_slot(gk, amask);
    bool placed = false;
    for (uint32_t it = 0; it <= amask && !placed; it++) {
      const uint32_t cur = atomicCAS(&atab[h].gram, kEmptyGram, gk);
      if (cur == kEmptyGram || cur == gk) {
        atomicOr(&atab[h].offs, 1ull << a);
        atomicMax(&atab[h].maxst, (unsigned long long)s);
        placed = true;
      } else {
        h = (h + 1) & amask;
      }
    }
    if (!placed) atomicExch(&status->error, 7ull);
  }
}

template <class M>
struct ScanCtx {
  M m;
  Geo g;
  const uint64_t* bkey;
  uint64_t bmask;
  unsigned long long* blo;
  const uint64_t* pkey;
  uint64_t pmask;
  unsigned long long* plo;
  LevelDev* ld;
  uint32_t pretail;
  uint64_t fp_tail;
  const unsigned long long* maxpst;  // last pair start per first-block slot
  struct Cand* q;                    // candidate windows for k_candidates
  unsigned long long* qn;            // candidates appended (may exceed qcap)
  uint64_t qcap;
};

// A proposed window: start p, the block k whose scan thread proposed it,
// kind 0 (full-length key) or 1 (the short tail key).
struct Cand {
  uint64_t p;
  uint32_t k;
  uint32_t kind;
};

// A full-length window at p (inside a run ending at av) matches slot sl.
template <class M>
__device__ __forceinline__ void on_block_hit(const ScanCtx<M>& C, uint32_t sl, uint64_t p,
                                             uint64_t av) {
  const Geo& g = C.g;
  min_pos(&C.blo[sl], p);
  if (p > C.maxpst[sl]) return;  // no pair starting with this slot can begin here or later
  if (p + 2 * g.b <= av) {
    uint64_t fp2 = window_fast(C.m, g.T, g.Hs, g.PB, g.Bb, p + g.b, g.b);
    uint32_t s2 = tbl_find(C.bkey, C.bmask, fp2);
    if (s2 != kNoSlot) {
      uint32_t ps = tbl_find(C.pkey, C.pmask, ((uint64_t)sl << 32) | s2);
      if (ps != kNoSlot) min_pos(&C.plo[ps], p);
    }
  }
  if (g.r && sl == C.pretail && p + g.b + g.r <= av &&
      window_fast(C.m, g.T, g.Hs, g.PB, g.Br, p + g.b, g.r) == C.fp_tail)
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

// Full-length candidate window at p: fingerprint -> block slot.
template <class M>
__device__ __forceinline__ void try_block(const ScanCtx<M>& C, uint64_t k, uint64_t s, uint64_t av,
                                          uint64_t p, uint32_t& ncand, uint32_t& nhit) {
  uint64_t avp;
  if (!window_in_run(C.g, k, s, av, p, C.g.b, &avp)) return;
  ncand++;
  const uint64_t fp = window_fast(C.m, C.g.T, C.g.Hs, C.g.PB, C.g.Bb, p, C.g.b);
  const uint32_t sl = tbl_find(C.bkey, C.bmask, fp);
  if (sl != kNoSlot) {
    nhit++;
    on_block_hit(C, sl, p, avp);
  }
}

template <class M>
__device__ __forceinline__ void try_tail(const ScanCtx<M>& C, uint64_t k, uint64_t s, uint64_t av,
                                         uint64_t p) {
  uint64_t avp;
  if (!window_in_run(C.g, k, s, av, p, C.g.r, &avp)) return;
  if (window_fast(C.m, C.g.T, C.g.Hs, C.g.PB, C.g.Br, p, C.g.r) == C.fp_tail)
    min_pos(&C.ld->lo_tail, p);
}

// Queue a proposed window for k_candidates (one slot claim per group of
// lanes that arrive together); when the queue is full, test it here.
template <class M>
__device__ __forceinline__ void propose(const ScanCtx<M>& C, uint64_t k, uint64_t s, uint64_t av,
                                        uint64_t p, uint32_t kind, uint32_t& ncand, uint32_t& nhit) {
  uint64_t avp;
  if (!window_in_run(C.g, k, s, av, p, kind ? C.g.r : C.g.b, &avp)) return;
  const unsigned active = __activemask();
  const unsigned lane = threadIdx.x & 31;
  const int leader = __ffs(active) - 1;
  unsigned long long base = 0;
  if ((int)lane == leader) base = atomicAdd(C.qn, (unsigned long long)__popc(active));
  base = __shfl_sync(active, base, leader);
  const unsigned long long idx = base + __popc(active & ((1u << lane) - 1u));
  if (idx < C.qcap) {
    C.q[idx] = Cand{p, (uint32_t)k, kind};
  } else if (kind) {
    try_tail(C, k, s, av, p);
  } else {
    try_block(C, k, s, av, p, ncand, nhit);
  }
}

// Copy T[a, a+cnt) into a thread's shared-memory slot: 16-byte loads for the
// aligned body when the text is 16-byte aligned, bytes for the rest.
__device__ __forceinline__ void stage(uint8_t* slot, const uint8_t* __restrict__ T, uint64_t n,
                                      uint64_t a, uint32_t cnt, bool aligned16) {
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

template <class M>
__global__ void __launch_bounds__(kScanThreads, 3) k_scan_anchor(ScanCtx<M> C0, GramP gp, uint64_t cpb,
                                                             const AnchorSet* __restrict__ atab,
                                                             uint32_t amask,
                                                             const uint32_t* __restrict__ bitmap_g,
                                                             uint32_t bm_smem_words,
                                                             const uint32_t* __restrict__ secbits_g) {
  extern __shared__ uint32_t smem[];
  uint32_t* sec = smem;                               // kSecBits / 32 words
  uint32_t* bms = smem + kSecBits / 32;               // bm_smem_words words
  uint8_t* slots = (uint8_t*)(bms + bm_smem_words);
  uint8_t* slot = slots + threadIdx.x * kSlotBytes;
  ScanCtx<M> C = C0;
  C.pretail = C.ld->pretail_slot;
  C.fp_tail = C.ld->fp_tail;
  const Geo& g = C.g;
  const bool anchorless = C.ld->anchorless == 1u;
  const bool tail_sec = C.ld->tail_anchorless == 2u;
  const uint32_t tail_gram = C.ld->tail_gram, tail_a = C.ld->tail_a;
  for (uint32_t i = threadIdx.x; i < kSecBits / 32; i += blockDim.x) sec[i] = secbits_g[i];
  for (uint32_t i = threadIdx.x; i < bm_smem_words; i += blockDim.x) bms[i] = bitmap_g[i];
  __syncthreads();
  const uint32_t* bitmap = bm_smem_words ? bms : bitmap_g;
  const bool check_sec = anchorless || tail_sec;
  const bool aligned16 = (((uintptr_t)g.T) & 15) == 0;
  const uint32_t w = gp.w, rb = gp.rb, rw = gp.rw, sbits = gp.sbits, fbits = gp.fbits;
  const uint64_t total = g.c * cpb;
  uint32_t ncand = 0, nhit = 0;
  for (uint64_t wi = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; wi < total;
       wi += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t k = wi / cpb, j = wi - k * cpb;
    const uint64_t s = g.st[k], len = blen(g, k);
    const uint64_t p0 = s + j * kAnchorQ;
    if (p0 >= s + len) continue;
    const uint64_t av = avail_end(g, k);
    // Gram positions x in [p0, xe): owned by this thread and able to anchor a
    // window that fits in the run (anchors of a length-L window lie below
    // its start + W_L; windows without anchors start at their first gram).
    uint64_t xe = p0 + kAnchorQ < s + len ? p0 + kAnchorQ : s + len;
    uint64_t xm = av >= g.b ? av - g.b + gp.W : 0;
    if (g.r && av >= g.r) {
      const uint64_t xr = av - g.r + (gp.Wr ? gp.Wr : 1);
      if (xr > xm) xm = xr;
    }
    const uint64_t gram_end = av + 1 >= w ? av + 1 - w : 0;  // grams must fit in the run
    if (xm > gram_end) xm = gram_end;
    if (xe > xm) xe = xm;
    if (xe <= p0) continue;
    const uint32_t nx = (uint32_t)(xe - p0);
    stage(slot, g.T, g.n, p0, nx + w - 1, aligned16);
    // Pass 1: roll the gram hash; mark positions whose gram is selected and
    // passes the bitmap filter (m0/m1), or hits the first-gram filter of keys
    // without an anchor (q0/q1).
    unsigned long long m0 = 0, m1 = 0, q0 = 0, q1 = 0;
    uint32_t gh = 0;
    for (uint32_t i = 0; i < w; i++) gh = gh * rb + slot[i];
    for (uint32_t i = 0; i < nx; i++) {
      if (i) gh = gh * rb - (uint32_t)slot[i - 1] * rw + slot[i + w - 1];
      if (check_sec) {
        const uint32_t sb = sec_bit(gh);
        if ((sec[sb >> 5] >> (sb & 31)) & 1u) {
          if (i < 64) q0 |= 1ull << i;
          else q1 |= 1ull << (i - 64);
        }
      }
      const uint32_t mix = gh * kFibMul;
      if (sbits && (mix >> (32 - sbits))) continue;
      const uint32_t bit = (mix << sbits) >> (32 - fbits);
      if (!((bitmap[bit >> 5] >> (bit & 31)) & 1u)) continue;
      if (i < 64) m0 |= 1ull << i;
      else m1 |= 1ull << (i - 64);
    }
    // Pass 2: the marked positions (rare).
    for (int half = 0; half < 2; half++) {
      unsigned long long mm = half ? m1 : m0, qq = half ? q1 : q0;
      while (mm | qq) {
        const uint32_t bi = __ffsll(mm | qq) - 1;
        const unsigned long long one = 1ull << bi;
        const bool is_anchor = mm & one, is_sec = qq & one;
        mm &= ~one;
        qq &= ~one;
        const uint32_t i = bi + 64u * half;
        const uint64_t x = p0 + i;
        uint32_t gx = 0;
        for (uint32_t t = 0; t < w; t++) gx = gx * rb + slot[i + t];
        if (is_sec) {
          if (anchorless) propose(C, k, s, av, x, 0, ncand, nhit);
          if (tail_sec) propose(C, k, s, av, x, 1, ncand, nhit);
        }
        if (!is_anchor) continue;
        const uint32_t gk = gram_key(gx);
        if (gk == tail_gram && x >= tail_a) propose(C, k, s, av, x - tail_a, 1, ncand, nhit);
        unsigned long long offs = 0, maxst = 0;
        for (uint32_t h = gram_slot(gk, amask), it = 0; it <= amask; h = (h + 1) & amask, it++) {
          const uint32_t eg = atab[h].gram;
          if (eg == gk) {
            offs = atab[h].offs;
            maxst = atab[h].maxst;
            break;
          }
          if (eg == kEmptyGram) break;
        }
        // A window that starts after every key anchored on this gram cannot
        // be the leftmost occurrence of any of them, nor of a pair that
        // starts with one of them (both are at or before the key's start).
        while (offs) {
          const uint32_t a = __ffsll(offs) - 1;
          offs &= offs - 1;
          if (a <= x && x - a <= maxst) propose(C, k, s, av, x - a, 0, ncand, nhit);
        }
      }
    }
  }
  if (ncand) atomicAdd(&C.ld->cands, (unsigned long long)ncand);
  if (nhit) atomicAdd(&C.ld->hits, (unsigned long long)nhit);
}

// Test the queued candidate windows: one per thread.
template <class M>
__global__ void __launch_bounds__(256) k_candidates(ScanCtx<M> C0) {
  ScanCtx<M> C = C0;
  C.pretail = C.ld->pretail_slot;
  C.fp_tail = C.ld->fp_tail;
  const unsigned long long qn = *C.qn;
  const uint64_t n = qn < C.qcap ? qn : C.qcap;
  uint32_t ncand = 0, nhit = 0;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const Cand e = C.q[i];
    const uint64_t s = C.g.st[e.k];
    const uint64_t av = avail_end(C.g, e.k);
    if (e.kind) try_tail(C, e.k, s, av, e.p);
    else try_block(C, e.k, s, av, e.p, ncand, nhit);
  }
  if (ncand) atomicAdd(&C.ld->cands, (unsigned long long)ncand);
  if (nhit) atomicAdd(&C.ld->hits, (unsigned long long)nhit);
}

// 4a. Pair results: leftmost when the slot minimum is the pair's own start;
// otherwise queue a verification of the earlier occurrence.
__global__ void k_pair_jobs(Geo g, const uint32_t* __restrict__ slotP,
                            const unsigned long long* __restrict__ plo, uint64_t* __restrict__ plo_k,
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
        lo = sp == kTailPair ? ld->lo_tailpair : plo[sp];
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
__global__ void __launch_bounds__(256) k_verify(const uint8_t* __restrict__ T, const Job* __restrict__ jobs,
                                                const LevelDev* ld, uint64_t ppj,
                                                unsigned int* mismatch) {
  const uint64_t njobs = ld->njobs;
  const unsigned lane = threadIdx.x & 31;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x / 32);
  for (uint64_t w = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) / 32; w < njobs * ppj;
       w += warps) {
    const uint64_t jb = w / ppj, piece = w - jb * ppj;
    const Job J = jobs[jb];
    const uint64_t off = piece * kPiece;
    if (off >= J.len) continue;
    if (*(volatile unsigned int*)&mismatch[jb]) continue;
    const uint64_t end = off + kPiece < J.len ? off + kPiece : J.len;
    bool diff = false;
    for (uint64_t x = off + lane; x < end; x += 32) diff |= T[J.a + x] != T[J.b + x];
    if (__any_sync(0xFFFFFFFFu, diff) && lane == 0) atomicOr(&mismatch[jb], 1u);
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
    uint64_t fp = window_fast(m, g.T, g.Hs, g.PB, BL, p0, klen);
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
                             const unsigned long long* __restrict__ blo, const uint32_t* __restrict__ mw,
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
        p = slotB[k] == kNoSlot ? ld->lo_tail : blo[slotB[k]];
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
  uint64_t* bkey;
  uint32_t* brep;
  unsigned long long* blo;
  unsigned long long* maxpst;
  uint64_t bcap;
  uint64_t* pkey;
  unsigned long long* plo;
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
    if (i < a.bcap) {
      a.bkey[i] = kNone;
      a.brep[i] = 0xFFFFFFFFu;
      a.blo[i] = kNone;
      a.maxpst[i] = 0;
    }
    if (i < a.pcap) {
      a.pkey[i] = kNone;
      a.plo[i] = kNone;
    }
    if (i < a.c) a.mismatch[i] = 0;
    if (a.atab && i < a.acap) {
      a.atab[i].gram = kEmptyGram;
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
GramP choose_gram(uint64_t b, uint64_t r, uint32_t S) {
  (void)S;
  uint32_t w = 16;
  if (w > b / 2) w = (uint32_t)(b / 2 > 0 ? b / 2 : 1);
  GramP gp;
  gp.w = w;
  gp.W = (uint32_t)(b - w + 1 < kAnchorWmax ? b - w + 1 : kAnchorWmax);
  gp.sbits = gp.W >= 64 ? 3 : gp.W >= 32 ? 2 : gp.W >= 16 ? 1 : 0;
  gp.Wr = (r && r >= w) ? (uint32_t)(r - w + 1 < kAnchorWmax ? r - w + 1 : kAnchorWmax) : 0;
  gp.fbits = 12;
  gp.rb = 0x01000193u;
  uint32_t rw = 1;
  for (uint32_t i = 0; i < w; i++) rw *= gp.rb;
  gp.rw = rw;
  return gp;
}

uint64_t pow2_at_least(uint64_t x) {
  uint64_t p = 16;
  while (p < x) p <<= 1;
  return p;
}

struct LevelWork {
  uint64_t *fpB, *bkey, *pkey, *plo_k, *job_of, *susp;
  unsigned long long* maxpst;
  uint32_t *slotB, *brep, *slotP, *wpop;
  unsigned long long *blo, *plo, *exlo;
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
  g.Hs = ctx.Hs;
  g.PB = ctx.PB;
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
  const bool anchored = !ctx.dense_scan;
  const GramP gp = choose_gram(b, r, t->S);
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
  // Candidate queue: a few candidates per covered window is plenty; more
  // are tested inline by the scan.
  const uint64_t cov_l = (c - 1) * b + (len_last < b ? len_last : b);
  uint64_t qcap = cov_l / 2 + 4096;
  if (qcap > (64ull << 20)) qcap = 64ull << 20;

  // Scratch: carved from the build's arena (a dry carving sizes it).
  Arena& A = ctx.arena;
  LevelWork W;
  AnchorSet* atab = nullptr;
  uint32_t *bitmap = nullptr, *secbits = nullptr, *sagg = nullptr;
  Cand* q = nullptr;
  unsigned long long* qn = nullptr;
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
    W.bkey = A.take<uint64_t>(bcap);
    W.brep = A.take<uint32_t>(bcap);
    W.blo = A.take<unsigned long long>(bcap);
    W.maxpst = A.take<unsigned long long>(bcap);
    W.pkey = A.take<uint64_t>(pcap);
    W.plo = A.take<unsigned long long>(pcap);
    W.ld = A.take<LevelDev>(1);
    W.wpop = A.take<uint32_t>(words);
    sagg = A.take<uint32_t>(scan_scratch_words(words));
    if (anchored) {
      atab = A.take<AnchorSet>(acap);
      bitmap = A.take<uint32_t>(bwords);
      secbits = A.take<uint32_t>(kSecBits / 32);
      q = A.take<Cand>(qcap);
      qn = A.take<unsigned long long>(1);
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

  InitArgs ia{W.bkey, W.brep, W.blo, W.maxpst, bcap, W.pkey, W.plo, pcap, W.mismatch, c,
              atab, acap, bitmap, bwords, secbits, qn, W.ld};
  {
    uint64_t top = bcap > acap ? bcap : acap;
    if (bwords > top) top = bwords;
    BT_LAUNCH(k_level_init<<<grid_for(top, T), T, 0, s>>>(ia));
  }
  BT_LAUNCH(k_block_fp<M><<<gc, T, 0, s>>>(m, g, W.fpB, W.slotB, W.bkey, bcap - 1, W.brep, W.ld, ctx.st));
  BT_LAUNCH(k_pair_insert<<<gc, T, 0, s>>>(g, W.slotB, W.slotP, W.pkey, pcap - 1, W.maxpst, W.ld,
                                           ctx.st));
  if (!anchored) {
    ProfScope ps("window_scan", s, cov_l);
    BT_LAUNCH(k_scan<M><<<grid_for(c * cpb, T), T, 0, s>>>(m, g, cpb, W.bkey, bcap - 1, W.blo, W.pkey,
                                                            pcap - 1, W.plo, W.ld, 0));
  } else {
    BT_LAUNCH(k_anchor_keys<<<gc, T, 0, s>>>(g, gq, W.slotB, atab, (uint32_t)(acap - 1), bitmap, secbits,
                                             W.ld, ctx.st));
    ScanCtx<M> C{m, g, W.bkey, bcap - 1, W.blo, W.pkey, pcap - 1, W.plo, W.ld, 0, 0, W.maxpst, q, qn, qcap};
    const uint64_t cpa = (b + kAnchorQ - 1) / kAnchorQ;
    const uint32_t bm_smem = bwords <= kSmemBitmapWords ? (uint32_t)bwords : 0;
    const size_t smem = (kSecBits / 32 + bm_smem) * 4 + (size_t)kScanThreads * kSlotBytes;
    static bool attr_set = false;
    if (!attr_set) {
      BT_CUDA(cudaFuncSetAttribute(k_scan_anchor<M>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)(((size_t)kSecBits / 32 + kSmemBitmapWords) * 4 +
                                         (size_t)kScanThreads * kSlotBytes)));
      attr_set = true;
    }
    ProfScope ps("window_scan", s, cov_l);
    BT_LAUNCH(k_scan_anchor<M><<<grid_for(c * cpa, kScanThreads, 152 * 8), kScanThreads, smem, s>>>(
        C, gq, cpa, atab, (uint32_t)(acap - 1), bitmap, bm_smem, secbits));
    BT_LAUNCH(k_candidates<M><<<152 * 16, 256, 0, s>>>(C));
    if (r)
      BT_LAUNCH(k_scan<M><<<grid_for(c * cpb, T), T, 0, s>>>(m, g, cpb, W.bkey, bcap - 1, W.blo, W.pkey,
                                                              pcap - 1, W.plo, W.ld, 1));
  }
  BT_CUDA(cudaGetLastError());

  // Pairs: verify, resolve collisions exactly, mark.
  const uint64_t ppj_pair = (2 * b + kPiece - 1) / kPiece;
  BT_LAUNCH(k_pair_jobs<<<gc, T, 0, s>>>(g, W.slotP, W.plo, W.plo_k, W.pm, W.jobs, W.job_of, W.ld, ctx.st));
  BT_LAUNCH(k_verify<<<grid_for(c * ppj_pair * 32, T), T, 0, s>>>(ctx.T, W.jobs, W.ld, ppj_pair, W.mismatch));
  BT_LAUNCH(k_pair_apply<<<gc, T, 0, s>>>(g, W.job_of, W.mismatch, W.susp, W.exlo, W.ld, ctx.st));
  BT_TRY(exact_pass(m, g, cpb, 1, W, s));
  BT_LAUNCH(k_pair_exact_apply<<<gc, T, 0, s>>>(g, W.susp, W.exlo, W.pm, W.plo_k, W.ld));
  BT_LAUNCH(k_mark<<<grid_for(words * 32, T), T, 0, s>>>(g, W.slotP, W.pm, v.mw, W.wpop));
  BT_CUDA(cudaGetLastError());
  BT_TRY(scan_u32(W.wpop, v.mr, words, s, sagg));

  // Blocks: leftmost occurrences, verified; pointers.
  BT_LAUNCH(k_reset_jobs<<<gc, T, 0, s>>>(W.mismatch, c, W.ld));
  const uint64_t ppj_blk = (b + kPiece - 1) / kPiece;
  BT_LAUNCH(k_block_jobs<<<gc, T, 0, s>>>(g, W.slotB, W.blo, v.mw, t->prune, v.lo, W.jobs, W.job_of, W.ld,
                                ctx.st));
  BT_LAUNCH(k_verify<<<grid_for(c * ppj_blk * 32, T), T, 0, s>>>(ctx.T, W.jobs, W.ld, ppj_blk, W.mismatch));
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
  return BT_OK;
}

}  // namespace

int build_levels(BuildCtx& ctx) {
  if (ctx.t->q == Mersenne61::Q) return all_levels(Mersenne61{}, ctx);
  return all_levels(SmallMod{ctx.t->q}, ctx);
}

}  // namespace bt
