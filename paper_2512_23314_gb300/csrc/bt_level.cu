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
#include <cstdio>

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
};

struct Geo {
  const uint8_t* T;
  uint64_t n;
  const uint64_t* Hs;
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

// 1. Block fingerprints and block-table insertion.
template <class M>
__global__ void k_block_fp(M m, Geo g, uint64_t* __restrict__ fpB, uint32_t* __restrict__ slotB,
                           uint64_t* bkey, uint64_t bmask, uint32_t* brep, LevelDev* ld,
                           Status* status) {
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < g.c;
       k += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t s = g.st[k], len = blen(g, k);
    uint64_t fp = window_fp(m, g.T, g.Hs, g.B, len == g.b ? g.Bb : g.Br, s, len);
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
                              uint64_t* pkey, uint64_t pmask, LevelDev* ld, Status* status) {
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k + 1 < g.c;
       k += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t sp = kNoSlot;
    if (g.st[k + 1] == g.st[k] + g.b) {
      atomicAdd(&ld->npairs, 1u);
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
template <class M>
__global__ void __launch_bounds__(256) k_scan(M m, Geo g, uint64_t cpb,
                                             const uint64_t* __restrict__ bkey, uint64_t bmask,
                                             unsigned long long* blo,
                                             const uint64_t* __restrict__ pkey, uint64_t pmask,
                                             unsigned long long* plo, LevelDev* ld) {
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
    if (p0 + g.b <= av) {
      uint64_t fp = window_fp(m, g.T, g.Hs, g.B, g.Bb, p0, g.b);
      for (uint64_t p = p0; p < pend && p + g.b <= av; p++) {
        if (p > p0) {
          uint64_t out = (uint64_t)g.T[p - 1] + 1, in = (uint64_t)g.T[p + g.b - 1] + 1;
          fp = m.add(m.sub(m.mul(fp, g.B), m.mul(out, g.Bb)), in);
        }
        uint32_t sl = tbl_find(bkey, bmask, fp);
        if (sl == kNoSlot) continue;
        min_pos(&blo[sl], p);
        if (p + 2 * g.b <= av) {
          uint64_t fp2 = window_fp(m, g.T, g.Hs, g.B, g.Bb, p + g.b, g.b);
          uint32_t s2 = tbl_find(bkey, bmask, fp2);
          if (s2 != kNoSlot) {
            uint32_t ps = tbl_find(pkey, pmask, ((uint64_t)sl << 32) | s2);
            if (ps != kNoSlot) min_pos(&plo[ps], p);
          }
        }
        if (g.r && sl == pretail && p + g.b + g.r <= av &&
            window_fp(m, g.T, g.Hs, g.B, g.Br, p + g.b, g.r) == fp_tail)
          min_pos(&ld->lo_tailpair, p);
      }
    }
    if (g.r && p0 + g.r <= av) {
      uint64_t fp = window_fp(m, g.T, g.Hs, g.B, g.Br, p0, g.r);
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

// 4a. Pair results: leftmost when the slot minimum is the pair's own start;
// otherwise queue a verification of the earlier occurrence.
__global__ void k_pair_jobs(Geo g, const uint32_t* __restrict__ slotP,
                            const unsigned long long* __restrict__ plo, uint64_t* __restrict__ plo_k,
                            uint8_t* __restrict__ pm, Job* jobs, uint64_t* job_of, LevelDev* ld,
                            Status* status) {
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k + 1 < g.c;
       k += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t sp = slotP[k];
    pm[k] = 0;
    job_of[k] = kNone;
    if (sp == kNoSlot) continue;
    uint64_t lo = sp == kTailPair ? ld->lo_tailpair : plo[sp];
    uint64_t s = g.st[k];
    plo_k[k] = lo;
    if (lo == s) {
      pm[k] = 1;
    } else if (lo < s) {
      uint64_t len = g.b + blen(g, k + 1);
      unsigned long long id = atomicAdd(&ld->njobs, 1ull);
      jobs[id] = Job{lo, s, len, k};
      job_of[k] = id;
      atomicAdd(&status->verify_bytes, 2ull * len);
    } else {
      atomicExch(&status->error, 3ull);  // the pair's own window was not seen
    }
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
                             const unsigned int* __restrict__ mismatch, uint64_t* susp, LevelDev* ld,
                             Status* status) {
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k + 1 < g.c;
       k += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t id = job_of[k];
    if (id == kNone || !mismatch[id]) continue;
    atomicAdd(&status->collisions, 1ull);
    susp[atomicAdd(&ld->nsusp, 1ull)] = k;
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
    uint64_t fp = window_fp(m, g.T, g.Hs, g.B, BL, p0, klen);
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

__global__ void k_init_exlo(Geo g, const uint64_t* __restrict__ susp, unsigned long long* exlo,
                            const LevelDev* ld) {
  const uint64_t ns = ld->nsusp;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < ns;
       i += (uint64_t)gridDim.x * blockDim.x)
    exlo[i] = g.st[susp[i]];
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
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < g.c;
       k += (uint64_t)gridDim.x * blockDim.x) {
    job_of[k] = kNone;
    lo[k] = kNone;
    if (!all && is_marked(mw, k)) continue;
    uint64_t s = g.st[k], len = blen(g, k);
    uint64_t p = slotB[k] == kNoSlot ? ld->lo_tail : blo[slotB[k]];
    lo[k] = p;
    if (p == s) continue;
    if (p > s) {
      atomicExch(&status->error, 4ull);
      continue;
    }
    unsigned long long id = atomicAdd(&ld->njobs, 1ull);
    jobs[id] = Job{p, s, len, k};
    job_of[k] = id;
    atomicAdd(&status->verify_bytes, 2ull * len);
  }
}

__global__ void k_block_apply(Geo g, const uint64_t* __restrict__ job_of,
                              const unsigned int* __restrict__ mismatch, uint64_t* susp, LevelDev* ld,
                              Status* status) {
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < g.c;
       k += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t id = job_of[k];
    if (id == kNone || !mismatch[id]) continue;
    atomicAdd(&status->collisions, 1ull);
    susp[atomicAdd(&ld->nsusp, 1ull)] = k;
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

uint64_t pow2_at_least(uint64_t x) {
  uint64_t p = 16;
  while (p < x) p <<= 1;
  return p;
}

struct LevelWork {
  uint64_t *fpB, *bkey, *pkey, *plo_k, *job_of, *susp;
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
  BT_LAUNCH(k_init_exlo<<<grid_for(g.c, T), T, 0, s>>>(g, W.susp, W.exlo, W.ld));
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

  Scratch sc(s);
  LevelWork W;
  BT_TRY(sc.alloc(&W.fpB, c));
  BT_TRY(sc.alloc(&W.slotB, c));
  BT_TRY(sc.alloc(&W.slotP, c));
  BT_TRY(sc.alloc(&W.pm, c));
  BT_TRY(sc.alloc(&W.plo_k, c));
  BT_TRY(sc.alloc(&W.job_of, c));
  BT_TRY(sc.alloc(&W.susp, c));
  BT_TRY(sc.alloc(&W.exlo, c));
  BT_TRY(sc.alloc(&W.jobs, c));
  BT_TRY(sc.alloc(&W.mismatch, c));
  BT_TRY(sc.alloc(&W.bkey, bcap));
  BT_TRY(sc.alloc(&W.brep, bcap));
  BT_TRY(sc.alloc(&W.blo, bcap));
  BT_TRY(sc.alloc(&W.pkey, pcap));
  BT_TRY(sc.alloc(&W.plo, pcap));
  BT_TRY(sc.alloc(&W.ld, 1));
  const uint64_t words = (c + 31) / 32;
  BT_TRY(sc.alloc(&W.wpop, words));
  // Persistent level arrays.
  BT_CUDA(cudaMallocAsync(&v.mw, words * sizeof(uint32_t) + 4, s));
  BT_CUDA(cudaMallocAsync(&v.mr, (words + 1) * sizeof(uint32_t), s));
  BT_CUDA(cudaMallocAsync(&v.ptr, c * sizeof(uint32_t) + 4, s));
  BT_CUDA(cudaMallocAsync(&v.off, c * sizeof(uint64_t) + 8, s));
  BT_CUDA(cudaMallocAsync(&v.lo, c * sizeof(uint64_t) + 8, s));

  BT_CUDA(cudaMemsetAsync(W.bkey, 0xFF, bcap * sizeof(uint64_t), s));
  BT_CUDA(cudaMemsetAsync(W.brep, 0xFF, bcap * sizeof(uint32_t), s));
  BT_CUDA(cudaMemsetAsync(W.blo, 0xFF, bcap * sizeof(uint64_t), s));
  BT_CUDA(cudaMemsetAsync(W.pkey, 0xFF, pcap * sizeof(uint64_t), s));
  BT_CUDA(cudaMemsetAsync(W.plo, 0xFF, pcap * sizeof(uint64_t), s));
  BT_CUDA(cudaMemsetAsync(W.ld, 0xFF, sizeof(LevelDev), s));
  BT_CUDA(cudaMemsetAsync(&W.ld->npairs, 0, sizeof(unsigned int), s));
  BT_CUDA(cudaMemsetAsync(&W.ld->njobs, 0, 2 * sizeof(unsigned long long), s));
  BT_CUDA(cudaMemsetAsync(W.mismatch, 0, c * sizeof(unsigned int), s));

  const unsigned T = 256;
  const unsigned gc = grid_for(c, T);
  BT_LAUNCH(k_block_fp<M><<<gc, T, 0, s>>>(m, g, W.fpB, W.slotB, W.bkey, bcap - 1, W.brep, W.ld, ctx.st));
  BT_LAUNCH(k_pair_insert<<<gc, T, 0, s>>>(g, W.slotB, W.slotP, W.pkey, pcap - 1, W.ld, ctx.st));
  {
    ProfScope ps("window_scan", s, (c - 1) * b + (len_last < b ? len_last : b));
    BT_LAUNCH(k_scan<M><<<grid_for(c * cpb, T), T, 0, s>>>(m, g, cpb, W.bkey, bcap - 1, W.blo, W.pkey, pcap - 1,
                                                  W.plo, W.ld));
  }
  BT_CUDA(cudaGetLastError());

  // Pairs: verify, resolve collisions exactly, mark.
  const uint64_t ppj_pair = (2 * b + kPiece - 1) / kPiece;
  BT_LAUNCH(k_pair_jobs<<<gc, T, 0, s>>>(g, W.slotP, W.plo, W.plo_k, W.pm, W.jobs, W.job_of, W.ld, ctx.st));
  BT_LAUNCH(k_verify<<<grid_for(c * ppj_pair * 32, T), T, 0, s>>>(ctx.T, W.jobs, W.ld, ppj_pair, W.mismatch));
  BT_LAUNCH(k_pair_apply<<<gc, T, 0, s>>>(g, W.job_of, W.mismatch, W.susp, W.ld, ctx.st));
  BT_TRY(exact_pass(m, g, cpb, 1, W, s));
  BT_LAUNCH(k_pair_exact_apply<<<gc, T, 0, s>>>(g, W.susp, W.exlo, W.pm, W.plo_k, W.ld));
  BT_LAUNCH(k_mark<<<grid_for(words * 32, T), T, 0, s>>>(g, W.slotP, W.pm, v.mw, W.wpop));
  BT_CUDA(cudaGetLastError());
  BT_TRY(scan_u32(W.wpop, v.mr, words, s));

  // Blocks: leftmost occurrences, verified; pointers.
  BT_CUDA(cudaMemsetAsync(&W.ld->njobs, 0, 2 * sizeof(unsigned long long), s));
  BT_CUDA(cudaMemsetAsync(W.mismatch, 0, c * sizeof(unsigned int), s));
  const uint64_t ppj_blk = (b + kPiece - 1) / kPiece;
  BT_LAUNCH(k_block_jobs<<<gc, T, 0, s>>>(g, W.slotB, W.blo, v.mw, t->prune, v.lo, W.jobs, W.job_of, W.ld,
                                ctx.st));
  BT_LAUNCH(k_verify<<<grid_for(c * ppj_blk * 32, T), T, 0, s>>>(ctx.T, W.jobs, W.ld, ppj_blk, W.mismatch));
  BT_LAUNCH(k_block_apply<<<gc, T, 0, s>>>(g, W.job_of, W.mismatch, W.susp, W.ld, ctx.st));
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
  ctx.verify_bytes = ctx.st_host->verify_bytes;
  ctx.collisions = ctx.st_host->collisions;
  if (ctx.st_host->error) return BT_EINTERNAL;
  return BT_OK;
}

template <class M>
int all_levels(const M& m, BuildCtx& ctx) {
  bt_tree* t = ctx.t;
  Level& r = t->lv[0];
  r.c = (t->n + r.b - 1) / r.b;
  BT_CUDA(cudaMallocAsync(&r.st, r.c * sizeof(uint64_t), ctx.s));
  BT_LAUNCH(k_level_start<<<grid_for(r.c, 256), 256, 0, ctx.s>>>(r.c, r.b, r.st));
  uint64_t last_start = (r.c - 1) * r.b;
  for (uint32_t l = 0; l < t->L; l++) {
    BT_TRY(level_pass(m, ctx, l, last_start));
    last_start = ctx.st_host->last_start;
  }
  return BT_OK;
}

}  // namespace

int build_levels(BuildCtx& ctx) {
  if (ctx.t->q == Mersenne61::Q) return all_levels(Mersenne61{}, ctx);
  return all_levels(SmallMod{ctx.t->q}, ctx);
}

}  // namespace bt
