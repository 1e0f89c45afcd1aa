// bt_batch.cuh -- types shared by the host driver and the persistent kernel of
// the batched build (bt_batch.cu).
//
// A batch is built by one persistent kernel per size class of documents.
// Every CTA takes the next document from a device work queue (an atomic
// counter over the documents in decreasing length) and builds that
// document's whole tree by itself, level by level (section 3's levels, the
// Karp-Rabin pass of section 3.1, then the pruning post-pass and the
// rank/select counters), with a barrier of the CTA between the steps.  No
// step of a document needs the host, so one launch builds thousands of
// documents, each with the same result as a standalone build.
#pragma once

#include "bt_internal.cuh"

namespace bt {

constexpr uint32_t kBMaxLevels = 40;       // documents with more levels use the standard path
constexpr uint64_t kBMaxText = 1ull << 30; // longest document of the batched path
// Selected grams (anchors of the window scan on levels with long blocks): a
// 16-byte gram is selected when its 32-bit hash is below 2^(32 - 6), one
// position in 64 on average; a document keeps up to n/32 + 1024 of them.
constexpr uint32_t kGramW = 16;
constexpr uint32_t kGramSelShift = 26;
constexpr uint64_t kAnchorMinB = 1024;  // levels with b >= this scan by anchors (BT_FLAG_ANCHOR_ALL: 32)
__host__ __device__ inline uint64_t gram_list_cap(uint64_t n) { return n / 32 + 1024; }

// One document of a batch (host -> device).
struct BDoc {
  const uint8_t* T;     // device text
  uint64_t n;
  uint32_t sigma, L;
  uint32_t index;       // position in the caller's arrays
  uint32_t lv_off;      // first entry of this document in the level arrays
};

// Per level of a finished document (device -> host).
struct BLevelRes {
  uint64_t c, b, nmarked;
  uint32_t arity, cw;
  uint64_t stats[BT_ST_FIELDS];
};

// Per document (device -> host).
struct BRes {
  int status;              // BT_OK, BT_EINVAL (alphabet), BT_ENOMEM (pool), BT_EINTERNAL
  uint32_t S;
  uint64_t leaf_bytes;     // bytes of leaf text
  uint64_t out_off;        // the tree's arrays: pool + out_off
  uint64_t out_bytes;      // bytes taken from the pool (or needed, with BT_ENOMEM)
  // SM clock cycles the CTA spent per phase: set-up (alphabet, prefix
  // fingerprints), tables (block and pair fingerprints), window scan,
  // verification / marks / pointers / split, pruning, output and counters.
  unsigned long long cycles[6];
  int16_t sym[256];
};

// Where the arrays of a finished tree lie in its pool region, in bytes from
// the region's start.  The same function runs on the device (to write the
// tree) and on the host (to point the bt_tree at it).
struct OutLevel {
  uint64_t st, mw, mr, ptr, off, cnt, pc;
};
__host__ __device__ inline uint64_t out_align(uint64_t x) { return (x + 255) & ~255ull; }
__host__ __device__ inline uint64_t out_align16(uint64_t x) { return (x + 15) & ~15ull; }

// c[l]: blocks of level l after pruning; cw[l]: counter bytes; S symbols;
// leaf_alloc: leaf text bytes (rounded).  Returns the region's size.
__host__ __device__ inline uint64_t out_layout(uint32_t L, const uint64_t* c, const uint32_t* cw, uint32_t S,
                                               uint64_t leaf_alloc, OutLevel* lv, uint64_t* view,
                                               uint64_t* pre, uint64_t* leaf, uint64_t* sym) {
  uint64_t o = 0;
  *view = o;
  o = out_align16(o + sizeof(TreeView));
  for (uint32_t l = 0; l < L; l++) {
    const uint64_t words = (c[l] + 31) / 32;
    lv[l].st = o;
    o = out_align16(o + c[l] * 8 + 8);
    lv[l].mw = o;
    o = out_align16(o + words * 4 + 4);
    lv[l].mr = o;
    o = out_align16(o + (words + 1) * 4);
    lv[l].ptr = o;
    o = out_align16(o + c[l] * 4 + 4);
    lv[l].off = o;
    o = out_align16(o + c[l] * 8 + 8);
    lv[l].cnt = o;
    o = out_align16(o + c[l] * S * cw[l] + 4);
    lv[l].pc = o;
    o = out_align16(o + c[l] * S * cw[l] + 4);
  }
  *pre = o;
  o = out_align16(o + (c[0] + 1) * (uint64_t)S * 8 + 8);
  *leaf = o;
  o = out_align16(o + leaf_alloc + 16);
  *sym = o;
  o = out_align16(o + 256 * sizeof(int16_t));
  return o;
}

// Scratch of one CTA for one document: offsets in bytes from the CTA's
// region.  Level l may hold at most cmax[l] = ceil(n / b_l) blocks.
struct ScratchLayout {
  uint64_t H;                                   // u64[n + 1]
  uint64_t lpos, lhash;                         // u32[gram_list_cap(n)]: selected grams in text order
  uint64_t st[kBMaxLevels], lo[kBMaxLevels], off[kBMaxLevels];  // u64[cmax]
  uint64_t ptr[kBMaxLevels], mw[kBMaxLevels], mr[kBMaxLevels];  // u32
  uint64_t temp;                                // per-level work area (reused)
  uint64_t total;
};

__host__ __device__ inline uint64_t pow2_ge(uint64_t x) {
  uint64_t p = 16;
  while (p < x) p <<= 1;
  return p;
}

// Bytes of the per-level work area for a level of at most cm blocks: the
// level pass (fingerprints, slots, pair results, jobs, suspects, block and
// pair tables) or the pruning pass, whichever is larger.
__host__ __device__ inline uint64_t temp_bytes(uint64_t cm) {
  const uint64_t cap = pow2_ge(2 * cm);
  const uint64_t level = out_align(cm * 8 + 8) * 5      // fpB, plo, job_of, susp, exlo
                         + out_align(cm * 4 + 4) * 4    // slotB, slotP, mismatch, wpop
                         + out_align(cm + 8)            // pm
                         + out_align(cm * 32 + 32)      // jobs
                         + out_align(cm * 8 + 8)        // exact-scan powers
                         + out_align(cap * 32) + out_align(cap * 16)
                         + out_align(cap * 8);          // anchor table
  const uint64_t prune = out_align(cm + 8) * 5          // hit_v, hit2, tgt_w, gone, mk2
                         + out_align(cm * 4 + 4) * 7    // state, indeg, fq x2, nidx, wpop, ptr2
                         + out_align(cm * 8 + 8) * 5;   // t1, t2, st2, off2, lo2
  return level > prune ? level : prune;
}

__host__ __device__ inline uint64_t scratch_layout(uint64_t n, uint32_t L, const uint64_t* b, ScratchLayout* s) {
  uint64_t o = 0, cm_max = 1;
  s->H = o;
  o = out_align(o + (n + 1) * 8);
  s->lpos = o;
  o = out_align(o + gram_list_cap(n) * 4);
  s->lhash = o;
  o = out_align(o + gram_list_cap(n) * 4);
  for (uint32_t l = 0; l < L; l++) {
    const uint64_t cm = (n + b[l] - 1) / b[l];
    const uint64_t words = (cm + 31) / 32;
    if (cm > cm_max) cm_max = cm;
    s->st[l] = o;
    o = out_align(o + cm * 8 + 8);
    s->lo[l] = o;
    o = out_align(o + cm * 8 + 8);
    s->off[l] = o;
    o = out_align(o + cm * 8 + 8);
    s->ptr[l] = o;
    o = out_align(o + cm * 4 + 4);
    s->mw[l] = o;
    o = out_align(o + words * 4 + 4);
    s->mr[l] = o;
    o = out_align(o + (words + 1) * 4 + 4);
  }
  s->temp = o;
  o = out_align(o + temp_bytes(cm_max));
  s->total = o;
  return o;
}

// Kernel parameters of one class launch.
struct BParams {
  const BDoc* docs;
  uint32_t ndocs;
  unsigned int* next;             // work-queue counter
  const uint64_t* sizes;          // block sizes, docs[d].lv_off + l
  BRes* res;
  BLevelRes* lres;
  char* scratch;
  uint64_t scratch_per_cta;
  char* pool;
  unsigned long long* pool_used;
  uint64_t pool_cap;
  uint64_t B;                     // Karp-Rabin base
  const uint64_t* pw32;           // (B^32)^i for i <= blockDim.x
  int prune;
  uint64_t max_rounds;
  uint32_t dyn_words;             // 32-bit words of dynamic shared memory
  uint32_t scan_u;                // window run: consecutive positions per lane of the scan (1-8)
  uint64_t anchor_min_b;          // levels with b at least this scan by anchors
};

}  // namespace bt
