// bt_batch.cu -- batched construction: a persistent, level-synchronous kernel
// with a per-document work queue.
//
// Each CTA of k_batch repeatedly takes the next document of the batch from a
// device work queue (an atomic counter; the documents come in decreasing
// expected work, length times levels) and builds its whole block tree by
// itself:
//
//   1. alphabet (byte histogram -> dense symbol map, sigma check);
//   2. Karp-Rabin prefix fingerprints H(p) at every position (section 2, the
//      all-prefix form of section 4.1: Horner per 32-byte chunk, then a scan
//      of the chunks with (h1, P1) (x) (h2, P2) = (h1 P2 + h2, P1 P2)), and
//      the list of selected 16-byte grams (the scan's anchors on levels of
//      long blocks);
//   3. for every level (section 3): block and pair fingerprints into
//      open-addressing tables, a scan of the windows of the level's runs of
//      consecutive blocks (section 3.1: phi(p, p+b) = H(p+b) - H(p) B^b,
//      rolled from window to window, or only the windows that the selected
//      grams propose on levels of long blocks; table probe, atomicMin of the
//      leftmost window per key, the pair joined at p+b), byte verification
//      of every accepted minimum with an exact
//      rescan of a key whose fingerprint collided, marks (a pair is marked
//      when its leftmost occurrence is its own start, a block in no pair is
//      marked), back-pointers (ptr, off), and the tau-way split of marked
//      blocks into the next level;
//   4. the pruning post-pass (section 3.1, "Optional Pruning"), with the same
//      four conditions and the same right-to-left rule as the standard path,
//      resolved by frontier rounds over the candidates;
//   5. the rank/select counters, level-1 prefix counts and leaf text, written
//      with the tree's arrays into a region of the batch's output pool taken
//      with one atomic add.
//
// Between steps the CTA meets at a barrier; nothing waits on another CTA, on
// another launch or on the host.  The tree of every document is the one
// bt_build_ex builds for it alone: the same readings of the paper, the same
// sizing, marking, pointer and pruning rules, every match verified.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <memory>
#include <mutex>
#include <queue>
#include <thread>
#include <vector>

#include <chrono>

#include "bt_batch.cuh"

namespace bt {

int plan_sizes(uint64_t n, uint32_t tau, uint32_t leaf, const bt_opts& o, std::vector<uint64_t>& b);
uint64_t base_for(uint64_t seed, uint64_t q);
unsigned device_sm_count();

namespace {

constexpr uint32_t kFull = 0xFFFFFFFFu;
constexpr uint32_t kBTailPair = 0xFFFFFFFEu;
constexpr uint32_t kMaxBThreads = 1024;

struct __align__(32) BSlot {
  unsigned long long key, lo, maxpst, pad;
};
struct __align__(16) PSlot {
  unsigned long long key, lo;
};
struct BJob {
  uint64_t a, b, len, idx;
};

enum : uint32_t { P_UNDEC = 0, P_PRUNED = 1, P_KEPT = 2, P_NOTCAND = 3 };

// Shared state of a CTA.
struct Cta {
  uint32_t doc;
  int err;
  uint64_t n;
  uint32_t S, L;
  int16_t sym[256];
  unsigned int hist[256];
  ScratchLayout sl;
  uint64_t c[kBMaxLevels];
  uint64_t nmarked[kBMaxLevels];
  uint32_t arity[kBMaxLevels];
  uint64_t stats[kBMaxLevels][BT_ST_FIELDS];
  uint64_t last_start;
  // current level
  uint64_t r, Bb, Br, B1;
  uint64_t bmask, pmask;
  uint64_t rtab[256];  // (a + 1) B^b for every byte a
  uint32_t bshift;
  unsigned long long fp_tail, lo_tail, lo_tailpair;
  uint32_t pretail;
  unsigned int npairs, njobs, nsusp;
  uint32_t nsel;                      // selected grams of the document (kNoList: none kept)
  unsigned int anchorless;            // some key of the level has no selected gram
  uint32_t tail_g, tail_a, tail_anchored;  // anchor of the short tail key
  unsigned long long verify_bytes, collisions;
  unsigned long long lastk;
  // scans
  uint32_t wtot[32];
  uint64_t wsum[32];
  uint64_t carry;
  // pruning worklists
  unsigned int wl[3];
  unsigned long long undecided;
  // output
  char* out;
  uint64_t out_off, out_bytes;
  // phase timing (SM cycles)
  unsigned long long cyc[6];
  long long t_mark;
};

// Adds the cycles since the last mark to phase `ph` (thread 0; call right
// after a barrier).
__device__ __forceinline__ void tmark(Cta& C, int ph) {
  if (threadIdx.x == 0) {
    const long long t = clock64();
    C.cyc[ph] += (unsigned long long)(t - C.t_mark);
    C.t_mark = t;
  }
}

__device__ __forceinline__ bool cta_failed(Cta& C) { return __syncthreads_or(C.err != 0) != 0; }
__device__ __forceinline__ void fail(Cta& C, int code) { atomicCAS(&C.err, 0, code); }

__device__ __forceinline__ void min_pos(unsigned long long* a, uint64_t p) {
  if (*(volatile unsigned long long*)a > p) atomicMin(a, (unsigned long long)p);
}
// The same without the read: an atomic whose result is not used (a reduction
// the thread does not wait for), for the scan's frequent hits.
__device__ __forceinline__ void red_min(unsigned long long* a, uint64_t p) { atomicMin(a, (unsigned long long)p); }

template <class M>
__device__ __forceinline__ uint64_t phi(const M& m, const uint64_t* __restrict__ H, uint64_t BL, uint64_t p,
                                        uint64_t len) {
  return m.sub(H[p + len], m.mul(H[p], BL));
}

template <class Slot>
__device__ __forceinline__ uint32_t t_insert(Slot* t, uint64_t mask, uint64_t key) {
  uint64_t h = mix64(key) & mask;
  for (uint64_t it = 0; it <= mask; it++) {
    unsigned long long old = *(volatile unsigned long long*)&t[h].key;
    if (old == kNone) old = atomicCAS(&t[h].key, (unsigned long long)kNone, (unsigned long long)key);
    if (old == kNone || old == key) return (uint32_t)h;
    h = (h + 1) & mask;
  }
  return kNoSlot;
}

template <class Slot>
__device__ __forceinline__ uint32_t t_find(const Slot* t, uint64_t mask, uint64_t key) {
  uint64_t h = mix64(key) & mask;
  for (uint64_t it = 0; it <= mask; it++) {
    const uint64_t k = t[h].key;
    if (k == key) return (uint32_t)h;
    if (k == kNone) return kNoSlot;
    h = (h + 1) & mask;
  }
  return kNoSlot;
}

// Exclusive prefix sum of in[0, n) into out[0, n]; out[n] = total.  in and
// out may be the same array.
__device__ void cta_scan_u32(const uint32_t* in, uint32_t* out, uint64_t n, Cta& C) {
  const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t carry = 0;
  for (uint64_t base = 0; base < n; base += blockDim.x) {
    const uint64_t i = base + threadIdx.x;
    const uint32_t v = i < n ? in[i] : 0u;
    uint32_t x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t o = __shfl_up_sync(kFull, x, d);
      if ((int)lane >= d) x += o;
    }
    if (lane == 31) C.wtot[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint32_t w = lane < nw ? C.wtot[lane] : 0u;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t o = __shfl_up_sync(kFull, w, d);
        if ((int)lane >= d) w += o;
      }
      C.wtot[lane] = w;
    }
    __syncthreads();
    const uint32_t before = warp ? C.wtot[warp - 1] : 0u;
    if (i < n) out[i] = carry + before + x - v;
    const uint32_t tot = C.wtot[nw - 1];
    __syncthreads();
    carry += tot;
  }
  if (threadIdx.x == 0) out[n] = carry;
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Level geometry.
// ---------------------------------------------------------------------------
struct LV {
  const uint8_t* T;
  uint64_t n, c, b;
  uint64_t* st;
};

__device__ __forceinline__ uint64_t blen(const LV& g, uint64_t k) {
  const uint64_t s = g.st[k];
  return g.n - s < g.b ? g.n - s : g.b;
}

// End of block k and of up to two following blocks consecutive with it.
__device__ __forceinline__ uint64_t avail_end(const LV& g, uint64_t k) {
  uint64_t e = g.st[k] + blen(g, k);
  if (k + 1 < g.c && g.st[k + 1] == e) {
    e += blen(g, k + 1);
    if (k + 2 < g.c && g.st[k + 2] == e) e += blen(g, k + 2);
  }
  return e;
}

__device__ __forceinline__ bool marked(const uint32_t* mw, uint64_t k) { return (mw[k >> 5] >> (k & 31)) & 1u; }
__device__ __forceinline__ uint64_t mrank(const uint32_t* mw, const uint32_t* mr, uint64_t k) {
  return mr[k >> 5] + __popc(mw[k >> 5] & ((1u << (k & 31)) - 1u));
}

// 16 bytes of T starting at any x, from the two aligned 16-byte units that
// cover them (the text buffer is padded, so the second unit is readable).
__device__ __forceinline__ uint4 load16u(const uint8_t* __restrict__ T, uint64_t x) {
  const uint64_t x0 = x & ~15ull;
  const uint32_t d = (uint32_t)(x & 15);
  const uint4 u0 = *(const uint4*)(T + x0);
  if (d == 0) return u0;
  const uint4 u1 = *(const uint4*)(T + x0 + 16);
  const uint32_t q = d >> 2, sh = 8 * (d & 3);
  const uint32_t w[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
  uint32_t o[5];
#pragma unroll
  for (int i = 0; i < 5; i++) o[i] = w[(q + i) & 7];
  return make_uint4(__funnelshift_r(o[0], o[1], sh), __funnelshift_r(o[1], o[2], sh),
                    __funnelshift_r(o[2], o[3], sh), __funnelshift_r(o[3], o[4], sh));
}

// Do T[a, a+len) and T[b, b+len) differ?  G lanes (lane gl of them) compare
// 16 bytes each per step.
__device__ __forceinline__ bool differs(const uint8_t* __restrict__ T, uint64_t a, uint64_t b, uint64_t len,
                                        unsigned gl, unsigned G) {
  bool diff = false;
  for (uint64_t y = 16ull * gl; y < len; y += 16ull * G) {
    const uint4 va = load16u(T, a + y), vb = load16u(T, b + y);
    const uint64_t cnt = len - y < 16 ? len - y : 16;
    const uint32_t xa[4] = {va.x ^ vb.x, va.y ^ vb.y, va.z ^ vb.z, va.w ^ vb.w};
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const uint64_t lo = 4ull * q;
      if (lo >= cnt) break;
      const uint32_t mk = cnt - lo >= 4 ? kFull : ((1u << (8 * (cnt - lo))) - 1u);
      diff |= (xa[q] & mk) != 0;
    }
  }
  return diff;
}

// Verify jobs[0, nj): mismatch[i] = 1 when the two ranges differ.  Groups of
// G lanes (about len/16, a power of two up to 32) take one job each.
__device__ void verify_jobs(const uint8_t* __restrict__ T, const BJob* jobs, uint32_t nj, uint64_t maxlen,
                            unsigned int* mismatch) {
  unsigned G = 1;
  while (G < 32 && 16ull * G < maxlen) G <<= 1;
  const unsigned lane = threadIdx.x & 31, grp = lane / G, gl = lane % G, gpw = 32 / G;
  const unsigned gmask = (G == 32 ? kFull : ((1u << G) - 1u)) << (grp * G);
  const unsigned nw = blockDim.x >> 5, warp = threadIdx.x >> 5;
  // Warp-uniform loop: every lane reaches every ballot.
  for (uint64_t base = (uint64_t)warp * gpw; base < nj; base += (uint64_t)nw * gpw) {
    const uint64_t j = base + grp;
    bool diff = false;
    if (j < nj) {
      const BJob J = jobs[j];
      diff = differs(T, J.a, J.b, J.len, gl, G);
    }
    const unsigned bal = __ballot_sync(kFull, diff);
    if (j < nj && gl == 0) mismatch[j] = (bal & gmask) ? 1u : 0u;
  }
}

// ---------------------------------------------------------------------------
// Document set-up: alphabet and prefix fingerprints.
// ---------------------------------------------------------------------------
__device__ void alphabet(const uint8_t* __restrict__ T, uint64_t n, uint32_t sigma, Cta& C) {
  for (uint32_t i = threadIdx.x; i < 256; i += blockDim.x) C.hist[i] = 0;
  __syncthreads();
  const uint64_t nv = n / 16;
  for (uint64_t i = threadIdx.x; i < nv; i += blockDim.x) {
    const uint4 q = ((const uint4*)T)[i];
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
      for (int s = 0; s < 4; s++) atomicAdd(&C.hist[(w[a] >> (8 * s)) & 0xFF], 1u);
  }
  for (uint64_t i = nv * 16 + threadIdx.x; i < n; i += blockDim.x) atomicAdd(&C.hist[T[i]], 1u);
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t S = 0;
    for (int i = 0; i < 256; i++) C.sym[i] = C.hist[i] ? (int16_t)S++ : (int16_t)-1;
    C.S = S;
    if (S > sigma) C.err = BT_EINVAL;
  }
  __syncthreads();
}

// H[p] for every p in [0, n]: chunks of 32 bytes, blockDim.x chunks per tile.
// pw[i] = X^i with X = B^32, i <= 1024.
template <class M>
__device__ void prefix_pass(const M& m, const uint8_t* __restrict__ T, uint64_t n, uint64_t B,
                            const uint64_t* __restrict__ pw, uint64_t* __restrict__ H, Cta& C) {
  const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const uint64_t tile = (uint64_t)blockDim.x * 32;
  if (threadIdx.x == 0) C.carry = 0;
  __syncthreads();
  for (uint64_t t0 = 0; t0 < n; t0 += tile) {
    const uint64_t carry = C.carry;
    const uint64_t p0 = t0 + 32ull * threadIdx.x;
    const uint32_t cnt = p0 < n ? (uint32_t)(n - p0 < 32 ? n - p0 : 32) : 0u;
    uint64_t h = 0;
    if (cnt == 32) {
      const uint4 v0 = *(const uint4*)(T + p0), v1 = *(const uint4*)(T + p0 + 16);
      const uint32_t wv[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
      for (int i = 0; i < 32; i++) h = m.add(m.mul(h, B), (uint64_t)((wv[i >> 2] >> (8 * (i & 3))) & 0xFFu) + 1);
    } else {
      for (uint32_t i = 0; i < cnt; i++) h = m.add(m.mul(h, B), (uint64_t)T[p0 + i] + 1);
    }
    // Inclusive scan of the chunk values (each chunk shifts by X = B^32).
    uint64_t x = h;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint64_t o = __shfl_up_sync(kFull, x, d);
      if ((int)lane >= d) x = m.add(m.mul(o, pw[d]), x);
    }
    if (lane == 31) C.wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint64_t w = lane < nw ? C.wsum[lane] : 0ull;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint64_t o = __shfl_up_sync(kFull, w, d);
        if ((int)lane >= d) w = m.add(m.mul(o, pw[32 * d]), w);
      }
      C.wsum[lane] = w;
    }
    __syncthreads();
    const uint64_t wp = warp ? C.wsum[warp - 1] : 0ull;
    const uint64_t incl = m.add(m.mul(wp, pw[lane + 1]), x);  // chunks [0, j] of the tile
    const uint64_t up = __shfl_up_sync(kFull, incl, 1);
    const uint64_t excl = lane ? up : wp;                      // chunks [0, j)
    uint64_t hh = m.add(m.mul(carry, pw[threadIdx.x]), excl);  // H(p0)
    if (cnt == 32) {
      const uint4 v0 = *(const uint4*)(T + p0), v1 = *(const uint4*)(T + p0 + 16);
      const uint32_t wv[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
      for (int i = 0; i < 32; i++) {
        H[p0 + i] = hh;
        hh = m.add(m.mul(hh, B), (uint64_t)((wv[i >> 2] >> (8 * (i & 3))) & 0xFFu) + 1);
      }
    } else {
      for (uint32_t i = 0; i < cnt; i++) {
        H[p0 + i] = hh;
        hh = m.add(m.mul(hh, B), (uint64_t)T[p0 + i] + 1);
      }
    }
    if (cnt && p0 + cnt == n) H[n] = hh;
    if (threadIdx.x == blockDim.x - 1) C.carry = m.add(m.mul(carry, pw[blockDim.x]), incl);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// One level.
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// Selected grams: the anchors of the window scan on levels with long blocks.
// A window's anchor is its first 16-byte gram whose hash is selected; a
// window equal to a key has the key's anchor gram at the key's anchor offset,
// so on those levels only the selected grams of the level's runs are read and
// each proposes the windows that would have it as their anchor.  The grams
// are selected once per document; a level looks them up in the list.
// ---------------------------------------------------------------------------
constexpr uint32_t kNoList = 0xFFFFFFFFu;        // the list overflowed: no anchors
constexpr unsigned long long kNoAnchor = ~0ull;  // empty anchor-table entry

__device__ __forceinline__ uint32_t gram_hash(uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3) {
  uint32_t h = w0 * 0x9E3779B1u;
  uint32_t t = w1 * 0x85EBCA77u;
  h ^= __funnelshift_l(t, t, 13);
  t = w2 * 0xC2B2AE3Du;
  h ^= __funnelshift_l(t, t, 7);
  t = w3 * 0x27D4EB2Fu;
  h ^= __funnelshift_l(t, t, 19);
  h ^= h >> 16;
  h *= 0x7FEB352Du;
  h ^= h >> 15;
  h *= 0x846CA68Bu;
  h ^= h >> 16;
  return h;
}

// Bit of the shared-memory filter for a window's first 8 bytes (lo, hi as
// little-endian words), the test of the blocks that have no selected gram.
__device__ __forceinline__ uint32_t prefix_bit(uint32_t lo, uint32_t hi, uint32_t fshift) {
  const uint32_t t = hi * 0x85EBCA77u;
  return ((lo * 0x9E3779B1u) ^ __funnelshift_l(t, t, 15)) * 0xC2B2AE3Du >> fshift;
}

__device__ __forceinline__ uint32_t anchor_slot(uint32_t g, uint64_t mask) {
  return (uint32_t)(((uint64_t)g * 0x9E3779B97F4A7C15ull >> 32) & mask);
}

// Exclusive sum of one value per thread over the CTA; *total = the sum.
__device__ uint32_t cta_excl_u32(uint32_t v, Cta& C, uint32_t* total) {
  const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t o = __shfl_up_sync(kFull, x, d);
    if ((int)lane >= d) x += o;
  }
  if (lane == 31) C.wtot[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < nw ? C.wtot[lane] : 0u;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t o = __shfl_up_sync(kFull, w, d);
      if ((int)lane >= d) w += o;
    }
    C.wtot[lane] = w;
  }
  __syncthreads();
  const uint32_t r = (warp ? C.wtot[warp - 1] : 0u) + x - v;
  *total = C.wtot[nw - 1];
  __syncthreads();
  return r;
}

// The selected grams of T[0, n) in text order: positions and hashes, at most
// cap of them (C.nsel = their number, or kNoList if there are more).  A
// thread takes 32 consecutive positions of a tile, from 12 aligned words
// (the text is followed by at least 48 readable bytes).
__device__ void gram_list_pass(const uint8_t* __restrict__ T, uint64_t n, uint32_t* __restrict__ lpos,
                               uint32_t* __restrict__ lhash, uint64_t cap, Cta& C) {
  if (threadIdx.x == 0) C.nsel = 0;
  __syncthreads();
  const uint64_t npos = n >= kGramW ? n - kGramW + 1 : 0;
  const uint64_t tile = (uint64_t)blockDim.x * 32;
  for (uint64_t t0 = 0; t0 < npos; t0 += tile) {
    const uint64_t x0 = t0 + 32ull * threadIdx.x;
    uint32_t w[12];
    uint32_t mask = 0;
    if (x0 < npos) {
      const uint32_t* wp = (const uint32_t*)(T + x0);
#pragma unroll
      for (int k = 0; k < 12; k++) w[k] = wp[k];
#pragma unroll
      for (int i = 0; i < 32; i++) {
        const int q = i >> 2, sh = 8 * (i & 3);
        const uint32_t h = gram_hash(__funnelshift_r(w[q], w[q + 1], sh), __funnelshift_r(w[q + 1], w[q + 2], sh),
                                     __funnelshift_r(w[q + 2], w[q + 3], sh), __funnelshift_r(w[q + 3], w[q + 4], sh));
        if ((h >> kGramSelShift) == 0 && x0 + i < npos) mask |= 1u << i;
      }
    }
    uint32_t total;
    const uint32_t before = cta_excl_u32(__popc(mask), C, &total);
    const uint32_t base = C.nsel;
    if (base != kNoList && (uint64_t)base + total <= cap) {
      uint32_t o = base + before;
#pragma unroll
      for (int i = 0; i < 32; i++) {
        if (!((mask >> i) & 1u)) continue;
        const int q = i >> 2, sh = 8 * (i & 3);
        lpos[o] = (uint32_t)(x0 + i);
        lhash[o] = gram_hash(__funnelshift_r(w[q], w[q + 1], sh), __funnelshift_r(w[q + 1], w[q + 2], sh),
                             __funnelshift_r(w[q + 2], w[q + 3], sh), __funnelshift_r(w[q + 3], w[q + 4], sh));
        o++;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) C.nsel = (base == kNoList || (uint64_t)base + total > cap) ? kNoList : base + total;
    __syncthreads();
  }
}

// First index i of the sorted a[0, n) with a[i] >= x.
__device__ __forceinline__ uint32_t lower_bound_u32(const uint32_t* __restrict__ a, uint32_t n, uint64_t x) {
  uint32_t lo = 0, hi = n;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

struct Work {
  uint64_t *fpB, *job_of, *susp, *exBL;
  unsigned long long* exlo;
  uint32_t *slotB, *slotP, *wpop;
  unsigned int* mismatch;
  uint8_t* pm;
  BJob* jobs;
  BSlot* bt;
  PSlot* pt;
  unsigned long long* at;  // anchor table: (gram hash << 32) | anchor offset
};

__device__ __forceinline__ char* carve(char*& p, uint64_t bytes) {
  char* q = p;
  p += out_align(bytes);
  return q;
}

__device__ Work carve_level(char* temp, uint64_t c, uint64_t bcap, uint64_t pcap) {
  Work W;
  char* p = temp;
  W.fpB = (uint64_t*)carve(p, c * 8 + 8);
  W.exBL = (uint64_t*)carve(p, c * 8 + 8);  // (the unused pair-lo slot of the layout)
  W.job_of = (uint64_t*)carve(p, c * 8 + 8);
  W.susp = (uint64_t*)carve(p, c * 8 + 8);
  W.exlo = (unsigned long long*)carve(p, c * 8 + 8);
  W.slotB = (uint32_t*)carve(p, c * 4 + 4);
  W.slotP = (uint32_t*)carve(p, c * 4 + 4);
  W.mismatch = (unsigned int*)carve(p, c * 4 + 4);
  W.wpop = (uint32_t*)carve(p, c * 4 + 4);
  W.pm = (uint8_t*)carve(p, c + 8);
  W.jobs = (BJob*)carve(p, c * 32 + 32);
  carve(p, c * 8 + 8);
  W.bt = (BSlot*)carve(p, bcap * 32);
  W.pt = (PSlot*)carve(p, pcap * 16);
  W.at = (unsigned long long*)carve(p, bcap * 8);
  return W;
}

// Exact leftmost occurrence of every suspect key (a fingerprint collision
// was found by verification): every window before the key's start, inside a
// run, whose fingerprint equals the key's is compared byte by byte.
template <class M>
__device__ void exact_pass(const M& m, const LV& g, const uint64_t* H, const Work& W, int pair, uint64_t B,
                           Cta& C) {
  const uint32_t ns = C.nsusp;
  // Key fingerprint, length and B^length of each suspect (in the job array).
  for (uint32_t i = threadIdx.x; i < ns; i += blockDim.x) {
    const uint64_t k = W.susp[i];
    uint64_t klen = blen(g, k), kfp = W.fpB[k];
    if (pair) {
      const uint64_t l2 = blen(g, k + 1);
      kfp = m.add(m.mul(kfp, pow_mod(m, B, l2)), W.fpB[k + 1]);
      klen += l2;
    }
    W.jobs[i] = BJob{kfp, pow_mod(m, B, klen), klen, g.st[k]};
  }
  __syncthreads();
  const uint64_t per = g.c * g.b;
  for (uint64_t w = threadIdx.x; w < (uint64_t)ns * per; w += blockDim.x) {
    const uint64_t i = w / per, rest = w - i * per;
    const uint64_t k = rest / g.b, j = rest - k * g.b;
    if (j >= blen(g, k)) continue;
    const BJob J = W.jobs[i];
    const uint64_t p = g.st[k] + j;
    if (p >= J.idx) continue;
    if (p + J.len > avail_end(g, k)) continue;
    if (phi(m, H, J.b, p, J.len) != J.a) continue;
    bool eq = true;
    for (uint64_t x = 0; x < J.len && eq; x++) eq = g.T[p + x] == g.T[J.idx + x];
    if (eq) min_pos(&W.exlo[i], p);
  }
  __syncthreads();
}

// A window of the scan whose fingerprint passed the filter: the block-table
// probe; for a match, the slot minimum, the pair that ends in the short tail,
// and the pair joined at p + b.  Out of line: matches are few, and the scan
// loop keeps its registers for the loads in flight.
struct ScanArgs {
  const uint64_t* H;
  BSlot* bt;
  PSlot* pt;
  uint64_t bmask, pmask, b, r, Bb, Br, fp_tail;
  uint32_t pretail;
  unsigned long long* lo_tailpair;
};

template <class M>
__device__ __forceinline__ void window_hit(const M& m, const ScanArgs& A, uint64_t p, uint64_t av, uint64_t x,
                                        uint64_t hb) {
  const uint32_t sl = t_find(A.bt, A.bmask, x);
  if (sl == kNoSlot) return;
  red_min(&A.bt[sl].lo, p);
  if (A.r && sl == A.pretail && p + A.b + A.r <= av && m.sub(A.H[p + A.b + A.r], m.mul(hb, A.Br)) == A.fp_tail)
    min_pos(A.lo_tailpair, p);
  if (p <= A.bt[sl].maxpst && p + 2 * A.b <= av) {
    const uint64_t fp2 = m.sub(A.H[p + 2 * A.b], m.mul(hb, A.Bb));
    const uint32_t s2 = t_find(A.bt, A.bmask, fp2);
    if (s2 != kNoSlot) {
      const uint32_t ps = t_find(A.pt, A.pmask, ((uint64_t)sl << 32) | s2);
      if (ps != kNoSlot) red_min(&A.pt[ps].lo, p);
    }
  }
}

template <class M>
__device__ void level_pass(const M& m, const BParams& P, const BDoc& D, Cta& C, char* scr, uint32_t l,
                           uint32_t* filt, uint32_t filt_words_max) {
  const uint64_t* bsz = P.sizes + D.lv_off;
  const uint64_t n = C.n, c = C.c[l], b = bsz[l];
  const bool last = l + 1 == C.L;
  const unsigned tid = threadIdx.x, nt = blockDim.x;
  LV g{D.T, n, c, b, (uint64_t*)(scr + C.sl.st[l])};
  const uint64_t* H = (const uint64_t*)(scr + C.sl.H);
  uint64_t* lo = (uint64_t*)(scr + C.sl.lo[l]);
  uint64_t* off = (uint64_t*)(scr + C.sl.off[l]);
  uint32_t* ptr = (uint32_t*)(scr + C.sl.ptr[l]);
  uint32_t* mw = (uint32_t*)(scr + C.sl.mw[l]);
  uint32_t* mr = (uint32_t*)(scr + C.sl.mr[l]);
  const uint64_t bcap = pow2_ge(2 * c), pcap = pow2_ge(2 * c);
  const Work W = carve_level(scr + C.sl.temp, c, bcap, pcap);

  if (tid == 0) {
    const uint64_t len_last = n - C.last_start;
    C.r = len_last < b ? len_last : 0;
    C.Bb = pow_mod(m, P.B, b);
    C.Br = C.r ? pow_mod(m, P.B, C.r) : 0;
    C.B1 = P.B % m.q();
    C.bmask = bcap - 1;
    C.pmask = pcap - 1;
    C.bshift = (b & (b - 1)) == 0 ? (uint32_t)(__ffsll((long long)b) - 1) : 0xFFu;
    C.fp_tail = kNone;
    C.lo_tail = kNone;
    C.lo_tailpair = kNone;
    C.pretail = kNoSlot;
    C.npairs = 0;
    C.njobs = 0;
    C.nsusp = 0;
    C.verify_bytes = 0;
    C.collisions = 0;
    C.lastk = 0;
  }
  for (uint64_t i = tid; i < bcap; i += nt) W.bt[i] = BSlot{kNone, kNone, 0, 0};
  for (uint64_t i = tid; i < pcap; i += nt) W.pt[i] = PSlot{kNone, kNone};
  for (uint64_t i = tid; i < c; i += nt) W.mismatch[i] = 0;
  __syncthreads();
  tmark(C, 3);
  const uint64_t r = C.r, Bb = C.Bb, Br = C.Br, bmask = C.bmask, pmask = C.pmask;

  // Block fingerprints; full-length blocks into the block table (the slot's
  // leftmost window starts at the block's own start).
  for (uint64_t k = tid; k < c; k += nt) {
    const uint64_t s = g.st[k], len = blen(g, k);
    const uint64_t fp = phi(m, H, len == b ? Bb : Br, s, len);
    W.fpB[k] = fp;
    if (len == b) {
      const uint32_t slot = t_insert(W.bt, bmask, fp);
      W.slotB[k] = slot;
      if (slot == kNoSlot) {
        fail(C, BT_EINTERNAL);
        continue;
      }
      min_pos(&W.bt[slot].lo, s);
    } else {
      W.slotB[k] = kNoSlot;
      C.fp_tail = fp;
      atomicMin(&C.lo_tail, (unsigned long long)s);
    }
  }
  if (cta_failed(C)) return;
  // Pairs of consecutive blocks: one pair-table slot per (slot, slot); the
  // pair ending in the short tail is kept in the CTA's scalars.
  for (uint64_t k = tid; k + 1 < c; k += nt) {
    W.slotP[k] = kNoSlot;
    if (g.st[k + 1] != g.st[k] + b) continue;
    atomicAdd(&C.npairs, 1u);
    const uint32_t sk = W.slotB[k];
    if (sk == kNoSlot) {
      fail(C, BT_EINTERNAL);
      continue;
    }
    if (*(volatile unsigned long long*)&W.bt[sk].maxpst < g.st[k])
      atomicMax(&W.bt[sk].maxpst, (unsigned long long)g.st[k]);
    if (W.slotB[k + 1] == kNoSlot) {
      W.slotP[k] = kBTailPair;
      C.pretail = sk;
      atomicMin(&C.lo_tailpair, (unsigned long long)g.st[k]);
    } else {
      const uint32_t sp = t_insert(W.pt, pmask, ((uint64_t)sk << 32) | W.slotB[k + 1]);
      W.slotP[k] = sp;
      if (sp == kNoSlot) {
        fail(C, BT_EINTERNAL);
        continue;
      }
      min_pos(&W.pt[sp].lo, g.st[k]);
    }
  }
  if (cta_failed(C)) return;
  // Levels of long blocks scan by anchors: every full-length block registers
  // its first selected gram (hash, offset from the block's start) in the
  // anchor table, each distinct (hash, offset) once.  Registering every block,
  // not one per table slot, keeps the proposals complete when different
  // contents share a fingerprint.  A block without a selected gram puts its
  // first 8 bytes into the shared-memory filter instead, and the scan then
  // also tests every window's first 8 bytes against it.
  const uint32_t* lpos = (const uint32_t*)(scr + C.sl.lpos);
  const uint32_t* lhash = (const uint32_t*)(scr + C.sl.lhash);
  const uint32_t nsel = C.nsel;
  const uint64_t amask = bcap - 1;
  uint32_t fwords = 32, fshift = 32 - 10;  // 32 words = 2^10 bits
  while (fwords < c && fwords < filt_words_max) {
    fwords <<= 1;
    fshift--;
  }
  const bool anch = b >= P.anchor_min_b && nsel != kNoList;
  if (anch) {
    if (tid == 0) {
      C.anchorless = 0;
      C.tail_anchored = 0;
      if (r >= kGramW) {
        const uint64_t ts = C.last_start;
        const uint32_t j = lower_bound_u32(lpos, nsel, ts);
        if (j < nsel && lpos[j] + kGramW <= ts + r) {
          C.tail_g = lhash[j];
          C.tail_a = (uint32_t)(lpos[j] - ts);
          C.tail_anchored = 1;
        }
      }
    }
    for (uint64_t i = tid; i < bcap; i += nt) W.at[i] = kNoAnchor;
    for (uint32_t i = tid; i < fwords; i += nt) filt[i] = 0;
    __syncthreads();
    for (uint64_t k = tid; k < c; k += nt) {
      if (W.slotB[k] == kNoSlot) continue;
      const uint64_t s0 = g.st[k];
      const uint32_t j = lower_bound_u32(lpos, nsel, s0);
      if (j >= nsel || lpos[j] + kGramW > s0 + b) {
        // No selected gram: the block's first 8 bytes go to the filter that
        // the per-window pass of the scan tests.
        const uint32_t* w3 = (const uint32_t*)(D.T + (s0 & ~3ull));
        const uint32_t sh = 8 * (uint32_t)(s0 & 3);
        const uint32_t bit = prefix_bit(__funnelshift_r(w3[0], w3[1], sh), __funnelshift_r(w3[1], w3[2], sh), fshift);
        atomicOr(&filt[bit >> 5], 1u << (bit & 31));
        atomicAdd(&C.anchorless, 1u);
        continue;
      }
      const unsigned long long e = ((unsigned long long)lhash[j] << 32) | (uint32_t)(lpos[j] - s0);
      uint32_t h = anchor_slot(lhash[j], amask);
      for (uint64_t it = 0; it <= amask; it++) {
        const unsigned long long cur = *(volatile unsigned long long*)&W.at[h];
        if (cur == e) break;
        if (cur == kNoAnchor) {
          const unsigned long long old = atomicCAS(&W.at[h], kNoAnchor, e);
          if (old == kNoAnchor || old == e) break;
        }
        h = (uint32_t)((h + 1) & amask);
      }
    }
    __syncthreads();
  }
  // A bitmap of the full-length block fingerprints in shared memory (about
  // 32 bits per key): a window whose fingerprint's bit is clear matches no
  // key, so only the few that pass probe the table in global memory.
  const uint64_t fmask = (uint64_t)fwords * 32 - 1;
  if (!anch) {
    for (uint32_t i = tid; i < fwords; i += nt) filt[i] = 0;
    for (uint32_t a = tid; a < 256; a += nt) C.rtab[a] = m.mul(a + 1, Bb);
    __syncthreads();
    for (uint64_t k = tid; k < c; k += nt)
      if (W.slotB[k] != kNoSlot) {
        const uint64_t bit = W.fpB[k] & fmask;
        atomicOr(&filt[bit >> 5], 1u << (bit & 31));
      }
  }
  __syncthreads();
  tmark(C, 1);

  // The window scan: every window [p, p+b) inside a run (and [p, p+r) for the
  // short tail).  When b is a multiple of 32, a warp takes CH = 32 Re
  // consecutive positions of one block (block, run end and bounds are warp
  // values, positions 32-bit) and lane l the Re positions from p0 + l Re,
  // rolling the fingerprint from one to the next.  Otherwise every thread
  // maps its positions to blocks itself.  The short tail's windows are tested only where their first four
  // bytes equal the tail's.
  {
    const uint32_t pretail = C.pretail, bshift = C.bshift;
    const uint64_t fp_tail = C.fp_tail;
    uint32_t tail4 = 0, tail4_mask = 0;
    if (r) {
      const uint64_t ts = C.last_start;
      for (uint32_t i = 0; i < 4 && i < r; i++) {
        tail4 |= (uint32_t)D.T[ts + i] << (8 * i);
        tail4_mask |= 0xFFu << (8 * i);
      }
    }
    const ScanArgs A{H, W.bt, W.pt, bmask, pmask, b, r, Bb, Br, fp_tail, pretail, &C.lo_tailpair};
    if (anch) {
      // A warp per present block k: its selected grams x (the list entries
      // in [s_k, s_k + len_k)) propose, for every key anchored on the gram's
      // hash at offset a, the window at p = x - a.  As a < b, p lies in
      // block k or in block k-1 when that one ends where k starts; the
      // window must end within the run of p's block.
      const unsigned lane = tid & 31, nw = nt >> 5;
      const bool tail_anch = r && C.tail_anchored;
      const uint32_t tail_g = C.tail_g, tail_a = C.tail_a;
      for (uint64_t k = tid >> 5; k < c; k += nw) {
        const uint64_t s = g.st[k];
        const uint64_t len = n - s < b ? n - s : b, e0 = s + len;
        uint64_t av = e0;  // run end of block k
        uint64_t nxt = 0;  // length of block k+1 when it follows k
        if (k + 1 < c && g.st[k + 1] == e0) {
          nxt = n - e0 < b ? n - e0 : b;
          av = e0 + nxt;
          if (k + 2 < c && g.st[k + 2] == av) av += n - av < b ? n - av : b;
        }
        const bool prev = k > 0 && g.st[k - 1] + b == s;  // block k-1 ends where k starts
        const uint64_t av_prev = e0 + nxt;                // run end of block k-1
        uint32_t j0 = 0, j1 = 0;
        if (lane == 0) {
          j0 = lower_bound_u32(lpos, nsel, s);
          j1 = lower_bound_u32(lpos, nsel, e0);
        }
        j0 = __shfl_sync(kFull, j0, 0);
        j1 = __shfl_sync(kFull, j1, 0);
        for (uint32_t j = j0 + lane; j < j1; j += 32) {
          const uint64_t x = lpos[j];
          const uint32_t gh = lhash[j];
          uint32_t h = anchor_slot(gh, amask);
          for (uint64_t it = 0; it <= amask; it++) {
            const unsigned long long en = W.at[h];
            if (en == kNoAnchor) break;
            if ((uint32_t)(en >> 32) == gh && (uint32_t)en <= x) {
              const uint64_t p = x - (uint32_t)en;
              const uint64_t pav = p >= s ? av : (prev ? av_prev : 0);
              if (p + b <= pav) {
                const uint64_t hb = H[p + b];
                window_hit(m, A, p, pav, m.sub(hb, m.mul(H[p], Bb)), hb);
              }
            }
            h = (uint32_t)((h + 1) & amask);
          }
          if (tail_anch && gh == tail_g && tail_a <= x) {
            const uint64_t p = x - tail_a;
            const uint64_t pav = p >= s ? av : (prev ? av_prev : 0);
            if (p + r <= pav && phi(m, H, Br, p, r) == fp_tail) min_pos(&C.lo_tail, p);
          }
        }
      }
      const uint32_t nal = C.anchorless;
      if (nal || (r && !tail_anch)) {
        // Blocks without a selected gram, and the short tail without one:
        // every window, where its first 8 bytes pass the blocks' filter
        // (then its fingerprint decides) or its first 4 bytes equal the
        // tail's.  A warp takes 256 consecutive positions of a block, a lane
        // 8 of them, from 5 aligned words.
        constexpr uint32_t Rp = 8, CHp = 32 * Rp;
        const uint64_t cpbp = (b + CHp - 1) / CHp;
        const bool all_present = c == (n + b - 1) / b;
        const uint8_t* T = D.T;
        for (uint64_t item = tid >> 5; item < c * cpbp; item += nw) {
          const uint64_t k = item / cpbp, jc = item - k * cpbp;
          uint64_t s, av;
          if (all_present) {
            s = k * b;
            av = (k + 3) * b < n ? (k + 3) * b : n;
          } else {
            s = g.st[k];
            const uint64_t s1 = k + 1 < c ? g.st[k + 1] : kNone, s2 = k + 2 < c ? g.st[k + 2] : kNone;
            const uint64_t e0 = s + (n - s < b ? n - s : b);
            av = e0;
            if (s1 == e0) {
              av = s1 + (n - s1 < b ? n - s1 : b);
              if (s2 == av) av = s2 + (n - s2 < b ? n - s2 : b);
            }
          }
          const uint64_t send = s + (n - s < b ? n - s : b);
          const uint64_t p = s + jc * CHp + lane * Rp;
          if (p >= send) continue;
          const uint64_t pend = p + Rp < send ? p + Rp : send;
          const uint32_t* wa = (const uint32_t*)(T + (p & ~3ull));
          const uint32_t sa = 8 * (uint32_t)(p & 3);
          uint32_t t[4];
          {
            uint32_t w[5];
#pragma unroll
            for (int q = 0; q < 5; q++) w[q] = wa[q];
#pragma unroll
            for (int q = 0; q < 4; q++) t[q] = __funnelshift_r(w[q], w[q + 1], sa);
          }
#pragma unroll
          for (uint32_t i = 0; i < Rp; i++) {
            const uint64_t q = p + i;
            if (q >= pend) break;
            const uint32_t lo = __funnelshift_r(t[i >> 2], t[(i >> 2) + 1], 8 * (i & 3));
            if (nal && q + b <= av) {
              const uint32_t hi = __funnelshift_r(t[(i >> 2) + 1], t[(i >> 2) + 2], 8 * (i & 3));
              const uint32_t bit = prefix_bit(lo, hi, fshift);
              if ((filt[bit >> 5] >> (bit & 31)) & 1u) {
                const uint64_t hb = H[q + b];
                window_hit(m, A, q, av, m.sub(hb, m.mul(H[q], Bb)), hb);
              }
            }
            if (r && !tail_anch && q + r <= av && (lo & tail4_mask) == tail4 && phi(m, H, Br, q, r) == fp_tail)
              min_pos(&C.lo_tail, q);
          }
        }
      }
    } else if (b % 32 == 0) {
      // A lane takes a run of Re consecutive positions: the first window's
      // fingerprint comes from two prefix fingerprints, each next one rolls
      // in one step from the text bytes, phi(p+1, p+1+b) = B phi(p, p+b) +
      // (T[p+b] + 1) - (T[p] + 1) B^b (the last term from a table in shared
      // memory), so the loads per window are a few text bytes.
      constexpr int R = 8;
      const uint32_t Rmax = P.scan_u && P.scan_u < (uint32_t)R ? P.scan_u : (uint32_t)R;
      const uint32_t Re = b / 32 < Rmax ? (uint32_t)(b / 32) : Rmax;  // positions per lane
      const uint32_t CH = 32 * Re;
      const uint64_t cpb = (b + CH - 1) / CH;
      const unsigned lane = tid & 31, nw = nt >> 5;
      const uint8_t* T = D.T;
      const uint64_t B1 = C.B1;
      const uint64_t* rtab = C.rtab;
      // Every block of the level present: block k starts at k b and its run
      // ends at min(n, (k + 3) b), with no loads.
      const bool all_present = c == (n + b - 1) / b;
      for (uint64_t item = tid >> 5; item < c * cpb; item += nw) {
        const uint64_t k = item / cpb, jc = item - k * cpb;
        uint64_t s, av;
        if (all_present) {
          s = k * b;
          av = (k + 3) * b < n ? (k + 3) * b : n;
        } else {
          // The three starts are loaded together, then the run end follows.
          s = g.st[k];
          const uint64_t s1 = k + 1 < c ? g.st[k + 1] : kNone, s2 = k + 2 < c ? g.st[k + 2] : kNone;
          const uint64_t e0 = s + (n - s < b ? n - s : b);
          av = e0;
          if (s1 == e0) {
            av = s1 + (n - s1 < b ? n - s1 : b);
            if (s2 == av) av = s2 + (n - s2 < b ? n - s2 : b);
          }
        }
        const uint64_t send = s + (n - s < b ? n - s : b);
        const uint32_t p = (uint32_t)(s + jc * CH + lane * Re);
        if (p >= send) continue;
        const uint32_t pend = (uint32_t)(p + Re < send ? p + Re : send);
        // Text bytes [p, p+12) and [p+b, p+b+8) from aligned words (a
        // document's bytes are followed by at least 48 readable bytes).
        const uint32_t* wa = (const uint32_t*)(T + (p & ~3u));
        const uint32_t sa = 8 * (p & 3);
        const uint32_t a0 = wa[0], a1 = wa[1], a2 = wa[2];
        const uint32_t ta0 = __funnelshift_r(a0, a1, sa), ta1 = __funnelshift_r(a1, a2, sa);
        uint32_t ta2 = 0;
        if (r) ta2 = __funnelshift_r(a2, wa[3], sa);
        const bool full0 = p + b <= av;
        uint64_t x = 0;
        uint32_t tb0 = 0, tb1 = 0;
        if (full0) {
          const uint32_t q = p + (uint32_t)b;
          const uint32_t* wb = (const uint32_t*)(T + (q & ~3u));
          const uint32_t sb = 8 * (q & 3);
          const uint32_t b0 = wb[0], b1 = wb[1], b2 = wb[2];
          tb0 = __funnelshift_r(b0, b1, sb);
          tb1 = __funnelshift_r(b1, b2, sb);
          x = m.sub(H[q], m.mul(H[p], Bb));
        }
#pragma unroll
        for (int i = 0; i < R; i++) {
          if (i >= (int)Re) break;
          const uint32_t q = p + i;
          if (q >= pend) break;
          if (q + b <= av) {
            const uint64_t bit = x & fmask;
            if ((filt[bit >> 5] >> (bit & 31)) & 1u) window_hit(m, A, q, av, x, H[q + b]);
            if (i + 1 < R) {
              const uint32_t lo = i < 4 ? ta0 : ta1, ins = i < 4 ? tb0 : tb1;
              const uint32_t sh = 8 * (i & 3);
              x = m.sub(m.add(m.mul(x, B1), ((ins >> sh) & 0xFFu) + 1), rtab[(lo >> sh) & 0xFFu]);
            }
          }
          if (r && q + r <= av) {
            const uint32_t v = i < 4 ? __funnelshift_r(ta0, ta1, 8 * (i & 3)) : __funnelshift_r(ta1, ta2, 8 * (i & 3));
            if ((v & tail4_mask) == tail4 && phi(m, H, Br, q, r) == fp_tail) min_pos(&C.lo_tail, q);
          }
        }
      }
    } else {
      for (uint64_t w = tid; w < c * b; w += nt) {
        const uint64_t k = bshift != 0xFFu ? w >> bshift : w / b;
        const uint64_t j = w - k * b;
        if (j >= blen(g, k)) continue;
        const uint64_t p = g.st[k] + j, av = avail_end(g, k);
        if (p + b <= av) {
          const uint64_t hb = H[p + b];
          const uint64_t x = m.sub(hb, m.mul(H[p], Bb));
          const uint64_t bit = x & fmask;
          if ((filt[bit >> 5] >> (bit & 31)) & 1u) window_hit(m, A, p, av, x, hb);
        }
        if (r && p + r <= av && phi(m, H, Br, p, r) == fp_tail) min_pos(&C.lo_tail, p);
      }
    }
  }
  __syncthreads();
  tmark(C, 2);

  // Pairs: leftmost when the minimum is the pair's own start; otherwise the
  // earlier occurrence is verified.
  for (uint64_t k = tid; k + 1 < c; k += nt) {
    W.pm[k] = 0;
    W.job_of[k] = kNone;
    const uint32_t sp = W.slotP[k];
    if (sp == kNoSlot) continue;
    const uint64_t lp = sp == kBTailPair ? C.lo_tailpair : W.pt[sp].lo;
    const uint64_t s = g.st[k];
    if (lp == s) {
      W.pm[k] = 1;
    } else if (lp < s) {
      const uint64_t len = b + blen(g, k + 1);
      const uint32_t id = atomicAdd(&C.njobs, 1u);
      W.jobs[id] = BJob{lp, s, len, k};
      W.job_of[k] = id;
      atomicAdd(&C.verify_bytes, 2ull * len);
    } else {
      fail(C, BT_EINTERNAL);  // the pair's own window was not seen
    }
  }
  if (cta_failed(C)) return;
  verify_jobs(g.T, W.jobs, C.njobs, 2 * b, W.mismatch);
  __syncthreads();
  for (uint64_t k = tid; k + 1 < c; k += nt) {
    const uint64_t id = W.job_of[k];
    if (id == kNone || !W.mismatch[id]) continue;
    atomicAdd(&C.collisions, 1ull);
    const uint32_t i = atomicAdd(&C.nsusp, 1u);
    W.susp[i] = k;
    W.exlo[i] = g.st[k];
  }
  __syncthreads();
  if (C.nsusp) {
    exact_pass(m, g, H, W, 1, P.B, C);
    for (uint32_t i = tid; i < C.nsusp; i += nt) W.pm[W.susp[i]] = W.exlo[i] == g.st[W.susp[i]];
    __syncthreads();
  }

  // Marks: a block in a leftmost pair, or in no pair.
  const uint64_t words = (c + 31) / 32;
  {
    const unsigned lane = tid & 31, nw = nt >> 5;
    for (uint64_t wb = tid >> 5; wb < words; wb += nw) {
      const uint64_t k = wb * 32 + lane;
      bool mk = false;
      if (k < c) {
        const bool left = k > 0 && W.slotP[k - 1] != kNoSlot;
        const bool right = k + 1 < c && W.slotP[k] != kNoSlot;
        mk = (left && W.pm[k - 1]) || (right && W.pm[k]) || (!left && !right);
      }
      const uint32_t bits = __ballot_sync(kFull, mk);
      if (lane == 0) {
        mw[wb] = bits;
        W.wpop[wb] = __popc(bits);
      }
    }
  }
  __syncthreads();
  cta_scan_u32(W.wpop, mr, words, C);

  // Leftmost occurrence of every block that becomes a pointer (of every
  // block when pruning needs it), verified.
  if (tid == 0) {
    C.njobs = 0;
    C.nsusp = 0;
  }
  for (uint64_t i = tid; i < c; i += nt) W.mismatch[i] = 0;
  __syncthreads();
  for (uint64_t k = tid; k < c; k += nt) {
    W.job_of[k] = kNone;
    lo[k] = kNone;
    if (!P.prune && marked(mw, k)) continue;
    const uint64_t s = g.st[k], len = blen(g, k);
    const uint64_t p = W.slotB[k] == kNoSlot ? C.lo_tail : W.bt[W.slotB[k]].lo;
    lo[k] = p;
    if (p < s) {
      const uint32_t id = atomicAdd(&C.njobs, 1u);
      W.jobs[id] = BJob{p, s, len, k};
      W.job_of[k] = id;
      atomicAdd(&C.verify_bytes, 2ull * len);
    } else if (p > s) {
      fail(C, BT_EINTERNAL);
    }
  }
  if (cta_failed(C)) return;
  verify_jobs(g.T, W.jobs, C.njobs, b, W.mismatch);
  __syncthreads();
  for (uint64_t k = tid; k < c; k += nt) {
    const uint64_t id = W.job_of[k];
    if (id == kNone || !W.mismatch[id]) continue;
    atomicAdd(&C.collisions, 1ull);
    const uint32_t i = atomicAdd(&C.nsusp, 1u);
    W.susp[i] = k;
    W.exlo[i] = g.st[k];
  }
  __syncthreads();
  if (C.nsusp) {
    exact_pass(m, g, H, W, 0, P.B, C);
    for (uint32_t i = tid; i < C.nsusp; i += nt) lo[W.susp[i]] = W.exlo[i];
    __syncthreads();
  }

  // Pointers of unmarked blocks: the block holding the leftmost occurrence
  // and the offset into it.
  for (uint64_t k = tid; k < c; k += nt) {
    if (marked(mw, k)) {
      ptr[k] = 0;
      off[k] = 0;
      continue;
    }
    const uint64_t p = lo[k], len = blen(g, k);
    uint64_t a = 0, z = c;
    while (a < z) {
      const uint64_t mid = (a + z) / 2;
      if (g.st[mid] <= p) a = mid + 1;
      else z = mid;
    }
    bool ok = a > 0;
    const uint64_t j = a - 1;
    if (ok) ok = p < g.st[j] + blen(g, j) && marked(mw, j) && p + len <= g.st[k];
    if (ok && p + len > g.st[j] + blen(g, j))
      ok = j + 1 < c && g.st[j + 1] == g.st[j] + blen(g, j) && marked(mw, j + 1);
    if (!ok) {
      fail(C, BT_EINTERNAL);
      continue;
    }
    ptr[k] = (uint32_t)j;
    off[k] = p - g.st[j];
  }
  if (cta_failed(C)) return;

  const uint64_t nm = mr[words];
  if (tid == 0) {
    C.nmarked[l] = nm;
    uint64_t* S = C.stats[l];
    S[BT_ST_NBLOCKS] = c;
    S[BT_ST_B] = b;
    S[BT_ST_COV] = (c - 1) * b + blen(g, c - 1);
    S[BT_ST_NMARKED] = nm;
    S[BT_ST_NPAIRS] = C.npairs;
    S[BT_ST_VERIFY_BYTES] = C.verify_bytes;
    S[BT_ST_COLLISIONS] = C.collisions;
    S[BT_ST_FINAL_BLOCKS] = c;
    S[BT_ST_CANDIDATES] = 0;
    S[BT_ST_HITS] = 0;
  }
  if (last) {
    if (tid == 0) C.arity[l] = 0;
    __syncthreads();
    tmark(C, 3);
    return;
  }
  // Children of marked blocks: rank r puts its children at r*arity + i.
  const uint64_t bn = bsz[l + 1];
  const uint32_t arity = (uint32_t)(b / bn);
  uint64_t* nst = (uint64_t*)(scr + C.sl.st[l + 1]);
  for (uint64_t wb = tid; wb < words; wb += nt)
    if (mw[wb]) atomicMax(&C.lastk, (unsigned long long)(wb * 32 + 31 - __clz(mw[wb])));
  __syncthreads();
  if (tid == 0) {
    C.arity[l] = arity;
    const uint64_t lk = C.lastk;
    if (nm == 0) {
      C.err = BT_EINTERNAL;
    } else {
      const uint64_t nch = (blen(g, lk) + bn - 1) / bn;
      const uint64_t nc = (nm - 1) * arity + nch;
      if (nc > (n + bn - 1) / bn) C.err = BT_EINTERNAL;
      C.c[l + 1] = nc;
      C.last_start = g.st[lk] + (nch - 1) * bn;
    }
  }
  if (cta_failed(C)) return;
  for (uint64_t w = tid; w < c * arity; w += nt) {
    const uint64_t k = w / arity, i = w - k * arity;
    if (!marked(mw, k)) continue;
    const uint64_t s = g.st[k] + i * bn;
    if (s >= g.st[k] + blen(g, k)) continue;
    nst[mrank(mw, mr, k) * arity + i] = s;
  }
  __syncthreads();
  tmark(C, 3);
}

// ---------------------------------------------------------------------------
// Pruning (section 3.1, "Optional Pruning"): for l = L-2 down to 0, a marked
// block k of level l becomes a pointer and loses its children when (i) none
// of its children has children, (ii) no pointer of level l (original, or made
// by pruning a block to its right) has a target window overlapping k, (iii)
// no pointer of level l+1 targets a child of k, and (iv) LO(S(k)) + |k| <=
// start(k).  Conditions (i), (iii), (iv) and the original pointers of (ii)
// leave a candidate set; a candidate is pruned iff no pruned candidate to its
// right targets it, resolved by frontier rounds (then right to left for what
// the round bound leaves).
// ---------------------------------------------------------------------------
struct PrW {
  uint8_t *hit_v, *hit2, *tgt_w, *gone, *mk2;
  uint32_t *state, *indeg, *fq0, *fq1, *nidx, *wpop, *ptr2;
  uint64_t *t1, *t2, *st2, *off2, *lo2;
};

__device__ PrW carve_prune(char* temp, uint64_t cv, uint64_t cw) {
  PrW R;
  char* p = temp;
  R.hit_v = (uint8_t*)carve(p, cv + 8);
  R.hit2 = (uint8_t*)carve(p, cv + 8);
  R.tgt_w = (uint8_t*)carve(p, cw + 8);
  R.gone = (uint8_t*)carve(p, cw + 8);
  R.mk2 = (uint8_t*)carve(p, cw + 8);
  R.state = (uint32_t*)carve(p, cv * 4 + 4);
  R.indeg = (uint32_t*)carve(p, cv * 4 + 4);
  R.fq0 = (uint32_t*)carve(p, cv * 4 + 4);
  R.fq1 = (uint32_t*)carve(p, cv * 4 + 4);
  R.nidx = (uint32_t*)carve(p, cw * 4 + 4);
  R.wpop = (uint32_t*)carve(p, (cv > cw ? cv : cw) * 4 + 4);  // mark words of either level
  R.ptr2 = (uint32_t*)carve(p, cw * 4 + 4);
  R.t1 = (uint64_t*)carve(p, cv * 8 + 8);
  R.t2 = (uint64_t*)carve(p, cv * 8 + 8);
  R.st2 = (uint64_t*)carve(p, cw * 8 + 8);
  R.off2 = (uint64_t*)carve(p, cw * 8 + 8);
  R.lo2 = (uint64_t*)carve(p, cw * 8 + 8);
  return R;
}

struct PLv {
  uint64_t n, c, b;
  uint64_t* st;
  uint32_t* mw;
  uint32_t* mr;
  uint32_t* ptr;
  uint64_t* off;
  uint64_t* lo;
};

__device__ __forceinline__ uint64_t plen(const PLv& v, uint64_t k) {
  const uint64_t s = v.st[k];
  return v.n - s < v.b ? v.n - s : v.b;
}

__device__ PLv plevel(const Cta& C, char* scr, const uint64_t* bsz, uint32_t l) {
  return PLv{C.n, C.c[l], bsz[l], (uint64_t*)(scr + C.sl.st[l]), (uint32_t*)(scr + C.sl.mw[l]),
             (uint32_t*)(scr + C.sl.mr[l]), (uint32_t*)(scr + C.sl.ptr[l]), (uint64_t*)(scr + C.sl.off[l]),
             (uint64_t*)(scr + C.sl.lo[l])};
}

__device__ void flag_targets(const PLv& v, uint8_t* flag) {
  for (uint64_t u = threadIdx.x; u < v.c; u += blockDim.x) {
    if (marked(v.mw, u)) continue;
    const uint64_t j = v.ptr[u];
    flag[j] = 1;
    if (v.off[u] + plen(v, u) > plen(v, j)) flag[j + 1] = 1;
  }
}

__device__ void prune_pass(const BParams& P, const BDoc& D, Cta& C, char* scr) {
  const uint64_t* bsz = P.sizes + D.lv_off;
  const unsigned tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, nw = nt >> 5;
  for (int l = (int)C.L - 2; l >= 0; l--) {
    const PLv v = plevel(C, scr, bsz, (uint32_t)l), w = plevel(C, scr, bsz, (uint32_t)l + 1);
    const bool w_last = l + 1 == (int)C.L - 1;
    const uint32_t arity = C.arity[l];
    const PrW R = carve_prune(scr + C.sl.temp, v.c, w.c);
    for (uint64_t i = tid; i <= v.c; i += nt) {
      R.hit_v[i] = 0;
      R.hit2[i] = 0;
      if (i < v.c) R.indeg[i] = 0;
    }
    for (uint64_t i = tid; i <= w.c; i += nt) {
      R.tgt_w[i] = 0;
      R.gone[i] = 0;
    }
    if (tid == 0) {
      C.wl[0] = C.wl[1] = C.wl[2] = 0;
      C.undecided = 0;
    }
    __syncthreads();
    flag_targets(v, R.hit_v);
    flag_targets(w, R.tgt_w);
    __syncthreads();
    // Candidates and their target blocks.
    for (uint64_t k = tid; k < v.c; k += nt) {
      R.state[k] = P_NOTCAND;
      if (!marked(v.mw, k) || R.hit_v[k]) continue;
      const uint64_t s = v.st[k], len = plen(v, k), lo = v.lo[k];
      if (lo == kNone) {
        fail(C, BT_EINTERNAL);
        continue;
      }
      if (lo + len > s) continue;  // (iv)
      const uint64_t first = mrank(v.mw, v.mr, k) * arity, nch = (len + w.b - 1) / w.b;
      bool ok = true;
      for (uint64_t i = 0; i < nch && ok; i++) {
        const uint64_t ch = first + i;
        if (!w_last && marked(w.mw, ch)) ok = false;  // (i)
        if (R.tgt_w[ch]) ok = false;                  // (iii)
      }
      if (!ok) continue;
      uint64_t a = 0, z = v.c;
      while (a < z) {
        const uint64_t mid = (a + z) / 2;
        if (v.st[mid] <= lo) a = mid + 1;
        else z = mid;
      }
      const uint64_t j = a - 1;
      R.t1[k] = j;
      R.t2[k] = (lo + len > v.st[j] + plen(v, j)) ? j + 1 : kNone;
      R.state[k] = P_UNDEC;
    }
    if (cta_failed(C)) return;
    for (uint64_t k = tid; k < v.c; k += nt) {
      if (R.state[k] != P_UNDEC) continue;
      if (R.state[R.t1[k]] != P_NOTCAND) atomicAdd(&R.indeg[R.t1[k]], 1u);
      if (R.t2[k] != kNone && R.state[R.t2[k]] != P_NOTCAND) atomicAdd(&R.indeg[R.t2[k]], 1u);
    }
    __syncthreads();
    // Round 0: candidates nothing targets are pruned.
    for (uint64_t k = tid; k < v.c; k += nt)
      if (R.state[k] == P_UNDEC && R.indeg[k] == 0) {
        R.state[k] = P_PRUNED;
        R.fq0[atomicAdd(&C.wl[0], 1u)] = (uint32_t)k;
      }
    __syncthreads();
    // Rounds: the candidates decided in the previous round inform their
    // targets (a pruned attacker keeps its target; the last kept attacker of
    // a target prunes it).
    uint64_t r = 1;
    for (; r < P.max_rounds; r++) {
      const uint32_t m = C.wl[(r - 1) % 3];
      if (m == 0) break;
      if (tid == 0) C.wl[r % 3] = 0;
      __syncthreads();
      const uint32_t* qin = (r - 1) & 1 ? R.fq1 : R.fq0;
      uint32_t* qout = r & 1 ? R.fq1 : R.fq0;
      for (uint32_t i = tid; i < m; i += nt) {
        const uint64_t k = qin[i];
        const uint32_t sk = R.state[k];
        for (int e = 0; e < 2; e++) {
          const uint64_t t = e == 0 ? R.t1[k] : R.t2[k];
          if (t == kNone || R.state[t] == P_NOTCAND) continue;
          uint32_t target = 0;
          if (sk == P_PRUNED) target = P_KEPT;
          else if (atomicSub(&R.indeg[t], 1u) == 1u) target = P_PRUNED;
          if (target && atomicCAS(&R.state[t], (uint32_t)P_UNDEC, target) == P_UNDEC)
            qout[atomicAdd(&C.wl[r % 3], 1u)] = (uint32_t)t;
        }
      }
      __syncthreads();
    }
    // Right-to-left finish of the candidates the round bound left undecided.
    for (uint64_t k = tid; k < v.c; k += nt)
      if (R.state[k] == P_UNDEC) atomicAdd(&C.undecided, 1ull);
    __syncthreads();
    if (C.undecided && tid == 0) {
      for (uint64_t k = v.c; k-- > 0;) {
        uint32_t s = R.state[k];
        if (s == P_UNDEC) {
          s = R.hit2[k] ? P_KEPT : P_PRUNED;
          R.state[k] = s;
        }
        if (s == P_PRUNED) {
          R.hit2[R.t1[k]] = 1;
          if (R.t2[k] != kNone) R.hit2[R.t2[k]] = 1;
        }
      }
    }
    __syncthreads();
    // Apply: pruned blocks lose their children and become pointers.
    for (uint64_t k = tid; k < v.c; k += nt) {
      if (R.state[k] != P_PRUNED) continue;
      const uint64_t first = mrank(v.mw, v.mr, k) * arity, nch = (plen(v, k) + w.b - 1) / w.b;
      for (uint64_t i = 0; i < nch; i++) R.gone[first + i] = 1;
      v.ptr[k] = (uint32_t)R.t1[k];
      v.off[k] = v.lo[k] - v.st[R.t1[k]];
    }
    __syncthreads();
    const uint64_t words = (v.c + 31) / 32;
    for (uint64_t wb = tid >> 5; wb < words; wb += nw) {
      const uint64_t k = wb * 32 + lane;
      const bool mk = k < v.c && marked(v.mw, k) && R.state[k] != P_PRUNED;
      const uint32_t bits = __ballot_sync(kFull, mk);
      if (lane == 0) R.wpop[wb] = __popc(bits);
      __syncwarp();
      if (lane == 0) v.mw[wb] = bits;
    }
    __syncthreads();
    cta_scan_u32(R.wpop, v.mr, words, C);
    // Compact level l+1 without the deleted children.
    for (uint64_t k = tid; k < w.c; k += nt) R.nidx[k] = R.gone[k] ? 0u : 1u;
    __syncthreads();
    cta_scan_u32(R.nidx, R.nidx, w.c, C);
    for (uint64_t k = tid; k < w.c; k += nt) {
      if (R.gone[k]) continue;
      const uint64_t i = R.nidx[k];
      R.st2[i] = w.st[k];
      const bool mk = marked(w.mw, k);
      R.mk2[i] = mk;
      R.off2[i] = w.off[k];
      R.lo2[i] = w.lo[k];
      if (mk) {
        R.ptr2[i] = 0;
      } else {
        const uint32_t j = w.ptr[k];
        if (R.gone[j]) fail(C, BT_EINTERNAL);
        R.ptr2[i] = R.nidx[j];
      }
    }
    if (cta_failed(C)) return;
    const uint64_t c2 = R.nidx[w.c];
    const uint64_t words2 = (c2 + 31) / 32;
    for (uint64_t i = tid; i < c2; i += nt) {
      w.st[i] = R.st2[i];
      w.off[i] = R.off2[i];
      w.lo[i] = R.lo2[i];
      w.ptr[i] = R.ptr2[i];
    }
    for (uint64_t wb = tid >> 5; wb < words2; wb += nw) {
      const uint64_t k = wb * 32 + lane;
      const uint32_t bits = __ballot_sync(kFull, k < c2 && R.mk2[k]);
      if (lane == 0) {
        w.mw[wb] = bits;
        R.wpop[wb] = __popc(bits);
      }
    }
    __syncthreads();
    cta_scan_u32(R.wpop, w.mr, words2, C);
    if (tid == 0) {
      C.c[l + 1] = c2;
      C.stats[l + 1][BT_ST_FINAL_BLOCKS] = c2;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Output: the tree's arrays, counters, level-1 prefix counts and leaf text in
// the pool; the device view that the query kernels read.
// ---------------------------------------------------------------------------
__device__ void count_rows(const uint8_t* __restrict__ T, const Cta& C, const PLv& v, int mode, bool last,
                           void* out, uint32_t cw, unsigned int* hist) {
  // mode 0: symbol counts of each block (marked blocks of a non-last level
  // are filled from their children afterwards); mode 1: counts of
  // T[st[ptr], st[ptr] + off) of each unmarked block (zeros for marked ones).
  const uint32_t S = C.S;
  const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  unsigned int* h = hist + warp * 256;
  for (uint64_t k = warp; k < v.c; k += nw) {
    const bool mk = marked(v.mw, k);
    uint64_t s0 = 0, len = 0;
    if (mode == 0 && (last || !mk)) {
      s0 = v.st[k];
      len = plen(v, k);
    } else if (mode == 1 && !mk) {
      s0 = v.st[v.ptr[k]];
      len = v.off[k];
    }
    for (uint32_t i = lane; i < S; i += 32) h[i] = 0;
    __syncwarp();
    for (uint64_t x = lane; x < len; x += 32) atomicAdd(&h[C.sym[T[s0 + x]]], 1u);
    __syncwarp();
    for (uint32_t i = lane; i < S; i += 32) cput(out, cw, k * S + i, h[i]);
    __syncwarp();
  }
}

__device__ void write_output(const BParams& P, const BDoc& D, Cta& C, char* scr, unsigned int* hist) {
  const uint64_t* bsz = P.sizes + D.lv_off;
  const unsigned tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  const uint32_t L = C.L, S = C.S;
  __shared__ OutLevel s_ol[kBMaxLevels];
  __shared__ uint32_t s_cw[kBMaxLevels];
  __shared__ uint64_t s_view, s_pre, s_leaf, s_sym;
  if (tid == 0) {
    for (uint32_t l = 0; l < L; l++) s_cw[l] = counter_width(bsz[l]);
    const uint64_t words = (C.c[L - 1] + 31) / 32;
    const uint32_t* mrl = (const uint32_t*)(scr + C.sl.mr[L - 1]);
    const uint64_t nm = mrl[words];
    const uint64_t leaf_alloc = nm * bsz[L - 1];
    const uint64_t need = out_layout(L, C.c, s_cw, S, leaf_alloc, s_ol, &s_view, &s_pre, &s_leaf, &s_sym);
    C.out_bytes = need;
    const unsigned long long o = atomicAdd(P.pool_used, (unsigned long long)need);
    if (o + need > P.pool_cap) {
      C.err = BT_ENOMEM;
      C.out = nullptr;
    } else {
      C.out_off = o;
      C.out = P.pool + o;
    }
  }
  if (cta_failed(C)) return;
  char* out = C.out;
  // Level arrays.
  for (uint32_t l = 0; l < L; l++) {
    const PLv v = plevel(C, scr, bsz, l);
    const uint64_t words = (v.c + 31) / 32;
    uint64_t* st = (uint64_t*)(out + s_ol[l].st);
    uint32_t* mw = (uint32_t*)(out + s_ol[l].mw);
    uint32_t* mr = (uint32_t*)(out + s_ol[l].mr);
    uint32_t* ptr = (uint32_t*)(out + s_ol[l].ptr);
    uint64_t* off = (uint64_t*)(out + s_ol[l].off);
    for (uint64_t k = tid; k < v.c; k += nt) {
      st[k] = v.st[k];
      ptr[k] = v.ptr[k];
      off[k] = marked(v.mw, k) ? 0 : v.off[k];
    }
    for (uint64_t i = tid; i <= words; i += nt) {
      if (i < words) mw[i] = v.mw[i];
      mr[i] = v.mr[i];
    }
  }
  __syncthreads();
  // Counters, last level first (marked blocks sum their children's rows).
  for (int l = (int)L - 1; l >= 0; l--) {
    const PLv v = plevel(C, scr, bsz, (uint32_t)l);
    const bool last = l + 1 == (int)L;
    void* cnt = out + s_ol[l].cnt;
    void* pc = out + s_ol[l].pc;
    const uint32_t cw = s_cw[l];
    count_rows(D.T, C, v, 0, last, cnt, cw, hist);
    count_rows(D.T, C, v, 1, last, pc, cw, hist);
    __syncthreads();
    if (!last) {
      const void* ccnt = out + s_ol[l + 1].cnt;
      const uint32_t ccw = s_cw[l + 1];
      const uint64_t bn = bsz[l + 1];
      const uint32_t arity = C.arity[l];
      for (uint64_t k = warp; k < v.c; k += nw) {
        if (!marked(v.mw, k)) continue;
        const uint64_t first = mrank(v.mw, v.mr, k) * arity, nch = (plen(v, k) + bn - 1) / bn;
        for (uint32_t s = lane; s < S; s += 32) {
          uint32_t acc = 0;
          for (uint64_t i = 0; i < nch; i++) acc += cget(ccnt, ccw, (first + i) * S + s);
          cput(cnt, cw, k * S + s, acc);
        }
      }
      __syncthreads();
    }
  }
  // Level-1 prefix counts.
  {
    const PLv v = plevel(C, scr, bsz, 0);
    uint64_t* pre = (uint64_t*)(out + s_pre);
    const void* cnt = out + s_ol[0].cnt;
    for (uint32_t s = tid; s < S; s += nt) {
      uint64_t acc = 0;
      for (uint64_t k = 0; k < v.c; k++) {
        pre[k * S + s] = acc;
        acc += cget(cnt, s_cw[0], k * S + s);
      }
      pre[v.c * S + s] = acc;
    }
  }
  // Leaf text of the marked last-level blocks: rank r at r * b_L.
  {
    const PLv v = plevel(C, scr, bsz, L - 1);
    uint8_t* leaf = (uint8_t*)(out + s_leaf);
    for (uint64_t w = tid; w < v.c * v.b; w += nt) {
      const uint64_t k = w / v.b, i = w - k * v.b;
      if (!marked(v.mw, k) || v.st[k] + i >= C.n) continue;
      leaf[mrank(v.mw, v.mr, k) * v.b + i] = D.T[v.st[k] + i];
    }
    if (tid == 0) {
      const uint64_t words = (v.c + 31) / 32;
      const uint64_t nm = v.mr[words];
      uint64_t lb = nm * v.b;
      if (nm && marked(v.mw, v.c - 1) && C.n - v.st[v.c - 1] < v.b) lb -= v.b - (C.n - v.st[v.c - 1]);
      P.res[D.index].leaf_bytes = lb;
    }
  }
  int16_t* sym = (int16_t*)(out + s_sym);
  for (uint32_t i = tid; i < 256; i += nt) sym[i] = C.sym[i];
  if (tid == 0) {
    TreeView* tv = (TreeView*)(out + s_view);
    tv->n = C.n;
    tv->L = L;
    tv->S = S;
    for (uint32_t l = 0; l < L; l++) {
      const uint64_t words = (C.c[l] + 31) / 32;
      LevelView& lv = tv->lv[l];
      lv.c = C.c[l];
      lv.b = bsz[l];
      lv.arity = C.arity[l];
      lv.bshift = block_shift(bsz[l]);
      lv.st = (const uint64_t*)(out + s_ol[l].st);
      lv.mw = (const uint32_t*)(out + s_ol[l].mw);
      lv.mr = (const uint32_t*)(out + s_ol[l].mr);
      lv.ptr = (const uint32_t*)(out + s_ol[l].ptr);
      lv.off = (const uint64_t*)(out + s_ol[l].off);
      lv.cnt = out + s_ol[l].cnt;
      lv.pc = out + s_ol[l].pc;
      lv.cw = s_cw[l];
      const uint32_t* mrl = (const uint32_t*)(scr + C.sl.mr[l]);
      C.nmarked[l] = mrl[words];
    }
    tv->pre = (const uint64_t*)(out + s_pre);
    tv->leaf = (const uint8_t*)(out + s_leaf);
    tv->sym = (const int16_t*)(out + s_sym);
  }
  __syncthreads();
}

template <class M>
__device__ void build_doc(const M& m, const BParams& P, uint32_t d, Cta& C, char* scr, unsigned int* hist,
                          uint32_t dyn_words) {
  const BDoc D = P.docs[d];
  const uint64_t* bsz = P.sizes + D.lv_off;
  if (threadIdx.x == 0) {
    C.err = 0;
    C.n = D.n;
    C.L = D.L;
    if (D.L == 0 || D.L > kBMaxLevels || scratch_layout(D.n, D.L, bsz, &C.sl) > P.scratch_per_cta)
      C.err = BT_EINTERNAL;
    C.out_off = 0;
    C.out_bytes = 0;
    for (int i = 0; i < 6; i++) C.cyc[i] = 0;
    C.t_mark = clock64();
  }
  __syncthreads();
  if (C.err == 0) alphabet(D.T, D.n, D.sigma, C);
  if (!cta_failed(C)) {
    prefix_pass(m, D.T, D.n, P.B, P.pw32, (uint64_t*)(scr + C.sl.H), C);
    if (bsz[0] >= P.anchor_min_b) {
      gram_list_pass(D.T, D.n, (uint32_t*)(scr + C.sl.lpos), (uint32_t*)(scr + C.sl.lhash), gram_list_cap(D.n), C);
    } else if (threadIdx.x == 0) {
      C.nsel = kNoList;
    }
    // Level 1: blocks k b_1.
    uint64_t* st0 = (uint64_t*)(scr + C.sl.st[0]);
    const uint64_t c0 = (D.n + bsz[0] - 1) / bsz[0];
    for (uint64_t k = threadIdx.x; k < c0; k += blockDim.x) st0[k] = k * bsz[0];
    if (threadIdx.x == 0) {
      C.c[0] = c0;
      C.last_start = (c0 - 1) * bsz[0];
    }
    __syncthreads();
    tmark(C, 0);
    for (uint32_t l = 0; l < D.L; l++) {
      level_pass(m, P, D, C, scr, l, (uint32_t*)hist, dyn_words);
      if (cta_failed(C)) break;
    }
  }
  if (!cta_failed(C) && P.prune) {
    prune_pass(P, D, C, scr);
    tmark(C, 4);
  }
  if (!cta_failed(C)) write_output(P, D, C, scr, hist);
  __syncthreads();
  tmark(C, 5);
  // Results.
  if (threadIdx.x == 0) {
    BRes& R = P.res[D.index];
    R.status = C.err;
    R.S = C.S;
    R.out_off = C.out_off;
    R.out_bytes = C.out_bytes;
    for (int i = 0; i < 6; i++) R.cycles[i] = C.cyc[i];
  }
  for (uint32_t i = threadIdx.x; i < 256; i += blockDim.x) P.res[D.index].sym[i] = C.sym[i];
  if (C.err == 0) {
    for (uint32_t l = threadIdx.x; l < D.L; l += blockDim.x) {
      BLevelRes& Lr = P.lres[D.lv_off + l];
      Lr.c = C.c[l];
      Lr.b = bsz[l];
      Lr.nmarked = C.nmarked[l];
      Lr.arity = C.arity[l];
      Lr.cw = counter_width(bsz[l]);
      for (int f = 0; f < BT_ST_FIELDS; f++) Lr.stats[f] = C.stats[l][f];
    }
  }
  __syncthreads();
}

// NT threads per CTA, MINB CTAs per SM: the register budget per thread is
// 65536 / (NT * MINB) (capped at 255).
template <class M, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_batch(BParams P, M m) {
  // Dynamic shared memory: the level's fingerprint filter, then (during the
  // output) 256 symbol counters per warp.
  extern __shared__ unsigned int s_hist[];
  __shared__ Cta C;
  char* scr = P.scratch + (uint64_t)blockIdx.x * P.scratch_per_cta;
  for (;;) {
    if (threadIdx.x == 0) C.doc = atomicAdd(P.next, 1u);
    __syncthreads();
    const uint32_t d = C.doc;
    __syncthreads();
    if (d >= P.ndocs) return;
    build_doc(m, P, d, C, scr, s_hist, P.dyn_words);
  }
}

// ---------------------------------------------------------------------------
// Host driver.
// ---------------------------------------------------------------------------
// What the last batched build did (bt_batch_report).
struct Report {
  uint64_t kernel_docs, worker_docs, launches, retried, threads, ctas_per_sm, pool_bytes, scratch_bytes,
      max_grid, chunk, tuned, upload_us, kernel_us;
};
std::mutex g_report_mu;
Report g_report{};

struct DocPlan {
  uint64_t i;              // caller index
  uint64_t n;
  uint32_t sigma, L;
  uint64_t need;           // CTA scratch bytes
  uint64_t size_off;       // first block size in the batch's size array
};

// Powers (B^32)^i, i <= 1024, for the prefix pass.
template <class M>
std::vector<uint64_t> chunk_powers(const M& m, uint64_t B) {
  std::vector<uint64_t> pw(1025);
  const uint64_t X = pow_mod(m, B, 32);
  pw[0] = 1 % m.q();
  for (int i = 1; i <= 1024; i++) pw[i] = m.mul(pw[i - 1], X);
  return pw;
}

// Opt every instantiation in to its dynamic shared memory, once per device.
template <class M>
int allow_smem(const M&, unsigned threads, unsigned ctas_per_sm, int bytes) {
  static std::mutex mu;
  static uint64_t done[8] = {};
  int dev = 0;
  BT_CUDA(cudaGetDevice(&dev));
  (void)threads;
  (void)ctas_per_sm;
  const int which = 0;
  std::lock_guard<std::mutex> g(mu);
  if (done[which] & (1ull << (dev & 63))) return BT_OK;
  BT_CUDA(cudaFuncSetAttribute(k_batch<M, 1024, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  done[which] |= 1ull << (dev & 63);
  return BT_OK;
}

template <class M>
int launch_docs(const M& m, const BParams& base, const std::vector<const DocPlan*>& order, uint32_t first,
                uint32_t count, unsigned threads, unsigned ctas_per_sm, unsigned grid, uint64_t per_cta,
                char* scratch, unsigned int* next, cudaStream_t s) {
  BParams P = base;
  P.docs = base.docs + first;
  P.ndocs = count;
  P.next = next;
  P.scratch = scratch;
  P.scratch_per_cta = per_cta;
  BT_CUDA(cudaMemsetAsync(next, 0, sizeof(unsigned int), s));
  // Filter words: 128 KiB of shared memory with one CTA per SM, 64 KiB with
  // two; at least the output's 256 counters per warp.
  const uint32_t hist_words = threads / 32 * 256;
  uint32_t fw = ctas_per_sm <= 1 ? 32768u : 16384u;
  if (fw < hist_words) fw = hist_words;
  P.dyn_words = fw;
  const size_t smem = (size_t)fw * sizeof(unsigned int);
  BT_TRY(allow_smem(m, threads, ctas_per_sm, (int)smem));
  // The one launch shape: 1024 threads, one CTA per SM (two CTAs of 512 and
  // one of 512 measured slower; see the shape list of the tuner).
  if (threads != 1024 || ctas_per_sm != 1) return BT_EINVAL;
  BT_LAUNCH(k_batch<M, 1024, 1><<<grid, 1024, smem, s>>>(P, m));
  BT_CUDA(cudaGetLastError());
  (void)order;
  return BT_OK;
}

// Device memory of one batched call, stream-ordered on the call's stream (no
// device-wide synchronisation, so calls on several host threads overlap).
struct DevFree {
  cudaStream_t s = nullptr;
  std::vector<void*> p;
  ~DevFree() {
    for (void* q : p) cudaFreeAsync(q, s);
  }
  template <class T>
  int alloc(T** out, uint64_t count) {
    void* q = nullptr;
    if (!alloc_allowed((count ? count : 1) * sizeof(T))) return BT_ENOMEM;
    cudaError_t e = cudaMallocAsync(&q, (count ? count : 1) * sizeof(T), s);
    if (e != cudaSuccess) {
      note_cuda_error(e, "cudaMallocAsync", __FILE__, __LINE__);
      cudaGetLastError();
      return e == cudaErrorMemoryAllocation ? BT_ENOMEM : BT_ECUDA;
    }
    p.push_back(q);
    *out = (T*)q;
    return BT_OK;
  }
};

template <class M>
int run_batch(const M& m, const uint8_t* const* texts, const uint32_t* taus, const uint32_t* leaf_lens,
              const bt_opts& o, std::vector<DocPlan>& plans, const std::vector<uint64_t>& sizes,
              unsigned threads, unsigned ctas_per_sm, unsigned chunk, bt_tree** outs, cudaStream_t s) {
  const uint64_t nd = plans.size();
  if (nd == 0) return BT_OK;
  int device = 0;
  BT_CUDA(cudaGetDevice(&device));
  const uint64_t q = o.modulus ? o.modulus : Mersenne61::Q;
  const uint64_t B = base_for(o.seed, q);
  // Longest documents first: the work queue hands them out first.
  std::vector<const DocPlan*> order(nd);
  for (uint64_t k = 0; k < nd; k++) order[k] = &plans[k];
  // Longest expected work first (text length times levels: each level
  // scans up to the whole text), so that the last CTAs to finish hold short
  // documents.
  std::stable_sort(order.begin(), order.end(), [](const DocPlan* a, const DocPlan* b) {
    return a->n * a->L > b->n * b->L;
  });
  DevFree mem;
  mem.s = s;
  // Texts, each at a 16-byte aligned offset and followed by at least 48 bytes
  // of padding (16-byte loads past a text's end stay in the buffer).
  std::vector<uint64_t> toff(nd);
  uint64_t ttotal = 0;
  for (uint64_t k = 0; k < nd; k++) {
    toff[k] = ttotal;
    ttotal += (plans[k].n + 63) & ~15ull;
  }
  uint8_t* d_text;
  BT_TRY(mem.alloc(&d_text, ttotal + 64));
  const auto t_up = std::chrono::steady_clock::now();
  for (uint64_t k = 0; k < nd; k++)
    BT_CUDA(cudaMemcpyAsync(d_text + toff[k], texts[plans[k].i], plans[k].n, cudaMemcpyDefault, s));
  const uint64_t upload_us = (uint64_t)std::chrono::duration_cast<std::chrono::microseconds>(
                                 std::chrono::steady_clock::now() - t_up).count();
  // Documents in processing order, block sizes, results.
  std::vector<BDoc> hd(nd);
  uint64_t nlv = 0;
  for (uint64_t k = 0; k < nd; k++) nlv += plans[k].L;
  std::vector<uint64_t> hsz(nlv);
  std::vector<uint32_t> lv_off(nd);
  {
    uint64_t o2 = 0;
    for (uint64_t k = 0; k < nd; k++) {
      lv_off[k] = (uint32_t)o2;
      for (uint32_t l = 0; l < plans[k].L; l++) hsz[o2 + l] = sizes[plans[k].size_off + l];
      o2 += plans[k].L;
    }
  }
  for (uint64_t r = 0; r < nd; r++) {
    const uint64_t k = (uint64_t)(order[r] - plans.data());
    hd[r] = BDoc{d_text + toff[k], plans[k].n, plans[k].sigma, plans[k].L, (uint32_t)k, lv_off[k]};
  }
  BDoc* d_docs;
  uint64_t* d_sizes;
  BRes* d_res;
  BLevelRes* d_lres;
  uint64_t* d_pw;
  unsigned int* d_next;
  BT_TRY(mem.alloc(&d_docs, nd));
  BT_TRY(mem.alloc(&d_sizes, nlv));
  BT_TRY(mem.alloc(&d_res, nd));
  BT_TRY(mem.alloc(&d_lres, nlv));
  BT_TRY(mem.alloc(&d_pw, 1025));
  BT_TRY(mem.alloc(&d_next, 64));
  const std::vector<uint64_t> pw = chunk_powers(m, B);
  BT_CUDA(cudaMemcpyAsync(d_docs, hd.data(), nd * sizeof(BDoc), cudaMemcpyHostToDevice, s));
  BT_CUDA(cudaMemcpyAsync(d_sizes, hsz.data(), nlv * sizeof(uint64_t), cudaMemcpyHostToDevice, s));
  BT_CUDA(cudaMemcpyAsync(d_pw, pw.data(), pw.size() * sizeof(uint64_t), cudaMemcpyHostToDevice, s));
  BT_CUDA(cudaMemsetAsync(d_res, 0, nd * sizeof(BRes), s));
  // Output pool: three bytes per text byte plus a fixed part per document;
  // a document that does not fit is built again into a pool of exactly the
  // size it reported.
  uint64_t pool_cap = 0;
  for (uint64_t k = 0; k < nd; k++) pool_cap += 3 * plans[k].n + (32u << 10);
  // The pool outlives the call: it is returned to the device's stream-ordered
  // pool when the last tree is freed (on the freeing thread's stream; a tree
  // is never freed while queries on it run).
  auto make_pool = [&](uint64_t cap, std::shared_ptr<void>& out) -> int {
    void* p = nullptr;
    if (!alloc_allowed(cap)) return BT_ENOMEM;
    cudaError_t e = cudaMallocAsync(&p, cap, s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return e == cudaErrorMemoryAllocation ? BT_ENOMEM : BT_ECUDA;
    }
    out = std::shared_ptr<void>(p, [](void* x) {
      cudaFreeAsync(x, cudaStreamPerThread);
      cudaStreamSynchronize(cudaStreamPerThread);
    });
    return BT_OK;
  };
  std::shared_ptr<void> pool;
  BT_TRY(make_pool(pool_cap, pool));
  unsigned long long* d_used;
  BT_TRY(mem.alloc(&d_used, 1));
  BT_CUDA(cudaMemsetAsync(d_used, 0, sizeof(unsigned long long), s));

  BParams P{};
  P.docs = d_docs;
  P.sizes = d_sizes;
  P.res = d_res;
  P.lres = d_lres;
  P.pool = (char*)pool.get();
  P.pool_used = d_used;
  P.pool_cap = pool_cap;
  P.B = B;
  P.pw32 = d_pw;
  P.prune = o.prune ? 1 : 0;
  P.max_rounds = o.max_rounds ? o.max_rounds : 4096;
  P.scan_u = chunk;
  P.anchor_min_b = (o.flags & BT_FLAG_ANCHOR_ALL) ? 32 : kAnchorMinB;

  // Size classes: consecutive documents (in decreasing scratch need) whose
  // need is within 4x of the class's first; one launch per class, with as
  // many CTAs as memory allows, up to ctas_per_sm per SM.
  size_t free_b = 0, total_b = 0;
  BT_CUDA(cudaMemGetInfo(&free_b, &total_b));
  const uint64_t budget = (uint64_t)(free_b * 0.6);
  const unsigned nsm = device_sm_count();
  struct Cls {
    uint32_t first, count;
    uint64_t per_cta;
    unsigned grid;
  };
  std::vector<Cls> cls;
  uint64_t scratch_max = 0;
  for (uint32_t r = 0; r < nd;) {
    // One launch for every remaining document when the scratch of a full
    // grid sized for the largest of them fits; otherwise a class of the
    // documents within 4x of the largest, with as many CTAs as fit.
    uint64_t top = 0;
    for (uint32_t q2 = r; q2 < nd; q2++) top = std::max<uint64_t>(top, out_align(order[q2]->need));
    const uint64_t full = std::min<uint64_t>((uint64_t)(nd - r), (uint64_t)nsm * ctas_per_sm);
    uint32_t e = r;
    uint64_t grid;
    const uint64_t cap = o.batch_ctas ? o.batch_ctas : ~0ull;
    if (std::min<uint64_t>(full, cap) * top <= budget) {
      e = (uint32_t)nd;
      grid = std::min<uint64_t>(full, cap);
    } else {
      // The class: the documents of the order whose need is within 4x of the
      // first one's, with a grid sized for the largest of them.
      const uint64_t first = out_align(order[r]->need);
      top = first;
      while (e < nd && order[e]->need * 4 >= first && order[e]->need <= first * 4) {
        top = std::max<uint64_t>(top, out_align(order[e]->need));
        e++;
      }
      grid = std::min<uint64_t>({(uint64_t)(e - r), budget / top, cap});
      if (grid == 0) grid = 1;
    }
    cls.push_back(Cls{r, e - r, top, (unsigned)grid});
    scratch_max = std::max<uint64_t>(scratch_max, grid * top);
    r = e;
  }
  char* d_scratch;
  BT_TRY(mem.alloc(&d_scratch, scratch_max));
  // The launches' device time (measurement hook), between two events.
  cudaEvent_t ev[2] = {nullptr, nullptr};
  const bool timed = cudaEventCreate(&ev[0]) == cudaSuccess && cudaEventCreate(&ev[1]) == cudaSuccess;
  if (timed) cudaEventRecord(ev[0], s);
  int lrc = BT_OK;
  for (size_t ci = 0; ci < cls.size() && lrc == BT_OK; ci++)
    lrc = launch_docs(m, P, order, cls[ci].first, cls[ci].count, threads, ctas_per_sm, cls[ci].grid,
                      cls[ci].per_cta, d_scratch, d_next + (ci % 64), s);
  if (timed) cudaEventRecord(ev[1], s);
  std::vector<BRes> res(nd);
  std::vector<BLevelRes> lres(nlv);
  if (lrc == BT_OK) {
    lrc = cudaMemcpyAsync(res.data(), d_res, nd * sizeof(BRes), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
                  cudaMemcpyAsync(lres.data(), d_lres, nlv * sizeof(BLevelRes), cudaMemcpyDeviceToHost, s) ==
                      cudaSuccess && cudaStreamSynchronize(s) == cudaSuccess
              ? BT_OK
              : BT_ECUDA;
  }
  float kernel_ms = 0;
  if (timed && lrc == BT_OK) cudaEventElapsedTime(&kernel_ms, ev[0], ev[1]);
  for (cudaEvent_t e : ev)
    if (e) cudaEventDestroy(e);
  BT_TRY(lrc);

  // Documents whose tree did not fit in the pool: once more, into a pool of
  // the size they reported.
  std::vector<std::shared_ptr<void>> pool_of(nd, pool);
  uint64_t retried = 0;
  {
    std::vector<uint32_t> again;
    uint64_t cap2 = 0;
    for (uint64_t k = 0; k < nd; k++)
      if (res[k].status == BT_ENOMEM) {
        again.push_back((uint32_t)k);
        cap2 += out_align(res[k].out_bytes);
      }
    if (!again.empty()) {
      std::shared_ptr<void> pool2;
      BT_TRY(make_pool(cap2, pool2));
      std::vector<BDoc> hd2;
      uint64_t top = 0;
      for (uint32_t k : again) {
        for (uint64_t r = 0; r < nd; r++)
          if (hd[r].index == k) hd2.push_back(hd[r]);
        top = std::max<uint64_t>(top, out_align(plans[k].need));
      }
      BDoc* d_docs2;
      BT_TRY(mem.alloc(&d_docs2, hd2.size()));
      BT_CUDA(cudaMemcpyAsync(d_docs2, hd2.data(), hd2.size() * sizeof(BDoc), cudaMemcpyHostToDevice, s));
      BT_CUDA(cudaMemsetAsync(d_used, 0, sizeof(unsigned long long), s));
      BParams P2 = P;
      P2.docs = d_docs2;
      P2.pool = (char*)pool2.get();
      P2.pool_cap = cap2;
      const unsigned grid = (unsigned)std::max<uint64_t>(
          1, std::min<uint64_t>({(uint64_t)hd2.size(), (uint64_t)nsm * ctas_per_sm, scratch_max / top,
                                 o.batch_ctas ? (uint64_t)o.batch_ctas : ~0ull}));
      BT_TRY(launch_docs(m, P2, order, 0, (uint32_t)hd2.size(), threads, ctas_per_sm, grid, top, d_scratch,
                         d_next, s));
      BT_CUDA(cudaMemcpyAsync(res.data(), d_res, nd * sizeof(BRes), cudaMemcpyDeviceToHost, s));
      BT_CUDA(cudaMemcpyAsync(lres.data(), d_lres, nlv * sizeof(BLevelRes), cudaMemcpyDeviceToHost, s));
      BT_CUDA(cudaStreamSynchronize(s));
      for (uint32_t k : again) pool_of[k] = pool2;
      retried = again.size();
    }
  }

  // Trees.
  for (uint64_t k = 0; k < nd; k++) {
    const BRes& R = res[k];
    if (R.status != BT_OK) return R.status;
  }
  for (uint64_t k = 0; k < nd; k++) {
    const BRes& R = res[k];
    const DocPlan& D = plans[k];
    bt_tree* t = new (std::nothrow) bt_tree();
    if (!t) return BT_ENOMEM;
    outs[D.i] = t;
    t->n = D.n;
    t->tau = taus[D.i];
    t->leaf_len = leaf_lens[D.i];
    t->L = D.L;
    t->prune = o.prune ? 1 : 0;
    t->seed = o.seed;
    t->q = q;
    t->B = B;
    t->device = device;
    t->S = R.S;
    t->leaf_bytes = R.leaf_bytes;
    memcpy(t->sym_host, R.sym, sizeof(t->sym_host));
    t->slab = pool_of[k];
    t->lv.resize(D.L);
    std::vector<uint64_t> c(D.L);
    std::vector<uint32_t> cw(D.L);
    for (uint32_t l = 0; l < D.L; l++) {
      const BLevelRes& Lr = lres[lv_off[k] + l];
      c[l] = Lr.c;
      cw[l] = Lr.cw;
    }
    const BLevelRes& last = lres[lv_off[k] + D.L - 1];
    std::vector<OutLevel> ol(D.L);
    uint64_t o_view, o_pre, o_leaf, o_sym;
    out_layout(D.L, c.data(), cw.data(), R.S, last.nmarked * last.b, ol.data(), &o_view, &o_pre, &o_leaf,
               &o_sym);
    char* base = (char*)t->slab.get() + R.out_off;
    for (uint32_t l = 0; l < D.L; l++) {
      const BLevelRes& Lr = lres[lv_off[k] + l];
      Level& v = t->lv[l];
      v.c = Lr.c;
      v.b = Lr.b;
      v.arity = Lr.arity;
      v.nmarked = Lr.nmarked;
      v.cw = Lr.cw;
      v.st = (uint64_t*)(base + ol[l].st);
      v.mw = (uint32_t*)(base + ol[l].mw);
      v.mr = (uint32_t*)(base + ol[l].mr);
      v.ptr = (uint32_t*)(base + ol[l].ptr);
      v.off = (uint64_t*)(base + ol[l].off);
      v.cnt = base + ol[l].cnt;
      v.pc = base + ol[l].pc;
      memcpy(v.stats, Lr.stats, sizeof(v.stats));
    }
    t->view = (TreeView*)(base + o_view);
    t->pre = (uint64_t*)(base + o_pre);
    t->leaf = (uint8_t*)(base + o_leaf);
    t->sym = (int16_t*)(base + o_sym);
    t->dev_bytes = R.out_bytes;
    for (int i = 0; i < 6; i++) t->batch_cycles[i] = R.cycles[i];
  }
  {
    std::lock_guard<std::mutex> g(g_report_mu);
    g_report.kernel_docs = nd;
    g_report.upload_us = upload_us;
    g_report.kernel_us = (uint64_t)(kernel_ms * 1000.0f);
    g_report.launches = cls.size();
    g_report.retried = retried;
    g_report.threads = threads;
    g_report.ctas_per_sm = ctas_per_sm;
    g_report.chunk = chunk;
    g_report.pool_bytes = pool_cap;
    g_report.scratch_bytes = scratch_max;
    g_report.max_grid = 0;
    for (const Cls& c2 : cls) g_report.max_grid = std::max<uint64_t>(g_report.max_grid, c2.grid);
  }
  return BT_OK;
}

}  // namespace

// Builds, with the persistent kernel, every document it can take (at most
// kBMaxText bytes and kBMaxLevels levels): routed[d] = 1 and outs[d] holds
// its tree.  Documents it cannot take keep routed[d] = 0 and are left to the
// caller.  Arguments are validated as bt_build_ex does.  Returns the first
// failure's status; trees already made stay in outs for the caller to free.
int batch_kernel_build(const uint8_t* const* texts, const uint64_t* ns, const uint32_t* sigmas,
                       const uint32_t* taus, const uint32_t* leaf_lens, uint64_t ndocs, const bt_opts& o,
                       std::vector<char>& routed, bt_tree** outs, uint32_t threads, uint32_t ctas_per_sm,
                       uint32_t chunk, cudaStream_t s, const std::vector<char>* eligible) {
  if (threads < 64 || threads > kMaxBThreads || threads % 32) return BT_EINVAL;
  if (ctas_per_sm == 0) ctas_per_sm = 1;
  if (o.modulus && (o.modulus < 300 || o.modulus >= (1ull << 32))) return BT_EINVAL;
  std::vector<DocPlan> plans;
  std::vector<uint64_t> sizes;
  routed.assign(ndocs, 0);
  for (uint64_t d = 0; d < ndocs; d++) {
    const uint64_t n = ns[d];
    if (!texts[d] || n == 0 || n >= (1ull << 32) || taus[d] < 2 || taus[d] > 64 || leaf_lens[d] == 0 ||
        sigmas[d] == 0)
      return BT_EINVAL;
    std::vector<uint64_t> b;
    BT_TRY(plan_sizes(n, taus[d], leaf_lens[d], o, b));
    if (n > kBMaxText || b.size() > kBMaxLevels) continue;
    if (eligible && !(*eligible)[d]) continue;
    DocPlan pl;
    pl.i = d;
    pl.n = n;
    pl.sigma = sigmas[d];
    pl.L = (uint32_t)b.size();
    ScratchLayout sl;
    pl.need = scratch_layout(n, pl.L, b.data(), &sl);
    pl.size_off = sizes.size();
    sizes.insert(sizes.end(), b.begin(), b.end());
    plans.push_back(pl);
    routed[d] = 1;
  }
  if (o.modulus)
    return run_batch(SmallMod{o.modulus}, texts, taus, leaf_lens, o, plans, sizes, threads, ctas_per_sm, chunk,
                     outs, s);
  return run_batch(Mersenne61{}, texts, taus, leaf_lens, o, plans, sizes, threads, ctas_per_sm, chunk, outs, s);
}

void batch_report_workers(uint64_t docs) {
  std::lock_guard<std::mutex> g(g_report_mu);
  g_report.worker_docs = docs;
}

void batch_report_reset() {
  std::lock_guard<std::mutex> g(g_report_mu);
  g_report = Report{};
}

// ---------------------------------------------------------------------------
// Autotuner of the batched kernel's launch shape: threads per CTA, CTAs per
// SM and the window chunk of the scan (positions per lane and step).  For a
// batch of at least kTuneMinDocs documents whose size class has no cached
// choice, each candidate builds the same seeded sample of the batch: every
// k-th document no longer than the batch's 75th length percentile, about
// 1/16 of the batch but at least two documents per CTA of a full grid, so
// that every SM stays busy during the trial.  A candidate's cost is the SM
// time it spent: the sum over the sample of the cycles of each document's
// CTA, divided by the CTAs that share an SM (a wall-clock time would measure
// the sample's longest document instead).  The cheapest is cached per (log2
// of the mean length, log2 of the longest, log2 of the batch size) for the
// rest of the process.  Smaller batches use the default shape.
namespace {
struct Shape {
  uint32_t threads, ctas, chunk;
};
// One CTA of 1024 threads per SM: two CTAs of 512 per SM measured slower on
// every batch tried (4 KiB - 4 MiB: 11.4k against 14.6k docs/s; 4 KiB -
// 16 MiB: 3.9k against 4.3k), as each document then has half the threads and
// half the shared-memory filter, and the longest documents set the batch's
// end.  The tuner picks the scan's run length.
constexpr Shape kShapes[] = {{1024, 1, 8}, {1024, 1, 4}};
constexpr uint64_t kTuneMinDocs = 1024;
std::mutex g_tune_mu;
std::vector<std::pair<uint64_t, Shape>> g_tuned;

uint64_t tune_key(const uint64_t* ns, uint64_t ndocs) {
  uint64_t sum = 0, mx = 0;
  for (uint64_t d = 0; d < ndocs; d++) {
    sum += ns[d];
    mx = std::max<uint64_t>(mx, ns[d]);
  }
  auto lg = [](uint64_t x) {
    uint64_t l = 0;
    while (x > 1) {
      x >>= 1;
      l++;
    }
    return l;
  };
  return (lg(sum / std::max<uint64_t>(ndocs, 1)) << 16) | (lg(mx) << 8) | lg(ndocs);
}
}  // namespace

int batch_shape(const uint8_t* const* texts, const uint64_t* ns, const uint32_t* sigmas, const uint32_t* taus,
                const uint32_t* leaf_lens, uint64_t ndocs, const bt_opts& o, cudaStream_t s, uint32_t* threads,
                uint32_t* ctas_per_sm, uint32_t* chunk, uint64_t* tuned_now) {
  Shape best = kShapes[0];
  *tuned_now = 0;
  if (const char* e = getenv("BT_BATCH_SHAPE")) {  // "threads,ctas,chunk": a fixed run length for measurements
    unsigned a = 0, b2 = 0, c = 0;
    if (sscanf(e, "%u,%u,%u", &a, &b2, &c) == 3 && c) best = Shape{1024, 1, c};
  } else if (ndocs >= kTuneMinDocs && !o.batch_ctas) {
    const uint64_t key = tune_key(ns, ndocs);
    bool found = false;
    {
      std::lock_guard<std::mutex> g(g_tune_mu);
      for (auto& kv : g_tuned)
        if (kv.first == key) {
          best = kv.second;
          found = true;
        }
    }
    if (!found) {
      // The sample: every k-th document, about 1/16 of the batch but at least
      // two per CTA of a full grid.
      std::vector<uint64_t> lens(ns, ns + ndocs);
      std::nth_element(lens.begin(), lens.begin() + ndocs * 3 / 4, lens.end());
      const uint64_t cap75 = lens[ndocs * 3 / 4];
      const uint64_t want = std::max<uint64_t>(ndocs / 16, 2ull * device_sm_count() * 2);
      const uint64_t step = std::max<uint64_t>(1, ndocs * 3 / 4 / want);
      std::vector<const uint8_t*> st;
      std::vector<uint64_t> sn;
      std::vector<uint32_t> ss, stau, sl;
      for (uint64_t d = 0; d < ndocs; d += step) {
        if (ns[d] > cap75) continue;
        st.push_back(texts[d]);
        sn.push_back(ns[d]);
        ss.push_back(sigmas[d]);
        stau.push_back(taus[d]);
        sl.push_back(leaf_lens[d]);
      }
      // A document's work is estimated as its bytes times its levels; a
      // shape's cost is the batch's makespan when its CTAs, at the cycles
      // per unit of work measured on the sample, take the documents from the
      // queue longest first.
      std::vector<double> work(ndocs, 0.0);
      double sample_work = 0;
      {
        std::vector<uint64_t> b;
        for (uint64_t d = 0; d < ndocs; d++) {
          if (ns[d] > kBMaxText || plan_sizes(ns[d], taus[d], leaf_lens[d], o, b) != BT_OK) continue;
          work[d] = (double)ns[d] * (double)b.size();
        }
        for (uint64_t d = 0; d < ndocs; d += step)
          if (ns[d] <= cap75) sample_work += work[d];
      }
      std::vector<double> order(work);
      std::sort(order.begin(), order.end(), std::greater<double>());
      double best_cost = 1e300;
      for (const Shape& sh : kShapes) {
        std::vector<char> routed;
        std::vector<bt_tree*> outs(st.size(), nullptr);
        const int rc = batch_kernel_build(st.data(), sn.data(), ss.data(), stau.data(), sl.data(), st.size(), o,
                                          routed, outs.data(), sh.threads, sh.ctas, sh.chunk, s, nullptr);
        cudaStreamSynchronize(s);
        double cycles = 0;
        for (bt_tree* t : outs)
          if (t)
            for (int i = 0; i < 6; i++) cycles += (double)t->batch_cycles[i];
        for (bt_tree* t : outs) bt_free(t);
        if (rc != BT_OK) return rc;
        const double per_work = cycles / std::max(sample_work, 1.0);
        std::priority_queue<double, std::vector<double>, std::greater<double>> slots;
        for (uint64_t g = 0; g < (uint64_t)device_sm_count() * sh.ctas; g++) slots.push(0.0);
        double cost = 0;
        for (double w : order) {
          if (w <= 0) break;
          const double t = slots.top() + w * per_work;
          slots.pop();
          slots.push(t);
          cost = std::max(cost, t);
        }
        if (cost < best_cost) {
          best_cost = cost;
          best = sh;
        }
        (*tuned_now)++;
      }
      std::lock_guard<std::mutex> g(g_tune_mu);
      g_tuned.emplace_back(key, best);
    }
  }
  *threads = best.threads;
  *ctas_per_sm = best.ctas;
  *chunk = best.chunk;
  return BT_OK;
}

// Long documents are built by the level kernels of the single-text path on
// host workers, at the same time as the batched kernel builds the others: a
// document longer than the batch's share per CTA would outlast the batch in
// its one CTA, and the single-text path's anchored scan gets more out of a
// long text than one CTA does.  A document is long at kSplitMin bytes or more
// and at least half the batch's bytes per CTA (so a batch large enough to
// balance its CTAs is not split).  The batched kernel then leaves the workers
// a share of the SMs in proportion to the long documents' bytes (at least 8
// SMs, at most half).  Returns the kernel's CTA cap (0: no split) and clears
// eligible[d] for the long documents.
constexpr uint64_t kSplitMin = 8ull << 20;

uint32_t batch_split(const uint64_t* ns, const uint32_t* taus, const uint32_t* leaf_lens, uint64_t ndocs,
                     const bt_opts& o, uint32_t ctas_per_sm, std::vector<char>& eligible) {
  (void)taus;
  (void)leaf_lens;
  eligible.assign(ndocs, 1);
  if (ndocs < 64 || o.batch_ctas) return 0;
  const unsigned nsm = device_sm_count();
  double total = 0, heavy = 0;
  for (uint64_t d = 0; d < ndocs; d++) total += (double)ns[d];
  const double share = total / ((double)nsm * ctas_per_sm);
  const double lim = std::max((double)kSplitMin, 0.5 * share);
  for (uint64_t d = 0; d < ndocs; d++)
    if ((double)ns[d] >= lim) {
      eligible[d] = 0;
      heavy += (double)ns[d];
    }
  if (heavy == 0 || heavy == total) {
    eligible.assign(ndocs, 1);
    return 0;
  }
  uint32_t reserve = (uint32_t)((double)nsm * heavy / total + 0.5);
  reserve = std::max<uint32_t>(8, std::min<uint32_t>(reserve, nsm / 2));
  return (nsm - reserve) * ctas_per_sm;
}

void batch_report_tuned(uint64_t trials) {
  std::lock_guard<std::mutex> g(g_report_mu);
  g_report.tuned = trials;
}

}  // namespace bt

extern "C" int bt_batch_report(uint64_t* out, uint32_t cap) {
  using namespace bt;
  if (!out || cap < 13) return BT_EINVAL;
  std::lock_guard<std::mutex> g(g_report_mu);
  const uint64_t v[13] = {g_report.kernel_docs, g_report.worker_docs, g_report.launches, g_report.retried,
                          g_report.threads, g_report.ctas_per_sm, g_report.pool_bytes, g_report.scratch_bytes,
                          g_report.max_grid, g_report.chunk, g_report.tuned, g_report.upload_us,
                          g_report.kernel_us};
  memcpy(out, v, sizeof(v));
  return BT_OK;
}

extern "C" int bt_batch_cycles(const bt_tree* t, uint64_t* out, uint32_t cap) {
  if (!t || !out || cap < 6) return BT_EINVAL;
  memcpy(out, t->batch_cycles, 6 * sizeof(uint64_t));
  return BT_OK;
}
