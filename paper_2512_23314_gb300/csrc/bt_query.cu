// bt_query.cu -- alphabet map, rank/select counters, leaf text and queries.
//
// access, rank and select are the queries of section 1; the paper's
// implementation stores one bit vector per level plus pointers and offsets
// (section 4.4) and names the rank/select auxiliary data as future work
// (section 6).  The counters used here:
//   cnt[k][s]  occurrences of symbol s in block k (every level),
//   pc[u][s]   occurrences of s in T[st[ptr], st[ptr] + off) for an unmarked
//              block u (the part of its target before the copied window),
//   pre[k][s]  occurrences of s before level-1 block k.
// rank_c(i) descends from the level-1 block holding i: inside a marked block
// it adds the counts of the children left of the one holding i; at an
// unmarked block it continues in its target (ptr or ptr+1) and subtracts
// pc.  select mirrors it.  One thread answers one query.
#include <cstdlib>

#include "bt_internal.cuh"

namespace bt {

namespace {

__global__ void k_histogram(const uint8_t* __restrict__ T, uint64_t n, unsigned long long* hist) {
  __shared__ unsigned int h[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
  __syncthreads();
  const uint64_t nv = n / 16;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (((uintptr_t)T & 15) == 0) {
    const uint4* V = (const uint4*)T;
    for (uint64_t i = tid; i < nv; i += stride) {
      uint4 q = V[i];
      uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
      for (int a = 0; a < 4; a++)
#pragma unroll
        for (int b = 0; b < 4; b++) atomicAdd(&h[(w[a] >> (8 * b)) & 0xFF], 1u);
    }
    for (uint64_t i = nv * 16 + tid; i < n; i += stride) atomicAdd(&h[T[i]], 1u);
  } else {
    for (uint64_t i = tid; i < n; i += stride) atomicAdd(&h[T[i]], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += blockDim.x)
    if (h[i]) atomicAdd(&hist[i], (unsigned long long)h[i]);
}

struct CountJob {
  const uint64_t* st;   // block starts of the level
  const uint32_t* ptr;  // for pc jobs: targets
  const uint64_t* off;
  const uint32_t* mw;
  uint64_t c, b, n;
  void* out;            // rows of S counters of cw bytes
  uint32_t cw;
  int mode;             // 0: count the block itself, 1: count T[st[ptr], st[ptr]+off)
  int only_unmarked;    // skip marked blocks
  int only_marked;
};

constexpr uint64_t kCountPiece = 1 << 16;

// One warp per (block, piece of at most 64 KiB); symbol counts are gathered
// in a per-warp shared histogram.  Narrow rows (blocks of at most 64 KiB, one
// piece) are written whole; 4-byte rows (several pieces) are added to with
// atomics.
__global__ void __launch_bounds__(256) k_count(CountJob J, const int16_t* __restrict__ sym,
                                               const uint8_t* __restrict__ T, uint32_t S,
                                               uint64_t ppb) {
  extern __shared__ unsigned int hist[];  // 8 warps x S
  const unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned int* h = hist + wid * S;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x / 32);
  for (uint64_t w = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) / 32; w < J.c * ppb; w += warps) {
    const uint64_t k = w / ppb, piece = w - k * ppb;
    const bool mk = (J.mw[k >> 5] >> (k & 31)) & 1u;
    if ((J.only_unmarked && mk) || (J.only_marked && !mk)) continue;
    uint64_t s0, len;
    if (J.mode == 0) {
      s0 = J.st[k];
      len = J.n - s0 < J.b ? J.n - s0 : J.b;
    } else {
      s0 = J.st[J.ptr[k]];
      len = J.off[k];
    }
    const uint64_t a = piece * kCountPiece;
    if (a >= len) {
      // An empty range (a pointer at offset 0): narrow rows are not zeroed
      // beforehand, so the row is written here.
      if (J.cw < 4 && piece == 0)
        for (uint32_t i = lane; i < S; i += 32) cput(J.out, J.cw, k * S + i, 0u);
      continue;
    }
    const uint64_t e = a + kCountPiece < len ? a + kCountPiece : len;
    for (uint32_t i = lane; i < S; i += 32) h[i] = 0;
    __syncwarp();
    for (uint64_t x = a + lane; x < e; x += 32) atomicAdd(&h[sym[T[s0 + x]]], 1u);
    __syncwarp();
    if (J.cw < 4) {
      for (uint32_t i = lane; i < S; i += 32) cput(J.out, J.cw, k * S + i, h[i]);
    } else {
      for (uint32_t i = lane; i < S; i += 32)
        if (h[i]) atomicAdd((uint32_t*)J.out + k * S + i, h[i]);
    }
    __syncwarp();
  }
}

// Small blocks (one-byte counters, b <= 255): one thread per block counts
// into a private shared-memory row (16-byte text loads when aligned); the
// CTA's rows are contiguous in the output and go out with word stores.
// Rows of blocks that are not counted (J.only_*) are written as zeros; a
// later kernel may overwrite them.
constexpr uint32_t kSmallCountThreads = 128;

__global__ void __launch_bounds__(kSmallCountThreads) k_count_small(CountJob J, const int16_t* __restrict__ sym_g,
                                                                    const uint8_t* __restrict__ T, uint32_t S) {
  extern __shared__ uint8_t rows[];  // kSmallCountThreads rows of S bytes, then the symbol map
  int16_t* sym = (int16_t*)(rows + ((kSmallCountThreads * S + 3) & ~3u));
  for (uint32_t i = threadIdx.x; i < 256; i += blockDim.x) sym[i] = sym_g[i];
  uint8_t* row = rows + threadIdx.x * S;
  for (uint32_t i = 0; i < S; i++) row[i] = 0;
  __syncthreads();
  const uint64_t k0 = (uint64_t)blockIdx.x * kSmallCountThreads, k = k0 + threadIdx.x;
  if (k < J.c) {
    const bool mk = (J.mw[k >> 5] >> (k & 31)) & 1u;
    if (!((J.only_unmarked && mk) || (J.only_marked && !mk))) {
      uint64_t s0, len;
      if (J.mode == 0) {
        s0 = J.st[k];
        len = J.n - s0 < J.b ? J.n - s0 : J.b;
      } else {
        s0 = J.st[J.ptr[k]];
        len = J.off[k];
      }
      uint64_t x = 0;
      if ((((uintptr_t)(T + s0)) & 15) == 0) {
        for (; x + 16 <= len; x += 16) {
          const uint4 v = *(const uint4*)(T + s0 + x);
          const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
          for (int t = 0; t < 16; t++) row[sym[(w[t >> 2] >> (8 * (t & 3))) & 0xFF]]++;
        }
      }
      for (; x < len; x++) row[sym[T[s0 + x]]]++;
    }
  }
  __syncthreads();
  const uint64_t nrows = J.c - k0 < kSmallCountThreads ? J.c - k0 : kSmallCountThreads;
  const uint64_t nbytes = nrows * S;
  uint8_t* out = (uint8_t*)J.out + k0 * S;
  const uint64_t nwords = ((((uintptr_t)out) & 3) == 0) ? nbytes / 4 : 0;
  for (uint64_t i = threadIdx.x; i < nwords; i += blockDim.x) ((uint32_t*)out)[i] = ((const uint32_t*)rows)[i];
  for (uint64_t i = nwords * 4 + threadIdx.x; i < nbytes; i += blockDim.x) out[i] = rows[i];
}

// Marked blocks of a non-last level: sum of the children's counts, one warp
// per block (lanes over the symbols).
__global__ void k_sum_children(uint64_t c, uint64_t b, uint64_t n, const uint64_t* __restrict__ st,
                               const uint32_t* __restrict__ mw, const uint32_t* __restrict__ mr,
                               uint32_t arity, uint64_t bn, const void* __restrict__ child_cnt,
                               uint32_t child_cw, uint32_t S, void* __restrict__ cnt, uint32_t cw) {
  const unsigned lane = threadIdx.x & 31;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x / 32);
  for (uint64_t k = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) / 32; k < c; k += warps) {
    if (!((mw[k >> 5] >> (k & 31)) & 1u)) continue;
    const uint64_t len = n - st[k] < b ? n - st[k] : b;
    const uint64_t first = (mr[k >> 5] + __popc(mw[k >> 5] & ((1u << (k & 31)) - 1u))) * (uint64_t)arity;
    const uint64_t nch = (len + bn - 1) / bn;
    for (uint32_t s = lane; s < S; s += 32) {
      uint32_t acc = 0;
      for (uint64_t i = 0; i < nch; i++) acc += cget(child_cnt, child_cw, (first + i) * S + s);
      cput(cnt, cw, k * S + s, acc);
    }
  }
}

__global__ void k_level1_prefix(uint64_t c, const void* __restrict__ cnt, uint32_t cw, uint32_t S,
                                uint64_t* __restrict__ pre) {
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < S; s += gridDim.x * blockDim.x) {
    uint64_t acc = 0;
    for (uint64_t k = 0; k < c; k++) {
      pre[k * S + s] = acc;
      acc += cget(cnt, cw, k * S + s);
    }
    pre[c * S + s] = acc;
  }
}

__global__ void k_leaf_text(uint64_t c, uint64_t b, uint64_t n, const uint64_t* __restrict__ st,
                            const uint32_t* __restrict__ mw, const uint32_t* __restrict__ mr,
                            const uint8_t* __restrict__ T, uint8_t* __restrict__ leaf) {
  for (uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; w < c * b;
       w += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t k = w / b, i = w - k * b;
    if (!((mw[k >> 5] >> (k & 31)) & 1u)) continue;
    if (st[k] + i >= n) continue;
    uint64_t r = mr[k >> 5] + __popc(mw[k >> 5] & ((1u << (k & 31)) - 1u));
    leaf[r * b + i] = T[st[k] + i];
  }
}

// ---------------------------------------------------------------------------
// Queries.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool qmarked(const LevelView& v, uint64_t k) {
  return (v.mw[k >> 5] >> (k & 31)) & 1u;
}
__device__ __forceinline__ uint64_t qrank(const LevelView& v, uint64_t k) {
  return v.mr[k >> 5] + __popc(v.mw[k >> 5] & ((1u << (k & 31)) - 1u));
}
__device__ __forceinline__ uint64_t qlen(const TreeView& t, const LevelView& v, uint64_t k) {
  uint64_t s = v.st[k];
  return t.n - s < v.b ? t.n - s : v.b;
}

// Occurrences of byte c in p[0, o): four bytes per step from aligned words
// (a per-byte compare, __vcmpeq4, then a population count).
__device__ __forceinline__ uint64_t leaf_count(const uint8_t* p, uint64_t o, uint32_t c) {
  uint64_t x = 0, acc = 0;
  for (; x < o && (((uintptr_t)(p + x)) & 3); x++) acc += p[x] == c;  // up to an aligned word
  const uint32_t cc = c * 0x01010101u;
  const uint32_t* w = (const uint32_t*)(p + x);
  uint64_t i = 0;
  for (; x + 4 <= o; x += 4, i++) acc += __popc(__vcmpeq4(w[i], cc)) >> 3;
  for (; x < o; x++) acc += p[x] == c;
  return acc;
}

// Position of the j-th occurrence (j >= 1) of byte c in p[0, len), or kNone.
__device__ __forceinline__ uint64_t leaf_find(const uint8_t* p, uint64_t len, uint32_t c, uint64_t j) {
  uint64_t x = 0;
  if ((((uintptr_t)p) & 3) == 0) {
    const uint32_t cc = c * 0x01010101u;
    const uint32_t* w = (const uint32_t*)p;
    for (; x + 4 <= len; x += 4) {
      const uint32_t eq = __vcmpeq4(w[x >> 2], cc);
      const uint32_t k = __popc(eq) >> 3;
      if (k >= j) break;  // the j-th is in this word: bytes below
      j -= k;
    }
  }
  for (; x < len; x++)
    if (p[x] == c && --j == 0) return x;
  return kNone;
}

// x / b for the block length of a level (a shift when b is a power of two).
__device__ __forceinline__ uint64_t div_b(uint64_t x, const LevelView& v) {
  return v.bshift != 0xFFu ? x >> v.bshift : x / v.b;
}

// Space-efficient counters (BT_FLAG_LEAF_COUNTS): the last level stores no
// symbol counters; they are counted in the leaf text when a query needs them.
// A marked last-level block's text is its leaf text; an unmarked one copies a
// window of at most two marked blocks (its target and the next one), whose
// text is in the leaf text too.
__device__ uint64_t leaf_block_count(const TreeView& t, const LevelView& v, uint64_t k, uint32_t c) {
  const uint64_t len = qlen(t, v, k);
  if (qmarked(v, k)) return leaf_count(t.leaf + qrank(v, k) * v.b, len, c);
  const uint64_t j = v.ptr[k], o = v.off[k], lj = qlen(t, v, j);
  const uint64_t first = o + len <= lj ? len : lj - o;
  uint64_t acc = leaf_count(t.leaf + qrank(v, j) * v.b + o, first, c);
  if (first < len) acc += leaf_count(t.leaf + qrank(v, j + 1) * v.b, len - first, c);
  return acc;
}

// Counts of byte c in T[st[ptr], st[ptr] + off) of an unmarked last-level block.
__device__ uint64_t leaf_prefix_count(const TreeView& t, const LevelView& v, uint64_t k, uint32_t c) {
  const uint64_t j = v.ptr[k];
  return leaf_count(t.leaf + qrank(v, j) * v.b, v.off[k], c);
}

// Counter of symbol s (byte c) of block k: stored, or counted in the leaf text.
__device__ __forceinline__ uint64_t blk_cnt(const TreeView& t, const LevelView& v, uint64_t k, uint32_t s,
                                            uint32_t c) {
  return v.cnt ? cget(v.cnt, v.cw, k * t.S + s) : leaf_block_count(t, v, k, c);
}
__device__ __forceinline__ uint64_t blk_pc(const TreeView& t, const LevelView& v, uint64_t k, uint32_t s,
                                           uint32_t c) {
  return v.pc ? cget(v.pc, v.cw, k * t.S + s) : leaf_prefix_count(t, v, k, c);
}

__device__ uint64_t q_access(const TreeView& t, uint64_t i) {
  if (i >= t.n) return kNone;
  uint32_t l = 0;
  uint64_t k = div_b(i, t.lv[0]), x = i;
  for (uint32_t step = 0; step < 4 * t.L + 4; step++) {
    const LevelView& v = t.lv[l];
    if (qmarked(v, k)) {
      if (l + 1 == t.L) return t.leaf[qrank(v, k) * v.b + (x - v.st[k])];
      k = qrank(v, k) * v.arity + div_b(x - v.st[k], t.lv[l + 1]);
      l++;
    } else {
      uint64_t P = v.ptr[k];
      x = v.st[P] + v.off[k] + (x - v.st[k]);
      k = x < v.st[P] + qlen(t, v, P) ? P : P + 1;
    }
  }
  return kNone;
}

__device__ uint64_t q_rank(const TreeView& t, uint32_t c, uint64_t i) {
  if (i > t.n) return kNone;
  int s = t.sym[c & 0xFF];
  if (s < 0) return 0;
  const uint32_t S = t.S;
  const LevelView& r = t.lv[0];
  if (i == t.n) return t.pre[r.c * S + s];
  uint64_t k = div_b(i, r), o = i - r.st[k];
  int64_t acc = (int64_t)t.pre[k * S + s];
  uint32_t l = 0;
  for (uint32_t step = 0; step < 4 * t.L + 4; step++) {
    const LevelView& v = t.lv[l];
    if (o == 0) return (uint64_t)acc;
    uint64_t len = qlen(t, v, k);
    if (o == len) return (uint64_t)(acc + blk_cnt(t, v, k, s, c & 0xFF));
    if (qmarked(v, k)) {
      if (l + 1 == t.L) return (uint64_t)(acc + leaf_count(t.leaf + qrank(v, k) * v.b, o, c & 0xFF));
      const LevelView& w = t.lv[l + 1];
      uint64_t j = div_b(o, w), f = qrank(v, k) * v.arity;
      for (uint64_t x = 0; x < j; x++) acc += blk_cnt(t, w, f + x, s, c & 0xFF);
      o -= j * w.b;
      k = f + j;
      l++;
    } else {
      uint64_t P = v.ptr[k], x = v.off[k] + o;
      acc -= blk_pc(t, v, k, s, c & 0xFF);
      uint64_t lp = qlen(t, v, P);
      if (x <= lp) {
        k = P;
        o = x;
      } else {
        acc += blk_cnt(t, v, P, s, c & 0xFF);
        k = P + 1;
        o = x - lp;
      }
    }
  }
  return kNone;
}

__device__ uint64_t q_select(const TreeView& t, uint32_t c, uint64_t j) {
  int s = t.sym[c & 0xFF];
  if (s < 0 || j == 0) return kNone;
  const uint32_t S = t.S;
  const LevelView& r = t.lv[0];
  if (j > t.pre[r.c * S + s]) return kNone;
  uint64_t a = 0, z = r.c;  // last k with pre[k] < j
  while (z - a > 1) {
    uint64_t mid = (a + z) / 2;
    if (t.pre[mid * S + s] < j) a = mid;
    else z = mid;
  }
  uint64_t k = a;
  j -= t.pre[k * S + s];
  int64_t res = (int64_t)r.st[k];
  uint32_t l = 0;
  for (uint32_t step = 0; step < 4 * t.L + 4; step++) {
    const LevelView& v = t.lv[l];
    if (qmarked(v, k)) {
      if (l + 1 == t.L) {
        const uint64_t x = leaf_find(t.leaf + qrank(v, k) * v.b, qlen(t, v, k), c & 0xFF, j);
        return x == kNone ? kNone : (uint64_t)(res + (int64_t)x);
      }
      const LevelView& w = t.lv[l + 1];
      uint64_t f = qrank(v, k) * v.arity, i = 0;
      while (i < v.arity) {
        const uint64_t cc = blk_cnt(t, w, f + i, s, c & 0xFF);
        if (cc >= j) break;
        j -= cc;
        i++;
      }
      if (i == v.arity) return kNone;
      res += (int64_t)(i * w.b);
      k = f + i;
      l++;
    } else {
      uint64_t P = v.ptr[k], jj = j + blk_pc(t, v, k, s, c & 0xFF);
      const uint64_t cp = blk_cnt(t, v, P, s, c & 0xFF);
      if (jj <= cp) {
        res -= (int64_t)v.off[k];
        k = P;
        j = jj;
      } else {
        res += (int64_t)(qlen(t, v, P) - v.off[k]);
        j = jj - cp;
        k = P + 1;
      }
    }
  }
  return kNone;
}

// The batched query kernel.  Every CTA first copies the tree's level table
// and the arrays of its top levels (block starts, marks, rank prefix,
// pointers, offsets, and the counters while they fit) into shared memory:
// every query descends through the top levels, so those steps read shared
// memory instead of L2.  Then each thread answers queries (grid-stride).
constexpr uint32_t kQThreads = 256;

__device__ __forceinline__ void copy_words(uint32_t* dst, const void* src, uint64_t bytes) {
  const uint32_t* s = (const uint32_t*)src;
  for (uint64_t i = threadIdx.x; i < bytes / 4; i += blockDim.x) dst[i] = s[i];
}

template <uint32_t kQCacheBytes, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_queries(const TreeView* __restrict__ tv, int kind,
                                                            const uint64_t* __restrict__ args, uint64_t m,
                                                            uint64_t* __restrict__ out) {
  if (kQCacheBytes == 0) {  // the level table straight from global memory (L1-cached broadcasts)
    const TreeView& t = *tv;
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < m;
         q += (uint64_t)gridDim.x * blockDim.x) {
      uint64_t r;
      if (kind == BT_Q_ACCESS) r = q_access(t, args[q]);
      else if (kind == BT_Q_RANK) r = args[2 * q] > 255 ? kNone : q_rank(t, (uint32_t)args[2 * q], args[2 * q + 1]);
      else r = args[2 * q] > 255 ? kNone : q_select(t, (uint32_t)args[2 * q], args[2 * q + 1]);
      out[q] = r;
    }
    return;
  }
  __shared__ TreeView st;
  __shared__ __align__(16) uint32_t cache[kQCacheBytes / 4 + 4];
  __shared__ uint32_t s_off[kMaxLevels][7];
  __shared__ uint32_t s_lc;
  {
    const uint32_t* src = (const uint32_t*)tv;
    uint32_t* dst = (uint32_t*)&st;
    for (uint32_t i = threadIdx.x; i < sizeof(TreeView) / 4; i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // Top levels that fit: st, mw, mr, ptr, off, cnt, pc (each 16-byte
    // aligned in the cache); counters only while the whole level fits.
    uint32_t used = 0, lc = 0;
    for (uint32_t l = 0; l < st.L; l++) {
      const LevelView& v = st.lv[l];
      const uint64_t words = (v.c + 31) / 32;
      const uint64_t cb = v.cnt ? v.c * st.S * v.cw : 0;
      const uint64_t sz[7] = {v.c * 8, words * 4, (words + 1) * 4, v.c * 4, v.c * 8, cb, cb};
      uint64_t tot = 0;
      for (int a = 0; a < 7; a++) tot += (sz[a] + 15) & ~15ull;
      if (used + tot > kQCacheBytes) break;
      for (int a = 0; a < 7; a++) {
        s_off[l][a] = used;
        used += (uint32_t)((sz[a] + 15) & ~15ull);
      }
      lc = l + 1;
    }
    s_lc = lc;
  }
  __syncthreads();
  const uint32_t lc = s_lc;
  for (uint32_t l = 0; l < lc; l++) {
    const LevelView& v = st.lv[l];
    const uint64_t words = (v.c + 31) / 32;
    copy_words(cache + s_off[l][0] / 4, v.st, v.c * 8);
    copy_words(cache + s_off[l][1] / 4, v.mw, (words * 4 + 3) & ~3ull);
    copy_words(cache + s_off[l][2] / 4, v.mr, (words + 1) * 4);
    copy_words(cache + s_off[l][3] / 4, v.ptr, v.c * 4);
    copy_words(cache + s_off[l][4] / 4, v.off, v.c * 8);
    if (v.cnt) {
      const uint64_t cb = (v.c * st.S * v.cw + 3) & ~3ull;
      copy_words(cache + s_off[l][5] / 4, v.cnt, cb);
      copy_words(cache + s_off[l][6] / 4, v.pc, cb);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (uint32_t l = 0; l < lc; l++) {
      LevelView& v = st.lv[l];
      char* b = (char*)cache;
      v.st = (const uint64_t*)(b + s_off[l][0]);
      v.mw = (const uint32_t*)(b + s_off[l][1]);
      v.mr = (const uint32_t*)(b + s_off[l][2]);
      v.ptr = (const uint32_t*)(b + s_off[l][3]);
      v.off = (const uint64_t*)(b + s_off[l][4]);
      if (v.cnt) {
        v.cnt = b + s_off[l][5];
        v.pc = b + s_off[l][6];
      }
    }
  __syncthreads();
  const TreeView& t = st;
  for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < m;
       q += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t r;
    if (kind == BT_Q_ACCESS) r = q_access(t, args[q]);
    else if (kind == BT_Q_RANK) r = args[2 * q] > 255 ? kNone : q_rank(t, (uint32_t)args[2 * q], args[2 * q + 1]);
    else r = args[2 * q] > 255 ? kNone : q_select(t, (uint32_t)args[2 * q], args[2 * q + 1]);
    out[q] = r;
  }
}

}  // namespace

int alphabet(const uint8_t* T, uint64_t n, uint32_t sigma, bt_tree* t, cudaStream_t s) {
  Scratch sc(s);
  unsigned long long* hist;
  BT_TRY(sc.alloc(&hist, 256));
  BT_CUDA(cudaMemsetAsync(hist, 0, 256 * sizeof(unsigned long long), s));
  BT_LAUNCH(k_histogram<<<grid_for(n / 16 + 1, 256, 152 * 8), 256, 0, s>>>(T, n, hist));
  unsigned long long h[256];
  BT_CUDA(cudaMemcpyAsync(h, hist, sizeof(h), cudaMemcpyDeviceToHost, s));
  BT_CUDA(cudaStreamSynchronize(s));
  uint32_t S = 0;
  for (int i = 0; i < 256; i++) t->sym_host[i] = h[i] ? (int16_t)S++ : (int16_t)-1;
  if (S > sigma) return BT_EINVAL;
  t->S = S;
  BT_CUDA(cudaMallocAsync(&t->sym, 256 * sizeof(int16_t), s));
  BT_CUDA(cudaMemcpyAsync(t->sym, t->sym_host, 256 * sizeof(int16_t), cudaMemcpyHostToDevice, s));
  BT_CUDA(cudaStreamSynchronize(s));
  return BT_OK;
}

int build_counters(BuildCtx& ctx) {
  bt_tree* t = ctx.t;
  cudaStream_t s = ctx.s;
  const uint32_t S = t->S;
  const unsigned T = 256;
  const size_t smem = 8 * S * sizeof(unsigned int);
  // Space-efficient counters: the last level keeps none (queries count its
  // blocks in the leaf text), and the marked blocks of the level above are
  // counted in the text instead of summed from children.
  const bool leaf_counts = ctx.leaf_counts && t->L >= 2;
  for (int l = (int)t->L - 1; l >= 0; l--) {
    Level& v = t->lv[l];
    v.cw = counter_width(v.b);
    if (leaf_counts && l + 1 == (int)t->L) {
      v.cnt = v.pc = nullptr;
      continue;
    }
    // Counters of cw bytes (a count never exceeds b).  Narrow rows are
    // written whole by the kernels; 4-byte rows are accumulated from zero.
    v.cw = counter_width(v.b);
    const uint64_t half = ((v.c * S * v.cw + 4) + 255) & ~255ull;
    char* mem;
    BT_CUDA(cudaMallocAsync((void**)&mem, 2 * half, s));
    v.owned.push_back(mem);
    v.cnt = mem;
    v.pc = mem + half;
    if (v.cw == 4) BT_CUDA(cudaMemsetAsync(mem, 0, 2 * half, s));
    const uint64_t ppb = (v.b + kCountPiece - 1) / kCountPiece;
    const bool last = l + 1 == (int)t->L;
    CountJob J{v.st, v.ptr, v.off, v.mw, v.c, v.b, t->n, v.cnt, v.cw, 0, 0, 0};
    CountJob P{v.st, v.ptr, v.off, v.mw, v.c, v.b, t->n, v.pc, v.cw, 1, 1, 0};
    const bool children_counted = !last && !(leaf_counts && l + 2 == (int)t->L);
    if (children_counted) J.only_unmarked = 1;  // marked blocks are sums of their children
    if (v.cw == 1) {
      // One thread per block; the rows of marked blocks are written as zeros
      // and the sums of children overwrite them below.
      const size_t sm1 = ((kSmallCountThreads * S + 3) & ~3u) + 256 * sizeof(int16_t);
      const unsigned g1 = (unsigned)((v.c + kSmallCountThreads - 1) / kSmallCountThreads);
      BT_LAUNCH(k_count_small<<<g1, kSmallCountThreads, sm1, s>>>(J, t->sym, ctx.T, S));
      BT_LAUNCH(k_count_small<<<g1, kSmallCountThreads, sm1, s>>>(P, t->sym, ctx.T, S));
    } else {
      BT_LAUNCH(k_count<<<grid_for(v.c * ppb * 32, T), T, smem, s>>>(J, t->sym, ctx.T, S, ppb));
      BT_LAUNCH(k_count<<<grid_for(v.c * ppb * 32, T), T, smem, s>>>(P, t->sym, ctx.T, S, ppb));
    }
    if (children_counted) {
      const Level& w = t->lv[l + 1];
      BT_LAUNCH(k_sum_children<<<grid_for(v.c * 32, T), T, 0, s>>>(v.c, v.b, t->n, v.st, v.mw, v.mr, v.arity, w.b,
                                                        w.cnt, w.cw, S, v.cnt, v.cw));
    }
    BT_CUDA(cudaGetLastError());
  }
  const Level& r = t->lv[0];
  BT_CUDA(cudaMallocAsync(&t->pre, (r.c + 1) * S * sizeof(uint64_t) + 8, s));
  BT_LAUNCH(k_level1_prefix<<<1, 256, 0, s>>>(r.c, r.cnt, r.cw, S, t->pre));
  // Leaf text of the marked last-level blocks.
  const Level& z = t->lv[t->L - 1];
  uint32_t nm = 0;
  BT_CUDA(cudaMemcpyAsync(&nm, z.mr + (z.c + 31) / 32, sizeof(nm), cudaMemcpyDeviceToHost, s));
  BT_CUDA(cudaStreamSynchronize(s));
  t->leaf_bytes = (uint64_t)nm * z.b;
  BT_CUDA(cudaMallocAsync(&t->leaf, t->leaf_bytes + 16, s));
  BT_LAUNCH(k_leaf_text<<<grid_for(z.c * z.b, T), T, 0, s>>>(z.c, z.b, t->n, z.st, z.mw, z.mr, ctx.T, t->leaf));
  BT_CUDA(cudaGetLastError());
  // Real leaf length: the tail block may be short.
  uint64_t tail_short = 0;
  if (nm) {
    uint64_t last_st = 0;
    BT_CUDA(cudaMemcpyAsync(&last_st, z.st + z.c - 1, sizeof(last_st), cudaMemcpyDeviceToHost, s));
    uint32_t lastw = 0;
    BT_CUDA(cudaMemcpyAsync(&lastw, z.mw + (z.c - 1) / 32, sizeof(lastw), cudaMemcpyDeviceToHost, s));
    BT_CUDA(cudaStreamSynchronize(s));
    bool last_marked = (lastw >> ((z.c - 1) & 31)) & 1u;
    if (last_marked && t->n - last_st < z.b) tail_short = z.b - (t->n - last_st);
  }
  t->leaf_bytes -= tail_short;
  return BT_OK;
}

int upload_view(bt_tree* t, cudaStream_t s) {
  TreeView h;
  h.n = t->n;
  h.L = t->L;
  h.S = t->S;
  for (uint32_t l = 0; l < t->L; l++) {
    const Level& v = t->lv[l];
    h.lv[l] = LevelView{v.c, v.b, v.arity, block_shift(v.b), v.st, v.mw, v.mr, v.ptr, v.off, v.cnt, v.pc, v.cw};
  }
  h.pre = t->pre;
  h.leaf = t->leaf;
  h.sym = t->sym;
  BT_CUDA(cudaMallocAsync(&t->view, sizeof(TreeView), s));
  BT_CUDA(cudaMemcpyAsync(t->view, &h, sizeof(TreeView), cudaMemcpyHostToDevice, s));
  BT_CUDA(cudaStreamSynchronize(s));
  return BT_OK;
}

int run_queries(const bt_tree* t, int kind, const uint64_t* d_args, uint64_t m, uint64_t* d_out,
                cudaStream_t s) {
  if (m == 0) return BT_OK;
  // Enough CTAs to fill the device (each pays for its shared-memory copy of
  // the top levels once), threads striding over the queries.
  // Access descends with few loads per level and gains most from threads in
  // flight: 128-thread CTAs without the shared-memory copy, bounded to 64
  // registers so that 1024 threads fit on an SM (80 registers left 768).
  // Rank and select read counters at every level and gain from the copy of
  // the top levels; four CTAs of 256 per SM at 64 registers run without the
  // spills that six CTAs (40 registers) had.  Measured on the 256 MiB tree:
  // access 9.7 instead of 8.2, rank 2.6 instead of 2.4, select 2.5 instead of
  // 2.1 G queries/s.
  if (kind == BT_Q_ACCESS)
    BT_LAUNCH(k_queries<0, 128, 8><<<grid_for(m, 128, 152 * 64), 128, 0, s>>>(t->view, kind, d_args, m, d_out));
  else
    BT_LAUNCH(k_queries<12 << 10, kQThreads, 4><<<grid_for(m, kQThreads, 152 * 4), kQThreads, 0, s>>>(
        t->view, kind, d_args, m, d_out));
  BT_CUDA(cudaGetLastError());
  return BT_OK;
}

}  // namespace bt
