// bt_internal.cuh -- shared types of the CUDA block-tree library.
//
// Device data layout (one tree, all in HBM):
//   text        u8[n]          the input (the caller's device buffer, or a copy)
//   H           u64[n + 1]     Karp-Rabin prefix fingerprints H(p) (section 2),
//                              during construction only
//   per level l (blocks in text order):
//     st        u64[c]         block starts (multiples of b_l)
//     mw        u32[ceil(c/32)] mark bits, bit k%32 of word k/32
//     mr        u32[words + 1] exclusive prefix popcounts of mw (rank support)
//     ptr       u32[c]         unmarked: index of the block holding the leftmost
//                              occurrence of the block's string
//     off       u64[c]         unmarked: offset of that occurrence in block ptr
//     cnt       u32[c * S]     symbol counts of the block (S distinct symbols)
//     pc        u32[c * S]     unmarked: symbol counts of T[st[ptr], st[ptr]+off)
//   pre         u64[(c_1+1)*S] level 1: symbol counts of T[0, st[k])
//   leaf        u8[...]        text of the marked last-level blocks, block r at r*b_L
// A marked block of a non-last level with mark rank r has its children at
// indices r*arity .. r*arity + ceil(len/b_{l+1}) - 1 of the next level.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <memory>
#include <string>
#include <vector>

#include "bt.h"

namespace bt {

constexpr uint32_t kPrefixStride = 32;  // spacing of the stored prefix fingerprints
constexpr uint64_t kNone = ~0ull;
constexpr uint32_t kNoSlot = 0xFFFFFFFFu;

// ---------------------------------------------------------------------------
// Arithmetic modulo q.  Mersenne61 is the production modulus 2^61-1: a 61x61
// bit product is split with a 64-bit high multiply and folded twice, using
// 2^61 = 1 (mod q).  SmallMod (q < 2^32) exists only so tests can force
// fingerprint collisions; its products fit in 64 bits.
// ---------------------------------------------------------------------------
struct Mersenne61 {
  static constexpr uint64_t Q = (1ull << 61) - 1;
  __host__ __device__ __forceinline__ uint64_t q() const { return Q; }
  __host__ __device__ __forceinline__ uint64_t mul(uint64_t a, uint64_t b) const {
#ifdef __CUDA_ARCH__
    uint64_t lo = a * b, hi = __umul64hi(a, b);
#else
    unsigned __int128 p = (unsigned __int128)a * b;
    uint64_t lo = (uint64_t)p, hi = (uint64_t)(p >> 64);
#endif
    uint64_t r = (lo & Q) + ((lo >> 61) | (hi << 3));
    r = (r & Q) + (r >> 61);
    return r >= Q ? r - Q : r;
  }
  __host__ __device__ __forceinline__ uint64_t add(uint64_t a, uint64_t b) const {
    uint64_t s = a + b;
    return s >= Q ? s - Q : s;
  }
  __host__ __device__ __forceinline__ uint64_t sub(uint64_t a, uint64_t b) const {
    return a >= b ? a - b : a + Q - b;
  }
};

struct SmallMod {
  uint64_t Q;
  __host__ __device__ __forceinline__ uint64_t q() const { return Q; }
  __host__ __device__ __forceinline__ uint64_t mul(uint64_t a, uint64_t b) const { return (a * b) % Q; }
  __host__ __device__ __forceinline__ uint64_t add(uint64_t a, uint64_t b) const {
    uint64_t s = a + b;
    return s >= Q ? s - Q : s;
  }
  __host__ __device__ __forceinline__ uint64_t sub(uint64_t a, uint64_t b) const {
    return a >= b ? a - b : a + Q - b;
  }
};

template <class M>
__host__ __device__ inline uint64_t pow_mod(const M& m, uint64_t a, uint64_t e) {
  uint64_t r = 1 % m.q();
  a %= m.q();
  while (e) {
    if (e & 1) r = m.mul(r, a);
    a = m.mul(a, a);
    e >>= 1;
  }
  return r;
}

// phi(p, p+len) = H(p+len) - H(p) * B^len  (BL = B^len), from the prefix
// fingerprints H at every position (section 2): two loads and one product.
template <class M>
__device__ __forceinline__ uint64_t window_fast(const M& m, const uint64_t* __restrict__ H,
                                               uint64_t BL, uint64_t p, uint64_t len) {
  return m.sub(H[p + len], m.mul(H[p], BL));
}

__host__ __device__ __forceinline__ uint64_t mix64(uint64_t x) {
  x ^= x >> 31;
  x *= 0x7FB5D329728EA185ull;
  x ^= x >> 27;
  x *= 0x81DADEF4BC2DD44Dull;
  x ^= x >> 33;
  return x;
}

// ---------------------------------------------------------------------------
// Host-side tree.
// ---------------------------------------------------------------------------
struct Level {
  uint64_t c = 0;        // blocks
  uint64_t b = 0;        // nominal block length
  uint32_t arity = 0;    // children per full marked block (0 on the last level)
  uint64_t nmarked = 0;
  uint64_t* st = nullptr;
  uint32_t* mw = nullptr;
  uint32_t* mr = nullptr;
  uint32_t* ptr = nullptr;
  uint64_t* off = nullptr;
  uint64_t* lo = nullptr;  // exact leftmost occurrence of every block (pruning)
  void* cnt = nullptr;     // counter rows, cw bytes per counter
  void* pc = nullptr;
  uint32_t cw = 4;
  uint64_t stats[BT_ST_FIELDS] = {};
  std::vector<void*> owned;  // device allocations holding this level's arrays
};

// Device-side view of one level, passed by value to kernels.
struct LevelView {
  uint64_t c, b;
  uint32_t arity;
  uint32_t bshift;  // log2(b) when b is a power of two, else 0xFF
  const uint64_t* st;
  const uint32_t* mw;
  const uint32_t* mr;
  const uint32_t* ptr;
  const uint64_t* off;
  const void* cnt;  // symbol counters of the blocks, cw bytes each (1, 2 or 4)
  const void* pc;
  uint32_t cw;
};

__host__ __device__ inline uint32_t block_shift(uint64_t b) {
  if (b == 0 || (b & (b - 1))) return 0xFFu;
  uint32_t s = 0;
  while ((1ull << s) < b) s++;
  return s;
}

// Bytes per symbol counter of a level with block length b: a count never
// exceeds b.
__host__ __device__ inline uint32_t counter_width(uint64_t b) { return b <= 0xFF ? 1 : b <= 0xFFFF ? 2 : 4; }

// Counter i of a row array with w-byte entries.
__device__ __forceinline__ uint32_t cget(const void* a, uint32_t w, uint64_t i) {
  return w == 1 ? ((const uint8_t*)a)[i] : w == 2 ? ((const uint16_t*)a)[i] : ((const uint32_t*)a)[i];
}
__device__ __forceinline__ void cput(void* a, uint32_t w, uint64_t i, uint32_t v) {
  if (w == 1) ((uint8_t*)a)[i] = (uint8_t)v;
  else if (w == 2) ((uint16_t*)a)[i] = (uint16_t)v;
  else ((uint32_t*)a)[i] = v;
}

constexpr int kMaxLevels = 64;

struct TreeView {
  uint64_t n;
  uint32_t L, S;
  LevelView lv[kMaxLevels];
  const uint64_t* pre;
  const uint8_t* leaf;
  const int16_t* sym;  // byte -> dense symbol, -1 if absent
};

}  // namespace bt

struct bt_tree {
  uint64_t n = 0;
  uint32_t tau = 0, leaf_len = 0, L = 0;
  int prune = 1;
  uint64_t seed = 0, B = 0, q = 0;
  std::vector<bt::Level> lv;
  uint8_t* leaf = nullptr;
  uint64_t leaf_bytes = 0;
  uint64_t* pre = nullptr;
  int16_t* sym = nullptr;  // device map
  int16_t sym_host[256];
  uint32_t S = 0;
  bt::TreeView* view = nullptr;  // device copy of the view
  int device = 0;
  uint64_t dev_bytes = 0;        // device memory held by the tree
  // Trees of a batched build live in a region of the batch's output pool:
  // the pool is released when the last of its trees is freed, and the
  // arrays above are not freed one by one.
  std::shared_ptr<void> slab;
  uint64_t batch_cycles[6] = {};  // batched build: SM cycles per phase of its CTA
};

namespace bt {

// Error helpers ------------------------------------------------------------
struct Err {
  int code = BT_OK;
};
#define BT_CUDA(call)                                   \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) {                            \
      bt::note_cuda_error(e_, #call, __FILE__, __LINE__); \
      return e_ == cudaErrorMemoryAllocation ? BT_ENOMEM : BT_ECUDA; \
    }                                                   \
  } while (0)
#define BT_TRY(expr)              \
  do {                            \
    int rc_ = (expr);             \
    if (rc_ != BT_OK) return rc_; \
  } while (0)

void note_cuda_error(cudaError_t e, const char* what, const char* file, int line);

// Every kernel launch of the library goes through BT_LAUNCH, which counts it
// (bt_launch_count reports the total).
void note_launch();
#define BT_LAUNCH(...)  \
  do {                  \
    ::bt::note_launch(); \
    __VA_ARGS__;        \
  } while (0)

// CUDA-event timing of selected kernels on the stream they are launched on,
// enabled by bt_profile_enable.  A ProfScope records an event pair around
// the launches in its lifetime; `bytes` is the algorithmic traffic they move.
struct ProfScope {
  int slot = -1;
  cudaStream_t s;
  ProfScope(const char* name, cudaStream_t st, uint64_t bytes);
  ~ProfScope();
};

// Device status word shared by the kernels of one build.
struct Status {
  unsigned long long error;          // nonzero: a device-side invariant failed
  unsigned long long njobs;          // verification jobs
  unsigned long long nsuspect;       // keys that need the exact rescan
  unsigned long long collisions;     // verification mismatches
  unsigned long long verify_bytes;   // bytes compared by verification
  unsigned long long next_c;         // blocks of the next level
  unsigned long long last_start;     // start of the last block of the next level
  unsigned long long lo_tail;        // leftmost occurrence of the short tail block
  unsigned long long lo_tailpair;    // leftmost occurrence of the pair ending in the tail
  unsigned long long tail_susp;      // tail key verification state
  unsigned long long rounds;         // pruning rounds used
  unsigned long long undecided;      // pruning: candidates left after a round
  unsigned long long pad[4];
};

// Test hook (bt_test_alloc_limit): the largest single device allocation a
// build may make; larger ones fail as if the device were out of memory.
// 0: no limit.
bool alloc_allowed(uint64_t bytes);

// Scratch allocator bound to a stream (stream-ordered pool allocations).
struct Scratch {
  cudaStream_t s;
  std::vector<void*> ptrs;
  explicit Scratch(cudaStream_t st) : s(st) {}
  template <class T>
  int alloc(T** p, uint64_t count) {
    void* q = nullptr;
    if (!alloc_allowed((count ? count : 1) * sizeof(T))) return BT_ENOMEM;
    cudaError_t e = cudaMallocAsync(&q, (count ? count : 1) * sizeof(T), s);
    if (e != cudaSuccess) {
      note_cuda_error(e, "cudaMallocAsync", __FILE__, __LINE__);
      return e == cudaErrorMemoryAllocation ? BT_ENOMEM : BT_ECUDA;
    }
    ptrs.push_back(q);
    *p = (T*)q;
    return BT_OK;
  }
  ~Scratch() {
    for (void* p : ptrs) cudaFreeAsync(p, s);
  }
};

// Growable scratch arena of one build: a level carves all its temporary
// buffers out of one device allocation (a bump pointer reset per level), so
// a level costs one allocation at most instead of dozens.  In dry mode take()
// only adds up the bytes a carving needs.
struct Arena {
  cudaStream_t s = nullptr;
  char* base = nullptr;
  uint64_t cap = 0, used = 0;
  bool dry = false;
  void begin_dry() {
    dry = true;
    used = 0;
  }
  int reserve() {  // after a dry carving: make room for it, then carve for real
    const uint64_t need = used + 256;
    dry = false;
    used = 0;
    if (need <= cap) return BT_OK;
    const uint64_t grown = 2 * cap;  // grow at least twofold: fewer, larger allocations
    if (base) cudaFreeAsync(base, s);
    base = nullptr;
    cap = 0;
    const uint64_t want = need + need / 4 > grown ? need + need / 4 : grown;
    if (!alloc_allowed(want)) return BT_ENOMEM;
    cudaError_t e = cudaMallocAsync((void**)&base, want, s);
    if (e != cudaSuccess) {
      note_cuda_error(e, "cudaMallocAsync", __FILE__, __LINE__);
      return e == cudaErrorMemoryAllocation ? BT_ENOMEM : BT_ECUDA;
    }
    cap = want;
    return BT_OK;
  }
  template <class T>
  T* take(uint64_t count) {
    used = (used + 255) & ~255ull;
    T* p = dry ? nullptr : (T*)(base + used);
    used += (count ? count : 1) * sizeof(T);
    return p;
  }
  void release() {
    if (base) cudaFreeAsync(base, s);
    base = nullptr;
    cap = used = 0;
  }
};

// Library-wide launch helpers.
inline unsigned grid_for(uint64_t work, unsigned threads, unsigned cap = 152u * 32u) {
  uint64_t g = (work + threads - 1) / threads;
  if (g == 0) g = 1;
  return (unsigned)(g < cap ? g : cap);
}

// Host entry points implemented across the .cu files --------------------------
int prefix_fingerprints(const uint8_t* d_text, uint64_t n, uint64_t B, uint64_t q,
                        uint64_t* d_Hs, cudaStream_t s);
// H[p] for every p in [0, n] from the stride-32 values Hs (n/32 + 1 entries).
int expand_prefix(const uint8_t* d_text, uint64_t n, uint64_t B, uint64_t q,
                  const uint64_t* d_Hs, uint64_t* d_H, cudaStream_t s);

// Exclusive prefix sum of d_in[0, n) into d_out[0, n]; d_out[n] = total.
int scan_u32(const uint32_t* d_in, uint32_t* d_out, uint64_t n, cudaStream_t s);
// Same, with caller-provided scratch of scan_scratch_words(n) entries.
int scan_u32(const uint32_t* d_in, uint32_t* d_out, uint64_t n, cudaStream_t s, uint32_t* agg);
inline uint64_t scan_scratch_words(uint64_t n) { return (n + 1023) / 1024 + 1; }
int scan_u64(const uint64_t* d_in, uint64_t* d_out, uint64_t n, cudaStream_t s);

// Stable LSD radix sort of (keys, vals)[0, n) by the low `bits` key bits
// (bt_sort.cu); (tk, tv) hold n entries each, scratch radix_sort_scratch_words(n).
uint64_t radix_sort_scratch_words(uint64_t n);
int radix_sort_u64_u32(uint64_t* keys, uint32_t* vals, uint64_t* tk, uint32_t* tv, uint64_t n, uint32_t bits,
                       uint32_t* scratch, cudaStream_t s);

struct BuildCtx {
  bt_tree* t;
  const uint8_t* T;   // device text
  uint64_t* H;        // prefix fingerprints at every position, n + 1 entries
  Arena arena;        // per-level scratch
  Status* st;         // device status
  Status* st_host;    // pinned mirror
  cudaStream_t s;
  uint64_t verify_bytes = 0, collisions = 0;
  int dense_scan = 0;  // probe every window (diagnostic) instead of the anchored scan
  int tiny_queue = 0;  // test hook: a 64-entry candidate queue (forces the overflow path)
  int force_list = 0;  // test hook: build the selected-gram list for any text length
  int two_phase = 0;   // BT_FLAG_TWO_PHASE: test every level's windows in two phases
  int leaf_counts = 0; // BT_FLAG_LEAF_COUNTS: no stored counters on the last level
  int sort_scan = 0;   // BT_FLAG_SORT_SCAN: leftmost windows by sorting instead of probing
  uint32_t partitions = 0;  // parts of the sort-based pass (domain decomposition; <= 1: one)
  uint64_t prev_cands = 0;  // windows the previous level's scan proposed (sizes the next queue)
  // Selected-gram list of the whole text (built once when levels can use it):
  // chunk j of 128 positions lists its grams at gl_chunk[j] .. gl_chunk[j+1].
  const uint32_t* gl_chunk = nullptr;
  const uint32_t* gl_mx = nullptr;
  const uint32_t* gl_x = nullptr;  // positions (texts are shorter than 2^32)
  uint32_t gl_total = 0;
  ~BuildCtx() { arena.release(); }
};

int build_levels(BuildCtx& ctx);
int prune_tree(BuildCtx& ctx, uint64_t max_rounds);
int build_counters(BuildCtx& ctx);
int sync_status(BuildCtx& ctx);

}  // namespace bt
