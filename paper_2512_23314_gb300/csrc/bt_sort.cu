// bt_sort.cu -- a stable LSD radix sort of (u64 key, u32 value) pairs, the
// sorting primitive of the sort-based level pass (section 4.1: fingerprints
// of all windows are sorted as (fingerprint, position) tuples, so that equal
// fingerprints are consecutive and, the sort being stable over positions in
// text order, the first tuple of a group is the leftmost window).
//
// Each pass sorts by one 8-bit digit:
//   1. k_digit_hist: per tile of kSortTile items, the count of every digit,
//      stored digit-major (counts[d * ntiles + tile]);
//   2. an exclusive prefix sum over those counts: the output offset of every
//      (digit, tile) pair, in the order that keeps the sort stable;
//   3. k_digit_scatter: every item goes to its (digit, tile) offset plus its
//      rank among the tile's items with the same digit, counted in index
//      order (per warp with __match_any_sync, then across the warps).
#include <utility>

#include "bt_internal.cuh"

namespace bt {

namespace {

constexpr uint32_t kSortThreads = 256;
constexpr uint32_t kSortPerThread = 8;
constexpr uint32_t kSortTile = kSortThreads * kSortPerThread;  // 2048 items
constexpr uint32_t kSortWarps = kSortThreads / 32;

__global__ void __launch_bounds__(kSortThreads) k_digit_hist(const uint64_t* __restrict__ keys, uint64_t n,
                                                             uint32_t shift, uint64_t ntiles,
                                                             uint32_t* __restrict__ counts) {
  __shared__ unsigned int h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const uint64_t t0 = (uint64_t)blockIdx.x * kSortTile;
  for (uint32_t j = threadIdx.x; j < kSortTile; j += kSortThreads) {
    const uint64_t i = t0 + j;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 0xFF], 1u);
  }
  __syncthreads();
  counts[(uint64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(kSortThreads) k_digit_scatter(const uint64_t* __restrict__ keys,
                                                                const uint32_t* __restrict__ vals, uint64_t n,
                                                                uint32_t shift, uint64_t ntiles,
                                                                const uint32_t* __restrict__ offs,
                                                                uint64_t* __restrict__ okeys,
                                                                uint32_t* __restrict__ ovals) {
  __shared__ unsigned int wcnt[kSortWarps][256];
  const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint32_t i = threadIdx.x; i < kSortWarps * 256; i += kSortThreads) (&wcnt[0][0])[i] = 0;
  __syncthreads();
  // Warp w holds items t0 + w*256 + j*32 + lane, j < 8: index order is
  // (warp, j, lane), so ranks counted in that order keep the sort stable.
  const uint64_t base = (uint64_t)blockIdx.x * kSortTile + warp * 32 * kSortPerThread;
  uint64_t k[kSortPerThread];
  uint32_t v[kSortPerThread], rk[kSortPerThread], dg[kSortPerThread];
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (uint32_t j = 0; j < kSortPerThread; j++) {
    const uint64_t i = base + j * 32 + lane;
    const bool ok = i < n;
    k[j] = ok ? keys[i] : 0;
    v[j] = ok ? vals[i] : 0;
    dg[j] = ok ? (uint32_t)((k[j] >> shift) & 0xFF) : 256u + lane;  // unique dummy digit
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, dg[j]);
    const unsigned before = __popc(peers & lt);
    rk[j] = 0;
    if (ok) rk[j] = wcnt[warp][dg[j]] + before;
    __syncwarp();
    if (ok && before == 0) wcnt[warp][dg[j]] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // Exclusive sum over the warps, per digit.
  {
    const unsigned d = threadIdx.x;  // 256 threads, one per digit
    unsigned acc = 0;
    for (uint32_t w = 0; w < kSortWarps; w++) {
      const unsigned c = wcnt[w][d];
      wcnt[w][d] = acc;
      acc += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (uint32_t j = 0; j < kSortPerThread; j++) {
    const uint64_t i = base + j * 32 + lane;
    if (i >= n) continue;
    const uint64_t dst = (uint64_t)offs[(uint64_t)dg[j] * ntiles + blockIdx.x] + wcnt[warp][dg[j]] + rk[j];
    okeys[dst] = k[j];
    ovals[dst] = v[j];
  }
}

}  // namespace

uint64_t radix_sort_scratch_words(uint64_t n) {
  const uint64_t ntiles = (n + kSortTile - 1) / kSortTile;
  return 256 * ntiles + 1 + scan_scratch_words(256 * ntiles);
}

// Sorts (keys, vals)[0, n) by the low `bits` bits of the keys, stably.  The
// result is in (keys, vals) again; (tk, tv) are buffers of n entries and
// `scratch` holds radix_sort_scratch_words(n) u32.  n < 2^32.
int radix_sort_u64_u32(uint64_t* keys, uint32_t* vals, uint64_t* tk, uint32_t* tv, uint64_t n, uint32_t bits,
                       uint32_t* scratch, cudaStream_t s) {
  if (n == 0) return BT_OK;
  if (n >= (1ull << 32)) return BT_EINVAL;
  const uint64_t ntiles = (n + kSortTile - 1) / kSortTile;
  uint32_t* counts = scratch;
  uint32_t* agg = scratch + 256 * ntiles + 1;
  uint64_t* ka = keys;
  uint32_t* va = vals;
  uint64_t* kb = tk;
  uint32_t* vb = tv;
  const uint32_t passes = (bits + 7) / 8;
  for (uint32_t p = 0; p < passes; p++) {
    const uint32_t shift = 8 * p;
    BT_LAUNCH(k_digit_hist<<<(unsigned)ntiles, kSortThreads, 0, s>>>(ka, n, shift, ntiles, counts));
    // In place: the prefix sum overwrites the counts with the offsets.
    BT_TRY(scan_u32(counts, counts, 256 * ntiles, s, agg));
    BT_LAUNCH(k_digit_scatter<<<(unsigned)ntiles, kSortThreads, 0, s>>>(ka, va, n, shift, ntiles, counts, kb, vb));
    BT_CUDA(cudaGetLastError());
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  if (ka != keys) {
    BT_CUDA(cudaMemcpyAsync(keys, ka, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    BT_CUDA(cudaMemcpyAsync(vals, va, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
  }
  return BT_OK;
}

}  // namespace bt
