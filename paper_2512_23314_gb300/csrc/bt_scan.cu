// bt_scan.cu -- device-wide prefix operations.
//
//  * scan_u32 / scan_u64: exclusive prefix sums (rank support of the mark
//    bit vectors, job offsets).
//  * prefix_fingerprints: the Karp-Rabin prefix H(32 j) of the whole text
//    (section 2 defines phi; Lemmas 7 and 8 of section 4.1 compute all
//    fingerprints with an all-prefix operation).  Each 32-byte chunk is hashed
//    by Horner, then the chunks are combined with the associative operator
//    (h1, P1) (x) (h2, P2) = (h1 * P2 + h2, P1 * P2) of the all-prefix lemma
//    (Lemma 1); every chunk has the same length, so P is a power of
//    B^32 determined by the number of chunks combined and is read from a
//    table instead of being carried.
// Three passes: a CTA-local scan of 1024 items, a single-CTA scan of the CTA
// aggregates, and a pass that folds each CTA's prefix into its items.
#include <cstdio>
#include <mutex>

#include "bt_internal.cuh"

namespace bt {

namespace {

constexpr int kTile = 1024;  // items per CTA (one per thread)

template <class T>
__device__ T cta_exclusive_sum(T v, T* sm, T* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T x = v;
  for (int d = 1; d < 32; d <<= 1) {
    T o = __shfl_up_sync(0xFFFFFFFFu, x, d);
    if (lane >= d) x += o;
  }
  if (lane == 31) sm[warp] = x;
  __syncthreads();
  if (warp == 0) {
    T w = sm[lane];
    for (int d = 1; d < 32; d <<= 1) {
      T o = __shfl_up_sync(0xFFFFFFFFu, w, d);
      if (lane >= d) w += o;
    }
    sm[lane] = w;
  }
  __syncthreads();
  T incl = x + (warp > 0 ? sm[warp - 1] : T(0));
  *total = sm[31];
  __syncthreads();
  return incl - v;
}

template <class T>
__global__ void __launch_bounds__(kTile) k_sum_local(const T* __restrict__ in, T* __restrict__ out,
                                                     uint64_t n, T* __restrict__ agg) {
  __shared__ T sm[32];
  uint64_t i = (uint64_t)blockIdx.x * kTile + threadIdx.x;
  T v = i < n ? in[i] : T(0);
  T tot;
  T e = cta_exclusive_sum(v, sm, &tot);
  if (i < n) out[i] = e;
  if (threadIdx.x == 0) agg[blockIdx.x] = tot;
}

// Exclusive scan of the aggregates by one CTA; agg[na] receives the total.
template <class T>
__global__ void __launch_bounds__(kTile) k_sum_aggs(T* agg, uint64_t na) {
  __shared__ T sm[32];
  T carry = 0;
  for (uint64_t base = 0; base < na; base += kTile) {
    uint64_t i = base + threadIdx.x;
    T v = i < na ? agg[i] : T(0);
    T tot;
    T e = cta_exclusive_sum(v, sm, &tot);
    if (i < na) agg[i] = carry + e;
    carry += tot;
  }
  if (threadIdx.x == 0) agg[na] = carry;
}

template <class T>
__global__ void __launch_bounds__(kTile) k_sum_add(T* out, uint64_t n, const T* __restrict__ agg) {
  uint64_t i = (uint64_t)blockIdx.x * kTile + threadIdx.x;
  if (i < n) out[i] += agg[blockIdx.x];
  if (i == 0) {
    uint64_t na = (n + kTile - 1) / kTile;
    out[n] = agg[na];
  }
}

template <class T>
int scan_sum(const T* in, T* out, uint64_t n, cudaStream_t s) {
  if (n == 0) {
    BT_CUDA(cudaMemsetAsync(out, 0, sizeof(T), s));
    return BT_OK;
  }
  uint64_t na = (n + kTile - 1) / kTile;
  if (na > (1ull << 31)) return BT_EINVAL;
  Scratch sc(s);
  T* agg;
  BT_TRY(sc.alloc(&agg, na + 1));
  BT_LAUNCH(k_sum_local<T><<<(unsigned)na, kTile, 0, s>>>(in, out, n, agg));
  BT_LAUNCH(k_sum_aggs<T><<<1, kTile, 0, s>>>(agg, na));
  BT_LAUNCH(k_sum_add<T><<<(unsigned)na, kTile, 0, s>>>(out, n, agg));
  BT_CUDA(cudaGetLastError());
  return BT_OK;
}

// ---------------------------------------------------------------------------
// Karp-Rabin all-prefix.
// ---------------------------------------------------------------------------

// Inclusive scan of chunk fingerprints within a CTA.  pw[i] = X^i, where X
// is B raised to the length of one item, for i <= 1024.
template <class M>
__device__ uint64_t cta_kr_scan(const M& m, uint64_t h, const uint64_t* __restrict__ pw,
                                uint64_t* sm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int d = 1; d < 32; d <<= 1) {
    uint64_t o = __shfl_up_sync(0xFFFFFFFFu, h, d);
    if (lane >= d) h = m.add(m.mul(o, pw[d]), h);
  }
  if (lane == 31) sm[warp] = h;
  __syncthreads();
  if (warp == 0) {
    uint64_t w = sm[lane];
    for (int d = 1; d < 32; d <<= 1) {
      uint64_t o = __shfl_up_sync(0xFFFFFFFFu, w, d);
      if (lane >= d) w = m.add(m.mul(o, pw[32 * d]), w);
    }
    sm[lane] = w;
  }
  __syncthreads();
  if (warp > 0) h = m.add(m.mul(sm[warp - 1], pw[lane + 1]), h);
  __syncthreads();
  return h;
}

// Horner fingerprint of each 32-byte chunk, scanned within the CTA; the
// CTA-inclusive value of chunk j goes to Hs[j+1], the CTA total to agg.
template <class M>
__global__ void __launch_bounds__(kTile) k_kr_local(M m, const uint8_t* __restrict__ T,
                                                    uint64_t nchunks, uint64_t B,
                                                    const uint64_t* __restrict__ pw1,
                                                    uint64_t* __restrict__ Hs,
                                                    uint64_t* __restrict__ agg) {
  __shared__ uint64_t sm[32];
  uint64_t j = (uint64_t)blockIdx.x * kTile + threadIdx.x;
  uint64_t h = 0;
  if (j < nchunks) {
    const uint8_t* p = T + j * kPrefixStride;
    if ((((uintptr_t)p) & 15) == 0) {  // two 16-byte loads
      const uint4 v0 = ((const uint4*)p)[0], v1 = ((const uint4*)p)[1];
      const uint32_t wv[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
      for (int i = 0; i < (int)kPrefixStride; i++)
        h = m.add(m.mul(h, B), (uint64_t)((wv[i >> 2] >> (8 * (i & 3))) & 0xFFu) + 1);
    } else {
#pragma unroll 8
      for (int i = 0; i < (int)kPrefixStride; i++) h = m.add(m.mul(h, B), (uint64_t)p[i] + 1);
    }
  }
  h = cta_kr_scan(m, h, pw1, sm);
  if (j < nchunks) Hs[j + 1] = h;
  uint64_t base = (uint64_t)blockIdx.x * kTile;
  uint64_t last = (nchunks - base < kTile ? nchunks - base : kTile) - 1;
  if (threadIdx.x == last) agg[blockIdx.x] = h;
}

// pre[i] = fingerprint of chunks [0, 1024 i): scan of the CTA totals by one
// CTA with X = B^(32*1024) (pw2[i] = X^i).
template <class M>
__global__ void __launch_bounds__(kTile) k_kr_aggs(M m, uint64_t* __restrict__ agg, uint64_t na,
                                                   const uint64_t* __restrict__ pw2) {
  __shared__ uint64_t sm[32];
  __shared__ uint64_t carry_s;
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  for (uint64_t base = 0; base < na; base += kTile) {
    uint64_t i = base + threadIdx.x;
    uint64_t v = i < na ? agg[i] : 0;
    uint64_t incl = cta_kr_scan(m, v, pw2, sm);
    uint64_t carry = carry_s;
    uint64_t g = m.add(m.mul(carry, pw2[threadIdx.x + 1]), incl);
    __syncthreads();
    uint64_t cnt = na - base < kTile ? na - base : kTile;
    if (i < na) agg[i] = g;  // inclusive prefix over CTA totals [0, i]
    if (threadIdx.x == cnt - 1) carry_s = g;
    __syncthreads();
  }
}

template <class M>
__global__ void __launch_bounds__(kTile) k_kr_add(M m, uint64_t* __restrict__ Hs, uint64_t nchunks,
                                                  const uint64_t* __restrict__ agg,
                                                  const uint64_t* __restrict__ pw1) {
  uint64_t j = (uint64_t)blockIdx.x * kTile + threadIdx.x;
  if (j == 0) Hs[0] = 0;
  if (j >= nchunks || blockIdx.x == 0) return;
  uint64_t pre = agg[blockIdx.x - 1];
  Hs[j + 1] = m.add(m.mul(pre, pw1[threadIdx.x + 1]), Hs[j + 1]);
}

template <class M>
int kr_prefix(const M& m, const uint8_t* T, uint64_t n, uint64_t B, uint64_t* Hs, cudaStream_t s) {
  uint64_t nchunks = n / kPrefixStride;
  if (nchunks == 0) {
    BT_CUDA(cudaMemsetAsync(Hs, 0, sizeof(uint64_t), s));
    return BT_OK;
  }
  uint64_t na = (nchunks + kTile - 1) / kTile;
  // Power tables: pw1[i] = P^i, pw2[i] = P^(1024 i), P = B^32.
  std::vector<uint64_t> h(2 * (kTile + 1));
  uint64_t P = pow_mod(m, B, kPrefixStride), P1024 = pow_mod(m, P, kTile);
  h[0] = 1 % m.q();
  h[kTile + 1] = 1 % m.q();
  for (int i = 1; i <= kTile; i++) {
    h[i] = m.mul(h[i - 1], P);
    h[kTile + 1 + i] = m.mul(h[kTile + i], P1024);
  }
  Scratch sc(s);
  uint64_t *pw, *agg;
  BT_TRY(sc.alloc(&pw, h.size()));
  BT_TRY(sc.alloc(&agg, na));
  BT_CUDA(cudaMemcpyAsync(pw, h.data(), h.size() * sizeof(uint64_t), cudaMemcpyHostToDevice, s));
  ProfScope ps("prefix_fingerprint", s, n);
  BT_LAUNCH(k_kr_local<M><<<(unsigned)na, kTile, 0, s>>>(m, T, nchunks, B, pw, Hs, agg));
  BT_LAUNCH(k_kr_aggs<M><<<1, kTile, 0, s>>>(m, agg, na, pw + kTile + 1));
  BT_LAUNCH(k_kr_add<M><<<(unsigned)na, kTile, 0, s>>>(m, Hs, nchunks, agg, pw));
  BT_CUDA(cudaGetLastError());
  // The host table must outlive the asynchronous copy.
  BT_CUDA(cudaStreamSynchronize(s));
  return BT_OK;
}

// H[p] at every position from the stride-32 values: the lane of chunk j
// extends Hs[j] by Horner over the chunk's bytes (section 2), keeping the 32
// prefixes in a shared-memory tile; the warp then writes the tile row by row
// so that each store covers 32 consecutive positions.
constexpr uint32_t kExpandWarps = 4;

template <class M>
__global__ void __launch_bounds__(32 * kExpandWarps) k_kr_expand(M m, const uint8_t* __restrict__ T,
                                                                uint64_t n, uint64_t B,
                                                                const uint64_t* __restrict__ Hs,
                                                                uint64_t* __restrict__ H) {
  __shared__ uint64_t tile[kExpandWarps][32][33];
  const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t nchunks = n / kPrefixStride + 1;  // the last one may be partial
  const uint64_t j0 = ((uint64_t)blockIdx.x * kExpandWarps + warp) * 32;
  const uint64_t j = j0 + lane;
  if (j < nchunks) {
    uint64_t h = Hs[j];
    const uint64_t p0 = j * kPrefixStride;
    if (p0 + kPrefixStride <= n && (((uintptr_t)(T + p0)) & 15) == 0) {
      // A full chunk: its 32 bytes are loaded before the multiply chain.
      const uint4 v0 = ((const uint4*)(T + p0))[0], v1 = ((const uint4*)(T + p0))[1];
      const uint32_t wv[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
      for (uint32_t i = 0; i < kPrefixStride; i++) {
        tile[warp][lane][i] = h;
        h = m.add(m.mul(h, B), (uint64_t)((wv[i >> 2] >> (8 * (i & 3))) & 0xFFu) + 1);
      }
    } else {
#pragma unroll 4
      for (uint32_t i = 0; i < kPrefixStride; i++) {
        tile[warp][lane][i] = h;
        if (p0 + i < n) h = m.add(m.mul(h, B), (uint64_t)T[p0 + i] + 1);
      }
    }
  }
  __syncwarp();
  for (uint32_t r = 0; r < 32 && j0 + r < nchunks; r++) {
    const uint64_t p = (j0 + r) * kPrefixStride + lane;
    if (p <= n) H[p] = tile[warp][r][lane];
  }
}

template <class M>
int kr_expand(const M& m, const uint8_t* T, uint64_t n, uint64_t B, const uint64_t* Hs, uint64_t* H,
              cudaStream_t s) {
  const uint64_t nchunks = n / kPrefixStride + 1;
  const uint64_t per_cta = 32ull * kExpandWarps;
  ProfScope ps("prefix_expand", s, n);
  BT_LAUNCH(k_kr_expand<M><<<(unsigned)((nchunks + per_cta - 1) / per_cta), 32 * kExpandWarps, 0, s>>>(
      m, T, n, B, Hs, H));
  BT_CUDA(cudaGetLastError());
  return BT_OK;
}

}  // namespace

int scan_u32(const uint32_t* in, uint32_t* out, uint64_t n, cudaStream_t s) {
  return scan_sum<uint32_t>(in, out, n, s);
}
int scan_u32(const uint32_t* in, uint32_t* out, uint64_t n, cudaStream_t s, uint32_t* agg) {
  if (n == 0) {
    BT_CUDA(cudaMemsetAsync(out, 0, sizeof(uint32_t), s));
    return BT_OK;
  }
  const uint64_t na = (n + kTile - 1) / kTile;
  BT_LAUNCH(k_sum_local<uint32_t><<<(unsigned)na, kTile, 0, s>>>(in, out, n, agg));
  BT_LAUNCH(k_sum_aggs<uint32_t><<<1, kTile, 0, s>>>(agg, na));
  BT_LAUNCH(k_sum_add<uint32_t><<<(unsigned)na, kTile, 0, s>>>(out, n, agg));
  BT_CUDA(cudaGetLastError());
  return BT_OK;
}
int scan_u64(const uint64_t* in, uint64_t* out, uint64_t n, cudaStream_t s) {
  return scan_sum<uint64_t>(in, out, n, s);
}

int prefix_fingerprints(const uint8_t* T, uint64_t n, uint64_t B, uint64_t q, uint64_t* Hs,
                        cudaStream_t s) {
  if (q == Mersenne61::Q) return kr_prefix(Mersenne61{}, T, n, B, Hs, s);
  return kr_prefix(SmallMod{q}, T, n, B, Hs, s);
}

int expand_prefix(const uint8_t* T, uint64_t n, uint64_t B, uint64_t q, const uint64_t* Hs, uint64_t* H,
                  cudaStream_t s) {
  if (q == Mersenne61::Q) return kr_expand(Mersenne61{}, T, n, B, Hs, H, s);
  return kr_expand(SmallMod{q}, T, n, B, Hs, H, s);
}

// ---------------------------------------------------------------------------
// Prefix fingerprints without allocation (bt_prefix_fingerprints_noalloc).
//
// Some callers cannot allocate device memory.  For example, a host runtime may
// reserve all device memory for its own allocator up front and forbid the
// libraries it loads to call cudaMalloc.  Code on a latency-critical path may
// also be unable to risk an allocation's implicit synchronisation or failure.
// This variant of the prefix-fingerprint pass takes its scratch (the two power
// tables and the per-CTA aggregates) from a fixed array in device memory
// instead of cudaMallocAsync.  Every GPU that loads the library holds the
// array until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr uint64_t kNoAllocMaxN = 1ull << 31;  // largest text accepted (2 GiB)
constexpr uint64_t kNoAllocAggs = (kNoAllocMaxN / kPrefixStride + kTile - 1) / kTile;
constexpr uint64_t kNoAllocWords = 2 * (kTile + 1) + kNoAllocAggs;  // 67586 u64, 528 KiB
constexpr int kNoAllocDevices = 64;
// The aggregate region holds exactly the CTA totals of the largest text, and
// the array is the two power tables plus that region.
static_assert(kNoAllocAggs == 65536, "one aggregate per 1024 chunks of 32 bytes of a 2 GiB text");
static_assert(kNoAllocWords == 2 * (kTile + 1) + 65536, "power tables + aggregates");

static __device__ __align__(256) uint64_t g_noalloc_scratch[kNoAllocWords];

std::mutex g_noalloc_mu;
uint64_t* g_noalloc_addr[kNoAllocDevices] = {};

// Device address of the scratch array on the current device.  In host code
// the array's name stands for a host-side shadow, not device memory, so the
// address is looked up once per device (the first call on a device does it)
// and cached.
int noalloc_scratch(uint64_t** out) {
  int dev = 0;
  BT_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocDevices) return BT_EINVAL;
  std::lock_guard<std::mutex> g(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
      note_cuda_error(e, "cudaGetSymbolAddress", __FILE__, __LINE__);
      return BT_ECUDA;
    }
    g_noalloc_addr[dev] = (uint64_t*)p;
  }
  *out = g_noalloc_addr[dev];
  return BT_OK;
}

// pw1[i] = P^i and pw2[i] = P^(1024 i) for i <= 1024, P = B^32, computed on
// the device so that no host buffer has to be copied.
template <class M>
__global__ void k_kr_powers(M m, uint64_t B, uint64_t* __restrict__ pw) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i > (uint64_t)kTile) return;
  const uint64_t P = pow_mod(m, B, kPrefixStride);
  pw[i] = pow_mod(m, P, i);
  pw[kTile + 1 + i] = pow_mod(m, pow_mod(m, P, kTile), i);
}

template <class M>
int kr_prefix_noalloc(const M& m, const uint8_t* T, uint64_t n, uint64_t B, uint64_t* Hs,
                      uint64_t* scratch, cudaStream_t s) {
  const uint64_t nchunks = n / kPrefixStride;
  if (nchunks == 0) {
    BT_CUDA(cudaMemsetAsync(Hs, 0, sizeof(uint64_t), s));
    return BT_OK;
  }
  const uint64_t na = (nchunks + kTile - 1) / kTile;
  uint64_t* pw = scratch;
  uint64_t* agg = scratch + 2 * (kTile + 1);
  BT_LAUNCH(k_kr_powers<M><<<(kTile + 1 + 255) / 256, 256, 0, s>>>(m, B, pw));
  BT_LAUNCH(k_kr_local<M><<<(unsigned)na, kTile, 0, s>>>(m, T, nchunks, B, pw, Hs, agg));
  BT_LAUNCH(k_kr_aggs<M><<<1, kTile, 0, s>>>(m, agg, na, pw + kTile + 1));
  BT_LAUNCH(k_kr_add<M><<<(unsigned)na, kTile, 0, s>>>(m, Hs, nchunks, agg, pw));
  BT_CUDA(cudaGetLastError());
  return BT_OK;
}

}  // namespace

}  // namespace bt

extern "C" int bt_prefix_fingerprints_noalloc(const uint8_t* d_text, uint64_t n, uint64_t seed,
                                              uint64_t modulus, uint32_t stride, uint64_t* d_out,
                                              void* stream) {
  using namespace bt;
  if (n > kNoAllocMaxN) return BT_ERANGE;  // before every other check
  if (!d_text || !d_out || stride != kPrefixStride) return BT_EINVAL;
  if (modulus && (modulus < 300 || modulus >= (1ull << 32))) return BT_EINVAL;
  uint64_t* scratch = nullptr;
  BT_TRY(noalloc_scratch(&scratch));
  const uint64_t q = modulus ? modulus : Mersenne61::Q;
  const uint64_t B = bt_fingerprint_base(seed, modulus);
  cudaStream_t s = stream ? (cudaStream_t)stream : cudaStreamPerThread;
  if (q == Mersenne61::Q) return kr_prefix_noalloc(Mersenne61{}, d_text, n, B, d_out, scratch, s);
  return kr_prefix_noalloc(SmallMod{q}, d_text, n, B, d_out, scratch, s);
}

namespace bt {
namespace {

// Integer-pipe microbenchmark: kMulChains independent chains of the 61-bit
// modular multiply the fingerprints use, `iters` steps each, per thread.  The
// base arrives at run time and every chain's result is stored, so nothing
// folds away.
constexpr int kMulChains = 8;

__global__ void __launch_bounds__(256) k_mulmod_bench(uint64_t B, uint32_t iters, uint64_t* __restrict__ out) {
  const Mersenne61 m;
  const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  uint64_t a[kMulChains];
#pragma unroll
  for (int u = 0; u < kMulChains; u++) a[u] = (t * kMulChains + u) % (Mersenne61::Q - 1) + 1;
  for (uint32_t i = 0; i < iters; i++) {
#pragma unroll
    for (int u = 0; u < kMulChains; u++) a[u] = m.mul(a[u], B);
  }
  uint64_t x = 0;
#pragma unroll
  for (int u = 0; u < kMulChains; u++) x ^= a[u];
  out[t] = x;
}

}  // namespace
}  // namespace bt

extern "C" int bt_mulmod_bench(uint32_t blocks, uint32_t iters, uint64_t seed, uint64_t* d_out, void* stream,
                               uint64_t* mulmods) {
  using namespace bt;
  if (!d_out || !mulmods || blocks == 0 || iters == 0) return BT_EINVAL;
  cudaStream_t s = stream ? (cudaStream_t)stream : cudaStreamPerThread;
  BT_LAUNCH(k_mulmod_bench<<<blocks, 256, 0, s>>>(bt_fingerprint_base(seed, 0), iters, d_out));
  BT_CUDA(cudaGetLastError());
  *mulmods = (uint64_t)blocks * 256 * iters * kMulChains;
  return BT_OK;
}
