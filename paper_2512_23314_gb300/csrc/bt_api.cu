// bt_api.cu -- the C ABI (include/bt.h) and the host side of a build.
//
// bt_build_ex: validate -> text on the device (H2D copy for host input) ->
// alphabet histogram -> Karp-Rabin prefix fingerprints -> the level loop of
// bt_level.cu (one device->host read of the next level's size per level) ->
// pruning (bt_prune.cu) -> counters and leaf text (bt_query.cu).  Every step
// runs in this library's kernels; the host only sizes buffers and launches.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <chrono>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "bt_internal.cuh"

namespace bt {

int alphabet(const uint8_t* T, uint64_t n, uint32_t sigma, bt_tree* t, cudaStream_t s);
int upload_view(bt_tree* t, cudaStream_t s);
int batch_kernel_build(const uint8_t* const* texts, const uint64_t* ns, const uint32_t* sigmas,
                       const uint32_t* taus, const uint32_t* leaf_lens, uint64_t ndocs, const bt_opts& o,
                       std::vector<char>& routed, bt_tree** outs, uint32_t threads, uint32_t ctas_per_sm,
                       uint32_t chunk, cudaStream_t s, const std::vector<char>* eligible);
uint32_t batch_split(const uint64_t* ns, const uint32_t* taus, const uint32_t* leaf_lens, uint64_t ndocs,
                     const bt_opts& o, uint32_t ctas_per_sm, std::vector<char>& eligible);
int batch_shape(const uint8_t* const* texts, const uint64_t* ns, const uint32_t* sigmas, const uint32_t* taus,
                const uint32_t* leaf_lens, uint64_t ndocs, const bt_opts& o, cudaStream_t s, uint32_t* threads,
                uint32_t* ctas_per_sm, uint32_t* chunk, uint64_t* tuned_now);
void batch_report_tuned(uint64_t trials);
void batch_report_workers(uint64_t docs);
void batch_report_reset();
int run_queries(const bt_tree* t, int kind, const uint64_t* d_args, uint64_t m, uint64_t* d_out,
                cudaStream_t s);

void note_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
  if (getenv("BT_VERBOSE"))
    fprintf(stderr, "bt: %s failed at %s:%d: %s\n", what, file, line, cudaGetErrorString(e));
}

static std::atomic<unsigned long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

static std::atomic<uint64_t> g_alloc_limit{0};
bool alloc_allowed(uint64_t bytes) {
  const uint64_t lim = g_alloc_limit.load(std::memory_order_relaxed);
  return lim == 0 || bytes <= lim;
}

namespace {
struct ProfRec {
  std::string name;
  cudaEvent_t a, b;
  uint64_t bytes;
};
std::mutex g_prof_mu;
std::vector<ProfRec> g_prof;
std::atomic<int> g_prof_on{0};
}  // namespace

ProfScope::ProfScope(const char* name, cudaStream_t st, uint64_t bytes) : s(st) {
  if (!g_prof_on.load()) return;
  ProfRec r{name, nullptr, nullptr, bytes};
  if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) return;
  cudaEventRecord(r.a, s);
  std::lock_guard<std::mutex> g(g_prof_mu);
  slot = (int)g_prof.size();
  g_prof.push_back(r);
}

ProfScope::~ProfScope() {
  if (slot < 0) return;
  std::lock_guard<std::mutex> g(g_prof_mu);
  cudaEventRecord(g_prof[slot].b, s);
}

int sync_status(BuildCtx& ctx) {
  BT_CUDA(cudaMemcpyAsync(ctx.st_host, ctx.st, sizeof(Status), cudaMemcpyDeviceToHost, ctx.s));
  BT_CUDA(cudaStreamSynchronize(ctx.s));
  return BT_OK;
}

// splitmix64 (Steele, Lea, Flood 2014): the seed -> base map.
static uint64_t splitmix(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

uint64_t base_for(uint64_t seed, uint64_t q) { return splitmix(seed) % (q - 256) + 256; }

// Streaming multiprocessors of the current device (cached per device).
unsigned device_sm_count() {
  static std::atomic<unsigned> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return 152;
  }
  unsigned v = cache[dev].load(std::memory_order_relaxed);
  if (v) return v;
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
    cudaGetLastError();
    n = 152;
  }
  cache[dev].store((unsigned)n, std::memory_order_relaxed);
  return (unsigned)n;
}

// Block sizes: b_L = leaf_len, b_l = tau * b_{l+1}, height the smallest h
// with s0 * leaf_len * tau^h >= n (section 3 assumes n = s * tau^h).
int plan_sizes(uint64_t n, uint32_t tau, uint32_t leaf, const bt_opts& o, std::vector<uint64_t>& b) {
  b.clear();
  if (o.level_sizes) {
    if (o.nlevels == 0 || o.nlevels > kMaxLevels) return BT_EINVAL;
    for (uint32_t l = 0; l < o.nlevels; l++) {
      uint64_t x = o.level_sizes[l];
      if (x == 0) return BT_EINVAL;
      if (l + 1 < o.nlevels) {
        uint64_t y = o.level_sizes[l + 1];
        if (y == 0 || x < 2 * y || x % y) return BT_EINVAL;
      }
      b.push_back(x);
    }
    return BT_OK;
  }
  unsigned __int128 size = (unsigned __int128)(o.root_arity ? o.root_arity : tau) * leaf;
  uint32_t h = 0;
  while (size < n) {
    size *= tau;
    if (++h >= (uint32_t)kMaxLevels) return BT_EINVAL;
  }
  b.resize(h + 1);
  b[h] = leaf;
  for (int l = (int)h - 1; l >= 0; l--) b[l] = b[l + 1] * tau;
  return BT_OK;
}

// Tree arrays come from the stream-ordered pool (cudaMallocAsync); they are
// returned the same way and the stream is synchronised once.
static void free_tree_memory(bt_tree* t) {
  cudaStream_t s = cudaStreamPerThread;
  for (Level& v : t->lv) {
    for (void* a : v.owned)
      if (a) cudaFreeAsync(a, s);
    v.owned.clear();
  }
  if (t->slab) {  // a batched tree: its arrays belong to the batch's pool
    t->slab.reset();
    return;
  }
  void* rest[] = {t->leaf, t->pre, t->sym, t->view};
  for (void* a : rest)
    if (a) cudaFreeAsync(a, s);
  cudaStreamSynchronize(s);
}

// Builds allocate and free their scratch through the device's stream-ordered
// pool.  By default the pool hands unused memory back to the driver at every
// synchronisation, so each level would map its scratch again; keep it cached
// for the life of the process instead (this changes only this process's pool).
static void keep_pool_memory(int device) {
  static std::mutex mu;
  static bool done[64] = {};
  if (device < 0 || device >= 64) return;
  std::lock_guard<std::mutex> g(mu);
  if (done[device]) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  cudaGetLastError();
  done[device] = true;
}

struct HostTrace {
  bool on = getenv("BT_TRACE") != nullptr;
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
  void mark(const char* what) {
    if (!on) return;
    auto t1 = std::chrono::steady_clock::now();
    fprintf(stderr, "bt-trace %s host %.3f ms\n", what,
            std::chrono::duration<double, std::milli>(t1 - t0).count());
    t0 = t1;
  }
};

static int build(const uint8_t* text, uint64_t n, uint32_t sigma, uint32_t tau, uint32_t leaf,
                 const bt_opts& o, cudaStream_t s, bt_tree* t) {
  HostTrace tr;
  std::vector<uint64_t> sizes;
  BT_TRY(plan_sizes(n, tau, leaf, o, sizes));
  t->n = n;
  t->tau = tau;
  t->leaf_len = leaf;
  t->L = (uint32_t)sizes.size();
  t->prune = o.prune ? 1 : 0;
  t->seed = o.seed;
  t->q = o.modulus ? o.modulus : Mersenne61::Q;
  t->B = base_for(o.seed, t->q);
  t->lv.resize(t->L);
  for (uint32_t l = 0; l < t->L; l++) t->lv[l].b = sizes[l];

  BT_CUDA(cudaGetDevice(&t->device));
  keep_pool_memory(t->device);
  Scratch sc(s);
  // Text on the device.
  cudaPointerAttributes pa;
  const uint8_t* dT = text;
  if (cudaPointerGetAttributes(&pa, text) != cudaSuccess || pa.type == cudaMemoryTypeHost ||
      pa.type == cudaMemoryTypeUnregistered) {
    cudaGetLastError();
    uint8_t* copy;
    BT_TRY(sc.alloc(&copy, n + 16));
    BT_CUDA(cudaMemcpyAsync(copy, text, n, cudaMemcpyHostToDevice, s));
    dT = copy;
  }
  BuildCtx ctx;
  ctx.t = t;
  ctx.T = dT;
  ctx.s = s;
  ctx.arena.s = s;
  ctx.dense_scan = (o.flags & BT_FLAG_DENSE_SCAN) ? 1 : 0;
  ctx.tiny_queue = (o.flags & BT_FLAG_TINY_QUEUE) ? 1 : 0;
  ctx.force_list = (o.flags & BT_FLAG_GRAM_LIST) ? 1 : 0;
  ctx.two_phase = (o.flags & BT_FLAG_TWO_PHASE) ? 1 : 0;
  ctx.leaf_counts = (o.flags & BT_FLAG_LEAF_COUNTS) ? 1 : 0;
  ctx.sort_scan = (o.flags & BT_FLAG_SORT_SCAN) ? 1 : 0;
  ctx.partitions = o.partitions;
  BT_TRY(sc.alloc(&ctx.st, 1));
  BT_CUDA(cudaMemsetAsync(ctx.st, 0, sizeof(Status), s));
  BT_CUDA(cudaMallocHost(&ctx.st_host, sizeof(Status)));
  struct HostFree {
    void* p;
    ~HostFree() { cudaFreeHost(p); }
  } hf{ctx.st_host};

  {
    ProfScope ps("phase_alphabet", s, n);
    BT_TRY(alphabet(dT, n, sigma, t, s));
  }
  tr.mark("setup+alphabet");
  {
    // Prefix fingerprints at every position, for the whole construction; the
    // stride-32 values are an intermediate step.
    Scratch hs(s);
    uint64_t* Hs;
    BT_TRY(hs.alloc(&Hs, n / kPrefixStride + 2));
    BT_TRY(sc.alloc(&ctx.H, n + 1));
    BT_TRY(prefix_fingerprints(dT, n, t->B, t->q, Hs, s));
    BT_TRY(expand_prefix(dT, n, t->B, t->q, Hs, ctx.H, s));
  }
  {
    ProfScope ps("phase_levels", s, 0);
    BT_TRY(build_levels(ctx));
  }
  tr.mark("levels");
  {
    ProfScope ps("phase_prune", s, 0);
    if (t->prune) BT_TRY(prune_tree(ctx, o.max_rounds));
    else
      for (Level& v : t->lv) v.stats[BT_ST_FINAL_BLOCKS] = v.c;
  }
  tr.mark("prune");
  {
    ProfScope ps("phase_counters", s, 0);
    BT_TRY(build_counters(ctx));
  }
  tr.mark("counters");
  for (Level& v : t->lv) v.lo = nullptr;  // lives in the level's allocation; no longer needed
  ctx.arena.release();
  BT_TRY(upload_view(t, s));
  uint64_t bytes = t->leaf_bytes + 16 + sizeof(TreeView) + 512 + (t->lv[0].c + 1) * t->S * 8;
  for (const Level& v : t->lv) {
    const uint64_t words = (v.c + 31) / 32;
    bytes += v.c * (8 + 4 + 8) + (2 * words + 1) * 4 + (v.cnt ? 2 * v.c * t->S * v.cw : 0);
  }
  t->dev_bytes = bytes;
  BT_CUDA(cudaStreamSynchronize(s));
  BT_TRY(sync_status(ctx));
  tr.mark("finish");
  if (ctx.st_host->error) return BT_EINTERNAL;
  return BT_OK;
}

static cudaStream_t as_stream(void* s) { return s ? (cudaStream_t)s : cudaStreamPerThread; }




// Documents not routed to the batched kernel: host workers, each issuing
// bt_build_ex on its own CUDA stream.
static int worker_builds(const uint8_t* const* texts, const uint64_t* ns, const uint32_t* sigmas,
                         const uint32_t* taus, const uint32_t* leaf_lens, uint64_t ndocs, const bt_opts* opts,
                         uint32_t nworkers, const std::vector<char>& routed, bt_tree** outs) {
  std::vector<uint64_t> todo;
  for (uint64_t d = 0; d < ndocs; d++)
    if (!routed[d]) todo.push_back(d);
  if (todo.empty()) return BT_OK;
  if (nworkers == 0) nworkers = 8;
  if (nworkers > todo.size()) nworkers = (uint32_t)todo.size();
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) {
    cudaGetLastError();
    return BT_ECUDA;
  }
  std::atomic<uint64_t> next{0};
  std::atomic<int> first_error{BT_OK};
  auto worker = [&]() {
    cudaSetDevice(device);
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      int expect = BT_OK;
      first_error.compare_exchange_strong(expect, BT_ECUDA);
      return;
    }
    for (;;) {
      const uint64_t j = next.fetch_add(1);
      if (j >= todo.size() || first_error.load() != BT_OK) break;
      const uint64_t d = todo[j];
      const int rc = bt_build_ex(texts[d], ns[d], sigmas[d], taus[d], leaf_lens[d], opts, s, &outs[d]);
      if (rc != BT_OK) {
        int expect = BT_OK;
        first_error.compare_exchange_strong(expect, rc);
      }
    }
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  };
  std::vector<std::thread> pool;
  for (uint32_t i = 0; i < nworkers; i++) {
    try {  // no exception may cross the C ABI: a thread that cannot start ends the batch
      pool.emplace_back(worker);
    } catch (...) {
      int expect = BT_OK;
      first_error.compare_exchange_strong(expect, BT_ENOMEM);
      break;
    }
  }
  for (auto& th : pool) th.join();
  return first_error.load();
}
namespace {

// One level of the canonical serialization, written on the device: the
// block count and length, the mark words (two 32-bit words per u64), the
// number of pointers, then (ptr, off) of every unmarked block in block order
// (unmarked block k goes to index k - rank of the marked blocks before it).
struct ExportLevel {
  const uint32_t* mw;
  const uint32_t* mr;
  const uint32_t* ptr;
  const uint64_t* off;
  uint64_t c, b, nptr;
  uint64_t at;  // u64 index of the level's first field in the serialization
};

__global__ void k_export_level(ExportLevel e, uint64_t* __restrict__ out) {
  const uint64_t words = (e.c + 31) / 32, mwords = (e.c + 63) / 64;
  uint64_t* marks = out + e.at + 2;
  uint64_t* pairs = marks + mwords + 1;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t t0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (t0 == 0) {
    out[e.at] = e.c;
    out[e.at + 1] = e.b;
    marks[mwords] = e.nptr;
  }
  for (uint64_t w = t0; w < mwords; w += stride) {
    const uint64_t lo = e.mw[2 * w], hi = 2 * w + 1 < words ? e.mw[2 * w + 1] : 0;
    marks[w] = lo | (hi << 32);
  }
  for (uint64_t k = t0; k < e.c; k += stride) {
    const uint32_t word = e.mw[k >> 5];
    if ((word >> (k & 31)) & 1u) continue;
    const uint64_t i = k - (e.mr[k >> 5] + __popc(word & ((1u << (k & 31)) - 1u)));
    pairs[2 * i] = e.ptr[k];
    pairs[2 * i + 1] = e.off[k];
  }
}

}  // namespace

}  // namespace bt

using namespace bt;

extern "C" {

void bt_opts_default(bt_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->prune = 1;
}

int bt_build_ex(const uint8_t* text, uint64_t n, uint32_t sigma, uint32_t tau, uint32_t leaf_len,
                const bt_opts* opts, void* stream, bt_tree** out) {
  if (!out) return BT_EINVAL;
  *out = nullptr;
  if (!text || n == 0 || n >= (1ull << 32) || tau < 2 || tau > 64 || leaf_len == 0 || sigma == 0)
    return BT_EINVAL;
  bt_opts o;
  if (opts) o = *opts;
  else bt_opts_default(&o);
  if (o.modulus && (o.modulus < 300 || o.modulus >= (1ull << 32))) return BT_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return BT_ECUDA;
  }
  bt_tree* t = new (std::nothrow) bt_tree();
  if (!t) return BT_ENOMEM;
  int rc = build(text, n, sigma, tau, leaf_len, o, as_stream(stream), t);
  if (rc != BT_OK) {
    cudaStreamSynchronize(as_stream(stream));
    free_tree_memory(t);
    delete t;
    return rc;
  }
  *out = t;
  return BT_OK;
}

int bt_build(const uint8_t* text, uint64_t n, uint32_t sigma, uint32_t tau, uint32_t leaf_len,
             bt_tree** out) {
  return bt_build_ex(text, n, sigma, tau, leaf_len, nullptr, nullptr, out);
}

int bt_build_batch(const uint8_t* const* texts, const uint64_t* ns, const uint32_t* sigmas,
                   const uint32_t* taus, const uint32_t* leaf_lens, uint64_t ndocs,
                   const bt_opts* opts, uint32_t nworkers, bt_tree** outs) {
  if (!outs || (ndocs && (!texts || !ns || !sigmas || !taus || !leaf_lens))) return BT_EINVAL;
  for (uint64_t d = 0; d < ndocs; d++) outs[d] = nullptr;
  if (ndocs == 0) return BT_OK;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return BT_ECUDA;
  }
  bt_opts o;
  if (opts) o = *opts;
  else bt_opts_default(&o);
  // The persistent batched kernel takes every document it can, except the
  // few whose work would outlast the rest of the batch on one CTA: those are
  // built at the same time by the single-text path on host workers (as is
  // every document the kernel cannot take, and every document with
  // BT_FLAG_BATCH_WORKERS).
  std::vector<char> routed(ndocs, 0);
  int rc = BT_OK, rc_split = BT_OK;
  uint64_t split_docs = 0;
  batch_report_reset();
  if (!(o.flags & BT_FLAG_BATCH_WORKERS)) {
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      return BT_ECUDA;
    }
    int device = 0;
    if (cudaGetDevice(&device) == cudaSuccess) keep_pool_memory(device);
    cudaGetLastError();
    uint32_t threads = 0, ctas = 0, chunk = 0;
    uint64_t trials = 0;
    rc = batch_shape(texts, ns, sigmas, taus, leaf_lens, ndocs, o, s, &threads, &ctas, &chunk, &trials);
    std::vector<char> eligible;
    bt_opts ok = o;
    const uint32_t cap = rc == BT_OK ? batch_split(ns, taus, leaf_lens, ndocs, o, ctas, eligible) : 0;
    std::thread split_thread;
    if (cap) {
      ok.batch_ctas = cap;
      std::vector<char> not_heavy(ndocs, 1);
      for (uint64_t d = 0; d < ndocs; d++) {
        not_heavy[d] = eligible[d];
        split_docs += !eligible[d];
      }
      try {
        split_thread = std::thread([&, not_heavy]() {
          cudaSetDevice(device);
          rc_split = worker_builds(texts, ns, sigmas, taus, leaf_lens, ndocs, opts, nworkers, not_heavy, outs);
        });
      } catch (...) {
        rc_split = BT_ENOMEM;
      }
    }
    if (rc == BT_OK && rc_split == BT_OK) {
      batch_report_reset();
      rc = batch_kernel_build(texts, ns, sigmas, taus, leaf_lens, ndocs, ok, routed, outs, threads, ctas, chunk,
                              s, cap ? &eligible : nullptr);
      batch_report_tuned(trials);
    }
    if (split_thread.joinable()) split_thread.join();
    if (rc == BT_OK) rc = rc_split;
    for (uint64_t d = 0; d < ndocs; d++)
      if (cap && !eligible[d]) routed[d] = 1;  // built by the split workers
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  if (rc == BT_OK) {
    uint64_t nw = split_docs;
    for (uint64_t d = 0; d < ndocs; d++) nw += !routed[d];
    batch_report_workers(nw);
    rc = worker_builds(texts, ns, sigmas, taus, leaf_lens, ndocs, opts, nworkers, routed, outs);
  }
  if (rc != BT_OK) {
    for (uint64_t d = 0; d < ndocs; d++) {
      bt_free(outs[d]);
      outs[d] = nullptr;
    }
  }
  return rc;
}

void bt_free(bt_tree* t) {
  if (!t) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(t->device);
  free_tree_memory(t);
  cudaSetDevice(cur);
  delete t;
}

static int single_query(const bt_tree* t, int kind, uint64_t a0, uint64_t a1, uint64_t* res) {
  if (!t) return BT_EINVAL;
  cudaStream_t s = cudaStreamPerThread;
  uint64_t* d;
  BT_CUDA(cudaMallocAsync(&d, 3 * sizeof(uint64_t), s));
  uint64_t h[2] = {a0, a1};
  int rc = BT_OK;
  if (cudaMemcpyAsync(d, h, sizeof(h), cudaMemcpyHostToDevice, s) != cudaSuccess) rc = BT_ECUDA;
  if (rc == BT_OK) rc = run_queries(t, kind, d, 1, d + 2, s);
  if (rc == BT_OK && cudaMemcpyAsync(res, d + 2, sizeof(uint64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    rc = BT_ECUDA;
  cudaFreeAsync(d, s);
  if (cudaStreamSynchronize(s) != cudaSuccess && rc == BT_OK) rc = BT_ECUDA;
  return rc;
}

int bt_access(const bt_tree* t, uint64_t i, uint8_t* out) {
  if (!t || !out) return BT_EINVAL;
  if (i >= t->n) return BT_ERANGE;
  uint64_t r;
  BT_TRY(single_query(t, BT_Q_ACCESS, i, 0, &r));
  if (r == kNone) return BT_EINTERNAL;
  *out = (uint8_t)r;
  return BT_OK;
}

int bt_rank(const bt_tree* t, uint8_t c, uint64_t i, uint64_t* out) {
  if (!t || !out) return BT_EINVAL;
  if (i > t->n) return BT_ERANGE;
  uint64_t r;
  BT_TRY(single_query(t, BT_Q_RANK, c, i, &r));
  if (r == kNone) return BT_EINTERNAL;
  *out = r;
  return BT_OK;
}

int bt_select(const bt_tree* t, uint8_t c, uint64_t j, uint64_t* out) {
  if (!t || !out) return BT_EINVAL;
  if (j == 0) return BT_ERANGE;
  uint64_t r;
  BT_TRY(single_query(t, BT_Q_SELECT, c, j, &r));
  if (r == kNone) return BT_ERANGE;
  *out = r;
  return BT_OK;
}

int bt_query_batch(const bt_tree* t, int kind, const uint64_t* d_args, uint64_t m, uint64_t* d_out,
                   void* stream) {
  if (!t || (m && (!d_args || !d_out))) return BT_EINVAL;
  if (kind != BT_Q_ACCESS && kind != BT_Q_RANK && kind != BT_Q_SELECT) return BT_EINVAL;
  return run_queries(t, kind, d_args, m, d_out, as_stream(stream));
}

uint32_t bt_levels(const bt_tree* t) { return t ? t->L : 0; }

uint64_t bt_device_bytes(const bt_tree* t) { return t ? t->dev_bytes : 0; }

int bt_stats(const bt_tree* t, uint64_t* out, uint64_t cap) {
  if (!t || !out || cap < (uint64_t)t->L * BT_ST_FIELDS) return BT_EINVAL;
  for (uint32_t l = 0; l < t->L; l++)
    memcpy(out + l * BT_ST_FIELDS, t->lv[l].stats, sizeof(uint64_t) * BT_ST_FIELDS);
  return BT_OK;
}

int bt_export(const bt_tree* t, uint8_t* buf, uint64_t cap, uint64_t* len) {
  if (!t || !len) return BT_EINVAL;
  // The layout needs each level's number of marked blocks (the last entry of
  // its rank prefix); the serialization itself is written on the device and
  // copied out once.
  cudaStream_t s = cudaStreamPerThread;
  const uint32_t L = t->L;
  std::vector<uint32_t> nm(L, 0);
  for (uint32_t l = 0; l < L; l++) {
    const Level& v = t->lv[l];
    BT_CUDA(cudaMemcpyAsync(&nm[l], v.mr + (v.c + 31) / 32, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  }
  BT_CUDA(cudaStreamSynchronize(s));
  std::vector<ExportLevel> ex(L);
  uint64_t at = 6;  // header: "BLKTREE1", n, tau, leaf_len, L, prune
  for (uint32_t l = 0; l < L; l++) {
    const Level& v = t->lv[l];
    ex[l] = ExportLevel{v.mw, v.mr, v.ptr, v.off, v.c, v.b, v.c - nm[l], at};
    at += 2 + (v.c + 63) / 64 + 1 + 2 * (v.c - nm[l]);
  }
  const uint64_t leaf_at = at + 1, leaf_pad = (t->leaf_bytes + 7) / 8 * 8;
  const uint64_t need = leaf_at * 8 + leaf_pad;
  *len = need;
  if (!buf) return BT_OK;
  if (cap < need) return BT_ERANGE;
  Scratch sc(s);
  uint64_t* d;
  BT_TRY(sc.alloc(&d, need / 8));
  const uint64_t head[6] = {0x31454552544B4C42ull, t->n, t->tau, t->leaf_len, L, (uint64_t)t->prune};
  BT_CUDA(cudaMemcpyAsync(d, head, sizeof(head), cudaMemcpyHostToDevice, s));
  for (uint32_t l = 0; l < L; l++)
    BT_LAUNCH(k_export_level<<<grid_for(t->lv[l].c, 256), 256, 0, s>>>(ex[l], d));
  const uint64_t lb = t->leaf_bytes;
  BT_CUDA(cudaMemcpyAsync(d + at, &lb, sizeof(lb), cudaMemcpyHostToDevice, s));
  if (leaf_pad) {
    BT_CUDA(cudaMemsetAsync((uint8_t*)(d + leaf_at) + leaf_pad - 8, 0, 8, s));
    if (lb) BT_CUDA(cudaMemcpyAsync(d + leaf_at, t->leaf, lb, cudaMemcpyDeviceToDevice, s));
  }
  BT_CUDA(cudaMemcpyAsync(buf, d, need, cudaMemcpyDeviceToHost, s));
  BT_CUDA(cudaStreamSynchronize(s));
  return BT_OK;
}

int bt_prefix_fingerprints(const uint8_t* d_text, uint64_t n, uint64_t seed, uint64_t modulus,
                           uint32_t stride, uint64_t* d_out, void* stream) {
  if (!d_text || !d_out || stride != kPrefixStride) return BT_EINVAL;
  if (modulus && (modulus < 300 || modulus >= (1ull << 32))) return BT_EINVAL;
  uint64_t q = modulus ? modulus : Mersenne61::Q;
  return prefix_fingerprints(d_text, n, base_for(seed, q), q, d_out, as_stream(stream));
}

uint64_t bt_fingerprint_base(uint64_t seed, uint64_t modulus) {
  return base_for(seed, modulus ? modulus : Mersenne61::Q);
}

void bt_profile_enable(int on) { g_prof_on.store(on ? 1 : 0); }

void bt_profile_reset(void) {
  std::lock_guard<std::mutex> g(g_prof_mu);
  for (ProfRec& r : g_prof) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  g_prof.clear();
}

int bt_profile_read(bt_profile_entry* out, uint32_t cap, uint32_t* count) {
  if (!count) return BT_EINVAL;
  std::lock_guard<std::mutex> g(g_prof_mu);
  std::vector<bt_profile_entry> agg;
  for (ProfRec& r : g_prof) {
    if (cudaEventSynchronize(r.b) != cudaSuccess) return BT_ECUDA;
    float ms = 0;
    if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) return BT_ECUDA;
    bt_profile_entry* e = nullptr;
    for (auto& x : agg)
      if (r.name == x.name) e = &x;
    if (!e) {
      agg.push_back(bt_profile_entry{});
      e = &agg.back();
      snprintf(e->name, sizeof(e->name), "%s", r.name.c_str());
    }
    e->launches++;
    e->ms += ms;
    e->bytes += r.bytes;
  }
  *count = (uint32_t)agg.size();
  if (out)
    for (uint32_t i = 0; i < agg.size() && i < cap; i++) out[i] = agg[i];
  return BT_OK;
}

uint64_t bt_launch_count(void) { return g_launches.load(); }

void bt_test_alloc_limit(uint64_t bytes) { g_alloc_limit.store(bytes); }

int bt_device_pool_used(uint64_t* out) {
  if (!out) return BT_EINVAL;
  int dev = 0;
  BT_CUDA(cudaGetDevice(&dev));
  cudaMemPool_t pool;
  BT_CUDA(cudaDeviceGetDefaultMemPool(&pool, dev));
  uint64_t used = 0;
  BT_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used));
  *out = used;
  return BT_OK;
}

int bt_device_pool_peak(uint64_t* out, int reset) {
  if (!out) return BT_EINVAL;
  int dev = 0;
  BT_CUDA(cudaGetDevice(&dev));
  cudaMemPool_t pool;
  BT_CUDA(cudaDeviceGetDefaultMemPool(&pool, dev));
  uint64_t high = 0;
  BT_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &high));
  *out = high;
  if (reset) {
    uint64_t zero = 0;  // resets the high-water mark to the bytes in use now
    BT_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &zero));
  }
  return BT_OK;
}

const char* bt_strerror(int status) {
  switch (status) {
    case BT_OK: return "ok";
    case BT_EINVAL: return "invalid argument";
    case BT_ERANGE: return "out of range";
    case BT_ENOMEM: return "out of memory";
    case BT_ECUDA: return "CUDA error";
    case BT_ETIMEOUT: return "device-side loop bound exceeded";
    case BT_EINTERNAL: return "internal invariant violated";
    default: return "unknown status";
  }
}

}  // extern "C"
