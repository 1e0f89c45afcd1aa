// bt_prune.cu -- the optional pruning pass (section 3.1, "Optional Pruning").
//
// The paper gives the intent: marked blocks that no pointer targets are
// removed.  The reading implemented here (identical to the CPU oracle's):
// levels are processed from the second-to-last up; on level l a marked block
// k becomes a pointer to LO(S(k)) and loses its children when
//   (i)   none of its children has children (or the next level is the last),
//   (ii)  no pointer of level l -- original, or created by pruning a block to
//         the right of k -- has a target window overlapping k,
//   (iii) no pointer of level l+1 (as it stands when level l starts) targets
//         one of k's children, and
//   (iv)  LO(S(k)) + |k| <= start(k).
// The sequential rule scans each level right to left.  Conditions (i), (iii),
// (iv) and the original pointers of (ii) are static, so they are evaluated in
// parallel; they leave a candidate set C.  A candidate j, once pruned, targets
// at most two blocks, both strictly to its left, so
//      pruned(k) = k in C  and  no pruned j > k in C targets k,
// a recurrence over a DAG whose edges point left.  It is resolved by
// frontier rounds (a candidate is decided once all candidates targeting it are
// decided: pruned if none of them was pruned), which gives exactly the
// sequential result; after `max_rounds` rounds a single thread finishes the
// undecided rest in right-to-left order.  Each round visits only the
// candidates the previous round decided (a worklist of block indices); wide
// frontiers go to multi-CTA launches, narrow ones to a single CTA that runs
// the remaining rounds without returning to the host.
#include <vector>

#include "bt_internal.cuh"

namespace bt {

namespace {

enum : uint32_t { UNDEC = 0, PRUNED = 1, KEPT = 2, NOTCAND = 3 };

// Per-level counters: prog[0..2] decisions of round r in prog[r % 3] (also the
// length of that round's worklist), prog[3] candidates left undecided, then
// the hand-over to the one-CTA tail (flag, first round it runs).
constexpr int kProg = 6, kTailFlag = 4, kTailRound = 5;
// Worklists narrower than this run in the one-CTA tail.
constexpr unsigned long long kTailFrontier = 4096;

struct PView {
  uint64_t n, c, b;
  const uint64_t* st;
  uint32_t* mw;
  const uint32_t* mr;
  const uint32_t* ptr;
  const uint64_t* off;
  const uint64_t* lo;
};

__device__ __forceinline__ uint64_t plen(const PView& v, uint64_t k) {
  uint64_t s = v.st[k];
  return v.n - s < v.b ? v.n - s : v.b;
}
__device__ __forceinline__ bool pmarked(const PView& v, uint64_t k) {
  return (v.mw[k >> 5] >> (k & 31)) & 1u;
}
__device__ __forceinline__ uint64_t prank(const PView& v, uint64_t k) {
  return v.mr[k >> 5] + __popc(v.mw[k >> 5] & ((1u << (k & 31)) - 1u));
}
__device__ uint64_t block_of(const PView& v, uint64_t p) {
  uint64_t a = 0, z = v.c;
  while (a < z) {
    uint64_t mid = (a + z) / 2;
    if (v.st[mid] <= p) a = mid + 1;
    else z = mid;
  }
  return a - 1;  // callers pass positions inside the level
}

// Flag every block that the target window of an unmarked block overlaps.
__global__ void k_flag_targets(PView v, uint8_t* __restrict__ flag) {
  for (uint64_t u = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; u < v.c;
       u += (uint64_t)gridDim.x * blockDim.x) {
    if (pmarked(v, u)) continue;
    uint64_t j = v.ptr[u];
    flag[j] = 1;
    if (v.off[u] + plen(v, u) > plen(v, j)) flag[j + 1] = 1;
  }
}

// Candidates: marked, conditions (i), (iii), (iv), and not overlapped by an
// original pointer of the level.  Their target blocks t1 (and t2 when the
// occurrence crosses into the next block).
__global__ void k_candidates(PView v, PView w, int w_last, uint32_t arity,
                             const uint8_t* __restrict__ hit_v, const uint8_t* __restrict__ tgt_w,
                             uint32_t* __restrict__ state, uint64_t* __restrict__ t1,
                             uint64_t* __restrict__ t2, Status* status) {
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < v.c;
       k += (uint64_t)gridDim.x * blockDim.x) {
    state[k] = NOTCAND;
    if (!pmarked(v, k) || hit_v[k]) continue;
    uint64_t s = v.st[k], len = plen(v, k);
    uint64_t lo = v.lo[k];
    if (lo == kNone) {
      atomicExch(&status->error, 11ull);
      continue;
    }
    if (lo + len > s) continue;  // (iv)
    uint64_t first = prank(v, k) * arity, nch = (len + w.b - 1) / w.b;
    bool ok = true;
    for (uint64_t i = 0; i < nch && ok; i++) {
      uint64_t ch = first + i;
      if (!w_last && pmarked(w, ch)) ok = false;  // (i)
      if (tgt_w[ch]) ok = false;                 // (iii)
    }
    if (!ok) continue;
    uint64_t j = block_of(v, lo);
    t1[k] = j;
    t2[k] = (lo + len > v.st[j] + plen(v, j)) ? j + 1 : kNone;
    state[k] = UNDEC;
  }
}

__global__ void k_indegree(PView v, const uint32_t* __restrict__ state, const uint64_t* __restrict__ t1,
                           const uint64_t* __restrict__ t2, uint32_t* __restrict__ indeg) {
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < v.c;
       k += (uint64_t)gridDim.x * blockDim.x) {
    if (state[k] != UNDEC) continue;
    if (state[t1[k]] != NOTCAND) atomicAdd(&indeg[t1[k]], 1u);
    if (t2[k] != kNone && state[t2[k]] != NOTCAND) atomicAdd(&indeg[t2[k]], 1u);
  }
}

// Frontier round 0: candidates nothing targets are pruned; they form the first
// worklist (fq[0, prog[0])).
__global__ void k_round0(PView v, uint32_t* __restrict__ state, const uint32_t* __restrict__ indeg,
                         uint32_t* __restrict__ fq, unsigned long long* prog) {
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < v.c;
       k += (uint64_t)gridDim.x * blockDim.x) {
    if (state[k] == UNDEC && indeg[k] == 0) {
      state[k] = PRUNED;
      fq[atomicAdd(&prog[0], 1ull)] = (uint32_t)k;
    }
  }
}

// Per-level scratch to its initial values in one launch.
__global__ void k_prune_init(uint8_t* hit_v, uint8_t* hit2, uint64_t nv, uint8_t* tgt_w, uint8_t* gone,
                             uint64_t nw, uint32_t* indeg, unsigned long long* prog) {
  const uint64_t top = (nv > nw ? nv : nw) + 1;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < top;
       i += (uint64_t)gridDim.x * blockDim.x) {
    if (i <= nv) {
      hit_v[i] = 0;
      hit2[i] = 0;
    }
    if (i < nv) indeg[i] = 0;
    if (i <= nw) {
      tgt_w[i] = 0;
      gone[i] = 0;
    }
    if (i < kProg) prog[i] = 0;
  }
}

// One frontier round for candidate k, decided in round r-1: it informs its
// targets (a pruned attacker keeps its target; a kept attacker lowers the
// target's count of undecided attackers, and at zero the target is pruned).
// Decisions of round r are counted in prog[r % 3] and appended to qout.
__device__ __forceinline__ void round_step(const PView& v, uint32_t* state, uint32_t* indeg,
                                           const uint64_t* __restrict__ t1, const uint64_t* __restrict__ t2,
                                           uint32_t r, unsigned long long* prog, uint32_t* qout, uint64_t k) {
  const uint32_t sk = state[k];
  for (int e = 0; e < 2; e++) {
    const uint64_t t = e == 0 ? t1[k] : t2[k];
    if (t == kNone || state[t] == NOTCAND) continue;
    uint32_t target = 0;
    if (sk == PRUNED) {
      target = KEPT;
    } else if (atomicSub(&indeg[t], 1u) == 1u) {
      target = PRUNED;
    }
    if (target && atomicCAS(&state[t], (uint32_t)UNDEC, target) == UNDEC)
      qout[atomicAdd(&prog[r % 3], 1ull)] = (uint32_t)t;
  }
}

// Round r over the worklist of round r-1 (fq + ((r-1) & 1) c, prog[(r-1) % 3]
// entries).  When that worklist is narrower than kTailFrontier the rounds
// from r on go to the one-CTA tail: round r records r in prog[kTailRound],
// sets prog[kTailFlag], and it and every later multi-CTA round return at once
// (every CTA of a launch reads the same count, so all take the same branch).
__global__ void k_round(PView v, uint32_t* state, uint32_t* indeg, const uint64_t* __restrict__ t1,
                        const uint64_t* __restrict__ t2, uint32_t* fq, uint32_t r, unsigned long long* prog) {
  if (*(volatile unsigned long long*)&prog[kTailFlag]) return;
  const unsigned long long m = *(volatile unsigned long long*)&prog[(r - 1) % 3];
  if (m < kTailFrontier) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      prog[kTailRound] = r;
      prog[kTailFlag] = 1;
    }
    return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) prog[(r + 1) % 3] = 0;
  const uint32_t* qin = fq + ((r - 1) & 1) * v.c;
  uint32_t* qout = fq + (r & 1) * v.c;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x)
    round_step(v, state, indeg, t1, t2, r, prog, qout, qin[i]);
}

// Rounds r0 (or the round the multi-CTA launches handed over at), r0+1, ...
// in one CTA until a round decides nothing or the bound is reached (narrow
// frontiers along deep dependency chains).
__global__ void k_rounds_tail(PView v, uint32_t* state, uint32_t* indeg, const uint64_t* __restrict__ t1,
                              const uint64_t* __restrict__ t2, uint32_t* fq, uint32_t r0, uint32_t rmax,
                              unsigned long long* prog) {
  uint32_t r = prog[kTailFlag] ? (uint32_t)prog[kTailRound] : r0;
  for (; r < rmax; r++) {
    __syncthreads();
    const unsigned long long m = *(volatile unsigned long long*)&prog[(r - 1) % 3];
    if (m == 0) return;
    if (threadIdx.x == 0) prog[(r + 1) % 3] = 0;
    const uint32_t* qin = fq + ((r - 1) & 1) * v.c;
    uint32_t* qout = fq + (r & 1) * v.c;
    for (uint64_t i = threadIdx.x; i < m; i += blockDim.x) round_step(v, state, indeg, t1, t2, r, prog, qout, qin[i]);
    __threadfence_block();
  }
}

// Right-to-left finish for candidates still undecided after the bound.
__global__ void k_finish_serial(PView v, uint32_t* state, const uint64_t* __restrict__ t1,
                                const uint64_t* __restrict__ t2, uint8_t* hit,
                                const unsigned long long* und) {
  if (*und == 0) return;
  for (uint64_t k = v.c; k-- > 0;) {
    uint32_t s = state[k];
    if (s == UNDEC) {
      s = hit[k] ? KEPT : PRUNED;
      state[k] = s;
    }
    if (s == PRUNED) {
      hit[t1[k]] = 1;
      if (t2[k] != kNone) hit[t2[k]] = 1;
    }
  }
}

__global__ void k_count_undecided(PView v, const uint32_t* __restrict__ state, unsigned long long* cnt) {
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < v.c;
       k += (uint64_t)gridDim.x * blockDim.x)
    if (state[k] == UNDEC) atomicAdd(cnt, 1ull);
}

// Apply: pruned blocks lose their children (marked gone on the next level,
// found through the mark rank before it changes) and become pointers.
__global__ void k_apply(PView v, uint32_t arity, uint64_t wb, const uint32_t* __restrict__ state,
                        const uint64_t* __restrict__ t1, uint32_t* __restrict__ ptr,
                        uint64_t* __restrict__ off, uint8_t* __restrict__ gone) {
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < v.c;
       k += (uint64_t)gridDim.x * blockDim.x) {
    if (state[k] != PRUNED) continue;
    uint64_t first = prank(v, k) * arity, nch = (plen(v, k) + wb - 1) / wb;
    for (uint64_t i = 0; i < nch; i++) gone[first + i] = 1;
    ptr[k] = (uint32_t)t1[k];
    off[k] = v.lo[k] - v.st[t1[k]];
  }
}

__global__ void k_clear_marks(PView v, const uint32_t* __restrict__ state, uint32_t* __restrict__ wpop) {
  const uint64_t words = (v.c + 31) / 32;
  for (uint64_t base = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) & ~31ull; base < words * 32;
       base += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t k = base + (threadIdx.x & 31);
    bool mk = k < v.c && pmarked(v, k) && state[k] != PRUNED;
    uint32_t bits = __ballot_sync(0xFFFFFFFFu, mk);
    if ((threadIdx.x & 31) == 0) {
      v.mw[base / 32] = bits;
      wpop[base / 32] = __popc(bits);
    }
  }
}

__global__ void k_keep(uint64_t c, const uint8_t* __restrict__ gone, uint64_t* __restrict__ keep) {
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < c;
       k += (uint64_t)gridDim.x * blockDim.x)
    keep[k] = gone[k] ? 0 : 1;
}

// Compact the next level without the deleted children; pointers are
// renumbered (their targets are never deleted: condition (iii)).
__global__ void k_compact(PView w, const uint8_t* __restrict__ gone, const uint64_t* __restrict__ nidx,
                          uint64_t* __restrict__ st2, uint8_t* __restrict__ mk2,
                          uint32_t* __restrict__ ptr2, uint64_t* __restrict__ off2,
                          uint64_t* __restrict__ lo2, Status* status) {
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < w.c;
       k += (uint64_t)gridDim.x * blockDim.x) {
    if (gone[k]) continue;
    uint64_t i = nidx[k];
    st2[i] = w.st[k];
    bool m = pmarked(w, k);
    mk2[i] = m;
    off2[i] = w.off[k];
    lo2[i] = w.lo[k];
    if (m) {
      ptr2[i] = 0;
    } else {
      uint32_t j = w.ptr[k];
      if (gone[j]) atomicExch(&status->error, 12ull);
      ptr2[i] = (uint32_t)nidx[j];
    }
  }
}

// Marks of the compacted level: c = *cnt blocks (known on the device only),
// packed into the words of an upper bound of cub blocks (the words past the
// last block hold zeros, so the rank prefix ends at the same total).
__global__ void k_pack_marks(const uint64_t* __restrict__ cnt, uint64_t cub, const uint8_t* __restrict__ mk,
                             uint32_t* __restrict__ mw, uint32_t* __restrict__ wpop) {
  const uint64_t c = *cnt, words = (cub + 31) / 32;
  for (uint64_t base = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) & ~31ull; base < words * 32;
       base += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t k = base + (threadIdx.x & 31);
    uint32_t bits = __ballot_sync(0xFFFFFFFFu, k < c && mk[k]);
    if ((threadIdx.x & 31) == 0) {
      mw[base / 32] = bits;
      wpop[base / 32] = __popc(bits);
    }
  }
}

PView view_of(const bt_tree* t, const Level& v) {
  return PView{t->n, v.c, v.b, v.st, v.mw, v.mr, v.ptr, v.off, v.lo};
}

}  // namespace

int prune_tree(BuildCtx& ctx, uint64_t max_rounds) {
  bt_tree* t = ctx.t;
  cudaStream_t s = ctx.s;
  const unsigned T = 256;
  if (max_rounds == 0) max_rounds = 4096;
  // New block counts of the compacted levels stay on the device until the
  // loop ends (no host round trip per level); cnt[l] for level l >= 1.
  uint64_t* cnt = nullptr;
  BT_CUDA(cudaMallocAsync((void**)&cnt, t->L * sizeof(uint64_t), s));
  struct Release {
    uint64_t* p;
    cudaStream_t s;
    ~Release() { cudaFreeAsync(p, s); }
  } release{cnt, s};
  BT_CUDA(cudaMemsetAsync(cnt, 0, t->L * sizeof(uint64_t), s));
  for (int l = (int)t->L - 2; l >= 0; l--) {
    Level& v = t->lv[l];
    Level& w = t->lv[l + 1];
    // Multi-CTA rounds before the one-CTA tail; a level of at most 16 Ki
    // blocks goes to the one-CTA rounds at once (launches cost more there).
    const uint32_t multi_rounds = v.c <= (16u << 10) ? 0 : 8;
    const int w_last = l + 1 == (int)t->L - 1;
    const uint64_t words = (v.c + 31) / 32;
    Arena& A = ctx.arena;
    uint8_t *hit_v = nullptr, *tgt_w = nullptr, *gone = nullptr, *hit2 = nullptr;
    uint32_t *state = nullptr, *indeg = nullptr, *fq = nullptr, *wpop = nullptr, *sagg = nullptr;
    uint64_t *t1 = nullptr, *t2 = nullptr, *keep = nullptr, *nidx = nullptr;
    uint32_t* sagg2 = nullptr;
    unsigned long long* prog = nullptr;
    auto carve = [&]() {
      hit_v = A.take<uint8_t>(v.c + 1);
      hit2 = A.take<uint8_t>(v.c + 1);
      tgt_w = A.take<uint8_t>(w.c + 1);
      gone = A.take<uint8_t>(w.c + 1);
      state = A.take<uint32_t>(v.c + 1);
      t1 = A.take<uint64_t>(v.c);
      t2 = A.take<uint64_t>(v.c);
      indeg = A.take<uint32_t>(v.c);
      fq = A.take<uint32_t>(2 * v.c);
      prog = A.take<unsigned long long>(kProg);
      wpop = A.take<uint32_t>(words);
      sagg = A.take<uint32_t>(scan_scratch_words(words));
      keep = A.take<uint64_t>(w.c);
      nidx = A.take<uint64_t>(w.c + 1);
      sagg2 = A.take<uint32_t>(scan_scratch_words((w.c + 31) / 32));
    };
    A.begin_dry();
    carve();
    BT_TRY(A.reserve());
    carve();
    PView pv = view_of(t, v), pw = view_of(t, w);
    const uint64_t top = (v.c > w.c ? v.c : w.c) + 1;
    BT_LAUNCH(k_prune_init<<<grid_for(top, T), T, 0, s>>>(hit_v, hit2, v.c, tgt_w, gone, w.c, indeg, prog));
    BT_LAUNCH(k_flag_targets<<<grid_for(v.c, T), T, 0, s>>>(pv, hit_v));
    BT_LAUNCH(k_flag_targets<<<grid_for(w.c, T), T, 0, s>>>(pw, tgt_w));
    BT_LAUNCH(k_candidates<<<grid_for(v.c, T), T, 0, s>>>(pv, pw, w_last, v.arity, hit_v, tgt_w, state, t1, t2,
                                                  ctx.st));
    BT_LAUNCH(k_indegree<<<grid_for(v.c, T), T, 0, s>>>(pv, state, t1, t2, indeg));
    BT_LAUNCH(k_round0<<<grid_for(v.c, T), T, 0, s>>>(pv, state, indeg, fq, prog));
    // Frontier rounds without host round trips: multi-CTA rounds while the
    // worklist is wide (each returns at once after the hand-over), then one
    // CTA for the narrow rest, then (only if the bound was hit) the
    // single-thread right-to-left finish.
    const uint32_t rmax = (uint32_t)(max_rounds < 0xFFFFFFF0u ? max_rounds : 0xFFFFFFF0u);
    uint32_t r = 1;
    for (; r <= multi_rounds && r < rmax; r++)
      BT_LAUNCH(k_round<<<grid_for(v.c, T, 152u * 8u), T, 0, s>>>(pv, state, indeg, t1, t2, fq, r, prog));
    BT_LAUNCH(k_rounds_tail<<<1, 1024, 0, s>>>(pv, state, indeg, t1, t2, fq, r, rmax, prog));
    BT_LAUNCH(k_count_undecided<<<grid_for(v.c, T), T, 0, s>>>(pv, state, prog + 3));
    BT_LAUNCH(k_finish_serial<<<1, 1, 0, s>>>(pv, state, t1, t2, hit2, prog + 3));
    BT_CUDA(cudaGetLastError());
    BT_LAUNCH(k_apply<<<grid_for(v.c, T), T, 0, s>>>(pv, v.arity, w.b, state, t1, v.ptr, v.off, gone));
    BT_LAUNCH(k_clear_marks<<<grid_for(words * 32, T), T, 0, s>>>(pv, state, wpop));
    BT_TRY(scan_u32(wpop, v.mr, words, s, sagg));

    // Compact the next level.  Its new block count c2 stays on the device
    // (nidx[w.c]); the arrays are sized for the old count w.c, an upper bound.
    BT_LAUNCH(k_keep<<<grid_for(w.c, T), T, 0, s>>>(w.c, gone, keep));
    BT_TRY(scan_u64(keep, nidx, w.c, s));
    {
      uint64_t *st2, *off2, *lo2;
      uint32_t *ptr2, *mw2, *mr2, *wpop2;
      uint8_t* mk2;
      const uint64_t cub = w.c, words2 = (cub + 31) / 32;
      auto al = [](uint64_t x) { return (x + 255) & ~255ull; };
      const uint64_t o_st = 0, o_off = al(cub * 8 + 8), o_lo = o_off + al(cub * 8 + 8),
                     o_ptr = o_lo + al(cub * 8 + 8), o_mw = o_ptr + al(cub * 4 + 4),
                     o_mr = o_mw + al(words2 * 4 + 4), total = o_mr + al((words2 + 1) * 4);
      char* mem;
      BT_CUDA(cudaMallocAsync((void**)&mem, total, s));
      st2 = (uint64_t*)(mem + o_st);
      off2 = (uint64_t*)(mem + o_off);
      lo2 = (uint64_t*)(mem + o_lo);
      ptr2 = (uint32_t*)(mem + o_ptr);
      mw2 = (uint32_t*)(mem + o_mw);
      mr2 = (uint32_t*)(mem + o_mr);
      BT_CUDA(cudaMallocAsync((void**)&mk2, cub + 8 + 4 * (words2 + 1), s));
      wpop2 = (uint32_t*)(((uintptr_t)(mk2 + cub + 1) + 3) & ~(uintptr_t)3);
      BT_LAUNCH(k_compact<<<grid_for(w.c, T), T, 0, s>>>(pw, gone, nidx, st2, mk2, ptr2, off2, lo2, ctx.st));
      BT_LAUNCH(k_pack_marks<<<grid_for(words2 * 32, T), T, 0, s>>>(nidx + w.c, cub, mk2, mw2, wpop2));
      BT_TRY(scan_u32(wpop2, mr2, words2, s, sagg2));
      BT_CUDA(cudaMemcpyAsync(cnt + l + 1, nidx + w.c, sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
      BT_CUDA(cudaGetLastError());
      cudaFreeAsync(mk2, s);
      for (void* a : w.owned) cudaFreeAsync(a, s);
      w.owned.assign(1, mem);
      w.st = st2;
      w.off = off2;
      w.lo = lo2;
      w.ptr = ptr2;
      w.mw = mw2;
      w.mr = mr2;
      // w.c keeps the upper bound until the loop ends: no later level of
      // this loop reads level l+1 again.
    }
  }
  // One host round trip for the whole pass: the new counts and the status.
  std::vector<uint64_t> c2(t->L, 0);
  BT_CUDA(cudaMemcpyAsync(c2.data(), cnt, t->L * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
  BT_TRY(sync_status(ctx));
  if (ctx.st_host->error) return BT_EINTERNAL;
  for (uint32_t l = 1; l < t->L; l++) {
    if (c2[l] == 0 || c2[l] > t->lv[l].c) return BT_EINTERNAL;
    t->lv[l].c = c2[l];
    t->lv[l].stats[BT_ST_FINAL_BLOCKS] = c2[l];
  }
  t->lv[0].stats[BT_ST_FINAL_BLOCKS] = t->lv[0].c;
  return BT_OK;
}

}  // namespace bt
