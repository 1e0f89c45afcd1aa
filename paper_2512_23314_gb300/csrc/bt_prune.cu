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
// undecided rest in right-to-left order.
#include "bt_internal.cuh"

namespace bt {

namespace {

enum : uint32_t { UNDEC = 0, PRUNED = 1, KEPT = 2, NOTCAND = 3 };

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
                           const uint64_t* __restrict__ t2, uint32_t* __restrict__ indeg,
                           uint32_t* __restrict__ dround) {
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < v.c;
       k += (uint64_t)gridDim.x * blockDim.x) {
    dround[k] = 0xFFFFFFFFu;
    if (state[k] != UNDEC) continue;
    if (state[t1[k]] != NOTCAND) atomicAdd(&indeg[t1[k]], 1u);
    if (t2[k] != kNone && state[t2[k]] != NOTCAND) atomicAdd(&indeg[t2[k]], 1u);
  }
}

__global__ void k_round0(PView v, uint32_t* __restrict__ state, const uint32_t* __restrict__ indeg,
                         uint32_t* __restrict__ dround, unsigned long long* prog) {
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < v.c;
       k += (uint64_t)gridDim.x * blockDim.x) {
    if (state[k] == UNDEC && indeg[k] == 0) {
      state[k] = PRUNED;
      dround[k] = 0;
      atomicAdd(&prog[0], 1ull);
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
    if (i < 4) prog[i] = 0;
  }
}

// One frontier round for candidate k: if k was decided in round r-1, it
// informs its targets (a pruned attacker keeps its target; a kept attacker
// lowers the target's count of undecided attackers, and at zero the target
// is pruned).  Decisions of round r are counted in prog[r % 3].
__device__ __forceinline__ void round_step(const PView& v, uint32_t* state, uint32_t* indeg,
                                           uint32_t* dround, const uint64_t* __restrict__ t1,
                                           const uint64_t* __restrict__ t2, uint32_t r,
                                           unsigned long long* prog, uint64_t k) {
  if (dround[k] != r - 1) return;
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
    if (target && atomicCAS(&state[t], (uint32_t)UNDEC, target) == UNDEC) {
      dround[t] = r;
      atomicAdd(&prog[r % 3], 1ull);
    }
  }
}

// Round r over all candidates.  A round after one that decided nothing has
// nothing to do (the decided set is a fixed point) and returns at once.
__global__ void k_round(PView v, uint32_t* state, uint32_t* indeg, uint32_t* dround,
                        const uint64_t* __restrict__ t1, const uint64_t* __restrict__ t2, uint32_t r,
                        unsigned long long* prog) {
  if (*(volatile unsigned long long*)&prog[(r - 1) % 3] == 0) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) prog[(r + 1) % 3] = 0;
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < v.c;
       k += (uint64_t)gridDim.x * blockDim.x)
    round_step(v, state, indeg, dround, t1, t2, r, prog, k);
}

// Rounds r0, r0+1, ... in one CTA until a round decides nothing or the
// bound is reached (deep dependency chains after the multi-CTA rounds).
__global__ void k_rounds_tail(PView v, uint32_t* state, uint32_t* indeg, uint32_t* dround,
                              const uint64_t* __restrict__ t1, const uint64_t* __restrict__ t2,
                              uint32_t r0, uint32_t rmax, unsigned long long* prog) {
  for (uint32_t r = r0; r < rmax; r++) {
    __syncthreads();
    if (*(volatile unsigned long long*)&prog[(r - 1) % 3] == 0) return;
    if (threadIdx.x == 0) prog[(r + 1) % 3] = 0;
    for (uint64_t k = threadIdx.x; k < v.c; k += blockDim.x)
      round_step(v, state, indeg, dround, t1, t2, r, prog, k);
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

__global__ void k_pack_marks(uint64_t c, const uint8_t* __restrict__ mk, uint32_t* __restrict__ mw,
                             uint32_t* __restrict__ wpop) {
  const uint64_t words = (c + 31) / 32;
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
  for (int l = (int)t->L - 2; l >= 0; l--) {
    Level& v = t->lv[l];
    Level& w = t->lv[l + 1];
    // Multi-CTA rounds before the one-CTA tail; a level of at most 16 Ki
    // blocks goes to the one-CTA rounds at once (launches cost more there).
    const uint32_t multi_rounds = v.c <= (16u << 10) ? 0 : 24;
    const int w_last = l + 1 == (int)t->L - 1;
    const uint64_t words = (v.c + 31) / 32;
    Arena& A = ctx.arena;
    uint8_t *hit_v = nullptr, *tgt_w = nullptr, *gone = nullptr, *hit2 = nullptr;
    uint32_t *state = nullptr, *indeg = nullptr, *dround = nullptr, *wpop = nullptr, *sagg = nullptr;
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
      dround = A.take<uint32_t>(v.c);
      prog = A.take<unsigned long long>(4);
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
    BT_LAUNCH(k_indegree<<<grid_for(v.c, T), T, 0, s>>>(pv, state, t1, t2, indeg, dround));
    BT_LAUNCH(k_round0<<<grid_for(v.c, T), T, 0, s>>>(pv, state, indeg, dround, prog));
    // Frontier rounds without host round trips: multi-CTA rounds that return
    // at once after the fixed point, then one CTA for deep chains, then (only
    // if the bound was hit) the single-thread right-to-left finish.
    const uint32_t rmax = (uint32_t)(max_rounds < 0xFFFFFFF0u ? max_rounds : 0xFFFFFFF0u);
    uint32_t r = 1;
    for (; r <= multi_rounds && r < rmax; r++)
      BT_LAUNCH(k_round<<<grid_for(v.c, T), T, 0, s>>>(pv, state, indeg, dround, t1, t2, r, prog));
    BT_LAUNCH(k_rounds_tail<<<1, 1024, 0, s>>>(pv, state, indeg, dround, t1, t2, r, rmax, prog));
    BT_LAUNCH(k_count_undecided<<<grid_for(v.c, T), T, 0, s>>>(pv, state, prog + 3));
    BT_LAUNCH(k_finish_serial<<<1, 1, 0, s>>>(pv, state, t1, t2, hit2, prog + 3));
    BT_CUDA(cudaGetLastError());
    t->lv[l].stats[BT_ST_FINAL_BLOCKS] = v.c;
    BT_LAUNCH(k_apply<<<grid_for(v.c, T), T, 0, s>>>(pv, v.arity, w.b, state, t1, v.ptr, v.off, gone));
    BT_LAUNCH(k_clear_marks<<<grid_for(words * 32, T), T, 0, s>>>(pv, state, wpop));
    BT_TRY(scan_u32(wpop, v.mr, words, s, sagg));

    // Compact the next level.
    BT_LAUNCH(k_keep<<<grid_for(w.c, T), T, 0, s>>>(w.c, gone, keep));
    BT_TRY(scan_u64(keep, nidx, w.c, s));
    uint64_t c2 = 0;
    BT_CUDA(cudaMemcpyAsync(&c2, nidx + w.c, sizeof(c2), cudaMemcpyDeviceToHost, s));
    BT_CUDA(cudaStreamSynchronize(s));
    if (c2 != w.c) {
      uint64_t *st2, *off2, *lo2;
      uint32_t *ptr2, *mw2, *mr2, *wpop2;
      uint8_t* mk2;
      const uint64_t words2 = (c2 + 31) / 32;
      auto al = [](uint64_t x) { return (x + 255) & ~255ull; };
      const uint64_t o_st = 0, o_off = al(c2 * 8 + 8), o_lo = o_off + al(c2 * 8 + 8),
                     o_ptr = o_lo + al(c2 * 8 + 8), o_mw = o_ptr + al(c2 * 4 + 4),
                     o_mr = o_mw + al(words2 * 4 + 4), total = o_mr + al((words2 + 1) * 4);
      char* mem;
      BT_CUDA(cudaMallocAsync((void**)&mem, total, s));
      st2 = (uint64_t*)(mem + o_st);
      off2 = (uint64_t*)(mem + o_off);
      lo2 = (uint64_t*)(mem + o_lo);
      ptr2 = (uint32_t*)(mem + o_ptr);
      mw2 = (uint32_t*)(mem + o_mw);
      mr2 = (uint32_t*)(mem + o_mr);
      BT_CUDA(cudaMallocAsync((void**)&mk2, c2 + 8 + 4 * (words2 + 1), s));
      wpop2 = (uint32_t*)(((uintptr_t)(mk2 + c2 + 1) + 3) & ~(uintptr_t)3);
      BT_LAUNCH(k_compact<<<grid_for(w.c, T), T, 0, s>>>(pw, gone, nidx, st2, mk2, ptr2, off2, lo2, ctx.st));
      BT_LAUNCH(k_pack_marks<<<grid_for(words2 * 32, T), T, 0, s>>>(c2, mk2, mw2, wpop2));
      BT_TRY(scan_u32(wpop2, mr2, words2, s, sagg2));
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
      w.c = c2;
    }
    w.stats[BT_ST_FINAL_BLOCKS] = w.c;
    BT_TRY(sync_status(ctx));
    if (ctx.st_host->error) return BT_EINTERNAL;
  }
  t->lv[0].stats[BT_ST_FINAL_BLOCKS] = t->lv[0].c;
  return BT_OK;
}

}  // namespace bt
