// qsgs_batch.cuh -- batched growth: many realizations per launch.
//
// Included at the end of qsgs_kernels.cu (one translation unit): it reuses
// the growth chunk, the step logic and the look-back scan of the single
// realization path.  A batch step is three launches for all members
// together -- growth over the concatenated candidate list, one commit over
// the marked and touched words of all members, and one control kernel with
// a thread per member -- so uneven realizations (different sizes, targets,
// step counts) advance side by side and each member's result is the one it
// gets alone: every draw is keyed by the member's own seed, step and voxel.
#pragma once

namespace qsgs {

// Largest member index m with key(m) <= x, for a key non-decreasing in m.
template <class Key>
__device__ __forceinline__ uint32_t find_member(const MemberDesc* d, uint32_t n, uint32_t x,
                                                Key key) {
  uint32_t lo = 0, hi = n;  // answer in [lo, hi)
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (key(d[mid]) <= x) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Prologue of a batch advance: lists every solid word of each running
// member (a superset of its front), used when the batch starts or its
// membership changed.  Member m's list entries (member-local word indices,
// any order) go to the batch list from word_base(m) on, counted by its run
// state's list_next.  A warp takes 8 consecutive 32-word groups per
// iteration (all loads first); groups of one member share one atomic.
constexpr int kBatchCommitGroups = 8;

// One 32-word group of member md (the slow path, at member boundaries).
__device__ __forceinline__ void batch_list_group(const MemberDesc& md, uint32_t gs,
                                                 uint32_t* list) {
  const uint32_t lane = threadIdx.x & 31u;
  RunState* st = md.st;
  const uint32_t w = gs + lane - md.word_base;
  const bool keep = gs + lane < md.word_end && st->status == kRunning && md.grid[w] != 0;
  const uint32_t bal = __ballot_sync(0xffffffffu, keep);
  uint32_t base = 0;
  if (lane == 0 && bal) base = atomicAdd(&st->list_next, (uint32_t)__popc(bal));
  base = __shfl_sync(0xffffffffu, base, 0);
  if (keep) list[md.word_base + base + __popc(bal & ((1u << lane) - 1u))] = w;
}

__global__ void __launch_bounds__(256, 2)
    k_batch_list_solid(const MemberDesc* __restrict__ d, const BatchState* bs, uint32_t* list) {
  constexpr int G = kBatchCommitGroups;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t n = bs->n_members;
  if (n == 0) return;
  const uint32_t ngroups = bs->total_words / 32u;  // member ranges are 32-aligned
  const uint32_t nsuper = (ngroups + G - 1) / G;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t sg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; sg < nsuper; sg += nwarps) {
    const uint32_t g0 = sg * G;
    const uint32_t glast = min(g0 + G, ngroups) - 1;
    // Members of the first and the last group, searched by two lanes at once.
    uint32_t mm = 0;
    if (lane < 2)
      mm = find_member(d, n, (lane ? glast : g0) * 32u,
                       [](const MemberDesc& x) { return x.word_base; });
    const uint32_t m0 = __shfl_sync(0xffffffffu, mm, 0);
    const uint32_t m1 = __shfl_sync(0xffffffffu, mm, 1);
    if (m0 != m1) {
      // A member boundary inside: group by group.
      uint32_t m = m0;
      for (uint32_t gi = g0; gi <= glast; ++gi) {
        while (m + 1 < n && d[m + 1].word_base <= gi * 32u) ++m;  // uniform
        batch_list_group(d[m], gi * 32u, list);
      }
      continue;
    }
    // Common case: every group of this warp belongs to one member.
    const MemberDesc& md = d[m0];
    RunState* st = md.st;
    if (st->status != kRunning) continue;
    const uint32_t lw0 = g0 * 32u - md.word_base;  // member-local first word
    const uint32_t nloc = md.word_end - md.word_base;
    uint32_t v[G], bal[G];
#pragma unroll
    for (int j = 0; j < G; ++j) {
      const uint32_t w = lw0 + j * 32u + lane;
      v[j] = (g0 + j <= glast && w < nloc) ? md.grid[w] : 0u;
    }
#pragma unroll
    for (int j = 0; j < G; ++j) bal[j] = __ballot_sync(0xffffffffu, v[j] != 0);
    uint32_t total = 0;
#pragma unroll
    for (int j = 0; j < G; ++j) total += (uint32_t)__popc(bal[j]);
    uint32_t base = 0;
    if (lane == 0 && total) base = atomicAdd(&st->list_next, total);
    base = __shfl_sync(0xffffffffu, base, 0);
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
    for (int j = 0; j < G; ++j) {
      if ((bal[j] >> lane) & 1u) list[md.word_base + base + __popc(bal[j] & lt)] = lw0 + j * 32u + lane;
      base += (uint32_t)__popc(bal[j]);
    }
  }
}

// Step commit of the batch (the work of k_commit, per member): a warp
// takes one super-group of 8 consecutive 32-word groups of one member per
// iteration, over the super-groups of the members that run the step only
// (laid out by k_batch_control: member m's start at commit_base(m)).  The
// group loads are issued together and list space is reserved with one
// atomic; as in k_commit, a member whose step list is under
// 1/kSparseFraction of its words takes the sparse path (bitmaps first, then
// only marked or touched words), the others the dense one (everything at
// once).  Member m's list entries (member-local word indices, any order) go
// to the batch list from word_base(m) on, counted by its list_next.
__global__ void __launch_bounds__(256, 2)
    k_batch_commit(const MemberDesc* __restrict__ d, const BatchState* bs, uint32_t* list) {
  constexpr int G = kBatchCommitGroups;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t n = bs->n_members;
  if (n == 0) return;
  const uint32_t nsuper = bs->total_supers;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t sg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; sg < nsuper; sg += nwarps) {
    // The member whose super-groups hold sg: the last one starting at or
    // before it (members that do not run have none, so never end there).
    uint32_t mm = 0;
    if (lane == 0) mm = find_member(d, n, sg, [](const MemberDesc& x) { return x.commit_base; });
    const uint32_t m0 = __shfl_sync(0xffffffffu, mm, 0);
    const MemberDesc& md = d[m0];
    RunState* st = md.st;
    const uint32_t nloc = md.word_end - md.word_base;
    const uint32_t ngl = (nloc + 31u) / 32u;                  // the member's groups
    const uint32_t lg0 = (sg - md.commit_base) * (uint32_t)G;  // its first group here
    const uint32_t lw0 = lg0 * 32u;                           // member-local first word
    uint32_t* touched = md.mark + bitmap_words(md.g);
    const uint32_t* cur = md.aux + (size_t)(st->t & 1u) * md.g.nwords;
    const bool sparse = commit_is_sparse(st->front_words, nloc);
    const bool jv = lane < (uint32_t)G && lg0 + lane < ngl;
    const uint32_t jl = (lw0 >> 5) + lane;
    const uint32_t mk = jv ? md.mark[jl] : 0u, tc = jv ? touched[jl] : 0u;
    uint32_t c[G], old[G], bal[G];
    if (sparse) {
      if (mk) md.mark[jl] = 0u;
      if (tc) touched[jl] = 0u;
      const uint32_t mt = mk | tc;
#pragma unroll
      for (int j = 0; j < G; ++j) {
        const uint32_t w = lw0 + j * 32u + lane;
        const bool act = (__shfl_sync(0xffffffffu, mt, j) >> lane) & 1u;  // set bits lie below nloc
        c[j] = act ? cur[w] : 0u;
        old[j] = act ? md.grid[w] : 0u;
        bal[j] = __ballot_sync(0xffffffffu, act);
      }
    } else {
#pragma unroll
      for (int j = 0; j < G; ++j) {
        const uint32_t w = lw0 + j * 32u + lane;
        const bool in = w < nloc;  // groups past the member's last hold no words
        c[j] = in ? cur[w] : 0u;
        old[j] = in ? md.grid[w] : 0u;
      }
      if (mk) md.mark[jl] = 0u;
      if (tc) touched[jl] = 0u;
#pragma unroll
      for (int j = 0; j < G; ++j) {
        const uint32_t mkw = __shfl_sync(0xffffffffu, mk, j);
        bal[j] = __ballot_sync(0xffffffffu, ((mkw >> lane) & 1u) || c[j] != 0);
      }
    }
    uint32_t claims = 0;
#pragma unroll
    for (int j = 0; j < G; ++j) {
      if (c[j]) md.grid[lw0 + j * 32u + lane] = old[j] | c[j];
      claims += (uint32_t)__popc(c[j]);
    }
    const uint32_t wc = __reduce_add_sync(0xffffffffu, claims);
    if (lane == 0 && wc) atomicAdd(&st->claimed, (unsigned long long)wc);
    uint32_t total = 0;
#pragma unroll
    for (int j = 0; j < G; ++j) total += (uint32_t)__popc(bal[j]);
    uint32_t base = 0;
    if (lane == 0 && total) base = atomicAdd(&st->list_next, total);
    base = __shfl_sync(0xffffffffu, base, 0);
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
    for (int j = 0; j < G; ++j) {
      if ((bal[j] >> lane) & 1u) list[md.word_base + base + __popc(bal[j] & lt)] = lw0 + j * 32u + lane;
      base += (uint32_t)__popc(bal[j]);
    }
  }
}

// Block per member: its run state into out[m] (16 threads, 16 bytes each),
// so that the host reads every member's state with one copy.
__global__ void __launch_bounds__(16) k_batch_gather_states(const MemberDesc* d, RunState* out) {
  const uint4* src = reinterpret_cast<const uint4*>(d[blockIdx.x].st);
  reinterpret_cast<uint4*>(out + blockIdx.x)[threadIdx.x] = src[threadIdx.x];
}
static_assert(sizeof(RunState) == 16 * sizeof(uint4), "one uint4 per gather thread");

// Thread per member: per-member step budget of this advance.
__global__ void k_batch_limits(MemberDesc* d, BatchState* bs) {
  for (uint32_t m = blockIdx.x * blockDim.x + threadIdx.x; m < bs->n_members;
       m += gridDim.x * blockDim.x)
    set_step_limit(d[m].st, bs->step_extra);
}

// One block, thread per member: close each member's step (none in the
// prologue), open the next, lay out the growth chunks of the members that
// run it, and set the while-loop condition.
__global__ void __launch_bounds__(kMaxBatchMembers)
    k_batch_control(MemberDesc* d, BatchState* bs, cudaGraphConditionalHandle cond, int use_cond,
                    int prologue) {
  __shared__ unsigned long long s_warp[kMaxBatchMembers / 32];
  __shared__ uint32_t s_active;
  const uint32_t n = bs->n_members;
  const uint32_t m = threadIdx.x;
  const uint32_t lane = m & 31u, warp = m >> 5;
  if (m == 0) s_active = 0;
  __syncthreads();
  uint32_t chunks = 0, supers = 0;
  if (m < n) {
    RunState* st = d[m].st;
    const uint32_t list_n = st->list_next;  // appended by the commit just before
    if (prologue) {
      st->front_acc = 0;
      st->claimed = 0;
      st->live = 0;
    } else {
      close_step(st);
    }
    begin_step(st);  // resets list_next for the next commit
    d[m].list_base = d[m].word_base;
    d[m].list_n = list_n;
    if (st->active) {
      chunks = (list_n + 31u) / 32u;
      const uint32_t groups = (d[m].word_end - d[m].word_base + 31u) / 32u;
      supers = (groups + kBatchCommitGroups - 1u) / kBatchCommitGroups;
      s_active = 1;  // benign race: every writer stores 1
    }
  }
  // Block-wide exclusive scan of the growth chunk counts (low half) and the
  // commit super-group counts (high half) of the members that run the step.
  const unsigned long long mine = chunks | ((unsigned long long)supers << 32);
  unsigned long long incl = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= (uint32_t)o) incl += y;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    unsigned long long x = s_warp[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= (uint32_t)o) x += y;
    }
    s_warp[lane] = x;  // inclusive warp totals
  }
  __syncthreads();
  const unsigned long long excl = (warp ? s_warp[warp - 1] : 0ull) + incl - mine;
  if (m < n) {
    d[m].chunk_base = (uint32_t)excl;
    d[m].commit_base = (uint32_t)(excl >> 32);
  }
  if (m == kMaxBatchMembers - 1) {
    const unsigned long long tot = s_warp[kMaxBatchMembers / 32 - 1];
    bs->total_chunks = (uint32_t)tot;
    bs->total_supers = (uint32_t)(tot >> 32);
  }
  if (m == 0) {
    bs->scan.iters += 1;  // control launches of this batch (launch accounting)
    bs->any_active = s_active;
    if (use_cond) cudaGraphSetConditional(cond, s_active);
  }
}

// Growth over the batch candidate list: warp chunk c belongs to the member
// whose chunk range holds c, so every warp serves one member at a time.
// Three blocks per SM like k_grow (the register cap costs a few spilled
// bytes; measured faster than two blocks per SM).  DK = kOpen when no
// member is periodic or has blocked cells (the open-domain code path of
// k_grow), else kRuntime, which decides per member.
#ifndef QSGS_BATCH_GROW_MIN_BLOCKS
#define QSGS_BATCH_GROW_MIN_BLOCKS 3
#endif
template <int DK>
__global__ void __launch_bounds__(kGrowThreads, QSGS_BATCH_GROW_MIN_BLOCKS)
    k_grow_batch(const MemberDesc* __restrict__ d, BatchState* bs,
                 const uint32_t* __restrict__ list, uint32_t tile) {
  extern __shared__ uint4 grow_smem_[];
  GrowWarpSmem* smem = reinterpret_cast<GrowWarpSmem*>(grow_smem_);
  __shared__ uint4 s_thr[kGrowWarps][8];  // seven blocks and a padding row, as in k_grow
  __shared__ PhiloxKeys s_keys[kGrowWarps];  // the warp's member's round keys
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t total = bs->total_chunks, n = bs->n_members;
  const uint32_t nwarps = gridDim.x * kGrowWarps;
  const uint32_t ntiles = (total + tile - 1) / tile;
  // The member of the warp's last chunk, its chunk range, thresholds (in
  // s_thr[warp]) and round keys (in s_keys[warp]) stay while the next chunk
  // is the same member's.
  uint32_t cur = 0xFFFFFFFFu, lo = 0, hi = 0, live_dirs = 0;
  // The warp's counters of its current member, added to the member's run
  // state when the warp moves on to another member and at the end (one
  // flush per chunk cost 3 % of the 96-member batch: its atomics all go to
  // a few run states).
  GrowCounters cnt{0, 0};
  for (uint32_t ti = blockIdx.x * kGrowWarps + warp; ti < ntiles;
       ti = next_chunk(&bs->scan.grow_next, nwarps)) {
    const uint32_t c_end = min(ti * tile + tile, total);
    for (uint32_t c = ti * tile; c < c_end; ++c) {
      if (c < lo || c >= hi) {  // warp-uniform
        if (cur != 0xFFFFFFFFu) flush_counters(d[cur].st, cnt);  // the previous member's
        cur = find_member(d, n, c, [](const MemberDesc& x) { return x.chunk_base; });
        lo = d[cur].chunk_base;
        hi = cur + 1 < n ? d[cur + 1].chunk_base : total;
        live_dirs = live_directions(d[cur].st);
        __syncwarp();  // the previous member's thresholds are no longer read
        load_thresholds<true>(d[cur].st, lane, s_thr[warp]);  // complemented, for fail_bits
        if (lane < 20) reinterpret_cast<uint32_t*>(&s_keys[warp])[lane] =
            reinterpret_cast<const uint32_t*>(&d[cur].keys)[lane];
        __syncwarp();
      }
      const MemberDesc& md = d[cur];
      const uint32_t t = md.st->t;
      const uint32_t j = (c - lo) * 32u + lane;
      const uint32_t w = j < md.list_n ? list[md.list_base + j] : 0xFFFFFFFFu;
      // The member's round keys are read by the Philox rounds from shared
      // memory: held in registers (k_grow takes them from the constant bank)
      // they made this kernel spill (100 vs 97 ms for the 96-member batch).
      const PhiloxKeys& keys = s_keys[warp];
      uint32_t* claims = md.aux + (size_t)(t & 1u) * md.g.nwords;
      uint32_t* other = md.aux + (size_t)((t & 1u) ^ 1u) * md.g.nwords;
      grow_chunk<DK>(md.g, md.grid, claims, other, md.mark, w, t, live_dirs, s_thr[warp], keys,
                     smem[warp], cnt);
    }
  }
  if (cur != 0xFFFFFFFFu) flush_counters(d[cur].st, cnt);
  finish_dispenser(&bs->scan.grow_next, &bs->scan.grow_done);
}

}  // namespace qsgs
