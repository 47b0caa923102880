// qsgs_batch.cuh -- batched growth: many realizations per launch.
//
// Included at the end of qsgs_kernels.cu (one translation unit): it reuses
// the growth chunk, the step logic and the look-back scan of the single
// realization path.  A batch step is three launches for all members
// together -- growth over the concatenated candidate list, one ordered
// commit scan over the batch word space, and one control kernel with a
// thread per member -- so uneven realizations (different sizes, targets,
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

// Commit over the batch word space (see CommitPolicy).  Prologue mode lists
// every solid word of each running member (a superset of its front, used
// when the batch starts or its membership changed); step mode ORs the
// claims of the members that ran a step into their grids, counts them per
// member, and lists marked or claimed words.  Also records where each
// member's entries start in the batch list.
struct BatchCommitPolicy {
  MemberDesc* d;
  BatchState* bs;
  uint32_t* list;
  int prologue;
  struct Item {
    uint32_t w;      // member-local word (0xFFFFFFFF: outside every member)
    uint32_t bits;   // 1: listed
    uint32_t extra;  // member index
    uint32_t c;      // claims of this step in the word
    uint32_t old;    // the word before the claims
    uint32_t flags;  // 1: lane 0 clears the warp's mark word; 2: clear the other claim word
  };
  __device__ bool active() const { return true; }
  __device__ bool emit_empty() const { return true; }
  __device__ uint32_t n_items() const { return bs->total_words; }
  __device__ uint32_t side(const Item&, int) const { return 0; }
  __device__ unsigned long long* side_sum(int) const { return nullptr; }
  __device__ Item load(uint32_t i, bool valid) const {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t n = bs->n_members;
    const uint32_t m = find_member(d, n, valid ? i : 0u,
                                   [](const MemberDesc& x) { return x.word_base; });
    const MemberDesc& md = d[m];
    const uint32_t w = i - md.word_base;
    const bool in_range = valid && i < md.word_end;
    const RunState* st = md.st;
    uint32_t keep = 0, c = 0, old = 0, flags = 0;
    if (prologue) {
      if (in_range && st->status == kRunning) keep = md.grid[w] ? 1u : 0u;
    } else if (st->active) {
      uint32_t mk = 0;
      if (lane == 0 && in_range) mk = md.mark[w >> 5];
      mk = __shfl_sync(0xffffffffu, mk, 0);
      if (in_range) {
        const uint32_t par = st->t & 1u;
        c = md.aux[(size_t)par * md.g.nwords + w];
        const uint32_t other = md.aux[(size_t)(par ^ 1u) * md.g.nwords + w];
        old = md.grid[w];
        keep = ((mk >> lane) & 1u) | (c ? 1u : 0u);
        flags = (lane == 0 && mk ? 1u : 0u) | (other ? 2u : 0u);
      }
    }
    return Item{in_range ? w : 0xFFFFFFFFu, keep, m, c, old, flags};
  }
  // Claims into the member's grid and their count; marks and the previous
  // claim grid cleared.  All lanes of a warp serve one member.
  __device__ void apply(const Item& it, bool) const {
    if (prologue) return;
    const MemberDesc& md = d[it.extra];
    RunState* st = md.st;
    if (!st->active) return;  // uniform over the warp
    if (it.w != 0xFFFFFFFFu) {
      if (it.flags & 1u) md.mark[it.w >> 5] = 0;
      if (it.flags & 2u) md.aux[(size_t)((st->t & 1u) ^ 1u) * md.g.nwords + it.w] = 0;
      if (it.c) md.grid[it.w] = it.old | it.c;
    }
    const uint32_t wc = __reduce_add_sync(0xffffffffu, (uint32_t)__popc(it.c));
    if ((threadIdx.x & 31u) == 0 && wc) atomicAdd(&st->claimed, (unsigned long long)wc);
  }
  __device__ uint32_t count(const Item& it) const { return it.bits; }
  __device__ void emit(const Item& it, unsigned long long off) const {
    if (it.w == 0) d[it.extra].list_base = (uint32_t)off;
    if (it.bits) list[off] = it.w;
  }
  __device__ void total(unsigned long long n) const { bs->list_total = (uint32_t)n; }
};

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
  __shared__ uint32_t s_warp[kMaxBatchMembers / 32];
  __shared__ uint32_t s_active;
  const uint32_t n = bs->n_members;
  const uint32_t m = threadIdx.x;
  const uint32_t lane = m & 31u, warp = m >> 5;
  if (m == 0) s_active = 0;
  __syncthreads();
  uint32_t chunks = 0;
  if (m < n) {
    RunState* st = d[m].st;
    if (prologue) {
      st->front_acc = 0;
      st->claimed = 0;
      st->live = 0;
    } else {
      close_step(st);
    }
    begin_step(st);
    const uint32_t next = m + 1 < n ? d[m + 1].list_base : bs->list_total;
    const uint32_t list_n = next - d[m].list_base;
    d[m].list_n = list_n;
    if (st->active) {
      chunks = (list_n + 31u) / 32u;
      s_active = 1;  // benign race: every writer stores 1
    }
  }
  // Block-wide exclusive scan of the chunk counts.
  uint32_t incl = chunks;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= (uint32_t)o) incl += y;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t x = s_warp[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= (uint32_t)o) x += y;
    }
    s_warp[lane] = x;  // inclusive warp totals
  }
  __syncthreads();
  const uint32_t excl = (warp ? s_warp[warp - 1] : 0u) + incl - chunks;
  if (m < n) d[m].chunk_base = excl;
  if (m == kMaxBatchMembers - 1) bs->total_chunks = s_warp[kMaxBatchMembers / 32 - 1];
  if (m == 0) {
    bs->scan.iters += 1;  // control launches of this batch (launch accounting)
    bs->any_active = s_active;
    if (use_cond) cudaGraphSetConditional(cond, s_active);
  }
}

// Growth over the batch candidate list: warp chunk c belongs to the member
// whose chunk range holds c, so every warp serves one member at a time.
__global__ void __launch_bounds__(kGrowThreads, 2)
    k_grow_batch(const MemberDesc* __restrict__ d, BatchState* bs,
                 const uint32_t* __restrict__ list) {
  extern __shared__ uint4 grow_smem_[];
  GrowWarpSmem* smem = reinterpret_cast<GrowWarpSmem*>(grow_smem_);
  __shared__ uint4 s_thr[kGrowWarps][7];
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t total = bs->total_chunks, n = bs->n_members;
  const uint32_t nwarps = gridDim.x * kGrowWarps;
  for (uint32_t c = blockIdx.x * kGrowWarps + warp; c < total;
       c = next_chunk(&bs->scan.grow_next, nwarps)) {
    const uint32_t m = find_member(d, n, c, [](const MemberDesc& x) { return x.chunk_base; });
    const MemberDesc& md = d[m];
    RunState* st = md.st;
    const uint32_t t = st->t;
    const uint32_t live_dirs = live_directions(st);
    load_thresholds(st, lane, s_thr[warp]);
    __syncwarp();
    const uint32_t j = (c - md.chunk_base) * 32u + lane;
    const uint32_t w = j < md.list_n ? list[md.list_base + j] : 0xFFFFFFFFu;
    const PhiloxKeys keys = md.keys;
    uint32_t* claims = md.aux + (size_t)(t & 1u) * md.g.nwords;
    GrowCounters cnt{0, 0};
    grow_chunk(md.g, md.grid, claims, md.mark, w, t, live_dirs, s_thr[warp], keys, smem[warp],
               cnt);
    flush_counters(st, cnt);
    __syncwarp();  // s_thr[warp] is rewritten by the next chunk
  }
  finish_dispenser(&bs->scan.grow_next, &bs->scan.grow_done);
}

}  // namespace qsgs
