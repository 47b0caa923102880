// qsgs_kernels.cu -- CUDA kernels of the LIETS QSGS generator (sm_103a).
//
// One realization lives in a caller-owned workspace: a run state, the
// bit-packed occupancy grid, an auxiliary bit grid (seed candidates, then the
// voxels claimed in the current step), the sorted active-front list and the
// scratch of the seed-spacing pass.  Every step of the hot loop is a fixed
// sequence of launches that read their sizes from the run state, so a step
// can be replayed from a CUDA graph without the host.
#include <cuda_runtime.h>

#include "qsgs_device.cuh"
#include "qsgs_launch.h"
#include "qsgs_scan.cuh"

namespace qsgs {

// ---------------------------------------------------------------------------
// Eq. 1 in integers: T(c) = min(2^32, floor(T_ref (20 Nt - 19 c) / Nt)).
// With num = 20 Nt - 19 c = a Nt + b (0 <= b < Nt), the quotient is
// T_ref a + floor(T_ref b / Nt), and T_ref b < 2^64 because T_ref <= 2^32
// and b < Nt < 2^32.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long eq1_threshold(unsigned long long t_ref,
                                                            unsigned long long nt,
                                                            unsigned long long c) {
  const unsigned long long two32 = 1ull << 32;
  if (nt == 0) return t_ref < two32 ? t_ref : two32;
  if (19ull * c >= 20ull * nt) return 0;
  const unsigned long long num = 20ull * nt - 19ull * c;
  const unsigned long long a = num / nt, b = num % nt;
  const unsigned long long q = t_ref * a + (t_ref * b) / nt;
  return q > two32 ? two32 : q;
}

// ---------------------------------------------------------------------------
// Run-state kernels (one thread).
// ---------------------------------------------------------------------------
__global__ void k_init_state(RunState* st, StateInit init) {
  st->solid = 0;
  st->nt = init.nt;
  for (int k = 0; k < 3; ++k) {
    st->t_ref[k] = init.t_ref[k];
    st->thr[k] = 0;
  }
  st->t_seed = init.t_seed;
  st->claimed = 0;
  st->live = 0;
  st->sum_front = 0;
  st->sum_draws = 0;
  st->front_n = 0;
  st->front_acc = 0;
  st->adj_n = 0;
  st->trim_keep = 0;
  st->front_words = 0;
  st->cand_n = 0;
  st->acc_n = 0;
  st->t = 0;
  st->max_steps = init.max_steps;
  st->step_limit = 0xFFFFFFFFu;
  st->status = kRunning;
  st->active = 0;
  st->trim_pending = 0;
  st->trim_parity = 0;
  st->error = 0;
  st->iters = 0;
  st->grow_next = 0;
  st->grow_done = 0;
  st->list_next = 0;
}

// Decides whether the next step runs.  Exits, tested in order: target
// reached, step limit, pause point of the current call.  Sets the Eq. 1
// thresholds of the step from the solid count before it.
__device__ void begin_step(RunState* st) {
  st->active = 0;
  st->list_next = 0;
  if (st->status != kRunning) return;
  if (st->solid >= st->nt) { st->status = kStatusDone; return; }
  if (st->t >= st->max_steps) { st->status = kStatusMaxSteps; return; }
  if (st->t >= st->step_limit) return;
  for (int k = 0; k < 3; ++k) st->thr[k] = eq1_threshold(st->t_ref[k], st->nt, st->solid);
  st->active = 1;
}

// Closes the step that just ran (if one did).  A step without a single
// attempt of positive probability is a fixed point: stalled, not counted.
// Otherwise the claims counted by the commit scan are added; if they
// overshoot Nt the solid count is capped and the exact-target trim is left
// pending (the run ends with this step).
__device__ void close_step(RunState* st) {
  if (st->active) {
    st->front_words = st->list_next;  // the list k_commit appended
    if (st->live == 0) {
      st->status = kStatusStalled;
    } else {
      st->sum_front += st->front_acc;  // |A_t|, counted by the growth kernel
      st->front_n = st->front_acc;
      const unsigned long long c = st->solid, k = st->claimed;
      if (c + k > st->nt) {
        st->trim_pending = 1;
        st->trim_parity = st->t & 1u;
        st->trim_keep = st->nt - c;
        st->solid = st->nt;
      } else {
        st->solid = c + k;
      }
      st->t += 1;
    }
  }
  st->front_acc = 0;
  st->claimed = 0;
  st->live = 0;
  st->iters += 1;
}

// Closes the step that just ran and opens the next.  With a graph
// conditional handle, also tells the enclosing while loop whether to go on.
// One warp: the 256-byte state comes in and goes back in one coalesced
// access each, and lane 0 works on the shared-memory copy, so the chain of
// dependent field reads costs shared-memory latency, not L2 latency.
__global__ void __launch_bounds__(32)
    k_step_control(RunState* st, cudaGraphConditionalHandle cond, int use_cond) {
  static_assert(sizeof(RunState) == 32 * sizeof(unsigned long long), "one word per lane");
  __shared__ RunState s;
  const uint32_t lane = threadIdx.x;
  reinterpret_cast<unsigned long long*>(&s)[lane] = reinterpret_cast<const unsigned long long*>(st)[lane];
  __syncwarp();
  if (lane == 0) {
    close_step(&s);
    begin_step(&s);
    if (use_cond) cudaGraphSetConditional(cond, s.active ? 1u : 0u);
  }
  __syncwarp();
  reinterpret_cast<unsigned long long*>(st)[lane] = reinterpret_cast<unsigned long long*>(&s)[lane];
}

__device__ void set_step_limit(RunState* st, uint32_t extra) {
  if (extra == 0) {
    st->step_limit = 0xFFFFFFFFu;
  } else {
    unsigned long long lim = (unsigned long long)st->t + extra;
    st->step_limit = lim > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)lim;
  }
  begin_step(st);
}

__global__ void k_set_step_limit(RunState* st, uint32_t extra) { set_step_limit(st, extra); }

__global__ void k_trim_done(RunState* st) { st->trim_pending = 0; }

__global__ void k_zero_front(RunState* st) { st->front_n = 0; }

// ---------------------------------------------------------------------------
// Shared helpers.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t ld_word(const uint32_t* p) { return *p; }

// ---------------------------------------------------------------------------
// Scan policies.
// ---------------------------------------------------------------------------
struct WordItem {
  uint32_t w;      // word index
  uint32_t bits;   // the word's set bits
  uint32_t extra;  // policy-specific second word
};

// Emit the voxel index of every set bit of a word, ascending.
__device__ __forceinline__ void emit_word_bits(const Geom& g, const WordItem& it, uint32_t* out,
                                               unsigned long long off) {
  const uint32_t r = fast_div(it.w, g.div_W);
  const uint32_t xw = it.w - r * g.W;
  const uint32_t v0 = r * g.nx + xw * 32u;
  uint32_t b = it.bits;
  while (b) {
    const int i = __ffs(b) - 1;
    b &= b - 1;
    out[off++] = v0 + (uint32_t)i;
  }
}

// Sec. 2.1 step 2: the Bernoulli candidate bits of one word, drawn from
// Philox block (v >> 2) word (v & 3) with the seeding tag.
__device__ __forceinline__ uint32_t seed_bits(const Geom& g, uint32_t w,
                                              unsigned long long t_seed,
                                              const PhiloxKeys& keys) {
  uint32_t bits = 0;
  if (t_seed != 0) {
    const uint32_t r = fast_div(w, g.div_W);
    const uint32_t xw = w - r * g.W;
    const uint32_t x0 = xw * 32u;
    const int len = (int)min(32u, g.nx - x0);
    const uint32_t v0 = r * g.nx + x0;
    const uint32_t g0 = v0 >> 2;        // first Philox block of the word
    const int s0 = (int)(v0 & 3u);      // bit i is voxel 4 * (g0 + j) + q with i = 4j + q - s0
    // The word's 32 voxels touch blocks g0 .. g0 + 8 (g0 + 7 when aligned).
#pragma unroll
    for (int j = 0; j < 9; ++j) {
      if (j == 8 && s0 == 0) break;
      const U4 blk = philox4x32_10(U4{g0 + (uint32_t)j, 0u, 0xFFFFFFFFu, kSeedTag}, keys);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = 4 * j + q - s0;
        if (i >= 0 && i < len && (unsigned long long)u4_word(blk, q) < t_seed) bits |= 1u << i;
      }
    }
  }
  if (g.blocked != nullptr && bits) bits &= ~g.blocked[w];  // R12: only unassigned cells
  return bits;
}

// The candidate bits of every word, written into the occupancy grid (empty
// until the seeds are placed): a grid-stride pass, one word per thread and
// iteration, so the Philox work runs with many resident warps and outside
// the ordered scan that lists the candidates.
__global__ void __launch_bounds__(256) k_seed_bits(Geom g, const RunState* st, uint32_t* grid,
                                                  const PhiloxKeys keys) {
  const unsigned long long t_seed = st->t_seed;
  for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < g.nwords;
       w += gridDim.x * blockDim.x)
    grid[w] = seed_bits(g, w, t_seed, keys);
}

// Lists the candidates of k_seed_bits in ascending voxel order and clears
// their bits from the grid again.
struct SeedCompactPolicy {
  Geom g;
  RunState* st;
  uint32_t* grid;          // candidate bits in, zero out
  uint32_t* cand;
  unsigned long long cap;  // entries cand can hold
  using Item = WordItem;
  __device__ uint32_t side(const Item&, int) const { return 0; }
  __device__ unsigned long long* side_sum(int) const { return nullptr; }
  __device__ void apply(const Item& it, bool valid) const {
    if (valid && it.bits) grid[it.w] = 0u;
  }
  __device__ bool active() const { return true; }
  __device__ bool emit_empty() const { return false; }
  __device__ uint32_t n_items() const { return g.nwords; }
  __device__ Item load(uint32_t w, bool valid) const {
    return Item{w, valid ? grid[w] : 0u, 0u};
  }
  __device__ uint32_t count(const Item& it) const { return __popc(it.bits); }
  // The word that straddles the capacity emits only its lowest (cap - off)
  // candidates, so the list holds exactly the first cap candidates.
  __device__ void emit(const Item& it, unsigned long long off) const {
    if (off >= cap) return;
    Item keep = it;
    if (off + __popc(it.bits) > cap) {
      uint32_t b = it.bits, low = 0;
      for (unsigned long long k = off; k < cap; ++k) {
        low |= b & (0u - b);  // lowest remaining candidate bit
        b &= b - 1;
      }
      keep.bits = low;
    }
    emit_word_bits(g, keep, cand, off);
  }
  // More candidates than the workspace holds (probability < 1e-15): the run
  // reports an overflow and keeps going on the first cap candidates.
  __device__ void total(unsigned long long n) const {
    if (n > cap) atomicOr(&st->error, kErrOverflow);
    st->cand_n = (uint32_t)(n > cap ? cap : n);
  }
};

// The candidate word list that drives the growth kernel: words that may
// hold front voxels (Sec. 2.3 step 2: solids with a void neighbour).
//
// Why "words marked by the last growth step, plus words that received
// claims" is enough: a voxel solid after step t with a void neighbour either
// is in New_t or was solid before with that neighbour already void (voids
// only shrink), i.e. it was a front voxel of step t.  So A_{t+1} = prune(A_t
// U New_t) lies in those words, and the growth kernel itself computes the
// exact front bits of every candidate word from the grid.
//
// The first list of a run (after seeding, or after the blocked cells or
// the state changed) is every word holding a solid voxel, in ascending word
// order: InitialListPolicy, an ordered look-back scan over the words.  The
// lists of later steps come from k_commit below.
struct InitialListPolicy {
  Geom g;
  RunState* st;
  const uint32_t* grid;
  uint32_t* list;
  struct Item {
    uint32_t w;     // word index
    uint32_t bits;  // 1: listed
  };
  __device__ bool active() const { return true; }
  __device__ bool emit_empty() const { return false; }
  __device__ uint32_t n_items() const { return g.nwords; }
  __device__ Item load(uint32_t w, bool valid) const {
    const uint32_t solid = valid ? grid[w] : 0u;
    return Item{w, solid ? 1u : 0u};
  }
  __device__ void apply(const Item&, bool) const {}
  __device__ uint32_t count(const Item& it) const { return it.bits; }
  __device__ uint32_t side(const Item&, int) const { return 0u; }
  __device__ unsigned long long* side_sum(int) const { return nullptr; }
  __device__ void emit(const Item& it, unsigned long long off) const { list[off] = it.w; }
  __device__ void total(unsigned long long n) const { st->front_words = (uint32_t)n; }
};

// Commit of a growth step: ORs the step's claims into the grid, counts them,
// appends marked or touched words to the next candidate list and clears the
// marks and touched bits (the growth kernel has already cleared the other
// claim grid).  A touched word holds claims and a marked one front voxels
// of this step: exactly the words of A_t U New_t.  The list is appended in
// any order -- the growth step gives the same result for any order of its
// list, every draw being keyed by (voxel, step, block) and claims ORed --
// but neighbouring words in ascending runs, so that a growth warp's 32 list
// entries are mostly neighbouring words, whose rows it reads from L1 (2 %
// of a 400^3 realization against lane-interleaved entries).
//
// Two paths, chosen per step by the size of the step's list (uniform):
//   - sparse (list < nwords / kSparseFraction): a warp reads 4 x 32 words
//     of both bitmaps (4096 grid words) at a time and serves the non-zero ones
//     in groups of kCommitGroup, a lane per grid word, loads first; the
//     work follows the front -- a region without it costs one coalesced
//     bitmap read per 1024 words, and no warp waits on another;
//   - dense: tiles of 2048 words, thread t of a block taking words base +
//     k * 256 + t (k < 8), every word's claims and grid word loaded together
//     with the bitmaps (no dependent round trip), one atomic per tile --
//     cheaper once the front occupies most words.
constexpr int kCommitThreads = 256;
constexpr int kCommitItems = 8;
constexpr int kCommitGroup = 8;
constexpr uint32_t kSparseFraction = 32;

// The commit of a step whose list holds list_n of nwords words takes the
// sparse path.
__device__ __forceinline__ bool commit_is_sparse(uint32_t list_n, uint32_t nwords) {
  return (unsigned long long)list_n * kSparseFraction < nwords;
}

// Lanes of a warp: the next (up to) kCommitGroup set bits of the uniform
// mask nz, as source lanes src[k] with their bitmap words mm[k] (0 past the
// last set bit); nz loses those bits.
__device__ __forceinline__ void next_group(uint32_t& nz, uint32_t m, uint32_t (&src)[kCommitGroup],
                                           uint32_t (&mm)[kCommitGroup]) {
#pragma unroll
  for (int k = 0; k < kCommitGroup; ++k) {
    const bool any = nz != 0u;
    src[k] = any ? (uint32_t)(__ffs(nz) - 1) : 0u;
    const uint32_t v = __shfl_sync(0xffffffffu, m, src[k]);
    mm[k] = any ? v : 0u;
    nz &= nz - 1u;
  }
}

// The sparse path (all lanes of the warp together): returns this lane's
// count of claimed voxels.  A warp reads kSparseRows rows of 32 bitmap
// words per iteration, all loads in flight together.
constexpr int kSparseRows = 4;

__device__ __forceinline__ uint32_t commit_sparse(const Geom& g, RunState* st, uint32_t* grid,
                                                  const uint32_t* claims, uint32_t* mark,
                                                  uint32_t* touched, uint32_t* list) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t nb = bitmap_words(g), nw = g.nwords;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  uint32_t claimed = 0;
  for (uint32_t r0 = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * (32u * kSparseRows);
       r0 < nb; r0 += nwarps * 32u * kSparseRows) {
    uint32_t mk[kSparseRows], tc[kSparseRows];
#pragma unroll
    for (int r = 0; r < kSparseRows; ++r) {
      const uint32_t j = r0 + r * 32u + lane;
      mk[r] = j < nb ? mark[j] : 0u;
      tc[r] = j < nb ? touched[j] : 0u;
    }
    // One list reservation for all words of the kSparseRows rows (a single
    // counter takes every step's appends: one atomic per warp iteration, not
    // per group).
    uint32_t words = 0;
#pragma unroll
    for (int r = 0; r < kSparseRows; ++r) words += (uint32_t)__popc(mk[r] | tc[r]);
    words = __reduce_add_sync(0xffffffffu, words);
    uint32_t base = 0;
    if (lane == 0 && words) base = atomicAdd(&st->list_next, words);
    base = __shfl_sync(0xffffffffu, base, 0);
#pragma unroll
    for (int r = 0; r < kSparseRows; ++r) {
      const uint32_t j0 = r0 + r * 32u;
      if (mk[r]) mark[j0 + lane] = 0u;
      if (tc[r]) touched[j0 + lane] = 0u;
      const uint32_t m = mk[r] | tc[r];
      uint32_t nz = __ballot_sync(0xffffffffu, m != 0u);
      while (nz) {  // warp-uniform
        uint32_t src[kCommitGroup], mm[kCommitGroup], c[kCommitGroup], old[kCommitGroup];
        bool act[kCommitGroup];
        next_group(nz, m, src, mm);
#pragma unroll
        for (int k = 0; k < kCommitGroup; ++k) {
          // (64-bit: near N = 2^32 with nx < 32 the word count nears 2^32
          // too; bits past nw are never set.)
          const unsigned long long w = (unsigned long long)(j0 + src[k]) * 32u + lane;
          act[k] = ((mm[k] >> lane) & 1u) && w < nw;
          c[k] = act[k] ? claims[w] : 0u;
          old[k] = act[k] ? grid[w] : 0u;
        }
#pragma unroll
        for (int k = 0; k < kCommitGroup; ++k) {
          if (c[k]) grid[(j0 + src[k]) * 32u + lane] = old[k] | c[k];
          claimed += (uint32_t)__popc(c[k]);
        }
#pragma unroll
        for (int k = 0; k < kCommitGroup; ++k) {
          if (act[k]) list[base + __popc(mm[k] & lt)] = (j0 + src[k]) * 32u + lane;
          base += (uint32_t)__popc(mm[k]);
        }
      }
    }
  }
  return claimed;
}

__global__ void __launch_bounds__(kCommitThreads, 3)
    k_commit(Geom g, RunState* st, uint32_t* grid, uint32_t* aux, uint32_t* mark,
             uint32_t* list) {
  constexpr int kWarps = kCommitThreads / 32;
  __shared__ uint32_t s_off[kCommitItems * kWarps];
  __shared__ uint32_t s_base;
  __shared__ unsigned long long s_claimed;
  if (!st->active) return;
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const uint32_t nw = g.nwords;
  uint32_t* touched = mark + bitmap_words(g);
  const uint32_t* claims = aux + (size_t)(st->t & 1u) * nw;
  const bool sparse = commit_is_sparse(st->front_words, nw);
  if (threadIdx.x == 0) s_claimed = 0;
  uint32_t claimed = 0;
  constexpr uint32_t kTile = kCommitThreads * kCommitItems;
  if (sparse) claimed = commit_sparse(g, st, grid, claims, mark, touched, list);
  for (uint32_t base = blockIdx.x * kTile; !sparse && base < nw; base += gridDim.x * kTile) {
    // Lane k < 8: the bitmap word of this warp's row k.
    const uint32_t row0 = base + lane * kCommitThreads + warp * 32u;
    const bool jv = lane < (uint32_t)kCommitItems && row0 < nw;
    const uint32_t jk = row0 >> 5;
    uint32_t c[kCommitItems], old[kCommitItems];
    uint32_t keep = 0;  // bit k: word k is listed
    const uint32_t mk = jv ? mark[jk] : 0u, tc = jv ? touched[jk] : 0u;
#pragma unroll
    for (int k = 0; k < kCommitItems; ++k) {
      const uint32_t w = base + k * kCommitThreads + threadIdx.x;
      const bool valid = w < nw;
      c[k] = valid ? claims[w] : 0u;
      old[k] = valid ? grid[w] : 0u;
    }
    if (mk) mark[jk] = 0u;
    if (tc) touched[jk] = 0u;
#pragma unroll
    for (int k = 0; k < kCommitItems; ++k) {
      const uint32_t mkk = __shfl_sync(0xffffffffu, mk, k);
      if (((mkk >> lane) & 1u) | (c[k] ? 1u : 0u)) keep |= 1u << k;
    }
#pragma unroll
    for (int k = 0; k < kCommitItems; ++k) {
      if (c[k]) grid[base + k * kCommitThreads + threadIdx.x] = old[k] | c[k];
      claimed += (uint32_t)__popc(c[k]);
    }
    // The tile's kept words in ascending order (k-major, then warp, then
    // lane), one atomic for the tile: a growth warp's 32 list entries are
    // then mostly neighbouring words, whose rows it reads from L1.
    uint32_t bk[kCommitItems], cnt_mine = 0;
#pragma unroll
    for (int k = 0; k < kCommitItems; ++k) {
      bk[k] = __ballot_sync(0xffffffffu, (keep >> k) & 1u);
      if (lane == (uint32_t)k) cnt_mine = (uint32_t)__popc(bk[k]);
    }
    if (lane < (uint32_t)kCommitItems) s_off[lane * kWarps + warp] = cnt_mine;
    __syncthreads();
    if (warp == 0) {
      static_assert(kCommitItems * kWarps == 64, "two counts per lane");
      const uint32_t a0 = s_off[2 * lane], a1 = s_off[2 * lane + 1];
      uint32_t incl = a0 + a1;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= (uint32_t)off) incl += y;
      }
      s_off[2 * lane] = incl - a0 - a1;
      s_off[2 * lane + 1] = incl - a1;
      const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
      if (lane == 0) s_base = tot ? atomicAdd(&st->list_next, tot) : 0u;
    }
    __syncthreads();
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
    for (int k = 0; k < kCommitItems; ++k)
      if ((keep >> k) & 1u)
        list[s_base + s_off[k * kWarps + warp] + __popc(bk[k] & lt)] =
            base + k * kCommitThreads + threadIdx.x;
    __syncthreads();  // s_off / s_base are reused by the next tile

  }
  const uint32_t wc = __reduce_add_sync(0xffffffffu, claimed);
  if (lane == 0 && wc) atomicAdd(&s_claimed, (unsigned long long)wc);
  __syncthreads();
  if (threadIdx.x == 0 && s_claimed) atomicAdd(&st->claimed, s_claimed);
}

// The front size |A| of the current grid (solids with a void in-domain
// 26-neighbour), counted once at the end of a growth call for the
// statistics.  Warp-cooperative: the 32 lanes hold 32 consecutive words,
// each neighbour row arrives in one coalesced load and the x-1 / x+1 bits
// come from the neighbouring lanes.
// Domain kind of a growth-path instantiation: the open domain (R6), the
// torus (R11), read from Geom at run time (batches mix both), or a phase
// that enters cells of earlier phases (R13; periodic read at run time).
enum DomainKind : int { kOpen = 0, kTorus = 1, kRuntime = 2, kInteract = 3 };

template <int DK>
__device__ __forceinline__ bool on_torus(const Geom& g) {
  return (DK == kRuntime || DK == kInteract) ? g.periodic != 0u : DK == kTorus;
}

// Cells of earlier phases (R12) are only looked at by the run-time and
// interacting kinds.
template <int DK>
__device__ __forceinline__ bool has_blocked(const Geom& g) {
  return DK == kInteract || (DK == kRuntime && g.blocked != nullptr);
}

template <int DK>
__device__ __forceinline__ void word_masks(const Geom& g, const uint32_t* __restrict__ grid,
                                           uint32_t w, uint32_t live_dirs, uint32_t (&V)[28],
                                           uint32_t (&Bm)[7], uint32_t& front, uint32_t& r,
                                           uint32_t& xw);

struct FrontCountPolicy {
  Geom g;
  RunState* st;
  const uint32_t* grid;
  using Item = WordItem;
  __device__ void apply(const Item&, bool) const {}
  __device__ bool active() const { return true; }
  __device__ bool emit_empty() const { return false; }
  __device__ uint32_t n_items() const { return g.nwords; }
  __device__ Item load(uint32_t w, bool valid) const {
    if (g.periodic || g.blocked) {  // the growth kernel's own neighbour masks
      uint32_t V[28], Bm[7] = {0, 0, 0, 0, 0, 0, 0}, front = 0, r, xw;
      if (valid) word_masks<kRuntime>(g, grid, w, (1u << 26) - 1u, V, Bm, front, r, xw);
      return Item{w, front, 0u};
    }
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t r = fast_div(w, g.div_W);
    const uint32_t xw = w - r * g.W;
    const uint32_t z = fast_div(r, g.div_ny);
    const uint32_t y = r - z * g.ny;
    const uint32_t self = valid ? grid[w] : 0u;
    const int64_t plane = (int64_t)g.W * g.ny;
    uint32_t solid_all = 0xFFFFFFFFu;
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz) {
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy) {
        const int yy = (int)y + dy, zz = (int)z + dz;
        const bool row_ok = valid && yy >= 0 && yy < (int)g.ny && zz >= 0 && zz < (int)g.nz;
        const int64_t q = (int64_t)w + (int64_t)dy * g.W + (int64_t)dz * plane;
        const uint32_t c0 = row_ok ? grid[q] : 0xFFFFFFFFu;
        uint32_t l = __shfl_up_sync(0xffffffffu, c0, 1);
        uint32_t rr = __shfl_down_sync(0xffffffffu, c0, 1);
        if (lane == 0 && row_ok && xw > 0) l = grid[q - 1];
        if (lane == 31 && row_ok && xw + 1 < g.W) rr = grid[q + 1];
        if (row_ok) {
          uint32_t c = c0;
          if (xw == g.W - 1) c |= g.pad_mask;
          if (xw == 0) l = 0xFFFFFFFFu;
          if (xw + 1 >= g.W) {
            rr = 0xFFFFFFFFu;
          } else if (xw + 1 == g.W - 1) {
            rr |= g.pad_mask;
          }
          uint32_t a = ((c << 1) | (l >> 31)) & ((c >> 1) | (rr << 31));
          if (dy != 0 || dz != 0) a &= c;
          solid_all &= a;
        }
      }
    }
    return Item{w, self & ~solid_all, 0u};
  }
  __device__ uint32_t count(const Item&) const { return 0u; }
  __device__ uint32_t side(const Item& it, int k) const { return k == 0 ? __popc(it.bits) : 0u; }
  __device__ unsigned long long* side_sum(int k) const { return k == 0 ? &st->front_n : nullptr; }
  __device__ void emit(const Item&, unsigned long long) const {}
  __device__ void total(unsigned long long) const {}
};

// The front count of an interacting phase (R13): a voxel is active if it has
// a void neighbour or an enterable one -- the growth kernel's own masks.
struct FrontCountInterPolicy {
  GeomInter g;
  RunState* st;
  const uint32_t* grid;
  using Item = WordItem;
  __device__ void apply(const Item&, bool) const {}
  __device__ bool active() const { return true; }
  __device__ bool emit_empty() const { return false; }
  __device__ uint32_t n_items() const { return g.nwords; }
  __device__ Item load(uint32_t w, bool valid) const {
    uint32_t V[28], Bm[7] = {0, 0, 0, 0, 0, 0, 0}, front = 0, r, xw;
    if (valid) word_masks<kInteract>(g, grid, w, (1u << 26) - 1u, V, Bm, front, r, xw);
    return Item{w, front, 0u};
  }
  __device__ uint32_t count(const Item&) const { return 0u; }
  __device__ uint32_t side(const Item& it, int k) const { return k == 0 ? __popc(it.bits) : 0u; }
  __device__ unsigned long long* side_sum(int k) const { return k == 0 ? &st->front_n : nullptr; }
  __device__ void emit(const Item&, unsigned long long) const {}
  __device__ void total(unsigned long long) const {}
};

// A count policy's side sum without the ordered scan: nothing is emitted,
// so no tile waits on its predecessors.  Each warp takes 32 consecutive
// items per iteration (the front policies' neighbour shuffles need
// consecutive words in consecutive lanes) and adds its warp total with one
// atomic.
template <class Policy>
__global__ void __launch_bounds__(256) k_side_sum(Policy pol) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t n = pol.n_items();
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  unsigned long long sum = 0;
  for (uint32_t w0 = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32u; w0 < n;
       w0 += nwarps * 32u) {
    const uint32_t w = w0 + lane;
    sum += pol.side(pol.load(w, w < n), 0);
  }
  const unsigned long long ws = __reduce_add_sync(0xffffffffu, (uint32_t)sum);
  if (lane == 0 && ws) atomicAdd(pol.side_sum(0), ws);
}

// The exact-target trim, once, after the step that overshot Nt.  The claim
// grid of that step holds exactly New_t (every success targets a voxel that
// was void when the step began); of New_t in ascending order only the first
// trim_keep voxels stay solid, the rest are cleared from the grid again.
struct TrimPolicy {
  Geom g;
  RunState* st;
  uint32_t* grid;
  const uint32_t* aux;  // two claim grids
  using Item = WordItem;
  __device__ uint32_t side(const Item&, int) const { return 0; }
  __device__ unsigned long long* side_sum(int) const { return nullptr; }
  __device__ void apply(const Item&, bool) const {}
  __device__ bool active() const { return st->trim_pending != 0; }
  __device__ bool emit_empty() const { return false; }
  __device__ uint32_t n_items() const { return g.nwords; }
  __device__ Item load(uint32_t w, bool valid) const {
    if (!valid) return Item{};
    return Item{w, aux[(size_t)st->trim_parity * g.nwords + w], 0u};
  }
  __device__ uint32_t count(const Item& it) const { return __popc(it.bits); }
  __device__ void emit(const Item& it, unsigned long long off) const {
    const unsigned long long keep = st->trim_keep;
    if (off + __popc(it.bits) <= keep) return;
    uint32_t drop = it.bits;
    if (off < keep) {
      uint32_t k = (uint32_t)(keep - off);
      uint32_t b = it.bits;
      while (k--) b &= b - 1;  // b = the bits beyond the first (keep - off)
      drop = b;
    }
    grid[it.w] &= ~drop;
  }
  __device__ void total(unsigned long long) const {}
};

// Seeds: the accepted candidates in ascending order, capped at Nt, written
// into the grid.
struct AcceptPolicy {
  Geom g;
  RunState* st;
  uint32_t* grid;
  const uint32_t* cand;
  const uint8_t* decision;  // nullptr: every candidate accepted
  struct Item {
    uint32_t v;
    uint32_t ok;
  };
  __device__ uint32_t side(const Item&, int) const { return 0; }
  __device__ unsigned long long* side_sum(int) const { return nullptr; }
  __device__ void apply(const Item&, bool) const {}
  __device__ bool active() const { return true; }
  __device__ bool emit_empty() const { return false; }
  __device__ uint32_t n_items() const { return st->cand_n; }
  __device__ Item load(uint32_t i, bool valid) const {
    if (!valid) return Item{};
    return Item{cand[i], decision ? (uint32_t)(decision[i] == 1) : 1u};
  }
  __device__ uint32_t count(const Item& it) const { return it.ok; }
  __device__ void emit(const Item& it, unsigned long long off) const {
    if (off < st->nt && it.v < g.n) {  // v >= N only after a timed-out scan
      const uint32_t r = fast_div(it.v, g.div_nx);
      const uint32_t x = it.v - r * g.nx;
      atomicOr(grid + (size_t)r * g.W + (x >> 5), 1u << (x & 31));
    }
  }
  __device__ void total(unsigned long long n) const {
    const unsigned long long placed = n < st->nt ? n : st->nt;
    st->acc_n = (uint32_t)placed;
    st->solid = placed;
  }
};

// Exclusive offsets of the spacing cells; the counts become fill cursors.
struct CellOffsetPolicy {
  RunState* st;
  uint32_t ncells;
  uint32_t* cell_count;  // in: per-cell counts; out: start offsets (cursors)
  uint32_t* start;       // out: ncells + 1 offsets
  struct Item {
    uint32_t i, c;
  };
  __device__ uint32_t side(const Item&, int) const { return 0; }
  __device__ unsigned long long* side_sum(int) const { return nullptr; }
  __device__ void apply(const Item&, bool) const {}
  __device__ bool active() const { return true; }
  __device__ bool emit_empty() const { return true; }
  __device__ uint32_t n_items() const { return ncells; }
  __device__ Item load(uint32_t i, bool valid) const {
    if (!valid) return Item{};
    return Item{i, cell_count[i]};
  }
  __device__ uint32_t count(const Item& it) const { return it.c; }
  __device__ void emit(const Item& it, unsigned long long off) const {
    start[it.i] = (uint32_t)off;
    cell_count[it.i] = (uint32_t)off;
  }
  __device__ void total(unsigned long long n) const { start[ncells] = (uint32_t)n; }
};

// ---------------------------------------------------------------------------
// Seed spacing (Sec. 2.3, Fig. 1 D): greedy in ascending index -- keep a
// candidate iff no kept candidate before it lies within L1 distance < s.
// Candidates are binned into cubic cells of edge s, so every conflict lies
// in the 27 surrounding cells.  The greedy choice is computed by rounds: a
// candidate is kept once every earlier conflicting candidate is rejected,
// and rejected once one of them is kept.  Each round settles at least the
// lowest undecided candidate, so n + 1 rounds always suffice.
// ---------------------------------------------------------------------------
struct CellGeom {
  uint32_t s, ncx, ncy, ncz;
  uint32_t periodic;  // torus: cells of width >= s tile each axis exactly
};

// Cell of coordinate u on an axis of n voxels and nc cells.  Open domain:
// width s (the last cell may be narrower).  Torus: nc = max(1, floor(n/s))
// cells of width >= s, so a point within distance < s of u, across the
// wrap too, lies in u's cell or one of its two neighbours.
__device__ __forceinline__ uint32_t cell_coord(const CellGeom& cg, uint32_t u, uint32_t n,
                                               uint32_t nc) {
  return cg.periodic ? (uint32_t)(((unsigned long long)u * nc) / n) : u / cg.s;
}

// Cell cu + du on an axis of nc cells; false if it lies outside the open
// domain, or repeats a cell already visited on a torus of fewer than 3 cells.
__device__ __forceinline__ bool cell_step(const CellGeom& cg, int cu, int du, uint32_t nc,
                                          uint32_t& out) {
  int v = cu + du;
  if (cg.periodic) {
    if ((nc == 1 && du != 0) || (nc == 2 && du == -1)) return false;
    v = v < 0 ? v + (int)nc : (v >= (int)nc ? v - (int)nc : v);
  } else if (v < 0 || v >= (int)nc) {
    return false;
  }
  out = (uint32_t)v;
  return true;
}

// L1 distance between two voxels, around the torus when periodic.
__device__ __forceinline__ int spacing_l1(const Geom& g, uint32_t x, uint32_t y, uint32_t z,
                                          uint32_t xj, uint32_t yj, uint32_t zj) {
  int dx = abs((int)xj - (int)x), dy = abs((int)yj - (int)y), dz = abs((int)zj - (int)z);
  if (g.periodic) {
    dx = min(dx, (int)g.nx - dx);
    dy = min(dy, (int)g.ny - dy);
    dz = min(dz, (int)g.nz - dz);
  }
  return dx + dy + dz;
}

__device__ __forceinline__ void decode_xyz(const Geom& g, uint32_t v, uint32_t& x, uint32_t& y,
                                           uint32_t& z) {
  const uint32_t r = fast_div(v, g.div_nx);
  x = v - r * g.nx;
  z = fast_div(r, g.div_ny);
  y = r - z * g.ny;
}

__global__ void k_cell_count(Geom g, CellGeom cg, const RunState* st, const uint32_t* cand,
                             uint32_t* count) {
  const uint32_t n = st->cand_n;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (cand[i] >= g.n) continue;  // only after a timed-out scan (reported)
    uint32_t x, y, z;
    decode_xyz(g, cand[i], x, y, z);
    const uint32_t cell = cell_coord(cg, x, g.nx, cg.ncx) +
                          cg.ncx * (cell_coord(cg, y, g.ny, cg.ncy) +
                                    cg.ncy * cell_coord(cg, z, g.nz, cg.ncz));
    atomicAdd(count + cell, 1u);
  }
}

__global__ void k_cell_fill(Geom g, CellGeom cg, const RunState* st, const uint32_t* cand,
                            uint32_t* cursor, uint32_t* items, uint8_t* decision) {
  const uint32_t n = st->cand_n;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    decision[i] = 0;
    if (cand[i] >= g.n) continue;  // only after a timed-out scan (reported)
    uint32_t x, y, z;
    decode_xyz(g, cand[i], x, y, z);
    const uint32_t cell = cell_coord(cg, x, g.nx, cg.ncx) +
                          cg.ncx * (cell_coord(cg, y, g.ny, cg.ncy) +
                                    cg.ncy * cell_coord(cg, z, g.nz, cg.ncz));
    items[atomicAdd(cursor + cell, 1u)] = i;
  }
}

// Earlier conflicts of candidate i: candidates j < i at L1 distance < s,
// found in the 27 cells around i.  One warp per candidate: lane c < 27 scans
// cell c.  Returns the count to every lane; with `out`, the conflicts are
// written to out[0 .. count) (grouped by cell; the rounds below do not
// depend on their order).  All 32 lanes must call it together.
__device__ __forceinline__ uint32_t scan_conflicts_warp(const Geom& g, const CellGeom& cg,
                                                        const uint32_t* cand,
                                                        const uint32_t* start,
                                                        const uint32_t* items, uint32_t i,
                                                        uint32_t* out,
                                                        unsigned long long out_cap = 0) {
  const uint32_t lane = threadIdx.x & 31u;
  if (cand[i] >= g.n) return 0;  // only after a timed-out scan (reported)
  uint32_t x, y, z;
  decode_xyz(g, cand[i], x, y, z);
  uint32_t k0 = 0, k1 = 0;
  if (lane < 27) {
    uint32_t xx, yy, zz;
    if (cell_step(cg, (int)cell_coord(cg, x, g.nx, cg.ncx), (int)(lane % 3u) - 1, cg.ncx, xx) &&
        cell_step(cg, (int)cell_coord(cg, y, g.ny, cg.ncy), (int)((lane / 3u) % 3u) - 1, cg.ncy,
                  yy) &&
        cell_step(cg, (int)cell_coord(cg, z, g.nz, cg.ncz), (int)(lane / 9u) - 1, cg.ncz, zz)) {
      const uint32_t cell = xx + cg.ncx * (yy + cg.ncy * zz);
      k0 = start[cell];
      k1 = start[cell + 1];
    }
  }
  auto conflicts = [&](uint32_t k, uint32_t& j) {
    j = items[k];
    if (j >= i || cand[j] >= g.n) return false;
    uint32_t xj, yj, zj;
    decode_xyz(g, cand[j], xj, yj, zj);
    return spacing_l1(g, x, y, z, xj, yj, zj) < (int)cg.s;
  };
  uint32_t mine = 0;
  for (uint32_t k = k0; k < k1; ++k) {
    uint32_t j;
    if (conflicts(k, j)) ++mine;
  }
  uint32_t incl = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= (uint32_t)o) incl += v;
  }
  if (out != nullptr && mine) {
    uint32_t pos = incl - mine;
    for (uint32_t k = k0; k < k1; ++k) {
      uint32_t j;
      if (conflicts(k, j)) {
        if (pos < out_cap) out[pos] = j;  // out_cap < count only after a timed-out scan
        ++pos;
      }
    }
  }
  return __shfl_sync(0xffffffffu, incl, 31);
}

__global__ void k_conflict_count(Geom g, CellGeom cg, const RunState* st, const uint32_t* cand,
                                 const uint32_t* start, const uint32_t* items, uint32_t* cnt) {
  const uint32_t n = st->cand_n;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nwarps) {
    const uint32_t c = scan_conflicts_warp(g, cg, cand, start, items, i, nullptr);
    if ((threadIdx.x & 31u) == 0) cnt[i] = c;
  }
}

// Exclusive offsets of the conflict lists (in place: counts -> offsets).
struct ConflictOffsetPolicy {
  RunState* st;
  uint32_t* off;  // in: counts; out: offsets, off[cand_n] = total
  struct Item {
    uint32_t i, c;
  };
  __device__ uint32_t side(const Item&, int) const { return 0; }
  __device__ unsigned long long* side_sum(int) const { return nullptr; }
  __device__ void apply(const Item&, bool) const {}
  __device__ bool active() const { return true; }
  __device__ bool emit_empty() const { return true; }
  __device__ uint32_t n_items() const { return st->cand_n; }
  __device__ Item load(uint32_t i, bool valid) const {
    if (!valid) return Item{};
    return Item{i, off[i]};
  }
  __device__ uint32_t count(const Item& it) const { return it.c; }
  __device__ void emit(const Item& it, unsigned long long o) const { off[it.i] = (uint32_t)o; }
  __device__ void total(unsigned long long n) const {
    off[st->cand_n] = (uint32_t)(n > 0xFFFFFFFFull ? 0xFFFFFFFFull : n);
    st->adj_n = n;
  }
};

__global__ void k_conflict_fill(Geom g, CellGeom cg, const RunState* st, const uint32_t* cand,
                                const uint32_t* start, const uint32_t* items, const uint32_t* off,
                                uint32_t* adj, unsigned long long cap) {
  if (st->adj_n > cap) return;
  const uint32_t n = st->cand_n;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nwarps) {
    const unsigned long long o = off[i];
    scan_conflicts_warp(g, cg, cand, start, items, i, adj + (o < cap ? o : cap),
                        o < cap ? cap - o : 0ull);
  }
}

// Rounds over the conflict lists (one block).  Each round settles at least
// the lowest undecided candidate, so cand_n + 1 rounds always suffice.  The
// decisions live in shared memory while they fit (kSpacingSmem candidates),
// else in the global array; they are copied out at the end.  Thread t owns
// candidates t + 1024 q; while there are at most 64 per thread (every
// candidate count that fits in shared memory) it keeps its undecided ones
// as a bit mask over q, so a round visits only undecided candidates, and
// one barrier per round both orders the decisions and tells whether any
// candidate is left.
constexpr uint32_t kSpacingSmem = 64 * 1024;
constexpr uint32_t kSpacingThreads = 1024;

// Settles candidate i if its earlier conflicts allow: 1 accepted (no
// earlier conflict accepted or pending), 2 rejected (one accepted);
// returns false while one is still pending.
__device__ __forceinline__ bool spacing_settle(uint32_t i, uint32_t n, const uint32_t* off,
                                               const uint32_t* adj, unsigned long long cap,
                                               uint8_t* dec) {
  bool pending = false;
  const unsigned long long k_end = off[i + 1] < cap ? off[i + 1] : cap;
  for (unsigned long long k = off[i]; k < k_end; ++k) {
    const uint32_t j = adj[k];
    if (j >= n) continue;  // only after a timed-out scan (reported)
    const uint8_t dj = ((volatile uint8_t*)dec)[j];
    if (dj == 1) {
      dec[i] = 2;
      return true;
    }
    if (dj == 0) pending = true;
  }
  if (pending) return false;
  dec[i] = 1;
  return true;
}

__global__ void __launch_bounds__(kSpacingThreads) k_spacing_rounds_csr(const RunState* st,
                                                                       const uint32_t* off,
                                                                       const uint32_t* adj,
                                                                       uint8_t* decision,
                                                                       unsigned long long cap) {
  extern __shared__ uint8_t s_decision[];
  if (st->adj_n > cap) return;
  const uint32_t n = st->cand_n;
  const bool in_smem = n <= kSpacingSmem;
  uint8_t* dec = in_smem ? s_decision : decision;
  for (uint32_t i = threadIdx.x; i < n; i += kSpacingThreads) dec[i] = 0;
  __syncthreads();
  if (n <= 64u * kSpacingThreads) {
    // und[h] bit q: candidate threadIdx.x + 1024 (32 h + q) is undecided.
    const uint32_t mine = threadIdx.x < n ? (n - 1u - threadIdx.x) / kSpacingThreads + 1u : 0u;
    uint32_t und[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint32_t cnt = mine > 32u * h ? min(mine - 32u * h, 32u) : 0u;
      und[h] = cnt == 32u ? 0xFFFFFFFFu : (1u << cnt) - 1u;
    }
    for (uint32_t round = 0; round <= n; ++round) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        for (uint32_t m = und[h]; m; m &= m - 1) {
          const uint32_t q = (uint32_t)__ffs(m) - 1u;
          if (spacing_settle(threadIdx.x + kSpacingThreads * (32u * h + q), n, off, adj, cap, dec))
            und[h] &= ~(1u << q);
        }
      }
      if (!__syncthreads_or((und[0] | und[1]) != 0u)) break;
    }
  } else {
    for (uint32_t round = 0; round <= n; ++round) {
      bool left = false;
      for (uint32_t i = threadIdx.x; i < n; i += kSpacingThreads)
        if (((volatile uint8_t*)dec)[i] == 0 && !spacing_settle(i, n, off, adj, cap, dec))
          left = true;
      if (!__syncthreads_or(left)) break;
    }
  }
  if (in_smem)
    for (uint32_t i = threadIdx.x; i < n; i += kSpacingThreads) decision[i] = s_decision[i];
}

// Fallback when the conflict lists exceed their buffer: one block runs all
// rounds and re-examines the 27 cells of every undecided candidate.

__global__ void __launch_bounds__(1024) k_spacing_rounds(Geom g, CellGeom cg, RunState* st,
                                                        const uint32_t* cand,
                                                        const uint32_t* start,
                                                        const uint32_t* items,
                                                        uint8_t* decision,
                                                        unsigned long long cap) {
  __shared__ uint32_t s_undecided;
  if (st->adj_n <= cap) return;
  const uint32_t n = st->cand_n;
  const int s = (int)cg.s;
  for (uint32_t round = 0; round <= n; ++round) {
    if (threadIdx.x == 0) s_undecided = 0;
    __syncthreads();
    uint32_t mine = 0;
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
      if (((volatile uint8_t*)decision)[i] != 0) continue;
      if (cand[i] >= g.n) {  // only after a timed-out scan (reported)
        decision[i] = 2;
        continue;
      }
      uint32_t x, y, z;
      decode_xyz(g, cand[i], x, y, z);
      const int cx = (int)cell_coord(cg, x, g.nx, cg.ncx);
      const int cy = (int)cell_coord(cg, y, g.ny, cg.ncy);
      const int cz = (int)cell_coord(cg, z, g.nz, cg.ncz);
      bool pending = false, rejected = false;
      for (int dz = -1; dz <= 1 && !rejected; ++dz) {
        uint32_t zz;
        if (!cell_step(cg, cz, dz, cg.ncz, zz)) continue;
        for (int dy = -1; dy <= 1 && !rejected; ++dy) {
          uint32_t yy;
          if (!cell_step(cg, cy, dy, cg.ncy, yy)) continue;
          for (int dx = -1; dx <= 1 && !rejected; ++dx) {
            uint32_t xx;
            if (!cell_step(cg, cx, dx, cg.ncx, xx)) continue;
            const uint32_t cell = xx + cg.ncx * (yy + cg.ncy * zz);
            for (uint32_t k = start[cell]; k < start[cell + 1]; ++k) {
              const uint32_t j = items[k];
              if (j >= i || cand[j] >= g.n) continue;  // only earlier candidates matter
              uint32_t xj, yj, zj;
              decode_xyz(g, cand[j], xj, yj, zj);
              if (spacing_l1(g, x, y, z, xj, yj, zj) >= s) continue;
              const uint8_t dj = ((volatile uint8_t*)decision)[j];
              if (dj == 1) { rejected = true; break; }
              if (dj == 0) pending = true;
            }
          }
        }
      }
      if (rejected) decision[i] = 2;
      else if (!pending) decision[i] = 1;
      else ++mine;
    }
    if (mine) atomicAdd(&s_undecided, mine);
    __syncthreads();
    const uint32_t left = s_undecided;
    __syncthreads();
    if (left == 0) break;
  }
}

// ---------------------------------------------------------------------------
// The growth step (Sec. 2.3 step 3, Algorithm 3).  Every front
// voxel a tries each void in-domain neighbour q = a + e_d (its targets)
// against the class threshold of Eq. 1, with the draw located by rank: the
// r-th target of class c takes word r & 3 of Philox block (a, 0, t, 0x200 |
// B_c + r >> 2), B = 0, 2, 5 for faces, edges, corners (growth_blocks); a
// success records q in this step's claim grid with a fire-and-forget
// atomicOr.  The occupancy grid is not written during the
// kernel, so every thread sees the start-of-step grid: the front, the void
// targets and the attempt count are those of Algorithm 3 exactly, and the
// claim grid ends up holding New_t (the commit scan ORs it into the grid).
//
// Work layout.  A warp takes 32 entries of the candidate word list (a
// superset of the words holding front voxels).  Phase 1: each lane builds,
// bit-parallel over its 32 voxels, the front bits (solid with a void
// in-domain neighbour), the 26 "void target" masks V_d (bit i: voxel i is
// solid, its d-neighbour is void and inside the domain, and d's class has a
// positive threshold) and the 7 Philox-block masks B_b (voxels with more
// targets of block b's class than the ranks before b); words that still
// hold front voxels are marked for
// the next candidate list.  Phase 2: the non-empty (word, block) masks are
// listed in shared memory as entries and the chunk's (voxel, block) pairs --
// one Philox call each -- are numbered through them; lane L takes the L-th
// 32nd of that range and walks it with a cursor (a binary search for its
// first entry, then bit by bit, two pairs per iteration), so every lane draws
// the same number of blocks whatever the density of its own word; passing
// draws are buffered and claimed by full warps.
// ---------------------------------------------------------------------------
constexpr int kGrowThreads = 256;
constexpr int kGrowWarps = kGrowThreads / 32;
#ifndef QSGS_GROW_MIN_BLOCKS
#define QSGS_GROW_MIN_BLOCKS 3  // resident blocks per SM the register budget aims for
#endif
constexpr int kGrowEntries = 7 * 32 + 1;  // non-empty masks of a chunk, plus one spare
constexpr int kGrowWins = 256;            // deferred claims buffered per warp

struct GrowWarpSmem {
  uint4 V[32][7];                // per lane word, per block b: V_{4b..4b+3}
  uint4 E[kGrowEntries];         // non-empty (word, block) masks: {voxels that draw
                                 // the block, voxel index of bit 0, counter word
                                 // kGrowTag | b, claim tag lane << 8 | b << 5}
  uint16_t P[kGrowEntries + 1];  // number of the first pair of each entry
  uint32_t w[32];                // per lane: word index
  uint32_t win[kGrowWins];       // draws that passed a threshold: tag | bit | pass bits << 16
};
// Dynamic shared memory of a growth block (one GrowWarpSmem per warp).
constexpr size_t kGrowSmemBytes = sizeof(GrowWarpSmem) * kGrowWarps;

// Direction index of offset (dx, dy, dz), evaluated at compile time.
__host__ __device__ constexpr int dir_index(int dx, int dy, int dz) {
  int found = -1;
  for (int d = 0; d < 26; ++d)
    if (kDirs[d].dx == dx && kDirs[d].dy == dy && kDirs[d].dz == dz) found = d;
  return found;
}

// V masks of the three directions that land in row (y+DY, z+DZ).
// V masks of the three directions that land in row (y+DY, z+DZ); `front`
// collects every void neighbour, live class or not.
// Word xw of a row (x-1 / x+1 neighbour words in l / rr) as occupancy: pad
// bits solid; on the torus the x wrap is folded in -- voxel nx-1 (bit p of
// the last word) is the x-1 neighbour of voxel 0, and voxel 0 the x+1
// neighbour of voxel nx-1.
template <int DK>
__device__ __forceinline__ void row_words(const Geom& g, const uint32_t* __restrict__ row,
                                          uint32_t xw, uint32_t& c, uint32_t& l, uint32_t& rr) {
  c = __ldg(row + xw);
  if (xw == g.W - 1) c |= g.pad_mask;
  l = xw > 0 ? __ldg(row + xw - 1) : 0xFFFFFFFFu;
  rr = 0xFFFFFFFFu;
  if (xw + 1 < g.W) {
    rr = __ldg(row + xw + 1);
    if (xw + 1 == g.W - 1) rr |= g.pad_mask;
  }
  if (on_torus<DK>(g)) {
    const uint32_t p = (g.nx - 1) & 31u;
    if (xw == 0) l = (__ldg(row + g.W - 1) >> p) << 31;
    if (xw == g.W - 1) {
      const uint32_t first = __ldg(row) & 1u;
      if (p == 31) rr = first;
      else c = (c & ~(2u << p)) | (first << (p + 1));
    }
  }
}

// The masks of the three directions that land in row (y+DY, z+DZ), from the
// row's words around the voxel's word (c) as occupancy, its x-1 / x+1
// neighbour words in l / rr; `front` collects every void neighbour.
template <int DZ, int DY>
__device__ __forceinline__ void row_masks_from(uint32_t c, uint32_t l, uint32_t rr, uint32_t self,
                                               const uint32_t (&live)[3], uint32_t (&V)[28],
                                               uint32_t& front) {
  const uint32_t at_minus = (c << 1) | (l >> 31);  // bit i: voxel x-1 of this row
  const uint32_t at_plus = (c >> 1) | (rr << 31);  // bit i: voxel x+1 of this row
  constexpr int dm = dir_index(-1, DY, DZ), d0 = dir_index(0, DY, DZ), dp = dir_index(1, DY, DZ);
  const uint32_t vm = ~at_minus & self, vp = ~at_plus & self;
  front |= vm | vp;
  V[dm] = vm & live[dir_cls(dm)];
  if (d0 >= 0) {
    constexpr int d = d0 < 0 ? 26 : d0;
    const uint32_t v0 = ~c & self;
    front |= v0;
    V[d] = v0 & live[dir_cls(d < 26 ? d : 0)];
  }
  V[dp] = vp & live[dir_cls(dp)];
}

template <int DZ, int DY, int DK, bool kInterior = false>
__device__ __forceinline__ void row_masks(const Geom& g, const uint32_t* __restrict__ grid,
                                          uint32_t y, uint32_t z, uint32_t r, uint32_t xw,
                                          uint32_t self, const uint32_t (&live)[3],
                                          uint32_t (&V)[28], uint32_t& front) {
  int yy = (int)y + DY, zz = (int)z + DZ;
  if (on_torus<DK>(g)) {  // the torus: every row exists
    yy = yy < 0 ? yy + (int)g.ny : (yy >= (int)g.ny ? yy - (int)g.ny : yy);
    zz = zz < 0 ? zz + (int)g.nz : (zz >= (int)g.nz ? zz - (int)g.nz : zz);
  }
  uint32_t c = 0xFFFFFFFFu, l = 0xFFFFFFFFu, rr = 0xFFFFFFFFu;  // outside: solid
  if (kInterior || (yy >= 0 && yy < (int)g.ny && zz >= 0 && zz < (int)g.nz)) {
    const size_t ro = (size_t)((uint32_t)zz * g.ny + (uint32_t)yy) * g.W;
    row_words<DK>(g, grid + ro, xw, c, l, rr);
    if (has_blocked<DK>(g)) {  // cells of earlier phases are not void either
      uint32_t bc, bl, br;
      row_words<DK>(g, g.blocked + ro, xw, bc, bl, br);
      c |= bc;
      l |= bl;
      rr |= br;
    }
  }
  row_masks_from<DZ, DY>(c, l, rr, self, live, V, front);
}

// The same for an interacting phase (R13): besides the void targets, cells
// of earlier phases that may be entered -- in the packed grid of the
// direction's class and not yet this phase's -- are targets, and they make
// a voxel active; they need no live class (their grid holds only labels
// with a positive interaction probability for that class).
template <int DZ, int DY>
__device__ __forceinline__ void row_masks_inter(const Geom& g, const uint32_t* __restrict__ grid,
                                                uint32_t y, uint32_t z, uint32_t xw, uint32_t self,
                                                const uint32_t (&live)[3], uint32_t (&V)[28],
                                                uint32_t& front) {
  constexpr int dm = dir_index(-1, DY, DZ), d0 = dir_index(0, DY, DZ), dp = dir_index(1, DY, DZ);
  constexpr int cls_x = dir_cls(dm);                // class of the x-1 / x+1 directions
  constexpr int cls_0 = d0 >= 0 ? dir_cls(d0) : 0;  // class of the centre direction
  int yy = (int)y + DY, zz = (int)z + DZ;
  if (g.periodic) {
    yy = yy < 0 ? yy + (int)g.ny : (yy >= (int)g.ny ? yy - (int)g.ny : yy);
    zz = zz < 0 ? zz + (int)g.nz : (zz >= (int)g.nz ? zz - (int)g.nz : zz);
  }
  uint32_t c = 0xFFFFFFFFu, l = 0xFFFFFFFFu, rr = 0xFFFFFFFFu;  // outside: solid
  uint32_t exc = 0, exl = 0, exr = 0, e0c = 0;                   // outside: none
  const GeomInter& gi = static_cast<const GeomInter&>(g);  // the kind's own geometry
  if (yy >= 0 && yy < (int)g.ny && zz >= 0 && zz < (int)g.nz) {
    const size_t ro = (size_t)((uint32_t)zz * g.ny + (uint32_t)yy) * g.W;
    row_words<kInteract>(g, grid + ro, xw, c, l, rr);
    uint32_t a, b, e;
    row_words<kInteract>(g, gi.enter + (size_t)cls_x * g.nwords + ro, xw, a, b, e);
    exc = a & ~c;
    exl = b & ~l;
    exr = e & ~rr;
    if (d0 >= 0) {
      row_words<kInteract>(g, gi.enter + (size_t)cls_0 * g.nwords + ro, xw, a, b, e);
      e0c = a & ~c;
    }
    uint32_t bc, bl, br;  // cells of earlier phases are not void
    row_words<kInteract>(g, g.blocked + ro, xw, bc, bl, br);
    c |= bc;
    l |= bl;
    rr |= br;
  }
  const uint32_t vm = ~((c << 1) | (l >> 31)) & self, vp = ~((c >> 1) | (rr << 31)) & self;
  const uint32_t em = ((exc << 1) | (exl >> 31)) & self, ep = ((exc >> 1) | (exr << 31)) & self;
  front |= vm | vp | em | ep;
  V[dm] = (vm & live[cls_x]) | em;
  if (d0 >= 0) {
    constexpr int d = d0 < 0 ? 26 : d0;
    const uint32_t v0 = ~c & self, e0 = e0c & self;
    front |= v0 | e0;
    V[d] = (v0 & live[cls_0]) | e0;
  }
  V[dp] = (vp & live[cls_x]) | ep;
}

// R1, the growth draws: a voxel's targets (V bits) are drawn class by class
// in rank order -- faces from blocks 0-1, edges from 2-4, corners from 5-6;
// block B_c + k (B = 0, 2, 5) serves the class's targets of rank 4k .. 4k+3,
// word j the one of rank 4k + j.  A voxel thus draws block B_c + k iff it
// has more than 4k targets of class c.  The counts come bit-parallel over
// the word's 32 voxels from carry-save adders (sum = a ^ b ^ c, carry = the
// majority) on the direction masks of each class.
__device__ __forceinline__ void csa(uint32_t a, uint32_t b, uint32_t c, uint32_t& sum,
                                    uint32_t& carry) {
  sum = a ^ b ^ c;
  carry = (a & b) | (c & (a ^ b));
}

// Class of growth block b (faces 0-1, edges 2-4, corners 5-6), the first
// block and the first direction of class c, and its number of directions.
__host__ __device__ constexpr int block_class(int b) { return b < 2 ? 0 : (b < 5 ? 1 : 2); }
__host__ __device__ constexpr int class_first_block(int c) { return c == 0 ? 0 : (c == 1 ? 2 : 5); }
__host__ __device__ constexpr int class_first_dir(int c) { return c == 0 ? 0 : (c == 1 ? 6 : 18); }
__host__ __device__ constexpr int class_dirs(int c) { return c == 0 ? 6 : (c == 1 ? 12 : 8); }

__device__ __forceinline__ void growth_blocks(const uint32_t (&V)[28], uint32_t (&Bm)[7]) {
  // Faces (6): count = fo + 2 ft + 4 f4.
  uint32_t s1, c1, s2, c2, ft, f4;
  csa(V[0], V[1], V[2], s1, c1);
  csa(V[3], V[4], V[5], s2, c2);
  const uint32_t fo = s1 ^ s2, fk = s1 & s2;
  csa(c1, c2, fk, ft, f4);
  Bm[0] = fo | ft | f4;    // >= 1
  Bm[1] = f4 & (fo | ft);  // >= 5
  // Edges (12): count = eo + 2 et + 4 eq + 8 ee.
  uint32_t a1, b1, a2, b2, a3, b3, a4, b4, o1, k1, t1, m1, t2, m2, eq, ee;
  csa(V[6], V[7], V[8], a1, b1);
  csa(V[9], V[10], V[11], a2, b2);
  csa(V[12], V[13], V[14], a3, b3);
  csa(V[15], V[16], V[17], a4, b4);
  csa(a1, a2, a3, o1, k1);
  const uint32_t eo = o1 ^ a4, k2 = o1 & a4;
  csa(b1, b2, b3, t1, m1);
  csa(b4, k1, k2, t2, m2);
  const uint32_t et = t1 ^ t2, m3 = t1 & t2;
  csa(m1, m2, m3, eq, ee);
  Bm[2] = eo | et | eq | ee;   // >= 1
  Bm[3] = ee | (eq & (eo | et));  // >= 5
  Bm[4] = ee & (eo | et | eq);    // >= 9
  // Corners (8): count = co + 2 ct + 4 cq + 8 ce.
  uint32_t p1, q1, p2, q2, o2, k3, u1, n1;
  csa(V[18], V[19], V[20], p1, q1);
  csa(V[21], V[22], V[23], p2, q2);
  csa(p1, p2, V[24], o2, k3);
  const uint32_t co = o2 ^ V[25], k4 = o2 & V[25];
  csa(q1, q2, k3, u1, n1);
  const uint32_t ct = u1 ^ k4, n2 = u1 & k4;
  const uint32_t cq = n1 ^ n2, ce = n1 & n2;
  Bm[5] = co | ct | cq | ce;      // >= 1
  Bm[6] = ce | (cq & (co | ct));  // >= 5
}

// The targets of class c of voxel i of a lane word, as a mask over the
// class's directions in order (bit k: direction class_first_dir(c) + k), from
// the word's direction masks (Vw[b] holds V[4b .. 4b+3]).
__device__ __forceinline__ uint32_t vbit(uint32_t v, uint32_t i) { return (v >> i) & 1u; }
__device__ __forceinline__ uint32_t class_targets(const uint4* Vw, uint32_t i, int c) {
  if (c == 0) {  // faces: V[0..5]
    const uint4 a = Vw[0], b = Vw[1];
    return vbit(a.x, i) | vbit(a.y, i) << 1 | vbit(a.z, i) << 2 | vbit(a.w, i) << 3 |
           vbit(b.x, i) << 4 | vbit(b.y, i) << 5;
  }
  if (c == 1) {  // edges: V[6..17]
    const uint4 a = Vw[1], b = Vw[2], e = Vw[3], f = Vw[4];
    return vbit(a.z, i) | vbit(a.w, i) << 1 | vbit(b.x, i) << 2 | vbit(b.y, i) << 3 |
           vbit(b.z, i) << 4 | vbit(b.w, i) << 5 | vbit(e.x, i) << 6 | vbit(e.y, i) << 7 |
           vbit(e.z, i) << 8 | vbit(e.w, i) << 9 | vbit(f.x, i) << 10 | vbit(f.y, i) << 11;
  }
  const uint4 a = Vw[4], b = Vw[5], e = Vw[6];  // corners: V[18..25]
  return vbit(a.z, i) | vbit(a.w, i) << 1 | vbit(b.x, i) << 2 | vbit(b.y, i) << 3 |
         vbit(b.z, i) << 4 | vbit(b.w, i) << 5 | vbit(e.x, i) << 6 | vbit(e.y, i) << 7;
}


// Position of the r-th (from 0) set bit of m (r < popc(m)).
__device__ __forceinline__ uint32_t nth_bit(uint32_t m, uint32_t r) {
  for (uint32_t k = 0; k < r; ++k) m &= m - 1;
  return (uint32_t)(__ffs(m) - 1);
}

struct GrowCounters {
  uint32_t draws, front;  // Philox blocks drawn (= attempts with a live void target), |A_t|
};

// Per-direction thresholds of one instance as T - 1 (a draw succeeds iff
// r <= T - 1), grouped by Philox block, and the mask of live directions
// (classes with T > 0).  Written by lanes 0..27 of a warp or block.
// kComplement stores ~(T - 1) instead: r + ~(T - 1) carries out of 32 bits
// exactly when r > T - 1, which fail_bits below reads off the carry flag.
template <bool kComplement = false>
__device__ __forceinline__ void load_thresholds(const RunState* st, uint32_t lane, uint4* thr) {
  if (lane < 28) {  // word j = lane & 3 of block b = lane >> 2: a target of rank r of class c
    const int b = (int)lane >> 2, c = block_class(b);
    const int r = 4 * (b - class_first_block(c)) + ((int)lane & 3);
    const unsigned long long T = r < class_dirs(c) ? st->thr[c] : 0ull;
    const uint32_t t1 = T ? (uint32_t)(T - 1) : 0u;  // dead: never tested
    reinterpret_cast<uint32_t*>(thr)[lane] = kComplement ? ~t1 : t1;
  }
}

// Interacting phases (R13): per direction the larger of the Eq. 1 threshold
// and the largest threshold of entering an earlier phase's cell along its
// class, complemented; the draw loop tests against it and the claims apply
// the target's own threshold.
// Eight entries: thr[7] = the Eq. 1 thresholds T - 1 of the three classes
// themselves (not complemented), for the claims.
__device__ __forceinline__ void load_thresholds_inter(const RunState* st, const GeomInter& g,
                                                      uint32_t lane, uint4* thr) {
  if (lane < 28) {  // word j = lane & 3 of block b = lane >> 2: a target of rank r of class c
    const int b = (int)lane >> 2, c = block_class(b);
    const bool real = 4 * (b - class_first_block(c)) + ((int)lane & 3) < class_dirs(c);
    const unsigned long long T = real ? st->thr[c] : 0ull;
    uint32_t t1 = T ? (uint32_t)(T - 1) : 0u;  // dead: never tested
    if (real) t1 = max(t1, g.enter_thr[c]);  // row 0: the largest per class
    reinterpret_cast<uint32_t*>(thr)[lane] = ~t1;
  } else if (lane < 31) {
    const unsigned long long T = st->thr[lane - 28];
    reinterpret_cast<uint32_t*>(thr)[lane] = T ? (uint32_t)(T - 1) : 0u;
  }
}

__device__ __forceinline__ uint32_t live_directions(const RunState* st) {
  uint32_t live_dirs = 0;
#pragma unroll
  for (int d = 0; d < 26; ++d)
    if (st->thr[dir_cls(d)] != 0) live_dirs |= 1u << d;
  return live_dirs;
}

// Word and bit of the d-neighbour of bit i of word w (in the domain, or on
// the torus).
template <int DK>
__device__ __forceinline__ void claim_target(const Geom& g, uint32_t w, uint32_t i, int d,
                                             uint32_t& wq, uint32_t& bit) {
  if (!on_torus<DK>(g)) {
    const int xi = (int)i + dir_dx(d);  // -1 .. 32: target bit, word carry
    wq = (uint32_t)((int)w + (dir_dy(d) + (int)g.ny * dir_dz(d)) * (int)g.W + (xi >> 5));
    bit = 1u << (xi & 31);
    return;
  }
  const uint32_t r = fast_div(w, g.div_W);
  const uint32_t z = fast_div(r, g.div_ny);
  const int y = (int)(r - z * g.ny) + dir_dy(d);
  const int zz = (int)z + dir_dz(d);
  const int x = (int)((w - r * g.W) * 32u + i) + dir_dx(d);
  const uint32_t xq = x < 0 ? g.nx - 1 : (x >= (int)g.nx ? 0u : (uint32_t)x);
  const uint32_t yq = y < 0 ? g.ny - 1 : (y >= (int)g.ny ? 0u : (uint32_t)y);
  const uint32_t zq = zz < 0 ? g.nz - 1 : (zz >= (int)g.nz ? 0u : (uint32_t)zz);
  wq = (zq * g.ny + yq) * g.W + (xq >> 5);
  bit = 1u << (xq & 31u);
}

// Claims of buffered draws: a draw's direction j wins when it passed its
// threshold and its target is a void in-domain neighbour (bit i of V_{4b+j}).
// Every claim also sets its word's touched bit, so that the commit's sparse
// path visits only marked and touched words.  (Setting it only in steps
// whose commit is sparse measured 1 % slower.)
__device__ __forceinline__ void claim(uint32_t* claims, uint32_t* touched, uint32_t wq,
                                      uint32_t bit) {
  // Fire-and-forget: the claim grid collects New_t; nobody waits.
  atomicOr(claims + wq, bit);
  atomicOr(touched + (wq >> 5), 1u << (wq & 31u));
}

// The claims of one buffered draw x (tag | bit | pass bits << 16).
template <int DK>
__device__ __forceinline__ void claim_entry(const Geom& g, uint32_t* claims, uint32_t* touched,
                                            const GrowWarpSmem& S, uint32_t x) {
  const uint32_t owner = (x >> 8) & 31u, b = (x >> 5) & 7u, i = x & 31u;
  // Word j of block b is the voxel's target of rank r0 + j of class c.
  const int c = block_class((int)b);
  const uint32_t r0 = 4u * (b - (uint32_t)class_first_block(c));
  const uint32_t m = class_targets(S.V[owner], i, c);
  const uint32_t n = (uint32_t)__popc(m);
  uint32_t win = n > r0 ? (x >> 16) & ((1u << min(4u, n - r0)) - 1u) : 0u;
  const uint32_t wo = S.w[owner];
  while (win) {
    const uint32_t j = __ffs(win) - 1;
    win &= win - 1;
    const int d = class_first_dir(c) + (int)nth_bit(m, r0 + j);
    uint32_t wq, bit;
    claim_target<DK>(g, wo, i, d, wq, bit);
    claim(claims, touched, wq, bit);
  }
}

template <int DK>
__device__ __forceinline__ void claim_wins(const Geom& g, uint32_t* claims, uint32_t* touched,
                                           const GrowWarpSmem& S, uint32_t nwin, uint32_t lane) {
  for (uint32_t k = lane; k < nwin; k += 32) claim_entry<DK>(g, claims, touched, S, S.win[k]);
}

// Claims of an interacting phase (R13).  The draw loop tested a block's
// words against the larger of the Eq. 1 and the largest interaction
// threshold of their class, so the block is drawn again here (a few per
// cent of the pairs) and each candidate direction is tested against its own
// target's threshold: Eq. 1 for a void cell, I^{n,m} for a cell of phase m.
template <int DK>
__device__ __forceinline__ void claim_entry_inter(const Geom& g, uint32_t* claims,
                                                  uint32_t* touched, const GrowWarpSmem& S,
                                                  uint32_t x, uint32_t t, const PhiloxKeys& keys,
                                                  const uint4* nthr) {
  const GeomInter& gi = static_cast<const GeomInter&>(g);  // the kind's own geometry
  const uint4 eq1 = nthr[7];  // Eq. 1 thresholds T - 1 per class (load_thresholds_inter)
  const uint32_t owner = (x >> 8) & 31u, b = (x >> 5) & 7u, i = x & 31u;
  // Word j of block b is the voxel's target of rank r0 + j of class c.
  const int cb = block_class((int)b);
  const uint32_t r0 = 4u * (b - (uint32_t)class_first_block(cb));
  const uint32_t m = class_targets(S.V[owner], i, cb);
  const uint32_t n = (uint32_t)__popc(m);
  uint32_t win = n > r0 ? (x >> 16) & ((1u << min(4u, n - r0)) - 1u) : 0u;
  if (!win) return;
  const uint32_t wo = S.w[owner];
  const uint32_t ro = fast_div(wo, g.div_W);
  const uint32_t v = ro * g.nx + (wo - ro * g.W) * 32u + i;
  const U4 rnd = philox4x32_10(U4{v, 0u, t, kGrowTag | b}, keys);
  while (win) {
    const uint32_t j = __ffs(win) - 1;
    win &= win - 1;
    const int d = class_first_dir(cb) + (int)nth_bit(m, r0 + j);
    uint32_t wq, bit;
    claim_target<DK>(g, wo, i, d, wq, bit);
    const uint32_t rq = fast_div(wq, g.div_W);
    const uint32_t q = rq * g.nx + (wq - rq * g.W) * 32u + (uint32_t)(__ffs(bit) - 1);
    const uint32_t lab = gi.labels[q];
    const int c = dir_cls(d);
    const uint32_t th = lab ? gi.enter_thr[lab * 3u + (uint32_t)c]
                            : (c == 0 ? eq1.x : (c == 1 ? eq1.y : eq1.z));
    if (u4_word(rnd, (int)j) <= th) claim(claims, touched, wq, bit);
  }
}

template <int DK>
__device__ __forceinline__ void claim_wins_inter(const Geom& g, uint32_t* claims,
                                                 uint32_t* touched, const GrowWarpSmem& S,
                                                 uint32_t nwin,
                                                 uint32_t lane, uint32_t t,
                                                 const PhiloxKeys& keys, const uint4* nthr) {
  for (uint32_t k = lane; k < nwin; k += 32)
    claim_entry_inter<DK>(g, claims, touched, S, S.win[k], t, keys, nthr);
}

// Bit-parallel over the 32 voxels of word w: the 26 void-target masks V_d
// (V[26], V[27] zero), the 7 Philox-block masks and the front bits; also the
// word's row r and word-in-row xw.
template <int DK>
__device__ __forceinline__ void word_masks(const Geom& g, const uint32_t* __restrict__ grid,
                                           uint32_t w, uint32_t live_dirs, uint32_t (&V)[28],
                                           uint32_t (&Bm)[7], uint32_t& front, uint32_t& r,
                                           uint32_t& xw) {  // declared before FrontCountPolicy
  const uint32_t self = __ldg(grid + w);
  r = fast_div(w, g.div_W);
  xw = w - r * g.W;
  const uint32_t z = fast_div(r, g.div_ny);
  const uint32_t y = r - z * g.ny;
  // Per class: all ones if its threshold is positive (live), else zero.
  const uint32_t live[3] = {0u - (live_dirs & 1u), 0u - ((live_dirs >> 6) & 1u),
                            0u - ((live_dirs >> 18) & 1u)};
  if constexpr (DK == kInteract) {
    row_masks_inter<-1, -1>(g, grid, y, z, xw, self, live, V, front);
    row_masks_inter<-1, 0>(g, grid, y, z, xw, self, live, V, front);
    row_masks_inter<-1, 1>(g, grid, y, z, xw, self, live, V, front);
    row_masks_inter<0, -1>(g, grid, y, z, xw, self, live, V, front);
    row_masks_inter<0, 0>(g, grid, y, z, xw, self, live, V, front);
    row_masks_inter<0, 1>(g, grid, y, z, xw, self, live, V, front);
    row_masks_inter<1, -1>(g, grid, y, z, xw, self, live, V, front);
    row_masks_inter<1, 0>(g, grid, y, z, xw, self, live, V, front);
    row_masks_inter<1, 1>(g, grid, y, z, xw, self, live, V, front);
  } else if (DK == kOpen && y >= 1 && y + 1 < g.ny && z >= 1 && z + 1 < g.nz) {
    // On the open domain, words whose nine neighbour rows all lie inside the
    // grid (almost all of them) take a copy without the per-row bounds tests
    // and branches (4 % of the 400^3 growth time).  The torus and run-time
    // kinds keep one copy: there the second one costs more in register
    // spills than it saves.
    row_masks<-1, -1, DK, true>(g, grid, y, z, r, xw, self, live, V, front);
    row_masks<-1, 0, DK, true>(g, grid, y, z, r, xw, self, live, V, front);
    row_masks<-1, 1, DK, true>(g, grid, y, z, r, xw, self, live, V, front);
    row_masks<0, -1, DK, true>(g, grid, y, z, r, xw, self, live, V, front);
    row_masks<0, 0, DK, true>(g, grid, y, z, r, xw, self, live, V, front);
    row_masks<0, 1, DK, true>(g, grid, y, z, r, xw, self, live, V, front);
    row_masks<1, -1, DK, true>(g, grid, y, z, r, xw, self, live, V, front);
    row_masks<1, 0, DK, true>(g, grid, y, z, r, xw, self, live, V, front);
    row_masks<1, 1, DK, true>(g, grid, y, z, r, xw, self, live, V, front);
  } else {
    row_masks<-1, -1, DK>(g, grid, y, z, r, xw, self, live, V, front);
    row_masks<-1, 0, DK>(g, grid, y, z, r, xw, self, live, V, front);
    row_masks<-1, 1, DK>(g, grid, y, z, r, xw, self, live, V, front);
    row_masks<0, -1, DK>(g, grid, y, z, r, xw, self, live, V, front);
    row_masks<0, 0, DK>(g, grid, y, z, r, xw, self, live, V, front);
    row_masks<0, 1, DK>(g, grid, y, z, r, xw, self, live, V, front);
    row_masks<1, -1, DK>(g, grid, y, z, r, xw, self, live, V, front);
    row_masks<1, 0, DK>(g, grid, y, z, r, xw, self, live, V, front);
    row_masks<1, 1, DK>(g, grid, y, z, r, xw, self, live, V, front);
  }
  V[26] = 0;
  V[27] = 0;
  growth_blocks(V, Bm);
}

// Bit j set: word j of r fails its threshold (r_j > T_j - 1), for the four
// words of a Philox block against the complemented thresholds nthr_j =
// ~(T_j - 1): the carry out of r_j + nthr_j, shifted in word by word (w
// first, so that x lands in bit 0).  Eight integer adds, no compare/select.
__device__ __forceinline__ uint32_t fail_bits(const U4& r, const uint4& nthr) {
  uint32_t acc;
  asm("{\n\t.reg .u32 s;\n\t"
      "add.cc.u32 s, %1, %2;\n\t"
      "addc.u32 %0, %9, %9;\n\t"
      "add.cc.u32 s, %3, %4;\n\t"
      "addc.u32 %0, %0, %0;\n\t"
      "add.cc.u32 s, %5, %6;\n\t"
      "addc.u32 %0, %0, %0;\n\t"
      "add.cc.u32 s, %7, %8;\n\t"
      "addc.u32 %0, %0, %0;\n\t}"
      : "=&r"(acc)
      : "r"(r.w), "r"(nthr.w), "r"(r.z), "r"(nthr.z), "r"(r.y), "r"(nthr.y), "r"(r.x),
        "r"(nthr.x), "r"(0u));
  return acc;
}

// Index of the highest set bit of m (0xFFFFFFFF for m = 0) and 1 << i
// (0 for i > 31): the PTX bfind and shl semantics, so that an exhausted mask
// needs no test.
__device__ __forceinline__ uint32_t top_bit(uint32_t m) {
  uint32_t i;
  asm("bfind.u32 %0, %1;" : "=r"(i) : "r"(m));
  return i;
}

__device__ __forceinline__ uint32_t bit_at(uint32_t i) {
  uint32_t b;
  asm("shl.b32 %0, %1, %2;" : "=r"(b) : "r"(1u), "r"(i));
  return b;
}

// One warp, one chunk of up to 32 candidate words (w = 0xFFFFFFFF: no word
// for this lane).  All 32 lanes must call it together.
template <int DK>
__device__ __forceinline__ void grow_chunk(const Geom& g, const uint32_t* __restrict__ grid,
                                           uint32_t* claims, uint32_t* other, uint32_t* mark,
                                           uint32_t w, uint32_t t, uint32_t live_dirs,
                                           const uint4* nthr,
                                           const PhiloxKeys& keys, GrowWarpSmem& S,
                                           GrowCounters& cnt) {
  const uint32_t lane = threadIdx.x & 31;
  uint32_t* touched = mark + bitmap_words(g);
  // Phase 1: masks of this lane's word.
  uint32_t Bm[7] = {0, 0, 0, 0, 0, 0, 0};
  uint32_t v0 = 0;
  if (w != 0xFFFFFFFFu) {
    uint32_t V[28], front = 0, r, xw;
    word_masks<DK>(g, grid, w, live_dirs, V, Bm, front, r, xw);
    cnt.front += __popc(front);
    // A word holding front voxels now may hold some after the step too.
    if (front) atomicOr(mark + (w >> 5), 1u << (w & 31));
    // The other claim grid takes the next step's claims.  Its only non-zero
    // words hold the previous step's claims (already in the grid), and
    // every word claimed then is on this step's list: clearing listed words
    // leaves it all zero for the next step.
    other[w] = 0;
#pragma unroll
    for (int b = 0; b < 7; ++b) S.V[lane][b] = make_uint4(V[4 * b], V[4 * b + 1], V[4 * b + 2], V[4 * b + 3]);
    S.w[lane] = w;
    v0 = r * g.nx + xw * 32u;
  }
  // Phase 2.  Pairs and non-empty masks of the lanes, counted by one warp
  // scan (pairs in the low half-word: at most 7 * 32 * 32 = 7168).
  uint32_t items = 0, ents = 0;
#pragma unroll
  for (int b = 0; b < 7; ++b) {
    items += __popc(Bm[b]);
    ents += Bm[b] ? 1u : 0u;
  }
  const uint32_t mine = items | (ents << 16);
  uint32_t incl = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= (uint32_t)o) incl += y;
  }
  const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
  const uint32_t total = tot & 0xFFFFu, n_ent = tot >> 16;
  cnt.draws += total;  // one Philox block per pair; every pair has a live void target
  if (total == 0) return;  // warp-uniform
  {
    const uint32_t excl = incl - mine;
    uint32_t e = excl >> 16, p = excl & 0xFFFFu;
#pragma unroll
    for (int b = 0; b < 7; ++b) {
      if (Bm[b]) {
        S.E[e] = make_uint4(Bm[b], v0, kGrowTag | (uint32_t)b, (lane << 8) | ((uint32_t)b << 5));
        S.P[e] = (uint16_t)p;
        ++e;
        p += __popc(Bm[b]);
      }
    }
  }
  __syncwarp();
  // Lane L draws pairs [s, s + n): an even split of the chunk's total.  Pairs
  // are numbered entry by entry, highest voxel bit first within an entry.
  const uint32_t per = total >> 5, extra = total & 31u;
  const uint32_t n = per + (lane < extra ? 1u : 0u);
  const uint32_t s = lane * per + min(lane, extra);
  uint32_t k = 0;  // the last entry whose first pair is at or before s
#pragma unroll
  for (uint32_t step = 128; step; step >>= 1)
    if (k + step < n_ent && S.P[k + step] <= s) k += step;
  uint4 E = S.E[k];
  uint32_t m = E.x;
  for (uint32_t j = S.P[k]; j < s; ++j) m ^= bit_at(top_bit(m));  // pairs before s
  // Each lane draws two pairs per iteration (two independent Philox chains
  // in flight hide the multiply latency).  After a lane's pair empties the
  // cursor's mask the cursor moves to the next entry (index at most n_ent:
  // the spare entry is read, never used).  Draws that pass a threshold (a
  // few per cent) are buffered and claimed together, so the claim work runs
  // on full warps instead of one or two lanes of every iteration.  va / vb:
  // the lane has a pair left (always, but in the last iteration).
  const uint32_t full = per >> 1;  // iterations in which every lane has both pairs
  uint32_t nwin = 0;
  auto draw2 = [&](const bool va, const bool vb) {
    const uint32_t ia = top_bit(m);
    m ^= bit_at(ia);
    const uint32_t xa = E.y + ia, cwa = E.z, ta = E.w | ia;
    if (va && m == 0) {
      E = S.E[++k];
      m = E.x;
    }
    const uint32_t ib = top_bit(m);
    m ^= bit_at(ib);
    const uint32_t xb = E.y + ib, cwb = E.z, tb = E.w | ib;
    if (vb && m == 0) {
      E = S.E[++k];
      m = E.x;
    }
    const U4 ra = philox4x32_10(U4{xa, 0u, t, cwa}, keys);
    const U4 rb = philox4x32_10(U4{xb, 0u, t, cwb}, keys);
    const uint32_t pa = va ? fail_bits(ra, nthr[cwa & 7u]) ^ 0xFu : 0u;  // passing words
    const uint32_t pb = vb ? fail_bits(rb, nthr[cwb & 7u]) ^ 0xFu : 0u;
    const uint32_t lt = (1u << lane) - 1u;
    const uint32_t bala = __ballot_sync(0xffffffffu, pa != 0);
    const uint32_t balb = __ballot_sync(0xffffffffu, pb != 0);
    if (pa) S.win[nwin + __popc(bala & lt)] = ta | (pa << 16);
    nwin += __popc(bala);
    if (pb) S.win[nwin + __popc(balb & lt)] = tb | (pb << 16);
    nwin += __popc(balb);
    if (nwin > (uint32_t)kGrowWins - 64u) {
      __syncwarp();
      if constexpr (DK == kInteract)
        claim_wins_inter<DK>(g, claims, touched, S, nwin, lane, t, keys, nthr);
      else
        claim_wins<DK>(g, claims, touched, S, nwin, lane);
      __syncwarp();
      nwin = 0;
    }
  };
  for (uint32_t it = 0; it < full; ++it) draw2(true, true);
  if ((per & 1u) | extra) draw2(2u * full < n, 2u * full + 1u < n);
  __syncwarp();
  if constexpr (DK == kInteract)
    claim_wins_inter<DK>(g, claims, touched, S, nwin, lane, t, keys, nthr);
  else
    claim_wins<DK>(g, claims, touched, S, nwin, lane);
  __syncwarp();  // S.E, S.P, S.V and S.win are rewritten by the next chunk
}

// `draws` is warp-uniform (a chunk total); `front` is per lane.  live is
// the number of Philox blocks drawn: zero exactly when no pair had a void
// target with a positive threshold (the stall test).
__device__ __forceinline__ void flush_counters(RunState* st, GrowCounters& c) {
  const uint32_t wf = __reduce_add_sync(0xffffffffu, c.front);
  if ((threadIdx.x & 31) == 0) {
    if (c.draws) {
      atomicAdd(&st->live, (unsigned long long)c.draws);
      atomicAdd(&st->sum_draws, (unsigned long long)c.draws);
    }
    if (wf) atomicAdd(&st->front_acc, (unsigned long long)wf);
  }
  c = GrowCounters{0, 0};
}

// Chunk dispenser of the growth kernels: a warp's first tile (of `tile`
// consecutive 32-word chunks) is its global warp index, later ones come from
// an atomic counter, so warps that drew cheap tiles take more.  The last block to finish puts the counters back
// to zero, which leaves every launch (a graph replay included) starting
// from a clean dispenser.
__device__ __forceinline__ uint32_t next_chunk(uint32_t* next, uint32_t nwarps) {
  uint32_t c = 0;
  if ((threadIdx.x & 31) == 0) c = atomicAdd(next, 1u) + nwarps;
  return __shfl_sync(0xffffffffu, c, 0);
}

__device__ __forceinline__ void finish_dispenser(uint32_t* next, uint32_t* done) {
  __syncthreads();  // every warp of the block has taken its last chunk
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(done, 1u) == gridDim.x - 1) {
      *next = 0;
      *done = 0;
    }
  }
}

// The kernel-parameter geometry of a kind: GeomInter for interacting phases.
template <int DK>
struct GeomOf {
  using type = Geom;
};
template <>
struct GeomOf<kInteract> {
  using type = GeomInter;
};

template <int DK>
__global__ void __launch_bounds__(kGrowThreads, QSGS_GROW_MIN_BLOCKS)
    k_grow(typename GeomOf<DK>::type g, const uint32_t* __restrict__ cand,
           const uint32_t* __restrict__ grid,
           uint32_t* aux, uint32_t* mark, RunState* st, const PhiloxKeys keys, uint32_t tile) {
  extern __shared__ uint4 grow_smem_[];
  GrowWarpSmem* smem = reinterpret_cast<GrowWarpSmem*>(grow_smem_);
  // Seven Philox blocks, and an eighth row: kInteract's Eq. 1 slot, else
  // padding, so that every index (b & 7) a cursor may form is in the array.
  __shared__ uint4 s_thr[8];
  if (!st->active) return;
  const uint32_t n = st->front_words;
  const uint32_t t = st->t;
  const uint32_t live_dirs = live_directions(st);
  if constexpr (DK == kInteract)
    load_thresholds_inter(st, g, threadIdx.x, s_thr);
  else
    load_thresholds<true>(st, threadIdx.x, s_thr);  // complemented, for fail_bits
  __syncthreads();
  uint32_t* claims = aux + (size_t)(t & 1u) * g.nwords;  // this step's claim grid
  uint32_t* other = aux + (size_t)((t & 1u) ^ 1u) * g.nwords;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t nwarps = gridDim.x * kGrowWarps;
  const uint32_t nchunks = (n + 31) / 32;
  const uint32_t ntiles = (nchunks + tile - 1) / tile;
  GrowCounters cnt{0, 0};
  auto entry = [&](uint32_t c) -> uint32_t {
    const uint32_t idx = c * 32u + lane;
    const uint32_t w = idx < n ? cand[idx] : 0xFFFFFFFFu;
    return w < g.nwords ? w : 0xFFFFFFFFu;  // >= nwords only after a timed-out scan (reported)
  };
  for (uint32_t ti = blockIdx.x * kGrowWarps + warp; ti < ntiles;
       ti = next_chunk(&st->grow_next, nwarps)) {
    const uint32_t c_end = min(ti * tile + tile, nchunks);
    for (uint32_t c = ti * tile; c < c_end; ++c)
      grow_chunk<DK>(g, grid, claims, other, mark, entry(c), t, live_dirs, s_thr, keys,
                     smem[warp], cnt);
  }
  flush_counters(st, cnt);
  finish_dispenser(&st->grow_next, &st->grow_done);
}

// ---------------------------------------------------------------------------
// Comparator: the full-field sweep of Algorithm 2 (Sec. 2.2) with the same
// keyed draws.  Every voxel draws every Philox block each step -- the cost
// model of the vectorized procedure, which generates a random field per
// direction over the whole grid -- and the successes are claimed exactly as
// in the list-driven step, so the result is the same bit for bit (the
// oracle pins Algorithm 2 == Algorithm 3).  A thread takes one word, a warp
// 32 consecutive words.  Counters: |A_t| and the live pairs as in k_grow;
// sum_draws counts every block drawn.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
    k_grow_fullfield(Geom g, const uint32_t* __restrict__ grid, uint32_t* aux, uint32_t* mark,
                     RunState* st, const PhiloxKeys keys) {
  __shared__ uint4 s_thr[7];
  if (!st->active) return;
  const uint32_t t = st->t;
  const uint32_t live_dirs = live_directions(st);
  load_thresholds(st, threadIdx.x, s_thr);
  __syncthreads();
  uint32_t* claims = aux + (size_t)(t & 1u) * g.nwords;
  uint32_t* other = aux + (size_t)((t & 1u) ^ 1u) * g.nwords;  // cleared as in k_grow
  uint32_t* touched = mark + bitmap_words(g);
  const uint32_t stride = gridDim.x * blockDim.x;
  const uint32_t rounds = (g.nwords + stride - 1) / stride;  // uniform: every lane loops alike
  uint32_t front_n = 0, live_n = 0;
  unsigned long long drawn = 0;
  for (uint32_t k = 0; k < rounds; ++k) {
    const uint32_t w = k * stride + blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= g.nwords) continue;
    uint32_t V[28], Bm[7] = {0, 0, 0, 0, 0, 0, 0}, front = 0, r, xw;
    word_masks<kRuntime>(g, grid, w, live_dirs, V, Bm, front, r, xw);
    front_n += __popc(front);
    if (front) atomicOr(mark + (w >> 5), 1u << (w & 31));
    other[w] = 0;
    const uint32_t x0 = xw * 32u;
    const uint32_t len = min(32u, g.nx - x0);
    const uint32_t v0 = r * g.nx + x0;
#pragma unroll
    for (int b = 0; b < 7; ++b) live_n += __popc(Bm[b]);
    for (uint32_t i = 0; i < len; ++i) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        // The voxel's targets of class c (bit k: direction class_first_dir(c)
        // + k); word j of block class_first_block(c) + kb is the one of rank
        // 4 kb + j.
        uint32_t m = 0;
#pragma unroll
        for (int k = 0; k < class_dirs(c); ++k) m |= ((V[class_first_dir(c) + k] >> i) & 1u) << k;
        const uint32_t n = (uint32_t)__popc(m);
#pragma unroll
        for (int kb = 0; kb < (class_dirs(c) + 3) / 4; ++kb) {
          const int b = class_first_block(c) + kb;
          const uint4 th = s_thr[b];
          const U4 rnd = philox4x32_10(U4{v0 + i, 0u, t, kGrowTag | (uint32_t)b}, keys);
          uint32_t win = (rnd.x <= th.x ? 1u : 0u) | (rnd.y <= th.y ? 2u : 0u) |
                         (rnd.z <= th.z ? 4u : 0u) | (rnd.w <= th.w ? 8u : 0u);
          const uint32_t r0 = 4u * (uint32_t)kb;
          win = n > r0 ? win & ((1u << min(4u, n - r0)) - 1u) : 0u;
          while (win) {
            const uint32_t j = __ffs(win) - 1;
            win &= win - 1;
            uint32_t wq, bit;
            claim_target<kRuntime>(g, w, i, class_first_dir(c) + (int)nth_bit(m, r0 + j), wq,
                                   bit);
            claim(claims, touched, wq, bit);
          }
        }
      }
    }
    drawn += 7ull * len;
  }
  const uint32_t wf = __reduce_add_sync(0xffffffffu, front_n);
  const uint32_t wl = __reduce_add_sync(0xffffffffu, live_n);
  unsigned long long wd = drawn;
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) wd += __shfl_xor_sync(0xffffffffu, wd, o);
  if ((threadIdx.x & 31) == 0) {
    if (wl) atomicAdd(&st->live, (unsigned long long)wl);
    if (wd) atomicAdd(&st->sum_draws, wd);
    if (wf) atomicAdd(&st->front_acc, (unsigned long long)wf);
  }
}

}  // namespace qsgs

#include "qsgs_batch.cuh"

namespace qsgs {

// ---------------------------------------------------------------------------
// Philox throughput probe: every thread draws `per_thread` blocks with
// distinct counters and folds them into one word, so nothing is optimised
// away.  Its rate is the ALU ceiling the growth kernel is compared with.
// ---------------------------------------------------------------------------
#ifndef QSGS_PROBE_ILP
#define QSGS_PROBE_ILP 2  // independent blocks in flight per thread
#endif
__global__ void __launch_bounds__(256) k_philox_rate(PhiloxKeys keys, uint32_t per_thread,
                                                     unsigned long long* out) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t acc[QSGS_PROBE_ILP];
#pragma unroll
  for (int j = 0; j < QSGS_PROBE_ILP; ++j) acc[j] = 0;
  for (uint32_t k = 0; k < per_thread; k += QSGS_PROBE_ILP) {
#pragma unroll
    for (int j = 0; j < QSGS_PROBE_ILP; ++j) {
      const U4 r = philox4x32_10(U4{tid, 0u, k + j, kGrowTag}, keys);
      acc[j] ^= r.x ^ r.y ^ r.z ^ r.w;
    }
  }
  uint32_t a = 0;
#pragma unroll
  for (int j = 0; j < QSGS_PROBE_ILP; ++j) a ^= acc[j];
  const uint32_t wsum = __reduce_add_sync(0xffffffffu, a & 0xFFFFu);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, (unsigned long long)wsum);
}

cudaError_t launch_philox_rate(uint64_t seed, uint32_t blocks, uint32_t per_thread,
                               unsigned long long* out, cudaStream_t s) {
  k_philox_rate<<<blocks, 256, 0, s>>>(make_philox_keys(seed), per_thread, out);
  return cudaGetLastError();
}

static int num_sms();

// ---------------------------------------------------------------------------
// L2 probes: the roof the growth step's gathers and claims would hit if the
// L2 bound it.  k_l2_read streams an L2-resident buffer `passes` times with
// 16-byte loads that bypass L1 (ld.global.cg), each pass starting every
// thread at a different 16-byte element so no SM re-reads its own lines;
// k_l2_red issues fire-and-forget atomicOr (reductions without a return
// value, the claims' kind) to scattered words of an L2-resident buffer.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(512) k_l2_read(const uint4* __restrict__ buf, uint32_t n16,
                                                 uint32_t passes, unsigned long long* out) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t nthreads = gridDim.x * blockDim.x;
  uint32_t acc = 0;
  for (uint32_t p = 0; p < passes; ++p) {
    // Pass p shifts every thread by p * 4099 elements (mod n16): the
    // elements a thread reads change from pass to pass.
    uint32_t i = (uint32_t)(((unsigned long long)tid + (unsigned long long)p * 4099u) % n16);
    uint32_t k = tid;
    // Four independent loads per iteration keep enough bytes in flight.  The
    // launcher guarantees n16 >= 4 * nthreads, so i stays below n16 with one
    // conditional subtraction per step.
    for (; k + 3u * nthreads < n16; k += 4u * nthreads) {
      uint32_t i1 = i + nthreads, i2 = i + 2u * nthreads, i3 = i + 3u * nthreads;
      i1 = i1 >= n16 ? i1 - n16 : i1;
      i2 = i2 >= n16 ? i2 - n16 : i2;
      i3 = i3 >= n16 ? i3 - n16 : i3;
      const uint4 a = __ldcg(buf + i), b = __ldcg(buf + i1), c = __ldcg(buf + i2),
                  d = __ldcg(buf + i3);
      acc ^= a.x ^ a.y ^ a.z ^ a.w ^ b.x ^ b.y ^ b.z ^ b.w ^ c.x ^ c.y ^ c.z ^ c.w ^ d.x ^ d.y ^
             d.z ^ d.w;
      i += 4u * nthreads;
      i = i >= n16 ? i - n16 : i;
    }
    for (; k < n16; k += nthreads) {
      const uint4 a = __ldcg(buf + i);
      acc ^= a.x ^ a.y ^ a.z ^ a.w;
      i += nthreads;
      i = i >= n16 ? i - n16 : i;
    }
  }
  const uint32_t wsum = __reduce_add_sync(0xffffffffu, acc & 0xFFFFu);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, (unsigned long long)wsum);
}

__global__ void __launch_bounds__(512) k_l2_red(uint32_t* buf, uint32_t nwords,
                                                uint32_t per_thread) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  // A multiplicative walk over the words (odd stride: a permutation mod a
  // power of two, scattered otherwise): neighbouring lanes hit words far
  // apart, like claims into a large grid.
  uint32_t x = tid * 2654435761u;
  for (uint32_t k = 0; k < per_thread; ++k) {
    atomicOr(buf + (x % nwords), 1u << (k & 31u));
    x += 0x9E3779B9u;
  }
}

cudaError_t launch_l2_read(const void* buf, uint64_t n16, uint32_t passes,
                           unsigned long long* out, cudaStream_t s) {
  const uint32_t blocks = (uint32_t)num_sms() * 4u;
  k_l2_read<<<blocks, 512, 0, s>>>(static_cast<const uint4*>(buf), (uint32_t)n16, passes, out);
  return cudaGetLastError();
}

uint32_t l2_read_threads() { return (uint32_t)num_sms() * 4u * 512u; }

cudaError_t launch_l2_red(void* buf, uint64_t nwords, uint32_t per_thread, uint32_t blocks,
                          cudaStream_t s) {
  k_l2_red<<<blocks, 512, 0, s>>>(static_cast<uint32_t*>(buf), (uint32_t)nwords, per_thread);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Fetch: bit grid -> uint8 phase map (x fastest), 16 voxels per thread.
// ---------------------------------------------------------------------------
__global__ void k_unpack_u8(Geom g, const uint32_t* grid, uint8_t* out, unsigned long long vb,
                            unsigned long long ve) {
  // Voxels [vb, ve) of the grid into out[0 .. ve - vb).
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x * 16ull;
  for (unsigned long long v0 = vb + ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) * 16ull;
       v0 < ve; v0 += stride) {
    uint32_t r = fast_div((uint32_t)v0, g.div_nx);
    uint32_t x = (uint32_t)v0 - r * g.nx;
    uint8_t b[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      b[k] = 0;
      if (v0 + k < ve) b[k] = (uint8_t)((grid[(size_t)r * g.W + (x >> 5)] >> (x & 31)) & 1u);
      if (++x == g.nx) { x = 0; ++r; }
    }
    uint8_t* o = out + (v0 - vb);
    if (v0 + 16 <= ve && ((reinterpret_cast<uintptr_t>(o) & 15u) == 0)) {
      uint4 pk;
      pk.x = b[0] | (b[1] << 8) | (b[2] << 16) | ((uint32_t)b[3] << 24);
      pk.y = b[4] | (b[5] << 8) | (b[6] << 16) | ((uint32_t)b[7] << 24);
      pk.z = b[8] | (b[9] << 8) | (b[10] << 16) | ((uint32_t)b[11] << 24);
      pk.w = b[12] | (b[13] << 8) | (b[14] << 16) | ((uint32_t)b[15] << 24);
      *reinterpret_cast<uint4*>(o) = pk;
    } else {
      for (int k = 0; k < 16 && v0 + k < ve; ++k) o[k] = b[k];
    }
  }
}

// ---------------------------------------------------------------------------
// Phase maps (R12): the label of this phase into a uint8 map (other bytes
// untouched), and this phase's cells ORed into a packed blocked grid.
// ---------------------------------------------------------------------------
__global__ void k_label_u8(Geom g, const uint32_t* grid, uint8_t* out, uint8_t label) {
  for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < g.nwords;
       w += gridDim.x * blockDim.x) {
    uint32_t bits = grid[w];
    if (!bits) continue;
    const uint32_t r = fast_div(w, g.div_W);
    const uint32_t v0 = r * g.nx + (w - r * g.W) * 32u;
    while (bits) {
      const uint32_t i = __ffs(bits) - 1;
      bits &= bits - 1;
      out[v0 + i] = label;
    }
  }
}

__global__ void k_or_words(uint32_t n, const uint32_t* src, uint32_t* dst) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    if (src[i]) dst[i] |= src[i];
}

// ---------------------------------------------------------------------------
// Host launchers.
// ---------------------------------------------------------------------------
static int g_num_sms = 0;

static int num_sms() {
  if (g_num_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 1;
  }
  return g_num_sms;
}

static uint32_t scan_grid(uint64_t max_items) {
  const uint64_t tiles = (max_items + kScanTile - 1) / kScanTile;
  uint64_t blocks = (uint64_t)num_sms() * 4;
  if (blocks > tiles) blocks = tiles;
  return (uint32_t)(blocks ? blocks : 1);
}

static uint32_t side_sum_grid(uint64_t nwords) {
  const uint64_t need = (nwords + 255) / 256;
  const uint64_t cap = (uint64_t)num_sms() * 4;
  return (uint32_t)(need < cap ? (need ? need : 1) : cap);
}

static uint32_t seed_bits_grid(uint64_t nwords) {
  const uint64_t need = (nwords + 255) / 256;
  const uint64_t cap = (uint64_t)num_sms() * 8;  // 8 blocks of 256 threads per SM
  return (uint32_t)(need < cap ? (need ? need : 1) : cap);
}

static uint32_t commit_grid(uint64_t nwords) {
  constexpr uint64_t kTile = kCommitThreads * kCommitItems;
  const uint64_t tiles = (nwords + kTile - 1) / kTile;
  uint64_t blocks = (uint64_t)num_sms() * 3;
  if (blocks > tiles) blocks = tiles;
  return (uint32_t)(blocks ? blocks : 1);
}

static uint32_t batch_commit_grid(uint64_t max_words) {
  const uint64_t supers = (max_words / 32 + kBatchCommitGroups - 1) / kBatchCommitGroups;
  const uint64_t warps_needed = supers ? supers : 1;
  uint64_t blocks = (warps_needed + 7) / 8;
  const uint64_t cap = (uint64_t)num_sms() * 4;
  if (blocks > cap) blocks = cap;
  return (uint32_t)(blocks ? blocks : 1);
}

Geom make_geom(uint32_t nx, uint32_t ny, uint32_t nz, uint32_t periodic) {
  Geom g{};
  g.periodic = periodic ? 1u : 0u;
  g.blocked = nullptr;
  g.nx = nx;
  g.ny = ny;
  g.nz = nz;
  g.W = (nx + 31) / 32;
  g.nrows = ny * nz;
  g.nwords = g.W * g.nrows;
  g.n = nx * ny * nz;
  const uint32_t tail = nx - (g.W - 1) * 32;  // voxels in the last word
  g.pad_mask = tail == 32 ? 0u : ~((1u << tail) - 1u);
  g.div_nx = make_fastdiv(nx);
  g.div_ny = make_fastdiv(ny);
  g.div_W = make_fastdiv(g.W);
  return g;
}

// The geometry of an interacting phase's kernels: Geom plus the step
// buffers' interaction pointers.
GeomInter geom_inter(const Geom& g, const StepBuffers& b) {
  GeomInter gi{};
  static_cast<Geom&>(gi) = g;
  gi.enter = b.enter;
  gi.labels = b.labels;
  gi.enter_thr = b.enter_thr;
  return gi;
}

// Every launch goes through LAUNCH so that the tracer counts (and, when
// profiling, times) it.
#define QSGS_LAUNCH_SMEM(tr, cls, s, kernel, grid, block, smem, ...) \
  do {                                                               \
    cudaError_t e_ = (tr).before((cls), (s));                        \
    if (e_ != cudaSuccess) return e_;                                \
    kernel<<<(grid), (block), (smem), (s)>>>(__VA_ARGS__);           \
    e_ = cudaGetLastError();                                         \
    if (e_ != cudaSuccess) return e_;                                \
    e_ = (tr).after((s));                                            \
    if (e_ != cudaSuccess) return e_;                                \
  } while (0)
#define QSGS_LAUNCH(tr, cls, s, kernel, grid, block, ...) \
  QSGS_LAUNCH_SMEM(tr, cls, s, kernel, grid, block, 0, __VA_ARGS__)

// The growth kernels use more than the default 48 KB of shared memory; the
// opt-in is a per-device function attribute, set once per device before
// their first launch (handle creation does it, outside any stream capture).
cudaError_t prepare_kernels() {
  static bool done[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
  e = cudaFuncSetAttribute(k_grow<kOpen>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kGrowSmemBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_grow<kTorus>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kGrowSmemBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_grow<kRuntime>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kGrowSmemBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_grow<kInteract>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kGrowSmemBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_grow_batch<kOpen>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kGrowSmemBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_grow_batch<kRuntime>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kGrowSmemBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_spacing_rounds_csr, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kSpacingSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_grow<kOpen>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_grow<kTorus>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_grow<kRuntime>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_grow<kInteract>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_grow_batch<kOpen>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_grow_batch<kRuntime>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
  if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
  return e;
}

cudaError_t launch_init_state(RunState* st, const StateInit& init, cudaStream_t s, Tracer& tr) {
  QSGS_LAUNCH(tr, kClsSeed, s, k_init_state, 1, 1, st, init);
  return cudaSuccess;
}

cudaError_t launch_seed(const Geom& g, const SeedBuffers& b, uint32_t k0, uint32_t k1,
                        uint32_t spin_limit, cudaStream_t s, Tracer& tr) {
  ScanCtl ctl{b.st, b.scan_status, spin_limit};
  // Candidate bits into the empty grid, then the candidates (ascending) into
  // the list buffer.
  QSGS_LAUNCH(tr, kClsSeed, s, k_seed_bits, seed_bits_grid(g.nwords), 256, g, b.st, b.grid,
              make_philox_keys((uint64_t)k1 << 32 | k0));
  SeedCompactPolicy sp{g, b.st, b.grid, b.list, b.cand_cap};
  QSGS_LAUNCH(tr, kClsSeed, s, k_lookback_scan<SeedCompactPolicy>, scan_grid(g.nwords),
              kScanThreads, sp, ctl);
  const uint8_t* decision = nullptr;
  if (b.cg.s >= 2) {
    const CellGeom cg{b.cg.s, b.cg.ncx, b.cg.ncy, b.cg.ncz, g.periodic};
    const uint32_t ncells = cg.ncx * cg.ncy * cg.ncz;
    cudaError_t e = cudaMemsetAsync(b.cell_count, 0, (size_t)ncells * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    const uint32_t blocks = (uint32_t)num_sms() * 4;
    QSGS_LAUNCH(tr, kClsSeed, s, k_cell_count, blocks, 256, g, cg, b.st, b.list, b.cell_count);
    CellOffsetPolicy cp{b.st, ncells, b.cell_count, b.cell_start};
    QSGS_LAUNCH(tr, kClsSeed, s, k_lookback_scan<CellOffsetPolicy>, scan_grid(ncells),
                kScanThreads, cp, ctl);
    QSGS_LAUNCH(tr, kClsSeed, s, k_cell_fill, blocks, 256, g, cg, b.st, b.list, b.cell_count,
                b.cell_items, b.decision);
    QSGS_LAUNCH(tr, kClsSeed, s, k_conflict_count, blocks, 256, g, cg, b.st, b.list, b.cell_start,
                b.cell_items, b.conf_off);
    ConflictOffsetPolicy op{b.st, b.conf_off};
    QSGS_LAUNCH(tr, kClsSeed, s, k_lookback_scan<ConflictOffsetPolicy>, scan_grid(g.n),
                kScanThreads, op, ctl);
    QSGS_LAUNCH(tr, kClsSeed, s, k_conflict_fill, blocks, 256, g, cg, b.st, b.list, b.cell_start,
                b.cell_items, b.conf_off, b.adj, b.adj_cap);
    QSGS_LAUNCH_SMEM(tr, kClsSeed, s, k_spacing_rounds_csr, 1, 1024, kSpacingSmem, b.st,
                     b.conf_off, b.adj, b.decision, b.adj_cap);
    QSGS_LAUNCH(tr, kClsSeed, s, k_spacing_rounds, 1, 1024, g, cg, b.st, b.list, b.cell_start,
                b.cell_items, b.decision, b.adj_cap);
    decision = b.decision;
  }
  AcceptPolicy ap{g, b.st, b.grid, b.list, decision};
  QSGS_LAUNCH(tr, kClsSeed, s, k_lookback_scan<AcceptPolicy>, scan_grid(g.n), kScanThreads, ap,
              ctl);
  // Initial candidate words (Sec. 2.3 step 2) replace the candidate list.
  InitialListPolicy cp{g, b.st, b.grid, b.list};
  QSGS_LAUNCH(tr, kClsFront, s, k_lookback_scan<InitialListPolicy>, scan_grid(g.nwords), kScanThreads,
              cp, ctl);
  QSGS_LAUNCH(tr, kClsStepCtl, s, k_step_control, 1, 32, b.st, (cudaGraphConditionalHandle)0, 0);
  return cudaSuccess;
}

cudaError_t launch_step(const Geom& g, const StepBuffers& b, uint32_t k0, uint32_t k1,
                        uint32_t spin_limit, GrowShape shape, cudaStream_t s, Tracer& tr,
                        cudaGraphConditionalHandle cond, int use_cond, int fullfield) {
  (void)spin_limit;  // no waits in a step of the single-realization path
  if (fullfield) {
    const uint64_t need = ((uint64_t)g.nwords + 255) / 256;
    const uint64_t cap = (uint64_t)num_sms() * 8;
    const uint32_t blocks = (uint32_t)(need < cap ? (need ? need : 1) : cap);
    QSGS_LAUNCH(tr, kClsGrow, s, k_grow_fullfield, blocks, 256, g, b.grid, b.aux, b.mark, b.st,
                make_philox_keys((uint64_t)k1 << 32 | k0));
  } else {
    if (b.enter)
      QSGS_LAUNCH_SMEM(tr, kClsGrow, s, k_grow<kInteract>, shape.blocks, kGrowThreads,
                       kGrowSmemBytes, geom_inter(g, b), b.list, b.grid, b.aux, b.mark, b.st,
                       make_philox_keys((uint64_t)k1 << 32 | k0), shape.tile);
    else if (g.blocked)
      QSGS_LAUNCH_SMEM(tr, kClsGrow, s, k_grow<kRuntime>, shape.blocks, kGrowThreads,
                       kGrowSmemBytes, g, b.list, b.grid, b.aux, b.mark, b.st,
                       make_philox_keys((uint64_t)k1 << 32 | k0), shape.tile);
    else if (g.periodic)
      QSGS_LAUNCH_SMEM(tr, kClsGrow, s, k_grow<kTorus>, shape.blocks, kGrowThreads,
                       kGrowSmemBytes, g, b.list, b.grid, b.aux, b.mark, b.st,
                       make_philox_keys((uint64_t)k1 << 32 | k0), shape.tile);
    else
      QSGS_LAUNCH_SMEM(tr, kClsGrow, s, k_grow<kOpen>, shape.blocks, kGrowThreads,
                       kGrowSmemBytes, g, b.list, b.grid, b.aux, b.mark, b.st,
                       make_philox_keys((uint64_t)k1 << 32 | k0), shape.tile);
  }
  QSGS_LAUNCH(tr, kClsFront, s, k_commit, commit_grid(g.nwords), kCommitThreads, g, b.st, b.grid,
              b.aux, b.mark, b.list);
  QSGS_LAUNCH(tr, kClsStepCtl, s, k_step_control, 1, 32, b.st, cond, use_cond);
  return cudaSuccess;
}

cudaError_t launch_epilogue(const Geom& g, const StepBuffers& b, uint32_t spin_limit,
                            cudaStream_t s, Tracer& tr) {
  ScanCtl ctl{b.st, b.scan_status, spin_limit};
  TrimPolicy tp{g, b.st, b.grid, b.aux};
  QSGS_LAUNCH(tr, kClsTrim, s, k_lookback_scan<TrimPolicy>, scan_grid(g.nwords), kScanThreads, tp,
              ctl);
  QSGS_LAUNCH(tr, kClsTrim, s, k_zero_front, 1, 1, b.st);
  // The final front count (a statistic): an unordered sum over all words.
  if (b.enter) {  // an interacting phase counts enterable neighbours too
    FrontCountInterPolicy fi{geom_inter(g, b), b.st, b.grid};
    QSGS_LAUNCH(tr, kClsTrim, s, k_side_sum<FrontCountInterPolicy>, side_sum_grid(g.nwords), 256,
                fi);
    QSGS_LAUNCH(tr, kClsTrim, s, k_trim_done, 1, 1, b.st);
    return cudaSuccess;
  }
  FrontCountPolicy fp{g, b.st, b.grid};
  QSGS_LAUNCH(tr, kClsTrim, s, k_side_sum<FrontCountPolicy>, side_sum_grid(g.nwords), 256, fp);
  QSGS_LAUNCH(tr, kClsTrim, s, k_trim_done, 1, 1, b.st);
  return cudaSuccess;
}

cudaError_t launch_set_step_limit(RunState* st, uint32_t extra, cudaStream_t s, Tracer& tr) {
  QSGS_LAUNCH(tr, kClsStepCtl, s, k_set_step_limit, 1, 1, st, extra);
  return cudaSuccess;
}

cudaError_t launch_unpack_u8(const Geom& g, const uint32_t* grid, uint8_t* out, uint64_t vb,
                             uint64_t ve, cudaStream_t s, Tracer& tr) {
  const uint64_t chunks = (ve - vb + 15) / 16;
  uint64_t blocks = (chunks + 255) / 256;
  const uint64_t cap = (uint64_t)num_sms() * 16;
  if (blocks > cap) blocks = cap;
  if (blocks == 0) blocks = 1;
  QSGS_LAUNCH(tr, kClsFetch, s, k_unpack_u8, (uint32_t)blocks, 256, g, grid, out,
              (unsigned long long)vb, (unsigned long long)ve);
  return cudaSuccess;
}

// Resident blocks per SM of a growth kernel (its registers and shared
// memory decide); the default grids are exactly one wave of them, since the
// kernels take their chunks from a dispenser.
template <class K>
static uint32_t grow_wave(K kernel) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kGrowThreads,
                                                    kGrowSmemBytes) != cudaSuccess ||
      per_sm <= 0) {
    (void)cudaGetLastError();
    per_sm = 2;
  }
  return (uint32_t)num_sms() * (uint32_t)per_sm;
}

uint32_t default_grow_blocks() {
  static uint32_t blocks = 0;
  if (!blocks) blocks = grow_wave(k_grow<kOpen>);
  return blocks;
}

uint32_t default_batch_grow_blocks() {
  static uint32_t blocks = 0;
  if (!blocks) blocks = grow_wave(k_grow_batch<kRuntime>);
  return blocks;
}

cudaError_t launch_label_u8(const Geom& g, const uint32_t* grid, uint8_t* out, uint8_t label,
                            cudaStream_t s, Tracer& tr) {
  uint64_t blocks = ((uint64_t)g.nwords + 255) / 256;
  const uint64_t cap = (uint64_t)num_sms() * 8;
  if (blocks > cap) blocks = cap;
  QSGS_LAUNCH(tr, kClsFetch, s, k_label_u8, (uint32_t)(blocks ? blocks : 1), 256, g, grid, out,
              label);
  return cudaSuccess;
}

cudaError_t launch_or_words(uint32_t n, const uint32_t* src, uint32_t* dst, cudaStream_t s,
                            Tracer& tr) {
  uint64_t blocks = ((uint64_t)n + 255) / 256;
  const uint64_t cap = (uint64_t)num_sms() * 8;
  if (blocks > cap) blocks = cap;
  QSGS_LAUNCH(tr, kClsFetch, s, k_or_words, (uint32_t)(blocks ? blocks : 1), 256, n, src, dst);
  return cudaSuccess;
}

// Interacting phases (R13): from the labels of earlier phases, the packed
// grid of all their cells (blocked) and, per class k, of the cells whose
// label may be entered along class k (bit `label` of sets[k]).  A thread per
// word; bits at x >= nx stay 0.
struct LabelSets {
  uint32_t bits[3][8];  // per class: a 256-bit set of labels
};

__global__ void k_pack_labels(Geom g, const uint8_t* __restrict__ labels, uint32_t* blocked,
                              uint32_t* enter, LabelSets sets) {
  for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < g.nwords;
       w += gridDim.x * blockDim.x) {
    const uint32_t r = fast_div(w, g.div_W);
    const uint32_t x0 = (w - r * g.W) * 32u;
    const uint32_t len = min(32u, g.nx - x0);
    const uint8_t* row = labels + (size_t)r * g.nx + x0;
    uint32_t b = 0, e0 = 0, e1 = 0, e2 = 0;
    for (uint32_t i = 0; i < len; ++i) {
      const uint32_t lab = row[i];
      b |= (lab != 0u ? 1u : 0u) << i;
      e0 |= ((sets.bits[0][lab >> 5] >> (lab & 31u)) & 1u) << i;
      e1 |= ((sets.bits[1][lab >> 5] >> (lab & 31u)) & 1u) << i;
      e2 |= ((sets.bits[2][lab >> 5] >> (lab & 31u)) & 1u) << i;
    }
    blocked[w] = b;
    enter[w] = e0;
    enter[(size_t)g.nwords + w] = e1;
    enter[2 * (size_t)g.nwords + w] = e2;
  }
}

cudaError_t launch_pack_labels(const Geom& g, const uint8_t* labels, uint32_t* blocked,
                               uint32_t* enter, const uint32_t (&sets)[3][8], cudaStream_t s,
                               Tracer& tr) {
  LabelSets ls;
  for (int k = 0; k < 3; ++k)
    for (int j = 0; j < 8; ++j) ls.bits[k][j] = sets[k][j];
  uint64_t blocks = ((uint64_t)g.nwords + 255) / 256;
  const uint64_t cap = (uint64_t)num_sms() * 8;
  if (blocks > cap) blocks = cap;
  QSGS_LAUNCH(tr, kClsSeed, s, k_pack_labels, (uint32_t)(blocks ? blocks : 1), 256, g, labels,
              blocked, enter, ls);
  return cudaSuccess;
}

cudaError_t launch_grow_only(const Geom& g, const StepBuffers& b, uint32_t k0, uint32_t k1,
                             GrowShape shape, cudaStream_t s, Tracer& tr) {
  if (b.enter)
    QSGS_LAUNCH_SMEM(tr, kClsGrow, s, k_grow<kInteract>, shape.blocks, kGrowThreads,
                     kGrowSmemBytes, geom_inter(g, b), b.list, b.grid, b.aux, b.mark, b.st,
                     make_philox_keys((uint64_t)k1 << 32 | k0), shape.tile);
  else if (g.blocked)
    QSGS_LAUNCH_SMEM(tr, kClsGrow, s, k_grow<kRuntime>, shape.blocks, kGrowThreads,
                     kGrowSmemBytes, g, b.list, b.grid, b.aux, b.mark, b.st,
                     make_philox_keys((uint64_t)k1 << 32 | k0), shape.tile);
  else if (g.periodic)
    QSGS_LAUNCH_SMEM(tr, kClsGrow, s, k_grow<kTorus>, shape.blocks, kGrowThreads, kGrowSmemBytes,
                     g, b.list, b.grid, b.aux, b.mark, b.st,
                     make_philox_keys((uint64_t)k1 << 32 | k0), shape.tile);
  else
    QSGS_LAUNCH_SMEM(tr, kClsGrow, s, k_grow<kOpen>, shape.blocks, kGrowThreads, kGrowSmemBytes,
                     g, b.list, b.grid, b.aux, b.mark, b.st,
                     make_philox_keys((uint64_t)k1 << 32 | k0), shape.tile);
  return cudaSuccess;
}

cudaError_t launch_front_list(const Geom& g, const StepBuffers& b, uint32_t spin_limit,
                              cudaStream_t s, Tracer& tr) {
  ScanCtl ctl{b.st, b.scan_status, spin_limit};
  InitialListPolicy cp{g, b.st, b.grid, b.list};
  QSGS_LAUNCH(tr, kClsFront, s, k_lookback_scan<InitialListPolicy>, scan_grid(g.nwords), kScanThreads,
              cp, ctl);
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Front count on library-owned static scratch (no allocation anywhere): the
// look-back scan of FrontCountPolicy with its run state and tile status
// words in a file-scope device array instead of a caller workspace.
// ---------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_front_scratch[kFrontScratchBytes];

uint64_t front_scratch_max_words() {
  const uint64_t tiles = (kFrontScratchBytes - sizeof(RunState)) / sizeof(unsigned long long) - 2;
  return tiles * kScanTile;
}

// The device address of the scratch, looked up once per device with that
// device current (the lookup may load the module: not inside a capture).
static cudaError_t front_scratch(void** ptr) {
  static void* addr[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_front_scratch);
    if (e != cudaSuccess) return e;
    addr[dev] = p;
  }
  *ptr = addr[dev];
  return cudaSuccess;
}

cudaError_t front_count_static(const Geom& g, const uint32_t* grid, uint32_t spin_limit,
                               cudaStream_t s, unsigned long long* front, uint32_t* error) {
  void* base = nullptr;
  cudaError_t e = front_scratch(&base);
  if (e != cudaSuccess) return e;
  RunState* st = static_cast<RunState*>(base);
  unsigned long long* status =
      reinterpret_cast<unsigned long long*>(static_cast<unsigned char*>(base) + sizeof(RunState));
  // What must start at zero: the run state (front count, tile dispenser,
  // epoch, error) and the status word of every tile this grid uses.
  const uint64_t tiles = ((uint64_t)g.nwords + kScanTile - 1) / kScanTile + 2;
  e = cudaMemsetAsync(base, 0, sizeof(RunState) + tiles * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  Tracer quiet;
  ScanCtl ctl{st, status, spin_limit};
  FrontCountPolicy fp{g, st, grid};
  const uint64_t blocks64 = (uint64_t)num_sms() * 4 < tiles ? (uint64_t)num_sms() * 4 : tiles;
  const uint32_t blocks = (uint32_t)(blocks64 ? blocks64 : 1);
  QSGS_LAUNCH(quiet, kClsTrim, s, k_lookback_scan<FrontCountPolicy>, blocks, kScanThreads, fp, ctl);
  RunState host{};
  e = cudaMemcpyAsync(&host, st, sizeof(RunState), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  *front = host.front_n;
  *error = host.error;
  return cudaSuccess;
}

cudaError_t launch_batch_prologue(const BatchBuffers& b, uint32_t spin_limit, cudaStream_t s,
                                  Tracer& tr, cudaGraphConditionalHandle cond, int use_cond) {
  (void)spin_limit;  // no waits in the batch commit
  QSGS_LAUNCH(tr, kClsStepCtl, s, k_batch_limits, (b.max_members + 255) / 256, 256, b.d, b.bs);
  QSGS_LAUNCH(tr, kClsFront, s, k_batch_list_solid, batch_commit_grid(b.max_words), 256, b.d,
              b.bs, b.list);
  QSGS_LAUNCH(tr, kClsStepCtl, s, k_batch_control, 1, kMaxBatchMembers, b.d, b.bs, cond, use_cond,
              1);
  return cudaSuccess;
}

cudaError_t launch_batch_gather_states(const BatchBuffers& b, uint32_t n, RunState* out,
                                       cudaStream_t s, Tracer& tr) {
  if (n) QSGS_LAUNCH(tr, kClsStepCtl, s, k_batch_gather_states, n, 16, b.d, out);
  return cudaSuccess;
}

cudaError_t launch_batch_step(const BatchBuffers& b, uint32_t spin_limit, GrowShape shape,
                              cudaStream_t s, Tracer& tr, cudaGraphConditionalHandle cond,
                              int use_cond) {
  (void)spin_limit;
  if (b.open_only)
    QSGS_LAUNCH_SMEM(tr, kClsGrow, s, k_grow_batch<kOpen>, shape.blocks, kGrowThreads,
                     kGrowSmemBytes, b.d, b.bs, b.list, shape.tile);
  else
    QSGS_LAUNCH_SMEM(tr, kClsGrow, s, k_grow_batch<kRuntime>, shape.blocks, kGrowThreads,
                     kGrowSmemBytes, b.d, b.bs, b.list, shape.tile);
  QSGS_LAUNCH(tr, kClsFront, s, k_batch_commit, batch_commit_grid(b.max_words), 256, b.d, b.bs,
              b.list);
  QSGS_LAUNCH(tr, kClsStepCtl, s, k_batch_control, 1, kMaxBatchMembers, b.d, b.bs, cond, use_cond,
              0);
  return cudaSuccess;
}

}  // namespace qsgs

