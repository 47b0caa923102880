// qsgs_scan.cuh -- single-pass prefix scan with decoupled look-back.
//
// One persistent kernel template serves every order-preserving pass of the
// generator (candidate compaction, front rebuild, exact trim, seed cap,
// cell offsets).  Blocks take tiles from an atomic dispenser, so a tile
// only ever waits on tiles already held by running blocks (Merrill &
// Garland, "Single-pass parallel prefix scan with decoupled look-back",
// NVIDIA TR 2016).  Every wait is bounded: after `spin_limit` polls the
// block records kErrTimeout in the run state and carries on with a zero
// prefix, so a fault is reported instead of hanging the GPU.
#pragma once

#include "qsgs_device.cuh"

namespace qsgs {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;                         // items per thread
constexpr int kScanTile = kScanThreads * kScanItems;  // items per tile

// Tile status word: [63:62] flag, [61:33] launch epoch, [32:0] value.
constexpr unsigned long long kFlagAggregate = 1ull << 62;
constexpr unsigned long long kFlagPrefix = 2ull << 62;
constexpr unsigned long long kValueMask = (1ull << 33) - 1;
constexpr uint32_t kEpochMask = (1u << 29) - 1;

struct ScanCtl {
  RunState* st;                  // epoch, tile dispenser, completion count, error
  unsigned long long* status;    // one word per tile (zeroed before first use)
  uint32_t spin_limit;
};

__device__ __forceinline__ unsigned long long tile_word(unsigned long long flag, uint32_t epoch,
                                                        unsigned long long value) {
  return flag | ((unsigned long long)(epoch & kEpochMask) << 33) | (value & kValueMask);
}

// Policy interface:
//   bool active() const                  -- uniform: false skips the launch
//   uint32_t n_items() const             -- number of items (read on device)
//   Item load(uint32_t i, bool valid) const
//                                        -- called by all 32 lanes of a warp
//                                           together (lane l gets item base+l,
//                                           so warp-cooperative loaders may use
//                                           shuffles); invalid lanes get
//                                           i = n_items and must not touch it;
//                                           reads only (no stores)
//   void apply(const Item&, bool valid) const
//                                        -- the item's side effects (stores),
//                                           called by all lanes after every
//                                           load of the tile was issued
//   uint32_t count(const Item&) const    -- outputs of the item
//   void emit(const Item&, unsigned long long prefix) const
//   bool emit_empty() const              -- also emit items with count 0
//   void total(unsigned long long) const -- called once with the grand total
//   uint32_t side(const Item&, int k) const     -- extra per-item values k = 0, 1,
//   unsigned long long* side_sum(int k) const   --   summed into these counters
//                                                   (nullptr: not summed)
//
// Tile layout: a tile holds kScanTile items; thread t of the block handles
// items base + k * kScanThreads + t for k < kScanItems, so every warp works
// on 32 consecutive items at a time (coalesced loads).  The order of the
// outputs is the order of the items: offsets are taken over (k, warp, lane)
// in that nesting.  The loads of all kScanItems items are issued before any
// store of the tile (side effects, shared-memory offsets), so a thread has
// all of them in flight at once instead of one memory round trip per item.
template <class Policy>
__global__ void __launch_bounds__(kScanThreads, 2) k_lookback_scan(Policy pol, ScanCtl ctl) {
  constexpr int kWarps = kScanThreads / 32;
  __shared__ uint32_t s_tile;
  __shared__ unsigned long long s_prefix;
  __shared__ uint32_t s_off[kScanItems * kWarps];  // warp totals, then their offsets
  __shared__ uint32_t s_agg;

  if (!pol.active()) return;
  const uint32_t n_items = pol.n_items();
  const uint32_t ntiles = (uint32_t)(((unsigned long long)n_items + kScanTile - 1) / kScanTile);
  const uint32_t epoch = *(volatile uint32_t*)&ctl.st->scan_epoch;
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  if (ntiles == 0 && blockIdx.x == 0 && threadIdx.x == 0) pol.total(0);

  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(&ctl.st->scan_tile, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    if (tile >= ntiles) break;

    typename Policy::Item it[kScanItems];
    uint32_t cnt[kScanItems], lex[kScanItems];
    uint32_t side0 = 0, side1 = 0;
    const unsigned long long base = (unsigned long long)tile * kScanTile + threadIdx.x;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      const unsigned long long i = base + (unsigned long long)k * kScanThreads;
      const bool valid = i < n_items;
      it[k] = pol.load(valid ? (uint32_t)i : n_items, valid);
    }
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      const unsigned long long i = base + (unsigned long long)k * kScanThreads;
      pol.apply(it[k], i < n_items);
    }
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      const unsigned long long i = base + (unsigned long long)k * kScanThreads;
      const bool valid = i < n_items;
      cnt[k] = valid ? pol.count(it[k]) : 0u;
      if (valid) {
        side0 += pol.side(it[k], 0);
        side1 += pol.side(it[k], 1);
      }
      uint32_t incl = cnt[k];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (uint32_t)o) incl += y;
      }
      lex[k] = incl - cnt[k];
      if (lane == 31) s_off[k * kWarps + warp] = incl;
    }
    if (pol.side_sum(0) != nullptr) {
      const uint32_t ws = __reduce_add_sync(0xffffffffu, side0);
      if (lane == 0 && ws) atomicAdd(pol.side_sum(0), (unsigned long long)ws);
    }
    if (pol.side_sum(1) != nullptr) {
      const uint32_t ws = __reduce_add_sync(0xffffffffu, side1);
      if (lane == 0 && ws) atomicAdd(pol.side_sum(1), (unsigned long long)ws);
    }
    __syncthreads();

    // Exclusive offsets of the kScanItems x kWarps warp totals (k-major),
    // two per lane of warp 0.
    if (warp == 0) {
      static_assert(kScanItems * kWarps == 64, "two warp totals per lane");
      const uint32_t a = s_off[2 * lane], b = s_off[2 * lane + 1];
      uint32_t incl = a + b;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (uint32_t)o) incl += y;
      }
      const uint32_t excl = incl - a - b;
      s_off[2 * lane] = excl;
      s_off[2 * lane + 1] = excl + a;
      if (lane == 31) s_agg = incl;
    }
    __syncthreads();
    const uint32_t aggregate = s_agg;

    // Decoupled look-back by warp 0: each round reads the 32 tiles before
    // the current window in parallel, waits (bounded) until all of them have
    // published, and stops at the nearest inclusive prefix.
    if (warp == 0) {
      unsigned long long prefix = 0;
      if (tile == 0) {
        if (lane == 0) atomicExch(&ctl.status[0], tile_word(kFlagPrefix, epoch, aggregate));
      } else {
        if (lane == 0) atomicExch(&ctl.status[tile], tile_word(kFlagAggregate, epoch, aggregate));
        int64_t window_end = (int64_t)tile - 1;  // highest tile of the window
        for (;;) {
          const int64_t p = window_end - (int64_t)lane;  // lane 0 = nearest predecessor
          unsigned long long w = kFlagPrefix;           // tiles before 0: empty prefix
          if (p >= 0) {
            uint32_t polls = 0;
            for (;;) {
              w = *(volatile unsigned long long*)&ctl.status[p];
              if ((w >> 62) != 0 && (uint32_t)((w >> 33) & kEpochMask) == (epoch & kEpochMask)) break;
              if (++polls > ctl.spin_limit) {
                atomicOr(&ctl.st->error, kErrTimeout);
                w = kFlagPrefix;  // give up: treat as a zero inclusive prefix
                break;
              }
              __nanosleep(32);
            }
          }
          const bool is_prefix = (w & (3ull << 62)) == kFlagPrefix;
          const uint32_t pmask = __ballot_sync(0xffffffffu, is_prefix);
          // Lanes up to and including the nearest inclusive prefix contribute.
          const int stop = pmask ? __ffs(pmask) - 1 : 31;
          unsigned long long v = ((int)lane <= stop) ? (w & kValueMask) : 0ull;
#pragma unroll
          for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
          prefix += v;
          if (pmask) break;
          window_end -= 32;
        }
        if (lane == 0)
          atomicExch(&ctl.status[tile], tile_word(kFlagPrefix, epoch, prefix + aggregate));
      }
      if (lane == 0) {
        s_prefix = prefix;
        if (tile == ntiles - 1) pol.total(prefix + aggregate);
      }
    }
    __syncthreads();

    const unsigned long long tile_prefix = s_prefix;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      const unsigned long long i = base + (unsigned long long)k * kScanThreads;
      if (i < n_items && (cnt[k] || pol.emit_empty()))
        pol.emit(it[k], tile_prefix + s_off[k * kWarps + warp] + lex[k]);
    }
    __syncthreads();  // s_tile / s_off / s_prefix are reused by the next tile
  }

  // The last block to finish re-arms the dispenser for the next launch.
  if (threadIdx.x == 0) {
    __threadfence();
    const uint32_t done = atomicAdd(&ctl.st->scan_done, 1u);
    if (done == gridDim.x - 1) {
      ctl.st->scan_tile = 0;
      ctl.st->scan_done = 0;
      ctl.st->scan_epoch = (epoch + 1) & kEpochMask;
      __threadfence();
    }
  }
}

}  // namespace qsgs
