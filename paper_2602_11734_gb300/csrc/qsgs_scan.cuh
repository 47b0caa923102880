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
constexpr int kScanItems = 8;                         // default items per thread
constexpr int kScanTile = kScanThreads * kScanItems;  // default items per tile
constexpr int kScanMinTile = kScanThreads;             // smallest tile (1 item per thread):
                                                       // sizes the tile-status array

// Items per thread of a policy: Policy::kItems if it declares one, else 8.
template <class P, class = void>
struct ItemsPerThread {
  static constexpr int value = kScanItems;
};
template <class P>
struct ItemsPerThread<P, decltype((void)P::kItems, void())> {
  static constexpr int value = P::kItems;
};

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
//   Item load(uint32_t i) const          -- i < n_items
//   uint32_t count(const Item&) const    -- outputs of the item
//   void emit(const Item&, unsigned long long prefix) const
//   void total(unsigned long long) const -- called once with the grand total
//   uint32_t side(const Item&, int k) const     -- extra per-item values k = 0, 1,
//   unsigned long long* side_sum(int k) const   --   summed into these counters
//                                                   (nullptr: not summed)
//   static constexpr bool kBatched              -- true: items are loaded by
//   void load_run(uint32_t first, uint32_t n, Item (&it)[kItems]) const
//                                                   (n consecutive valid items)
//   static constexpr int kItems (optional)      -- items per thread (default 8);
//                                                   with 1, the 32 lanes of a
//                                                   warp hold consecutive items
template <class Policy>
__global__ void __launch_bounds__(kScanThreads, 2) k_lookback_scan(Policy pol, ScanCtl ctl) {
  __shared__ uint32_t s_tile;
  __shared__ unsigned long long s_prefix;
  __shared__ uint32_t s_warp[kScanThreads / 32];

  constexpr int kItems = ItemsPerThread<Policy>::value;
  constexpr int kTile = kScanThreads * kItems;
  if (!pol.active()) return;
  const uint32_t n_items = pol.n_items();
  const uint32_t ntiles = (uint32_t)(((unsigned long long)n_items + kTile - 1) / kTile);
  const uint32_t epoch = *(volatile uint32_t*)&ctl.st->scan_epoch;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (ntiles == 0 && blockIdx.x == 0 && threadIdx.x == 0) pol.total(0);

  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(&ctl.st->scan_tile, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    if (tile >= ntiles) break;

    typename Policy::Item it[kItems];
    uint32_t cnt[kItems];
    uint32_t mine = 0, side0 = 0, side1 = 0;
    const unsigned long long base =
        (unsigned long long)tile * kTile + (unsigned long long)threadIdx.x * kItems;
    const uint32_t n_valid =
        base >= n_items ? 0u : (uint32_t)min((unsigned long long)kItems, n_items - base);
    if constexpr (Policy::kBatched) {
      // Called by every thread (warp-cooperative loaders need all lanes).
      pol.load_run((uint32_t)min(base, (unsigned long long)n_items), n_valid, it);
    } else {
#pragma unroll
      for (int k = 0; k < kItems; ++k)
        if ((uint32_t)k < n_valid) it[k] = pol.load((uint32_t)(base + k));
    }
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
      cnt[k] = 0;
      if ((uint32_t)k < n_valid) {
        cnt[k] = pol.count(it[k]);
        side0 += pol.side(it[k], 0);
        side1 += pol.side(it[k], 1);
      }
      mine += cnt[k];
    }

    if (pol.side_sum(0) != nullptr) {
      const uint32_t ws = __reduce_add_sync(0xffffffffu, side0);
      if (lane == 0 && ws) atomicAdd(pol.side_sum(0), (unsigned long long)ws);
    }
    if (pol.side_sum(1) != nullptr) {
      const uint32_t ws = __reduce_add_sync(0xffffffffu, side1);
      if (lane == 0 && ws) atomicAdd(pol.side_sum(1), (unsigned long long)ws);
    }

    // Block-wide exclusive scan of the per-thread counts.
    uint32_t incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      uint32_t w = lane < kScanThreads / 32 ? s_warp[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      if (lane < kScanThreads / 32) s_warp[lane] = w;  // inclusive warp totals
    }
    __syncthreads();
    const uint32_t warp_excl = warp ? s_warp[warp - 1] : 0;
    const uint32_t aggregate = s_warp[kScanThreads / 32 - 1];

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
          const int64_t p = window_end - lane;  // lane 0 = nearest predecessor
          unsigned long long w = kFlagPrefix;  // tiles before 0: empty prefix
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
          unsigned long long v = (lane <= stop) ? (w & kValueMask) : 0ull;
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

    unsigned long long off = s_prefix + warp_excl + (incl - mine);
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
      if (cnt[k] || pol.emit_empty()) {
        if (base + k < n_items) pol.emit(it[k], off);
      }
      off += cnt[k];
    }
    __syncthreads();  // s_tile / s_warp / s_prefix are reused by the next tile
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
