// qsgs_device.cuh -- device primitives of the QSGS generator (sm_103a).
//
// Grid geometry with division by invariant integers, the Philox4x32-10
// counter-based generator, the 26-direction table of the growth step and
// the device-resident run state.  Written for this library; it shares
// nothing with the CPU oracle.
#pragma once

#include <cstdint>

namespace qsgs {

// ---------------------------------------------------------------------------
// Unsigned division by an invariant 32-bit divisor with one multiply-high
// (Granlund & Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994, Sec. 4, the round-up method):
//   l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1,
//   t = umulhi(m, n), q = (t + ((n - t) >> min(l,1))) >> max(l-1, 0).
// Exact for every 32-bit n and every 1 <= d < 2^32.
// ---------------------------------------------------------------------------
struct FastDiv {
  uint32_t d, m, s1, s2;
};

inline FastDiv make_fastdiv(uint32_t d) {
  FastDiv f{};
  f.d = d;
  uint32_t l = 0;
  while (l < 32 && (1ull << l) < d) ++l;
  f.m = (uint32_t)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
  f.s1 = l < 1 ? l : 1;
  f.s2 = l > 0 ? l - 1 : 0;
  return f;
}

__host__ __device__ inline uint32_t fast_div(uint32_t n, const FastDiv& f) {
#ifdef __CUDA_ARCH__
  uint32_t t = __umulhi(n, f.m);
#else
  uint32_t t = (uint32_t)(((uint64_t)n * f.m) >> 32);
#endif
  return (t + ((n - t) >> f.s1)) >> f.s2;
}

// ---------------------------------------------------------------------------
// Grid geometry.  Voxel v = x + nx (y + ny z); row r = y + ny z.  The
// occupancy grid is bit-packed, x fastest: row r holds W = ceil(nx/32)
// 32-bit words, bit (x & 31) of word r*W + (x >> 5).  Bits at x >= nx in
// the last word of a row are kept zero.
// ---------------------------------------------------------------------------
struct Geom {
  uint32_t nx, ny, nz;
  uint32_t W;        // words per row
  uint32_t nrows;    // ny * nz
  uint32_t nwords;   // W * nrows
  uint32_t n;        // nx * ny * nz (< 2^32)
  uint32_t pad_mask; // bits of the last word of a row that lie at x >= nx
  uint32_t periodic; // 1: neighbours wrap around every axis (a torus)
  FastDiv div_nx, div_ny, div_W;
  const uint32_t* blocked;  // packed cells of earlier phases (R12), or nullptr
};

// Word bitmaps: one bit per grid word (bit w & 31 of word w >> 5).  The mark
// area of a workspace holds two of them: the marks (words that hold front
// voxels in the current step, set by the growth kernel) and, right after,
// the touched bits (words that received a claim in the current step).
__host__ __device__ __forceinline__ uint32_t bitmap_words(const Geom& g) {
  return (g.nwords >> 5) + 1u;
}

// The geometry of an interacting phase (R13), passed to that kind's kernels
// only (so that Geom, which every kernel takes, keeps its size).
struct GeomInter : Geom {
  const uint32_t* enter;      // three packed grids (class face, edge, corner;
                              // nwords apart): cells of earlier phases that
                              // may be entered along that class
  const uint8_t* labels;      // labels of earlier phases, 0 = unassigned
  const uint32_t* enter_thr;  // [label * 3 + class]: floor(I 2^32) - 1; row
                              // 0 (no label): per class the largest of them
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
// easy as 1, 2, 3", SC'11): ten rounds, each two 32x32->64 products
// (multipliers 0xD2511F53, 0xCD9E8D57) and a key bumped by the Weyl
// constants (0x9E3779B9, 0xBB67AE85).
// ---------------------------------------------------------------------------
struct U4 {
  uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    const uint32_t lo0 = 0xD2511F53u * c.x;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// The ten round keys of a 64-bit seed, precomputed on the host so that a
// kernel can take them as (constant-bank) parameters.
struct PhiloxKeys {
  uint32_t k0[10], k1[10];
};

inline PhiloxKeys make_philox_keys(uint64_t seed) {
  PhiloxKeys k{};
  uint32_t a = (uint32_t)seed, b = (uint32_t)(seed >> 32);
  for (int i = 0; i < 10; ++i) {
    k.k0[i] = a;
    k.k1[i] = b;
    a += 0x9E3779B9u;
    b += 0xBB67AE85u;
  }
  return k;
}

// Philox4x32-10 with precomputed round keys (each round's two products as
// 64-bit multiplies; separate 32-bit high and low products measured slower).
__device__ __forceinline__ U4 philox4x32_10(U4 c, const PhiloxKeys& key) {
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
    const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
    c = U4{(uint32_t)(p1 >> 32) ^ c.y ^ key.k0[i], (uint32_t)p1,
           (uint32_t)(p0 >> 32) ^ c.w ^ key.k1[i], (uint32_t)p0};
  }
  return c;
}

__device__ __forceinline__ uint32_t u4_word(const U4& r, int j) {
  return j == 0 ? r.x : (j == 1 ? r.y : (j == 2 ? r.z : r.w));
}

// Stream tags of the counter's fourth word: seeding draws and growth draws
// never share a counter.
constexpr uint32_t kSeedTag = 0x100u;
constexpr uint32_t kGrowTag = 0x200u;

// ---------------------------------------------------------------------------
// Directions.  d = 0..5 faces, 6..17 edges, 18..25 corners; within a class
// ordered by (dz, dy, dx) lexicographically.  A growth attempt along d is
// drawn by the rank of d among the source's targets of its class (counter
// word 3 = 0x200 | block; see growth_blocks in qsgs_kernels.cu).  A
// neighbourhood position packs the offset as (dz+1)*9 + (dy+1)*3 + (dx+1).
// ---------------------------------------------------------------------------
struct Dir {
  int dx, dy, dz, cls;
};

// The table itself is only read in constant expressions; device code uses
// the packed scalar forms below (2 bits per direction and field).
constexpr Dir kDirs[26] = {
    // faces
    {0, 0, -1, 0}, {0, -1, 0, 0}, {-1, 0, 0, 0}, {1, 0, 0, 0}, {0, 1, 0, 0}, {0, 0, 1, 0},
    // edges
    {0, -1, -1, 1}, {-1, 0, -1, 1}, {1, 0, -1, 1}, {0, 1, -1, 1},
    {-1, -1, 0, 1}, {1, -1, 0, 1}, {-1, 1, 0, 1}, {1, 1, 0, 1},
    {0, -1, 1, 1}, {-1, 0, 1, 1}, {1, 0, 1, 1}, {0, 1, 1, 1},
    // corners
    {-1, -1, -1, 2}, {1, -1, -1, 2}, {-1, 1, -1, 2}, {1, 1, -1, 2},
    {-1, -1, 1, 2}, {1, -1, 1, 2}, {-1, 1, 1, 2}, {1, 1, 1, 2},
};

constexpr uint64_t pack_dir_field(int field) {
  uint64_t m = 0;
  for (int d = 0; d < 26; ++d) {
    int v = field == 0 ? kDirs[d].dx + 1
          : field == 1 ? kDirs[d].dy + 1
          : field == 2 ? kDirs[d].dz + 1
                       : kDirs[d].cls;
    m |= (uint64_t)v << (2 * d);
  }
  return m;
}

constexpr uint64_t kDxPacked = pack_dir_field(0);
constexpr uint64_t kDyPacked = pack_dir_field(1);
constexpr uint64_t kDzPacked = pack_dir_field(2);
constexpr uint64_t kClsPacked = pack_dir_field(3);

__host__ __device__ constexpr int dir_dx(int d) { return (int)((kDxPacked >> (2 * d)) & 3) - 1; }
__host__ __device__ constexpr int dir_dy(int d) { return (int)((kDyPacked >> (2 * d)) & 3) - 1; }
__host__ __device__ constexpr int dir_dz(int d) { return (int)((kDzPacked >> (2 * d)) & 3) - 1; }
__host__ __device__ constexpr int dir_cls(int d) { return (int)((kClsPacked >> (2 * d)) & 3); }

__host__ __device__ __forceinline__ int nb_pos(int dx, int dy, int dz) {
  return (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
}

__host__ __device__ __forceinline__ int dir_pos(int d) {
  return nb_pos(dir_dx(d), dir_dy(d), dir_dz(d));
}

constexpr uint32_t kNbAll = (1u << 27) - 1u;
constexpr uint32_t kNbCentre = 1u << 13;

// ---------------------------------------------------------------------------
// Device-resident run state (one per realization, 256 bytes, in the
// caller's workspace).  Kernels of a step read it; the one-thread step
// kernels write it, so the host never has to synchronise between steps.
// ---------------------------------------------------------------------------
enum : int32_t { kRunning = -1 };
enum : uint32_t { kErrTimeout = 1u, kErrOverflow = 2u };

struct alignas(256) RunState {
  unsigned long long solid;      // c_t (solid voxels)
  unsigned long long nt;         // target count
  unsigned long long thr[3];     // Eq. 1 thresholds for this step
  unsigned long long t_ref[3];   // floor(G_ref 2^32) per class
  unsigned long long t_seed;     // floor(cd 2^32)
  unsigned long long claimed;    // |New_t|, counted by the front rebuild
  unsigned long long live;       // attempts with a positive threshold
  unsigned long long sum_front;  // sum over steps of |A_t| (statistics)
  unsigned long long sum_draws;  // Philox blocks drawn by growth steps
  unsigned long long front_n;    // |A_t| (front voxels)
  unsigned long long front_acc;  // |A_{t+1}| being counted by the rebuild
  unsigned long long adj_n;      // spacing: total earlier-conflict entries
  unsigned long long trim_keep;  // exact target: claims of the last step kept
  uint32_t front_words;          // entries of the front word list
  uint32_t cand_n;               // Bernoulli candidates
  uint32_t acc_n;                // seeds placed
  uint32_t t;                    // steps executed
  uint32_t max_steps;            // total step limit (0xFFFFFFFF = none)
  uint32_t step_limit;           // pause point of the current call
  int32_t status;                // kRunning or a QSGS_* status
  uint32_t active;               // the next step runs
  uint32_t trim_pending;         // the last step overshot Nt: trim before fetch
  uint32_t trim_parity;          // claim grid of that step
  uint32_t error;                // kErr* bits
  uint32_t iters;                // step-control launches (closed/opened steps)
  uint32_t scan_epoch;           // look-back scan launch counter
  uint32_t scan_tile;            // look-back scan tile dispenser
  uint32_t scan_done;            // look-back scan blocks finished
  uint32_t grow_next;            // growth chunk dispenser (zero between launches)
  uint32_t grow_done;            // growth blocks finished (zero between launches)
  uint32_t list_next;            // entries appended to the next candidate list
};

// ---------------------------------------------------------------------------
// Batches: many realizations advanced by the same launches.  Member m's
// words occupy [word_base, word_base + nwords) of a batch word space whose
// ranges start at multiples of 32, so the 32 lanes of a warp that scan 32
// consecutive batch words always serve one member.  The batch candidate
// list is the concatenation of the members' candidate lists (local word
// indices); member m's entries start at list_base.
// ---------------------------------------------------------------------------
constexpr uint32_t kMaxBatchMembers = 1024;  // one control block, thread per member

struct alignas(16) MemberDesc {
  Geom g;
  uint32_t* grid;
  uint32_t* aux;        // two claim grids
  uint32_t* mark;
  RunState* st;
  PhiloxKeys keys;
  uint32_t word_base;   // first batch word (multiple of 32)
  uint32_t word_end;    // word_base + nwords
  uint32_t list_base;   // first entry in the batch candidate list
  uint32_t list_n;      // entries of this member
  uint32_t chunk_base;  // first growth chunk (32 entries) of this member
  uint32_t commit_base; // first commit super-group of this member (0 groups if it does not run)
  uint32_t pad_[2];
};

struct BatchState {
  RunState scan;          // growth chunk dispenser, control-launch counter (iters)
  uint32_t n_members;
  uint32_t total_words;   // end of the batch word space
  uint32_t total_chunks;  // growth chunks of this step
  uint32_t any_active;    // some member runs the next step
  uint32_t step_extra;    // per-member step budget of the current advance (0: none)
  uint32_t total_supers;  // commit super-groups of the members that run this step
  uint32_t pad_[2];
};

}  // namespace qsgs

