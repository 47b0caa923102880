// qsgs_launch.h -- internal interface between the C ABI and the kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "qsgs_device.cuh"

namespace qsgs {

// Kernel classes of the launch counter and the optional event profiler.
enum KernelClass : int { kClsSeed, kClsGrow, kClsStepCtl, kClsTrim, kClsFront, kClsFetch, kNumClasses };
inline const char* kernel_class_name(int c) {
  static const char* names[kNumClasses] = {"seed", "grow", "step_ctl", "epilogue", "commit", "fetch"};
  return (c >= 0 && c < kNumClasses) ? names[c] : "?";
}

// Counts every kernel launch; when enabled, brackets each launch with a pair
// of CUDA events and turns them into per-class totals at collect().
class Tracer {
 public:
  uint64_t launches = 0;
  uint64_t count[kNumClasses] = {};
  double ms[kNumClasses] = {};

  bool enabled() const { return enabled_; }

  cudaError_t enable(bool on) {
    reset();
    enabled_ = on;
    return cudaSuccess;
  }

  void reset() {
    for (int c = 0; c < kNumClasses; ++c) { count[c] = 0; ms[c] = 0.0; }
    for (auto& p : pending_) { free_.push_back(p.start); free_.push_back(p.stop); }
    pending_.clear();
  }

  cudaError_t before(int cls, cudaStream_t s) {
    ++launches;
    if (!enabled_) return cudaSuccess;
    Pending p{cls, take(), take()};
    if (!p.start || !p.stop) return cudaErrorMemoryAllocation;
    pending_.push_back(p);
    return cudaEventRecord(p.start, s);
  }

  cudaError_t after(cudaStream_t s) {
    if (!enabled_ || pending_.empty()) return cudaSuccess;
    return cudaEventRecord(pending_.back().stop, s);
  }

  // Call after the stream has been synchronised.
  cudaError_t collect() {
    cudaError_t err = cudaSuccess;
    for (auto& p : pending_) {
      float t = 0.f;
      cudaError_t e = cudaEventElapsedTime(&t, p.start, p.stop);
      if (e == cudaSuccess) { count[p.cls] += 1; ms[p.cls] += t; } else { err = e; }
      free_.push_back(p.start);
      free_.push_back(p.stop);
    }
    pending_.clear();
    return err;
  }

  ~Tracer() {
    reset();
    for (auto e : free_) cudaEventDestroy(e);
  }

 private:
  struct Pending {
    int cls;
    cudaEvent_t start, stop;
  };
  cudaEvent_t take() {
    if (!free_.empty()) {
      cudaEvent_t e = free_.back();
      free_.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
  }
  bool enabled_ = false;
  std::vector<Pending> pending_;
  std::vector<cudaEvent_t> free_;
};

// Terminal statuses written into RunState::status (same values as the
// public QSGS_* codes).
enum : int32_t { kStatusDone = 0, kStatusStalled = 1, kStatusMaxSteps = 2 };

struct StateInit {
  unsigned long long nt;
  unsigned long long t_ref[3];
  unsigned long long t_seed;
  uint32_t max_steps;
};

struct CellGeomHost {
  uint32_t s, ncx, ncy, ncz;
};

struct SeedBuffers {
  RunState* st;
  unsigned long long* scan_status;
  uint32_t* grid;
  uint32_t* aux;
  uint32_t* list;        // seed candidates, then the candidate word list
  uint32_t* mark;        // one bit per word (growth kernel -> commit scan)
  uint32_t* cell_count;  // spacing only
  uint32_t* cell_start;
  uint32_t* cell_items;
  uint8_t* decision;
  uint32_t* conf_off;            // cand_n + 1 conflict-list offsets
  uint32_t* adj;                 // conflict lists
  unsigned long long adj_cap;    // entries adj can hold
  unsigned long long cand_cap;   // seed candidates list, cell_items and decision hold
  CellGeomHost cg;
};

struct StepBuffers {
  RunState* st;
  unsigned long long* scan_status;
  uint32_t* grid;
  uint32_t* aux;   // two claim grids (step parity)
  uint32_t* mark;  // one bit per word: still holds front voxels
  uint32_t* list;  // candidate word list (ascending)
  // Interacting phase (R13): the fields of GeomInter, all nullptr otherwise.
  const uint32_t* enter;
  const uint8_t* labels;
  const uint32_t* enter_thr;
};

Geom make_geom(uint32_t nx, uint32_t ny, uint32_t nz, uint32_t periodic);
// Launch shape of a growth kernel: thread blocks, and chunks of 32
// candidate words a warp takes per dispenser grab (its "front tile").
struct GrowShape {
  uint32_t blocks;
  uint32_t tile;
};
constexpr uint32_t kMaxGrowTile = 16;
uint32_t default_grow_blocks();        // one wave of k_grow (after prepare_kernels)
uint32_t default_batch_grow_blocks();  // one wave of k_grow_batch
// Front count with library-owned static scratch (kFrontScratchBytes of
// device memory in the library image; no allocation).  Serves grids of up
// to front_scratch_max_words() words; concurrent calls share the scratch.
constexpr size_t kFrontScratchBytes = 64 * 1024;
uint64_t front_scratch_max_words();
cudaError_t front_count_static(const Geom& g, const uint32_t* grid, uint32_t spin_limit,
                               cudaStream_t s, unsigned long long* front, uint32_t* error);
// Per-device function attributes (shared-memory opt-in) of the growth
// kernels; call before their first launch on the current device.
cudaError_t prepare_kernels();

cudaError_t launch_init_state(RunState* st, const StateInit& init, cudaStream_t s, Tracer& tr);
cudaError_t launch_seed(const Geom& g, const SeedBuffers& b, uint32_t k0, uint32_t k1,
                        uint32_t spin_limit, cudaStream_t s, Tracer& tr);
// One growth step: k_grow, the commit scan (claims into the grid, their
// count, the next candidate list) and the step control.  With use_cond, the step control
// also sets the graph conditional `cond` (while-loop body).
cudaError_t launch_step(const Geom& g, const StepBuffers& b, uint32_t k0, uint32_t k1,
                        uint32_t spin_limit, GrowShape shape, cudaStream_t s, Tracer& tr,
                        cudaGraphConditionalHandle cond, int use_cond, int fullfield);
// Exact-target trim (a no-op unless the last step overshot Nt) and the
// front count of the current grid.
cudaError_t launch_epilogue(const Geom& g, const StepBuffers& b, uint32_t spin_limit,
                            cudaStream_t s, Tracer& tr);
cudaError_t launch_set_step_limit(RunState* st, uint32_t extra, cudaStream_t s, Tracer& tr);
// The growth kernel alone (the timing probe: it is idempotent on the grid,
// the claim grid and the marks).
cudaError_t launch_grow_only(const Geom& g, const StepBuffers& b, uint32_t k0, uint32_t k1,
                             GrowShape shape, cudaStream_t s, Tracer& tr);
// Rebuilds a realization's candidate list from its grid (all solid words).
cudaError_t launch_front_list(const Geom& g, const StepBuffers& b, uint32_t spin_limit,
                              cudaStream_t s, Tracer& tr);

struct BatchBuffers {
  MemberDesc* d;
  BatchState* bs;
  uint32_t* list;
  uint32_t max_members;
  uint64_t max_words;
  uint32_t open_only;  // no member is periodic or has blocked cells
};

// Batch step limits, prologue commit (lists every running member's solid
// words) and prologue control (which sets the loop condition `cond` when
// use_cond is set).
cudaError_t launch_batch_prologue(const BatchBuffers& b, uint32_t spin_limit, cudaStream_t s,
                                  Tracer& tr, cudaGraphConditionalHandle cond, int use_cond);
// Run states of members 0 .. n-1 into out[0 .. n) (device).
cudaError_t launch_batch_gather_states(const BatchBuffers& b, uint32_t n, RunState* out,
                                       cudaStream_t s, Tracer& tr);
// One step of every member that runs: batched growth, commit and control.
cudaError_t launch_batch_step(const BatchBuffers& b, uint32_t spin_limit, GrowShape shape,
                              cudaStream_t s, Tracer& tr, cudaGraphConditionalHandle cond,
                              int use_cond);
cudaError_t launch_philox_rate(uint64_t seed, uint32_t blocks, uint32_t per_thread,
                               unsigned long long* out, cudaStream_t s);
// L2 probes: `passes` reads of n16 16-byte elements through L2 (the grid is
// 4 blocks of 512 threads per SM; needs n16 >= 4 * that many threads), and
// blocks x 512 threads issuing per_thread reductions each into nwords words.
uint32_t l2_read_threads();
cudaError_t launch_l2_read(const void* buf, uint64_t n16, uint32_t passes,
                           unsigned long long* out, cudaStream_t s);
cudaError_t launch_l2_red(void* buf, uint64_t nwords, uint32_t per_thread, uint32_t blocks,
                          cudaStream_t s);
// Phase maps: `label` into out[v] for every solid voxel v (other bytes
// untouched); src words ORed into dst (n words).
cudaError_t launch_label_u8(const Geom& g, const uint32_t* grid, uint8_t* out, uint8_t label,
                            cudaStream_t s, Tracer& tr);
// Interacting phases (R13): packed grids of the earlier phases' cells and,
// per class, of the enterable ones (three grids nwords apart) from a label
// map; sets[k] holds the labels that class k may enter (bit m of word m>>5).
cudaError_t launch_pack_labels(const Geom& g, const uint8_t* labels, uint32_t* blocked,
                               uint32_t* enter, const uint32_t (&sets)[3][8], cudaStream_t s,
                               Tracer& tr);
cudaError_t launch_or_words(uint32_t n, const uint32_t* src, uint32_t* dst, cudaStream_t s,
                            Tracer& tr);
// Voxels [vb, ve) of the grid as one byte each into out[0 .. ve - vb).
cudaError_t launch_unpack_u8(const Geom& g, const uint32_t* grid, uint8_t* out, uint64_t vb,
                             uint64_t ve, cudaStream_t s, Tracer& tr);

}  // namespace qsgs
