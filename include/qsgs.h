/*
 * qsgs.h -- C ABI of the GB300 LIETS QSGS porous-media generator.
 *
 * The library generates one solid phase on a 3-D voxel grid by the
 * list-indexed explicit time-stepping (LIETS) form of the Quartet Structure
 * Generation Set of arXiv 2602.11734 (Wang & Al Kobaisi):
 *   - Bernoulli seeding with probability c_d                (Sec. 2.1 step 2)
 *   - seed spacing s by diamond (L1-ball) exclusion          (Sec. 2.3, Fig. 1 D)
 *   - the active front: solids with a void 26-neighbour      (Sec. 2.3 step 2)
 *   - front-only directional growth, 6 face / 12 edge /
 *     8 corner directions                                   (Sec. 2.3 step 3, Algorithm 3)
 *   - the volume-fraction law of the growth probabilities    (Eq. 1)
 *   - the front update prune(A U New)                        (Sec. 2.3 step 4)
 * with an exact final solid count (the last step keeps the lowest-index
 * claims only).  All arithmetic is integer: draws are 32-bit Philox4x32-10
 * words keyed by the realization seed, and probabilities p enter as
 * thresholds floor(p 2^32).  Results are bit-identical for any launch order.
 *
 * Conventions
 *   - Voxel v = x + nx (y + ny z), x fastest; N = nx ny nz must be < 2^32.
 *   - Pointers marked "device" are CUDA device pointers of the current
 *     device; "host" pointers are ordinary host memory.
 *   - Ownership: the caller allocates and frees the device workspace, every
 *     output buffer and the CUDA stream.  A handle owns only host-side
 *     metadata; creating or destroying one allocates or frees no device
 *     memory.  Work is enqueued on the caller's stream.
 *   - Errors: every function returns an int.  0 (QSGS_OK) is success;
 *     positive values are run statuses; negative values are errors.  No C++
 *     exception crosses this interface.  qsgs_strerror() names every code.
 *   - Thread safety: a handle must not be used from two host threads at
 *     once; distinct handles are independent.
 */
#ifndef QSGS_H
#define QSGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes (>= 0) ---------------------------------------------- */
#define QSGS_OK 0          /* done: the solid count equals the target       */
#define QSGS_STALLED 1     /* no growth attempt can succeed any more         */
#define QSGS_MAX_STEPS 2   /* the total step limit (params.max_steps) hit    */
#define QSGS_RUNNING 3     /* this call's step budget is used up; call again */

/* ---- error codes (< 0) ------------------------------------------------ */
#define QSGS_ERR_INVALID -1   /* bad parameter or argument                   */
#define QSGS_ERR_WORKSPACE -2 /* workspace missing, misaligned or too small  */
#define QSGS_ERR_CUDA -3      /* a CUDA runtime call failed                  */
#define QSGS_ERR_TIMEOUT -4   /* a bounded device-side wait gave up          */
#define QSGS_ERR_STATE -5     /* call out of order (e.g. grow before seed)   */
#define QSGS_ERR_NOMEM -6     /* host allocation failed                      */

/* ---- fetch formats ---------------------------------------------------- */
/* Step kernels of a single realization (qsgs_set_mode). */
#define QSGS_MODE_LIETS 0     /* growth from the front list only (Algorithm 3) */
#define QSGS_MODE_FULLFIELD 1 /* comparator: full-field sweep (Algorithm 2)   */

#define QSGS_FMT_U8 0     /* uint8[N], 1 = solid, 0 = void, x fastest        */
#define QSGS_FMT_PACKED 1 /* uint32[nz*ny*W], W = ceil(nx/32): bit (x & 31)
                             of word (y + ny z) W + (x >> 5); bits at
                             x >= nx are 0                                   */

/* ---- fetch destinations (the dst_is_device argument of qsgs_fetch) ----- */
#define QSGS_DST_HOST 0        /* host memory of any kind                     */
#define QSGS_DST_DEVICE 1      /* device memory                               */
#define QSGS_DST_HOST_MAPPED 2 /* page-locked host memory mapped into the
                                  device's address space over the whole
                                  [dst, dst + bytes) (cudaHostAlloc, or
                                  cudaHostRegister of the whole range)        */

/* Generation parameters (the problem statement of Sec. 2.1 and Sec. 3.2).
 *   nx, ny, nz   grid dimensions, each >= 1, product < 2^32
 *   cd           seed (core) probability c_d in [0, 1]
 *   g_face       reference growth probability G_ref of the 6 face directions
 *   g_edge       ... of the 12 edge directions
 *   g_corner     ... of the 8 corner directions            (each in [0, 1])
 *   spacing_s    minimum L1 distance between seeds (0 or 1: no spacing)
 *   target_solid_fraction  phi_s in [0, 1], used when target_count == 0:
 *                Nt = floor(phi_s N + 0.5)
 *   target_count Nt directly (<= N); 0 = derive from the fraction
 *   seed         64-bit key of the realization's random numbers
 *   max_steps    total growth-step limit; 0 = none (2^32 - 1)          */
typedef struct qsgs_params {
  uint32_t nx, ny, nz;
  double cd;
  double g_face, g_edge, g_corner;
  uint32_t spacing_s;
  double target_solid_fraction;
  uint64_t target_count;
  uint64_t seed;
  uint32_t max_steps;
  uint32_t periodic;  /* 0: open domain; 1: periodic (a torus: neighbours and the
                         spacing distance wrap, the roll of Sec. 2.2); each
                         dimension must then be >= 3 */
} qsgs_params;

/* Run statistics.
 *   solid_count  current solid voxels c
 *   target_count Nt
 *   front_size   |A|, the current active front
 *   n_candidates Bernoulli candidates drawn by qsgs_seed
 *   n_seeds      seeds placed (after spacing and the cap at Nt)
 *   sum_front    sum over executed steps of |A_t| (growth work done)
 *   steps        growth steps executed
 *   status       QSGS_RUNNING while more steps can run, else the final
 *                status (QSGS_OK / QSGS_STALLED / QSGS_MAX_STEPS)           */
typedef struct qsgs_stats {
  uint64_t solid_count;
  uint64_t target_count;
  uint64_t front_size;
  uint64_t n_candidates;
  uint64_t n_seeds;
  uint64_t sum_front;
  uint32_t steps;
  int32_t status;
  uint64_t launches; /* kernels this handle has launched since creation  */
  uint64_t sum_draws; /* Philox blocks drawn by growth steps (sum over t)  */
} qsgs_stats;

/* One kernel class of the optional event profiler (qsgs_profile).
 *   name      "seed", "grow", "step_ctl", "trim", "front" or "fetch"
 *   launches  kernels of that class timed so far
 *   total_ms  their summed CUDA-event durations on the handle's stream  */
typedef struct qsgs_profile_entry {
  char name[16];
  uint64_t launches;
  double total_ms;
} qsgs_profile_entry;

typedef struct qsgs_handle qsgs_handle;

/* Library ABI version (major * 10000 + minor * 100 + patch). */
int qsgs_version(void);

/* Text of a status or error code; never NULL. */
const char* qsgs_strerror(int code);

/* Validates params and returns 0 with *nt, *t_seed, t_ref[0..2] set to the
 * integer forms of Nt, floor(cd 2^32) and floor(G 2^32) (face, edge,
 * corner), or QSGS_ERR_INVALID.  Host only; touches no device. */
int qsgs_check_params(const qsgs_params* params, uint64_t* nt, uint64_t* t_seed,
                      uint64_t t_ref[3]);

/* Device workspace bytes needed for params (0 if params are invalid).  The
 * workspace holds the run state, the bit grid and two claim grids of
 * nz*ny*ceil(nx/32) words each, the candidate list (the larger of that word
 * count and the seed-candidate capacity) and, when spacing_s >= 2, the
 * spacing scratch.  Seed arrays are sized for the Bernoulli candidate count
 * (N cd plus eight standard deviations plus 4096, at most N): a realization
 * with more candidates -- probability below 1e-15 -- makes qsgs_grow_until
 * and qsgs_query return QSGS_ERR_WORKSPACE.  Host only. */
size_t qsgs_workspace_bytes(const qsgs_params* params);

/* Binds a realization to a caller-allocated device workspace.
 *   params          host, copied
 *   dev_workspace   device, >= qsgs_workspace_bytes(params) bytes, 256-byte
 *                   aligned; owned by the caller and must outlive the handle
 *   bytes           its size
 *   cuda_stream     a cudaStream_t (NULL = the legacy default stream); all
 *                   work of this handle is enqueued on it
 *   out             host; receives the handle
 * Returns QSGS_OK, QSGS_ERR_INVALID, QSGS_ERR_WORKSPACE, QSGS_ERR_NOMEM or
 * QSGS_ERR_CUDA.  Enqueues the workspace initialisation (no host wait). */
int qsgs_create(const qsgs_params* params, void* dev_workspace, size_t bytes, void* cuda_stream,
                qsgs_handle** out);

/* Seeding, spacing, the seed cap and the initial front (Sec. 2.1 step 2,
 * Sec. 2.3 steps 1-2).  Asynchronous on the handle's stream.  May be
 * called again to restart the realization from scratch.
 * Returns QSGS_OK or QSGS_ERR_CUDA. */
int qsgs_seed(qsgs_handle* h);

/* Runs growth steps (Sec. 2.3 steps 3-5 with Eq. 1) until the target is
 * reached, growth stalls, params.max_steps is hit, or max_steps further
 * steps have run in this call (0 = no per-call limit).  Blocks until the
 * stream has finished them and fills *out (may be NULL).
 * Returns the status (QSGS_OK, QSGS_STALLED, QSGS_MAX_STEPS, QSGS_RUNNING)
 * or QSGS_ERR_STATE (not seeded), QSGS_ERR_CUDA, QSGS_ERR_TIMEOUT,
 * QSGS_ERR_WORKSPACE (more seed candidates than the workspace holds). */
int qsgs_grow_until(qsgs_handle* h, uint32_t max_steps, qsgs_stats* out);

/* Copies the phase map out.
 *   dst            host or device buffer (dst_is_device says which)
 *   bytes          its size: >= N for QSGS_FMT_U8, >= 4 nz ny W for
 *                  QSGS_FMT_PACKED
 *   fmt            QSGS_FMT_U8 or QSGS_FMT_PACKED
 *   dst_is_device  QSGS_DST_HOST, QSGS_DST_DEVICE or QSGS_DST_HOST_MAPPED
 * Blocks until the copy is complete.  Returns QSGS_OK, QSGS_ERR_INVALID
 * (fmt, size or destination kind), QSGS_ERR_STATE or QSGS_ERR_CUDA.  A U8
 * fetch to QSGS_DST_HOST memory stages through the candidate-list area of
 * the workspace in slabs of its size, so it is only allowed when the
 * realization has finished (status != QSGS_RUNNING).  To
 * QSGS_DST_HOST_MAPPED memory the device writes the uint8 map directly (no
 * staging, allowed at any time); a dst that the CUDA runtime does not know
 * as mapped host memory is served like QSGS_DST_HOST.  The caller
 * guarantees that the mapping covers all of [dst, dst + bytes). */
int qsgs_fetch(qsgs_handle* h, void* dst, size_t bytes, int fmt, int dst_is_device);

/* Synchronises the handle's stream and fills *out.  Returns QSGS_OK,
 * QSGS_ERR_CUDA, QSGS_ERR_TIMEOUT (a device wait gave up) or
 * QSGS_ERR_WORKSPACE (more seed candidates than the workspace holds). */
int qsgs_query(qsgs_handle* h, qsgs_stats* out);

/* Checkpoint and resume of a realization (Sec. 2.3, Algorithm 3: what one
 * growth step carries to the next is the phase array, the active front, the
 * step counter t and the solid count c_t; the front is a function of the
 * phase array, and every draw is keyed by (seed, voxel, t) and the rank of
 * its direction among the voxel's start-of-step targets, all of which the
 * snapshot restores, so a realization resumed from a snapshot takes
 * exactly the steps it would have taken uninterrupted).
 *
 * qsgs_snapshot_bytes: bytes of a snapshot of a realization with these
 * params (256-byte header, 256-byte run state, the packed grid: 512 + 4
 * nz ny ceil(nx/32)), or 0 if the params are invalid.  Host only.
 *
 * qsgs_snapshot: writes the realization's state between growth calls --
 * after qsgs_seed, or after a qsgs_grow_until that returned any status --
 * into dst.
 *   dst        host or device buffer of >= qsgs_snapshot_bytes bytes, owned
 *              by the caller; dst_kind is QSGS_DST_HOST, QSGS_DST_DEVICE or
 *              QSGS_DST_HOST_MAPPED (written like QSGS_DST_HOST)
 * Blocks until the snapshot is complete.  Returns QSGS_OK, QSGS_ERR_INVALID
 * (argument, size or kind), QSGS_ERR_STATE (not seeded, or a batch member
 * whose exact-target trim is still pending: call qsgs_batch_query first),
 * QSGS_ERR_TIMEOUT / QSGS_ERR_WORKSPACE (the run already failed) or
 * QSGS_ERR_CUDA.
 *
 * qsgs_restore: makes the handle continue the snapshotted realization.
 *   src        host or device buffer written by qsgs_snapshot; src_kind as
 *              dst_kind above; read during the call only
 * The handle must have been created with the same params (every field
 * equal); its earlier state, if any, is replaced.  Cells of earlier phases
 * and interactions (qsgs_set_blocked, qsgs_set_interaction) are not part of
 * a snapshot: set them on the handle as for the original run, before the
 * restore.  The next qsgs_grow_until (alone or in a batch) rebuilds the
 * candidate list from the grid first.  Blocks.  Returns QSGS_OK,
 * QSGS_ERR_INVALID (argument, size, kind, or a buffer that is not a
 * snapshot of a realization with these params) or QSGS_ERR_CUDA. */
size_t qsgs_snapshot_bytes(const qsgs_params* params);
int qsgs_snapshot(qsgs_handle* h, void* dst, size_t bytes, int dst_kind);
int qsgs_restore(qsgs_handle* h, const void* src, size_t bytes, int src_kind);

/* Turns the event profiler on (enable != 0) or off and clears its totals.
 * While on, every kernel launch of the handle is bracketed by CUDA events
 * on its stream; totals are collected at each host synchronisation.  Adds
 * a small per-launch cost, so timed runs leave it off.  Returns QSGS_OK,
 * QSGS_ERR_INVALID or QSGS_ERR_CUDA (event creation failed). */
int qsgs_set_profiling(qsgs_handle* h, int enable);

/* Copies up to max_entries profiler totals into out (host) and returns the
 * number of kernel classes (>= 0), or QSGS_ERR_INVALID. */
int qsgs_profile(qsgs_handle* h, qsgs_profile_entry* out, int max_entries);

/* Calibration probe: times Philox4x32-10 blocks drawn as fast as the GPU
 * can, with no memory traffic -- the ALU ceiling of the growth step, whose
 * work is one Philox block per front voxel and four targets of a direction
 * class.
 *   n_blocks   blocks to time (rounded up to whole threads)
 *   dev_out    device, 8 bytes: receives a checksum (keeps the work live)
 *   cuda_stream  stream to run on (NULL = legacy default stream)
 *   ms         host: elapsed milliseconds for n_blocks blocks
 * Blocks until done.  Returns QSGS_OK, QSGS_ERR_INVALID or QSGS_ERR_CUDA. */
int qsgs_bench_philox(uint64_t n_blocks, void* dev_out, void* cuda_stream, double* ms);

/* Calibration probes of the L2 roof (no counterpart in the paper).  The
 * growth step reads neighbour words of an L2-resident bit grid and claims
 * voxels with fire-and-forget atomicOr; these two kernels measure what the
 * L2 itself sustains for that kind of traffic on this GPU, so a step's
 * bytes and claims can be set against a measured peak.
 *
 * qsgs_bench_l2_read: reads the whole buffer `passes` times with 16-byte
 * loads that bypass L1 (each pass shifts every thread to other elements),
 * after one untimed pass that brings it into L2.
 *   dev_buf   device, read only, 16-byte aligned; bytes a multiple of 16,
 *             at least 64 bytes per probe thread (4 blocks of 512 threads
 *             per SM: 19.9 MB on 152 SMs) and below 64 GiB; pick it well
 *             below the L2 size (129 MB) to stay resident
 *   dev_out   device, 8 bytes, 8-byte aligned: receives a checksum
 *   ms        host: elapsed milliseconds of the timed passes
 *             (bytes read = bytes * passes)
 * qsgs_bench_l2_atomic: n_ops atomicOr reductions (no value returned) to
 * scattered words of the buffer, after an untimed warm-up.
 *   dev_buf   device, 4-byte aligned, bytes / 4 words (< 2^32); its
 *             contents are overwritten
 *   ms        host: elapsed milliseconds scaled to n_ops reductions
 * Both block until done and return QSGS_OK, QSGS_ERR_INVALID or
 * QSGS_ERR_CUDA. */
int qsgs_bench_l2_read(const void* dev_buf, size_t bytes, uint32_t passes, void* dev_out,
                       void* cuda_stream, double* ms);
int qsgs_bench_l2_atomic(void* dev_buf, size_t bytes, uint64_t n_ops, void* cuda_stream,
                         double* ms);

/* Releases the handle (host memory only).  NULL is ignored. */
void qsgs_destroy(qsgs_handle* h);

/* Tuning knob: thread blocks of the growth kernel (0 = one wave: as many
 * blocks as all SMs hold at once).  Results do not depend on it.  Returns
 * QSGS_OK or QSGS_ERR_INVALID. */
int qsgs_set_grow_blocks(qsgs_handle* h, uint32_t blocks);

/* Tuning knob: front tile of the growth kernel -- the number of 32-word
 * chunks of the candidate list a warp takes per grab from the kernel's
 * chunk dispenser (1..16; 0 = 1).  Larger tiles mean fewer dispenser
 * atomics and coarser load balance.  Results do not depend on it.  Returns
 * QSGS_OK or QSGS_ERR_INVALID. */
int qsgs_set_grow_tile(qsgs_handle* h, uint32_t chunks);

/* Comparator switch (Algorithm 2 of Sec. 2.2 against the list-driven
 * Algorithm 3).  QSGS_MODE_FULLFIELD makes every later growth step of this
 * handle a full-field sweep: every voxel draws every Philox block each step
 * (the work of the vectorized procedure, which generates a random field per
 * direction over the whole grid) and the successes are claimed as in the
 * list-driven step, so the realization is the same bit for bit; only its
 * cost and stats.sum_draws (every block drawn) differ.  QSGS_MODE_LIETS
 * (the default) switches back.  Batches always use the list-driven step;
 * qsgs_time_grow always times it.  Returns QSGS_OK, QSGS_ERR_INVALID, or
 * QSGS_ERR_STATE for QSGS_MODE_FULLFIELD on an interacting phase
 * (qsgs_set_interaction). */
int qsgs_set_mode(qsgs_handle* h, int mode);

/* Failure-detection knob (no counterpart in the paper): how many polls a
 * device-side wait of this handle's order-preserving passes (seeding,
 * first candidate list, trim, front count) makes before it gives up,
 * records the timeout and lets the kernel finish; the next query or grow
 * call then returns QSGS_ERR_TIMEOUT (the realization is invalid; reseed).
 * 0 = the default 2^20 polls (about a second).  Returns QSGS_OK or
 * QSGS_ERR_INVALID. */
int qsgs_set_spin_limit(qsgs_handle* h, uint32_t polls);

/* Later growing phases (Sec. 2.1 step 4 with independent discrete phases,
 * reading R12): a phase is generated on the cells no earlier phase holds.
 *   dev_blocked  device, read only, owned by the caller: the packed grid
 *                (QSGS_FMT_PACKED layout of this handle's dims) of the cells
 *                of all earlier phases; NULL = none (the first phase).  It
 *                must stay valid and unchanged from qsgs_seed to the last
 *                fetch; 4-byte aligned.
 * Blocked cells are never seeds, never void targets and never count as void
 * neighbours; targets stay fractions of the whole domain.  Set it before
 * qsgs_seed.  Batches use each member's own setting.  Returns QSGS_OK or
 * QSGS_ERR_INVALID. */
int qsgs_set_blocked(qsgs_handle* h, const void* dev_blocked);

/* Interacting growing phases (Sec. 2.1 step 4, second case; reading R13):
 * the phase grows into cells of earlier phases as well.
 *   dev_labels  device, read only, owned by the caller: one byte per voxel
 *               (x fastest), 0 = unassigned, m = a cell of earlier phase m;
 *               NULL clears the interaction (and the blocked cells).  It must
 *               stay valid and unchanged from qsgs_seed to the last fetch.
 *   probs       host: probs[3 (m - 1) + k] = the interaction probability
 *               I^{n,m} in [0, 1] of class k (face, edge, corner) for the
 *               labels m = 1 .. n_labels; read during the call only
 *   n_labels    0 .. 255
 *   dev_scratch device, owned by the caller, qsgs_interaction_bytes(params)
 *               bytes, 16-byte aligned: packed grids and thresholds the
 *               handle derives from the labels; valid as long as dev_labels
 * A move along class k from a voxel of this phase into a cell of phase m
 * succeeds with probability floor(I^{n,m}_k 2^32) / 2^32 (a constant: Eq. 1
 * scales the growth probabilities only); the cell becomes this phase's and
 * counts towards its target.  Voids are entered as in an independent phase;
 * seeds only fall on unassigned cells; a voxel with a void or an enterable
 * neighbour is active.  With all I = 0 this is qsgs_set_blocked of the
 * labelled cells.  Set it before qsgs_seed.  Single realizations in
 * QSGS_MODE_LIETS only: batches reject such members and qsgs_set_mode
 * rejects QSGS_MODE_FULLFIELD while it is set.  Returns QSGS_OK,
 * QSGS_ERR_INVALID, QSGS_ERR_WORKSPACE (scratch too small), QSGS_ERR_STATE
 * (full-field mode) or QSGS_ERR_CUDA. */
size_t qsgs_interaction_bytes(const qsgs_params* params);
int qsgs_set_interaction(qsgs_handle* h, const uint8_t* dev_labels, const double* probs,
                         uint32_t n_labels, void* dev_scratch, size_t scratch_bytes);

/* Phase-map composition: writes `label` into dev_dst[v] (device uint8 map
 * of N bytes, x fastest) for every solid voxel v of this realization and
 * leaves the other bytes unchanged.  Blocks.  Returns QSGS_OK,
 * QSGS_ERR_INVALID, QSGS_ERR_STATE (not seeded) or QSGS_ERR_CUDA. */
int qsgs_fetch_label(qsgs_handle* h, void* dev_dst, size_t bytes, uint8_t label);

/* ORs this realization's packed grid into dev_dst (device, >= 4 nz ny W
 * bytes, 4-byte aligned): accumulates the blocked grid of the next phase.
 * Blocks.  Returns QSGS_OK, QSGS_ERR_INVALID, QSGS_ERR_STATE or
 * QSGS_ERR_CUDA. */
int qsgs_fetch_or(qsgs_handle* h, void* dev_dst, size_t bytes);

/* Tuning probe (no counterpart in the paper): replays the growth kernel of
 * the handle's next step `reps` times with `grow_blocks` thread blocks (0 =
 * default) and writes the mean milliseconds per launch to *ms (host).  The
 * realization is left exactly as it was (the step's claims and marks are
 * idempotent and its counters are restored), so an autotuner can time grid
 * sizes on the real mid-run state.  The handle must be between steps of a
 * running realization (after qsgs_grow_until returned QSGS_RUNNING).
 * Blocks.  Returns QSGS_OK, QSGS_ERR_INVALID, QSGS_ERR_STATE or
 * QSGS_ERR_CUDA. */
int qsgs_time_grow(qsgs_handle* h, uint32_t grow_blocks, uint32_t reps, double* ms);

/* Front size of a packed grid, without any allocation (no counterpart in the
 * paper).  Counts the solid voxels with a void in-domain 26-neighbour (the
 * front |A| of Sec. 2.3, the front_size qsgs_query reports at the end of a
 * run) of a grid in the library's packed layout: bit x of word
 * (z * ny + y) * ceil(nx / 32) + x / 32, pad bits zero.
 *
 * For callers that may not allocate device memory: code that runs under a
 * pool-only allocator (a framework that owns all device memory, where a
 * stray cudaMalloc would bypass its accounting or fail once the pool holds
 * the device), or a real-time path where an allocation may block or fail.
 * The call uses 64 KiB of scratch that lives in the library's own device
 * image (a static __device__ array, held by every device that loads the
 * library until the process exits) and allocates nothing, on the device or
 * the host.
 *   dev_grid     device, read only, ceil(nx/32) * ny * nz words
 *   nx, ny, nz   grid size (nx * ny * nz < 2^32)
 *   cuda_stream  stream to run on (NULL = legacy default stream)
 *   front_out    host: receives the count
 * Limit: at most 16,707,584 words (e.g. 800^3 or 32 x 4096 x 4079 fit,
 * 1024^3 does not); larger grids return QSGS_ERR_WORKSPACE before touching
 * the device.  The first call on a device does the set-up: it looks up the
 * scratch address with that device current (this may load the library's
 * device code), so make that first call before any stream capture.  Each
 * call zeroes the scratch it uses (run state and tile status words) on the
 * stream before the count.
 * Calls share the one scratch per device: overlapping calls (other streams
 * or host threads) race and must be serialised by the caller.  The call
 * copies the count to the host and synchronises cuda_stream before it
 * returns.  Returns QSGS_OK, QSGS_ERR_INVALID, QSGS_ERR_WORKSPACE,
 * QSGS_ERR_TIMEOUT or QSGS_ERR_CUDA. */
int qsgs_front_count_static(const uint32_t* dev_grid, uint32_t nx, uint32_t ny, uint32_t nz,
                            void* cuda_stream, uint64_t* front_out);

/* ---- batches ------------------------------------------------------------
 * A batch advances many realizations (its members: ordinary handles, each
 * with its own workspace) with the same launches: one growth launch over
 * the concatenation of all members' candidate lists, one commit scan over
 * all members' words and one control kernel with a thread per member, per
 * step, replayed from one CUDA graph until no member has a step left.
 * Every member gets exactly the result it gets alone (its draws are keyed
 * by its own seed, step and voxel).  The paper runs one realization at a
 * time; batching serves the many realizations that uncertainty
 * quantification needs (Sec. 1).
 *
 * Ownership: the caller owns the batch workspace (device) and stream and
 * the member handles, which must outlive their membership.  A batch holds
 * host metadata, a few events and kSeedStreams (8) private streams used to
 * seed members concurrently. */
typedef struct qsgs_batch qsgs_batch;

/* Device workspace bytes for up to max_members (<= 1024) members whose
 * words (nz*ny*ceil(nx/32) each, rounded up to 32) total at most max_words
 * (< 2^32).  0 if the limits are invalid.  Host only. */
size_t qsgs_batch_workspace_bytes(uint32_t max_members, uint64_t max_words);

/* Creates an empty batch on a caller workspace (256-byte aligned) and
 * stream (a non-default stream enables the CUDA graph).  Returns QSGS_OK,
 * QSGS_ERR_INVALID, QSGS_ERR_WORKSPACE, QSGS_ERR_NOMEM or QSGS_ERR_CUDA. */
int qsgs_batch_create(uint32_t max_members, uint64_t max_words, void* dev_workspace, size_t bytes,
                      void* cuda_stream, qsgs_batch** out);

/* Sets the members (host array of n handles; replaces the previous set).
 * Members keep their run state: a member may join mid-run and leave
 * mid-run (qsgs_grow_until on a handle that left rebuilds its candidate
 * list first).  The batch stream waits for each member's own stream.
 * Blocks until the member table is on the device.  Must not be called while
 * an advance is in flight.  Returns QSGS_OK, QSGS_ERR_INVALID (also for a
 * handle of an interacting phase, qsgs_set_interaction), QSGS_ERR_WORKSPACE
 * (too many words) or QSGS_ERR_CUDA. */
int qsgs_batch_set_members(qsgs_batch* b, qsgs_handle* const* members, uint32_t n);

/* Seeds (or re-seeds) every member, up to 16 at a time on private streams;
 * the batch stream waits for all.  On a non-default stream, with no
 * profiler on, the first call for a set of members captures all of their
 * seeding into one CUDA graph that later calls replay; changing the
 * members or a member's settings (qsgs_set_*) makes the next call capture
 * again.  Asynchronous.  Returns QSGS_OK or an error. */
int qsgs_batch_seed(qsgs_batch* b);

/* Enqueues on the batch stream: every running member advances until it is
 * done, stalls, hits its step limit or has run max_steps more steps (0 = no
 * per-call limit).  Asynchronous; qsgs_batch_query waits.  Returns QSGS_OK,
 * QSGS_ERR_STATE (a member not seeded) or QSGS_ERR_CUDA. */
int qsgs_batch_advance(qsgs_batch* b, uint32_t max_steps);

/* Waits for the batch stream, runs the exact-target trim and the final
 * front count of members whose run has ended, and fills per_member[0..n)
 * (host array, may be NULL if n = 0) in member order.  The members' run
 * states are gathered into the batch workspace on the batch stream and read
 * with one copy.  Returns QSGS_OK,
 * QSGS_ERR_TIMEOUT, QSGS_ERR_INVALID or QSGS_ERR_CUDA. */
int qsgs_batch_query(qsgs_batch* b, qsgs_stats* per_member, uint32_t n);

/* qsgs_batch_seed + qsgs_batch_advance + qsgs_batch_query. */
int qsgs_batch_run(qsgs_batch* b, uint32_t max_steps, qsgs_stats* per_member, uint32_t n);

/* Tuning knob: thread blocks of the batched growth kernel (0 = one wave: as
 * many blocks as all SMs hold at once). */
int qsgs_batch_set_grow_blocks(qsgs_batch* b, uint32_t blocks);

/* Tuning knob: front tile of the batched growth kernel (as
 * qsgs_set_grow_tile; 1..16, 0 = 1). */
int qsgs_batch_set_grow_tile(qsgs_batch* b, uint32_t chunks);

/* Event profiler of the batch's own launches (see qsgs_set_profiling);
 * while on, advances use direct launches instead of the graph. */
int qsgs_batch_set_profiling(qsgs_batch* b, int enable);
int qsgs_batch_profile(qsgs_batch* b, qsgs_profile_entry* out, int max_entries);

/* Releases the batch's host metadata, events and private streams (not the
 * members or the workspace).  NULL is ignored. */
void qsgs_batch_destroy(qsgs_batch* b);

#ifdef __cplusplus
}
#endif
#endif /* QSGS_H */
