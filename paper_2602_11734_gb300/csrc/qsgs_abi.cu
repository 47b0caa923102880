// qsgs_abi.cu -- the extern "C" boundary of libqsgs (see include/qsgs.h).
//
// Host-side only: parameter validation, workspace carve-up, launch order
// and synchronisation.  All generation work runs in the kernels of
// qsgs_kernels.cu; nothing here computes voxels.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <cstddef>
#include <atomic>
#include <new>
#include <utility>
#include <vector>

#include "../../include/qsgs.h"
#include "qsgs_launch.h"
#include "qsgs_scan.cuh"

using namespace qsgs;

namespace {

constexpr size_t kAlign = 256;
constexpr uint32_t kSpinLimit = 1u << 20;  // bounded look-back polls (about 1 s)
constexpr uint32_t kStepsPerSync = 8;      // steps enqueued between host checks

size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

struct Layout {
  size_t state, scan_status, grid, aux, mark, list, cell_count, cell_start, cell_items, decision;
  size_t conf_off, adj, total;
  uint64_t adj_cap;
  uint64_t cand_cap;  // seed candidates the workspace holds
  uint64_t list_bytes;  // size of the list area (also the u8 fetch staging slab)
  uint64_t ntiles;
  CellGeomHost cg;
};

struct Ints {
  uint64_t nt, t_seed, t_ref[3];
};

int check_params(const qsgs_params* p, Ints* out) {
  if (!p) return QSGS_ERR_INVALID;
  if (p->nx == 0 || p->ny == 0 || p->nz == 0) return QSGS_ERR_INVALID;
  if (p->periodic > 1) return QSGS_ERR_INVALID;
  if (p->periodic && (p->nx < 3 || p->ny < 3 || p->nz < 3)) return QSGS_ERR_INVALID;
  const uint64_t n = (uint64_t)p->nx * p->ny * p->nz;
  if (n >= (1ull << 32)) return QSGS_ERR_INVALID;
  const double vals[4] = {p->cd, p->g_face, p->g_edge, p->g_corner};
  for (double v : vals)
    if (!(v >= 0.0 && v <= 1.0)) return QSGS_ERR_INVALID;
  uint64_t nt;
  if (p->target_count != 0) {
    nt = p->target_count;
  } else {
    if (!(p->target_solid_fraction >= 0.0 && p->target_solid_fraction <= 1.0)) return QSGS_ERR_INVALID;
    nt = (uint64_t)std::floor(p->target_solid_fraction * (double)n + 0.5);
  }
  if (nt > n) return QSGS_ERR_INVALID;
  const double two32 = 4294967296.0;
  out->nt = nt;
  out->t_seed = (uint64_t)std::floor(p->cd * two32);
  out->t_ref[0] = (uint64_t)std::floor(p->g_face * two32);
  out->t_ref[1] = (uint64_t)std::floor(p->g_edge * two32);
  out->t_ref[2] = (uint64_t)std::floor(p->g_corner * two32);
  return QSGS_OK;
}

// Seed candidates a workspace provides for: the number of candidates is
// Binomial(N, P) with P = floor(cd 2^32) / 2^32, so the mean plus eight
// standard deviations plus 4096 (capped at N) is exceeded with probability
// below 1e-15; a run that exceeds it reports QSGS_ERR_WORKSPACE.
uint64_t candidate_capacity(uint64_t n, double cd) {
  const double pr = std::floor(cd * 4294967296.0) / 4294967296.0;
  const double mean = (double)n * pr;
  const double cap = mean + 8.0 * std::sqrt(mean * (1.0 - pr)) + 4096.0;
  return cap >= (double)n ? n : (uint64_t)std::ceil(cap);
}

Layout make_layout(const qsgs_params* p) {
  Layout L{};
  const uint64_t n = (uint64_t)p->nx * p->ny * p->nz;
  const uint64_t W = (p->nx + 31) / 32;
  const uint64_t nwords = W * p->ny * p->nz;
  L.cand_cap = candidate_capacity(n, p->cd);
  uint64_t ncells = 0;
  if (p->spacing_s >= 2) {
    const uint32_t s = p->spacing_s;
    if (p->periodic) {  // cells of width >= s tile the torus exactly
      auto cells = [s](uint32_t n) { return n / s ? n / s : 1u; };
      L.cg = CellGeomHost{s, cells(p->nx), cells(p->ny), cells(p->nz)};
    } else {
      L.cg = CellGeomHost{s, (p->nx + s - 1) / s, (p->ny + s - 1) / s, (p->nz + s - 1) / s};
    }
    ncells = (uint64_t)L.cg.ncx * L.cg.ncy * L.cg.ncz;
  }
  uint64_t max_items = n > nwords ? n : nwords;
  if (ncells > max_items) max_items = ncells;
  L.ntiles = (max_items + kScanTile - 1) / kScanTile + 1;
  size_t off = 0;
  L.state = off; off = align_up(off + sizeof(RunState));
  L.scan_status = off; off = align_up(off + L.ntiles * sizeof(unsigned long long));
  L.grid = off; off = align_up(off + nwords * 4);
  L.aux = off; off = align_up(off + 2 * nwords * 4);  // claim grids of even / odd steps
  L.mark = off; off = align_up(off + 2 * (nwords / 32 + 1) * 4);  // marks, touched bits
  // Seed candidates (at most cand_cap), then the candidate word list (at
  // most nwords); u32 entries.
  L.list_bytes = (L.cand_cap > nwords ? L.cand_cap : nwords) * 4;
  L.list = off; off = align_up(off + L.list_bytes);
  if (ncells) {
    const uint64_t cap = L.cand_cap;
    L.cell_count = off; off = align_up(off + ncells * 4);
    L.cell_start = off; off = align_up(off + (ncells + 1) * 4);
    L.cell_items = off; off = align_up(off + cap * 4);
    L.decision = off; off = align_up(off + cap);
    L.conf_off = off; off = align_up(off + (cap + 1) * 4);
    // Conflict lists: 16 per candidate (more: the list-free fallback runs).
    L.adj_cap = 16 * cap < n ? 16 * cap : n;
    L.adj = off; off = align_up(off + L.adj_cap * 4);
  }
  L.total = off;
  return L;
}

}  // namespace

struct qsgs_handle {
  qsgs_params p;
  Ints ints;
  Geom g;
  Layout L;
  cudaStream_t stream;
  uint8_t* ws;
  RunState* st;
  unsigned long long* scan_status;
  uint32_t* grid;
  uint32_t* aux;
  uint32_t* list;
  uint32_t* mark;
  uint32_t *cell_count, *cell_start, *cell_items, *conf_off, *adj;
  uint8_t* decision;
  uint32_t k0, k1;
  uint32_t grow_blocks;
  uint32_t grow_tile;
  int mode;  // QSGS_MODE_LIETS or QSGS_MODE_FULLFIELD
  uint32_t spin_limit;  // polls before a device-side wait gives up
  bool seeded;
  cudaError_t last_cuda;
  Tracer tracer;
  // Whole-run graph: while (active) { grow; front; control } then the
  // exact-target epilogue.  Built on first use; direct launches when the
  // profiler is on, the stream is the legacy default stream, or building
  // the graph failed.
  cudaGraph_t graph;
  cudaGraphExec_t graph_exec;
  bool graph_tried;
  uint32_t iters_seen;
  // Set while a batch advances the realization: its own candidate list is
  // out of date and is rebuilt before qsgs_grow_until continues alone.
  bool list_stale;
  // The exact-target epilogue has run since the run ended (batch members).
  bool finalized;
  // Changes whenever a setter changes what seeding launches (a batch's
  // captured seeding graph is valid only for the versions it saw).
  uint64_t seed_version;
  // Interacting phase (R13): the label thresholds copied to the scratch, and
  // the device pointers of GeomInter (nullptr for an independent phase).
  std::vector<uint32_t> enter_thr;
  const uint32_t* dev_enter;
  const uint8_t* dev_labels;
  const uint32_t* dev_enter_thr;
};

namespace {

std::atomic<uint64_t> g_seed_versions{0};
uint64_t next_seed_version() { return ++g_seed_versions; }

int cuda_fail(qsgs_handle* h, cudaError_t e) {
  if (h) h->last_cuda = e;
  return QSGS_ERR_CUDA;
}

int read_state(qsgs_handle* h, RunState* out) {
  cudaError_t e = cudaMemcpyAsync(out, h->st, sizeof(RunState), cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e);
  e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e);
  e = h->tracer.collect();
  if (e != cudaSuccess) return cuda_fail(h, e);
  if (out->error & kErrTimeout) return QSGS_ERR_TIMEOUT;
  if (out->error & kErrOverflow) return QSGS_ERR_WORKSPACE;
  return QSGS_OK;
}

void fill_stats(const qsgs_handle* h, const RunState& s, qsgs_stats* out) {
  if (!out) return;
  out->solid_count = s.solid;
  out->target_count = s.nt;
  out->front_size = s.front_n;
  (void)s.front_words;
  out->n_candidates = s.cand_n;
  out->n_seeds = s.acc_n;
  out->sum_front = s.sum_front;
  out->steps = s.t;
  out->status = s.status == kRunning ? QSGS_RUNNING : s.status;
  out->launches = h->tracer.launches;
  out->sum_draws = s.sum_draws;
}

StepBuffers step_buffers(const qsgs_handle* h) {
  return StepBuffers{h->st,   h->scan_status, h->grid,       h->aux,
                     h->mark, h->list,        h->dev_enter,  h->dev_labels,
                     h->dev_enter_thr};
}

// Seeding, spacing, the seed cap and the initial candidate list (Sec. 2.1
// step 2, Sec. 2.3 steps 1-2), enqueued on `stream`.
int seed_on_stream(qsgs_handle* h, cudaStream_t stream) {
  const size_t grids = (size_t)h->g.nwords * 4;
  cudaError_t e = cudaMemsetAsync(h->grid, 0, grids, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->aux, 0, 2 * grids, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->mark, 0, 2 * (size_t)bitmap_words(h->g) * 4, stream);
  if (e != cudaSuccess) return cuda_fail(h, e);
  StateInit init{};
  init.nt = h->ints.nt;
  for (int k = 0; k < 3; ++k) init.t_ref[k] = h->ints.t_ref[k];
  init.t_seed = h->ints.t_seed;
  init.max_steps = h->p.max_steps ? h->p.max_steps : 0xFFFFFFFFu;
  e = launch_init_state(h->st, init, stream, h->tracer);
  if (e != cudaSuccess) return cuda_fail(h, e);
  SeedBuffers b{h->st,         h->scan_status, h->grid,     h->aux,
                h->list,       h->mark,        h->cell_count,  h->cell_start, h->cell_items,
                h->decision,   h->conf_off,    h->adj,        h->L.adj_cap,
                h->L.cand_cap, h->L.cg};
  e = launch_seed(h->g, b, h->k0, h->k1, h->spin_limit, stream, h->tracer);
  if (e != cudaSuccess) return cuda_fail(h, e);
  h->seeded = true;
  h->list_stale = false;
  h->finalized = false;
  h->iters_seen = 0;
  return QSGS_OK;
}

void destroy_graph(qsgs_handle* h) {
  if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
  if (h->graph) cudaGraphDestroy(h->graph);
  h->graph_exec = nullptr;
  h->graph = nullptr;
}

// Captures the whole growth loop of this handle into one graph: a while
// node whose body is kGraphStepsPerIteration steps (each one's last kernel
// sets the loop condition), followed by the exact-target epilogue.  Kernel arguments are fixed per
// handle, so the graph is built once and relaunched by every call.
constexpr int kGraphStepsPerIteration = 4;

cudaError_t build_graph(qsgs_handle* h) {
  cudaError_t e = cudaGraphCreate(&h->graph, 0);
  if (e != cudaSuccess) return e;
  cudaGraphConditionalHandle cond;
  e = cudaGraphConditionalHandleCreate(&cond, h->graph, 1, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) return e;
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = cond;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t loop;
  e = cudaGraphAddNode(&loop, h->graph, nullptr, nullptr, 0, &cp);
  if (e != cudaSuccess) return e;
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  const StepBuffers b = step_buffers(h);
  Tracer capture_tracer;  // launches inside the graph are counted from iters
  e = cudaStreamBeginCaptureToGraph(h->stream, body, nullptr, nullptr, 0,
                                    cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  // kGraphStepsPerIteration steps per evaluation of the loop condition: each
  // step's kernels return at once when the step is not active, so the copies
  // after the last step of a run cost a few microseconds of empty launches,
  // against one conditional evaluation saved per step otherwise.
  cudaError_t le = cudaSuccess;
  for (int u = 0; u < kGraphStepsPerIteration && le == cudaSuccess; ++u)
    le = launch_step(h->g, b, h->k0, h->k1, kSpinLimit, GrowShape{h->grow_blocks, h->grow_tile},
                     h->stream, capture_tracer, cond, 1, h->mode == QSGS_MODE_FULLFIELD);
  cudaGraph_t captured = nullptr;
  e = cudaStreamEndCapture(h->stream, &captured);
  if (le != cudaSuccess) return le;
  if (e != cudaSuccess) return e;
  e = cudaStreamBeginCaptureToGraph(h->stream, h->graph, &loop, nullptr, 1,
                                    cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  le = launch_epilogue(h->g, b, h->spin_limit, h->stream, capture_tracer);
  e = cudaStreamEndCapture(h->stream, &captured);
  if (le != cudaSuccess) return le;
  if (e != cudaSuccess) return e;
  return cudaGraphInstantiate(&h->graph_exec, h->graph, 0);
}


// ---------------------------------------------------------------------------
// Batches.
// ---------------------------------------------------------------------------
constexpr uint32_t kSeedStreams = 16;  // members seeded concurrently

struct BatchLayout {
  size_t state, descs, states, list, total;
};

BatchLayout make_batch_layout(uint32_t max_members, uint64_t max_words) {
  BatchLayout L{};
  size_t off = 0;
  L.state = off; off = align_up(off + sizeof(BatchState));
  L.descs = off; off = align_up(off + (size_t)max_members * sizeof(MemberDesc));
  L.states = off; off = align_up(off + (size_t)max_members * sizeof(RunState));
  L.list = off; off = align_up(off + (max_words ? max_words : 1) * 4);
  L.total = off;
  return L;
}

}  // namespace

struct qsgs_batch {
  uint32_t max_members;
  uint64_t max_words;
  BatchLayout L;
  cudaStream_t stream;
  uint8_t* ws;
  BatchBuffers buf;
  std::vector<qsgs_handle*> members;
  std::vector<MemberDesc> host_descs;
  std::vector<RunState> host_states;
  uint32_t grow_blocks;
  uint32_t grow_tile;
  uint32_t iters_seen;
  cudaGraph_t graph;
  cudaGraphExec_t graph_exec;
  bool graph_tried;
  cudaStream_t seed_streams[kSeedStreams];
  cudaEvent_t seed_events[kSeedStreams];
  cudaEvent_t fork;
  // Every member's seeding captured into one graph, for the members (and
  // their seed versions) in seed_key; rebuilt when they change.
  cudaGraphExec_t seed_exec;
  std::vector<std::pair<const qsgs_handle*, uint64_t>> seed_key;
  bool seed_graph_failed;  // capture failed for seed_key: launch directly
  Tracer tracer;
  cudaError_t last_cuda;
};

namespace {

void destroy_batch_graph(qsgs_batch* b) {
  if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->graph_exec = nullptr;
  b->graph = nullptr;
}

// [step limits, prologue commit, prologue control] then while (any member
// active) { batched growth, commit, control }.  Nothing in it depends on
// the membership, which the kernels read from the workspace.
cudaError_t build_batch_graph(qsgs_batch* b) {
  cudaError_t e = cudaGraphCreate(&b->graph, 0);
  if (e != cudaSuccess) return e;
  cudaGraphConditionalHandle cond;
  e = cudaGraphConditionalHandleCreate(&cond, b->graph, 0, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) return e;
  Tracer capture_tracer;
  e = cudaStreamBeginCaptureToGraph(b->stream, b->graph, nullptr, nullptr, 0,
                                    cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t le = launch_batch_prologue(b->buf, kSpinLimit, b->stream, capture_tracer, cond, 1);
  cudaGraph_t captured = nullptr;
  e = cudaStreamEndCapture(b->stream, &captured);
  if (le != cudaSuccess) return le;
  if (e != cudaSuccess) return e;
  // The loop node goes after everything captured so far.
  size_t n_nodes = 0;
  e = cudaGraphGetNodes(b->graph, nullptr, &n_nodes);
  if (e != cudaSuccess) return e;
  std::vector<cudaGraphNode_t> nodes(n_nodes);
  e = cudaGraphGetNodes(b->graph, nodes.data(), &n_nodes);
  if (e != cudaSuccess) return e;
  std::vector<cudaGraphNode_t> leaves;
  for (auto nd : nodes) {
    size_t n_out = 0;
    e = cudaGraphNodeGetDependentNodes(nd, nullptr, nullptr, &n_out);
    if (e != cudaSuccess) return e;
    if (n_out == 0) leaves.push_back(nd);
  }
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = cond;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t loop;
  e = cudaGraphAddNode(&loop, b->graph, leaves.data(), nullptr, leaves.size(), &cp);
  if (e != cudaSuccess) return e;
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  e = cudaStreamBeginCaptureToGraph(b->stream, body, nullptr, nullptr, 0,
                                    cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  le = launch_batch_step(b->buf, kSpinLimit, GrowShape{b->grow_blocks, b->grow_tile}, b->stream,
                         capture_tracer, cond, 1);
  e = cudaStreamEndCapture(b->stream, &captured);
  if (le != cudaSuccess) return le;
  if (e != cudaSuccess) return e;
  return cudaGraphInstantiate(&b->graph_exec, b->graph, 0);
}

int batch_fail(qsgs_batch* b, cudaError_t e) {
  if (b) b->last_cuda = e;
  return QSGS_ERR_CUDA;
}

}  // namespace

namespace {

// ---------------------------------------------------------------------------
// Snapshots: [0, 256) header, [256, 512) the run state, then the packed
// grid (4 nwords bytes).
// ---------------------------------------------------------------------------
constexpr char kSnapMagic[8] = {'Q', 'S', 'G', 'S', 'S', 'N', 'P', '1'};
constexpr uint32_t kSnapVersion = 1;
constexpr size_t kSnapHeader = 256;
constexpr size_t kSnapState = kSnapHeader + sizeof(RunState);

struct SnapHeader {
  char magic[8];
  uint32_t version;
  uint32_t nwords;
  uint64_t total_bytes;
  qsgs_params params;
};
static_assert(sizeof(SnapHeader) <= kSnapHeader, "snapshot header fits its slot");
static_assert(sizeof(RunState) == 256, "run state slot");

size_t snapshot_bytes(const Geom& g) { return kSnapState + (size_t)g.nwords * 4; }

// The generation parameters two handles must share for a snapshot of one
// to continue on the other (compared field by field: no padding bytes).
bool same_params(const qsgs_params& a, const qsgs_params& b) {
  return a.nx == b.nx && a.ny == b.ny && a.nz == b.nz && a.cd == b.cd && a.g_face == b.g_face &&
         a.g_edge == b.g_edge && a.g_corner == b.g_corner && a.spacing_s == b.spacing_s &&
         a.target_solid_fraction == b.target_solid_fraction && a.target_count == b.target_count &&
         a.seed == b.seed && a.max_steps == b.max_steps && a.periodic == b.periodic;
}

cudaMemcpyKind copy_kind(int kind, bool to_device_buffer) {
  if (kind == QSGS_DST_DEVICE) return cudaMemcpyDeviceToDevice;
  return to_device_buffer ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost;
}

// Times `fn` (which enqueues one probe launch on s) between two events.
template <class F>
int time_probe(cudaStream_t s, F fn, float* ms) {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (e == cudaSuccess) e = cudaEventRecord(a, s);
  if (e == cudaSuccess) e = fn();
  if (e == cudaSuccess) e = cudaEventRecord(b, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  return e == cudaSuccess ? QSGS_OK : QSGS_ERR_CUDA;
}

}  // namespace

extern "C" {

int qsgs_version(void) { return 100; }

const char* qsgs_strerror(int code) {
  switch (code) {
    case QSGS_OK: return "ok: target solid count reached";
    case QSGS_STALLED: return "stalled: no growth attempt can succeed";
    case QSGS_MAX_STEPS: return "step limit reached";
    case QSGS_RUNNING: return "running: call budget used, more steps remain";
    case QSGS_ERR_INVALID: return "invalid parameter or argument";
    case QSGS_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case QSGS_ERR_CUDA: return "CUDA runtime error";
    case QSGS_ERR_TIMEOUT: return "bounded device wait timed out";
    case QSGS_ERR_STATE: return "call out of order";
    case QSGS_ERR_NOMEM: return "host allocation failed";
    default: return "unknown code";
  }
}

int qsgs_check_params(const qsgs_params* params, uint64_t* nt, uint64_t* t_seed, uint64_t t_ref[3]) {
  Ints ints{};
  const int rc = check_params(params, &ints);
  if (rc != QSGS_OK) return rc;
  if (nt) *nt = ints.nt;
  if (t_seed) *t_seed = ints.t_seed;
  if (t_ref)
    for (int k = 0; k < 3; ++k) t_ref[k] = ints.t_ref[k];
  return QSGS_OK;
}

size_t qsgs_workspace_bytes(const qsgs_params* params) {
  Ints ints{};
  if (check_params(params, &ints) != QSGS_OK) return 0;
  return make_layout(params).total;
}

int qsgs_create(const qsgs_params* params, void* dev_workspace, size_t bytes, void* cuda_stream,
                qsgs_handle** out) {
  if (!out) return QSGS_ERR_INVALID;
  *out = nullptr;
  Ints ints{};
  int rc = check_params(params, &ints);
  if (rc != QSGS_OK) return rc;
  const Layout L = make_layout(params);
  if (!dev_workspace || bytes < L.total || (reinterpret_cast<uintptr_t>(dev_workspace) % kAlign))
    return QSGS_ERR_WORKSPACE;
  if (prepare_kernels() != cudaSuccess) return QSGS_ERR_CUDA;
  qsgs_handle* h = new (std::nothrow) qsgs_handle();
  if (!h) return QSGS_ERR_NOMEM;
  h->p = *params;
  h->ints = ints;
  h->g = make_geom(params->nx, params->ny, params->nz, params->periodic);
  h->L = L;
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  h->ws = static_cast<uint8_t*>(dev_workspace);
  h->st = reinterpret_cast<RunState*>(h->ws + L.state);
  h->scan_status = reinterpret_cast<unsigned long long*>(h->ws + L.scan_status);
  h->grid = reinterpret_cast<uint32_t*>(h->ws + L.grid);
  h->aux = reinterpret_cast<uint32_t*>(h->ws + L.aux);
  h->list = reinterpret_cast<uint32_t*>(h->ws + L.list);
  h->mark = reinterpret_cast<uint32_t*>(h->ws + L.mark);
  const bool spacing = params->spacing_s >= 2;
  h->cell_count = spacing ? reinterpret_cast<uint32_t*>(h->ws + L.cell_count) : nullptr;
  h->cell_start = spacing ? reinterpret_cast<uint32_t*>(h->ws + L.cell_start) : nullptr;
  h->cell_items = spacing ? reinterpret_cast<uint32_t*>(h->ws + L.cell_items) : nullptr;
  h->decision = spacing ? h->ws + L.decision : nullptr;
  h->conf_off = spacing ? reinterpret_cast<uint32_t*>(h->ws + L.conf_off) : nullptr;
  h->adj = spacing ? reinterpret_cast<uint32_t*>(h->ws + L.adj) : nullptr;
  h->k0 = (uint32_t)params->seed;
  h->k1 = (uint32_t)(params->seed >> 32);
  h->grow_blocks = default_grow_blocks();
  h->grow_tile = 1;
  h->mode = QSGS_MODE_LIETS;
  h->spin_limit = kSpinLimit;
  h->seeded = false;
  h->seed_version = next_seed_version();
  h->last_cuda = cudaSuccess;
  h->graph = nullptr;
  h->graph_exec = nullptr;
  h->graph_tried = false;
  h->iters_seen = 0;
  h->list_stale = false;
  h->finalized = false;
  h->dev_enter = nullptr;
  h->dev_labels = nullptr;
  h->dev_enter_thr = nullptr;
  // The scan status words must start with flag 0; the run state is set by
  // qsgs_seed.
  cudaError_t e = cudaMemsetAsync(h->ws, 0, L.grid, h->stream);
  if (e != cudaSuccess) {
    delete h;
    return QSGS_ERR_CUDA;
  }
  *out = h;
  return QSGS_OK;
}

int qsgs_seed(qsgs_handle* h) {
  if (!h) return QSGS_ERR_INVALID;
  return seed_on_stream(h, h->stream);
}

int qsgs_grow_until(qsgs_handle* h, uint32_t max_steps, qsgs_stats* out) {
  if (!h) return QSGS_ERR_INVALID;
  if (!h->seeded) return QSGS_ERR_STATE;
  const StepBuffers b = step_buffers(h);
  cudaError_t e = cudaSuccess;
  if (h->list_stale) {
    e = launch_front_list(h->g, b, h->spin_limit, h->stream, h->tracer);
    if (e != cudaSuccess) return cuda_fail(h, e);
    h->list_stale = false;
  }
  e = launch_set_step_limit(h->st, max_steps, h->stream, h->tracer);
  if (e != cudaSuccess) return cuda_fail(h, e);
  RunState s{};
  if (!h->tracer.enabled() && h->stream != nullptr && !h->graph_tried) {
    h->graph_tried = true;
    if (build_graph(h) != cudaSuccess) {
      destroy_graph(h);
      (void)cudaGetLastError();
    }
  }
  if (!h->tracer.enabled() && h->graph_exec) {
    e = cudaGraphLaunch(h->graph_exec, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e);
    const int rc = read_state(h, &s);
    if (rc != QSGS_OK) return rc;
    // Count the kernels the graph ran: three per loop iteration, four in
    // the epilogue.
    h->tracer.launches += 3ull * (s.iters - h->iters_seen) + 4ull;
    h->iters_seen = s.iters;
  } else {
    // At most kStepsPerSync steps between host checks, and no more than
    // the call's budget (a step that is not active returns at once, but is
    // still a launch the profiler would time).
    uint32_t launched = 0;
    for (;;) {
      const uint32_t left = max_steps ? max_steps - launched : kStepsPerSync;
      const uint32_t burst = left < kStepsPerSync ? left : kStepsPerSync;
      if (burst == 0) break;  // the call's budget is spent
      launched += burst;
      for (uint32_t k = 0; k < burst; ++k) {
        e = launch_step(h->g, b, h->k0, h->k1, kSpinLimit, GrowShape{h->grow_blocks, h->grow_tile},
                        h->stream, h->tracer, (cudaGraphConditionalHandle)0, 0,
                        h->mode == QSGS_MODE_FULLFIELD);
        if (e != cudaSuccess) return cuda_fail(h, e);
      }
      const int rc = read_state(h, &s);
      if (rc != QSGS_OK) return rc;
      if (s.status != kRunning || !s.active) break;
    }
    e = launch_epilogue(h->g, b, h->spin_limit, h->stream, h->tracer);
    if (e != cudaSuccess) return cuda_fail(h, e);
    const int rc = read_state(h, &s);
    if (rc != QSGS_OK) return rc;
    h->iters_seen = s.iters;
  }
  fill_stats(h, s, out);
  return s.status == kRunning ? QSGS_RUNNING : s.status;
}

int qsgs_query(qsgs_handle* h, qsgs_stats* out) {
  if (!h) return QSGS_ERR_INVALID;
  RunState s{};
  const int rc = read_state(h, &s);
  if (rc != QSGS_OK) return rc;
  fill_stats(h, s, out);
  return QSGS_OK;
}

int qsgs_fetch(qsgs_handle* h, void* dst, size_t bytes, int fmt, int dst_is_device) {
  if (!h || !dst) return QSGS_ERR_INVALID;
  if (!h->seeded) return QSGS_ERR_STATE;
  if (dst_is_device != QSGS_DST_HOST && dst_is_device != QSGS_DST_DEVICE &&
      dst_is_device != QSGS_DST_HOST_MAPPED)
    return QSGS_ERR_INVALID;
  const size_t n = h->g.n, packed = (size_t)h->g.nwords * 4;
  const cudaMemcpyKind kind =
      dst_is_device == QSGS_DST_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  cudaError_t e = cudaSuccess;
  if (fmt == QSGS_FMT_PACKED) {
    if (bytes < packed) return QSGS_ERR_INVALID;
    e = cudaMemcpyAsync(dst, h->grid, packed, kind, h->stream);
  } else if (fmt == QSGS_FMT_U8) {
    if (bytes < n) return QSGS_ERR_INVALID;
    // Mapped host memory: its device address, if the runtime knows it.
    void* mapped = nullptr;
    if (dst_is_device == QSGS_DST_HOST_MAPPED &&
        cudaHostGetDevicePointer(&mapped, dst, 0) != cudaSuccess) {
      mapped = nullptr;
      (void)cudaGetLastError();  // not mapped host memory: staged below
    }
    if (dst_is_device == QSGS_DST_DEVICE || mapped) {
      // Straight into device memory, or over the host link into mapped host
      // memory (16-byte stores: no staging and no separate copy).
      uint8_t* out = static_cast<uint8_t*>(dst_is_device == QSGS_DST_DEVICE ? dst : mapped);
      e = launch_unpack_u8(h->g, h->grid, out, 0, n, h->stream, h->tracer);
    } else {
      RunState s{};
      const int rc = read_state(h, &s);
      if (rc != QSGS_OK) return rc;
      if (s.status == kRunning) return QSGS_ERR_STATE;  // the front area is still live
      // Staged through the candidate-list area in slabs of its size (the
      // stream orders each slab's copy before the next slab's unpack).
      uint8_t* staging = reinterpret_cast<uint8_t*>(h->list);
      const size_t slab = (size_t)(h->L.list_bytes & ~(uint64_t)15);
      for (size_t vb = 0; vb < n && e == cudaSuccess; vb += slab) {
        const size_t ve = vb + slab < n ? vb + slab : n;
        e = launch_unpack_u8(h->g, h->grid, staging, vb, ve, h->stream, h->tracer);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(static_cast<uint8_t*>(dst) + vb, staging, ve - vb, kind, h->stream);
      }
    }
  } else {
    return QSGS_ERR_INVALID;
  }
  if (e != cudaSuccess) return cuda_fail(h, e);
  e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e);
  e = h->tracer.collect();
  if (e != cudaSuccess) return cuda_fail(h, e);
  return QSGS_OK;
}

int qsgs_set_profiling(qsgs_handle* h, int enable) {
  if (!h) return QSGS_ERR_INVALID;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e);
  e = h->tracer.collect();
  if (e == cudaSuccess) e = h->tracer.enable(enable != 0);
  if (e != cudaSuccess) return cuda_fail(h, e);
  return QSGS_OK;
}

int qsgs_profile(qsgs_handle* h, qsgs_profile_entry* out, int max_entries) {
  if (!h || max_entries < 0 || (max_entries > 0 && !out)) return QSGS_ERR_INVALID;
  for (int c = 0; c < kNumClasses && c < max_entries; ++c) {
    std::memset(out[c].name, 0, sizeof(out[c].name));
    std::strncpy(out[c].name, kernel_class_name(c), sizeof(out[c].name) - 1);
    out[c].launches = h->tracer.count[c];
    out[c].total_ms = h->tracer.ms[c];
  }
  return kNumClasses;
}

int qsgs_bench_philox(uint64_t n_blocks, void* dev_out, void* cuda_stream, double* ms) {
  if (!dev_out || !ms || n_blocks == 0) return QSGS_ERR_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  int sms = 0, dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return QSGS_ERR_CUDA;
  const uint32_t blocks = (uint32_t)sms * 8u;  // 2048 threads per SM
  const uint64_t threads = (uint64_t)blocks * 256u;
  uint64_t per = (n_blocks + threads - 1) / threads;
  per = (per + 3) & ~3ull;  // whole groups of independent blocks per thread
  if (per > 0xFFFFFFFFull) return QSGS_ERR_INVALID;
  cudaEvent_t a = nullptr, b = nullptr;
  e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (e == cudaSuccess) e = cudaMemsetAsync(dev_out, 0, sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = cudaEventRecord(a, s);
  if (e == cudaSuccess)
    e = launch_philox_rate(0x0123456789ABCDEFull, blocks, (uint32_t)per,
                           static_cast<unsigned long long*>(dev_out), s);
  if (e == cudaSuccess) e = cudaEventRecord(b, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (e != cudaSuccess) return QSGS_ERR_CUDA;
  *ms = (double)t * (double)n_blocks / (double)(threads * per);  // scaled to n_blocks
  return QSGS_OK;
}

size_t qsgs_snapshot_bytes(const qsgs_params* params) {
  Ints ints{};
  if (check_params(params, &ints) != QSGS_OK) return 0;
  return snapshot_bytes(make_geom(params->nx, params->ny, params->nz, params->periodic));
}

int qsgs_snapshot(qsgs_handle* h, void* dst, size_t bytes, int dst_kind) {
  if (!h || !dst) return QSGS_ERR_INVALID;
  if (dst_kind != QSGS_DST_HOST && dst_kind != QSGS_DST_DEVICE &&
      dst_kind != QSGS_DST_HOST_MAPPED)
    return QSGS_ERR_INVALID;
  const size_t need = snapshot_bytes(h->g);
  if (bytes < need) return QSGS_ERR_INVALID;
  if (!h->seeded) return QSGS_ERR_STATE;
  RunState s{};
  const int rc = read_state(h, &s);  // synchronises: the step is closed
  if (rc != QSGS_OK) return rc;
  // Between calls the exact-target trim has run (a batch member's only at
  // qsgs_batch_query); a pending trim needs the claim grid, which a
  // snapshot does not hold.
  if (s.trim_pending) return QSGS_ERR_STATE;
  SnapHeader hd{};
  std::memcpy(hd.magic, kSnapMagic, sizeof(kSnapMagic));
  hd.version = kSnapVersion;
  hd.nwords = h->g.nwords;
  hd.total_bytes = need;
  hd.params = h->p;
  unsigned char head[kSnapState] = {};
  std::memcpy(head, &hd, sizeof(hd));
  std::memcpy(head + kSnapHeader, &s, sizeof(s));
  uint8_t* out = static_cast<uint8_t*>(dst);
  cudaError_t e = cudaSuccess;
  if (dst_kind == QSGS_DST_DEVICE)
    e = cudaMemcpyAsync(out, head, kSnapState, cudaMemcpyHostToDevice, h->stream);
  else
    std::memcpy(out, head, kSnapState);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out + kSnapState, h->grid, (size_t)h->g.nwords * 4,
                        copy_kind(dst_kind, false), h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);  // `head` is on this stack
  return e == cudaSuccess ? QSGS_OK : cuda_fail(h, e);
}

int qsgs_restore(qsgs_handle* h, const void* src, size_t bytes, int src_kind) {
  if (!h || !src) return QSGS_ERR_INVALID;
  if (src_kind != QSGS_DST_HOST && src_kind != QSGS_DST_DEVICE &&
      src_kind != QSGS_DST_HOST_MAPPED)
    return QSGS_ERR_INVALID;
  const size_t need = snapshot_bytes(h->g);
  if (bytes < need) return QSGS_ERR_INVALID;
  const uint8_t* in = static_cast<const uint8_t*>(src);
  unsigned char head[kSnapState];
  cudaError_t e = cudaSuccess;
  if (src_kind == QSGS_DST_DEVICE) {
    e = cudaMemcpyAsync(head, in, kSnapState, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e);
  } else {
    std::memcpy(head, in, kSnapState);
  }
  SnapHeader hd;
  std::memcpy(&hd, head, sizeof(hd));
  if (std::memcmp(hd.magic, kSnapMagic, sizeof(kSnapMagic)) != 0 || hd.version != kSnapVersion ||
      hd.nwords != h->g.nwords || hd.total_bytes != need || !same_params(hd.params, h->p))
    return QSGS_ERR_INVALID;
  RunState s;
  std::memcpy(&s, head + kSnapHeader, sizeof(s));
  if (s.trim_pending || s.error || s.nt != h->ints.nt) return QSGS_ERR_INVALID;
  // Everything a step carries over is the grid and these counters; the
  // transient fields of a step and of the look-back scans start afresh.
  s.claimed = 0;
  s.live = 0;
  s.front_acc = 0;
  s.active = 0;
  s.step_limit = 0xFFFFFFFFu;
  s.scan_tile = 0;
  s.scan_done = 0;
  s.grow_next = 0;
  s.grow_done = 0;
  s.list_next = 0;
  s.front_words = 0;
  const size_t grids = (size_t)h->g.nwords * 4;
  e = cudaMemcpyAsync(h->grid, in + kSnapState, grids, copy_kind(src_kind, true), h->stream);
  // Claim grids, marks and touched bits are all zero between steps of a
  // fresh run; so are the look-back status words before their first use.
  if (e == cudaSuccess) e = cudaMemsetAsync(h->aux, 0, 2 * grids, h->stream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(h->mark, 0, 2 * (size_t)bitmap_words(h->g) * 4, h->stream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(h->scan_status, 0, h->L.ntiles * sizeof(unsigned long long), h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->st, &s, sizeof(s), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);  // `s` is on this stack
  if (e != cudaSuccess) return cuda_fail(h, e);
  h->seeded = true;
  h->list_stale = true;  // the candidate list is rebuilt from the grid
  h->finalized = s.status != kRunning;
  h->iters_seen = s.iters;
  return QSGS_OK;
}

int qsgs_bench_l2_read(const void* dev_buf, size_t bytes, uint32_t passes, void* dev_out,
                       void* cuda_stream, double* ms) {
  if (!dev_buf || !dev_out || !ms || passes == 0 || bytes % 16 ||
      (reinterpret_cast<uintptr_t>(dev_buf) % 16) || (reinterpret_cast<uintptr_t>(dev_out) % 8))
    return QSGS_ERR_INVALID;
  const uint64_t n16 = bytes / 16;
  if (n16 < 4ull * l2_read_threads() || n16 >= (1ull << 32)) return QSGS_ERR_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  unsigned long long* out = static_cast<unsigned long long*>(dev_out);
  // One untimed pass brings the buffer into L2.
  cudaError_t e = launch_l2_read(dev_buf, n16, 1, out, s);
  if (e != cudaSuccess) return QSGS_ERR_CUDA;
  float t = 0.f;
  const int rc = time_probe(s, [&] { return launch_l2_read(dev_buf, n16, passes, out, s); }, &t);
  if (rc != QSGS_OK) return rc;
  *ms = t;
  return QSGS_OK;
}

int qsgs_bench_l2_atomic(void* dev_buf, size_t bytes, uint64_t n_ops, void* cuda_stream,
                         double* ms) {
  if (!dev_buf || !ms || n_ops == 0 || bytes < 4 || (reinterpret_cast<uintptr_t>(dev_buf) % 4))
    return QSGS_ERR_INVALID;
  const uint64_t nwords = bytes / 4;
  if (nwords >= (1ull << 32)) return QSGS_ERR_INVALID;
  int sms = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return QSGS_ERR_CUDA;
  const uint32_t blocks = (uint32_t)sms * 4u;
  const uint64_t threads = (uint64_t)blocks * 512u;
  const uint64_t per = (n_ops + threads - 1) / threads;
  if (per > 0xFFFFFFFFull) return QSGS_ERR_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = launch_l2_red(dev_buf, nwords, 4, blocks, s);  // untimed warm-up
  if (e != cudaSuccess) return QSGS_ERR_CUDA;
  float t = 0.f;
  const int rc = time_probe(
      s, [&] { return launch_l2_red(dev_buf, nwords, (uint32_t)per, blocks, s); }, &t);
  if (rc != QSGS_OK) return rc;
  *ms = (double)t * (double)n_ops / (double)(threads * per);  // scaled to n_ops
  return QSGS_OK;
}

void qsgs_destroy(qsgs_handle* h) {
  if (!h) return;
  destroy_graph(h);
  delete h;
}


size_t qsgs_batch_workspace_bytes(uint32_t max_members, uint64_t max_words) {
  if (max_members == 0 || max_members > kMaxBatchMembers || max_words >= (1ull << 32)) return 0;
  return make_batch_layout(max_members, max_words).total;
}

int qsgs_batch_create(uint32_t max_members, uint64_t max_words, void* dev_workspace, size_t bytes,
                      void* cuda_stream, qsgs_batch** out) {
  if (!out) return QSGS_ERR_INVALID;
  *out = nullptr;
  if (max_members == 0 || max_members > kMaxBatchMembers || max_words >= (1ull << 32))
    return QSGS_ERR_INVALID;
  const BatchLayout L = make_batch_layout(max_members, max_words);
  if (!dev_workspace || bytes < L.total || (reinterpret_cast<uintptr_t>(dev_workspace) % kAlign))
    return QSGS_ERR_WORKSPACE;
  if (prepare_kernels() != cudaSuccess) return QSGS_ERR_CUDA;
  qsgs_batch* b = new (std::nothrow) qsgs_batch();
  if (!b) return QSGS_ERR_NOMEM;
  b->max_members = max_members;
  b->max_words = max_words;
  b->L = L;
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  b->ws = static_cast<uint8_t*>(dev_workspace);
  b->buf = BatchBuffers{reinterpret_cast<MemberDesc*>(b->ws + L.descs),
                        reinterpret_cast<BatchState*>(b->ws + L.state),
                        reinterpret_cast<uint32_t*>(b->ws + L.list), max_members, max_words};
  b->grow_blocks = default_batch_grow_blocks();
  b->grow_tile = 1;
  b->iters_seen = 0;
  b->graph = nullptr;
  b->graph_exec = nullptr;
  b->graph_tried = false;
  b->seed_exec = nullptr;
  b->seed_graph_failed = false;
  b->last_cuda = cudaSuccess;
  cudaError_t e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  for (uint32_t k = 0; k < kSeedStreams && e == cudaSuccess; ++k) {
    e = cudaStreamCreateWithFlags(&b->seed_streams[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->seed_events[k], cudaEventDisableTiming);
  }
  // State and scan tile words start at zero; no members yet.
  if (e == cudaSuccess) e = cudaMemsetAsync(b->ws, 0, L.list, b->stream);
  if (e != cudaSuccess) {
    qsgs_batch_destroy(b);
    return QSGS_ERR_CUDA;
  }
  *out = b;
  return QSGS_OK;
}

int qsgs_batch_set_members(qsgs_batch* b, qsgs_handle* const* members, uint32_t n) {
  if (!b || (n && !members) || n > b->max_members) return QSGS_ERR_INVALID;
  std::vector<MemberDesc> descs(n);
  uint64_t words = 0;
  uint32_t open_only = 1;
  for (uint32_t m = 0; m < n; ++m) {
    qsgs_handle* h = members[m];
    if (!h || h->dev_enter) return QSGS_ERR_INVALID;  // interacting phases: single path only
    if (h->g.periodic || h->g.blocked) open_only = 0;
    MemberDesc& d = descs[m];
    std::memset(&d, 0, sizeof(d));
    d.g = h->g;
    d.grid = h->grid;
    d.aux = h->aux;
    d.mark = h->mark;
    d.st = h->st;
    d.keys = make_philox_keys(h->p.seed);
    d.word_base = (uint32_t)words;
    d.word_end = (uint32_t)(words + h->g.nwords);
    words += ((uint64_t)h->g.nwords + 31) / 32 * 32;
  }
  if (words > b->max_words) return QSGS_ERR_WORKSPACE;
  // The batch stream waits for each member's own stream (its seeding).
  cudaError_t e = cudaSuccess;
  for (uint32_t m = 0; m < n && e == cudaSuccess; ++m) {
    if (members[m]->stream == b->stream) continue;
    e = cudaEventRecord(b->fork, members[m]->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->fork, 0);
  }
  if (e == cudaSuccess && n)
    e = cudaMemcpyAsync(b->buf.d, descs.data(), n * sizeof(MemberDesc), cudaMemcpyHostToDevice,
                        b->stream);
  uint32_t sizes[2] = {n, (uint32_t)words};
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(reinterpret_cast<uint8_t*>(b->buf.bs) + offsetof(BatchState, n_members),
                        sizes, sizeof(sizes), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);  // host copies are staged
  if (e != cudaSuccess) return batch_fail(b, e);
  b->members.assign(members, members + n);
  b->host_descs = descs;
  // The growth kernel's domain kind is fixed in the graph: a change of kind
  // rebuilds it at the next advance.
  if (open_only != b->buf.open_only) {
    destroy_batch_graph(b);
    b->graph_tried = false;
    b->buf.open_only = open_only;
  }
  for (qsgs_handle* h : b->members) h->list_stale = true;
  return QSGS_OK;
}

namespace {

// Seeding of every member, forked from the batch stream onto the seed
// streams and joined back: launched directly, or captured into the seeding
// graph.
cudaError_t enqueue_batch_seeding(qsgs_batch* b) {
  cudaError_t e = cudaEventRecord(b->fork, b->stream);
  for (uint32_t k = 0; k < kSeedStreams && e == cudaSuccess; ++k)
    e = cudaStreamWaitEvent(b->seed_streams[k], b->fork, 0);
  for (size_t m = 0; m < b->members.size() && e == cudaSuccess; ++m)
    if (seed_on_stream(b->members[m], b->seed_streams[m % kSeedStreams]) != QSGS_OK)
      e = b->members[m]->last_cuda != cudaSuccess ? b->members[m]->last_cuda
                                                  : cudaErrorUnknown;
  for (uint32_t k = 0; k < kSeedStreams && e == cudaSuccess; ++k) {
    e = cudaEventRecord(b->seed_events[k], b->seed_streams[k]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->seed_events[k], 0);
  }
  return e;
}

// The seeding graph for the current members, captured once per membership
// (and member seed versions); false if it cannot be used.
bool seed_graph_ready(qsgs_batch* b) {
  if (b->stream == nullptr || b->tracer.enabled()) return false;
  std::vector<std::pair<const qsgs_handle*, uint64_t>> key;
  key.reserve(b->members.size());
  for (qsgs_handle* h : b->members) {
    if (h->tracer.enabled()) return false;  // the profiler times direct launches
    key.emplace_back(h, h->seed_version);
  }
  if (key == b->seed_key) return b->seed_exec != nullptr;
  if (b->seed_exec) cudaGraphExecDestroy(b->seed_exec);
  b->seed_exec = nullptr;
  b->seed_key = key;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    const cudaError_t le = enqueue_batch_seeding(b);
    e = cudaStreamEndCapture(b->stream, &g);
    if (le != cudaSuccess) e = le;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->seed_exec, g, 0);
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    if (b->seed_exec) cudaGraphExecDestroy(b->seed_exec);
    b->seed_exec = nullptr;
    (void)cudaGetLastError();
    for (qsgs_handle* h : b->members) h->last_cuda = cudaSuccess;
  }
  return b->seed_exec != nullptr;
}

}  // namespace

int qsgs_batch_seed(qsgs_batch* b) {
  if (!b) return QSGS_ERR_INVALID;
  // One graph launch replays every member's seeding (captured on the first
  // call for these members; 88.8 -> 87.6 ms for the 96-member batch with
  // 16 seed streams, against 1,800-odd direct launches).
  if (!b->members.empty() && seed_graph_ready(b)) {
    const cudaError_t ge = cudaGraphLaunch(b->seed_exec, b->stream);
    if (ge != cudaSuccess) return batch_fail(b, ge);
    for (qsgs_handle* h : b->members) {  // what seed_on_stream records
      h->seeded = true;
      h->finalized = false;
      h->iters_seen = 0;
      h->list_stale = true;
    }
    return QSGS_OK;
  }
  // Direct launches (the profiler is on, the legacy stream, or no graph).
  const cudaError_t e = enqueue_batch_seeding(b);
  if (e != cudaSuccess) return batch_fail(b, e);
  for (qsgs_handle* h : b->members) h->list_stale = true;
  return QSGS_OK;
}

int qsgs_batch_advance(qsgs_batch* b, uint32_t max_steps) {
  if (!b) return QSGS_ERR_INVALID;
  if (b->members.empty()) return QSGS_OK;
  for (qsgs_handle* h : b->members)
    if (!h->seeded) return QSGS_ERR_STATE;
  cudaError_t e = cudaMemcpyAsync(
      reinterpret_cast<uint8_t*>(b->buf.bs) + offsetof(BatchState, step_extra), &max_steps,
      sizeof(max_steps), cudaMemcpyHostToDevice, b->stream);
  if (e != cudaSuccess) return batch_fail(b, e);
  if (!b->tracer.enabled() && b->stream != nullptr && !b->graph_tried) {
    b->graph_tried = true;
    if (build_batch_graph(b) != cudaSuccess) {
      destroy_batch_graph(b);
      (void)cudaGetLastError();
    }
  }
  if (!b->tracer.enabled() && b->graph_exec) {
    e = cudaGraphLaunch(b->graph_exec, b->stream);
    if (e != cudaSuccess) return batch_fail(b, e);
    return QSGS_OK;
  }
  e = launch_batch_prologue(b->buf, kSpinLimit, b->stream, b->tracer,
                            (cudaGraphConditionalHandle)0, 0);
  if (e != cudaSuccess) return batch_fail(b, e);
  for (;;) {
    for (uint32_t k = 0; k < kStepsPerSync; ++k) {
      e = launch_batch_step(b->buf, kSpinLimit, GrowShape{b->grow_blocks, b->grow_tile}, b->stream,
                            b->tracer,
                            (cudaGraphConditionalHandle)0, 0);
      if (e != cudaSuccess) return batch_fail(b, e);
    }
    uint32_t any = 0;
    e = cudaMemcpyAsync(&any, reinterpret_cast<uint8_t*>(b->buf.bs) + offsetof(BatchState, any_active),
                        sizeof(any), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e == cudaSuccess) e = b->tracer.collect();
    if (e != cudaSuccess) return batch_fail(b, e);
    if (!any) break;
  }
  return QSGS_OK;
}

int qsgs_batch_query(qsgs_batch* b, qsgs_stats* per_member, uint32_t n) {
  if (!b || (n && !per_member)) return QSGS_ERR_INVALID;
  const size_t nm = b->members.size();
  b->host_states.resize(nm);
  // Every member's run state, gathered on the device, in one copy.
  RunState* gathered = reinterpret_cast<RunState*>(b->ws + b->L.states);
  auto read_all = [&]() -> cudaError_t {
    cudaError_t e = launch_batch_gather_states(b->buf, (uint32_t)nm, gathered, b->stream,
                                               b->tracer);
    if (e == cudaSuccess && nm)
      e = cudaMemcpyAsync(b->host_states.data(), gathered, nm * sizeof(RunState),
                          cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    return e;
  };
  cudaError_t e = read_all();
  if (e != cudaSuccess) return batch_fail(b, e);
  // Members whose run ended: exact-target trim and final front count, once.
  bool any_final = false;
  for (size_t m = 0; m < nm; ++m) {
    qsgs_handle* h = b->members[m];
    if (b->host_states[m].status != kRunning && !h->finalized) {
      e = launch_epilogue(h->g, step_buffers(h), h->spin_limit, b->stream, h->tracer);
      if (e != cudaSuccess) return batch_fail(b, e);
      h->finalized = true;
      any_final = true;
    }
  }
  if (any_final) {
    e = read_all();
    if (e != cudaSuccess) return batch_fail(b, e);
  }
  int rc = QSGS_OK;
  for (size_t m = 0; m < nm; ++m) {
    if (b->host_states[m].error & kErrTimeout) rc = QSGS_ERR_TIMEOUT;
    if (b->host_states[m].error & kErrOverflow) rc = QSGS_ERR_WORKSPACE;
    if (m < n) fill_stats(b->members[m], b->host_states[m], &per_member[m]);
  }
  return rc;
}

int qsgs_batch_run(qsgs_batch* b, uint32_t max_steps, qsgs_stats* per_member, uint32_t n) {
  int rc = qsgs_batch_seed(b);
  if (rc == QSGS_OK) rc = qsgs_batch_advance(b, max_steps);
  if (rc == QSGS_OK) rc = qsgs_batch_query(b, per_member, n);
  return rc;
}

int qsgs_batch_set_grow_blocks(qsgs_batch* b, uint32_t blocks) {
  if (!b) return QSGS_ERR_INVALID;
  b->grow_blocks = blocks ? blocks : default_batch_grow_blocks();
  destroy_batch_graph(b);  // the grid size is baked into the graph
  b->graph_tried = false;
  return QSGS_OK;
}

int qsgs_set_spin_limit(qsgs_handle* h, uint32_t polls) {
  if (!h) return QSGS_ERR_INVALID;
  h->spin_limit = polls ? polls : kSpinLimit;
  destroy_graph(h);  // the limit is a launch argument inside the graph
  h->graph_tried = false;
  h->seed_version = next_seed_version();
  return QSGS_OK;
}

int qsgs_set_blocked(qsgs_handle* h, const void* dev_blocked) {
  if (!h) return QSGS_ERR_INVALID;
  if (dev_blocked && (reinterpret_cast<uintptr_t>(dev_blocked) % 4)) return QSGS_ERR_INVALID;
  h->g.blocked = static_cast<const uint32_t*>(dev_blocked);
  h->dev_enter = nullptr;  // an independent phase: no interaction
  h->dev_labels = nullptr;
  h->dev_enter_thr = nullptr;
  destroy_graph(h);  // the geometry (with the pointer) is baked into the graph
  h->graph_tried = false;
  h->seed_version = next_seed_version();
  return QSGS_OK;
}

int qsgs_fetch_label(qsgs_handle* h, void* dev_dst, size_t bytes, uint8_t label) {
  if (!h || !dev_dst || bytes < (size_t)h->g.n) return QSGS_ERR_INVALID;
  if (!h->seeded) return QSGS_ERR_STATE;
  cudaError_t e = launch_label_u8(h->g, h->grid, static_cast<uint8_t*>(dev_dst), label, h->stream,
                                  h->tracer);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess) e = h->tracer.collect();
  return e == cudaSuccess ? QSGS_OK : cuda_fail(h, e);
}

int qsgs_fetch_or(qsgs_handle* h, void* dev_dst, size_t bytes) {
  if (!h || !dev_dst || bytes < (size_t)h->g.nwords * 4 ||
      (reinterpret_cast<uintptr_t>(dev_dst) % 4))
    return QSGS_ERR_INVALID;
  if (!h->seeded) return QSGS_ERR_STATE;
  cudaError_t e = launch_or_words(h->g.nwords, h->grid, static_cast<uint32_t*>(dev_dst),
                                  h->stream, h->tracer);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess) e = h->tracer.collect();
  return e == cudaSuccess ? QSGS_OK : cuda_fail(h, e);
}

size_t qsgs_interaction_bytes(const qsgs_params* p) {
  Ints ints;
  if (check_params(p, &ints) != QSGS_OK) return 0;
  const uint64_t W = (p->nx + 31) / 32;
  const uint64_t nwords = W * p->ny * p->nz;
  return (size_t)(4 * nwords * 4 + 256 * 3 * 4);
}

int qsgs_set_interaction(qsgs_handle* h, const uint8_t* dev_labels, const double* probs,
                         uint32_t n_labels, void* dev_scratch, size_t scratch_bytes) {
  if (!h) return QSGS_ERR_INVALID;
  if (!dev_labels) {  // back to an independent first phase
    h->g.blocked = nullptr;
    h->dev_enter = nullptr;
    h->dev_labels = nullptr;
    h->dev_enter_thr = nullptr;
    destroy_graph(h);
    h->graph_tried = false;
    h->seed_version = next_seed_version();
    return QSGS_OK;
  }
  if (n_labels > 255 || (n_labels && !probs) || !dev_scratch ||
      (reinterpret_cast<uintptr_t>(dev_scratch) % 16))
    return QSGS_ERR_INVALID;
  if (h->mode != QSGS_MODE_LIETS) return QSGS_ERR_STATE;
  for (uint32_t i = 0; i < 3 * n_labels; ++i)
    if (!(probs[i] >= 0.0 && probs[i] <= 1.0)) return QSGS_ERR_INVALID;
  const size_t nwords = h->g.nwords;
  if (scratch_bytes < 4 * nwords * 4 + 256 * 3 * 4) return QSGS_ERR_WORKSPACE;
  // Thresholds floor(I 2^32) - 1 per label and class; row 0 (no label)
  // holds the largest per class; sets of the labels each class may enter.
  h->enter_thr.assign(256 * 3, 0u);
  uint32_t sets[3][8] = {};
  for (uint32_t m = 1; m <= n_labels; ++m)
    for (uint32_t k = 0; k < 3; ++k) {
      const double pr = probs[3 * (m - 1) + k];
      const uint64_t T = (uint64_t)std::floor(pr * 4294967296.0);
      if (T == 0) continue;
      const uint32_t t1 = (uint32_t)(T - 1);
      h->enter_thr[m * 3 + k] = t1;
      sets[k][m >> 5] |= 1u << (m & 31u);
      if (t1 > h->enter_thr[k]) h->enter_thr[k] = t1;
    }
  uint32_t* blocked = static_cast<uint32_t*>(dev_scratch);
  uint32_t* enter = blocked + nwords;
  uint32_t* thr = enter + 3 * nwords;
  Geom g = h->g;
  cudaError_t e = cudaMemcpyAsync(thr, h->enter_thr.data(), 256 * 3 * 4, cudaMemcpyHostToDevice,
                                  h->stream);
  if (e == cudaSuccess) e = launch_pack_labels(g, dev_labels, blocked, enter, sets, h->stream,
                                               h->tracer);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e);
  h->g.blocked = blocked;
  h->dev_enter = enter;
  h->dev_labels = dev_labels;
  h->dev_enter_thr = thr;
  destroy_graph(h);  // the geometry (with the pointers) is baked into the graph
  h->graph_tried = false;
  h->seed_version = next_seed_version();
  return QSGS_OK;
}

int qsgs_set_mode(qsgs_handle* h, int mode) {
  if (!h || (mode != QSGS_MODE_LIETS && mode != QSGS_MODE_FULLFIELD)) return QSGS_ERR_INVALID;
  if (mode == QSGS_MODE_FULLFIELD && h->dev_enter) return QSGS_ERR_STATE;
  if (mode != h->mode) {
    h->mode = mode;
    destroy_graph(h);  // the step kernel is baked into the graph
    h->graph_tried = false;
    h->seed_version = next_seed_version();
  }
  return QSGS_OK;
}

int qsgs_set_grow_tile(qsgs_handle* h, uint32_t chunks) {
  if (!h || chunks > kMaxGrowTile) return QSGS_ERR_INVALID;
  h->grow_tile = chunks ? chunks : 1;
  destroy_graph(h);  // the tile is baked into the graph
  h->graph_tried = false;
  h->seed_version = next_seed_version();
  return QSGS_OK;
}

int qsgs_batch_set_grow_tile(qsgs_batch* b, uint32_t chunks) {
  if (!b || chunks > kMaxGrowTile) return QSGS_ERR_INVALID;
  b->grow_tile = chunks ? chunks : 1;
  destroy_batch_graph(b);
  b->graph_tried = false;
  return QSGS_OK;
}

int qsgs_set_grow_blocks(qsgs_handle* h, uint32_t blocks) {
  if (!h) return QSGS_ERR_INVALID;
  h->grow_blocks = blocks ? blocks : default_grow_blocks();
  destroy_graph(h);
  h->graph_tried = false;
  h->seed_version = next_seed_version();
  return QSGS_OK;
}

int qsgs_time_grow(qsgs_handle* h, uint32_t grow_blocks, uint32_t reps, double* ms) {
  if (!h || !ms || reps == 0) return QSGS_ERR_INVALID;
  if (!h->seeded || h->list_stale) return QSGS_ERR_STATE;
  RunState saved{};
  int rc = read_state(h, &saved);
  if (rc != QSGS_OK) return rc;
  if (saved.status != kRunning) return QSGS_ERR_STATE;
  const uint32_t blocks = grow_blocks ? grow_blocks : default_grow_blocks();
  const StepBuffers b = step_buffers(h);
  Tracer quiet;  // probe launches are not counted as the run's launches
  // A run paused by its step budget has step t listed but not opened: open
  // it (thresholds of step t) for the replays; the saved state goes back.
  cudaError_t e = launch_set_step_limit(h->st, 1, h->stream, quiet);
  RunState open{};
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e);
  rc = read_state(h, &open);
  if (rc != QSGS_OK) return rc;
  if (!open.active) {
    e = cudaMemcpyAsync(h->st, &saved, sizeof(RunState), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    return e == cudaSuccess ? QSGS_ERR_STATE : cuda_fail(h, e);
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const GrowShape shape{blocks, h->grow_tile};
  if (e == cudaSuccess) e = launch_grow_only(h->g, b, h->k0, h->k1, shape, h->stream, quiet);
  if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
  for (uint32_t k = 0; k < reps && e == cudaSuccess; ++k)
    e = launch_grow_only(h->g, b, h->k0, h->k1, shape, h->stream, quiet);
  if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  // Put back the counters the replays accumulated; the grid, the claim grid
  // and the marks are unchanged by repeating the same step.
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->st, &saved, sizeof(RunState), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(h, e);
  *ms = (double)t / reps;
  return QSGS_OK;
}

int qsgs_front_count_static(const uint32_t* dev_grid, uint32_t nx, uint32_t ny, uint32_t nz,
                            void* cuda_stream, uint64_t* front_out) {
  if (!dev_grid || !front_out || nx == 0 || ny == 0 || nz == 0) return QSGS_ERR_INVALID;
  const uint64_t words = (uint64_t)((nx + 31u) / 32u) * ny * nz;
  if ((uint64_t)nx * ny * nz > 0xFFFFFFFFull) return QSGS_ERR_INVALID;
  if (words > front_scratch_max_words()) return QSGS_ERR_WORKSPACE;
  const Geom g = make_geom(nx, ny, nz, 0);
  unsigned long long front = 0;
  uint32_t error = 0;
  const cudaError_t e =
      front_count_static(g, dev_grid, kSpinLimit, static_cast<cudaStream_t>(cuda_stream), &front,
                         &error);
  if (e != cudaSuccess) return QSGS_ERR_CUDA;
  if (error & kErrTimeout) return QSGS_ERR_TIMEOUT;
  *front_out = front;
  return QSGS_OK;
}

int qsgs_batch_set_profiling(qsgs_batch* b, int enable) {
  if (!b) return QSGS_ERR_INVALID;
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e == cudaSuccess) e = b->tracer.collect();
  if (e == cudaSuccess) e = b->tracer.enable(enable != 0);
  if (e != cudaSuccess) return batch_fail(b, e);
  return QSGS_OK;
}

int qsgs_batch_profile(qsgs_batch* b, qsgs_profile_entry* out, int max_entries) {
  if (!b || max_entries < 0 || (max_entries > 0 && !out)) return QSGS_ERR_INVALID;
  for (int c = 0; c < kNumClasses && c < max_entries; ++c) {
    std::memset(out[c].name, 0, sizeof(out[c].name));
    std::strncpy(out[c].name, kernel_class_name(c), sizeof(out[c].name) - 1);
    out[c].launches = b->tracer.count[c];
    out[c].total_ms = b->tracer.ms[c];
  }
  return kNumClasses;
}

void qsgs_batch_destroy(qsgs_batch* b) {
  if (!b) return;
  destroy_batch_graph(b);
  if (b->seed_exec) cudaGraphExecDestroy(b->seed_exec);
  for (uint32_t k = 0; k < kSeedStreams; ++k) {
    if (b->seed_streams[k]) cudaStreamDestroy(b->seed_streams[k]);
    if (b->seed_events[k]) cudaEventDestroy(b->seed_events[k]);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  delete b;
}

}  // extern "C"
