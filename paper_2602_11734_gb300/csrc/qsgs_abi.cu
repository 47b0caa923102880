// qsgs_abi.cu -- the extern "C" boundary of libqsgs (see include/qsgs.h).
//
// Host-side only: parameter validation, workspace carve-up, launch order
// and synchronisation.  All generation work runs in the kernels of
// qsgs_kernels.cu; nothing here computes voxels.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

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
  uint64_t ntiles;
  CellGeomHost cg;
};

struct Ints {
  uint64_t nt, t_seed, t_ref[3];
};

int check_params(const qsgs_params* p, Ints* out) {
  if (!p) return QSGS_ERR_INVALID;
  if (p->nx == 0 || p->ny == 0 || p->nz == 0) return QSGS_ERR_INVALID;
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

Layout make_layout(const qsgs_params* p) {
  Layout L{};
  const uint64_t n = (uint64_t)p->nx * p->ny * p->nz;
  const uint64_t W = (p->nx + 31) / 32;
  const uint64_t nwords = W * p->ny * p->nz;
  uint64_t ncells = 0;
  if (p->spacing_s >= 2) {
    const uint32_t s = p->spacing_s;
    L.cg = CellGeomHost{s, (p->nx + s - 1) / s, (p->ny + s - 1) / s, (p->nz + s - 1) / s};
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
  L.mark = off; off = align_up(off + (nwords / 32 + 1) * 4);
  // Seed candidates (at most N), then the candidate word list (at most
  // nwords); u32 entries.
  const uint64_t list_bytes = (n > nwords ? n : nwords) * 4;
  L.list = off; off = align_up(off + list_bytes);
  if (ncells) {
    L.cell_count = off; off = align_up(off + ncells * 4);
    L.cell_start = off; off = align_up(off + (ncells + 1) * 4);
    L.cell_items = off; off = align_up(off + n * 4);
    L.decision = off; off = align_up(off + n);
    L.conf_off = off; off = align_up(off + (n + 1) * 4);
    L.adj_cap = n;
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
};

namespace {

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
  return StepBuffers{h->st, h->scan_status, h->grid, h->aux, h->mark, h->list};
}

void destroy_graph(qsgs_handle* h) {
  if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
  if (h->graph) cudaGraphDestroy(h->graph);
  h->graph_exec = nullptr;
  h->graph = nullptr;
}

// Captures the whole growth loop of this handle into one graph: a while
// node whose body is one step (its last kernel sets the loop condition),
// followed by the exact-target epilogue.  Kernel arguments are fixed per
// handle, so the graph is built once and relaunched by every call.
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
  cudaError_t le = launch_step(h->g, b, h->k0, h->k1, kSpinLimit, h->grow_blocks, h->stream,
                               capture_tracer, cond, 1);
  cudaGraph_t captured = nullptr;
  e = cudaStreamEndCapture(h->stream, &captured);
  if (le != cudaSuccess) return le;
  if (e != cudaSuccess) return e;
  e = cudaStreamBeginCaptureToGraph(h->stream, h->graph, &loop, nullptr, 1,
                                    cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  le = launch_epilogue(h->g, b, kSpinLimit, h->stream, capture_tracer);
  e = cudaStreamEndCapture(h->stream, &captured);
  if (le != cudaSuccess) return le;
  if (e != cudaSuccess) return e;
  return cudaGraphInstantiate(&h->graph_exec, h->graph, 0);
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
  qsgs_handle* h = new (std::nothrow) qsgs_handle();
  if (!h) return QSGS_ERR_NOMEM;
  h->p = *params;
  h->ints = ints;
  h->g = make_geom(params->nx, params->ny, params->nz);
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
  h->seeded = false;
  h->last_cuda = cudaSuccess;
  h->graph = nullptr;
  h->graph_exec = nullptr;
  h->graph_tried = false;
  h->iters_seen = 0;
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
  const size_t grids = (size_t)h->g.nwords * 4;
  cudaError_t e = cudaMemsetAsync(h->grid, 0, grids, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->aux, 0, 2 * grids, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->mark, 0, (h->g.nwords / 32 + 1) * 4, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e);
  StateInit init{};
  init.nt = h->ints.nt;
  for (int k = 0; k < 3; ++k) init.t_ref[k] = h->ints.t_ref[k];
  init.t_seed = h->ints.t_seed;
  init.max_steps = h->p.max_steps ? h->p.max_steps : 0xFFFFFFFFu;
  e = launch_init_state(h->st, init, h->stream, h->tracer);
  if (e != cudaSuccess) return cuda_fail(h, e);
  SeedBuffers b{h->st,         h->scan_status, h->grid,     h->aux,
                h->list,       h->mark,        h->cell_count,  h->cell_start, h->cell_items,
                h->decision,   h->conf_off,    h->adj,        h->L.adj_cap,
                h->L.cg};
  e = launch_seed(h->g, b, h->k0, h->k1, kSpinLimit, h->stream, h->tracer);
  if (e != cudaSuccess) return cuda_fail(h, e);
  h->seeded = true;
  h->iters_seen = 0;
  return QSGS_OK;
}

int qsgs_grow_until(qsgs_handle* h, uint32_t max_steps, qsgs_stats* out) {
  if (!h) return QSGS_ERR_INVALID;
  if (!h->seeded) return QSGS_ERR_STATE;
  cudaError_t e = launch_set_step_limit(h->st, max_steps, h->stream, h->tracer);
  if (e != cudaSuccess) return cuda_fail(h, e);
  const StepBuffers b = step_buffers(h);
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
    for (;;) {
      for (uint32_t k = 0; k < kStepsPerSync; ++k) {
        e = launch_step(h->g, b, h->k0, h->k1, kSpinLimit, h->grow_blocks, h->stream, h->tracer,
                        (cudaGraphConditionalHandle)0, 0);
        if (e != cudaSuccess) return cuda_fail(h, e);
      }
      const int rc = read_state(h, &s);
      if (rc != QSGS_OK) return rc;
      if (s.status != kRunning || !s.active) break;
    }
    e = launch_epilogue(h->g, b, kSpinLimit, h->stream, h->tracer);
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
  const size_t n = h->g.n, packed = (size_t)h->g.nwords * 4;
  const cudaMemcpyKind kind = dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  cudaError_t e = cudaSuccess;
  if (fmt == QSGS_FMT_PACKED) {
    if (bytes < packed) return QSGS_ERR_INVALID;
    e = cudaMemcpyAsync(dst, h->grid, packed, kind, h->stream);
  } else if (fmt == QSGS_FMT_U8) {
    if (bytes < n) return QSGS_ERR_INVALID;
    if (dst_is_device) {
      e = launch_unpack_u8(h->g, h->grid, static_cast<uint8_t*>(dst), h->stream, h->tracer);
    } else {
      RunState s{};
      const int rc = read_state(h, &s);
      if (rc != QSGS_OK) return rc;
      if (s.status == kRunning) return QSGS_ERR_STATE;  // the front area is still live
      uint8_t* staging = reinterpret_cast<uint8_t*>(h->list);
      e = launch_unpack_u8(h->g, h->grid, staging, h->stream, h->tracer);
      if (e == cudaSuccess) e = cudaMemcpyAsync(dst, staging, n, kind, h->stream);
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

void qsgs_destroy(qsgs_handle* h) {
  if (!h) return;
  destroy_graph(h);
  delete h;
}

}  // extern "C"
