// api.cu -- the C ABI of libqtv (include/qtv.h): argument validation, handle
// workspace, and dispatch to the kernels.  Nothing here computes on the host.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "qtv_internal.cuh"

namespace qtv {

namespace {
thread_local std::string g_err;

// Makes the handle's device current for the scope of an API call.


bool capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return false;
  return cs != cudaStreamCaptureStatusNone;
}

template <typename T>
int grow(T*& p, uint64_t& cap, uint64_t want, cudaStream_t st, const char* what) {
  if (want <= cap && p) return QTV_OK;
  if (capturing(st))
    return set_error(QTV_ERR_STATE, "%s: workspace must grow to %llu entries during stream capture;"
                     " call qtv_reserve before capturing", what, (unsigned long long)want);
  if (p) {
    cudaFree(p);
    p = nullptr;
    cap = 0;
  }
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&p), want * sizeof(T));
  if (e != cudaSuccess) {
    p = nullptr;
    return check_cuda(e, what);
  }
  cap = want;
  return QTV_OK;
}

int validate_grid(const qtv_grid* g) {
  if (!g) return set_error(QTV_ERR_ARG, "grid is NULL");
  if (g->nx < 0 || g->ny < 0 || g->nz < 0)
    return set_error(QTV_ERR_ARG, "negative grid size (%d, %d, %d)", g->nx, g->ny, g->nz);
  if (g->periodic != 0) return set_error(QTV_ERR_ARG, "periodic grids are not supported");
  if (g->nx > 64 * kMaxWarpsX)
    return set_error(QTV_ERR_ARG, "nx = %d exceeds the supported maximum %d", g->nx,
                     64 * kMaxWarpsX);
  const unsigned long long n = (unsigned long long)g->nx * g->ny * g->nz;
  if (n >> 60) return set_error(QTV_ERR_ARG, "grid too large");
  if (!(g->h > 0.f)) return set_error(QTV_ERR_ARG, "grid spacing h must be positive");
  return QTV_OK;
}

// Grow the handle workspace to what one identification call needs.
int grow_identify(qtv_handle h, const qtv_grid& g, uint64_t capacity, const void* psi,
                  cudaStream_t st) {
  IdentNeeds n;
  int rc = identify_needs(h, h->num_sms, g, capacity, psi, 0, &n);
  if (rc) return rc;
  if (n.staging > 0xFFFFFFFFull)
    return set_error(QTV_ERR_ARG, "staging above 2^32 records is not supported");
  rc = grow(h->ws.staging, h->ws.staging_cap, n.staging > 0 ? n.staging : 1, st,
            "cudaMalloc(staging)");
  if (!rc && n.seg) rc = grow(h->ws.seg, h->ws.seg_cap, n.seg, st, "cudaMalloc(seg)");
  if (!rc && n.table) rc = grow(h->ws.table, h->ws.table_cap, n.table, st, "cudaMalloc(table)");
  if (!rc && n.seg_off)
    rc = grow(h->ws.seg_off, h->ws.seg_off_cap, n.seg_off, st, "cudaMalloc(seg_off)");
  if (!rc && n.tiles) rc = grow(h->ws.tiles, h->ws.tiles_cap, n.tiles, st, "cudaMalloc(tiles)");
  return rc;
}

IdentScratch scratch_of(qtv_handle h) {
  IdentScratch sc;
  sc.staging = h->ws.staging;
  sc.staging_cap = h->ws.staging_cap;
  sc.seg = h->ws.seg;
  sc.seg_cap = h->ws.seg_cap;
  sc.table = h->ws.table;
  sc.table_cap = h->ws.table_cap;
  sc.seg_off = h->ws.seg_off;
  sc.seg_off_cap = h->ws.seg_off_cap;
  sc.tiles = h->ws.tiles;
  sc.tiles_cap = h->ws.tiles_cap;
  sc.counters = h->ws.counters;
  return sc;
}
}  // namespace

int set_error(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int check_cuda(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return QTV_OK;
  // clear the runtime's last-error state (a failed non-launch call would
  // otherwise be reported again by the next launch check)
  (void)cudaGetLastError();
  return set_error(QTV_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

namespace {
cudaEvent_t take_event(qtv_handle h) {
  if (!h->event_pool.empty()) {
    cudaEvent_t e = h->event_pool.back();
    h->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}
const char* kKernelNames[K_COUNT] = {"sweep",     "seg_scan",  "scatter",      "stats",
                                     "localize",  "emit_pack", "batch",        "encode",
                                     "network",   "head",      "node_form",    "node_scan",
                                     "node_scatter", "density",   "refine",       "graph",
                                     "lines",     "curves",    "thin",      "reduce",
                                     "node_faces"};
}  // namespace

// Inside a stream capture the records become event-record nodes of the graph
// (cudaEventRecordExternal), so each replay times the launch.
TraceScope::TraceScope(qtv_handle h_, int k, cudaStream_t s) : h(h_), kernel(k), st(s) {
  if (!h || !h->trace_on || (h->trace_only >= 0 && h->trace_only != k)) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return;
  captured = cs == cudaStreamCaptureStatusActive;
  a = take_event(h);
  b = take_event(h);
  if (a && b) cudaEventRecordWithFlags(a, st, captured ? cudaEventRecordExternal : 0u);
}

TraceScope::~TraceScope() {
  if (!a || !b) {
    if (a) h->event_pool.push_back(a);
    if (b) h->event_pool.push_back(b);
    return;
  }
  cudaEventRecordWithFlags(b, st, captured ? cudaEventRecordExternal : 0u);
  h->trace.push_back(TraceRec{kernel, a, b});
}

// Double-buffered device state of qtv_identify_localize_host: call i uses
// buffer i % 2; its copy from the host runs on the pipe's own stream and waits
// only for the call that used the same buffer two calls earlier.
struct HostPipe {
  cudaStream_t copy = nullptr;
  cudaEvent_t ready[2] = {nullptr, nullptr}, done[2] = {nullptr, nullptr};
  bool used[2] = {false, false};
  float2* psi[2] = {nullptr, nullptr};
  size_t psi_bytes = 0;
  uint64_t* ids[2] = {nullptr, nullptr};
  int8_t* w[2] = {nullptr, nullptr};
  float* xyz[2] = {nullptr, nullptr};
  float* resid[2] = {nullptr, nullptr};
  uint8_t* flags[2] = {nullptr, nullptr};
  uint64_t* count[2] = {nullptr, nullptr};
  qtv_sample* pack[2] = {nullptr, nullptr};
  uint64_t cap = 0;
  int next = 0;
};

namespace {
void pipe_free_buffers(HostPipe* p, bool field, bool outputs) {
  for (int b = 0; b < 2; ++b) {
    if (field) {
      cudaFree(p->psi[b]);
      p->psi[b] = nullptr;
    }
    if (outputs) {
      cudaFree(p->ids[b]);
      cudaFree(p->w[b]);
      cudaFree(p->xyz[b]);
      cudaFree(p->resid[b]);
      cudaFree(p->flags[b]);
      cudaFree(p->count[b]);
      cudaFree(p->pack[b]);
      p->ids[b] = nullptr;
      p->w[b] = nullptr;
      p->xyz[b] = nullptr;
      p->resid[b] = nullptr;
      p->flags[b] = nullptr;
      p->count[b] = nullptr;
      p->pack[b] = nullptr;
    }
  }
  if (field) p->psi_bytes = 0;
  if (outputs) p->cap = 0;
}
}  // namespace

void host_pipe_free(HostPipe* p) {
  if (!p) return;
  pipe_free_buffers(p, true, true);
  for (int b = 0; b < 2; ++b) {
    if (p->ready[b]) cudaEventDestroy(p->ready[b]);
    if (p->done[b]) cudaEventDestroy(p->done[b]);
  }
  if (p->copy) cudaStreamDestroy(p->copy);
  delete p;
}

}  // namespace qtv

using namespace qtv;

extern "C" {

int qtv_version(void) { return (1 << 16) | 0; }

const char* qtv_last_error_string(void) { return g_err.c_str(); }

int qtv_create(qtv_handle* out, int device) {
  if (!out) return set_error(QTV_ERR_ARG, "out is NULL");
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return check_cuda(e, "cudaGetDeviceCount");
  if (device < 0 || device >= ndev)
    return set_error(QTV_ERR_ARG, "device %d out of range (%d devices)", device, ndev);
  DeviceGuard dg(device);
  if (!dg.ok) return set_error(QTV_ERR_CUDA, "cudaSetDevice(%d) failed", device);
  qtv_handle h = new (std::nothrow) qtv_handle_s();
  if (!h) return set_error(QTV_ERR_ARG, "out of host memory");
  h->device = device;
  e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) {
    delete h;
    return check_cuda(e, "cudaDeviceGetAttribute(SM count)");
  }
  e = cudaMalloc(reinterpret_cast<void**>(&h->ws.counters), 8 * sizeof(unsigned long long));
  if (e != cudaSuccess) {
    delete h;
    return check_cuda(e, "cudaMalloc(counters)");
  }
  *out = h;
  return QTV_OK;
}

int qtv_destroy(qtv_handle h) {
  if (!h) return QTV_OK;
  DeviceGuard dg(h->device);
  cudaDeviceSynchronize();
  cudaFree(h->ws.staging);
  cudaFree(h->ws.seg);
  cudaFree(h->ws.seg_off);
  cudaFree(h->ws.counters);
  cudaFree(h->ws.pack);
  cudaFree(h->ws.table);
  cudaFree(h->ws.tiles);
  locator_free(h->loc);
  batch_free(h->batch);
  node_work_free(h->node);
  graph_work_free(h->graph);
  line_work_free(h->lines);
  reduce_work_free(h->reduce);
  node_faces_work_free(h->nodef);
  host_pipe_free(h->pipe);
  cudaFree(h->refine_counter);
  for (auto& r : h->trace) {
    cudaEventDestroy(r.start);
    cudaEventDestroy(r.stop);
  }
  for (auto e : h->event_pool) cudaEventDestroy(e);
  delete h;
  return QTV_OK;
}

int qtv_configure_sweep(qtv_handle h, int variant, int warps_per_tile, int stages,
                        int ctas_per_sm) {
  if (!h) return set_error(QTV_ERR_ARG, "handle is NULL");
  if (variant < -1 || variant > 1) return set_error(QTV_ERR_ARG, "unknown sweep variant %d", variant);
  if (warps_per_tile < 0 || warps_per_tile > 16 || stages < 0 || stages > 3 || ctas_per_sm < 0)
    return set_error(QTV_ERR_ARG, "sweep shape out of range");
  if (variant == 1 && warps_per_tile != 0 && warps_per_tile != 2 && warps_per_tile != 4 &&
      warps_per_tile != 8)
    return set_error(QTV_ERR_ARG, "bit-sliced sweep: %d warps per tile (2, 4 or 8)",
                     warps_per_tile);
  h->sweep_variant = variant;
  h->sweep_nwt = warps_per_tile;
  h->sweep_stages = stages;
  h->sweep_ctas = ctas_per_sm;
  return QTV_OK;
}

int qtv_inject_scan_hold(qtv_handle h, int64_t hold_tile, int64_t spin_cycles) {
  if (!h) return set_error(QTV_ERR_ARG, "handle is NULL");
  if (hold_tile < -1 || spin_cycles < 0)
    return set_error(QTV_ERR_ARG, "scan hold: tile %lld, spin limit %lld", (long long)hold_tile,
                     (long long)spin_cycles);
  h->scan_hold_tile = hold_tile;
  h->scan_spin_limit = spin_cycles;
  return QTV_OK;
}

int qtv_trace_enable(qtv_handle h, int on) {
  if (!h) return set_error(QTV_ERR_ARG, "handle is NULL");
  h->trace_on = on != 0;
  return QTV_OK;
}

int qtv_trace_filter(qtv_handle h, const char* name) {
  if (!h) return set_error(QTV_ERR_ARG, "handle is NULL");
  if (!name || !name[0]) {
    h->trace_only = -1;
    return QTV_OK;
  }
  for (int k = 0; k < K_COUNT; ++k)
    if (strcmp(name, kKernelNames[k]) == 0) {
      h->trace_only = k;
      return QTV_OK;
    }
  return set_error(QTV_ERR_ARG, "unknown kernel name '%s'", name);
}

int qtv_trace_read(qtv_handle h, qtv_trace_entry* out, int max_entries, int* n_entries,
                   int reset) {
  if (!h) return set_error(QTV_ERR_ARG, "handle is NULL");
  if (!n_entries || (max_entries > 0 && !out)) return set_error(QTV_ERR_ARG, "NULL output");
  DeviceGuard dg(h->device);
  double tot[K_COUNT] = {0};
  uint32_t cnt[K_COUNT] = {0};
  for (auto& r : h->trace) {
    cudaError_t e = cudaEventSynchronize(r.stop);
    if (e != cudaSuccess) return check_cuda(e, "cudaEventSynchronize(trace)");
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, r.start, r.stop);
    if (e != cudaSuccess) return check_cuda(e, "cudaEventElapsedTime(trace)");
    tot[r.kernel] += ms;
    cnt[r.kernel] += 1;
  }
  int n = 0;
  for (int k = 0; k < K_COUNT; ++k) {
    if (!cnt[k]) continue;
    if (n < max_entries) {
      memset(out[n].name, 0, sizeof out[n].name);
      strncpy(out[n].name, kKernelNames[k], sizeof out[n].name - 1);
      out[n].launches = cnt[k];
      out[n].total_ms = (float)tot[k];
    }
    ++n;
  }
  *n_entries = n;
  if (reset) {
    for (auto& r : h->trace) {
      h->event_pool.push_back(r.start);
      h->event_pool.push_back(r.stop);
    }
    h->trace.clear();
  }
  return QTV_OK;
}

int qtv_reserve(qtv_handle h, const qtv_grid* grid, uint64_t max_faces) {
  if (!h) return set_error(QTV_ERR_ARG, "handle is NULL");
  int rc = validate_grid(grid);
  if (rc) return rc;
  DeviceGuard dg(h->device);
  if (max_faces > 0xFFFFFFFFull)
    return set_error(QTV_ERR_ARG, "max_faces above 2^32-1 is not supported");
  // psi alignment decides the kernel; reserve for the staged sweep's layout
  rc = grow_identify(h, *grid, max_faces, reinterpret_cast<const void*>(256), nullptr);
  if (rc) return rc;
  rc = grow(h->ws.pack, h->ws.pack_cap, max_faces > 0 ? max_faces : 1, nullptr,
            "cudaMalloc(pack)");
  if (rc) return rc;
  return check_cuda(cudaDeviceSynchronize(), "qtv_reserve");
}

int qtv_identify(qtv_handle h, const qtv_grid* grid, const void* psi, uint64_t* face_ids,
                 int8_t* winding, uint64_t capacity, uint64_t* count, qtv_stats* stats,
                 void* stream) {
  if (!h) return set_error(QTV_ERR_ARG, "handle is NULL");
  int rc = validate_grid(grid);
  if (rc) return rc;
  if (!count) return set_error(QTV_ERR_ARG, "count is NULL");
  if (capacity > 0 && (!face_ids || !winding))
    return set_error(QTV_ERR_ARG, "face_ids / winding are NULL with capacity %llu",
                     (unsigned long long)capacity);
  if (capacity > 0xFFFFFFFFull)
    return set_error(QTV_ERR_ARG, "capacity above 2^32-1 is not supported");
  const qtv_grid& g = *grid;
  const unsigned long long nn = (unsigned long long)g.nx * g.ny * g.nz;
  if (nn > 0 && !psi) return set_error(QTV_ERR_ARG, "psi is NULL");
  if (reinterpret_cast<uintptr_t>(psi) & 7u)
    return set_error(QTV_ERR_ARG, "psi must be 8-byte aligned");
  DeviceGuard dg(h->device);
  if (!dg.ok) return set_error(QTV_ERR_CUDA, "cudaSetDevice failed");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (nn == 0 || g.nx < 1 || g.ny < 1 || g.nz < 1) {
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(uint64_t), st);
    if (e == cudaSuccess && stats) e = cudaMemsetAsync(stats, 0, sizeof(qtv_stats), st);
    return check_cuda(e, "cudaMemsetAsync(count)");
  }
  rc = grow_identify(h, g, capacity, psi, st);
  if (rc) return rc;
  return identify_launch(h, g, reinterpret_cast<const float2*>(psi), face_ids, winding, capacity,
                         count, stats, st, scratch_of(h), 0);
}

int qtv_identify_localize(qtv_handle h, const qtv_grid* grid, const void* psi,
                          uint64_t* face_ids, int8_t* winding, uint64_t capacity, uint64_t* count,
                          float* xyz, float* resid, uint8_t* flags, qtv_stats* stats,
                          void* stream) {
  if (!h) return set_error(QTV_ERR_ARG, "handle is NULL");
  int rc = validate_grid(grid);
  if (rc) return rc;
  if (!count) return set_error(QTV_ERR_ARG, "count is NULL");
  if (capacity > 0 && (!face_ids || !winding || !xyz || !resid || !flags))
    return set_error(QTV_ERR_ARG, "an output is NULL with capacity %llu",
                     (unsigned long long)capacity);
  if (capacity > 0xFFFFFFFFull)
    return set_error(QTV_ERR_ARG, "capacity above 2^32-1 is not supported");
  const qtv_grid& g = *grid;
  const unsigned long long nn = (unsigned long long)g.nx * g.ny * g.nz;
  if (nn > 0 && !psi) return set_error(QTV_ERR_ARG, "psi is NULL");
  if (reinterpret_cast<uintptr_t>(psi) & 7u)
    return set_error(QTV_ERR_ARG, "psi must be 8-byte aligned");
  DeviceGuard dg(h->device);
  if (!dg.ok) return set_error(QTV_ERR_CUDA, "cudaSetDevice failed");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (nn == 0 || g.nx < 1 || g.ny < 1 || g.nz < 1) {
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(uint64_t), st);
    if (e == cudaSuccess && stats) e = cudaMemsetAsync(stats, 0, sizeof(qtv_stats), st);
    return check_cuda(e, "cudaMemsetAsync(count)");
  }
  rc = grow_identify(h, g, capacity, psi, st);
  if (rc) return rc;
  return identify_launch(h, g, reinterpret_cast<const float2*>(psi), face_ids, winding, capacity,
                         count, stats, st, scratch_of(h), 0, capacity > 0 ? xyz : nullptr, resid,
                         flags);
}

int qtv_node_circulation(qtv_handle h, const qtv_grid* grid, const void* psi, uint64_t* node_ids,
                         int8_t* circ, uint64_t capacity, uint64_t* count, int8_t* dense,
                         void* stream) {
  if (!h) return set_error(QTV_ERR_ARG, "handle is NULL");
  int rc = validate_grid(grid);
  if (rc) return rc;
  if (!count) return set_error(QTV_ERR_ARG, "count is NULL");
  if (capacity > 0 && (!node_ids || !circ))
    return set_error(QTV_ERR_ARG, "an output list is NULL with capacity %llu",
                     (unsigned long long)capacity);
  if (capacity > 0xFFFFFFFFull)
    return set_error(QTV_ERR_ARG, "capacity above 2^32-1 is not supported");
  const qtv_grid& g = *grid;
  const unsigned long long nn = (unsigned long long)g.nx * g.ny * g.nz;
  if (nn >> 52) return set_error(QTV_ERR_ARG, "grid of 2^52 nodes or more");
  if (nn > 0 && !psi) return set_error(QTV_ERR_ARG, "psi is NULL");
  if (reinterpret_cast<uintptr_t>(psi) & 7u)
    return set_error(QTV_ERR_ARG, "psi must be 8-byte aligned");
  DeviceGuard dg(h->device);
  if (!dg.ok) return set_error(QTV_ERR_CUDA, "cudaSetDevice failed");
  return node_circulation_launch(h, g, reinterpret_cast<const float2*>(psi), node_ids, circ,
                                 capacity, count, dense, reinterpret_cast<cudaStream_t>(stream));
}

int qtv_density_error(qtv_handle h, const qtv_grid* grid, const void* psi, const float* xyz,
                      uint64_t n, const uint64_t* n_dev, float* rho, double* out, void* stream) {
  if (!h) return set_error(QTV_ERR_ARG, "handle is NULL");
  int rc = validate_grid(grid);
  if (rc) return rc;
  if (!out) return set_error(QTV_ERR_ARG, "out is NULL");
  const qtv_grid& g = *grid;
  const unsigned long long nn = (unsigned long long)g.nx * g.ny * g.nz;
  if (nn == 0) return set_error(QTV_ERR_ARG, "empty grid");
  if (!psi) return set_error(QTV_ERR_ARG, "psi is NULL");
  if (reinterpret_cast<uintptr_t>(psi) & 7u)
    return set_error(QTV_ERR_ARG, "psi must be 8-byte aligned");
  if (n > 0 && !xyz)
    return set_error(QTV_ERR_ARG, "xyz is NULL with n = %llu", (unsigned long long)n);
  DeviceGuard dg(h->device);
  if (!dg.ok) return set_error(QTV_ERR_CUDA, "cudaSetDevice failed");
  return density_error_launch(h, g, reinterpret_cast<const float2*>(psi), xyz, n, n_dev, rho, out,
                              reinterpret_cast<cudaStream_t>(stream));
}

int qtv_refine_samples(qtv_handle h, const qtv_grid* grid, const void* psi, const float* xyz0,
                       const uint64_t* face_ids, uint64_t n, const uint64_t* n_dev, int max_iter,
                       float tol, float* xyz, float* rho, float* tangent, float* detj,
                       int32_t* iters, uint8_t* flags, void* stream) {
  if (!h) return set_error(QTV_ERR_ARG, "handle is NULL");
  int rc = validate_grid(grid);
  if (rc) return rc;
  if (n == 0) return QTV_OK;
  if ((xyz0 == nullptr) == (face_ids == nullptr))
    return set_error(QTV_ERR_ARG, "give exactly one of xyz0 and face_ids");
  if (!psi || !xyz || !flags) return set_error(QTV_ERR_ARG, "a required pointer is NULL");
  if (reinterpret_cast<uintptr_t>(psi) & 7u)
    return set_error(QTV_ERR_ARG, "psi must be 8-byte aligned");
  const qtv_grid& g = *grid;
  if ((unsigned long long)g.nx * g.ny * g.nz == 0) return set_error(QTV_ERR_ARG, "empty grid");
  if (max_iter < 0) return set_error(QTV_ERR_ARG, "max_iter must be >= 0");
  if (!(tol > 0.f)) return set_error(QTV_ERR_ARG, "tol must be positive");
  DeviceGuard dg(h->device);
  if (!dg.ok) return set_error(QTV_ERR_CUDA, "cudaSetDevice failed");
  return refine_launch(h, g, reinterpret_cast<const float2*>(psi), xyz0, face_ids, n, n_dev,
                       max_iter, tol, xyz, rho, tangent, detj, iters, flags,
                       reinterpret_cast<cudaStream_t>(stream));
}

int qtv_face_graph(qtv_handle h, const qtv_grid* grid, const uint64_t* face_ids, uint64_t n,
                   const uint64_t* n_dev, uint32_t* nbr, uint8_t* deg, uint32_t* comp,
                   uint64_t* ncomp, void* stream) {
  if (!h) return set_error(QTV_ERR_ARG, "handle is NULL");
  int rc = validate_grid(grid);
  if (rc) return rc;
  if (!ncomp) return set_error(QTV_ERR_ARG, "ncomp is NULL");
  if (n > 0 && (!face_ids || !nbr || !deg || !comp))
    return set_error(QTV_ERR_ARG, "a required pointer is NULL");
  if (n >= 0xFFFFFFFFull) return set_error(QTV_ERR_ARG, "2^32 - 1 faces or more");
  const qtv_grid& g = *grid;
  if ((unsigned long long)g.ny * g.nz >= 0xFFFFFFFFull)
    return set_error(QTV_ERR_ARG, "too many grid rows");
  DeviceGuard dg(h->device);
  if (!dg.ok) return set_error(QTV_ERR_CUDA, "cudaSetDevice failed");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (n == 0 || (unsigned long long)g.nx * g.ny * g.nz == 0) {
    const cudaError_t e = cudaMemsetAsync(ncomp, 0, sizeof(uint64_t), st);
    return check_cuda(e, "cudaMemsetAsync(ncomp)");
  }
  return face_graph_launch(h, g, face_ids, n, n_dev, nbr, deg, comp, ncomp, st);
}

int qtv_line_pieces(qtv_handle h, uint64_t n, const uint64_t* n_dev, const uint32_t* nbr,
                    const uint8_t* deg, const uint32_t* comp, const float* xyz,
                    const uint64_t* face_ids, const int8_t* winding, qtv_piece* pieces,
                    uint64_t piece_cap, uint32_t* nodes, uint64_t node_cap, uint64_t* counts,
                    void* stream) {
  if (!h) return set_error(QTV_ERR_ARG, "handle is NULL");
  if (!counts) return set_error(QTV_ERR_ARG, "counts is NULL");
  if (n >= 0xFFFFFFFFull / 11) return set_error(QTV_ERR_ARG, "too many samples");
  if (n > 0 && (!nbr || !deg || !comp || !xyz))
    return set_error(QTV_ERR_ARG, "a required pointer is NULL");
  if ((face_ids == nullptr) != (winding == nullptr))
    return set_error(QTV_ERR_ARG, "give both face_ids and winding, or neither");
  if ((piece_cap > 0 && !pieces) || (node_cap > 0 && !nodes))
    return set_error(QTV_ERR_ARG, "an output is NULL with a nonzero capacity");
  DeviceGuard dg(h->device);
  if (!dg.ok) return set_error(QTV_ERR_CUDA, "cudaSetDevice failed");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (n == 0) {
    const cudaError_t e = cudaMemsetAsync(counts, 0, 2 * sizeof(uint64_t), st);
    return check_cuda(e, "cudaMemsetAsync(counts)");
  }
  return line_pieces_launch(h, n, n_dev, nbr, deg, comp, xyz, face_ids, winding, pieces,
                            piece_cap, nodes, node_cap, counts, st);
}

int qtv_piece_curves(qtv_handle h, const float* xyz, const uint32_t* nodes,
                     const qtv_piece* pieces, uint64_t npieces, const uint64_t* npieces_dev,
                     int per_segment, float* curve, uint64_t curve_cap, uint64_t* curve_first,
                     float* length, uint64_t* total, void* stream) {
  if (!h) return set_error(QTV_ERR_ARG, "handle is NULL");
  if (!total) return set_error(QTV_ERR_ARG, "total is NULL");
  if (per_segment < 1 || per_segment > 1024)
    return set_error(QTV_ERR_ARG, "per_segment must be in [1, 1024]");
  if (npieces >= 0xFFFFFFFFull) return set_error(QTV_ERR_ARG, "too many pieces");
  if (npieces > 0 && (!xyz || !nodes || !pieces || !curve_first || !length))
    return set_error(QTV_ERR_ARG, "a required pointer is NULL");
  if (curve_cap > 0 && !curve) return set_error(QTV_ERR_ARG, "curve is NULL");
  DeviceGuard dg(h->device);
  if (!dg.ok) return set_error(QTV_ERR_CUDA, "cudaSetDevice failed");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (npieces == 0) {
    const cudaError_t e = cudaMemsetAsync(total, 0, sizeof(uint64_t), st);
    return check_cuda(e, "cudaMemsetAsync(total)");
  }
  return piece_curves_launch(h, xyz, nodes, pieces, npieces, npieces_dev, per_segment, curve,
                             curve_cap, curve_first, length, total, st);
}

int qtv_identify_localize_host(qtv_handle h, const qtv_grid* grid, const void* psi_host,
                               uint64_t capacity, qtv_sample* host_out, uint64_t* host_count,
                               void* stream) {
  if (!h) return set_error(QTV_ERR_ARG, "handle is NULL");
  int rc = validate_grid(grid);
  if (rc) return rc;
  if (!host_count) return set_error(QTV_ERR_ARG, "host_count is NULL");
  if (capacity > 0 && !host_out) return set_error(QTV_ERR_ARG, "host_out is NULL");
  if (capacity > 0xFFFFFFFFull)
    return set_error(QTV_ERR_ARG, "capacity above 2^32-1 is not supported");
  const qtv_grid& g = *grid;
  const unsigned long long nn = (unsigned long long)g.nx * g.ny * g.nz;
  if (nn > 0 && !psi_host) return set_error(QTV_ERR_ARG, "psi_host is NULL");
  DeviceGuard dg(h->device);
  if (!dg.ok) return set_error(QTV_ERR_CUDA, "cudaSetDevice failed");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (capturing(st)) return set_error(QTV_ERR_STATE, "not available during stream capture");
  if (!h->pipe) {
    HostPipe* p = new (std::nothrow) HostPipe();
    if (!p) return set_error(QTV_ERR_ARG, "out of host memory");
    cudaError_t e = cudaStreamCreateWithFlags(&p->copy, cudaStreamNonBlocking);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
      e = cudaEventCreateWithFlags(&p->ready[b], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->done[b], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
      host_pipe_free(p);
      return check_cuda(e, "host pipe streams and events");
    }
    h->pipe = p;
  }
  HostPipe* p = h->pipe;
  const size_t bytes = (size_t)nn * sizeof(float2);
  // (re)allocation synchronises the device, so no call in flight uses the old buffers
  cudaError_t e = cudaSuccess;
  if (bytes > p->psi_bytes) {
    pipe_free_buffers(p, true, false);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b)
      e = cudaMalloc(reinterpret_cast<void**>(&p->psi[b]), bytes > 0 ? bytes : 16);
    if (e != cudaSuccess) {
      pipe_free_buffers(p, true, false);
      return check_cuda(e, "cudaMalloc(host pipe field)");
    }
    p->psi_bytes = bytes;
  }
  const uint64_t cap = capacity > 0 ? capacity : 1;
  if (cap > p->cap) {
    pipe_free_buffers(p, false, true);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
      e = cudaMalloc(reinterpret_cast<void**>(&p->ids[b]), cap * sizeof(uint64_t));
      if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&p->w[b]), cap);
      if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&p->xyz[b]), cap * 12);
      if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&p->resid[b]), cap * 4);
      if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&p->flags[b]), cap);
      if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&p->count[b]), 8);
      if (e == cudaSuccess)
        e = cudaMalloc(reinterpret_cast<void**>(&p->pack[b]), cap * sizeof(qtv_sample));
    }
    if (e != cudaSuccess) {
      pipe_free_buffers(p, false, true);
      return check_cuda(e, "cudaMalloc(host pipe outputs)");
    }
    p->cap = cap;
  }
  const int b = p->next;
  p->next ^= 1;
  rc = grow_identify(h, g, capacity, p->psi[b], st);
  if (rc) return rc;
  // copy of the field: waits only for the call that used this buffer before
  if (p->used[b]) e = cudaStreamWaitEvent(p->copy, p->done[b], 0);
  if (e == cudaSuccess && bytes > 0)
    e = cudaMemcpyAsync(p->psi[b], psi_host, bytes, cudaMemcpyHostToDevice, p->copy);
  if (e == cudaSuccess) e = cudaEventRecord(p->ready[b], p->copy);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, p->ready[b], 0);
  if (e != cudaSuccess) return check_cuda(e, "host pipe copy");
  if (nn == 0 || g.nx < 1 || g.ny < 1 || g.nz < 1) {
    e = cudaMemsetAsync(p->count[b], 0, sizeof(uint64_t), st);
  } else {
    rc = identify_launch(h, g, p->psi[b], p->ids[b], p->w[b], capacity, p->count[b], nullptr, st,
                         scratch_of(h), 0, capacity > 0 ? p->xyz[b] : nullptr, p->resid[b],
                         p->flags[b]);
    if (rc) return rc;
    if (capacity > 0) {
      rc = emit_pack_launch(h, capacity, p->ids[b], p->w[b], p->xyz[b], p->resid[b], p->flags[b],
                            p->pack[b], st);
      if (rc) return rc;
      e = cudaMemcpyAsync(host_out, p->pack[b], capacity * sizeof(qtv_sample),
                          cudaMemcpyDeviceToHost, st);
    }
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(host_count, p->count[b], sizeof(uint64_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaEventRecord(p->done[b], st);
  if (e != cudaSuccess) return check_cuda(e, "host pipe results");
  p->used[b] = true;
  return QTV_OK;
}

int qtv_thin_pieces(qtv_handle h, const float* xyz, const uint32_t* nodes, const qtv_piece* pieces,
                    uint64_t npieces, uint64_t nnodes, float box, float* out_xyz, uint64_t out_cap,
                    qtv_piece* out_pieces, uint64_t* total, void* stream) {
  if (!h) return set_error(QTV_ERR_ARG, "handle is NULL");
  if (!total) return set_error(QTV_ERR_ARG, "total is NULL");
  if (!(box > 0.f)) return set_error(QTV_ERR_ARG, "box must be positive");
  if (npieces > 0 && (!xyz || !nodes || !pieces || !out_pieces))
    return set_error(QTV_ERR_ARG, "a required pointer is NULL");
  if (out_cap > 0 && !out_xyz) return set_error(QTV_ERR_ARG, "out_xyz is NULL");
  if (nnodes >= 0xFFFFFFFFull || npieces > nnodes)
    return set_error(QTV_ERR_ARG, "bad node or piece count");
  DeviceGuard dg(h->device);
  if (!dg.ok) return set_error(QTV_ERR_CUDA, "cudaSetDevice failed");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (npieces == 0) {
    const cudaError_t e = cudaMemsetAsync(total, 0, sizeof(uint64_t), st);
    return check_cuda(e, "cudaMemsetAsync(total)");
  }
  return thin_pieces_launch(h, xyz, nodes, pieces, npieces, nnodes, box, out_xyz, out_cap,
                            out_pieces, total, st);
}

int qtv_box_reduce(qtv_handle h, uint64_t n, const uint64_t* n_dev, const uint32_t* nbr,
                   const uint8_t* deg, int stride, const float* xyz, float box, int max_passes,
                   uint32_t* label, double* out_xyz, uint64_t* counts, void* stream) {
  if (!h) return set_error(QTV_ERR_ARG, "handle is NULL");
  if (!counts) return set_error(QTV_ERR_ARG, "counts is NULL");
  if (n > 0 && (!nbr || !deg || !xyz || !label || !out_xyz))
    return set_error(QTV_ERR_ARG, "a required pointer is NULL");
  if (n >= 0xFFFFFFFFull) return set_error(QTV_ERR_ARG, "too many nodes (%llu)", (unsigned long long)n);
  if (stride < 1 || stride > 64) return set_error(QTV_ERR_ARG, "neighbour stride %d (1 to 64)", stride);
  if (!(box > 0.f && box <= 32.f)) return set_error(QTV_ERR_ARG, "box must be in (0, 32]");
  if (max_passes < 1 || max_passes > 64)
    return set_error(QTV_ERR_ARG, "max_passes %d (1 to 64)", max_passes);
  DeviceGuard dg(h->device);
  if (!dg.ok) return set_error(QTV_ERR_CUDA, "cudaSetDevice failed");
  return box_reduce_launch(h, n, n_dev, nbr, deg, stride, xyz, box, max_passes, label, out_xyz,
                           counts, reinterpret_cast<cudaStream_t>(stream));
}

int qtv_node_graph(qtv_handle h, const qtv_grid* grid, const uint64_t* node_ids, uint64_t n,
                   const uint64_t* n_dev, uint32_t* nbr, uint8_t* deg, uint32_t* comp,
                   uint64_t* ncomp, void* stream) {
  if (!h) return set_error(QTV_ERR_ARG, "handle is NULL");
  int rc = validate_grid(grid);
  if (rc) return rc;
  if (!ncomp) return set_error(QTV_ERR_ARG, "ncomp is NULL");
  if (n > 0 && (!node_ids || !nbr || !deg || !comp))
    return set_error(QTV_ERR_ARG, "a required pointer is NULL");
  if (n >= 0xFFFFFFFFull) return set_error(QTV_ERR_ARG, "2^32 - 1 nodes or more");
  const qtv_grid& g = *grid;
  if ((unsigned long long)g.ny * g.nz >= 0xFFFFFFFFull)
    return set_error(QTV_ERR_ARG, "too many grid rows");
  DeviceGuard dg(h->device);
  if (!dg.ok) return set_error(QTV_ERR_CUDA, "cudaSetDevice failed");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (n == 0 || (unsigned long long)g.nx * g.ny * g.nz == 0) {
    const cudaError_t e = cudaMemsetAsync(ncomp, 0, sizeof(uint64_t), st);
    return check_cuda(e, "cudaMemsetAsync(ncomp)");
  }
  return face_graph_launch(h, g, node_ids, n, n_dev, nbr, deg, comp, ncomp, st, true);
}

int qtv_localize(qtv_handle h, const qtv_grid* grid, const void* psi, const uint64_t* face_ids,
                 const int8_t* winding, uint64_t n, const uint64_t* n_dev, int mode,
                 float fallback_resid, float* xyz, float* resid, uint8_t* flags, void* stream) {
  if (!h) return set_error(QTV_ERR_ARG, "handle is NULL");
  int rc = validate_grid(grid);
  if (rc) return rc;
  if (mode != QTV_PLAIN && mode != QTV_LEARNED)
    return set_error(QTV_ERR_ARG, "unknown localization mode %d", mode);
  if (n == 0) return QTV_OK;
  if (!psi || !face_ids || !winding || !xyz || !resid || !flags)
    return set_error(QTV_ERR_ARG, "a required pointer is NULL");
  if (reinterpret_cast<uintptr_t>(psi) & 7u)
    return set_error(QTV_ERR_ARG, "psi must be 8-byte aligned");
  DeviceGuard dg(h->device);
  if (!dg.ok) return set_error(QTV_ERR_CUDA, "cudaSetDevice failed");
  if (mode == QTV_LEARNED)
    return locator_localize(h, single_geo(*grid, reinterpret_cast<const float2*>(psi)), face_ids,
                            winding, n,
                            n_dev, fallback_resid, xyz, resid, flags,
                            reinterpret_cast<cudaStream_t>(stream));
  return localize_launch(h, *grid, reinterpret_cast<const float2*>(psi), face_ids, winding, n, n_dev,
                         xyz, resid, flags, reinterpret_cast<cudaStream_t>(stream));
}

int qtv_emit_samples(qtv_handle h, uint64_t n, const uint64_t* face_ids, const int8_t* winding,
                     const float* xyz, const float* resid, const uint8_t* flags,
                     qtv_sample* host_out, void* stream) {
  if (!h) return set_error(QTV_ERR_ARG, "handle is NULL");
  if (n == 0) return QTV_OK;
  if (!face_ids || !winding || !xyz || !resid || !host_out)
    return set_error(QTV_ERR_ARG, "a required pointer is NULL");
  DeviceGuard dg(h->device);
  if (!dg.ok) return set_error(QTV_ERR_CUDA, "cudaSetDevice failed");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int rc = grow(h->ws.pack, h->ws.pack_cap, n, st, "cudaMalloc(pack)");
  if (rc) return rc;
  rc = emit_pack_launch(h, n, face_ids, winding, xyz, resid, flags, h->ws.pack, st);
  if (rc) return rc;
  return check_cuda(cudaMemcpyAsync(host_out, h->ws.pack, n * sizeof(qtv_sample),
                                    cudaMemcpyDeviceToHost, st),
                    "cudaMemcpyAsync(samples)");
}

}  // extern "C"
