// batch.cu -- many snapshots through one pass.
//
// A batch plan holds up to kMaxSnaps snapshots of any (uneven) grid sizes.
// Their work units, (plane, band, x tile) triples, are numbered consecutively
// and cut into one contiguous range per CTA of ONE persistent sweep launch, so
// CTAs run across snapshot boundaries and no launch drains between
// snapshots.  The per-segment face totals of all snapshots form one sequence:
// one scan and one expand pass give one face list in which every snapshot
// owns a contiguous, face-id ordered slice, and one localization pass (plain
// or learned) covers all faces.  The whole sequence is captured once into a
// CUDA graph and replayed by qtv_batch_run; it is captured again only when
// the output buffers or the localization mode change.
//
// Autotuning.  The shape of the sweep (warps per x tile, resident CTAs per SM,
// height of the z blocks) is picked by timing the sweep on the plan's own
// fields over a small grid of candidates; the choice is cached in a text file
// keyed by device and grid sizes.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "localize_impl.cuh"
#include "qtv_internal.cuh"

namespace qtv {

struct BatchPlan {
  int n = 0;
  std::vector<qtv_grid> grids;
  std::vector<const float2*> psis;
  TileConfig tc;
  qtv_batch_info info{};
  // scratch
  uint32_t* staging = nullptr;
  uint64_t staging_cap = 0;  // words
  uint4* table = nullptr;
  uint64_t table_cap = 0;
  unsigned int* segf = nullptr;
  unsigned long long* seg_off = nullptr;
  uint64_t seg_cap = 0;
  unsigned long long* tiles = nullptr;
  uint64_t tiles_cap = 0;
  unsigned long long* counters = nullptr;
  uint64_t* count_buf = nullptr;  // [kMaxSnaps + 1] offsets of the counting pass
  SweepBranches br{};  // streams and events of concurrent group sweeps
  // captured graph and what it was captured for
  cudaStream_t cap = nullptr;
  cudaGraphExec_t exec = nullptr;
  struct Key {
    uint64_t* face_ids;
    int8_t* winding;
    uint64_t capacity;
    uint64_t* offsets;
    float* xyz;
    float* resid;
    uint8_t* flags;
    int mode;
    float thresh;
    uint64_t locator_version;
    bool operator==(const Key& o) const {
      return face_ids == o.face_ids && winding == o.winding && capacity == o.capacity &&
             offsets == o.offsets && xyz == o.xyz && resid == o.resid && flags == o.flags &&
             mode == o.mode && thresh == o.thresh && locator_version == o.locator_version;
    }
  } key{};
  bool have_graph = false;
};

void batch_free(BatchPlan* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (int i = 0; i < b->br.n; ++i) {
    cudaStreamDestroy(b->br.streams[i]);
    cudaEventDestroy(b->br.join[i]);
  }
  if (b->br.n) cudaEventDestroy(b->br.fork);
  cudaFree(b->staging);
  cudaFree(b->table);
  cudaFree(b->segf);
  cudaFree(b->seg_off);
  cudaFree(b->tiles);
  cudaFree(b->counters);
  cudaFree(b->count_buf);
  delete b;
}

namespace {

// plain localization of the concatenated face list (Sec. 3.3.3, Eq. 6)
__global__ void batch_localize_kernel(const __grid_constant__ FaceGeo geo,
                                      const uint64_t* __restrict__ face_ids,
                                      const int8_t* __restrict__ winding, unsigned long long n,
                                      const uint64_t* __restrict__ n_dev, float* __restrict__ xyz,
                                      float* __restrict__ resid, uint8_t* __restrict__ flags) {
  unsigned long long nn = n;
  if (n_dev) {
    const unsigned long long d = *n_dev;
    nn = d < n ? d : n;
  }
  for (unsigned long long f = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; f < nn;
       f += (unsigned long long)gridDim.x * blockDim.x) {
    const GridGeo& g = geo.g[geo_snapshot(geo, f)];
    float p[3], r;
    uint8_t fl;
    loc::localize_face(g.psi, g.nx, g.ny, g.nz, g.h, g.ox, g.oy, g.oz, face_ids[f], winding[f], p,
                       &r, &fl);
    xyz[3 * f + 0] = p[0];
    xyz[3 * f + 1] = p[1];
    xyz[3 * f + 2] = p[2];
    resid[f] = r;
    flags[f] = fl;
  }
}

template <typename T>
int grow(T** p, uint64_t* cap, uint64_t need, const char* what) {
  if (need <= *cap) return QTV_OK;
  cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), need * sizeof(T));
  if (e != cudaSuccess) return check_cuda(e, what);
  *cap = need;
  return QTV_OK;
}

int ensure_scratch(BatchPlan* b, const BatchLayout& L) {
  int rc = grow(&b->staging, &b->staging_cap, L.recs_need * (uint64_t)L.rec_words,
                "cudaMalloc(batch staging)");
  if (!rc) rc = grow(&b->table, &b->table_cap, L.table_need, "cudaMalloc(batch table)");
  // segment totals are addressed as pairs of u32 by the scratch descriptor
  const uint64_t nseg = ((uint64_t)L.fin.nseg + 1) & ~1ull;
  if (!rc && nseg > b->seg_cap) {
    cudaFree(b->segf);
    cudaFree(b->seg_off);
    b->segf = nullptr;
    b->seg_off = nullptr;
    b->seg_cap = 0;
    cudaError_t e = cudaMalloc(&b->segf, nseg * sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMalloc(&b->seg_off, nseg * sizeof(unsigned long long));
    if (e != cudaSuccess) return check_cuda(e, "cudaMalloc(batch segments)");
    b->seg_cap = nseg;
  }
  if (!rc) rc = grow(&b->tiles, &b->tiles_cap, (uint64_t)L.ntiles, "cudaMalloc(batch tiles)");
  return rc;
}

IdentScratch scratch_of(BatchPlan* b) {
  IdentScratch sc;
  sc.staging = b->staging;
  sc.staging_cap = b->staging_cap;
  sc.seg = reinterpret_cast<uint2*>(b->segf);
  sc.seg_cap = b->seg_cap / 2;
  sc.table = b->table;
  sc.table_cap = b->table_cap;
  sc.seg_off = b->seg_off;
  sc.seg_off_cap = b->seg_cap;
  sc.tiles = b->tiles;
  sc.tiles_cap = b->tiles_cap;
  sc.counters = b->counters;
  return sc;
}

FaceGeo geo_of(const BatchPlan* b, const uint64_t* offsets) {
  FaceGeo g;
  g.n = b->n;
  g.offsets = offsets;
  for (int i = 0; i < b->n; ++i) {
    const qtv_grid& q = b->grids[i];
    g.g[i].psi = b->psis[i];
    g.g[i].nx = q.nx;
    g.g[i].ny = q.ny;
    g.g[i].nz = q.nz;
    g.g[i].h = q.h;
    g.g[i].ox = q.origin[0];
    g.g[i].oy = q.origin[1];
    g.g[i].oz = q.origin[2];
  }
  return g;
}

std::string tune_key(const BatchPlan* b, int device, int num_sms) {
  cudaDeviceProp prop;
  std::string name = "device";
  if (cudaGetDeviceProperties(&prop, device) == cudaSuccess) name = prop.name;
  for (auto& c : name)
    if (c == ' ' || c == '\t') c = '_';
  std::string k = name + "|sms=" + std::to_string(num_sms) + "|";
  for (int i = 0; i < b->n; ++i) {
    const qtv_grid& g = b->grids[i];
    if (i) k += ",";
    k += std::to_string(g.nx) + "x" + std::to_string(g.ny) + "x" + std::to_string(g.nz);
  }
  return k;
}

constexpr const char* kTuneTag = "qtv-tune-v3";

bool tune_lookup(const char* path, const std::string& key, TileConfig* tc, float* ms) {
  if (!path || !*path) return false;
  FILE* f = fopen(path, "r");
  if (!f) return false;
  char line[4096];
  bool found = false;
  while (fgets(line, sizeof line, f)) {
    char tag[32], k[3500];
    int var = 0, nwt = 0, ctas = 0, conc = 0, stages = 3;
    float zs = 0.f, t = 0.f;
    if (sscanf(line, "%31s %3499s %d %d %d %f %d %d %f", tag, k, &var, &nwt, &ctas, &zs, &conc,
               &stages, &t) != 9)
      continue;
    if (strcmp(tag, kTuneTag) != 0 || (key != k && strcmp(k, "*") != 0)) continue;
    tc->variant = var;
    tc->nwt = nwt;
    tc->ctas_per_sm = ctas;
    tc->zscale = zs;
    tc->concurrent = conc;
    tc->stages = stages;
    *ms = t;
    found = true;  // the last matching line wins
  }
  fclose(f);
  return found;
}

void tune_store(const char* path, const std::string& key, const TileConfig& tc, float ms) {
  if (!path || !*path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s %s %d %d %d %.3f %d %d %.6f\n", kTuneTag, key.c_str(), tc.variant, tc.nwt,
          tc.ctas_per_sm, tc.zscale, tc.concurrent, tc.stages, ms);
  fclose(f);
}

// Times the sweeps of each candidate shape on the plan's fields; returns the
// fastest (median of 3 timed launches after one warm-up).  Candidates: one
// tile width for all snapshots (64 to 1024 columns), or per-snapshot widths
// with one sweep per width group (serial or concurrent), each with a few
// occupancies and z-block heights.
int autotune(qtv_handle h, BatchPlan* b, uint64_t faces, cudaStream_t st, TileConfig* best,
             float* best_ms, int* ncand) {
  std::vector<TileConfig> cands;
  auto add = [&](int nwt, int ctas, float zs, int conc, int variant = 0, int stages = 3) {
    TileConfig tc;
    tc.nwt = nwt;
    tc.ctas_per_sm = ctas;
    tc.zscale = zs;
    tc.concurrent = conc;
    tc.variant = variant;
    tc.stages = stages;
    BatchLayout L;
    if (batch_layout(h->num_sms, b->n, b->grids.data(), b->psis.data(), tc, faces, 0, &L) ==
        QTV_OK) {
      if (conc && !L.concurrent) return;  // one group: same as serial
      cands.push_back(tc);
    }
  };
  for (int nwt : {2, 4, 8, 16}) {
    int bps = 0;
    size_t smem = 0;
    if (bulk_variant_occupancy(nwt, &bps, &smem)) continue;
    std::vector<int> occ = {bps, std::max(1, (3 * bps) / 4), std::max(1, bps / 2)};
    std::sort(occ.begin(), occ.end());
    occ.erase(std::unique(occ.begin(), occ.end()), occ.end());
    for (int c : occ)
      for (float zs : {0.5f, 1.f, 2.f}) add(nwt, c, zs, 0);
  }
  for (int conc : {0, 1})
    for (int c : {0, 2, 1})
      for (float zs : {0.5f, 1.f, 2.f}) add(0, c, zs, conc);
  // bit-sliced sweep: one tile width for all snapshots
  for (int nwt : {2, 4, 8})
    for (int stages : {2, 3}) {
      int bps = 0;
      size_t smem = 0;
      if (bits_variant_occupancy(nwt, stages, &bps, &smem)) continue;
      std::vector<int> occ = {bps, std::max(1, bps / 2)};
      occ.erase(std::unique(occ.begin(), occ.end()), occ.end());
      for (int c : occ)
        for (float zs : {1.f, 2.f}) add(nwt, c, zs, 0, 1, stages);
    }
  if (cands.empty()) return set_error(QTV_ERR_ARG, "no sweep shape fits this batch");
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return check_cuda(cudaGetLastError(), "event");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return check_cuda(cudaGetLastError(), "event");
  }
  int rc = QTV_OK;
  *best_ms = 1e30f;
  for (const TileConfig& tc : cands) {
    BatchLayout L;
    rc = batch_layout(h->num_sms, b->n, b->grids.data(), b->psis.data(), tc, faces, 0, &L);
    if (!rc) rc = ensure_scratch(b, L);
    if (rc) break;
    IdentScratch sc = scratch_of(b);
    float t[3];
    for (int r = 0; r < 4 && !rc; ++r) {
      cudaEventRecord(e0, st);
      rc = batch_sweep_only(h, L, sc, st, &b->br);
      cudaEventRecord(e1, st);
      if (!rc) rc = check_cuda(cudaEventSynchronize(e1), "autotune sync");
      if (!rc && r > 0) cudaEventElapsedTime(&t[r - 1], e0, e1);
    }
    if (rc) break;
    std::sort(t, t + 3);
    if (t[1] < *best_ms) {
      *best_ms = t[1];
      *best = tc;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ncand = (int)cands.size();
  return rc;
}

}  // namespace
}  // namespace qtv

using namespace qtv;

extern "C" {

int qtv_batch_plan(qtv_handle h, int n, const qtv_grid* grids, const void* const* psis,
                   const char* tune_cache, void* stream) {
  if (!h) return set_error(QTV_ERR_ARG, "handle is NULL");
  if (n < 1 || n > kMaxSnaps)
    return set_error(QTV_ERR_ARG, "%d snapshots (1 to %d supported)", n, kMaxSnaps);
  if (!grids || !psis) return set_error(QTV_ERR_ARG, "grids or psis is NULL");
  for (int i = 0; i < n; ++i) {
    const qtv_grid& g = grids[i];
    if (g.nx < 2 || g.ny < 1 || g.nz < 1 || (g.nx & 1) || g.nx > 64 * kMaxWarpsX)
      return set_error(QTV_ERR_ARG, "snapshot %d: grid %d x %d x %d (even nx in [2, %d], "
                       "ny, nz >= 1 required)", i, g.nx, g.ny, g.nz, 64 * kMaxWarpsX);
    if (g.periodic != 0) return set_error(QTV_ERR_ARG, "snapshot %d: periodic grids are not supported", i);
    if (!(g.h > 0.f)) return set_error(QTV_ERR_ARG, "snapshot %d: grid spacing must be positive", i);
    if (!psis[i] || (reinterpret_cast<uintptr_t>(psis[i]) & 15u))
      return set_error(QTV_ERR_ARG, "snapshot %d: psi is NULL or not 16-byte aligned", i);
  }
  DeviceGuard dg(h->device);
  if (!dg.ok) return set_error(QTV_ERR_CUDA, "cudaSetDevice failed");
  cudaError_t e = cudaSuccess;
  batch_free(h->batch);
  h->batch = nullptr;
  BatchPlan* b = new (std::nothrow) BatchPlan();
  if (!b) return set_error(QTV_ERR_ARG, "out of host memory");
  h->batch = b;
  b->n = n;
  b->grids.assign(grids, grids + n);
  for (int i = 0; i < n; ++i) b->psis.push_back(reinterpret_cast<const float2*>(psis[i]));
  e = cudaMalloc(&b->counters, 8 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&b->count_buf, (kMaxSnaps + 1) * sizeof(uint64_t));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) return check_cuda(e, "qtv_batch_plan allocation");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);

  // branch streams for concurrent group sweeps: one per distinct row width
  {
    std::vector<int> widths;
    for (int i = 0; i < n; ++i) {
      const int w = (grids[i].nx + 63) / 64;
      if (std::find(widths.begin(), widths.end(), w) == widths.end()) widths.push_back(w);
    }
    if (widths.size() > 1) {
      e = cudaEventCreateWithFlags(&b->br.fork, cudaEventDisableTiming);
      if (e != cudaSuccess) return check_cuda(e, "cudaEventCreate(fork)");
      for (size_t i = 0; i < widths.size(); ++i) {
        e = cudaStreamCreateWithFlags(&b->br.streams[i], cudaStreamNonBlocking);
        if (e == cudaSuccess)
          e = cudaEventCreateWithFlags(&b->br.join[i], cudaEventDisableTiming);
        if (e != cudaSuccess) {
          if (b->br.streams[i]) cudaStreamDestroy(b->br.streams[i]);
          return check_cuda(e, "branch stream");
        }
        b->br.n = (int)i + 1;
      }
    }
  }
  // counting pass with the default shape (the bit-sliced sweep where a grid
  // is wider than the nibble sweep takes): the face total sizes the staging
  // of the candidates (face totals do not depend on the staging size)
  BatchLayout L0;
  TileConfig t0;
  int rc = batch_layout(h->num_sms, n, b->grids.data(), b->psis.data(), t0, 0, 0, &L0);
  if (rc == QTV_ERR_ARG) {
    t0.variant = 1;
    rc = batch_layout(h->num_sms, n, b->grids.data(), b->psis.data(), t0, 0, 0, &L0);
  }
  if (rc) return rc;
  rc = ensure_scratch(b, L0);
  if (rc) return rc;
  const bool tr = h->trace_on;
  h->trace_on = false;
  rc = batch_launch(h, L0, scratch_of(b), nullptr, nullptr, 0, b->count_buf + n, b->count_buf,
                    nullptr, 0, st, true, nullptr);
  h->trace_on = tr;
  if (rc) return rc;
  uint64_t total = 0;
  e = cudaMemcpyAsync(&total, b->count_buf + n, sizeof total, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return check_cuda(e, "qtv_batch_plan counting pass");
  if (total == QTV_COUNT_TIMEOUT)
    return set_error(QTV_ERR_TIMEOUT, "qtv_batch_plan: a bounded device wait gave up");
  b->info.faces = total;
  unsigned long long nodes = 0;
  for (int i = 0; i < n; ++i)
    nodes += (unsigned long long)grids[i].nx * grids[i].ny * grids[i].nz;
  b->info.nodes = nodes;

  const std::string key = tune_key(b, h->device, h->num_sms);
  float ms = 0.f;
  TileConfig tc;
  if (tune_lookup(tune_cache, key, &tc, &ms)) {
    BatchLayout Lc;
    if (batch_layout(h->num_sms, n, b->grids.data(), b->psis.data(), tc, total, 0, &Lc) ==
        QTV_OK) {
      b->tc = tc;
      b->info.source = 1;
      b->info.tuned_ms = ms;
    }
  }
  if (b->info.source == 0) {
    int ncand = 0;
    rc = autotune(h, b, total, st, &tc, &ms, &ncand);
    if (rc) return rc;
    b->tc = tc;
    b->info.source = 2;
    b->info.tuned_ms = ms;
    b->info.candidates = ncand;
    tune_store(tune_cache, key, tc, ms);
  }
  b->info.warps_per_tile = b->tc.nwt;
  b->info.ctas_per_sm = b->tc.ctas_per_sm;
  b->info.zscale = b->tc.zscale;
  b->info.concurrent = b->tc.concurrent;
  b->info.variant = b->tc.variant;
  b->info.stages = b->tc.stages;
  BatchLayout L;
  rc = batch_layout(h->num_sms, n, b->grids.data(), b->psis.data(), b->tc, total, 0, &L);
  if (rc) return rc;
  b->info.grid = 0;
  for (const BulkLayout& g : L.groups) b->info.grid += g.grid;
  b->info.sweeps = (int)L.groups.size();
  b->info.tile_columns = b->tc.variant == 1 ? 31 * L.fin.s[0].nwt : 64 * b->tc.nwt;
  return QTV_OK;
}

int qtv_batch_info_get(qtv_handle h, qtv_batch_info* out) {
  if (!h || !out) return set_error(QTV_ERR_ARG, "handle or out is NULL");
  if (!h->batch) return set_error(QTV_ERR_STATE, "no batch plan");
  *out = h->batch->info;
  return QTV_OK;
}

int qtv_batch_run(qtv_handle h, uint64_t* face_ids, int8_t* winding, uint64_t capacity,
                  uint64_t* offsets, float* xyz, float* resid, uint8_t* flags, int mode,
                  float fallback_resid, void* stream) {
  if (!h) return set_error(QTV_ERR_ARG, "handle is NULL");
  BatchPlan* b = h->batch;
  if (!b) return set_error(QTV_ERR_STATE, "no batch plan (call qtv_batch_plan first)");
  if (!offsets) return set_error(QTV_ERR_ARG, "offsets is NULL");
  if (capacity > 0 && (!face_ids || !winding))
    return set_error(QTV_ERR_ARG, "face_ids / winding are NULL with capacity %llu",
                     (unsigned long long)capacity);
  const bool loc = xyz != nullptr;
  if (loc && (!resid || !flags)) return set_error(QTV_ERR_ARG, "xyz given without resid / flags");
  if (mode != QTV_PLAIN && mode != QTV_LEARNED)
    return set_error(QTV_ERR_ARG, "unknown localization mode %d", mode);
  DeviceGuard dg(h->device);
  if (!dg.ok) return set_error(QTV_ERR_CUDA, "cudaSetDevice failed");
  cudaError_t e = cudaSuccess;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  BatchPlan::Key key{face_ids, winding, capacity, offsets, xyz, resid, flags,
                     loc ? mode : -1, loc ? fallback_resid : 0.f, 0};
  if (loc && mode == QTV_LEARNED) {
    int rc = locator_prepare(h, capacity, &key.locator_version);
    if (rc) return rc;
  }
  if (!b->have_graph || !(key == b->key)) {
    BatchLayout L;
    int rc = batch_layout(h->num_sms, b->n, b->grids.data(), b->psis.data(), b->tc, capacity, 0, &L);
    if (!rc) rc = ensure_scratch(b, L);
    if (rc) return rc;
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    b->have_graph = false;
    const bool tr = h->trace_on;
    h->trace_on = false;
    e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      h->trace_on = tr;
      return check_cuda(e, "cudaStreamBeginCapture");
    }
    rc = batch_launch(h, L, scratch_of(b), face_ids, winding, capacity, offsets + b->n, offsets,
                      nullptr, 0, b->cap, true, &b->br);
    if (!rc && loc && capacity > 0) {
      const FaceGeo geo = geo_of(b, offsets);
      if (mode == QTV_LEARNED) {
        rc = locator_localize(h, geo, face_ids, winding, capacity, offsets + b->n, fallback_resid,
                              xyz, resid, flags, b->cap);
      } else {
        unsigned long long blocks = (capacity + 255) / 256;
        if (blocks > 65535ull * 4) blocks = 65535ull * 4;
        batch_localize_kernel<<<(unsigned)blocks, 256, 0, b->cap>>>(
            geo, face_ids, winding, capacity, offsets + b->n, xyz, resid, flags);
        rc = check_cuda(cudaGetLastError(), "batch_localize_kernel launch");
      }
    }
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(b->cap, &graph);
    h->trace_on = tr;
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (e != cudaSuccess) return check_cuda(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return check_cuda(e, "cudaGraphInstantiate");
    b->key = key;
    b->have_graph = true;
  }
  TraceScope ts(h, K_BATCH, st);
  return check_cuda(cudaGraphLaunch(b->exec, st), "cudaGraphLaunch(batch)");
}

}  // extern "C"
