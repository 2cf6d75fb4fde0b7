// qtv_internal.cuh -- shared device helpers and host-side plumbing of libqtv.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/qtv.h"

namespace qtv {

// ---------------------------------------------------------------------------
// Error reporting (thread-local text behind qtv_last_error_string).
// ---------------------------------------------------------------------------
int set_error(int code, const char* fmt, ...);
int check_cuda(cudaError_t e, const char* what);

// ---------------------------------------------------------------------------
// Programmatic dependent launch.  A kernel launched by launch_dependent may
// start while the previous kernel of the stream is still running: its blocks
// wait in pdl_wait() (first statement, before any global memory access) until
// that kernel has finished and its writes are visible.  pdl_trigger() in the
// previous kernel lets the dependent launch before all of its blocks exit
// (once every block has triggered); without it, at exit.  Outside such a
// launch both are no-ops.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_dependent(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                    cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

// Makes a device current for a scope and restores the caller's device.
struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// Workspace owned by a handle.
struct Workspace {
  uint32_t* staging = nullptr;        // staged face records of the sweep
  uint64_t staging_cap = 0;           // records
  uint2* seg = nullptr;               // per (plane, band) segment {count, base}
  uint64_t seg_cap = 0;               // entries
  unsigned long long* counters = nullptr;  // [0] staging bump, [1] overflow, [2..] spare
  unsigned long long* seg_off = nullptr;   // per segment output offset (exclusive scan)
  uint64_t seg_off_cap = 0;
  qtv_sample* pack = nullptr;         // emission staging (device)
  uint64_t pack_cap = 0;
  uint4* table = nullptr;             // per (plane, band, warp) record table
  uint64_t table_cap = 0;
  unsigned long long* tiles = nullptr;  // look-back state of the segment scan
  uint64_t tiles_cap = 0;
};

// Raw scratch pointers of one identification call (handle workspace or the
// static array of qtv_identify_static).
struct IdentScratch {
  uint32_t* staging = nullptr;  // face records (register sweep) / lane-row records (staged sweep)
  uint64_t staging_cap = 0;
  uint2* seg = nullptr;         // per (plane, band): {count, base} (register sweep) or
                                // two u32 face totals per entry (staged sweep)
  uint64_t seg_cap = 0;
  uint4* table = nullptr;       // staged sweep: per (plane, band, warp) entry
  uint64_t table_cap = 0;
  unsigned long long* seg_off = nullptr;
  uint64_t seg_off_cap = 0;
  unsigned long long* tiles = nullptr;
  uint64_t tiles_cap = 0;
  unsigned long long* counters = nullptr;  // 8 words
};

// Entries of each scratch array that one call needs.
struct IdentNeeds {
  uint64_t staging = 0, seg = 0, table = 0, seg_off = 0, tiles = 0;
};

}  // namespace qtv

#include <vector>

namespace qtv {
struct Locator;  // learned locator state (locator.cu)
void locator_free(Locator* L);
enum KernelId {
  K_SWEEP = 0, K_SEG_SCAN, K_SCATTER, K_STATS, K_LOCALIZE, K_EMIT_PACK, K_BATCH,
  K_ENCODE, K_NETWORK, K_HEAD, K_NODE_FORM, K_NODE_SCAN, K_NODE_SCATTER, K_DENSITY, K_REFINE, K_GRAPH, K_LINES, K_CURVES, K_THIN, K_REDUCE, K_NODE_FACES, K_COUNT
};
struct BatchPlan;  // batched snapshots (batch.cu)
void batch_free(BatchPlan* b);
struct NodeWork;   // node-form and density-error workspace (node_form.cu)
void node_work_free(NodeWork* w);
struct GraphWork;  // face-graph workspace (graph.cu)
void graph_work_free(GraphWork* w);
struct LineWork;   // line-extraction workspace (lines.cu)
void line_work_free(LineWork* w);
struct ReduceWork;  // box-reduction workspace (reduce.cu)
void reduce_work_free(ReduceWork* w);
struct NodeFacesWork;  // node form from a face list (node_faces.cu)
void node_faces_work_free(NodeFacesWork* w);
struct HostPipe;   // double-buffered device copies for calls from host memory (api.cu)
void host_pipe_free(HostPipe* p);
struct TraceRec {
  int kernel;
  cudaEvent_t start, stop;
};
}  // namespace qtv

struct qtv_handle_s {
  int device = 0;
  int num_sms = 0;
  qtv::Workspace ws;
  bool trace_on = false;
  int trace_only = -1;                   // trace one kernel name only (-1 = all)
  std::vector<qtv::TraceRec> trace;      // recorded, not yet read
  std::vector<cudaEvent_t> event_pool;   // free events
  qtv::Locator* loc = nullptr;           // learned locator (weights, Adam state, buffers)
  qtv::BatchPlan* batch = nullptr;       // batch plan, scratch and captured graph
  qtv::NodeWork* node = nullptr;         // node-form / density-error workspace
  qtv::GraphWork* graph = nullptr;       // face-graph workspace
  qtv::LineWork* lines = nullptr;        // line-extraction workspace
  qtv::ReduceWork* reduce = nullptr;     // box-reduction workspace
  qtv::NodeFacesWork* nodef = nullptr;   // node form from a face list
  qtv::HostPipe* pipe = nullptr;         // calls from host memory
  unsigned long long* refine_counter = nullptr;  // work counter of the refinement kernel
  // sweep shape of single-snapshot calls (qtv_configure_sweep); -1 / 0 = default
  int sweep_variant = -1, sweep_nwt = 0, sweep_stages = 0, sweep_ctas = 0;
  // failure injection (qtv_inject_scan_hold): a look-back tile of the segment
  // scan that never publishes its state (-1: none) and the spin limit, in SM
  // cycles, of the look-back waits (0: the default of about 2^32)
  long long scan_hold_tile = -1;
  long long scan_spin_limit = 0;
};

namespace qtv {
// Records start/stop events around a launch while tracing is enabled.
struct TraceScope {
  qtv_handle h;
  int kernel;
  cudaStream_t st;
  cudaEvent_t a = nullptr, b = nullptr;
  bool captured = false;
  TraceScope(qtv_handle h_, int k, cudaStream_t s);
  ~TraceScope();
};
}  // namespace qtv

namespace qtv {

// ---------------------------------------------------------------------------
// Identification launch (identify.cu)
// ---------------------------------------------------------------------------
struct SweepArgs {
  const float2* psi;
  int nx, ny, nz;
  int nbands;      // ceil(ny / kRows)
  int kchunk;      // planes per work item
  int nitems;      // nbands * ceil(nz / kchunk)
  uint32_t* staging;
  unsigned long long staging_cap;
  unsigned long long* staging_top;
  uint2* seg;      // [nz][nbands]
  qtv_stats* stats;
};

constexpr int kRows = 7;          // owned rows per band (plus one halo row)
constexpr int kMaxWarpsX = 32;    // nx <= 64 * 32

// max_warps bounds the resident warps of the staged sweep (0 = no bound); it
// bounds the staging slack that per-warp record chunks can leave unused.
int identify_needs(qtv_handle h, int num_sms, const qtv_grid& g, uint64_t capacity,
                   const void* psi, uint64_t max_warps, IdentNeeds* n);
int identify_launch(qtv_handle h, const qtv_grid& g, const float2* psi, uint64_t* face_ids,
                    int8_t* winding, uint64_t capacity, uint64_t* count, qtv_stats* stats,
                    cudaStream_t st, const IdentScratch& sc, uint64_t max_warps,
                    float* xyz = nullptr, float* resid = nullptr, uint8_t* flags = nullptr);

// Bulk-copy staged sweeps (sweep_bulk.cu, sweep_bits.cu): even nx and a
// 16-byte aligned psi; nx <= 1024 for the nibble sweep, <= 2048 for the
// bit-sliced one.
struct BulkNeeds {
  uint64_t recs = 0, table = 0, seg_off = 0, tiles = 0, segf = 0;
};

// One snapshot of a sweep.  Its work units are (plane, band, x tile) triples
// in (z block, band, tile, plane) order; units, segments ((plane, band)
// pairs) and table entries ((plane, band, tile, warp)) of all snapshots are
// numbered consecutively.
struct SnapDesc {
  const float2* psi = nullptr;
  int nx = 0, ny = 0, nz = 0;
  int nbands = 0;   // ceil(ny / kRows)
  int ntx = 1;      // x tiles per row
  int st = 0;       // x stride of the tiles (even); tile t stages columns
                    // [t st, t st + st + 2), the last one [t st, nx)
  int hblock = 1;   // planes per z block
  int nwt = 1;      // warps per x tile (tile width 64 nwt columns)
  int nstk = 0;     // bit-sliced sweep: columns of stacked last tiles (0: none)
  long long unit0 = 0, seg0 = 0, tab0 = 0;  // first unit / segment / table entry
};
constexpr int kMaxSnaps = QTV_BATCH_MAX;

// Kernel parameters of the sweep and the expand pass (passed by value).
struct BulkParams {
  SnapDesc s[kMaxSnaps];
  int nsnap = 0;
  int nwt = 0;      // warps per tile of the sweep launch (its CTA width)
  long long units = 0, nseg = 0;
  uint32_t* recs = nullptr;
  unsigned long long recs_cap = 0;   // records
  unsigned long long* counters = nullptr;  // [0] chunk top, [1] status bits, [2] scan ticket
  uint4* table = nullptr;
  unsigned int* segf = nullptr;      // pierced faces per segment (zeroed before)
};

// Tunable shape of a sweep: warps per x tile for every snapshot (0: per
// snapshot, one tile as wide as its row), resident CTAs per SM (0: as many as
// fit), a factor on the z-block height, and whether the sweeps of snapshot
// groups of different tile widths run concurrently (each on a share of the
// GPU in proportion to its nodes) or one after the other.
// variant 0: nibble sweep (7-row bands, 64 columns per warp); variant 1:
// bit-sliced sweep (16-row bands, 31 columns per warp, 2 or 3 ring stages).
struct TileConfig {
  int nwt = 0;
  int ctas_per_sm = 0;
  float zscale = 1.f;
  int concurrent = 0;
  int variant = 0;
  int stages = 3;
};

// One sweep launch: the snapshots of one group (same warps per tile), units
// numbered within the group, segments and table entries numbered globally.
struct BulkLayout {
  BulkParams p;
  int grid = 0, threads = 0;
  size_t smem = 0;
};

// A whole pass: the sweep launches of all groups, and the parameters of the
// expand pass over all snapshots in their given order.
struct BatchLayout {
  std::vector<BulkLayout> groups;
  std::vector<int> group_of;
  BulkParams fin;
  int variant = 0, stages = 3;
  int rec_words = 6;  // 32-bit words per staged record
  bool concurrent = false;
  int expand_blocks = 1;
  long long ntiles = 0;  // scan tiles
  unsigned long long recs_need = 0, table_need = 0;
};

// Streams and events for concurrent sweeps (fork from and join into the
// launching stream).
struct SweepBranches {
  int n = 0;
  cudaStream_t streams[kMaxSnaps];
  cudaEvent_t fork;
  cudaEvent_t join[kMaxSnaps];
};

// Geometry of the faces of one call: one grid, or the concatenated face lists
// of several snapshots (snapshot s owns faces [offsets[s], offsets[s + 1]);
// offsets is device memory and is read only when n > 1).
struct GridGeo {
  const float2* psi = nullptr;
  int nx = 0, ny = 0, nz = 0;
  float h = 1.f, ox = 0.f, oy = 0.f, oz = 0.f;
};
struct FaceGeo {
  GridGeo g[kMaxSnaps];
  int n = 0;
  const uint64_t* offsets = nullptr;
};
inline FaceGeo single_geo(const qtv_grid& g, const float2* psi) {
  FaceGeo f;
  f.n = 1;
  f.g[0].psi = psi;
  f.g[0].nx = g.nx;
  f.g[0].ny = g.ny;
  f.g[0].nz = g.nz;
  f.g[0].h = g.h;
  f.g[0].ox = g.origin[0];
  f.g[0].oy = g.origin[1];
  f.g[0].oz = g.origin[2];
  return f;
}
#ifdef __CUDACC__
// (i, j, k) of the linear node index lin = (k ny + j) nx + i; two divisions,
// in 32 bits whenever lin fits (every grid below 2^32 nodes)
__device__ __forceinline__ void split_lin(unsigned long long lin, long long nx, long long ny,
                                          long long& i, long long& j, long long& k) {
  if ((lin >> 32) == 0ull) {
    const uint32_t l = (uint32_t)lin, q1 = l / (uint32_t)nx, q2 = q1 / (uint32_t)ny;
    i = (long long)(l - q1 * (uint32_t)nx);
    j = (long long)(q1 - q2 * (uint32_t)ny);
    k = (long long)q2;
  } else {
    const unsigned long long q1 = lin / (unsigned long long)nx, q2 = q1 / (unsigned long long)ny;
    i = (long long)(lin - q1 * (unsigned long long)nx);
    j = (long long)(q1 - q2 * (unsigned long long)ny);
    k = (long long)q2;
  }
}

// snapshot of face f: the largest s with offsets[s] <= f
__device__ __forceinline__ int geo_snapshot(const FaceGeo& G, unsigned long long f) {
  if (G.n <= 1) return 0;
  int lo = 0, hi = G.n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(G.offsets + mid) <= f) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}
#endif

int bulk_variant_occupancy(int nw, int* ctas_per_sm, size_t* smem);
// bit-sliced sweep (sweep_bits.cu)
int bits_variant_occupancy(int nw, int stages, int* ctas_per_sm, size_t* smem);
void bits_sweep_launch(const BulkParams& p, int grid, int nw, int stages, size_t smem,
                       cudaStream_t st);
// resident CTAs per SM of the bit-sliced expand kernel (its launch bound)
constexpr int kBitsExpandCtasPerSm = 3;
// (tile, warp) steps per band row the bit-sliced expand handles (31 columns
// each: nx up to 2976); the nibble sweep's expand handles 32
constexpr int kBitsBandWarps = 96;
constexpr int kNibbleBandWarps = 32;
cudaError_t bits_expand_launch(const BulkParams& p, int blocks, const unsigned long long* seg_off,
                               uint64_t* face_ids, int8_t* winding, unsigned long long capacity,
                               uint64_t* offsets, cudaStream_t st);
int batch_layout(int num_sms, int nsnap, const qtv_grid* grids, const float2* const* psis,
                 const TileConfig& tc, uint64_t capacity, uint64_t max_warps, BatchLayout* B);
int batch_launch(qtv_handle h, BatchLayout& B, const IdentScratch& sc, uint64_t* face_ids,
                 int8_t* winding, uint64_t capacity, uint64_t* count, uint64_t* offsets,
                 qtv_stats* stats, unsigned long long scanned, cudaStream_t st, bool expand_always,
                 const SweepBranches* br);
int batch_sweep_only(qtv_handle h, BatchLayout& B, const IdentScratch& sc, cudaStream_t st,
                     const SweepBranches* br);
// whether a staged sweep (variant 1: bit-sliced, 0: nibble) can take a grid
bool sweep_bulk_supported(int variant, int nx, int ny, int nz, const void* psi);
// the staged sweep a single-snapshot call of handle h takes for a grid: the
// handle's variant when it can, else the nibble sweep when that can, else -1
// (the register sweep of identify.cu)
int staged_variant(const qtv_handle_s* h, int nx, int ny, int nz, const void* psi);
int bulk_needs(qtv_handle h, int num_sms, const qtv_grid& g, uint64_t capacity,
               uint64_t max_warps, BulkNeeds* n);
int bulk_identify(qtv_handle h, const qtv_grid& g, const float2* psi, uint64_t* face_ids,
                  int8_t* winding, uint64_t capacity, uint64_t* count, qtv_stats* stats,
                  cudaStream_t st, const IdentScratch& sc, uint64_t max_warps,
                  float* xyz = nullptr, float* resid = nullptr, uint8_t* flags = nullptr);

// Box-mean reduction of a sample graph (reduce.cu)
int box_reduce_launch(qtv_handle h, uint64_t n, const uint64_t* n_dev, const uint32_t* nbr,
                      const uint8_t* deg, int stride, const float* xyz, float box, int max_passes,
                      uint32_t* label, double* out_xyz, uint64_t* counts, cudaStream_t st);

// Localization launch (localize.cu)
int localize_launch(qtv_handle h, const qtv_grid& g, const float2* psi, const uint64_t* face_ids,
                    const int8_t* winding, uint64_t n, const uint64_t* n_dev, float* xyz,
                    float* resid, uint8_t* flags, cudaStream_t st);

// Learned localization with plain fallback (locator.cu); n faces (at most
// *n_dev when n_dev is given) processed in chunks of locator rows
int locator_localize(qtv_handle h, const FaceGeo& geo, const uint64_t* face_ids,
                     const int8_t* winding, uint64_t n, const uint64_t* n_dev, float thresh,
                     float* xyz, float* resid, uint8_t* flags, cudaStream_t st);
// Allocates the locator's row buffers for the chunk that n faces use (outside
// stream capture) and reports how often they have been reallocated (a graph
// that captured them is stale once this changes); QTV_ERR_STATE when no
// locator is loaded.
int locator_prepare(qtv_handle h, uint64_t n, uint64_t* generation);

// C[M][N] = A[M][K] B[N][K]^T on tcgen05 (locator_tc.cu); epi 0 FP32 (split K
// summed in order), 1 relu(. + bias) BF16, 2 masked by mask > 0 BF16
int tc_gemm(const uint16_t* A, long long lda, const uint16_t* B, long long ldb, long long M, int N,
            long long K, int splits, int epi, float* C, long long ldc, float* part, uint16_t* O,
            long long ldo, uint16_t* OT, long long ldot, const float* bias, const uint16_t* mask,
            long long ldm, unsigned int* status, cudaStream_t st);
// The whole network, fused (locator_tc.cu): Y[M][3] from X[M][128] (W1, W2
// BF16; biases and W3 FP32); X 16-byte aligned, M below 2^31.
int tc_mlp_forward(const uint16_t* X, long long M, const uint16_t* W1, const uint16_t* W2,
                   const float* b1, const float* b2, const float* w3, const float* b3, float* Y,
                   unsigned int* status, int num_sms, cudaStream_t st);

// rows[r] = first index a with ids[a] >= (r nx) << shift, r in [0, R]
// (graph.cu); ids ascending, n or *n_dev of them
cudaError_t row_table_launch(const uint64_t* ids, unsigned long long n, const uint64_t* n_dev,
                             int nx, long long R, int shift, uint32_t* rows, int num_sms,
                             cudaStream_t st);
// Node form of the circulation: vortex nodes in ascending order with their
// three ring windings, optional dense field (node_form.cu)
int node_circulation_launch(qtv_handle h, const qtv_grid& g, const float2* psi,
                            uint64_t* node_ids, int8_t* circ, uint64_t capacity, uint64_t* count,
                            int8_t* dense, cudaStream_t st);
// Density error of Eq. 7 at n sample points (node_form.cu)
int density_error_launch(qtv_handle h, const qtv_grid& g, const float2* psi, const float* xyz,
                         uint64_t n, const uint64_t* n_dev, float* rho, double* out,
                         cudaStream_t st);

// Sample refinement in the plane normal to the pseudo-vorticity (refine.cu)
int refine_launch(qtv_handle h, const qtv_grid& g, const float2* psi, const float* xyz0,
                  const uint64_t* face_ids, uint64_t n, const uint64_t* n_dev, int max_iter,
                  float tol, float* xyz, float* rho, float* tangent, float* detj, int32_t* iters,
                  uint8_t* flags, cudaStream_t st);

// Face graph and connected components (graph.cu)
// (nodes: the list holds vortex-node indices and the graph is 6-connected)
int face_graph_launch(qtv_handle h, const qtv_grid& g, const uint64_t* face_ids, uint64_t n,
                      const uint64_t* n_dev, uint32_t* nbr, uint8_t* deg, uint32_t* comp,
                      uint64_t* ncomp, cudaStream_t st, bool nodes = false);

// Line pieces and curves of a sample graph (lines.cu)
int line_pieces_launch(qtv_handle h, uint64_t n, const uint64_t* n_dev, const uint32_t* nbr,
                       const uint8_t* deg, const uint32_t* comp, const float* xyz,
                       const uint64_t* face_ids, const int8_t* winding, qtv_piece* pieces,
                       uint64_t piece_cap, uint32_t* nodes, uint64_t node_cap, uint64_t* counts,
                       cudaStream_t st);
int piece_curves_launch(qtv_handle h, const float* xyz, const uint32_t* nodes,
                        const qtv_piece* pieces, uint64_t np, const uint64_t* np_dev, int per,
                        float* curve, uint64_t curve_cap, uint64_t* curve_first, float* length,
                        uint64_t* total, cudaStream_t st);

// Arc-length thinning of line pieces (lines.cu)
int thin_pieces_launch(qtv_handle h, const float* xyz, const uint32_t* nodes,
                       const qtv_piece* pieces, uint64_t np, uint64_t nnodes, float box,
                       float* out_xyz, uint64_t out_cap, qtv_piece* out_pieces, uint64_t* total,
                       cudaStream_t st);

// Emission pack (localize.cu)
int emit_pack_launch(qtv_handle h, uint64_t n, const uint64_t* face_ids, const int8_t* winding, const float* xyz,
                     const float* resid, const uint8_t* flags, qtv_sample* out, cudaStream_t st);

}  // namespace qtv
