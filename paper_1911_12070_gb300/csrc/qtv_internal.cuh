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
enum KernelId { K_SWEEP = 0, K_SEG_SCAN, K_SCATTER, K_STATS, K_LOCALIZE, K_EMIT_PACK, K_COUNT };
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
  std::vector<qtv::TraceRec> trace;      // recorded, not yet read
  std::vector<cudaEvent_t> event_pool;   // free events
  qtv::Locator* loc = nullptr;           // learned locator (weights, Adam state, buffers)
};

namespace qtv {
// Records start/stop events around a launch while tracing is enabled.
struct TraceScope {
  qtv_handle h;
  int kernel;
  cudaStream_t st;
  cudaEvent_t a = nullptr, b = nullptr;
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
int identify_needs(int num_sms, const qtv_grid& g, uint64_t capacity, const void* psi,
                   uint64_t max_warps, IdentNeeds* n);
int identify_launch(qtv_handle h, const qtv_grid& g, const float2* psi, uint64_t* face_ids,
                    int8_t* winding, uint64_t capacity, uint64_t* count, qtv_stats* stats,
                    cudaStream_t st, const IdentScratch& sc, uint64_t max_warps,
                    float* xyz = nullptr, float* resid = nullptr, uint8_t* flags = nullptr);

// Bulk-copy staged sweep with per-warp compaction (sweep_bulk.cu): even
// nx <= 1024, 16-byte aligned psi.
struct BulkNeeds {
  uint64_t recs = 0, table = 0, seg_off = 0, tiles = 0, segf = 0;
};
bool sweep_bulk_supported(int nx, int ny, int nz, const void* psi);
int bulk_needs(int num_sms, const qtv_grid& g, uint64_t capacity, uint64_t max_warps,
               BulkNeeds* n);
int bulk_identify(qtv_handle h, const qtv_grid& g, const float2* psi, uint64_t* face_ids,
                  int8_t* winding, uint64_t capacity, uint64_t* count, qtv_stats* stats,
                  cudaStream_t st, const IdentScratch& sc, uint64_t max_warps,
                  float* xyz = nullptr, float* resid = nullptr, uint8_t* flags = nullptr);

// Localization launch (localize.cu)
int localize_launch(qtv_handle h, const qtv_grid& g, const float2* psi, const uint64_t* face_ids,
                    const int8_t* winding, uint64_t n, const uint64_t* n_dev, float* xyz,
                    float* resid, uint8_t* flags, cudaStream_t st);

// Learned localization with plain fallback (locator.cu)
int locator_localize(qtv_handle h, const qtv_grid& g, const float2* psi, const uint64_t* face_ids,
                     const int8_t* winding, uint64_t n, const uint64_t* n_dev, float thresh,
                     float* xyz, float* resid, uint8_t* flags, cudaStream_t st);

// Emission pack (localize.cu)
int emit_pack_launch(qtv_handle h, uint64_t n, const uint64_t* face_ids, const int8_t* winding, const float* xyz,
                     const float* resid, const uint8_t* flags, qtv_sample* out, cudaStream_t st);

}  // namespace qtv
