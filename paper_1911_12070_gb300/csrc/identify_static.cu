// identify_static.cu -- qtv_identify_static: identification that allocates
// nothing.  Its scratch (the compaction staging records, the per-segment
// table and the counters that qtv_identify keeps in handle workspace) lives in
// one file-scope __device__ array of fixed size, so the call needs neither a
// handle nor any cudaMalloc.  Everything else runs through the same launch
// code as qtv_identify.
#include <mutex>

#include "qtv_internal.cuh"

namespace qtv {
namespace {

// Layout of the scratch array.  Staging holds up to one 24-byte record per
// pierced face, plus the slack that per-warp record chunks may leave unused
// (2 chunks of 32 records for each of at most kMaxWarps resident warps).
constexpr unsigned long long kMaxWarps = 4096;
constexpr unsigned long long kStagingWords =
    6ull * ((unsigned long long)QTV_STATIC_MAX_FACES + 2ull * 32 * kMaxWarps + 32);
constexpr unsigned long long kTableEntries = (unsigned long long)QTV_STATIC_MAX_WARP_SEGMENTS;
constexpr unsigned long long kTileEntries = 256;
constexpr unsigned long long kStagingBytes = kStagingWords * 4ull;
constexpr unsigned long long kTableBytes = kTableEntries * 16ull;
constexpr unsigned long long kSegBytes = (unsigned long long)QTV_STATIC_MAX_SEGMENTS * 8ull;
constexpr unsigned long long kSegOffBytes = (unsigned long long)QTV_STATIC_MAX_SEGMENTS * 8ull;
constexpr unsigned long long kTileBytes = kTileEntries * 8ull;
constexpr unsigned long long kCounterBytes = 256ull;
constexpr unsigned long long kStaticBytes =
    kTableBytes + kSegBytes + kSegOffBytes + kTileBytes + kCounterBytes + kStagingBytes;

// The scratch.  In host code this name is only a host-side stand-in: the
// device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
unsigned char* g_addr[kMaxDevices] = {};
int g_num_sms[kMaxDevices] = {};

// Once per device, with that device current: resolve the device address of
// the scratch array and the SM count.
int setup_device(int dev, unsigned char** addr, int* num_sms) {
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return check_cuda(e, "cudaGetSymbolAddress(static scratch)");
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return check_cuda(e, "cudaDeviceGetAttribute(SM count)");
    g_num_sms[dev] = sms;
    g_addr[dev] = static_cast<unsigned char*>(p);
  }
  *addr = g_addr[dev];
  *num_sms = g_num_sms[dev];
  return QTV_OK;
}

}  // namespace
}  // namespace qtv

using namespace qtv;

extern "C" int qtv_identify_static(const qtv_grid* grid, const void* psi, uint64_t* face_ids,
                                   int8_t* winding, uint64_t capacity, uint64_t* count,
                                   void* stream) {
  if (!grid) return set_error(QTV_ERR_ARG, "grid is NULL");
  const qtv_grid& g = *grid;
  if (g.nx < 0 || g.ny < 0 || g.nz < 0)
    return set_error(QTV_ERR_ARG, "negative grid size (%d, %d, %d)", g.nx, g.ny, g.nz);
  if (g.periodic != 0) return set_error(QTV_ERR_ARG, "periodic grids are not supported");
  if (g.nx > 64 * kMaxWarpsX)
    return set_error(QTV_ERR_ARG, "nx = %d exceeds the supported maximum %d", g.nx,
                     64 * kMaxWarpsX);
  if (!(g.h > 0.f)) return set_error(QTV_ERR_ARG, "grid spacing h must be positive");
  if (!count) return set_error(QTV_ERR_ARG, "count is NULL");
  if (capacity > 0 && (!face_ids || !winding))
    return set_error(QTV_ERR_ARG, "face_ids / winding are NULL with capacity %llu",
                     (unsigned long long)capacity);
  if (capacity > QTV_STATIC_MAX_FACES)
    return set_error(QTV_ERR_ARG,
                     "qtv_identify_static: capacity %llu exceeds the static scratch limit of "
                     "%u faces (QTV_STATIC_MAX_FACES); use qtv_identify with a handle",
                     (unsigned long long)capacity, (unsigned)QTV_STATIC_MAX_FACES);
  const unsigned long long nbands = ((unsigned long long)g.ny + kRows - 1) / kRows;
  const unsigned long long nseg = nbands * (unsigned long long)g.nz;
  if (nseg > QTV_STATIC_MAX_SEGMENTS)
    return set_error(QTV_ERR_ARG,
                     "qtv_identify_static: grid needs %llu segments (nz * ceil(ny / %d)), above "
                     "the static scratch limit of %u (QTV_STATIC_MAX_SEGMENTS)",
                     nseg, kRows, (unsigned)QTV_STATIC_MAX_SEGMENTS);
  const unsigned long long nn = (unsigned long long)g.nx * g.ny * g.nz;
  if (nn > 0 && !psi) return set_error(QTV_ERR_ARG, "psi is NULL");
  if (reinterpret_cast<uintptr_t>(psi) & 7u)
    return set_error(QTV_ERR_ARG, "psi must be 8-byte aligned");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return check_cuda(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return set_error(QTV_ERR_ARG, "device %d unsupported", dev);
  unsigned char* base = nullptr;
  int num_sms = 0;
  int rc = setup_device(dev, &base, &num_sms);
  if (rc) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (nn == 0) return check_cuda(cudaMemsetAsync(count, 0, sizeof(uint64_t), st), "cudaMemsetAsync");
  IdentNeeds need;
  // the nibble sweep: its staging grows with the pierced faces, not the grid
  qtv_handle_s tmp;
  tmp.device = dev;
  tmp.num_sms = num_sms;
  tmp.sweep_variant = 0;
  rc = identify_needs(&tmp, num_sms, g, capacity, psi, kMaxWarps, &need);
  if (rc) return rc;
  if (need.table > kTableEntries)
    return set_error(QTV_ERR_ARG,
                     "qtv_identify_static: grid needs %llu (plane, band, warp) table entries "
                     "(nz * ceil(ny / 7) * ceil(nx / 64)), above the static scratch limit of %u "
                     "(QTV_STATIC_MAX_WARP_SEGMENTS)",
                     (unsigned long long)need.table, (unsigned)QTV_STATIC_MAX_WARP_SEGMENTS);
  if (need.staging > kStagingWords || need.seg > QTV_STATIC_MAX_SEGMENTS ||
      need.seg_off > QTV_STATIC_MAX_SEGMENTS || need.tiles > kTileEntries)
    return set_error(QTV_ERR_ARG, "qtv_identify_static: request exceeds the static scratch");
  unsigned char* p = base;
  IdentScratch sc;
  sc.table = reinterpret_cast<uint4*>(p);
  sc.table_cap = kTableEntries;
  p += kTableBytes;
  sc.seg = reinterpret_cast<uint2*>(p);
  sc.seg_cap = QTV_STATIC_MAX_SEGMENTS;
  p += kSegBytes;
  sc.seg_off = reinterpret_cast<unsigned long long*>(p);
  sc.seg_off_cap = QTV_STATIC_MAX_SEGMENTS;
  p += kSegOffBytes;
  sc.tiles = reinterpret_cast<unsigned long long*>(p);
  sc.tiles_cap = kTileEntries;
  p += kTileBytes;
  sc.counters = reinterpret_cast<unsigned long long*>(p);
  p += kCounterBytes;
  sc.staging = reinterpret_cast<uint32_t*>(p);
  sc.staging_cap = kStagingWords;
  // identify_launch only reads the SM count, the sweep choice and the (off)
  // trace switch of its handle argument; a stack handle carries them without
  // any allocation.
  return identify_launch(&tmp, g, reinterpret_cast<const float2*>(psi), face_ids, winding,
                         capacity, count, nullptr, st, sc, kMaxWarps);
}
