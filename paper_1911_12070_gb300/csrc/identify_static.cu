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

constexpr unsigned long long kStagingBytes = (unsigned long long)QTV_STATIC_MAX_FACES * 4ull;
constexpr unsigned long long kSegBytes = (unsigned long long)QTV_STATIC_MAX_SEGMENTS * 8ull;
constexpr unsigned long long kSegOffBytes = (unsigned long long)QTV_STATIC_MAX_SEGMENTS * 8ull;
constexpr unsigned long long kCounterBytes = 256ull;
constexpr unsigned long long kStaticBytes = kStagingBytes + kSegBytes + kSegOffBytes + kCounterBytes;

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
  uint32_t* staging = reinterpret_cast<uint32_t*>(base);
  uint2* seg = reinterpret_cast<uint2*>(base + kStagingBytes);
  unsigned long long* seg_off = reinterpret_cast<unsigned long long*>(base + kStagingBytes + kSegBytes);
  unsigned long long* counters =
      reinterpret_cast<unsigned long long*>(base + kStagingBytes + kSegBytes + kSegOffBytes);
  // identify_launch only reads the SM count and the (off) trace switch of its
  // handle argument; a stack handle carries them without any allocation.
  qtv_handle_s tmp;
  tmp.device = dev;
  tmp.num_sms = num_sms;
  return identify_launch(&tmp, g, reinterpret_cast<const float2*>(psi), face_ids, winding,
                         capacity, count, nullptr, st, staging, capacity, seg, seg_off, counters);
}
