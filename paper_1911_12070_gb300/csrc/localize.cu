// localize.cu -- density-guided sub-grid localization (Sec. 3.3.3, Eq. 6) of
// a list of pierced plaquettes (see localize_impl.cuh), and packing of
// samples for emission.
#include "localize_impl.cuh"

namespace qtv {
namespace {

// One face per thread (two per thread with both faces' loads in flight was
// slower: 75 registers cost more occupancy than the second face hid latency).
constexpr int kLocThreads = 256;

__global__ void __launch_bounds__(kLocThreads) localize_kernel(
    const float2* __restrict__ psi, int nx, int ny, int nz, float h, float ox, float oy, float oz,
    const uint64_t* __restrict__ face_ids, const int8_t* __restrict__ winding,
    unsigned long long n, const uint64_t* __restrict__ n_dev, float* __restrict__ xyz,
    float* __restrict__ resid, uint8_t* __restrict__ flags) {
  pdl_wait();  // the face list (and its count) of the previous kernel
  unsigned long long nn = n;
  if (n_dev) {
    const unsigned long long d = *n_dev;
    nn = d < n ? d : n;
  }
  for (unsigned long long f = (unsigned long long)blockIdx.x * kLocThreads + threadIdx.x; f < nn;
       f += (unsigned long long)gridDim.x * kLocThreads) {
    float p[3], r;
    uint8_t fl;
    loc::localize_face(psi, nx, ny, nz, h, ox, oy, oz, face_ids[f], winding[f], p, &r, &fl);
    xyz[3 * f + 0] = p[0];
    xyz[3 * f + 1] = p[1];
    xyz[3 * f + 2] = p[2];
    resid[f] = r;
    flags[f] = fl;
  }
}

__global__ void emit_pack_kernel(unsigned long long n, const uint64_t* __restrict__ face_ids,
                                 const int8_t* __restrict__ winding, const float* __restrict__ xyz,
                                 const float* __restrict__ resid, const uint8_t* __restrict__ flags,
                                 qtv_sample* __restrict__ out) {
  for (unsigned long long f = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; f < n;
       f += (unsigned long long)gridDim.x * blockDim.x) {
    qtv_sample s;
    s.x = xyz[3 * f];
    s.y = xyz[3 * f + 1];
    s.z = xyz[3 * f + 2];
    s.resid = resid[f];
    s.face_id = face_ids[f];
    s.winding = winding[f];
    s.flags = flags ? flags[f] : 0;
    s.reserved0 = 0;
    s.reserved1 = 0;
    out[f] = s;
  }
}

}  // namespace

int localize_launch(qtv_handle h, const qtv_grid& g, const float2* psi, const uint64_t* face_ids,
                    const int8_t* winding, uint64_t n, const uint64_t* n_dev, float* xyz,
                    float* resid, uint8_t* flags, cudaStream_t st) {
  if (n == 0) return QTV_OK;
  TraceScope ts(h, K_LOCALIZE, st);
  unsigned long long blocks = (n + kLocThreads - 1) / kLocThreads;
  if (blocks > 65535ull * 4) blocks = 65535ull * 4;
  cudaError_t e = launch_dependent(localize_kernel, dim3((unsigned)blocks), dim3(kLocThreads), 0,
                                   st, psi, g.nx, g.ny, g.nz, g.h, g.origin[0], g.origin[1],
                                   g.origin[2], face_ids, winding, (unsigned long long)n, n_dev,
                                   xyz, resid, flags);
  if (e == cudaSuccess) e = cudaGetLastError();
  return check_cuda(e, "localize_kernel launch");
}

int emit_pack_launch(qtv_handle h, uint64_t n, const uint64_t* face_ids, const int8_t* winding,
                     const float* xyz, const float* resid, const uint8_t* flags, qtv_sample* out,
                     cudaStream_t st) {
  if (n == 0) return QTV_OK;
  TraceScope ts(h, K_EMIT_PACK, st);
  unsigned long long blocks = (n + 255) / 256;
  if (blocks > 65535ull * 4) blocks = 65535ull * 4;
  emit_pack_kernel<<<(unsigned)blocks, 256, 0, st>>>(n, face_ids, winding, xyz, resid, flags, out);
  return check_cuda(cudaGetLastError(), "emit_pack_kernel launch");
}

}  // namespace qtv
