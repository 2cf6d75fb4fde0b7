// node_faces.cu -- the node form of the circulation (Sec. 2.2.2) from the
// pierced-face list of the identification instead of from psi.
//
// The ring of node (i, j, k) in a grid plane (its eight in-plane neighbours,
// counter-clockwise about the plane normal) encloses exactly the four
// plaquettes of that plane that have the node as a corner.  Every interior
// edge of those plaquettes is run once in each direction and cancels, so the
// ring's integer circulation S is the sum of the four plaquette windings W
// (each edge term being the same integer branch crossing in both forms):
//   S_xy(i,j,k) = sum of W_xy over the xy faces with min corner (i-1|i, j-1|j, k)
//   S_yz(i,j,k) = sum of W_yz over the yz faces with min corner (i, j-1|j, k-1|k)
//   S_zx(i,j,k) = sum of W_zx over the zx faces with min corner (i-1|i, j, k-1|k)
// Faces with W = 0 are absent from the list and add nothing.  So the vortex
// nodes follow from the 1e-2 faces per node of the face list, not from
// another pass over psi: per node row (j, k) one warp adds the windings of
// the faces in the four face rows (j-1|j, k-1|k) into a shared-memory row of
// packed per-plane sums (only the columns a face reached are read and
// reset), and stages the row's nodes with a non-zero S in ascending x in a
// block of a staging buffer; a scan over the rows' counts and a scatter that
// copies each row's block to its place give the list in ascending node
// order, as the psi form (node_form.cu) gives it.
//
// Exactness.  The identification reports W mod 4 (winding 2 for W = +-2, a
// face whose four edges are exact +-pi ties), so a face of winding 2 makes the
// sums unknown: such a face sets *tie and the outputs are not to be used.
// Rings through non-finite nodes count 0 in the psi form, while the
// identification drops the faces touching such a node: the field must be
// finite (qtv_stats.nonfinite == 0 for the identification that made the
// list).  Rings that leave the grid count 0, as in the psi form.
#include <cstdio>

#include "qtv_internal.cuh"

namespace qtv {

struct NodeFacesWork {
  uint32_t* rows = nullptr;              // face-row table: R + 1 entries
  uint32_t* rowcnt = nullptr;            // vortex nodes per node row
  unsigned long long* rowoff = nullptr;  // exclusive prefix within a scan block
  unsigned long long* boff = nullptr;    // scan-block offsets
  unsigned long long* rowbase = nullptr;  // first staging entry of each row
  unsigned long long* stage = nullptr;   // staged vortex nodes
  unsigned long long* flags = nullptr;   // staging top
  uint64_t cap = 0;                      // rows provided for
  uint64_t bcap = 0;                     // scan blocks provided for
  uint64_t scap = 0;                     // staging entries provided for
};

void node_faces_work_free(NodeFacesWork* w) {
  if (!w) return;
  cudaFree(w->rows);
  cudaFree(w->rowcnt);
  cudaFree(w->rowoff);
  cudaFree(w->boff);
  cudaFree(w->rowbase);
  cudaFree(w->stage);
  cudaFree(w->flags);
  delete w;
}

namespace {

constexpr int kNfWarps = 8;            // warps (node rows in flight) per CTA
constexpr int kScanThreads = 1024;
constexpr int kScanPer = 4;            // rows per scan thread
constexpr long long kScanRows = (long long)kScanThreads * kScanPer;
constexpr uint32_t kBias = 0x00080808u;  // S + 8 in bytes 0 (xy), 1 (yz), 2 (zx)
constexpr unsigned FULL = 0xffffffffu;
constexpr uint32_t kStageChunk = 1024;  // staging entries a warp reserves at a time

struct NfArgs {
  const uint64_t* ids;
  const int8_t* w;
  unsigned long long n;
  const uint64_t* n_dev;
  int nx, ny, nz;
  long long R;  // node rows: ny * nz
  const uint32_t* rows;
  uint32_t* rowcnt;
  unsigned long long* rowbase;  // first staging entry of a row
  unsigned long long* stage;    // staged vortex nodes: x << 32 | (S + 8) bytes
  unsigned long long stage_cap;
  unsigned long long* top;      // staging bump counter
  const unsigned long long* rowoff;
  const unsigned long long* boff;
  uint64_t* node_ids;
  int8_t* circ;
  unsigned long long capacity;
  unsigned int* tie;
};

// Vortex nodes per node row, staged in the row's block of the staging buffer
// (and the tie flag); node_faces_scatter then puts them in order.
// A warp's shared memory holds the packed sums of one node row (nx words,
// S + 8 in three bytes) and a bit mask of the columns that received a face
// (nx / 32 words): only those are read, listed and reset, so a row costs its
// faces, not its nx nodes.
__global__ void __launch_bounds__(kNfWarps * 32, 8) node_faces_kernel(const __grid_constant__ NfArgs a) {
  extern __shared__ uint32_t nf_acc[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int nwords = (nx + 31) >> 5;
  const int wstride = nx + nwords + (nx + 1) / 2;  // words per warp
  uint32_t* acc = nf_acc + (size_t)wib * (size_t)wstride;
  uint32_t* touched = acc + nx;
  uint16_t* cols = reinterpret_cast<uint16_t*>(touched + nwords);  // touched columns of a row
  unsigned long long chunk_at = 0;  // this warp's staging block (lane 0)
  uint32_t chunk_left = 0;
  for (int i = lane; i < nx; i += 32) acc[i] = kBias;
  for (int i = lane; i < nwords; i += 32) touched[i] = 0u;
  __syncwarp();
  const long long warps = (long long)gridDim.x * kNfWarps;
  for (long long r = (long long)blockIdx.x * kNfWarps + wib; r < a.R; r += warps) {
    const int k = (int)((uint32_t)r / (uint32_t)ny), j = (int)r - k * ny;  // R < 2^31
    // face rows q = (j + dj, k + dk), dj = (q & 1) - 1, dk = (q >> 1) - 1:
    // xy faces of plane k, yz faces of all four, zx faces of row j.  Their
    // bounds come from six row-table entries read at once (lanes 0-5), and
    // the lanes stride over the four rows' faces as one range, so a row's
    // loads are in flight together.
    uint32_t rv = 0;
    if (lane < 6) {
      const int kk = lane < 3 ? k - 1 : k, jj = j - 1 + lane % 3;
      if (kk >= 0 && jj >= 0) rv = __ldg(a.rows + (long long)kk * ny + jj);
    }
    uint32_t lo[4], c[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int b0 = (q >> 1) * 3 + (q & 1);  // lane holding the row's first index
      const uint32_t l = __shfl_sync(FULL, rv, b0), h = __shfl_sync(FULL, rv, b0 + 1);
      const bool ok = j + (q & 1) - 1 >= 0 && k + (q >> 1) - 1 >= 0;
      lo[q] = l;
      c[q] = ok ? h - l : 0u;
    }
    const uint32_t total = c[0] + c[1] + c[2] + c[3];
    for (uint32_t t = (uint32_t)lane; t < total; t += 32) {
      int q = 0;
      uint32_t u = t;
      if (u >= c[0]) { u -= c[0]; q = 1;
        if (u >= c[1]) { u -= c[1]; q = 2;
          if (u >= c[2]) { u -= c[2]; q = 3; } } }
      const uint32_t f = (q == 0 ? lo[0] : q == 1 ? lo[1] : q == 2 ? lo[2] : lo[3]) + u;
      const int dj = (q & 1) - 1, dk = (q >> 1) - 1;
      const uint64_t id = __ldg(a.ids + f);
      const int o = (int)(id & 3u);
      const bool use = (o == 0 && dk == 0) || o == 1 || (o == 2 && dj == 0);
      if (!use) continue;
      const int wv = (int)a.w[f];
      if (wv != 1 && wv != -1) {
        atomicOr(a.tie, 1u);
        continue;
      }
      const unsigned long long rowbase =
          ((unsigned long long)(k + dk) * (unsigned long long)ny + (unsigned long long)(j + dj)) *
          (unsigned long long)nx;
      const int i = (int)((id >> 2) - rowbase);
      const uint32_t d = wv > 0 ? (1u << (8 * o)) : (0u - (1u << (8 * o)));
      atomicAdd(acc + i, d);
      atomicOr(touched + (i >> 5), 1u << (i & 31));
      if (o != 1 && i + 1 < nx) {
        atomicAdd(acc + i + 1, d);
        atomicOr(touched + ((i + 1) >> 5), 1u << ((i + 1) & 31));
      }
    }
    __syncwarp();
    // The touched columns, compacted in ascending order into the warp's column
    // list (lane l owns mask word l of each group of 32), then read one column
    // per lane: S of the three planes (rings leaving the grid count 0), the
    // vortex nodes ranked by a ballot, staged, and every column reset.
    const bool jin = j >= 1 && j <= ny - 2, kin = k >= 1 && k <= nz - 2;
    uint32_t ntouched = 0;
    for (int w0 = 0; w0 < nwords; w0 += 32) {
      const int wi = w0 + lane;
      uint32_t bits = 0;
      if (wi < nwords) {
        bits = touched[wi];
        touched[wi] = 0u;
      }
      const uint32_t pc = (uint32_t)__popc(bits);
      uint32_t incl = pc;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t u = __shfl_up_sync(FULL, incl, d);
        if (lane >= d) incl += u;
      }
      uint32_t pos = ntouched + incl - pc;
      for (uint32_t b = bits; b; b &= b - 1u) cols[pos++] = (uint16_t)(32 * wi + __ffs(b) - 1);
      ntouched += __shfl_sync(FULL, incl, 31);
    }
    __syncwarp();
    auto col_s = [&](uint32_t t, int& i, uint32_t& packed) -> bool {
      i = cols[t];
      const uint32_t v = acc[i];
      acc[i] = kBias;
      const bool iin = i >= 1 && i <= nx - 2;
      const int s0 = (iin && jin) ? (int)(v & 0xFFu) - 8 : 0;
      const int s1 = (jin && kin) ? (int)((v >> 8) & 0xFFu) - 8 : 0;
      const int s2 = (kin && iin) ? (int)((v >> 16) & 0xFFu) - 8 : 0;
      packed = (uint32_t)((s0 + 8) | ((s1 + 8) << 8) | ((s2 + 8) << 16));
      return (s0 | s1 | s2) != 0;
    };
    // the first 32 columns are read once and held; the row's total is known
    // before its staging block is reserved
    int i0 = 0;
    uint32_t p0 = 0;
    const bool v0 = (uint32_t)lane < ntouched && col_s((uint32_t)lane, i0, p0);
    const uint32_t bal0 = __ballot_sync(FULL, v0);
    uint32_t cnt = (uint32_t)__popc(bal0);
    for (uint32_t t0 = 32; t0 < ntouched; t0 += 32) {  // wide rows: count only
      const uint32_t t = t0 + (uint32_t)lane;
      bool v = false;
      if (t < ntouched) {
        const int ii = cols[t];
        const uint32_t vv = acc[ii];
        const bool iin = ii >= 1 && ii <= nx - 2;
        v = ((iin && jin) && (vv & 0xFFu) != 8u) || ((jin && kin) && ((vv >> 8) & 0xFFu) != 8u) ||
            ((kin && iin) && ((vv >> 16) & 0xFFu) != 8u);
      }
      cnt += (uint32_t)__popc(__ballot_sync(FULL, v));
    }
    unsigned long long off = 0;
    bool store = false;
    if (cnt) {
      unsigned long long base = 0;
      if (lane == 0) {
        if (cnt > kStageChunk) {
          base = atomicAdd(a.top, (unsigned long long)cnt);
        } else {
          if (cnt > chunk_left) {
            chunk_at = atomicAdd(a.top, (unsigned long long)kStageChunk);
            chunk_left = kStageChunk;
          }
          base = chunk_at;
          chunk_at += cnt;
          chunk_left -= cnt;
        }
        // the buffer holds four nodes per face plus every warp's part-used
        // block, so this cannot fail; if it did, nothing is written past it
        if (base + cnt > a.stage_cap) atomicOr(a.tie, 2u);
        a.rowbase[r] = base;
      }
      off = __shfl_sync(FULL, base, 0);
      store = off + cnt <= a.stage_cap;
    }
    if (lane == 0) a.rowcnt[r] = cnt;
    if (store && v0)
      a.stage[off + (unsigned)__popc(bal0 & ((1u << lane) - 1u))] =
          ((unsigned long long)(unsigned)i0 << 32) | p0;
    off += (unsigned)__popc(bal0);
    for (uint32_t t0 = 32; t0 < ntouched; t0 += 32) {
      const uint32_t t = t0 + (uint32_t)lane;
      int ii = 0;
      uint32_t pp = 0;
      const bool v = t < ntouched && col_s(t, ii, pp);
      const uint32_t bal = __ballot_sync(FULL, v);
      if (store && v)
        a.stage[off + (unsigned)__popc(bal & ((1u << lane) - 1u))] =
            ((unsigned long long)(unsigned)ii << 32) | pp;
      off += (unsigned)__popc(bal);
    }
    __syncwarp();  // the row is reset before the next one adds into it
  }
}

// The staged rows at their places in the ascending list.  A warp takes 32
// consecutive node rows (lane = row for their counts, staging blocks and
// offsets); their outputs are one contiguous range, which the lanes fill in
// order, each finding the row of its entry among the 32 by a binary search
// over the rows' exclusive counts.
__global__ void __launch_bounds__(256) node_faces_scatter(const __grid_constant__ NfArgs a) {
  const int lane = threadIdx.x & 31;
  const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long r0 = 32 * (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5); r0 < a.R;
       r0 += 32 * warps) {
    const long long r = r0 + lane;
    uint32_t cnt = 0;
    unsigned long long base = 0;
    if (r < a.R) {
      cnt = a.rowcnt[r];
      if (cnt) base = a.rowbase[r];
    }
    uint32_t incl = cnt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t u = __shfl_up_sync(FULL, incl, d);
      if (lane >= d) incl += u;
    }
    const uint32_t total = __shfl_sync(FULL, incl, 31);
    if (total == 0) continue;
    const uint32_t excl = incl - cnt;
    // the first output of row r0 (the rows' outputs follow it contiguously)
    const unsigned long long dst0 = a.boff[r0 / kScanRows] + a.rowoff[r0];
    for (uint32_t e0 = 0; e0 < total; e0 += 32) {  // uniform trip count: shuffles below
      const uint32_t e = e0 + (uint32_t)lane;
      int m = 0;  // the last row whose exclusive count is <= e
#pragma unroll
      for (int stp = 16; stp >= 1; stp >>= 1) {
        const uint32_t xv = __shfl_sync(FULL, excl, (m + stp) & 31);
        if (m + stp < 32 && xv <= e) m += stp;
      }
      const uint32_t em = __shfl_sync(FULL, excl, m);
      const unsigned long long bm = __shfl_sync(FULL, base, m);
      const unsigned long long dst = dst0 + e;
      if (e >= total || dst >= a.capacity) continue;
      const unsigned long long v = a.stage[bm + (e - em)];
      a.node_ids[dst] = (unsigned long long)(r0 + m) * (unsigned long long)a.nx + (v >> 32);
      a.circ[3 * dst] = (int8_t)((int)(v & 0xFFu) - 8);
      a.circ[3 * dst + 1] = (int8_t)((int)((v >> 8) & 0xFFu) - 8);
      a.circ[3 * dst + 2] = (int8_t)((int)((v >> 16) & 0xFFu) - 8);
    }
  }
}

// exclusive prefix of the row counts within blocks of kScanRows rows, and
// each block's total
__global__ void __launch_bounds__(kScanThreads) nf_scan_rows(const uint32_t* __restrict__ cnt,
                                                             long long R,
                                                             unsigned long long* __restrict__ rowoff,
                                                             unsigned long long* __restrict__ btot) {
  __shared__ unsigned long long wsum[kScanThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const long long r0 = (long long)blockIdx.x * kScanRows + (long long)tid * kScanPer;
  uint32_t c[kScanPer];
  unsigned long long local = 0;
#pragma unroll
  for (int q = 0; q < kScanPer; ++q) {
    c[q] = r0 + q < R ? cnt[r0 + q] : 0u;
    local += c[q];
  }
  unsigned long long incl = local;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const unsigned long long u = __shfl_up_sync(FULL, incl, d);
    if (lane >= d) incl += u;
  }
  if (lane == 31) wsum[w] = incl;
  __syncthreads();
  if (w == 0) {
    const unsigned long long v = wsum[lane];
    unsigned long long iv = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned long long u = __shfl_up_sync(FULL, iv, d);
      if (lane >= d) iv += u;
    }
    wsum[lane] = iv - v;
    if (lane == 31) btot[blockIdx.x] = iv;
  }
  __syncthreads();
  unsigned long long run = wsum[w] + incl - local;
#pragma unroll
  for (int q = 0; q < kScanPer; ++q) {
    if (r0 + q < R) rowoff[r0 + q] = run;
    run += c[q];
  }
}

// block totals -> exclusive block offsets, in place; the total into *count
__global__ void __launch_bounds__(kScanThreads) nf_scan_blocks(unsigned long long* __restrict__ b,
                                                               long long nb, uint64_t* count) {
  __shared__ unsigned long long wsum[kScanThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const long long per = (nb + kScanThreads - 1) / kScanThreads;
  const long long s0 = tid * per, s1 = s0 + per < nb ? s0 + per : nb;
  unsigned long long local = 0;
  for (long long s = s0; s < s1; ++s) local += b[s];
  unsigned long long incl = local;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const unsigned long long u = __shfl_up_sync(FULL, incl, d);
    if (lane >= d) incl += u;
  }
  if (lane == 31) wsum[w] = incl;
  __syncthreads();
  if (w == 0) {
    const unsigned long long v = wsum[lane];
    unsigned long long iv = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned long long u = __shfl_up_sync(FULL, iv, d);
      if (lane >= d) iv += u;
    }
    wsum[lane] = iv - v;
    if (lane == 31) *count = iv;
  }
  __syncthreads();
  unsigned long long run = wsum[w] + incl - local;
  for (long long s = s0; s < s1; ++s) {
    const unsigned long long t = b[s];
    b[s] = run;
    run += t;
  }
}

bool capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  return cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
}

}  // namespace
}  // namespace qtv

using namespace qtv;

QTV_API int qtv_node_circulation_faces(qtv_handle h, const qtv_grid* grid, const uint64_t* face_ids,
                                       const int8_t* winding, uint64_t n, const uint64_t* n_dev,
                                       uint64_t* node_ids, int8_t* circ, uint64_t capacity,
                                       uint64_t* count, uint32_t* tie, void* stream) {
  if (!h || !grid) return set_error(QTV_ERR_ARG, "handle or grid is NULL");
  if (!count || !tie) return set_error(QTV_ERR_ARG, "count and tie are required");
  if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1)
    return set_error(QTV_ERR_ARG, "grid %d x %d x %d", grid->nx, grid->ny, grid->nz);
  if (n > 0 && (!face_ids || !winding)) return set_error(QTV_ERR_ARG, "face list is NULL");
  if (capacity > 0 && (!node_ids || !circ)) return set_error(QTV_ERR_ARG, "output lists are NULL");
  if (n >= (1ull << 32)) return set_error(QTV_ERR_ARG, "more than 2^32 - 1 faces");
  const int nx = grid->nx, ny = grid->ny, nz = grid->nz;
  const size_t smem =
      (size_t)kNfWarps * (size_t)(nx + (nx + 31) / 32 + (nx + 1) / 2) * sizeof(uint32_t);
  if (smem > 200 * 1024)
    return set_error(QTV_ERR_ARG, "rows of %d nodes are too wide for the face-derived node form", nx);
  const long long R = (long long)ny * nz;
  if (R >= (1ll << 31)) return set_error(QTV_ERR_ARG, "ny * nz of 2^31 or more node rows");
  const long long nb = (R + kScanRows - 1) / kScanRows;
  long long blocks = (R + kNfWarps - 1) / kNfWarps;
  const long long maxb = (long long)h->num_sms * 8;
  if (blocks > maxb) blocks = maxb;
  // staging: at most four vortex nodes per face (a face is on four rings),
  // plus the part-used block of every warp
  const uint64_t scap = 4 * n + (uint64_t)blocks * kNfWarps * kStageChunk;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  NodeFacesWork* w = h->nodef;
  if (!w || w->cap < (uint64_t)R || w->bcap < (uint64_t)nb || w->scap < scap) {
    if (capturing(st)) return set_error(QTV_ERR_STATE, "workspace must grow outside stream capture");
    if (!w) w = h->nodef = new NodeFacesWork();
    const uint64_t ncap = w->cap > (uint64_t)R ? w->cap : (uint64_t)R;
    const uint64_t nbcap = w->bcap > (uint64_t)nb ? w->bcap : (uint64_t)nb;
    const uint64_t nscap = w->scap > scap ? w->scap : scap;
    cudaFree(w->rows);
    cudaFree(w->rowcnt);
    cudaFree(w->rowoff);
    cudaFree(w->boff);
    cudaFree(w->rowbase);
    cudaFree(w->stage);
    cudaFree(w->flags);
    w->rows = w->rowcnt = nullptr;
    w->rowoff = w->boff = w->rowbase = w->stage = w->flags = nullptr;
    w->cap = w->bcap = w->scap = 0;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&w->rows), (ncap + 1) * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&w->rowcnt), ncap * sizeof(uint32_t));
    if (e == cudaSuccess)
      e = cudaMalloc(reinterpret_cast<void**>(&w->rowoff), ncap * sizeof(unsigned long long));
    if (e == cudaSuccess)
      e = cudaMalloc(reinterpret_cast<void**>(&w->rowbase), ncap * sizeof(unsigned long long));
    if (e == cudaSuccess)
      e = cudaMalloc(reinterpret_cast<void**>(&w->boff), (nbcap + 1) * sizeof(unsigned long long));
    if (e == cudaSuccess)
      e = cudaMalloc(reinterpret_cast<void**>(&w->stage), nscap * sizeof(unsigned long long));
    if (e == cudaSuccess)
      e = cudaMalloc(reinterpret_cast<void**>(&w->flags), sizeof(unsigned long long));
    if (e != cudaSuccess) return check_cuda(e, "cudaMalloc(node-form-from-faces workspace)");
    w->cap = ncap;
    w->bcap = nbcap;
    w->scap = nscap;
  }
  static bool attr = false;
  if (!attr) {
    const cudaError_t e0 = cudaFuncSetAttribute(node_faces_kernel,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                200 * 1024);
    if (e0 != cudaSuccess) return check_cuda(e0, "cudaFuncSetAttribute(node_faces)");
    // all of the unified L1 / shared memory as shared memory: eight CTAs of
    // 8 warps fit on an SM for rows up to 1000 nodes
    const cudaError_t e1 = cudaFuncSetAttribute(node_faces_kernel,
                                                cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e1 != cudaSuccess) return check_cuda(e1, "cudaFuncSetAttribute(node_faces carveout)");
    attr = true;
  }
  TraceScope ts(h, K_NODE_FACES, st);
  cudaError_t e = cudaMemsetAsync(tie, 0, sizeof(uint32_t), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(w->flags, 0, sizeof(unsigned long long), st);
  if (e == cudaSuccess)
    e = row_table_launch(face_ids, n, n_dev, nx, R, 2, w->rows, h->num_sms, st);
  if (e != cudaSuccess) return check_cuda(e, "node form from faces: row table");
  NfArgs a;
  a.ids = face_ids;
  a.w = winding;
  a.n = n;
  a.n_dev = n_dev;
  a.nx = nx;
  a.ny = ny;
  a.nz = nz;
  a.R = R;
  a.rows = w->rows;
  a.rowcnt = w->rowcnt;
  a.rowbase = w->rowbase;
  a.stage = w->stage;
  a.stage_cap = w->scap;
  a.top = w->flags;
  a.rowoff = w->rowoff;
  a.boff = w->boff;
  a.node_ids = node_ids;
  a.circ = circ;
  a.capacity = capacity;
  a.tie = tie;
  node_faces_kernel<<<(int)blocks, kNfWarps * 32, smem, st>>>(a);
  nf_scan_rows<<<(int)nb, kScanThreads, 0, st>>>(w->rowcnt, R, w->rowoff, w->boff);
  nf_scan_blocks<<<1, kScanThreads, 0, st>>>(w->boff, nb, count);
  if (capacity > 0) {
    long long sblocks = (R + 255) / 256;  // 32 rows per warp
    if (sblocks > (long long)h->num_sms * 16) sblocks = (long long)h->num_sms * 16;
    node_faces_scatter<<<(int)sblocks, 256, 0, st>>>(a);
  }
  return check_cuda(cudaGetLastError(), "node form from faces");
}
