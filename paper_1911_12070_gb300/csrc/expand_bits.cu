// expand_bits.cu -- expand pass of the bit-sliced identification sweep
// (Sec. 2.2.2, Eq. 5): the per-lane records of sweep_bits.cu become the face
// list in ascending face-id order, at the offsets of the segment scan.
#include "bits_layout.cuh"
#include "qtv_internal.cuh"
#include "sweep_common.cuh"

namespace qtv {
namespace {

using namespace sweep;
using namespace bits;

// ---------------------------------------------------------------------------
// Expand: one warp per (snapshot, plane, band) segment writes its faces in
// ascending face-id order: row by row, within a row by x (tile, warp, lane
// order of the records), within a node by orientation.  A band row has up to
// kBitsBandWarps (tile, warp) steps (nx up to 2048 and more); lane l holds
// the table entries l E .. l E + E - 1, E = ceil(steps / 32).
// ---------------------------------------------------------------------------
constexpr int kExpandWarps = 8;
constexpr int kHeld = 3;  // record chunks (of 32) a warp keeps in registers
constexpr int kMaxE = (kBitsBandWarps + 31) / 32;  // table entries per lane
static_assert(kMaxE == 3, "the entry selection below handles three entries per lane");

// bits 4q..4q+3 of m spread to the low bit of bytes 0..3
__device__ __forceinline__ uint32_t spread4(uint32_t m, int q) {
  return (((m >> (4 * q)) & 0xFu) * 0x00204081u) & 0x01010101u;
}

// MAXE: table entries a lane may hold (1 when every band row has at most 32
// (tile, warp) steps, the common case, compiled without the wider selection)
template <int MAXE>
__global__ void __launch_bounds__(32 * kExpandWarps, kBitsExpandCtasPerSm) expand_bits_kernel(
    const __grid_constant__ BulkParams a, const unsigned long long* __restrict__ seg_off,
    uint64_t* __restrict__ face_ids, int8_t* __restrict__ winding, unsigned long long capacity,
    uint64_t* __restrict__ offsets) {
  __shared__ uint32_t s_rowbase[kExpandWarps][BR / 2];  // running offsets within rows
  __shared__ uint32_t s_base[kExpandWarps][BR];          // first face of each row
  pdl_wait();  // segment offsets and counts of the scan
  pdl_trigger();
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const uint2* __restrict__ table = reinterpret_cast<const uint2*>(a.table);
  const uint4* __restrict__ recs = reinterpret_cast<const uint4*>(a.recs);
  const unsigned long long recs_cap = a.recs_cap;
  const long long nseg = a.nseg;
  if (offsets && blockIdx.x == 0 && threadIdx.x < (unsigned)a.nsnap)
    offsets[threadIdx.x] = a.s[threadIdx.x].seg0 < nseg ? seg_off[a.s[threadIdx.x].seg0] : 0ull;
  if (capacity == 0) return;
  const long long nwarps = (long long)gridDim.x * kExpandWarps;
  auto locate = [&](long long sg, int& si, long long& local, int& NWs) {
    si = 0;
    while (si + 1 < a.nsnap && a.s[si + 1].seg0 <= sg) ++si;
    local = sg - a.s[si].seg0;
    NWs = a.s[si].ntx * a.s[si].nwt;
  };
  for (long long s = (long long)blockIdx.x * kExpandWarps + wib; s < nseg; s += nwarps) {
    int si, NW;
    long long local;
    locate(s, si, local, NW);
    const SnapDesc& sd = a.s[si];
    const int nbands = sd.nbands;
    const long long k = local / nbands;
    const long long band = local % nbands;
    // entry of (tile, warp) step i: ((band ntx + tile) nwt + warp) nz + k =
    // ebase + i nz; lane l holds steps l E + j (their record lane masks)
    const int E = MAXE == 1 ? 1 : (NW + 31) >> 5;
    const int NL = (NW + E - 1) / E;  // lanes holding steps
    const unsigned long long nzl = (unsigned long long)sd.nz;
    const unsigned long long ebase =
        (unsigned long long)sd.tab0 + (unsigned long long)band * (unsigned long long)NW * nzl +
        (unsigned long long)k;
    uint32_t em[MAXE];
#pragma unroll
    for (int j = 0; j < MAXE; ++j) {
      const int i = lane * E + j;
      em[j] = (j < E && i < NW) ? table[ebase + (unsigned long long)i * nzl].x : 0u;
    }
    const unsigned long long fbase = seg_off[s];  // loaded alongside the entries
    uint32_t n = 0;
#pragma unroll
    for (int j = 0; j < MAXE; ++j) n += __popc(em[j]);
    uint32_t incl = n;
#pragma unroll
    for (int dd = 1; dd < 32; dd <<= 1) {
      const uint32_t x = __shfl_up_sync(0xffffffffu, incl, dd);
      if (lane >= dd) incl += x;
    }
    const uint32_t start = lane < NL ? incl - n : 0xFFFFFFFFu;
    const uint32_t rtot = __shfl_sync(0xffffffffu, incl, 31);
    if (rtot == 0) continue;
    const unsigned long long nx = (unsigned)sd.nx, ny = (unsigned)sd.ny;
    const long long j0 = band * BR;
    const int nwt = sd.nwt;
    const uint32_t nchunks = (rtot + 31) / 32;

    // record of flattened index g = g0 + lane (zero past the end); ww = its
    // (tile, warp) step: the lane holding the step (the last lane whose first
    // record is at or before g), then the step among that lane's E
    auto load = [&](uint32_t g0, uint4& rec, int& ww) {
      const uint32_t g = g0 + lane;
      int lo = 0;
#pragma unroll
      for (int stp = 16; stp >= 1; stp >>= 1) {
        const int cand = lo + stp;
        const uint32_t sv = __shfl_sync(0xffffffffu, start, cand & 31);
        if (cand < NL && sv <= g) lo = cand;
      }
      uint32_t qi = g - __shfl_sync(0xffffffffu, start, lo);
      uint32_t mask = __shfl_sync(0xffffffffu, em[0], lo);
      int j = 0;
      if constexpr (MAXE > 1) if (E > 1) {  // warp-uniform
        const uint32_t m1 = __shfl_sync(0xffffffffu, em[1 % MAXE], lo);
        const uint32_t m2 = __shfl_sync(0xffffffffu, em[2 % MAXE], lo);
        const uint32_t c0 = __popc(mask), c1 = __popc(m1);
        if (qi >= c0) {
          qi -= c0;
          j = 1;
          mask = m1;
          if (qi >= c1) {
            qi -= c1;
            j = 2;
            mask = m2;
          }
        }
      }
      ww = lo * E + j;
      rec = make_uint4(0u, 0u, 0u, 0u);
      if (g < rtot) {
        const unsigned long long idx = (ebase + (unsigned long long)ww * nzl) * 32ull +
                                       (unsigned)(__fns(mask, 0, (int)qi + 1));
        if (idx < recs_cap) rec = recs[idx];
      }
    };
    // per-row face counts of a record, 4 rows per word (one byte each)
    auto counts = [&](const uint4& rec, uint32_t* cw) {
      const uint32_t mx = (rec.x | (rec.x >> 16)) & kRows16;
      const uint32_t my = (rec.y | (rec.y >> 16)) & kRows16;
      const uint32_t mz = (rec.z | (rec.z >> 16)) & kRows16;
#pragma unroll
      for (int q = 0; q < 4; ++q) cw[q] = spread4(mx, q) + spread4(my, q) + spread4(mz, q);
    };
    auto scan4 = [&](const uint32_t* cw, uint32_t* ex, uint32_t* tot) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        uint32_t v = cw[q];
#pragma unroll
        for (int dd = 1; dd < 32; dd <<= 1) {
          const uint32_t x = __shfl_up_sync(0xffffffffu, v, dd);
          if (lane >= dd) v += x;
        }
        ex[q] = v - cw[q];
        tot[q] = __shfl_sync(0xffffffffu, v, 31);
      }
    };

    // Faces per row (pass 1), then the running offset of each row within it
    // (pass 2), as 16-bit halves: row r in word 2 (r >> 2) + (r & 1), half
    // (r >> 1) & 1 (the layout of the byte counts' even and odd bytes).  A row
    // holds at most 3 nx faces, below 2^16.  With at most 32 (tile, warp)
    // steps a row (nx <= 992) a whole segment holds fewer than 3 x 16 x 992 <
    // 2^16 faces and the halves carry the running row bases themselves;
    // otherwise the rows' first faces are kept as 32-bit words in s_base.
    uint32_t racc[BR / 2];
#pragma unroll
    for (int q = 0; q < BR / 2; ++q) racc[q] = 0;
    auto add_tot = [&](const uint32_t* tot) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        racc[2 * q] += tot[q] & 0x00FF00FFu;
        racc[2 * q + 1] += (tot[q] >> 8) & 0x00FF00FFu;
      }
    };
    // pass 1: faces per row over the segment's records (byte sums over the
    // lanes: at most 3 x 32 per byte, no carry between bytes)
    auto tally = [&](const uint4& rec) {
      uint32_t cw[4], tot[4];
      counts(rec, cw);
#pragma unroll
      for (int q = 0; q < 4; ++q) tot[q] = __reduce_add_sync(0xffffffffu, cw[q]);
      add_tot(tot);
    };
    const unsigned long long lin0 = ((unsigned long long)k * ny + (unsigned long long)j0) * nx;
    // pass 2: the faces of a chunk of records at their row-major positions
    auto emit = [&](const uint4& rec, int ww) {
      uint32_t cw[4], ex[4], tot[4];
      counts(rec, cw);
      scan4(cw, ex, tot);
      const uint32_t mx = (rec.x | (rec.x >> 16)) & kRows16;
      const uint32_t my = (rec.y | (rec.y >> 16)) & kRows16;
      const uint32_t mz = (rec.z | (rec.z >> 16)) & kRows16;
      const uint32_t rows = mx | my | mz;
      if (rows) {
#pragma unroll
        for (int q = 0; q < BR / 2; ++q) s_rowbase[wib][q] = racc[q];
        // column of the record: tile ww / nwt at tile * st, warp ww % nwt of
        // the tile at 31 columns each, lane in the record
        const unsigned tile = (unsigned)ww / (unsigned)nwt;
        const uint32_t x = tile * (unsigned)sd.st + (uint32_t)BL * ((unsigned)ww - tile * (unsigned)nwt) +
                           (rec.w & 31u);
        uint32_t rm = rows;
        while (rm) {
          const int r = __ffs(rm) - 1;
          rm &= rm - 1u;
          const int q = r >> 2;
          const uint32_t exq = q == 0 ? ex[0] : (q == 1 ? ex[1] : (q == 2 ? ex[2] : ex[3]));
          uint32_t rb = (s_rowbase[wib][2 * q + (r & 1)] >> (16 * ((r >> 1) & 1))) & 0xFFFFu;
          if constexpr (MAXE > 1) rb += s_base[wib][r];
          unsigned long long pos = fbase + rb + ((exq >> (8 * (r & 3))) & 0xFFu);
          const unsigned long long lin = lin0 + (unsigned long long)((uint32_t)r * (uint32_t)nx + x);
          const uint32_t Ls[3] = {rec.x, rec.y, rec.z};
#pragma unroll
          for (int o = 0; o < 3; ++o) {
            const uint32_t L = (Ls[o] >> r) & 1u, H = (Ls[o] >> (16 + r)) & 1u;
            if (L | H) {
              if (pos < capacity) {
                face_ids[pos] = (lin << 2) | (unsigned)o;
                winding[pos] = (int8_t)(L ? (H ? -1 : 1) : 2);
              }
              ++pos;
            }
          }
        }
      }
      add_tot(tot);
    };
    // row totals -> each row's first face: 32-bit words shared with the lanes
    // (the running offsets within rows then start at zero), or for narrow
    // rows the 16-bit halves themselves
    auto bases = [&]() {
      uint32_t acc = 0;
      if constexpr (MAXE > 1) {
#pragma unroll
        for (int r = 0; r < BR; ++r) {
          const int wi = 2 * (r >> 2) + (r & 1), sh = 16 * ((r >> 1) & 1);
          if (lane == r) s_base[wib][r] = acc;
          acc += (racc[wi] >> sh) & 0xFFFFu;
        }
#pragma unroll
        for (int q = 0; q < BR / 2; ++q) racc[q] = 0;
        __syncwarp();
      } else {
        uint32_t out[BR / 2];
#pragma unroll
        for (int q = 0; q < BR / 2; ++q) out[q] = 0;
#pragma unroll
        for (int r = 0; r < BR; ++r) {
          const int wi = 2 * (r >> 2) + (r & 1), sh = 16 * ((r >> 1) & 1);
          out[wi] |= acc << sh;
          acc += (racc[wi] >> sh) & 0xFFFFu;
        }
#pragma unroll
        for (int q = 0; q < BR / 2; ++q) racc[q] = out[q];
      }
    };

    if (nchunks <= (uint32_t)kHeld) {
      // the usual case: every record load of the segment in flight at once,
      // the records held in registers for both passes
      uint4 hrec[kHeld];
      int hww[kHeld];
#pragma unroll
      for (int c = 0; c < kHeld; ++c)
        if ((uint32_t)c < nchunks) load(c * 32, hrec[c], hww[c]);
#pragma unroll
      for (int c = 0; c < kHeld; ++c)
        if ((uint32_t)c < nchunks) tally(hrec[c]);
      bases();
#pragma unroll
      for (int c = 0; c < kHeld; ++c)
        if ((uint32_t)c < nchunks) emit(hrec[c], hww[c]);
    } else {
      for (uint32_t c = 0; c < nchunks; ++c) {
        uint4 rec;
        int ww;
        load(c * 32, rec, ww);
        tally(rec);
      }
      bases();
      for (uint32_t c = 0; c < nchunks; ++c) {
        uint4 rec;
        int ww;
        load(c * 32, rec, ww);
        emit(rec, ww);
      }
    }
  }
}

}  // namespace

cudaError_t bits_expand_launch(const BulkParams& p, int blocks, const unsigned long long* seg_off,
                               uint64_t* face_ids, int8_t* winding, unsigned long long capacity,
                               uint64_t* offsets, cudaStream_t st) {
  bool wide = false;
  for (int i = 0; i < p.nsnap; ++i) wide |= p.s[i].ntx * p.s[i].nwt > 32;
  if (wide)
    return launch_dependent(expand_bits_kernel<kMaxE>, dim3(blocks), dim3(32 * kExpandWarps), 0,
                            st, p, seg_off, face_ids, winding, capacity, offsets);
  return launch_dependent(expand_bits_kernel<1>, dim3(blocks), dim3(32 * kExpandWarps), 0, st, p,
                          seg_off, face_ids, winding, capacity, offsets);
}

}  // namespace qtv
