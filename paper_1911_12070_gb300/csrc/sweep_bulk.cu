// sweep_bulk.cu -- identification sweep (Sec. 2.2.2, Eq. 5) with psi planes
// staged in shared memory by the bulk-copy engine, per-warp compaction of the
// pierced plaquettes, and a finalize pass that puts them in face-id order.
//
// Decomposition.  A CTA owns a band of 7 rows (+1 halo row) across the whole
// x extent and marches z; thread (w, l) owns columns x0 = 64 w + 2 l, x0 + 1.
// The edge values of each (edge direction, column) are packed one 4-bit field
// per row (value + 1), so the four-term plaquette sums of all rows of a column
// take three integer instructions.
//
// Staging.  Each plane's band rows are copied into one slot of a 3-deep ring
// in shared memory with cp.async.bulk (one copy per row, issued by lane 0 of
// the warp that owns the row index modulo the warp count; completion counted
// in bytes on the slot's mbarrier, which every warp arrives on once per fill).
// Threads read their 16-byte pairs and the x-neighbour column from shared
// memory.  Waits are bounded (about 2^32 SM cycles); a timeout sets a status
// bit that turns the reported count into QTV_COUNT_TIMEOUT.
//
// Edge test.  Phases follow the IEEE atan2 convention theta in [-pi, pi]
// with the sign of a zero imaginary part deciding +pi or -pi, so a node is in
// the lower half-plane (s = 1) iff the sign bit of Im psi is set.  The
// branch-crossing integer of edge a -> b is r = s_b - s_a when the edge
// crosses the branch cut (arg = +-pi) and 0 otherwise; with s_a != s_b this
// happens iff the sign bit of cross(a, b) = Re a Im b - Im a Re b is clear
// (s_a = 0) or set (s_a = 1).  The FP32 FMA evaluation
// fma(Re a, Im b, -RN(Im a Re b)) gives that sign bit exactly in every case
// that matters: when Re a and Re b have equal signs the two terms cannot
// cancel (and signed-zero results follow IEEE rules that match the atan2
// convention), and when they differ |d| > pi/2, so a wrong sign needs
// |sin d| < 2^-24, an edge within 1e-7 rad of +-pi (an ambiguous edge).
// Sign bits are gathered four bits per row with one funnel shift each.  A
// node with psi == 0 has no phase; it is read as phase 0, which makes every
// edge that touches it contribute 0.  Warps whose planes hold a zero or a
// non-finite node (detected by a product of |Re| + |Im|) take a path that
// masks those edges and drops the faces that touch non-finite nodes.
//
// Compaction.  Each warp, each plane, emits one 24-byte record per lane that
// has a pierced face: the six packed (W+4)^4 fields of its two columns and
// three orientations (rows 0..6) plus the lane index.  Record positions come
// from one warp ballot; records go to per-warp chunks of a staging buffer
// reserved with one global atomic per chunk (prefetched), and a 16-byte table
// entry per (plane, band, warp) says where they are and how many faces they
// hold.  A finalize pass scans the face totals in (plane, band) order (single
// pass, decoupled look-back) and expands the records of each segment row by
// row, in (warp, lane) order, which is ascending face-id order.
//
// Schedule.  Work units are (plane, band) pairs ordered (z block, band, plane)
// and cut into one contiguous range per CTA, so all CTAs get the same number
// of planes, and CTAs that hold neighbouring bands march the same z block at
// the same time (the halo row of a band is the first row of the next one and
// is then served by L2).
#include <algorithm>

#include "qtv_internal.cuh"
#include "sweep_common.cuh"

namespace qtv {
namespace {

using namespace sweep;

constexpr int R = kRows;
constexpr int RH = R + 1;
constexpr int kStages = 3;
constexpr uint32_t kOnes = 0x11111111u;
constexpr uint32_t kFours = 0x44444444u;
constexpr uint32_t kOwnedBits = 0x01111111u;  // bit 0 of the fields of rows 0..6
constexpr uint32_t kBit3 = 0x88888888u;
constexpr int kRecWords = 6;                   // 32-bit words per staged record

__device__ __forceinline__ uint32_t nz_fields(uint32_t d) {
  uint32_t t = d | (d >> 2);
  t = t | (t >> 1);
  return t & kOnes;
}

// acc' = (acc << 4) | top nibble of x: the sign bit of x lands in bit 3 of a
// new lowest field.  Push rows from the highest to the lowest.
__device__ __forceinline__ uint32_t push_sign(uint32_t acc, float x) {
  return __funnelshift_l(__float_as_uint(x), acc, 4);
}
// keep bit 3 of each field and move it to bit 0
__device__ __forceinline__ uint32_t fields_of(uint32_t acc) { return (acc & kBit3) >> 3; }

// sign bits of Im psi of one column over the RH rows (bit 0 of field r)
__device__ __forceinline__ uint32_t sbits_col(const float4* v, int p) {
  uint32_t acc = 0;
#pragma unroll
  for (int r = RH - 1; r >= 0; --r) acc = push_sign(acc, p ? v[r].w : v[r].y);
  return fields_of(acc);
}
__device__ __forceinline__ uint32_t sbits_nb(const float2* v) {
  uint32_t acc = 0;
#pragma unroll
  for (int r = RH - 1; r >= 0; --r) acc = push_sign(acc, v[r].y);
  return fields_of(acc);
}
// psi == 0 (both parts +-0) bits of a column
__device__ __forceinline__ uint32_t zbits_col(const float4* v, int p) {
  uint32_t z = 0;
#pragma unroll
  for (int r = 0; r < RH; ++r) {
    const uint32_t b = (__float_as_uint(p ? v[r].z : v[r].x) | __float_as_uint(p ? v[r].w : v[r].y)) << 1;
    if (b == 0u) z |= 1u << (4 * r);
  }
  return z;
}
__device__ __forceinline__ uint32_t zbits_nb(const float2* v) {
  uint32_t z = 0;
#pragma unroll
  for (int r = 0; r < RH; ++r)
    if (((__float_as_uint(v[r].x) | __float_as_uint(v[r].y)) << 1) == 0u) z |= 1u << (4 * r);
  return z;
}

// packed edge values (value + 1 per field) from tail/head s-bits, the
// cross-negative bits N and the edges E that touch a zero node
__device__ __forceinline__ uint32_t pack_edges(uint32_t SA, uint32_t SB, uint32_t N, uint32_t E) {
  return kOnes + (~SA & SB & ~N & ~E) - (SA & ~SB & N & ~E);
}

struct SmallSmem {
  uint2 xbits[2][kMaxWarpsX];  // {rz_k, ry_k+1} fields of column x0 of each warp
};

constexpr uint32_t kChunk = 32;     // records per staging chunk
constexpr uint32_t kLowWater = 12;  // prefetch the next chunk below this

// Edge fields of one step.  In: plane k (C, s-bits Sk0/Sk1, zero bits Zk*) and
// plane k+1 (N, neighbour column nbv).  ZERO masks edges at zero nodes.
template <bool ZERO>
__device__ __forceinline__ void step_edges(const float4* C, const float4* N, const float2* nbv,
                                           uint32_t Sk0, uint32_t Sk1, uint32_t Zk0,
                                           uint32_t Zk1, uint32_t& S0n, uint32_t& S1n,
                                           uint32_t& Z0n, uint32_t& Z1n, uint32_t& RZ0,
                                           uint32_t& RZ1, uint32_t& RX0n, uint32_t& RX1n,
                                           uint32_t& RY0n, uint32_t& RY1n) {
  S0n = sbits_col(N, 0);
  S1n = sbits_col(N, 1);
  const uint32_t SNn = sbits_nb(nbv);
  uint32_t az0 = 0, az1 = 0, ax0 = 0, ax1 = 0, ay0 = 0, ay1 = 0;
#pragma unroll
  for (int r = RH - 1; r >= 0; --r) {
    az0 = push_sign(az0, cross_f(C[r].x, C[r].y, N[r].x, N[r].y));
    az1 = push_sign(az1, cross_f(C[r].z, C[r].w, N[r].z, N[r].w));
    ax0 = push_sign(ax0, cross_f(N[r].x, N[r].y, N[r].z, N[r].w));
    ax1 = push_sign(ax1, cross_f(N[r].z, N[r].w, nbv[r].x, nbv[r].y));
    if (r < R) {
      ay0 = push_sign(ay0, cross_f(N[r].x, N[r].y, N[r + 1].x, N[r + 1].y));
      ay1 = push_sign(ay1, cross_f(N[r].z, N[r].w, N[r + 1].z, N[r + 1].w));
    }
  }
  uint32_t Ez0 = 0, Ez1 = 0, Ex0 = 0, Ex1 = 0, Ey0 = 0, Ey1 = 0;
  Z0n = 0;
  Z1n = 0;
  if (ZERO) {
    Z0n = zbits_col(N, 0);
    Z1n = zbits_col(N, 1);
    const uint32_t ZN = zbits_nb(nbv);
    Ez0 = Zk0 | Z0n;
    Ez1 = Zk1 | Z1n;
    Ex0 = Z0n | Z1n;
    Ex1 = Z1n | ZN;
    Ey0 = Z0n | (Z0n >> 4);
    Ey1 = Z1n | (Z1n >> 4);
  }
  RZ0 = pack_edges(Sk0, S0n, fields_of(az0), Ez0);
  RZ1 = pack_edges(Sk1, S1n, fields_of(az1), Ez1);
  RX0n = pack_edges(S0n, S1n, fields_of(ax0), Ex0);
  RX1n = pack_edges(S1n, SNn, fields_of(ax1), Ex1);
  RY0n = pack_edges(S0n & kOwnedBits, S0n >> 4, fields_of(ay0), Ey0);
  RY1n = pack_edges(S1n & kOwnedBits, S1n >> 4, fields_of(ay1), Ey1);
}

// non-finite bits of a column (one bit per field)
__device__ __forceinline__ uint32_t badbits_col(const float4* v, int p) {
  uint32_t b = 0;
#pragma unroll
  for (int r = 0; r < RH; ++r) {
    const float re = p ? v[r].z : v[r].x, im = p ? v[r].w : v[r].y;
    if (!(finite_f(re) && finite_f(im))) b |= 1u << (4 * r);
  }
  return b;
}
__device__ __forceinline__ uint32_t badbits_nb(const float2* v) {
  uint32_t b = 0;
#pragma unroll
  for (int r = 0; r < RH; ++r)
    if (!(finite_f(v[r].x) && finite_f(v[r].y))) b |= 1u << (4 * r);
  return b;
}

// product of |Re| + |Im| over the 3 columns of one plane: 0 when a node is
// zero, non-finite when a node is; also 0 / infinite on FP32 under- and
// overflow, which merely selects the masking path
__device__ __forceinline__ bool plane_special(const float4* v, const float2* nbv) {
  float prod = 1.f;
#pragma unroll
  for (int r = 0; r < RH; ++r)
    prod *= (fabsf(v[r].x) + fabsf(v[r].y)) * (fabsf(v[r].z) + fabsf(v[r].w)) *
            (fabsf(nbv[r].x) + fabsf(nbv[r].y));
  return !(prod > 0.f && prod <= 3.402823466e38f);
}

template <int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB) sweep_bulk_kernel(const __grid_constant__ BulkParams a) {
  extern __shared__ __align__(128) unsigned char dsm[];
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int w = tid >> 5;
  const int NW = blockDim.x >> 5;
  const int W = NW * 64;  // row pitch of a ring slot (the tile width), in elements
  float2* ring = reinterpret_cast<float2*>(dsm);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(dsm + (size_t)kStages * RH * W * sizeof(float2));
  SmallSmem& sm = *reinterpret_cast<SmallSmem*>(mbar + kStages);
  const int x0 = 64 * w + 2 * lane;  // tile-local column of this lane's pair
  const bool nbin = x0 + 2 < W;
  const uint32_t lt = (1u << lane) - 1u;

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&mbar[s], (uint32_t)NW);
    fence_mbar_init();
  }
  __syncthreads();

  uint32_t fill = 0, use = 0;  // planes issued / consumed by this CTA (uniform)
  bool timeout = false;
  // per-warp record chunk (uniform within the warp)
  uint32_t cb = 0, cl = 0, nb_l0 = 0;
  bool have_next = false;
  bool overflow = false;
  // columns [valid_w, W) of every row and rows [valid_r, RH) of every column
  // of every ring slot hold the padding value 1 (finite and nonzero, so that
  // padding never selects the masking path; faces that touch it are masked)
  int valid_w = W, valid_r = RH;

  const long long U = a.units;
  long long u = U * blockIdx.x / gridDim.x;
  const long long uend = U * (blockIdx.x + 1) / gridDim.x;

  while (u < uend) {
    int si = 0;
    while (si + 1 < a.nsnap && a.s[si + 1].unit0 <= u) ++si;
    const SnapDesc& sd = a.s[si];
    const int nx = sd.nx, ny = sd.ny, nz = sd.nz, ntx = sd.ntx;
    long long col;
    int kb, kblk;
    unit_pos(u - sd.unit0, (long long)sd.nbands * ntx, nz, sd.hblock, col, kb, kblk);
    const int band = (int)(col / ntx), tile = (int)(col % ntx);
    const int ke = (int)min((long long)kblk, (long long)kb + (uend - u));
    u += ke - kb;
    const int j0 = band * R;
    const int nrows = min(RH, ny - j0);
    const int klast = min(ke, nz - 1);
    const int nplanes = klast - kb + 1;
    const int nsteps = ke - kb;
    // tile: staged columns [xt0, xt0 + tw); this CTA owns the faces of the
    // lanes with x0 < own_end (the last pair of a non-final tile only feeds
    // its left neighbour and is owned by the next tile)
    const int xt0 = tile * sd.st;
    const bool last_tile = tile == ntx - 1;
    const int tw = last_tile ? nx - xt0 : sd.st + 2;
    const int own_end = last_tile ? tw : sd.st;
    const uint32_t row_bytes = (uint32_t)tw * 8u;
    const size_t plane = (size_t)nx * ny;

    if (tw < valid_w || nrows < valid_r) {
      const int cw = valid_w - tw;
      if (cw > 0)
        for (int idx = tid; idx < kStages * RH * cw; idx += blockDim.x)
          ring[(size_t)(idx / cw) * W + tw + idx % cw] = make_float2(1.f, 0.f);
      const int rr = valid_r - nrows;
      if (rr > 0) {
        const int per = rr * W;
        for (int idx = tid; idx < kStages * per; idx += blockDim.x) {
          const int sl = idx / per, rem = idx % per;
          ring[((size_t)sl * RH + nrows + rem / W) * W + rem % W] = make_float2(1.f, 0.f);
        }
      }
      fence_proxy_async();  // later bulk copies may land in rows written here
      __syncthreads();
    }
    valid_w = tw;
    valid_r = nrows;

    // every warp arrives once per fill, lane 0 copying the rows r == w (mod NW)
    auto issue = [&](int m) {
      if (lane == 0) {
        const int sl = fill % kStages;
        uint64_t* bar = &mbar[sl];
        float2* dst = ring + (size_t)sl * RH * W;
        const float2* src = sd.psi + (size_t)m * plane + (size_t)j0 * nx + xt0;
        uint32_t mine = 0;
        for (int r = w; r < nrows; r += NW) ++mine;
        fence_proxy_async();
        mbar_arrive_expect_tx(bar, row_bytes * mine);
        for (int r = w; r < nrows; r += NW)
          bulk_g2s(dst + (size_t)r * W, src + (size_t)r * nx, row_bytes, bar);
      }
      ++fill;
    };
    auto acquire = [&]() -> const float2* {
      const int sl = use % kStages;
      if (!mbar_wait(&mbar[sl], (use / kStages) & 1u)) timeout = true;
      ++use;
      return ring + (size_t)sl * RH * W;
    };

    // row validity and slot existence (bit 0 of each field)
    uint32_t rowv = 0, rowv1 = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (j0 + r < ny) rowv |= 1u << (4 * r);
      if (j0 + r + 1 < ny) rowv1 |= 1u << (4 * r);
    }
    const bool own = x0 < own_end;
    const bool c0 = own && x0 < tw, c1 = own && x0 + 1 < tw, c2 = own && x0 + 2 < tw;
    const uint32_t ex_xy0 = c1 ? rowv1 : 0u, ex_xy1 = c2 ? rowv1 : 0u;
    const uint32_t ex_yz0 = c0 ? rowv1 : 0u, ex_yz1 = c1 ? rowv1 : 0u;
    const uint32_t ex_zx0 = c1 ? rowv : 0u, ex_zx1 = c2 ? rowv : 0u;
    // table entry of (plane k, band, tile, warp w) = tbase + k * tstride
    const unsigned long long tstride = (unsigned long long)sd.nbands * ntx * NW;
    const unsigned long long tbase =
        (unsigned long long)sd.tab0 + ((unsigned long long)band * ntx + tile) * NW + w;
    unsigned int* const segf = a.segf + sd.seg0 + band;
    const unsigned sstride = (unsigned)sd.nbands;

    // ---- prologue: plane kb
    for (int i = 0; i < min(kStages, nplanes); ++i) issue(kb + i);
    float4 bufA[RH], bufB[RH];
    uint32_t Sk0, Sk1, Zk0 = 0, Zk1 = 0, RX0, RX1, RY0, RY1, RYN;
    bool bad_k;
    uint32_t Bk0 = 0, Bk1 = 0, BkN = 0;  // non-finite bits of plane k (masking path only)
    {
      const float2* sp = acquire();
      float2 nbv[RH];
#pragma unroll
      for (int r = 0; r < RH; ++r) {
        bufA[r] = *reinterpret_cast<const float4*>(sp + (size_t)r * W + x0);
        nbv[r] = nbin ? sp[(size_t)r * W + x0 + 2] : make_float2(1.f, 0.f);
      }
      bad_k = __any_sync(0xffffffffu, plane_special(bufA, nbv));
      Sk0 = sbits_col(bufA, 0);
      Sk1 = sbits_col(bufA, 1);
      const uint32_t SN = sbits_nb(nbv);
      uint32_t ax0 = 0, ax1 = 0, ay0 = 0, ay1 = 0, ayn = 0;
#pragma unroll
      for (int r = RH - 1; r >= 0; --r) {
        ax0 = push_sign(ax0, cross_f(bufA[r].x, bufA[r].y, bufA[r].z, bufA[r].w));
        ax1 = push_sign(ax1, cross_f(bufA[r].z, bufA[r].w, nbv[r].x, nbv[r].y));
        if (r < R) {
          ay0 = push_sign(ay0, cross_f(bufA[r].x, bufA[r].y, bufA[r + 1].x, bufA[r + 1].y));
          ay1 = push_sign(ay1, cross_f(bufA[r].z, bufA[r].w, bufA[r + 1].z, bufA[r + 1].w));
          ayn = push_sign(ayn, cross_f(nbv[r].x, nbv[r].y, nbv[r + 1].x, nbv[r + 1].y));
        }
      }
      uint32_t ZN = 0;
      if (bad_k) {
        Zk0 = zbits_col(bufA, 0);
        Zk1 = zbits_col(bufA, 1);
        ZN = zbits_nb(nbv);
        Bk0 = badbits_col(bufA, 0);
        Bk1 = badbits_col(bufA, 1);
        BkN = badbits_nb(nbv);
      }
      RX0 = pack_edges(Sk0, Sk1, fields_of(ax0), Zk0 | Zk1);
      RX1 = pack_edges(Sk1, SN, fields_of(ax1), Zk1 | ZN);
      RY0 = pack_edges(Sk0 & kOwnedBits, Sk0 >> 4, fields_of(ay0), Zk0 | (Zk0 >> 4));
      RY1 = pack_edges(Sk1 & kOwnedBits, Sk1 >> 4, fields_of(ay1), Zk1 | (Zk1 >> 4));
      RYN = pack_edges(SN & kOwnedBits, SN >> 4, fields_of(ayn), ZN | (ZN >> 4));
    }
    __syncthreads();  // slot of plane kb fully read
    if (kb + kStages <= klast) issue(kb + kStages);

    // one z step: plane k = kb + t in C, plane k + 1 loaded into Nn
    auto step = [&](float4(&C)[RH], float4(&Nn)[RH], int t) {
      const int k = kb + t;
      const bool has_up = k + 1 < nz;
      uint32_t S0n = 0, S1n = 0, Z0n = 0, Z1n = 0, RZ0 = kOnes, RZ1 = kOnes, RX0n = kOnes,
               RX1n = kOnes, RY0n = kOnes, RY1n = kOnes;
      uint32_t Bn0 = 0, Bn1 = 0, BnN = 0;
      bool bad_k1 = false;
      if (has_up) {
        const float2* sp = acquire();
        float2 nbv[RH];
#pragma unroll
        for (int r = 0; r < RH; ++r) {
          Nn[r] = *reinterpret_cast<const float4*>(sp + (size_t)r * W + x0);
          nbv[r] = nbin ? sp[(size_t)r * W + x0 + 2] : make_float2(1.f, 0.f);
        }
        bad_k1 = __any_sync(0xffffffffu, plane_special(Nn, nbv));
        if (bad_k || bad_k1) {
          step_edges<true>(C, Nn, nbv, Sk0, Sk1, Zk0, Zk1, S0n, S1n, Z0n, Z1n, RZ0, RZ1, RX0n,
                           RX1n, RY0n, RY1n);
          Bn0 = badbits_col(Nn, 0);
          Bn1 = badbits_col(Nn, 1);
          BnN = badbits_nb(nbv);
        } else {
          step_edges<false>(C, Nn, nbv, Sk0, Sk1, 0u, 0u, S0n, S1n, Z0n, Z1n, RZ0, RZ1, RX0n,
                            RX1n, RY0n, RY1n);
        }
      }
      if (lane == 0) sm.xbits[t & 1][w] = make_uint2(RZ0, RY0n);
      __syncthreads();
      if (has_up && k + 1 + kStages <= klast) issue(k + 1 + kStages);

      // neighbour-column fields from lane + 1 (lane 31: from warp w + 1)
      uint32_t RZN = __shfl_down_sync(0xffffffffu, RZ0, 1);
      uint32_t RYNn = __shfl_down_sync(0xffffffffu, RY0n, 1);
      if (lane == 31) {
        if (w + 1 < NW) {
          const uint2 xb = sm.xbits[t & 1][w + 1];
          RZN = xb.x;
          RYNn = xb.y;
        } else {
          RZN = kOnes;
          RYNn = kOnes;
        }
      }
      // plaquette windings, (W + 4) per field
      uint32_t d[6];
      d[0] = RX0 + RY1 + kFours - (RX0 >> 4) - RY0;    // xy, x0
      d[1] = RY0 + (RZ0 >> 4) + kFours - RY0n - RZ0;   // yz, x0
      d[2] = RZ0 + RX0n + kFours - RZ1 - RX0;          // zx, x0
      d[3] = RX1 + RYN + kFours - (RX1 >> 4) - RY1;    // xy, x0 + 1
      d[4] = RY1 + (RZ1 >> 4) + kFours - RY1n - RZ1;   // yz, x0 + 1
      d[5] = RZ1 + RX1n + kFours - RZN - RX1;          // zx, x0 + 1
      uint32_t keep[6] = {ex_xy0 * 0xFu, has_up ? ex_yz0 * 0xFu : 0u, has_up ? ex_zx0 * 0xFu : 0u,
                          ex_xy1 * 0xFu, has_up ? ex_yz1 * 0xFu : 0u, has_up ? ex_zx1 * 0xFu : 0u};
      if (bad_k || bad_k1) {
        const uint32_t bxy0 = Bk0 | Bk1 | (Bk0 >> 4) | (Bk1 >> 4);
        const uint32_t bxy1 = Bk1 | BkN | (Bk1 >> 4) | (BkN >> 4);
        const uint32_t byz0 = Bk0 | (Bk0 >> 4) | Bn0 | (Bn0 >> 4);
        const uint32_t byz1 = Bk1 | (Bk1 >> 4) | Bn1 | (Bn1 >> 4);
        const uint32_t bzx0 = Bk0 | Bk1 | Bn0 | Bn1;
        const uint32_t bzx1 = Bk1 | BkN | Bn1 | BnN;
        const uint32_t bb[6] = {bxy0, byz0, bzx0, bxy1, byz1, bzx1};
#pragma unroll
        for (int q = 0; q < 6; ++q) keep[q] &= ~((bb[q] & kOnes) * 0xFu);
      }
      uint32_t cnt = 0, anyw = 0;
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        d[q] = (d[q] ^ kFours) & keep[q];
        cnt += nz_fields(d[q]);
        anyw |= d[q];
      }
      // ---- per-warp compaction: one record per lane with faces
      const uint32_t bsum = (cnt & 0x0F0F0F0Fu) + ((cnt >> 4) & 0x0F0F0F0Fu);
      const uint32_t faces_w = __reduce_add_sync(0xffffffffu, (bsum * 0x01010101u) >> 24);
      const uint32_t bal = __ballot_sync(0xffffffffu, anyw != 0u);
      const uint32_t T = __popc(bal);
      uint32_t base1 = cb, base2 = 0, n1 = T;
      if (T > cl) {
        const uint32_t need = T - cl;
        uint32_t nbase, ncap;
        if (have_next && need <= kChunk) {
          nbase = __shfl_sync(0xffffffffu, nb_l0, 0);
          ncap = kChunk;
          have_next = false;
        } else {
          ncap = need > kChunk ? need : kChunk;
          uint32_t x = 0;
          if (lane == 0) {
            const unsigned long long got = atomicAdd(a.counters, (unsigned long long)ncap);
            x = (uint32_t)got;
            if (got + ncap > a.recs_cap) overflow = true;
          }
          nbase = __shfl_sync(0xffffffffu, x, 0);
        }
        n1 = cl;
        base2 = nbase;
        cb = nbase + need;
        cl = ncap - need;
      } else {
        cb += T;
        cl -= T;
      }
      if (cl < kLowWater && !have_next) {
        if (lane == 0) {
          const unsigned long long got = atomicAdd(a.counters, (unsigned long long)kChunk);
          nb_l0 = (uint32_t)got;
          if (got + kChunk > a.recs_cap) overflow = true;
        }
        have_next = true;
      }
      if (lane == 0) {
        a.table[tbase + (unsigned long long)k * tstride] =
            make_uint4(base1, base2, T | (n1 << 6) | (faces_w << 12), 0u);
        if (faces_w) atomicAdd(&segf[(size_t)k * sstride], faces_w);
      }
      if (anyw) {
        const uint32_t q = __popc(bal & lt);
        const unsigned long long idx =
            q < n1 ? (unsigned long long)base1 + q : (unsigned long long)base2 + (q - n1);
        if (idx < a.recs_cap) {
          uint2* p = reinterpret_cast<uint2*>(a.recs + idx * kRecWords);
          p[0] = make_uint2(d[0] | ((uint32_t)lane << 28), d[1] | ((uint32_t)(lane >> 4) << 28));
          p[1] = make_uint2(d[2], d[3]);
          p[2] = make_uint2(d[4], d[5]);
        }
      }
      // plane k + 1 becomes plane k
      Sk0 = S0n;
      Sk1 = S1n;
      Zk0 = Z0n;
      Zk1 = Z1n;
      RX0 = RX0n;
      RX1 = RX1n;
      RY0 = RY0n;
      RY1 = RY1n;
      RYN = RYNn;
      bad_k = bad_k1;
      Bk0 = Bn0;
      Bk1 = Bn1;
      BkN = BnN;
    };

    for (int t = 0; t < nsteps; t += 2) {
      step(bufA, bufB, t);
      if (t + 1 < nsteps) step(bufB, bufA, t + 1);
    }
    __syncthreads();
  }
  if (timeout) atomicOr(reinterpret_cast<unsigned int*>(a.counters + 1), 1u);
  if (overflow) atomicOr(reinterpret_cast<unsigned int*>(a.counters + 1), 2u);
}

// ---------------------------------------------------------------------------
// Finalize 1: exclusive scan of the per-segment face totals in (snapshot,
// plane, band) order, single pass with decoupled look-back over tiles taken by
// ticket.
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr long long kScanTile = (long long)kScanThreads * kScanItems;
constexpr unsigned long long kFlagA = 1ull << 62, kFlagP = 2ull << 62;
constexpr unsigned long long kValMask = (1ull << 62) - 1;

__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.volatile.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__global__ void __launch_bounds__(kScanThreads) v3_scan_kernel(
    const unsigned int* __restrict__ segf, long long nseg, unsigned long long* __restrict__ seg_off,
    uint64_t* count, unsigned long long* counters, unsigned long long* tiles, long long ntiles,
    qtv_stats* stats, unsigned long long scanned, long long hold_tile, long long spin_limit) {
  __shared__ unsigned long long s_warp[kScanThreads / 32];
  __shared__ unsigned long long s_prefix;
  __shared__ long long s_tile;
  pdl_wait();  // segment totals of the sweeps
  pdl_trigger();
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) s_tile = (long long)atomicAdd(counters + 2, 1ull);
  __syncthreads();
  const long long tile = s_tile;
  const long long s0 = tile * kScanTile + (long long)tid * kScanItems;
  uint32_t v[kScanItems];
  unsigned long long local = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const long long s = s0 + i;
    const uint32_t f = s < nseg ? __ldg(&segf[s]) : 0u;
    v[i] = f;
    local += f;
  }
  unsigned long long incl = local;
#pragma unroll
  for (int dd = 1; dd < 32; dd <<= 1) {
    const unsigned long long x = __shfl_up_sync(0xffffffffu, incl, dd);
    if (lane >= dd) incl += x;
  }
  if (lane == 31) s_warp[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    const unsigned long long x = lane < kScanThreads / 32 ? s_warp[lane] : 0ull;
    unsigned long long ix = x;
#pragma unroll
    for (int dd = 1; dd < 32; dd <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, ix, dd);
      if (lane >= dd) ix += y;
    }
    if (lane < kScanThreads / 32) s_warp[lane] = ix - x;
    if (lane == 31) {
      // ix: tile aggregate
      const unsigned long long agg = ix;
      unsigned long long prefix = 0;
      // a held tile (failure injection) never publishes, so a later tile's
      // look-back wait on it runs out
      const bool publish = tile != hold_tile;
      if (tile == 0) {
        if (publish) atomicExch(&tiles[0], kFlagP | agg);
      } else {
        if (publish) atomicExch(&tiles[tile], kFlagA | agg);
        long long p = tile - 1;
        while (p >= 0) {
          unsigned long long st = ld_volatile_u64(&tiles[p]);
          if ((st >> 62) == 0) {
            const long long t0 = clock64();
            while ((st >> 62) == 0) {
              st = ld_volatile_u64(&tiles[p]);
              if (clock64() - t0 > spin_limit) break;
            }
            if ((st >> 62) == 0) {
              atomicOr(reinterpret_cast<unsigned int*>(counters + 1), 4u);
              break;
            }
          }
          prefix += st & kValMask;
          if ((st >> 62) == 2) break;
          --p;
        }
        if (publish) atomicExch(&tiles[tile], kFlagP | (prefix + agg));
      }
      s_prefix = prefix;
      if (tile == ntiles - 1) {
        const unsigned long long status = ld_volatile_u64(counters + 1);
        *count = (status & 5ull) ? QTV_COUNT_TIMEOUT : prefix + agg;
        if (stats) {
          stats->pierced = prefix + agg;
          stats->faces_scanned = scanned;
        }
      }
    }
  }
  __syncthreads();
  unsigned long long run = s_prefix + s_warp[wid] + incl - local;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const long long s = s0 + i;
    if (s < nseg) seg_off[s] = run;
    run += v[i];
  }
}

// ---------------------------------------------------------------------------
// Finalize 2: one warp per (snapshot, plane, band) segment expands its
// records into face ids and windings at their final offsets: row by row, and
// within a row in flattened record order (tile, warp, lane), which is
// ascending x.
// ---------------------------------------------------------------------------
constexpr int kExpandWarps = 8;

// fields 0..6 of the packed count of pierced faces per row in a record
__device__ __forceinline__ uint32_t rec_row_counts(const uint32_t* dw) {
  uint32_t c = 0;
#pragma unroll
  for (int sl = 0; sl < kRecWords; ++sl) c += nz_fields(dw[sl] & 0x0FFFFFFFu);
  return c;
}

__global__ void __launch_bounds__(32 * kExpandWarps, 4) v3_expand_kernel(
    const __grid_constant__ BulkParams a, const unsigned long long* __restrict__ seg_off,
    uint64_t* __restrict__ face_ids, int8_t* __restrict__ winding, unsigned long long capacity,
    uint64_t* __restrict__ offsets) {
  __shared__ uint32_t s_rowbase[kExpandWarps][R];
  pdl_wait();  // segment offsets and counts of the scan
  pdl_trigger();
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const uint4* __restrict__ table = a.table;
  const uint32_t* __restrict__ recs = a.recs;
  const unsigned long long recs_cap = a.recs_cap;
  const long long nseg = a.nseg;
  if (offsets && blockIdx.x == 0 && threadIdx.x < (unsigned)a.nsnap)
    offsets[threadIdx.x] = a.s[threadIdx.x].seg0 < nseg ? seg_off[a.s[threadIdx.x].seg0] : 0ull;
  if (capacity == 0) return;
  const long long nwarps = (long long)gridDim.x * kExpandWarps;
  long long s = (long long)blockIdx.x * kExpandWarps + wib;
  // snapshot of segment s and its per-segment table geometry
  auto locate = [&](long long sg, int& si, long long& local, int& NWs) {
    si = 0;
    while (si + 1 < a.nsnap && a.s[si + 1].seg0 <= sg) ++si;
    local = sg - a.s[si].seg0;
    NWs = a.s[si].ntx * a.s[si].nwt;
  };
  // the next segment's table entries and offset are loaded one segment ahead
  uint4 e_next = make_uint4(0u, 0u, 0u, 0u);
  unsigned long long fb_next = 0;
  if (s < nseg) {
    int si, NWs;
    long long local;
    locate(s, si, local, NWs);
    if (lane < NWs) e_next = table[a.s[si].tab0 + local * NWs + lane];
    fb_next = seg_off[s];
  }
  for (; s < nseg; s += nwarps) {
    const uint4 e = e_next;
    const unsigned long long fbase = fb_next;
    int si, NW;
    long long local;
    locate(s, si, local, NW);
    if (s + nwarps < nseg) {
      int si2, NW2;
      long long local2;
      locate(s + nwarps, si2, local2, NW2);
      if (lane < NW2) e_next = table[a.s[si2].tab0 + local2 * NW2 + lane];
      fb_next = seg_off[s + nwarps];
    }
    const uint32_t n = e.z & 63u, n1 = (e.z >> 6) & 63u;
    uint32_t incl = n;
#pragma unroll
    for (int dd = 1; dd < 32; dd <<= 1) {
      const uint32_t x = __shfl_up_sync(0xffffffffu, incl, dd);
      if (lane >= dd) incl += x;
    }
    const uint32_t start = lane < NW ? incl - n : 0xFFFFFFFFu;
    const uint32_t rtot = __shfl_sync(0xffffffffu, incl, 31);
    if (rtot == 0) continue;
    const SnapDesc& sd = a.s[si];
    const int nbands = sd.nbands;
    const unsigned long long nx = (unsigned)sd.nx, ny = (unsigned)sd.ny;
    const long long k = local / nbands;
    const long long j0 = (local % nbands) * R;
    const int nwt = sd.nwt;  // warps per tile of this snapshot
    const uint32_t nchunks = (rtot + 31) / 32;

    // record of flattened index g = g0 + lane (zeros past the end)
    auto load = [&](uint32_t g0, uint32_t* dw, int& ww) {
      const uint32_t g = g0 + lane;
      int lo = 0;
#pragma unroll
      for (int stp = 16; stp >= 1; stp >>= 1) {
        const int cand = lo + stp;
        const uint32_t sv = __shfl_sync(0xffffffffu, start, cand & 31);
        if (cand < NW && sv <= g) lo = cand;
      }
      ww = lo;
      const uint32_t qi = g - __shfl_sync(0xffffffffu, start, lo);
      const uint32_t b1 = __shfl_sync(0xffffffffu, e.x, lo);
      const uint32_t b2 = __shfl_sync(0xffffffffu, e.y, lo);
      const uint32_t m1 = __shfl_sync(0xffffffffu, n1, lo);
      const unsigned long long idx =
          qi < m1 ? (unsigned long long)b1 + qi : (unsigned long long)b2 + (qi - m1);
#pragma unroll
      for (int sl = 0; sl < kRecWords; ++sl) dw[sl] = 0u;
      if (g < rtot && idx < recs_cap) {
        const uint2* p = reinterpret_cast<const uint2*>(recs + idx * kRecWords);
        const uint2 q0 = p[0], q1 = p[1], q2 = p[2];
        dw[0] = q0.x;
        dw[1] = q0.y;
        dw[2] = q1.x;
        dw[3] = q1.y;
        dw[4] = q2.x;
        dw[5] = q2.y;
      }
    };
    // per-row exclusive counts within the chunk (bytes: even rows, odd rows)
    auto scan_rows = [&](uint32_t cnt, uint32_t& exe, uint32_t& exo, uint32_t& te, uint32_t& to) {
      const uint32_t ce = cnt & 0x0F0F0F0Fu, co = (cnt >> 4) & 0x0F0F0F0Fu;
      uint32_t ie = ce, io = co;
#pragma unroll
      for (int dd = 1; dd < 32; dd <<= 1) {
        const uint32_t xe = __shfl_up_sync(0xffffffffu, ie, dd);
        const uint32_t xo = __shfl_up_sync(0xffffffffu, io, dd);
        if (lane >= dd) {
          ie += xe;
          io += xo;
        }
      }
      exe = ie - ce;
      exo = io - co;
      te = __shfl_sync(0xffffffffu, ie, 31);
      to = __shfl_sync(0xffffffffu, io, 31);
    };
    auto field8 = [](uint32_t ev, uint32_t od, int r) -> uint32_t {
      return ((r & 1) ? (od >> (8 * (r >> 1))) : (ev >> (8 * (r >> 1)))) & 0xFFu;
    };

    // pass 1 (several chunks only): per-row totals of the segment
    uint32_t rowtot[R];
#pragma unroll
    for (int r = 0; r < R; ++r) rowtot[r] = 0;
    uint32_t dw[kRecWords];
    int ww = 0;
    uint32_t cnt = 0, exe = 0, exo = 0, te = 0, to = 0;
    if (nchunks == 1) {
      load(0, dw, ww);
      cnt = rec_row_counts(dw);
      scan_rows(cnt, exe, exo, te, to);
#pragma unroll
      for (int r = 0; r < R; ++r) rowtot[r] = field8(te, to, r);
    } else {
      for (uint32_t c = 0; c < nchunks; ++c) {
        uint32_t tdw[kRecWords];
        int tww;
        load(c * 32, tdw, tww);
        uint32_t a0, a1, t0, t1;
        scan_rows(rec_row_counts(tdw), a0, a1, t0, t1);
#pragma unroll
        for (int r = 0; r < R; ++r) rowtot[r] += field8(t0, t1, r);
      }
    }
    uint32_t rowbase[R];
    {
      uint32_t acc = 0;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        rowbase[r] = acc;
        acc += rowtot[r];
      }
    }
    // pass 2: write
    for (uint32_t c = 0; c < nchunks; ++c) {
      if (nchunks > 1) {
        load(c * 32, dw, ww);
        cnt = rec_row_counts(dw);
        scan_rows(cnt, exe, exo, te, to);
      }
      // write this lane's faces: rows with faces, then slots with faces
      if (cnt) {
        const uint32_t rl = (dw[0] >> 28) | ((dw[1] >> 28) << 4);
#pragma unroll
        for (int r = 0; r < R; ++r) s_rowbase[wib][r] = rowbase[r];
        // first column of warp ww: tile ww / nwt at x = tile * st, warp
        // ww % nwt of the tile at 64 columns each
        const unsigned tw_i = (unsigned)ww / (unsigned)nwt;
        const unsigned long long xw =
            (unsigned long long)tw_i * (unsigned)sd.st + 64u * ((unsigned)ww - tw_i * (unsigned)nwt);
        uint32_t rm = nz_fields((dw[0] | dw[1]) & 0x0FFFFFFFu | dw[2] | dw[3] | dw[4] | dw[5]);
        while (rm) {
          const int f = __ffs(rm) - 1;
          const int r = f >> 2;
          rm &= rm - 1u;
          uint32_t rn = 0;
#pragma unroll
          for (int sl = 0; sl < 6; ++sl) rn |= ((dw[sl] >> f) & 0xFu) << (4 * sl);
          unsigned long long pos = fbase + s_rowbase[wib][r] + field8(exe, exo, r);
          const unsigned long long lin0 =
              ((unsigned long long)k * ny + (unsigned long long)(j0 + r)) * nx + xw + 2u * rl;
          uint32_t nzm = nz_fields(rn);
          while (nzm) {
            const int g = __ffs(nzm) - 1;
            nzm &= nzm - 1u;
            const int sl = g >> 2;
            const uint32_t nib = (rn >> g) & 0xFu;
            if (pos < capacity) {
              face_ids[pos] = ((lin0 + (unsigned long long)(sl >= 3)) << 2) | (unsigned)(sl % 3);
              winding[pos] = (int8_t)((int)(nib ^ 4u) - 4);
            }
            ++pos;
          }
        }
      }
#pragma unroll
      for (int r = 0; r < R; ++r) rowbase[r] += field8(te, to, r);
    }
  }
}

using BulkFn = void (*)(BulkParams);

BulkFn bulk_fn(int nw) {
  if (nw <= 2) return sweep_bulk_kernel<64, 8>;
  if (nw <= 4) return sweep_bulk_kernel<128, 4>;
  if (nw <= 8) return sweep_bulk_kernel<256, 2>;
  return sweep_bulk_kernel<512, 1>;
}

int bulk_fn_index(int nw) { return nw <= 2 ? 0 : (nw <= 4 ? 1 : (nw <= 8 ? 2 : 3)); }

size_t bulk_smem_for_warps(int nw) {
  return (size_t)kStages * RH * nw * 64 * sizeof(float2) + kStages * sizeof(uint64_t) +
         sizeof(SmallSmem);
}

// x tiles of a row of nx columns for tiles of nwt warps: one tile when it
// fits, else ntx tiles at an even stride st, each staging st + 2 <= 64 nwt
// columns (the last one the rest)
int snap_tiles(int nx, int nwt, int* ntx, int* st) {
  const int TX = 64 * nwt;
  if (nx <= TX) {
    *ntx = 1;
    *st = 0;
    return QTV_OK;
  }
  if (TX < 4) return set_error(QTV_ERR_ARG, "tile of %d columns too narrow", TX);
  const int n = (nx - 2 + (TX - 2) - 1) / (TX - 2);
  const int per = (nx - 2 + n - 1) / n;
  const int s = (per + 1) & ~1;
  if (s + 2 > TX || nx - (n - 1) * s > TX || nx - (n - 1) * s < 2)
    return set_error(QTV_ERR_ARG, "no tiling of nx = %d into %d-column tiles", nx, TX);
  *ntx = n;
  *st = s;
  return QTV_OK;
}

}  // namespace

// Sets the shared-memory opt-in of a sweep variant once; returns its maximum
// resident CTAs per SM.
int bulk_variant_occupancy(int nw, int* ctas_per_sm, size_t* smem) {
  static bool attr_set[4] = {false, false, false, false};
  const int which = bulk_fn_index(nw);
  BulkFn fn = bulk_fn(nw);
  if (!attr_set[which]) {
    cudaError_t e =
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e != cudaSuccess) return check_cuda(e, "cudaFuncSetAttribute(sweep_bulk)");
    attr_set[which] = true;
  }
  *smem = bulk_smem_for_warps(nw);
  int bps = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, nw * 32, *smem);
  if (e != cudaSuccess) return check_cuda(e, "occupancy(sweep_bulk)");
  if (bps < 1) return set_error(QTV_ERR_ARG, "sweep_bulk: no resident CTA with %d warps", nw);
  *ctas_per_sm = bps;
  return QTV_OK;
}

bool sweep_bulk_supported(int variant, int nx, int ny, int nz, const void* psi) {
  if (nx < 2 || ny < 1 || nz < 1 || (nx & 1)) return false;
  if (reinterpret_cast<uintptr_t>(psi) & 15u) return false;
  // bit-sliced: tiles of 31 nwt columns for any nwt, at most kBitsBandWarps
  // (tile, warp) steps per band row at nwt = 4 (tiles of 124 columns)
  if (variant == 1) return (nx + 123) / 124 * 4 <= kBitsBandWarps;
  if (nx > 1024) return false;
  return bulk_smem_for_warps((nx + 63) / 64) <= 227u * 1024u;
}

int batch_layout(int num_sms, int nsnap, const qtv_grid* grids, const float2* const* psis,
                 const TileConfig& tc, uint64_t capacity, uint64_t max_warps, BatchLayout* B) {
  if (nsnap < 1 || nsnap > kMaxSnaps)
    return set_error(QTV_ERR_ARG, "%d snapshots (1 to %d supported)", nsnap, kMaxSnaps);
  if (tc.nwt < 0 || tc.nwt > 16)
    return set_error(QTV_ERR_ARG, "tile of %d warps (1 to 16 supported)", tc.nwt);
  const bool bits = tc.variant == 1;
  if (tc.variant != 0 && tc.variant != 1)
    return set_error(QTV_ERR_ARG, "unknown sweep variant %d", tc.variant);
  if (bits && tc.nwt != 0 && tc.nwt != 2 && tc.nwt != 4 && tc.nwt != 8)
    return set_error(QTV_ERR_ARG, "bit-sliced sweep: %d warps per tile (2, 4 or 8)", tc.nwt);
  const int stages = tc.stages <= 2 ? 2 : 3;
  B->variant = tc.variant;
  B->stages = stages;
  B->rec_words = bits ? 4 : kRecWords;
  BulkParams& fin = B->fin;
  fin = BulkParams();
  fin.nsnap = nsnap;
  B->groups.clear();
  B->group_of.assign(nsnap, 0);
  long long nseg = 0, tab = 0;
  for (int i = 0; i < nsnap; ++i) {
    const qtv_grid& g = grids[i];
    if (!sweep_bulk_supported(tc.variant, g.nx, g.ny, g.nz, psis[i]))
      return set_error(QTV_ERR_ARG, "snapshot %d (%d x %d x %d): the staged sweep needs even nx "
                       "(<= 1024 for the nibble sweep) and a 16-byte aligned field", i, g.nx,
                       g.ny, g.nz);
    SnapDesc& d = fin.s[i];
    d.psi = psis[i];
    d.nx = g.nx;
    d.ny = g.ny;
    d.nz = g.nz;
    if (bits) {
      // 16-row bands; tiles of 31 nwt owned columns, each staging 2 more
      d.nbands = (g.ny + 15) / 16;
      d.nwt = tc.nwt > 0 ? tc.nwt : 4;
      d.st = 31 * d.nwt;
      d.ntx = (g.nx + d.st - 1) / d.st;
      // A last tile narrower than one warp would cost a whole CTA step per
      // plane and band for a few columns: the last tiles of nwt bands share
      // one CTA instead (one band per warp, each in its own 32-column strip
      // of the slot rows, which must fit the row pitch 31 nwt + 2).
      const int tw_last = g.nx - (d.ntx - 1) * d.st;
      d.nstk = (tw_last + 32 * (d.nwt - 1) <= 31 * d.nwt + 2) ? (d.nbands + d.nwt - 1) / d.nwt : 0;
      // warps of the last tile that own columns (a warp owns 31)
    } else {
      d.nbands = (g.ny + R - 1) / R;
      d.nwt = tc.nwt > 0 ? tc.nwt : (g.nx + 63) / 64;
      int rc = snap_tiles(g.nx, d.nwt, &d.ntx, &d.st);
      if (rc) return rc;
    }
    const int max_row_warps = bits ? kBitsBandWarps : kNibbleBandWarps;
    if (d.ntx * d.nwt > max_row_warps)
      return set_error(QTV_ERR_ARG, "snapshot %d: %d tiles of %d warps exceed %d warps per row",
                       i, d.ntx, d.nwt, max_row_warps);
    d.seg0 = nseg;
    d.tab0 = tab;
    nseg += (long long)d.nbands * g.nz;
    tab += (long long)d.nbands * g.nz * d.ntx * d.nwt;
  }
  fin.nseg = nseg;
  // groups: snapshots with the same warps per tile, in order of appearance
  std::vector<int> gw;
  for (int i = 0; i < nsnap; ++i) {
    int gi = 0;
    while (gi < (int)gw.size() && gw[gi] != fin.s[i].nwt) ++gi;
    if (gi == (int)gw.size()) gw.push_back(fin.s[i].nwt);
    B->group_of[i] = gi;
  }
  double total_nodes = 0;
  for (int i = 0; i < nsnap; ++i)
    total_nodes += (double)grids[i].nx * grids[i].ny * grids[i].nz;
  unsigned long long slack = kChunk;
  B->groups.resize(gw.size());
  for (size_t gi = 0; gi < gw.size(); ++gi) {
    BulkLayout& L = B->groups[gi];
    BulkParams& p = L.p;
    p = BulkParams();
    p.nwt = gw[gi];
    long long units = 0;
    double nodes = 0;
    for (int i = 0; i < nsnap; ++i) {
      if (B->group_of[i] != (int)gi) continue;
      SnapDesc d = fin.s[i];
      d.unit0 = units;
      units += d.nstk ? ((long long)d.nbands * (d.ntx - 1) + d.nstk) * d.nz
                      : (long long)d.nbands * d.ntx * d.nz;
      nodes += (double)d.nx * d.ny * d.nz;
      p.s[p.nsnap++] = d;
    }
    p.units = units;
    p.nseg = nseg;
    int bps = 0;
    size_t smem = 0;
    int rc = bits ? bits_variant_occupancy(p.nwt, stages, &bps, &smem)
                  : bulk_variant_occupancy(p.nwt, &bps, &smem);
    if (rc) return rc;
    if (tc.ctas_per_sm > 0 && tc.ctas_per_sm < bps) bps = tc.ctas_per_sm;
    long long grid = (long long)bps * num_sms;
    // concurrent groups share the GPU in proportion to their nodes
    if (tc.concurrent && gw.size() > 1)
      grid = (long long)((double)grid * nodes / total_nodes + 0.5);
    if (max_warps > 0 && grid * p.nwt > (long long)max_warps) grid = (long long)max_warps / p.nwt;
    if (grid > units) grid = units;
    if (grid < 1) grid = 1;
    // z blocks: the CTAs that a snapshot gets (in proportion to its units)
    // are spread over its (band, tile) columns
    for (int j = 0; j < p.nsnap; ++j) {
      SnapDesc& d = p.s[j];
      const long long cols =
          d.nstk ? (long long)d.nbands * (d.ntx - 1) + d.nstk : (long long)d.nbands * d.ntx;
      const double share = (double)grid * (double)(cols * d.nz) / (double)units;
      long long zblocks = (long long)(share / (double)cols + 0.5);
      if (zblocks < 1) zblocks = 1;
      if (zblocks > d.nz) zblocks = d.nz;
      long long H = (d.nz + zblocks - 1) / zblocks;
      H = (long long)((double)H * (tc.zscale > 0.f ? tc.zscale : 1.f) + 0.5);
      if (H < 1) H = 1;
      if (H > d.nz) H = d.nz;
      d.hblock = (int)H;
    }
    L.grid = (int)grid;
    L.threads = p.nwt * 32;
    L.smem = smem;
    slack += 2ull * kChunk * (unsigned long long)grid * p.nwt;
  }
  B->concurrent = tc.concurrent && gw.size() > 1;
  B->ntiles = (nseg + kScanTile - 1) / kScanTile;
  // records: nibble sweep, at most one per pierced face plus two partly used
  // chunks per warp of every sweep; bit-sliced sweep, fixed slots of 32 per
  // (plane, band, tile, warp)
  B->recs_need = bits ? (unsigned long long)tab * 32ull : capacity + slack;
  B->table_need = (unsigned long long)tab;
  B->expand_blocks = (int)std::min<long long>((nseg + kExpandWarps - 1) / kExpandWarps,
                                              (long long)num_sms * (bits ? kBitsExpandCtasPerSm : 4));
  return QTV_OK;
}

namespace {

int check_scratch(const BatchLayout& B, const IdentScratch& sc, bool scan) {
  if (sc.staging_cap < B.recs_need * B.rec_words || sc.table_cap < B.table_need ||
      sc.seg_cap * 2 < (uint64_t)B.fin.nseg ||
      (scan && (sc.seg_off_cap < (uint64_t)B.fin.nseg || sc.tiles_cap < (uint64_t)B.ntiles)))
    return set_error(QTV_ERR_CAPACITY, "identification scratch too small for this layout");
  return QTV_OK;
}

// The sweeps of all groups on st, or (concurrent) on the branch streams
// forked from and joined back into st.
int launch_sweeps(qtv_handle h, BatchLayout& B, const IdentScratch& sc, cudaStream_t st,
                  const SweepBranches* br) {
  const bool fork = B.concurrent && br && (int)B.groups.size() <= br->n;
  cudaError_t e = cudaSuccess;
  if (fork) {
    e = cudaEventRecord(br->fork, st);
    if (e != cudaSuccess) return check_cuda(e, "cudaEventRecord(fork)");
  }
  for (size_t gi = 0; gi < B.groups.size(); ++gi) {
    BulkLayout& L = B.groups[gi];
    BulkParams& p = L.p;
    p.recs = sc.staging;
    p.recs_cap = B.recs_need;
    p.counters = sc.counters;
    p.table = sc.table;
    p.segf = reinterpret_cast<unsigned int*>(sc.seg);
    cudaStream_t s = st;
    if (fork) {
      s = br->streams[gi];
      e = cudaStreamWaitEvent(s, br->fork, 0);
      if (e != cudaSuccess) return check_cuda(e, "cudaStreamWaitEvent(fork)");
    }
    {
      TraceScope ts(h, K_SWEEP, s);
      if (B.variant == 1) bits_sweep_launch(p, L.grid, p.nwt, B.stages, L.smem, s);
      else bulk_fn(p.nwt)<<<L.grid, L.threads, L.smem, s>>>(p);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return check_cuda(e, "sweep_bulk_kernel launch");
    if (fork) {
      e = cudaEventRecord(br->join[gi], s);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(st, br->join[gi], 0);
      if (e != cudaSuccess) return check_cuda(e, "sweep join");
    }
  }
  return QTV_OK;
}

}  // namespace

// The launches of one layout: scratch zeroing, sweeps, scan, expand.  count
// receives the total; offsets (optional) receives the first face of each
// snapshot (nsnap entries).
int batch_launch(qtv_handle h, BatchLayout& B, const IdentScratch& sc, uint64_t* face_ids,
                 int8_t* winding, uint64_t capacity, uint64_t* count, uint64_t* offsets,
                 qtv_stats* stats, unsigned long long scanned, cudaStream_t st, bool expand_always,
                 const SweepBranches* br) {
  int rc = check_scratch(B, sc, true);
  if (rc) return rc;
  cudaError_t e = cudaMemsetAsync(sc.counters, 0, 4 * sizeof(unsigned long long), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(sc.tiles, 0, B.ntiles * sizeof(unsigned long long), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(sc.seg, 0, B.fin.nseg * sizeof(unsigned int), st);
  if (e == cudaSuccess && stats) e = cudaMemsetAsync(stats, 0, sizeof(qtv_stats), st);
  if (e != cudaSuccess) return check_cuda(e, "cudaMemsetAsync(identify scratch)");
  rc = launch_sweeps(h, B, sc, st, br);
  if (rc) return rc;
  {
    TraceScope ts(h, K_SEG_SCAN, st);
    e = launch_dependent(v3_scan_kernel, dim3((unsigned)B.ntiles), dim3(kScanThreads), 0, st,
                         reinterpret_cast<const unsigned int*>(sc.seg), B.fin.nseg, sc.seg_off,
                         count, sc.counters, sc.tiles, B.ntiles, stats, scanned,
                         h ? h->scan_hold_tile : -1ll,
                         (h && h->scan_spin_limit > 0) ? h->scan_spin_limit : (1ll << 32));
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return check_cuda(e, "v3_scan_kernel launch");
  if (capacity > 0 || expand_always) {
    BulkParams& p = B.fin;
    p.recs = sc.staging;
    p.recs_cap = B.recs_need;
    p.counters = sc.counters;
    p.table = sc.table;
    p.segf = reinterpret_cast<unsigned int*>(sc.seg);
    TraceScope ts(h, K_SCATTER, st);
    if (B.variant == 1)
      e = bits_expand_launch(p, B.expand_blocks, sc.seg_off, face_ids, winding, capacity, offsets,
                             st);
    else
      e = launch_dependent(v3_expand_kernel, dim3((unsigned)B.expand_blocks),
                           dim3(32 * kExpandWarps), 0, st, p, sc.seg_off, face_ids, winding,
                           capacity, offsets);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return check_cuda(e, "v3_expand_kernel launch");
  }
  return QTV_OK;
}

// Sweeps alone (autotuning): zeroing and the sweep launches of one layout.
int batch_sweep_only(qtv_handle h, BatchLayout& B, const IdentScratch& sc, cudaStream_t st,
                     const SweepBranches* br) {
  int rc = check_scratch(B, sc, false);
  if (rc) return rc;
  cudaError_t e = cudaMemsetAsync(sc.counters, 0, 4 * sizeof(unsigned long long), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(sc.seg, 0, B.fin.nseg * sizeof(unsigned int), st);
  if (e != cudaSuccess) return check_cuda(e, "cudaMemsetAsync(sweep scratch)");
  return launch_sweeps(h, B, sc, st, br);
}

// Sweep shape of a single-snapshot call: the handle's choice
// (qtv_configure_sweep), else the library default.
constexpr int kDefaultSweepVariant = 1;

TileConfig handle_sweep_config(const qtv_handle_s* h) {
  TileConfig tc;
  tc.variant = (h && h->sweep_variant >= 0) ? h->sweep_variant : kDefaultSweepVariant;
  // the bit-sliced sweep runs its CTAs over z blocks twice as tall as the
  // even split (fewer run changes, measured slightly faster)
  if (tc.variant == 1) tc.zscale = 2.f;
  if (h) {
    tc.nwt = h->sweep_nwt;
    tc.ctas_per_sm = h->sweep_ctas;
    if (h->sweep_stages > 0) tc.stages = h->sweep_stages;
  }
  return tc;
}

int staged_variant(const qtv_handle_s* h, int nx, int ny, int nz, const void* psi) {
  const int v = handle_sweep_config(h).variant;
  if (sweep_bulk_supported(v, nx, ny, nz, psi)) return v;
  if (v != 0 && sweep_bulk_supported(0, nx, ny, nz, psi)) return 0;
  return -1;
}

namespace {
// Layout of a single snapshot in the handle's shape; a grid the bit-sliced
// sweep cannot tile (too many warps per row for the handle's tile width)
// takes the nibble sweep where that can.
int single_layout(qtv_handle h, int num_sms, const qtv_grid& g, const float2* psi,
                  uint64_t capacity, uint64_t max_warps, BatchLayout* B) {
  TileConfig tc = handle_sweep_config(h);
  int rc = batch_layout(num_sms, 1, &g, &psi, tc, capacity, max_warps, B);
  if (rc && tc.variant == 1 && sweep_bulk_supported(0, g.nx, g.ny, g.nz, psi)) {
    TileConfig t0;
    rc = batch_layout(num_sms, 1, &g, &psi, t0, capacity, max_warps, B);
  }
  return rc;
}
}  // namespace

int bulk_needs(qtv_handle h, int num_sms, const qtv_grid& g, uint64_t capacity,
               uint64_t max_warps, BulkNeeds* n) {
  BatchLayout B;
  // alignment is checked by the caller; sizing needs only a 16-byte aligned stand-in
  const float2* psi = reinterpret_cast<const float2*>(uintptr_t(256));
  const int rc = single_layout(h, num_sms, g, psi, capacity, max_warps, &B);
  if (rc) return rc;
  n->recs = B.recs_need * B.rec_words;  // staging words
  n->table = B.table_need;
  n->seg_off = (unsigned long long)B.fin.nseg;
  n->tiles = (unsigned long long)B.ntiles;
  n->segf = (unsigned long long)(B.fin.nseg + 1) / 2;  // uint2 entries holding nseg u32
  return QTV_OK;
}

int bulk_identify(qtv_handle h, const qtv_grid& g, const float2* psi, uint64_t* face_ids,
                  int8_t* winding, uint64_t capacity, uint64_t* count, qtv_stats* stats,
                  cudaStream_t st, const IdentScratch& sc, uint64_t max_warps, float* xyz,
                  float* resid, uint8_t* flags) {
  BatchLayout B;
  int rc = single_layout(h, h->num_sms, g, psi, capacity, max_warps, &B);
  if (rc) return rc;
  const unsigned long long nx = g.nx, ny = g.ny, nz = g.nz;
  const unsigned long long scanned =
      (nx - 1) * (ny - 1) * nz + nx * (ny - 1) * (nz - 1) + (nx - 1) * ny * (nz - 1);
  rc = batch_launch(h, B, sc, face_ids, winding, capacity, count, nullptr, stats, scanned, st,
                    false, nullptr);
  if (rc) return rc;
  if (xyz && capacity > 0)
    return localize_launch(h, g, psi, face_ids, winding, capacity, count, xyz, resid, flags, st);
  return QTV_OK;
}

}  // namespace qtv
