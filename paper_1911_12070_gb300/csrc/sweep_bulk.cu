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
// Staging.  Thread 0 copies the band rows of each plane into one slot of a
// 3-deep ring in shared memory with cp.async.bulk (one copy per row; completion
// counted in bytes on the slot's mbarrier).  Threads read their 16-byte pairs
// and the x-neighbour column from shared memory, so global latency is covered
// by the ring.  Waits are bounded (about 2^32 SM cycles); a timeout sets a
// status bit that turns the reported count into QTV_COUNT_TIMEOUT.
//
// Edge test.  The winding contribution of edge a -> b is r = s_b - s_a when
// the edge crosses the negative real axis and 0 otherwise (s = Im < 0).  With
// s_a != s_b that happens iff cross(a, b) = Re a Im b - Im a Re b has the sign
// of s_b - s_a.  Its FP32 FMA evaluation fma(Re a, Im b, -RN(Im a Re b)) has
// the exact sign in every case that matters: when Re a and Re b have equal
// signs the two terms cannot cancel, and when they differ |d| > pi/2, so a
// wrong sign needs |sin d| < 2^-24, an edge within 1e-7 rad of +-pi (an
// ambiguous edge).  Only the "cross > 0" bit is formed; a zero cross product
// (a node with psi == 0) needs both comparisons, so a warp whose planes hold a
// zero or non-finite node takes an exact path with both comparisons and drops
// the faces that touch non-finite nodes.
//
// Compaction.  Each warp, each plane, emits one 32-bit record per (lane, row)
// that has a pierced face: the six (W+4)^4 nibbles of the lane's two columns
// and three orientations, the lane and the row.  Record positions come from
// per-row warp ballots, so no shuffle scan and no cross-warp step is needed;
// records go to per-warp chunks of a staging buffer reserved with one global
// atomic per chunk (prefetched), and a 16-byte table entry per (plane, band,
// warp) says where they are and how many faces they hold.  A finalize pass
// scans the face totals in (plane, band) order (single pass, decoupled
// look-back) and expands the records of each segment in (row, warp, lane)
// order, which is ascending face-id order.
//
// Schedule.  Work units are (plane, band) pairs ordered (z block, band, plane)
// and cut into one contiguous range per CTA, so all CTAs get the same number
// of planes, and CTAs that hold neighbouring bands march the same z block at
// the same time (the halo row of a band is the first row of the next one and
// is then served by L2).
#include "qtv_internal.cuh"

namespace qtv {
namespace {

constexpr int R = kRows;
constexpr int RH = R + 1;
constexpr int kStages = 3;
constexpr uint32_t kOnes = 0x11111111u;
constexpr uint32_t kFours = 0x44444444u;
constexpr uint32_t kOwned = 0x0FFFFFFFu;
constexpr uint32_t kOwnedBits = 0x01111111u;  // bit 0 of the fields of rows 0..6

__device__ __forceinline__ uint32_t nz_fields(uint32_t d) {
  uint32_t t = d | (d >> 2);
  t = t | (t >> 1);
  return t & kOnes;
}

__device__ __forceinline__ bool finite_f(float v) { return fabsf(v) <= 3.402823466e38f; }

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase with the given parity; false after ~2^32 cycles.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > (1ll << 32)) return false;
  }
  return true;
}

__device__ __forceinline__ float cross_f(float ar, float ai, float br, float bi) {
  return fmaf(ar, bi, -(ai * br));
}

// s-bits (Im < 0) of one column over the RH rows, one bit per 4-bit field
__device__ __forceinline__ uint32_t sbits_col(const float4* v, int p) {
  uint32_t s = 0;
#pragma unroll
  for (int r = 0; r < RH; ++r)
    if ((p ? v[r].w : v[r].y) < 0.f) s |= 1u << (4 * r);
  return s;
}
__device__ __forceinline__ uint32_t sbits_nb(const float2* v) {
  uint32_t s = 0;
#pragma unroll
  for (int r = 0; r < RH; ++r)
    if (v[r].y < 0.f) s |= 1u << (4 * r);
  return s;
}

// packed edge values (value + 1 per field) from tail/head s-bits and the
// cross-sign bits
__device__ __forceinline__ uint32_t pack_fast(uint32_t SA, uint32_t SB, uint32_t CP) {
  return kOnes + (~SA & SB & CP) - (SA & ~SB & ~CP);
}
__device__ __forceinline__ uint32_t pack_exact(uint32_t SA, uint32_t SB, uint32_t CP, uint32_t CN) {
  return kOnes + (~SA & SB & CP) - (SA & ~SB & CN);
}

struct SmallSmem {
  uint2 xbits[2][kMaxWarpsX];  // {rz_k, ry_k+1} fields of column x0 of each warp
};

constexpr uint32_t kChunk = 64;    // records per staging chunk
constexpr uint32_t kLowWater = 24; // prefetch the next chunk below this

// Edge fields of one step.  In: plane k (cur, s-bits Sk0/Sk1) and plane k+1
// (nxt, nb column nbv).  EXACT selects both comparisons (zero nodes).
template <bool EXACT>
__device__ __forceinline__ void step_edges(const float4* cur, const float4* nxt, const float2* nbv,
                                           uint32_t Sk0, uint32_t Sk1, uint32_t& S0n,
                                           uint32_t& S1n, uint32_t& SNn, uint32_t& RZ0,
                                           uint32_t& RZ1, uint32_t& RX0n, uint32_t& RX1n,
                                           uint32_t& RY0n, uint32_t& RY1n) {
  S0n = sbits_col(nxt, 0);
  S1n = sbits_col(nxt, 1);
  SNn = sbits_nb(nbv);
  uint32_t pz0 = 0, pz1 = 0, px0 = 0, px1 = 0, py0 = 0, py1 = 0;
  uint32_t nz0 = 0, nz1 = 0, nx0 = 0, nx1 = 0, ny0 = 0, ny1 = 0;
#pragma unroll
  for (int r = 0; r < RH; ++r) {
    const uint32_t bit = 1u << (4 * r);
    const float cz0 = cross_f(cur[r].x, cur[r].y, nxt[r].x, nxt[r].y);
    const float cz1 = cross_f(cur[r].z, cur[r].w, nxt[r].z, nxt[r].w);
    const float cx0 = cross_f(nxt[r].x, nxt[r].y, nxt[r].z, nxt[r].w);
    const float cx1 = cross_f(nxt[r].z, nxt[r].w, nbv[r].x, nbv[r].y);
    if (cz0 > 0.f) pz0 |= bit;
    if (cz1 > 0.f) pz1 |= bit;
    if (cx0 > 0.f) px0 |= bit;
    if (cx1 > 0.f) px1 |= bit;
    if (EXACT) {
      if (cz0 < 0.f) nz0 |= bit;
      if (cz1 < 0.f) nz1 |= bit;
      if (cx0 < 0.f) nx0 |= bit;
      if (cx1 < 0.f) nx1 |= bit;
    }
    if (r < R) {
      const float cy0 = cross_f(nxt[r].x, nxt[r].y, nxt[r + 1].x, nxt[r + 1].y);
      const float cy1 = cross_f(nxt[r].z, nxt[r].w, nxt[r + 1].z, nxt[r + 1].w);
      if (cy0 > 0.f) py0 |= bit;
      if (cy1 > 0.f) py1 |= bit;
      if (EXACT) {
        if (cy0 < 0.f) ny0 |= bit;
        if (cy1 < 0.f) ny1 |= bit;
      }
    }
  }
  const uint32_t SY0 = S0n & kOwnedBits, SY1 = S1n & kOwnedBits;
  if (EXACT) {
    RZ0 = pack_exact(Sk0, S0n, pz0, nz0);
    RZ1 = pack_exact(Sk1, S1n, pz1, nz1);
    RX0n = pack_exact(S0n, S1n, px0, nx0);
    RX1n = pack_exact(S1n, SNn, px1, nx1);
    RY0n = pack_exact(SY0, S0n >> 4, py0, ny0);
    RY1n = pack_exact(SY1, S1n >> 4, py1, ny1);
  } else {
    RZ0 = pack_fast(Sk0, S0n, pz0);
    RZ1 = pack_fast(Sk1, S1n, pz1);
    RX0n = pack_fast(S0n, S1n, px0);
    RX1n = pack_fast(S1n, SNn, px1);
    RY0n = pack_fast(SY0, S0n >> 4, py0);
    RY1n = pack_fast(SY1, S1n >> 4, py1);
  }
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


struct V3Args {
  const float2* psi;
  int nx, ny, nz, nbands, hblock;
  uint32_t* recs;
  unsigned long long recs_cap;
  unsigned long long* counters;  // [0] chunk top, [1] status bits, [2] scan ticket
  uint4* table;                  // [(k * nbands + band) * NW + w]
};

// unit u of the (z block, band, plane) order -> band, plane, end of its z block
__device__ __forceinline__ void unit_pos(long long u, int nbands, int nz, int H, int& band, int& k,
                                         int& kend) {
  const long long full = nz / H;
  const long long per_full = (long long)nbands * H;
  long long zb, rem;
  int h;
  if (u < full * per_full) {
    zb = u / per_full;
    rem = u % per_full;
    h = H;
  } else {
    zb = full;
    rem = u - full * per_full;
    h = nz - (int)full * H;
  }
  band = (int)(rem / h);
  k = (int)zb * H + (int)(rem % h);
  kend = (int)zb * H + h;
}

template <int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB) sweep_bulk_kernel(V3Args a) {
  extern __shared__ __align__(128) unsigned char dsm[];
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int w = tid >> 5;
  const int NW = blockDim.x >> 5;
  const int W = NW * 64;  // row pitch of a ring slot, in elements
  float2* ring = reinterpret_cast<float2*>(dsm);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(dsm + (size_t)kStages * RH * W * sizeof(float2));
  SmallSmem& sm = *reinterpret_cast<SmallSmem*>(mbar + kStages);
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int x0 = 64 * w + 2 * lane;
  const bool c0 = x0 < nx, c1 = x0 + 1 < nx, c2 = x0 + 2 < nx;
  const bool nbin = x0 + 2 < W;
  const size_t plane = (size_t)nx * ny;
  const uint32_t row_bytes = (uint32_t)nx * 8u;
  const uint32_t lt = (1u << lane) - 1u;

  // columns [nx, W) of every slot row are never copied: fill them with 1 (a
  // finite, nonzero value, so that padding never sends a warp down the exact
  // path; faces that touch padding do not exist and are masked anyway)
  {
    const int pad = W - nx;
    for (int idx = tid; idx < kStages * RH * pad; idx += blockDim.x)
      ring[(size_t)(idx / pad) * W + nx + idx % pad] = make_float2(1.f, 0.f);
  }
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&mbar[s], 1);
    fence_mbar_init();
  }
  __syncthreads();

  uint32_t fill = 0, use = 0;  // planes issued / consumed by this CTA (uniform)
  bool timeout = false;
  // per-warp record chunk (uniform within the warp)
  uint32_t cb = 0, cl = 0, nb_l0 = 0;
  bool have_next = false;
  bool overflow = false;

  const long long U = (long long)a.nbands * nz;
  long long u = U * blockIdx.x / gridDim.x;
  const long long uend = U * (blockIdx.x + 1) / gridDim.x;

  while (u < uend) {
    int band, kb, kblk;
    unit_pos(u, a.nbands, nz, a.hblock, band, kb, kblk);
    const int ke = (int)min((long long)kblk, (long long)kb + (uend - u));
    u += ke - kb;
    const int j0 = band * R;
    const int nrows = min(RH, ny - j0);
    const int klast = min(ke, nz - 1);
    const int nplanes = klast - kb + 1;
    const int nsteps = ke - kb;

    if (nrows < RH) {  // rows beyond the grid are never copied: fill with 1
      const int per = (RH - nrows) * W;
      for (int idx = tid; idx < kStages * per; idx += blockDim.x) {
        const int s = idx / per, rem = idx % per;
        ring[((size_t)s * RH + nrows + rem / W) * W + rem % W] = make_float2(1.f, 0.f);
      }
      __syncthreads();
    }

    auto issue = [&](int m) {  // copy plane m of the band into the next slot
      if (tid == 0) {
        uint64_t* bar = &mbar[fill % kStages];
        float2* dst = ring + (size_t)(fill % kStages) * RH * W;
        fence_proxy_async();
        mbar_arrive_expect_tx(bar, row_bytes * (uint32_t)nrows);
        const float2* src = a.psi + (size_t)m * plane + (size_t)j0 * nx;
        for (int r = 0; r < nrows; ++r)
          bulk_g2s(dst + (size_t)r * W, src + (size_t)r * nx, row_bytes, bar);
      }
      ++fill;
    };
    auto acquire = [&]() -> const float2* {
      const int s = use % kStages;
      if (!mbar_wait(&mbar[s], (use / kStages) & 1u)) timeout = true;
      ++use;
      return ring + (size_t)s * RH * W;
    };

    // row validity and slot existence (bit 0 of each field)
    uint32_t rowv = 0, rowv1 = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (j0 + r < ny) rowv |= 1u << (4 * r);
      if (j0 + r + 1 < ny) rowv1 |= 1u << (4 * r);
    }
    const uint32_t ex_xy0 = c1 ? rowv1 : 0u, ex_xy1 = c2 ? rowv1 : 0u;
    const uint32_t ex_yz0 = c0 ? rowv1 : 0u, ex_yz1 = c1 ? rowv1 : 0u;
    const uint32_t ex_zx0 = c1 ? rowv : 0u, ex_zx1 = c2 ? rowv : 0u;

    // ---- prologue: plane kb
    for (int i = 0; i < min(kStages, nplanes); ++i) issue(kb + i);
    float4 bufA[RH], bufB[RH];
    uint32_t Sk0, Sk1, RX0, RX1, RY0, RY1, RYN;
    bool bad_k;
    uint32_t Bk0 = 0, Bk1 = 0, BkN = 0;  // non-finite bits of plane k (exact path only)
    {
      const float2* sp = acquire();
      float2 nbv[RH];
#pragma unroll
      for (int r = 0; r < RH; ++r) {
        bufA[r] = *reinterpret_cast<const float4*>(sp + (size_t)r * W + x0);
        nbv[r] = nbin ? sp[(size_t)r * W + x0 + 2] : make_float2(1.f, 0.f);
      }
      float prod = 1.f;
#pragma unroll
      for (int r = 0; r < RH; ++r)
        prod *= (fabsf(bufA[r].x) + fabsf(bufA[r].y)) * (fabsf(bufA[r].z) + fabsf(bufA[r].w)) *
                (fabsf(nbv[r].x) + fabsf(nbv[r].y));
      bad_k = __any_sync(0xffffffffu, !(prod > 0.f && prod <= 3.402823466e38f));
      Sk0 = sbits_col(bufA, 0);
      Sk1 = sbits_col(bufA, 1);
      const uint32_t SN = sbits_nb(nbv);
      uint32_t px0 = 0, px1 = 0, py0 = 0, py1 = 0, pyn = 0, qx0 = 0, qx1 = 0, qy0 = 0, qy1 = 0,
               qyn = 0;
#pragma unroll
      for (int r = 0; r < RH; ++r) {
        const uint32_t bit = 1u << (4 * r);
        const float cx0 = cross_f(bufA[r].x, bufA[r].y, bufA[r].z, bufA[r].w);
        const float cx1 = cross_f(bufA[r].z, bufA[r].w, nbv[r].x, nbv[r].y);
        if (cx0 > 0.f) px0 |= bit;
        if (cx1 > 0.f) px1 |= bit;
        if (cx0 < 0.f) qx0 |= bit;
        if (cx1 < 0.f) qx1 |= bit;
        if (r < R) {
          const float cy0 = cross_f(bufA[r].x, bufA[r].y, bufA[r + 1].x, bufA[r + 1].y);
          const float cy1 = cross_f(bufA[r].z, bufA[r].w, bufA[r + 1].z, bufA[r + 1].w);
          const float cyn = cross_f(nbv[r].x, nbv[r].y, nbv[r + 1].x, nbv[r + 1].y);
          if (cy0 > 0.f) py0 |= bit;
          if (cy1 > 0.f) py1 |= bit;
          if (cyn > 0.f) pyn |= bit;
          if (cy0 < 0.f) qy0 |= bit;
          if (cy1 < 0.f) qy1 |= bit;
          if (cyn < 0.f) qyn |= bit;
        }
      }
      RX0 = pack_exact(Sk0, Sk1, px0, qx0);
      RX1 = pack_exact(Sk1, SN, px1, qx1);
      RY0 = pack_exact(Sk0 & kOwnedBits, Sk0 >> 4, py0, qy0);
      RY1 = pack_exact(Sk1 & kOwnedBits, Sk1 >> 4, py1, qy1);
      RYN = pack_exact(SN & kOwnedBits, SN >> 4, pyn, qyn);
      if (bad_k) {
        Bk0 = badbits_col(bufA, 0);
        Bk1 = badbits_col(bufA, 1);
        BkN = badbits_nb(nbv);
      }
    }
    __syncthreads();  // slot of plane kb fully read
    if (kb + kStages <= klast) issue(kb + kStages);

    // one z step: plane k = kb + t in C, plane k + 1 loaded into N
    auto step = [&](float4(&C)[RH], float4(&N)[RH], int t) {
      const int k = kb + t;
      const bool has_up = k + 1 < nz;
      uint32_t S0n = 0, S1n = 0, SNn = 0, RZ0 = kOnes, RZ1 = kOnes, RX0n = kOnes, RX1n = kOnes,
               RY0n = kOnes, RY1n = kOnes;
      uint32_t Bn0 = 0, Bn1 = 0, BnN = 0;
      bool bad_k1 = false;
      if (has_up) {
        const float2* sp = acquire();
        float2 nbv[RH];
#pragma unroll
        for (int r = 0; r < RH; ++r) {
          N[r] = *reinterpret_cast<const float4*>(sp + (size_t)r * W + x0);
          nbv[r] = nbin ? sp[(size_t)r * W + x0 + 2] : make_float2(1.f, 0.f);
        }
        float prod = 1.f;
#pragma unroll
        for (int r = 0; r < RH; ++r)
          prod *= (fabsf(N[r].x) + fabsf(N[r].y)) * (fabsf(N[r].z) + fabsf(N[r].w)) *
                  (fabsf(nbv[r].x) + fabsf(nbv[r].y));
        bad_k1 = __any_sync(0xffffffffu, !(prod > 0.f && prod <= 3.402823466e38f));
        if (bad_k || bad_k1) {
          step_edges<true>(C, N, nbv, Sk0, Sk1, S0n, S1n, SNn, RZ0, RZ1, RX0n, RX1n, RY0n, RY1n);
          Bn0 = badbits_col(N, 0);
          Bn1 = badbits_col(N, 1);
          BnN = badbits_nb(nbv);
        } else {
          step_edges<false>(C, N, nbv, Sk0, Sk1, S0n, S1n, SNn, RZ0, RZ1, RX0n, RX1n, RY0n, RY1n);
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
        for (int s = 0; s < 6; ++s) keep[s] &= ~((bb[s] & kOnes) * 0xFu);
      }
      uint32_t cnt = 0, anyf = 0;
#pragma unroll
      for (int s = 0; s < 6; ++s) {
        d[s] = (d[s] ^ kFours) & keep[s];
        const uint32_t nzb = nz_fields(d[s]);
        cnt += nzb;
        anyf |= nzb;
      }
      // ---- per-warp compaction: one record per (lane, row) with faces
      const uint32_t bsum = (cnt & 0x0F0F0F0Fu) + ((cnt >> 4) & 0x0F0F0F0Fu);
      const uint32_t faces_w = __reduce_add_sync(0xffffffffu, (bsum * 0x01010101u) >> 24);
      {
        uint32_t bal[R], pre[R];
        uint32_t T = 0, rc_lo = 0, rc_hi = 0;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          bal[r] = __ballot_sync(0xffffffffu, (anyf >> (4 * r)) & 1u);
          pre[r] = T;
          const uint32_t c = __popc(bal[r]);
          T += c;
          if (r < 5) rc_lo |= c << (6 * r);
          else rc_hi |= c << (6 * (r - 5));
        }
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
        if (lane == 0)
          a.table[((size_t)k * a.nbands + band) * NW + w] =
              make_uint4(base1, base2, rc_lo, rc_hi | (n1 << 12) | (faces_w << 20));
#pragma unroll
        for (int r = 0; r < R; ++r) {
          if ((anyf >> (4 * r)) & 1u) {
            const uint32_t q = pre[r] + __popc(bal[r] & lt);
            const unsigned long long addr =
                q < n1 ? (unsigned long long)base1 + q : (unsigned long long)base2 + (q - n1);
            uint32_t rec = ((uint32_t)r << 29) | ((uint32_t)lane << 24);
#pragma unroll
            for (int s = 0; s < 6; ++s) rec |= ((d[s] >> (4 * r)) & 0xFu) << (4 * s);
            if (addr < a.recs_cap) a.recs[addr] = rec;
          }
        }
      }
      // plane k + 1 becomes plane k
      Sk0 = S0n;
      Sk1 = S1n;
      RX0 = RX0n;
      RX1 = RX1n;
      RY0 = RY0n;
      RY1 = RY1n;
      RYN = RYNn;
      bad_k = bad_k1;
      Bk0 = Bn0;
      Bk1 = Bn1;
      BkN = BnN;
      (void)SNn;
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
// Finalize 1: exclusive scan of the per-segment face totals in (plane, band)
// order, single pass with decoupled look-back over tiles taken by ticket.
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
    const uint4* __restrict__ table, int NW, long long nseg, unsigned long long* __restrict__ seg_off,
    uint64_t* count, unsigned long long* counters, unsigned long long* tiles, long long ntiles,
    qtv_stats* stats, unsigned long long scanned) {
  __shared__ unsigned long long s_warp[kScanThreads / 32];
  __shared__ unsigned long long s_prefix;
  __shared__ long long s_tile;
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
    uint32_t f = 0;
    if (s < nseg)
      for (int q = 0; q < NW; ++q) f += __ldg(&table[s * NW + q].w) >> 20;
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
      if (tile == 0) {
        atomicExch(&tiles[0], kFlagP | agg);
      } else {
        atomicExch(&tiles[tile], kFlagA | agg);
        long long p = tile - 1;
        while (p >= 0) {
          unsigned long long st = ld_volatile_u64(&tiles[p]);
          if ((st >> 62) == 0) {
            const long long t0 = clock64();
            while ((st >> 62) == 0) {
              st = ld_volatile_u64(&tiles[p]);
              if (clock64() - t0 > (1ll << 32)) break;
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
        atomicExch(&tiles[tile], kFlagP | (prefix + agg));
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
// Finalize 2: one warp per (plane, band) segment expands its records, in
// (row, warp, lane) order, into face ids and windings at their final offsets.
// ---------------------------------------------------------------------------
constexpr int kExpandWarps = 8;

__global__ void __launch_bounds__(32 * kExpandWarps) v3_expand_kernel(
    const uint4* __restrict__ table, int NW, long long nseg, int nbands, int nx, int ny,
    const uint32_t* __restrict__ recs, unsigned long long recs_cap,
    const unsigned long long* __restrict__ seg_off, uint64_t* __restrict__ face_ids,
    int8_t* __restrict__ winding, unsigned long long capacity) {
  __shared__ uint32_t s_start[kExpandWarps][R][kMaxWarpsX];
  __shared__ uint32_t s_wpre[kExpandWarps][R][kMaxWarpsX];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const long long nwarps = (long long)gridDim.x * kExpandWarps;
  for (long long s = (long long)blockIdx.x * kExpandWarps + wib; s < nseg; s += nwarps) {
    uint4 e = make_uint4(0u, 0u, 0u, 0u);
    if (lane < NW) e = table[s * NW + lane];
    const uint32_t base1 = e.x, base2 = e.y, n1 = (e.w >> 12) & 0xFFu;
    uint32_t rowstart[R];
    uint32_t run = 0, wp = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const uint32_t n = r < 5 ? (e.z >> (6 * r)) & 63u : (e.w >> (6 * (r - 5))) & 63u;
      uint32_t incl = n;
#pragma unroll
      for (int dd = 1; dd < 32; dd <<= 1) {
        const uint32_t x = __shfl_up_sync(0xffffffffu, incl, dd);
        if (lane >= dd) incl += x;
      }
      rowstart[r] = run;
      if (lane < NW) {
        s_start[wib][r][lane] = run + incl - n;
        s_wpre[wib][r][lane] = wp;
      }
      wp += n;
      run += __shfl_sync(0xffffffffu, incl, 31);
    }
    __syncwarp();
    const uint32_t rtot = run;
    if (rtot == 0) continue;
    const unsigned long long fbase = seg_off[s];
    const long long k = s / nbands;
    const int band = (int)(s % nbands);
    const long long j0 = (long long)band * R;
    unsigned long long fo = 0;
    for (uint32_t g0 = 0; g0 < rtot; g0 += 32) {
      const uint32_t g = g0 + lane;
      const bool valid = g < rtot;
      int r = 0;
#pragma unroll
      for (int rr = 1; rr < R; ++rr)
        if (rowstart[rr] <= g) r = rr;
      int ww = 0;
      for (int q = 1; q < NW; ++q)
        if (s_start[wib][r][q] <= g) ww = q;
      const uint32_t widx = g - s_start[wib][r][ww] + s_wpre[wib][r][ww];
      const uint32_t b1 = __shfl_sync(0xffffffffu, base1, ww);
      const uint32_t b2 = __shfl_sync(0xffffffffu, base2, ww);
      const uint32_t m1 = __shfl_sync(0xffffffffu, n1, ww);
      const unsigned long long addr =
          widx < m1 ? (unsigned long long)b1 + widx : (unsigned long long)b2 + (widx - m1);
      const uint32_t rec = (valid && addr < recs_cap) ? recs[addr] : 0u;
      const uint32_t nf = __popc(nz_fields(rec & 0x00FFFFFFu));
      uint32_t incl = nf;
#pragma unroll
      for (int dd = 1; dd < 32; dd <<= 1) {
        const uint32_t x = __shfl_up_sync(0xffffffffu, incl, dd);
        if (lane >= dd) incl += x;
      }
      unsigned long long pos = fbase + fo + (incl - nf);
      if (nf) {
        const uint32_t rrow = rec >> 29, rl = (rec >> 24) & 31u;
        const unsigned long long lin0 =
            ((unsigned long long)k * ny + (unsigned long long)(j0 + rrow)) * nx + 64u * ww + 2u * rl;
#pragma unroll
        for (int sl = 0; sl < 6; ++sl) {
          const uint32_t nib = (rec >> (4 * sl)) & 0xFu;
          if (nib) {
            if (pos < capacity) {
              face_ids[pos] = ((lin0 + (unsigned long long)(sl / 3)) << 2) | (unsigned)(sl % 3);
              winding[pos] = (int8_t)((int)(nib ^ 4u) - 4);
            }
            ++pos;
          }
        }
      }
      fo += __shfl_sync(0xffffffffu, incl, 31);
    }
  }
}

using BulkFn = void (*)(V3Args);

BulkFn bulk_fn(int nw) {
  if (nw <= 4) return sweep_bulk_kernel<128, 4>;
  if (nw <= 8) return sweep_bulk_kernel<256, 2>;
  return sweep_bulk_kernel<512, 1>;
}

struct BulkPlan {
  int grid = 0, nw = 0, hblock = 1;
  size_t smem = 0;
  long long nseg = 0, ntiles = 0;
  unsigned long long recs_need = 0, table_need = 0;
};

size_t bulk_smem_bytes(int nx) {
  const int nw = (nx + 63) / 64;
  return (size_t)kStages * RH * nw * 64 * sizeof(float2) + kStages * sizeof(uint64_t) +
         sizeof(SmallSmem);
}

int bulk_plan(int num_sms, const qtv_grid& g, uint64_t capacity, uint64_t max_warps,
              BulkPlan* p) {
  const int nw = (g.nx + 63) / 64;
  const int nbands = (g.ny + R - 1) / R;
  BulkFn fn = bulk_fn(nw);
  static bool attr_set[3] = {false, false, false};
  const int which = nw <= 4 ? 0 : (nw <= 8 ? 1 : 2);
  if (!attr_set[which]) {
    cudaError_t e =
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e != cudaSuccess) return check_cuda(e, "cudaFuncSetAttribute(sweep_bulk)");
    attr_set[which] = true;
  }
  p->smem = bulk_smem_bytes(g.nx);
  int bps = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, nw * 32, p->smem);
  if (e != cudaSuccess) return check_cuda(e, "occupancy(sweep_bulk)");
  if (bps < 1) return set_error(QTV_ERR_ARG, "sweep_bulk: no resident CTA for nx = %d", g.nx);
  const long long units = (long long)nbands * g.nz;
  long long grid = (long long)bps * num_sms;
  if (max_warps > 0 && grid * nw > (long long)max_warps) grid = (long long)max_warps / nw;
  if (grid > units) grid = units;
  if (grid < 1) grid = 1;
  long long zblocks = (grid + nbands / 2) / nbands;
  if (zblocks < 1) zblocks = 1;
  if (zblocks > g.nz) zblocks = g.nz;
  p->grid = (int)grid;
  p->nw = nw;
  p->hblock = (int)((g.nz + zblocks - 1) / zblocks);
  p->nseg = (long long)g.nz * nbands;
  p->ntiles = (p->nseg + kScanTile - 1) / kScanTile;
  p->recs_need = capacity + 2ull * kChunk * (unsigned long long)grid * nw + kChunk;
  p->table_need = (unsigned long long)p->nseg * nw;
  return QTV_OK;
}

}  // namespace

bool sweep_bulk_supported(int nx, int ny, int nz, const void* psi) {
  if (nx < 2 || ny < 1 || nz < 1 || (nx & 1) || nx > 1024) return false;
  if (reinterpret_cast<uintptr_t>(psi) & 15u) return false;
  return bulk_smem_bytes(nx) <= 227u * 1024u;
}

int bulk_needs(int num_sms, const qtv_grid& g, uint64_t capacity, uint64_t max_warps,
               BulkNeeds* n) {
  BulkPlan p;
  const int rc = bulk_plan(num_sms, g, capacity, max_warps, &p);
  if (rc) return rc;
  n->recs = p.recs_need;
  n->table = p.table_need;
  n->seg_off = (unsigned long long)p.nseg;
  n->tiles = (unsigned long long)p.ntiles;
  return QTV_OK;
}

int bulk_identify(qtv_handle h, const qtv_grid& g, const float2* psi, uint64_t* face_ids,
                  int8_t* winding, uint64_t capacity, uint64_t* count, qtv_stats* stats,
                  cudaStream_t st, const IdentScratch& sc, uint64_t max_warps) {
  BulkPlan p;
  int rc = bulk_plan(h->num_sms, g, capacity, max_warps, &p);
  if (rc) return rc;
  if (sc.staging_cap < p.recs_need || sc.table_cap < p.table_need ||
      sc.seg_off_cap < (uint64_t)p.nseg || sc.tiles_cap < (uint64_t)p.ntiles)
    return set_error(QTV_ERR_CAPACITY, "identification scratch too small for this grid");
  cudaError_t e = cudaMemsetAsync(sc.counters, 0, 4 * sizeof(unsigned long long), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(sc.tiles, 0, p.ntiles * sizeof(unsigned long long), st);
  if (e == cudaSuccess && stats) e = cudaMemsetAsync(stats, 0, sizeof(qtv_stats), st);
  if (e != cudaSuccess) return check_cuda(e, "cudaMemsetAsync(identify scratch)");
  V3Args a;
  a.psi = psi;
  a.nx = g.nx;
  a.ny = g.ny;
  a.nz = g.nz;
  a.nbands = (g.ny + R - 1) / R;
  a.hblock = p.hblock;
  a.recs = sc.staging;
  a.recs_cap = p.recs_need;
  a.counters = sc.counters;
  a.table = sc.table;
  {
    TraceScope ts(h, K_SWEEP, st);
    bulk_fn(p.nw)<<<p.grid, p.nw * 32, p.smem, st>>>(a);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return check_cuda(e, "sweep_bulk_kernel launch");
  const unsigned long long nx = g.nx, ny = g.ny, nz = g.nz;
  const unsigned long long scanned =
      (nx - 1) * (ny - 1) * nz + nx * (ny - 1) * (nz - 1) + (nx - 1) * ny * (nz - 1);
  {
    TraceScope ts(h, K_SEG_SCAN, st);
    v3_scan_kernel<<<(unsigned)p.ntiles, kScanThreads, 0, st>>>(
        sc.table, p.nw, p.nseg, sc.seg_off, count, sc.counters, sc.tiles, p.ntiles, stats, scanned);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return check_cuda(e, "v3_scan_kernel launch");
  if (capacity > 0) {
    long long blocks = (p.nseg + kExpandWarps - 1) / kExpandWarps;
    const long long maxb = (long long)h->num_sms * 16;
    if (blocks > maxb) blocks = maxb;
    TraceScope ts(h, K_SCATTER, st);
    v3_expand_kernel<<<(unsigned)blocks, 32 * kExpandWarps, 0, st>>>(
        sc.table, p.nw, p.nseg, a.nbands, g.nx, g.ny, sc.staging, p.recs_need, sc.seg_off, face_ids,
        winding, capacity);
    e = cudaGetLastError();
    if (e != cudaSuccess) return check_cuda(e, "v3_expand_kernel launch");
  }
  return QTV_OK;
}

}  // namespace qtv
