// sweep_bits.cu -- bit-sliced identification sweep (Sec. 2.2.2, Eq. 5).
//
// Decomposition.  A CTA owns a band of 16 rows (+1 halo row) of an x tile and
// marches z.  Lane l of warp w owns the grid column x = 31 w + l of the tile;
// lane 31 is the halo column of the warp (the first column of the next warp)
// and owns no faces, so every quantity of column x + 1 that a lane needs comes
// from lane l + 1 by a shuffle.  Each lane walks its 17 rows and keeps one bit
// per row in 32-bit words: the sign bit of Im psi (the half-plane of the node)
// and the sign bits of the cross products of its x, y and z edges.
//
// Edge test.  As in the nibble sweep (sweep_bulk.cu): with s the sign bit of
// Im psi (IEEE atan2 convention) and n the sign bit of the FP32 FMA value of
// cross(a, b) = Re a Im b - Im a Re b, the branch-crossing integer of edge
// a -> b is +1 when s_a = 0, s_b = 1, n = 0, and -1 when s_a = 1, s_b = 0,
// n = 1, else 0.  Per word of 17 rows: P = ~s_a & s_b & ~n, N = s_a & ~s_b &
// n, and Z = P | N.
//
// Plaquette sums.  W = r1 + r2 - r3 - r4 lies in {-1, 0, 1, 2} (four wrapped
// differences in (-pi, pi] add to a multiple of 2 pi in (-4 pi, 4 pi]), so W
// is fixed by W mod 4.  A term t = +-r has the 2-bit code (Z, N) for +r and
// (Z, P) for -r (1 = 01, -1 = 11); the sum of four codes mod 4 has low bit
// L = xor of the four Z and high bit H = xor of the four high bits xor the
// parity of the pairs of Z (the carry), so W = 1, 2, -1 for (L, H) = (1, 0),
// (0, 1), (1, 1).  Each orientation takes nine 3-input logic operations for
// 16 rows.
//
// Zero and non-finite nodes.  A warp-uniform test per plane (a packed FP32x2
// product of the Re and Im values, zero if a component of a node is, or
// non-finite) selects a path that builds zero-node bits (their edges count 0:
// phase 0) and non-finite bits (their faces are dropped).  Padding holds
// (1, 1), finite with nonzero components.
//
// Staging.  Planes of the band arrive by cp.async.bulk row copies (one per row,
// issued by the lanes of warp 0) into a ring of shared-memory slots with a
// "full" mbarrier (transaction bytes) and an "empty" mbarrier (one arrival per
// warp after it has read the slot) per slot, so warps are not held in lockstep.
// A lane keeps the 17 values of plane k in registers while it reads plane
// k + 1.  Waits are bounded (about 2^32 SM cycles); a timeout sets a status
// bit that turns the reported count into QTV_COUNT_TIMEOUT.
//
// Stacked last tiles.  A CTA's plane step costs about the same whatever the
// tile width (the sweep is latency-bound per CTA), so a last tile of a row
// that is narrower than one warp (16 columns at nx = 512) would cost a whole
// CTA unit per band and plane.  Instead the last tiles of NW consecutive
// bands share one unit: warp v takes band band0 + v as if it were warp 0 of
// that band's last tile, in its own 32-column strip of the slot rows.  Strip
// rows are too short for bulk copies to pay (each bulk copy has a fixed cost),
// so each warp fills its own strip with 16-byte cp.async copies, one commit
// group per plane, and the warps of a stacked unit run independently.
//
// Output and finalize.  Each lane with faces in a plane writes one 16-byte
// record (L and H words of the three orientations, 16 rows each, and the lane)
// into the fixed slot block of its (plane, band, tile, warp) step (32 records,
// one per lane); the step's table entry (ballot of the lanes with records,
// face count) is held by lane t % 32 and 32 consecutive planes' entries are
// stored at once; face totals per (plane, band) segment accumulate in shared
// memory for the CTA's run of planes and are added to the segment totals at
// its end.  The scan of the nibble sweep gives segment offsets, and the expand
// pass (expand_bits.cu) writes faces in ascending face-id order (row, then x,
// then orientation).
#include <algorithm>

#include "bits_layout.cuh"
#include "qtv_internal.cuh"
#include "sweep_common.cuh"

namespace qtv {
namespace {

using namespace sweep;
using namespace bits;

constexpr int kMaxRun = 256;      // planes per run (bounds the shared face totals)
constexpr int kTail = 8;          // padding elements after the ring (stacked strips)

// acc' = (acc << 1) | sign bit of x
__device__ __forceinline__ uint32_t push1(uint32_t acc, float x) {
  return __funnelshift_l(__float_as_uint(x), acc, 1);
}

struct Edge {
  uint32_t P, N, Z;
};

// edges a -> b from the sign words of a and b, the cross-sign word n, and the
// edges E that touch a zero node (contribute 0)
__device__ __forceinline__ Edge edge_words(uint32_t sa, uint32_t sb, uint32_t n, uint32_t E) {
  Edge e;
  e.P = ~sa & sb & ~n & ~E;
  e.N = sa & ~sb & n & ~E;
  e.Z = e.P | e.N;
  return e;
}

__device__ __forceinline__ Edge edge_words(uint32_t sa, uint32_t sb, uint32_t n) {
  Edge e;
  e.P = ~sa & sb & ~n;
  e.N = sa & ~sb & n;
  e.Z = e.P | e.N;
  return e;
}

// packed product of the (Re, Im) values of a plane: zero when a component of
// a node is zero, non-finite when a node is (or on FP32 under- or overflow,
// which merely selects the masking path)
__device__ __forceinline__ unsigned long long prod_step(unsigned long long acc, float2 v) {
  return mul_f32x2(acc, (unsigned long long)__float_as_uint(v.x) |
                            ((unsigned long long)__float_as_uint(v.y) << 32));
}
__device__ __forceinline__ bool prod_special(unsigned long long acc) {
  const float px = fabsf(__uint_as_float((uint32_t)acc)), py = fabsf(__uint_as_float((uint32_t)(acc >> 32)));
  return !(px > 0.f && px <= 3.402823466e38f && py > 0.f && py <= 3.402823466e38f);
}
constexpr unsigned long long kProdOne = 0x3f8000003f800000ull;  // (1.f, 1.f)

// sum mod 4 of four terms given as (low, high) bit words
__device__ __forceinline__ void mod4(uint32_t a, uint32_t a1, uint32_t b, uint32_t b1, uint32_t c,
                                     uint32_t c1, uint32_t d, uint32_t d1, uint32_t& L,
                                     uint32_t& H) {
  const uint32_t x = a ^ b, y = c ^ d;
  L = x ^ y;
  const uint32_t e2 = (a & b) ^ (c & d) ^ (x & y);
  H = a1 ^ b1 ^ c1 ^ d1 ^ e2;
}

__device__ __forceinline__ uint32_t zero_bit(float2 v) {
  return ((__float_as_uint(v.x) | __float_as_uint(v.y)) << 1) == 0u ? 1u : 0u;
}
__device__ __forceinline__ uint32_t bad_bit(float2 v) {
  return (finite_f(v.x) && finite_f(v.y)) ? 0u : 1u;
}

template <int NW, int MINB, int STAGES>
__global__ void __launch_bounds__(NW * 32, MINB) sweep_bits_kernel(const __grid_constant__ BulkParams a) {
  extern __shared__ __align__(128) unsigned char dsm[];
  pdl_trigger();  // the segment scan may queue behind this grid's blocks
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int w = tid >> 5;
  constexpr int W2 = BL * NW + 2;  // row pitch of a slot, in elements
  float2* ring = reinterpret_cast<float2*>(dsm);
  uint64_t* full =
      reinterpret_cast<uint64_t*>(dsm + ((size_t)STAGES * BRH * W2 + kTail) * sizeof(float2));
  uint64_t* empty = full + STAGES;
  unsigned int* s_faces = reinterpret_cast<unsigned int*>(empty + STAGES);  // [kMaxRun]
  // per warp: first node of its band's rows in the tile
  const float2** s_src = reinterpret_cast<const float2**>(s_faces + kMaxRun);
  const int xl = BL * w + lane;  // tile-local column of this lane

  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1u);
      mbar_init(&empty[s], (uint32_t)NW);
    }
    fence_mbar_init();
  }
  __syncthreads();

  uint32_t fill = 0, use = 0;  // planes issued (warp 0) / consumed, counted over the whole CTA
  bool timeout = false;
  int valid_w = W2, valid_r = BRH;  // padding bookkeeping, as in the nibble sweep
  bool stk_padded = false;          // the ring holds padding outside the stacked strips
  // padding past the last slot: the lanes of the last stacked strip read up to
  // 32 NW - W2 elements beyond a slot row
  for (int i = tid; i < kTail; i += blockDim.x)
    ring[(size_t)STAGES * BRH * W2 + i] = make_float2(1.f, 1.f);

  const long long U = a.units;
  long long u = U * blockIdx.x / gridDim.x;
  const long long uend = U * (blockIdx.x + 1) / gridDim.x;

  while (u < uend) {
    int si = 0;
    while (si + 1 < a.nsnap && a.s[si + 1].unit0 <= u) ++si;
    const SnapDesc& sd = a.s[si];
    const int nx = sd.nx, ny = sd.ny, nz = sd.nz, ntx = sd.ntx;
    // columns: (band, tile) of the tiles before the last, then (with
    // stacking) groups of NW bands whose narrow last tiles share a CTA, one
    // band per warp, else (band, tile) of every tile
    const int ntn = sd.nstk ? ntx - 1 : ntx;
    const long long nnorm = (long long)sd.nbands * ntn;
    long long col;
    int kb, kblk;
    unit_pos(u - sd.unit0, nnorm + sd.nstk, nz, sd.hblock, col, kb, kblk);
    const bool stk = col >= nnorm;
    const int band0 = stk ? (int)(col - nnorm) * NW : 0;  // first band of a stacked group
    const int band = stk ? band0 + w : (int)(col / ntn);  // this warp's band
    const int tile = stk ? ntx - 1 : (int)(col % ntn);
    const bool wok = band < sd.nbands;  // a stacked group may hold fewer than NW bands
    const int ke = (int)min(min((long long)kblk, (long long)kb + (uend - u)), (long long)kb + kMaxRun);
    u += ke - kb;
    const int j0 = band * BR;
    const int nrows = wok ? min(BRH, ny - j0) : 0;
    const int klast = min(ke, nz - 1);
    const int nplanes = klast - kb + 1;
    const int nsteps = ke - kb;
    const int xt0 = tile * sd.st;
    const bool last_tile = tile == ntx - 1;
    const int tw = last_tile ? nx - xt0 : sd.st + 2;
    const int own_end = last_tile ? tw : sd.st;
    const uint32_t row_bytes = (uint32_t)tw * 8u;
    // first node of this warp's band (stacked) or the CTA's band in the tile,
    // kept in shared memory (read once per plane by the copying lanes)
    __syncwarp();
    if (lane == 0) s_src[w] = sd.psi + (size_t)(wok ? band * BR : 0) * nx + xt0;
    __syncwarp();
    // tile-local column of this lane, and its column in a slot (a stacked
    // group puts band band0 + v at slot columns 32 v ..)
    const int xs = stk ? lane : xl;
    const int xc = stk ? 32 * w + lane : xl;

    if (stk) {
      if (!stk_padded) {
        for (int idx = tid; idx < STAGES * BRH * W2; idx += blockDim.x)
          ring[idx] = make_float2(1.f, 1.f);
        fence_proxy_async();
        __syncthreads();
        stk_padded = true;
      }
      valid_w = W2;  // a later unstacked run re-pads what it needs
      valid_r = BRH;
    } else {
      stk_padded = false;
      if (tw < valid_w || nrows < valid_r) {
        const int cw = valid_w - tw;
        if (cw > 0)
          for (int idx = tid; idx < STAGES * BRH * cw; idx += blockDim.x)
            ring[(size_t)(idx / cw) * W2 + tw + idx % cw] = make_float2(1.f, 1.f);
        const int rr = valid_r - nrows;
        if (rr > 0) {
          const int per = rr * W2;
          for (int idx = tid; idx < STAGES * per; idx += blockDim.x) {
            const int sl = idx / per, rem = idx % per;
            ring[((size_t)sl * BRH + nrows + rem / W2) * W2 + rem % W2] = make_float2(1.f, 1.f);
          }
        }
        fence_proxy_async();
        __syncthreads();
      }
      valid_w = tw;
      valid_r = nrows;
    }
    for (int i = tid; i < nsteps; i += blockDim.x) s_faces[i] = 0u;
    __syncthreads();

    // warp 0: plane m into the next slot once every warp has released it
    auto produce = [&](int m) {
      const uint32_t q = fill;
      const int sl = (int)(q % STAGES);
      if (q >= (uint32_t)STAGES && !mbar_wait(&empty[sl], ((q / STAGES) - 1u) & 1u)) timeout = true;
      if (lane == 0) {
        fence_proxy_async();
        mbar_arrive_expect_tx(&full[sl], row_bytes * (uint32_t)nrows);
      }
      __syncwarp();
      if (lane < nrows)
        bulk_g2s(ring + ((size_t)sl * BRH + lane) * W2,
                 s_src[0] + (size_t)m * ((size_t)nx * ny) + (size_t)lane * nx, row_bytes, &full[sl]);
      ++fill;
    };
    // Stacked group: each warp fills and reads only its own strip, so the
    // warps run independently, with 16-byte cp.async copies (a strip row is
    // too short for a bulk copy to pay) in one commit group per plane.  Lane
    // chunks: (row, 16-byte column pair) = (r0, c0) + i (dr, dc), row-major.
    // (plane m of a run sits in slot (m - kb) % STAGES)
    auto sfill = [&](int m) {
      if (m <= klast && wok) {
        const int nch = (int)(row_bytes >> 4);  // 16-byte chunks of a strip row (tw is even)
        const float2* src = s_src[w] + (size_t)m * ((size_t)nx * ny);
        float2* dst = ring + (size_t)((m - kb) % STAGES) * BRH * W2 + 32 * w;
        const int dr = 32 / nch, dc = 32 - dr * nch;
        int r = lane / nch, c = lane - (lane / nch) * nch;
        while (r < nrows) {
          cp_async16(dst + r * W2 + 2 * c, src + (size_t)r * nx + 2 * c);
          r += dr;
          c += dc;
          if (c >= nch) {
            c -= nch;
            ++r;
          }
        }
      }
      cp_async_commit();
    };
    auto acquire = [&](int m) -> const float2* {
      if (stk) {
        cp_async_wait<STAGES - 1>();
        __syncwarp();
        return ring + (size_t)((m - kb) % STAGES) * BRH * W2;
      }
      const int sl = (int)(use % STAGES);
      if (!mbar_wait(&full[sl], (use / STAGES) & 1u)) timeout = true;
      return ring + (size_t)sl * BRH * W2;
    };
    // done with plane m (a stacked warp refills its strip's slot at once)
    auto release = [&](int m) {
      __syncwarp();
      if (stk) {
        sfill(m + STAGES);
        return;
      }
      if (lane == 0) mbar_arrive(&empty[use % STAGES]);
      ++use;
    };

    // masks of the faces this lane owns (rows 0..15 of the band)
    const int avail = wok ? ny - j0 : 0;  // rows of the band that exist
    const uint32_t rv = avail >= BR ? kRows16 : ((1u << avail) - 1u);
    const uint32_t rv1 = avail - 1 >= BR ? kRows16 : (avail > 1 ? ((1u << (avail - 1)) - 1u) : 0u);
    const bool own = wok && lane < BL && xs < own_end;
    const uint32_t m_xy = (own && xs + 1 < tw) ? rv1 : 0u;
    const uint32_t m_yz = (own && xs < tw) ? rv1 : 0u;
    const uint32_t m_zx = (own && xs + 1 < tw) ? rv : 0u;
    // table entries of this (band, tile, warp): one per plane, contiguous in k;
    // records of entry e in the fixed slots 32 e .. 32 e + 31 (one per lane).
    // A stacked warp is warp 0 of its band's last tile; that tile's other
    // warps own no columns and get empty entries.
    const unsigned long long ebase =
        (unsigned long long)sd.tab0 +
        (((unsigned long long)band * ntx + tile) * NW + (stk ? 0 : w)) * nz;
    uint2* const table = reinterpret_cast<uint2*>(a.table);
    uint4* const recs = reinterpret_cast<uint4*>(a.recs);
    uint2 tent = make_uint2(0u, 0u);  // entry of step t held by lane t % 32

    if (stk) {
      for (int i = 0; i < STAGES; ++i) sfill(kb + i);
    } else if (w == 0) {
      for (int i = 0; i < min(STAGES, nplanes); ++i) produce(kb + i);
    }

    // ---- prologue: plane kb (values into vA)
    float2 vA[BRH], vB[BRH];
    uint32_t S0, S0n, ZB0 = 0, ZB0n = 0, BB0 = 0, BB0n = 0;
    Edge X0, Y0, Y0n;
    bool bad0;
    {
      const float2* sp = acquire(kb);
      uint32_t SX = 0, SY = 0;
      unsigned long long prod = kProdOne;
      S0 = 0;
#pragma unroll
      for (int r = BRH - 1; r >= 0; --r) {
        const float2 v = sp[r * W2 + xc];
        const float2 nb = sp[r * W2 + xc + 1];
        S0 = push1(S0, v.y);
        SX = push1(SX, cross_f(v.x, v.y, nb.x, nb.y));
        if (r < BR) SY = push1(SY, cross_f(v.x, v.y, vA[r + 1].x, vA[r + 1].y));
        prod = prod_step(prod, v);
        vA[r] = v;
      }
      release(kb);
      if (w == 0 && !stk && kb + STAGES <= klast) produce(kb + STAGES);
      bad0 = __any_sync(0xffffffffu, prod_special(prod));
      if (bad0) {
#pragma unroll
        for (int r = 0; r < BRH; ++r) {
          ZB0 |= zero_bit(vA[r]) << r;
          BB0 |= bad_bit(vA[r]) << r;
        }
      }
      S0n = __shfl_down_sync(0xffffffffu, S0, 1);
      const uint32_t SYn = __shfl_down_sync(0xffffffffu, SY, 1);
      ZB0n = __shfl_down_sync(0xffffffffu, ZB0, 1);
      BB0n = __shfl_down_sync(0xffffffffu, BB0, 1);
      X0 = edge_words(S0, S0n, SX, ZB0 | ZB0n);
      Y0 = edge_words(S0, S0 >> 1, SY, ZB0 | (ZB0 >> 1));
      Y0n = edge_words(S0n, S0n >> 1, SYn, ZB0n | (ZB0n >> 1));
    }

    // one z step: plane k = kb + t in V0 (values) and the plane-k words,
    // plane k + 1 read into V1
    auto step = [&](float2(&V0)[BRH], float2(&V1)[BRH], int t) {
      const int k = kb + t;
      const bool has_up = k + 1 < nz;
      uint32_t Lxy, Hxy, Lyz = 0, Hyz = 0, Lzx = 0, Hzx = 0;
      // xy faces of plane k: +x(r), +y_{x+1}(r), -x(r+1), -y_x(r)
      mod4(X0.Z, X0.N, Y0n.Z, Y0n.N, X0.Z >> 1, X0.P >> 1, Y0.Z, Y0.P, Lxy, Hxy);
      uint32_t Mxy = (Lxy | Hxy) & m_xy, Myz = 0, Mzx = 0;
      uint32_t S1 = 0, S1n = 0, ZB1 = 0, ZB1n = 0, BB1 = 0, BB1n = 0;
      Edge X1{0, 0, 0}, Y1{0, 0, 0}, Y1n{0, 0, 0};
      bool bad1 = false;
      if (has_up) {
        const float2* sp = acquire(k + 1);
        uint32_t SX = 0, SY = 0, SZ = 0;
        unsigned long long prod = kProdOne;
#pragma unroll
        for (int r = BRH - 1; r >= 0; --r) {
          const float2 v = sp[r * W2 + xc];
          const float2 nb = sp[r * W2 + xc + 1];
          S1 = push1(S1, v.y);
          SX = push1(SX, cross_f(v.x, v.y, nb.x, nb.y));
          SZ = push1(SZ, cross_f(V0[r].x, V0[r].y, v.x, v.y));
          if (r < BR) SY = push1(SY, cross_f(v.x, v.y, V1[r + 1].x, V1[r + 1].y));
          prod = prod_step(prod, v);
          V1[r] = v;
        }
        release(k + 1);
        if (w == 0 && !stk && k + 1 + STAGES <= klast) produce(k + 1 + STAGES);
        bad1 = __any_sync(0xffffffffu, prod_special(prod));
        S1n = __shfl_down_sync(0xffffffffu, S1, 1);
        const uint32_t SYn = __shfl_down_sync(0xffffffffu, SY, 1);
        const uint32_t SZn = __shfl_down_sync(0xffffffffu, SZ, 1);
        Edge Zk, Zkn;
        if (bad0 || bad1) {
          if (bad1) {
#pragma unroll
            for (int r = 0; r < BRH; ++r) {
              ZB1 |= zero_bit(V1[r]) << r;
              BB1 |= bad_bit(V1[r]) << r;
            }
          }
          ZB1n = __shfl_down_sync(0xffffffffu, ZB1, 1);
          BB1n = __shfl_down_sync(0xffffffffu, BB1, 1);
          X1 = edge_words(S1, S1n, SX, ZB1 | ZB1n);
          Y1 = edge_words(S1, S1 >> 1, SY, ZB1 | (ZB1 >> 1));
          Y1n = edge_words(S1n, S1n >> 1, SYn, ZB1n | (ZB1n >> 1));
          Zk = edge_words(S0, S1, SZ, ZB0 | ZB1);
          Zkn = edge_words(S0n, S1n, SZn, ZB0n | ZB1n);
        } else {
          X1 = edge_words(S1, S1n, SX);
          Y1 = edge_words(S1, S1 >> 1, SY);
          Y1n = edge_words(S1n, S1n >> 1, SYn);
          Zk = edge_words(S0, S1, SZ);
          Zkn = edge_words(S0n, S1n, SZn);
        }
        // yz faces of plane k: +y_k(r), +z(r+1), -y_{k+1}(r), -z(r)
        mod4(Y0.Z, Y0.N, Zk.Z >> 1, Zk.N >> 1, Y1.Z, Y1.P, Zk.Z, Zk.P, Lyz, Hyz);
        // zx faces of plane k: +z_x(r), +x_{k+1}(r), -z_{x+1}(r), -x_k(r)
        mod4(Zk.Z, Zk.N, X1.Z, X1.N, Zkn.Z, Zkn.P, X0.Z, X0.P, Lzx, Hzx);
        Myz = (Lyz | Hyz) & m_yz;
        Mzx = (Lzx | Hzx) & m_zx;
      }
      if (bad0 || bad1) {  // drop faces that touch a non-finite node
        Mxy &= ~(BB0 | BB0n | (BB0 >> 1) | (BB0n >> 1));
        Myz &= ~(BB0 | (BB0 >> 1) | BB1 | (BB1 >> 1));
        Mzx &= ~(BB0 | BB0n | BB1 | BB1n);
      }
      Lxy &= Mxy;
      Hxy &= Mxy;
      Lyz &= Myz;
      Hyz &= Myz;
      Lzx &= Mzx;
      Hzx &= Mzx;
      const uint32_t cnt = __popc(Mxy) + __popc(Myz) + __popc(Mzx);
      const bool anyf = cnt != 0u;

      // ---- output: records in the fixed slots of this warp step, the
      // table entry (lane mask, faces) held by lane t % 32 and stored for 32
      // steps at once, the face total added to the CTA's count of plane k
      const uint32_t faces_w = __reduce_add_sync(0xffffffffu, cnt);
      const uint32_t bal = __ballot_sync(0xffffffffu, anyf);
      const unsigned long long e = ebase + (unsigned long long)k;
      if (anyf && e * 32ull + lane < a.recs_cap)
        recs[e * 32ull + lane] =
            make_uint4(Lxy | (Hxy << 16), Lyz | (Hyz << 16), Lzx | (Hzx << 16), (uint32_t)lane);
      if (lane == (t & 31)) tent = make_uint2(bal, faces_w);
      if (((t & 31) == 31 || t == nsteps - 1) && wok) {
        if (lane <= (t & 31)) {
          const unsigned long long ei = ebase + (unsigned long long)(kb + (t & ~31) + lane);
          table[ei] = tent;
          if (stk)
            for (int v = 1; v < NW; ++v) table[ei + (unsigned long long)v * nz] = make_uint2(0u, 0u);
        }
      }
      if (lane == 0 && faces_w) {
        if (stk) atomicAdd(&a.segf[sd.seg0 + (size_t)k * sd.nbands + band], faces_w);
        else atomicAdd(&s_faces[t], faces_w);
      }
      // plane k + 1 becomes plane k
      S0 = S1;
      S0n = S1n;
      ZB0 = ZB1;
      ZB0n = ZB1n;
      BB0 = BB1;
      BB0n = BB1n;
      X0 = X1;
      Y0 = Y1;
      Y0n = Y1n;
      bad0 = bad1;
    };

    for (int t = 0; t < nsteps; t += 2) {
      step(vA, vB, t);
      if (t + 1 < nsteps) step(vB, vA, t + 1);
    }
    if (stk) cp_async_wait<0>();  // only empty groups are left
    __syncthreads();
    // face totals of the run's planes into the (plane, band) segments
    for (int i = tid; i < nsteps; i += blockDim.x)
      if (s_faces[i]) atomicAdd(&a.segf[sd.seg0 + (size_t)(kb + i) * sd.nbands + band], s_faces[i]);
    __syncthreads();
  }
  if (timeout) atomicOr(reinterpret_cast<unsigned int*>(a.counters + 1), 1u);
}

using BitsFn = void (*)(BulkParams);

template <int STAGES>
BitsFn bits_fn_stages(int nw) {
  if (nw <= 2) return sweep_bits_kernel<2, 8, STAGES>;
  if (nw <= 4) return sweep_bits_kernel<4, 4, STAGES>;
  return sweep_bits_kernel<8, 2, STAGES>;
}

BitsFn bits_fn(int nw, int stages) {
  return stages <= 2 ? bits_fn_stages<2>(nw) : bits_fn_stages<3>(nw);
}

int bits_fn_index(int nw, int stages) {
  return (nw <= 2 ? 0 : (nw <= 4 ? 1 : 2)) + (stages <= 2 ? 0 : 3);
}

}  // namespace

size_t bits_smem_bytes(int nw, int stages) {
  return ((size_t)stages * BRH * (BL * nw + 2) + kTail) * sizeof(float2) +
         2 * stages * sizeof(uint64_t) + kMaxRun * sizeof(unsigned int) +
         (size_t)nw * sizeof(const float2*);
}

int bits_variant_occupancy(int nw, int stages, int* ctas_per_sm, size_t* smem) {
  static bool attr_set[6] = {false, false, false, false, false, false};
  if (nw != 2 && nw != 4 && nw != 8)
    return set_error(QTV_ERR_ARG, "bit-sliced sweep: %d warps per tile (2, 4 or 8)", nw);
  const int which = bits_fn_index(nw, stages);
  BitsFn fn = bits_fn(nw, stages);
  if (!attr_set[which]) {
    cudaError_t e =
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e != cudaSuccess) return check_cuda(e, "cudaFuncSetAttribute(sweep_bits)");
    attr_set[which] = true;
  }
  *smem = bits_smem_bytes(nw, stages);
  int bps = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, nw * 32, *smem);
  if (e != cudaSuccess) return check_cuda(e, "occupancy(sweep_bits)");
  if (bps < 1) return set_error(QTV_ERR_ARG, "sweep_bits: no resident CTA with %d warps", nw);
  *ctas_per_sm = bps;
  return QTV_OK;
}

void bits_sweep_launch(const BulkParams& p, int grid, int nw, int stages, size_t smem,
                       cudaStream_t st) {
  bits_fn(nw, stages)<<<grid, nw * 32, smem, st>>>(p);
}


}  // namespace qtv
