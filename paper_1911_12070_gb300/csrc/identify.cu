// identify.cu -- circulation-based vortex identification (Sec. 2.2.2, Eq. 5)
// on every plaquette of a 3-D complex64 grid, with deterministic stream
// compaction of the pierced plaquettes into ascending face-id order.
//
// Arithmetic.  For a directed grid edge a -> b the wrapped phase difference
// d = arg(psi_b conj(psi_a)) in (-pi, pi] differs from theta_b - theta_a
// (theta = arg psi in (-pi, pi]) by 2 pi r with an integer r in {-1, 0, 1}.
// Summed around a closed loop the theta terms telescope, so the circulation of
// Eq. 5 on a plaquette is exactly 2 pi times the sum of its four r values.  r
// is decided without any transcendental function:
//   s(z) = (Im z < 0)             (lower half plane: theta in (-pi, 0))
//   r = +1  if s_a = 0, s_b = 1 and cross(a, b) > 0   (crosses the cut
//                                                     counter-clockwise)
//   r = -1  if s_a = 1, s_b = 0 and cross(a, b) < 0
//   r =  0  otherwise,
// with cross(a, b) = Re a Im b - Im a Re b = |a||b| sin d.  The sign of cross
// is evaluated exactly in FP32 by Kahan's 2x2 determinant (an error-free
// product split with one FMA; its relative error is below 2 ulp, so its sign
// is always right; Jeannerod, Louvet & Muller 2013), which makes r exact for
// every |d| < pi.  A node with psi == 0 gets s = 0 and cross = 0 on its edges,
// i.e. phase 0.
//
// Layout.  A CTA owns a band of kRows = 7 rows (y) across the full x extent
// and marches z over a chunk of planes.  Thread (warp w, lane l) owns the two
// nodes x0 = 64 w + 2 l, x0 + 1 of every band row, plus the band's halo row,
// in registers (one 16-byte load per row and plane).  The x-neighbour column
// x0 + 2 comes from lane l + 1 by warp shuffle; lane 31 gets it from warp
// w + 1 through shared memory.  The r values of each (edge direction, column)
// are packed one 4-bit field per row (value + 1), so the four-term plaquette
// sums of all rows of a column are three integer instructions.
//
// Compaction.  Faces of one (plane, band) segment are produced in face-id
// order (rows, then x, then orientation).  Per-row counts are scanned inside
// each warp, then across warps, then a segment is reserved in a staging buffer
// with one atomic; this is software-pipelined over two planes so that every
// plane needs a single __syncthreads.  A finalize pass scans the segment counts
// in (plane, band) order, which is ascending face-id order, and scatters the
// staged records to their final positions.
#include <cstdio>

#include "qtv_internal.cuh"

namespace qtv {
namespace {

constexpr int R = kRows;    // owned rows
constexpr int RH = R + 1;   // rows incl. halo (one 4-bit field each)
constexpr uint32_t kOnes = 0x11111111u;
constexpr uint32_t kFours = 0x44444444u;
constexpr uint32_t kOwned = 0x0FFFFFFFu;  // fields of rows 0..6

// value + 1 of the branch-crossing integer of edge a -> b (see header comment)
__device__ __forceinline__ uint32_t edge_term(float ar, float ai, float br, float bi) {
  const float p = ai * br;
  const float e = fmaf(ai, br, -p);  // ai*br - p, exact
  const float c = fmaf(ar, bi, -p);  // RN(ar*bi - p)
  const bool sa = ai < 0.f, sb = bi < 0.f;
  const uint32_t plus = (!sa && sb && c > e) ? 1u : 0u;
  const uint32_t minus = (sa && !sb && c < e) ? 1u : 0u;
  return 1u + plus - minus;
}

// nonzero 4-bit fields -> bit 0 of that field
__device__ __forceinline__ uint32_t nz_fields(uint32_t d) {
  uint32_t t = d | (d >> 2);
  t = t | (t >> 1);
  return t & kOnes;
}

__device__ __forceinline__ bool finite_f(float v) { return fabsf(v) <= 3.402823466e38f; }

struct Pending {
  uint32_t d[6];     // per slot: (W+4) ^ 4 per row field, 0 where no face
  uint32_t ex_e;     // warp-exclusive per-row counts, rows 0,2,4,6 (bytes)
  uint32_t ex_o;     // rows 1,3,5 (bytes)
};

struct SmemSweep {
  float2 xpsi[2][kMaxWarpsX][RH];  // column x0 of each warp, plane k+1
  uint2 xbits[2][kMaxWarpsX];      // {rz_k, ry_k+1} fields of column x0
  uint2 tot[2][kMaxWarpsX];        // warp row totals (bytes, even / odd rows)
  uint32_t offs[2][kMaxWarpsX][R]; // CTA offset of (row, warp) within segment
  uint32_t base[2];                // staging base of the segment
};

template <bool VEC>
__device__ __forceinline__ float4 load_pair(const float2* __restrict__ psi, long long idx, bool ok0,
                                            bool ok1) {
  if (VEC) {
    if (ok0) return __ldg(reinterpret_cast<const float4*>(psi + idx));
    return make_float4(0.f, 0.f, 0.f, 0.f);
  } else {
    float2 a = ok0 ? __ldg(psi + idx) : make_float2(0.f, 0.f);
    float2 b = ok1 ? __ldg(psi + idx + 1) : make_float2(0.f, 0.f);
    return make_float4(a.x, a.y, b.x, b.y);
  }
}

// Per-node non-finite bits of column p (0: x0, 1: x0+1) over the RH rows.
__device__ __forceinline__ uint32_t bad_bits_col(const float4* v, int p) {
  uint32_t b = 0;
#pragma unroll
  for (int r = 0; r < RH; ++r) {
    float re = p ? v[r].z : v[r].x, im = p ? v[r].w : v[r].y;
    if (!(finite_f(re) && finite_f(im))) b |= 1u << (4 * r);
  }
  return b;
}

template <bool VEC, int MAXT>
__global__ void __launch_bounds__(MAXT) sweep_kernel(SweepArgs a) {
  __shared__ SmemSweep sm;
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const int NW = blockDim.x >> 5;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int x0 = 64 * w + 2 * lane;
  const bool c0 = x0 < nx, c1 = x0 + 1 < nx, c2 = x0 + 2 < nx;
  const long long plane = (long long)nx * ny;

  for (int item = blockIdx.x; item < a.nitems; item += gridDim.x) {
    const int band = item % a.nbands;
    const int zc = item / a.nbands;
    const int j0 = band * R;
    const int kb = zc * a.kchunk;
    const int ke = min(nz, kb + a.kchunk);
    const int nsteps = ke - kb;

    // row validity (4-bit field per row, bit 0)
    uint32_t rowv = 0, rowv1 = 0;  // row exists / row and row+1 exist
#pragma unroll
    for (int r = 0; r < RH; ++r) {
      if (j0 + r < ny) rowv |= 1u << (4 * r);
      if (j0 + r + 1 < ny && r < R) rowv1 |= 1u << (4 * r);
    }
    rowv &= kOwned;
    // existence of each slot (p, o) on planes with k+1 < nz, and on the last plane
    const uint32_t ex_xy0 = c1 ? rowv1 : 0u, ex_xy1 = c2 ? rowv1 : 0u;
    const uint32_t ex_yz0 = c0 ? rowv1 : 0u, ex_yz1 = c1 ? rowv1 : 0u;
    const uint32_t ex_zx0 = c1 ? rowv : 0u, ex_zx1 = c2 ? rowv : 0u;

    auto row_index = [&](int r, int k) -> long long {
      return (long long)k * plane + (long long)(j0 + r) * nx + x0;
    };

    // ---- prologue: plane kb
    float4 cur[RH];
#pragma unroll
    for (int r = 0; r < RH; ++r) {
      const bool rok = j0 + r < ny;
      cur[r] = load_pair<VEC>(a.psi, row_index(r, kb), rok && c0, rok && c1);
    }
    uint32_t RX0 = 0, RY0 = 0, RY1 = 0;
#pragma unroll
    for (int r = 0; r < RH; ++r) {
      RX0 |= edge_term(cur[r].x, cur[r].y, cur[r].z, cur[r].w) << (4 * r);
      if (r < R) {
        RY0 |= edge_term(cur[r].x, cur[r].y, cur[r + 1].x, cur[r + 1].y) << (4 * r);
        RY1 |= edge_term(cur[r].z, cur[r].w, cur[r + 1].z, cur[r + 1].w) << (4 * r);
      }
    }
    if (lane == 0) {
#pragma unroll
      for (int r = 0; r < RH; ++r) sm.xpsi[1][w][r] = make_float2(cur[r].x, cur[r].y);
      sm.xbits[1][w] = make_uint2(0u, RY0);
    }
    bool bad_k;  // warp-uniform: some node of plane k (own or neighbour column) non-finite
    {
      float acc = 0.f;
#pragma unroll
      for (int r = 0; r < RH; ++r)
        acc += fabsf(cur[r].x) + fabsf(cur[r].y) + fabsf(cur[r].z) + fabsf(cur[r].w);
      bad_k = __any_sync(0xffffffffu, !(acc <= 3.402823466e38f));
    }
    __syncthreads();
    uint32_t RX1 = 0, RYN = 0;
    {
      const uint32_t ryn_sh = __shfl_down_sync(0xffffffffu, RY0, 1);
      float2 nb[RH];
#pragma unroll
      for (int r = 0; r < RH; ++r) {
        nb[r].x = __shfl_down_sync(0xffffffffu, cur[r].x, 1);
        nb[r].y = __shfl_down_sync(0xffffffffu, cur[r].y, 1);
      }
      RYN = ryn_sh;
      if (lane == 31) {
        if (w + 1 < NW) {
#pragma unroll
          for (int r = 0; r < RH; ++r) nb[r] = sm.xpsi[1][w + 1][r];
          RYN = sm.xbits[1][w + 1].y;
        } else {
#pragma unroll
          for (int r = 0; r < RH; ++r) nb[r] = make_float2(0.f, 0.f);
          RYN = 0x11111111u;
        }
      }
      float accn = 0.f;
#pragma unroll
      for (int r = 0; r < RH; ++r) {
        RX1 |= edge_term(cur[r].z, cur[r].w, nb[r].x, nb[r].y) << (4 * r);
        accn += fabsf(nb[r].x) + fabsf(nb[r].y);
      }
      bad_k = bad_k || __any_sync(0xffffffffu, !(accn <= 3.402823466e38f));
    }

    Pending p1{}, p2{};  // pending steps t-1 and t-2
    for (int t = 0; t < nsteps + 2; ++t) {
      const int k = kb + t;
      const bool compute = t < nsteps;
      const bool has_up = k + 1 < nz;
      float4 nxt[RH];
      uint32_t RZ0 = 0, RZ1 = 0, RX0n = 0, RY0n = 0, RY1n = 0;
      bool bad_k1 = false;
      if (compute) {
#pragma unroll
        for (int r = 0; r < RH; ++r) {
          const bool rok = has_up && j0 + r < ny;
          nxt[r] = load_pair<VEC>(a.psi, row_index(r, k + 1), rok && c0, rok && c1);
        }
        float acc0 = 0.f, acc1 = 0.f;
#pragma unroll
        for (int r = 0; r < RH; ++r) {
          RZ0 |= edge_term(cur[r].x, cur[r].y, nxt[r].x, nxt[r].y) << (4 * r);
          RZ1 |= edge_term(cur[r].z, cur[r].w, nxt[r].z, nxt[r].w) << (4 * r);
          RX0n |= edge_term(nxt[r].x, nxt[r].y, nxt[r].z, nxt[r].w) << (4 * r);
          if (r < R) {
            RY0n |= edge_term(nxt[r].x, nxt[r].y, nxt[r + 1].x, nxt[r + 1].y) << (4 * r);
            RY1n |= edge_term(nxt[r].z, nxt[r].w, nxt[r + 1].z, nxt[r + 1].w) << (4 * r);
          }
          acc0 += fabsf(nxt[r].x) + fabsf(nxt[r].y);
          acc1 += fabsf(nxt[r].z) + fabsf(nxt[r].w);
        }
        bad_k1 = !(acc0 + acc1 <= 3.402823466e38f);
        if (lane == 0) {
#pragma unroll
          for (int r = 0; r < RH; ++r) sm.xpsi[t & 1][w][r] = make_float2(nxt[r].x, nxt[r].y);
          sm.xbits[t & 1][w] = make_uint2(RZ0, RY0n);
        }
      }
      __syncthreads();

      // ---- CTA offsets of step t-1 (warp 0), segment reservation (thread 0)
      if (t >= 1 && t - 1 < nsteps && w == 0) {
        const int tp = (t - 1) & 1;
        uint2 tw = lane < NW ? sm.tot[tp][lane] : make_uint2(0u, 0u);
        // 16-bit fields: A0 = rows {0,2}, A1 = {4,6}, B0 = {1,3}, B1 = {5,7}
        uint32_t A0 = __byte_perm(tw.x, 0u, 0x4140), A1 = __byte_perm(tw.x, 0u, 0x4342);
        uint32_t B0 = __byte_perm(tw.y, 0u, 0x4140), B1 = __byte_perm(tw.y, 0u, 0x4342);
        const uint32_t oA0 = A0, oA1 = A1, oB0 = B0, oB1 = B1;
#pragma unroll
        for (int s = 1; s < 32; s <<= 1) {
          uint32_t u0 = __shfl_up_sync(0xffffffffu, A0, s), u1 = __shfl_up_sync(0xffffffffu, A1, s);
          uint32_t u2 = __shfl_up_sync(0xffffffffu, B0, s), u3 = __shfl_up_sync(0xffffffffu, B1, s);
          if (lane >= s) { A0 += u0; A1 += u1; B0 += u2; B1 += u3; }
        }
        const uint32_t T0 = __shfl_sync(0xffffffffu, A0, 31), T1 = __shfl_sync(0xffffffffu, A1, 31);
        const uint32_t U0 = __shfl_sync(0xffffffffu, B0, 31), U1 = __shfl_sync(0xffffffffu, B1, 31);
        const uint32_t e0 = A0 - oA0, e1 = A1 - oA1, f0 = B0 - oB0, f1 = B1 - oB1;
        uint32_t tot_r[R] = {T0 & 0xffffu, U0 & 0xffffu, T0 >> 16, U0 >> 16,
                             T1 & 0xffffu, U1 & 0xffffu, T1 >> 16};
        uint32_t ex_r[R] = {e0 & 0xffffu, f0 & 0xffffu, e0 >> 16, f0 >> 16,
                            e1 & 0xffffu, f1 & 0xffffu, e1 >> 16};
        uint32_t run = 0;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          if (lane < NW) sm.offs[tp][lane][r] = run + ex_r[r];
          run += tot_r[r];
        }
        if (lane == 0) {
          unsigned long long b = run ? atomicAdd(a.staging_top, (unsigned long long)run) : 0ull;
          sm.base[tp] = (uint32_t)b;
          const int kprev = k - 1;
          uint32_t cnt = run;
          a.seg[(long long)kprev * a.nbands + band] = make_uint2(cnt, (uint32_t)b);
          if (b + run > a.staging_cap) atomicAdd(a.staging_top + 1, 1ull);
        }
      }

      // ---- write the staged records of step t-2
      if (t >= 2) {
        const int tp = (t - 2) & 1;
        uint32_t any = 0;
#pragma unroll
        for (int s = 0; s < 6; ++s) any |= p2.d[s];
        any = nz_fields(any);
        if (any) {
          const uint32_t base = sm.base[tp];
          while (any) {
            const int f = __ffs(any) - 1;
            const int r = f >> 2;
            any &= ~(0xFu << f);
            const uint32_t exb = (r & 1) ? (p2.ex_o >> (8 * (r >> 1))) & 0xffu
                                         : (p2.ex_e >> (8 * (r >> 1))) & 0xffu;
            unsigned long long pos = (unsigned long long)base + sm.offs[tp][w][r] + exb;
#pragma unroll
            for (int s = 0; s < 6; ++s) {
              const uint32_t dv = (p2.d[s] >> f) & 0xFu;
              if (dv) {
                const int pcol = s / 3, o = s % 3;
                const int wv = (int)(dv ^ 4u) - 4;
                const uint32_t rec =
                    (((uint32_t)r * (uint32_t)nx + (uint32_t)(x0 + pcol)) << 5) |
                    ((uint32_t)o << 3) | (uint32_t)(wv + 4);
                if (pos < a.staging_cap) a.staging[pos] = rec;
                ++pos;
              }
            }
          }
        }
      }

      // ---- step t: neighbour column, plaquette windings, per-row counts
      Pending pc{};
      if (compute) {
        const int tb = t & 1;
        float2 nb[RH];
        uint32_t RZN = __shfl_down_sync(0xffffffffu, RZ0, 1);
        uint32_t RYNn = __shfl_down_sync(0xffffffffu, RY0n, 1);
#pragma unroll
        for (int r = 0; r < RH; ++r) {
          nb[r].x = __shfl_down_sync(0xffffffffu, nxt[r].x, 1);
          nb[r].y = __shfl_down_sync(0xffffffffu, nxt[r].y, 1);
        }
        if (lane == 31) {
          if (w + 1 < NW) {
#pragma unroll
            for (int r = 0; r < RH; ++r) nb[r] = sm.xpsi[tb][w + 1][r];
            const uint2 xb = sm.xbits[tb][w + 1];
            RZN = xb.x;
            RYNn = xb.y;
          } else {
#pragma unroll
            for (int r = 0; r < RH; ++r) nb[r] = make_float2(0.f, 0.f);
            RZN = 0x11111111u;
            RYNn = 0x11111111u;
          }
        }
        uint32_t RX1n = 0;
        float accn = 0.f;
#pragma unroll
        for (int r = 0; r < RH; ++r) {
          RX1n |= edge_term(nxt[r].z, nxt[r].w, nb[r].x, nb[r].y) << (4 * r);
          accn += fabsf(nb[r].x) + fabsf(nb[r].y);
        }
        bad_k1 = __any_sync(0xffffffffu, bad_k1 || !(accn <= 3.402823466e38f));

        // plaquette windings, W + 4 per 4-bit field
        uint32_t Wv[6];
        Wv[0] = RX0 + RY1 + kFours - (RX0 >> 4) - RY0;      // xy, p=0
        Wv[1] = RY0 + (RZ0 >> 4) + kFours - RY0n - RZ0;     // yz, p=0
        Wv[2] = RZ0 + RX0n + kFours - RZ1 - RX0;            // zx, p=0
        Wv[3] = RX1 + RYN + kFours - (RX1 >> 4) - RY1;      // xy, p=1
        Wv[4] = RY1 + (RZ1 >> 4) + kFours - RY1n - RZ1;     // yz, p=1
        Wv[5] = RZ1 + RX1n + kFours - RZN - RX1;            // zx, p=1
        const uint32_t exm[6] = {ex_xy0, has_up ? ex_yz0 : 0u, has_up ? ex_zx0 : 0u,
                                 ex_xy1, has_up ? ex_yz1 : 0u, has_up ? ex_zx1 : 0u};
        uint32_t keep[6];
#pragma unroll
        for (int s = 0; s < 6; ++s) keep[s] = exm[s] * 0xFu;  // field masks

        if (bad_k || bad_k1) {
          // rare path: drop faces that touch a non-finite node
          uint32_t bk0 = bad_bits_col(cur, 0), bk1 = bad_bits_col(cur, 1);
          uint32_t bu0 = bad_bits_col(nxt, 0), bu1 = bad_bits_col(nxt, 1);
          uint32_t bk2 = 0, bu2 = 0;
          if (c2) {
#pragma unroll
            for (int r = 0; r < RH; ++r) {
              if (j0 + r < ny) {
                float2 vk = __ldg(a.psi + row_index(r, k) + 2);
                if (!(finite_f(vk.x) && finite_f(vk.y))) bk2 |= 1u << (4 * r);
                if (has_up) {
                  float2 vu = __ldg(a.psi + row_index(r, k + 1) + 2);
                  if (!(finite_f(vu.x) && finite_f(vu.y))) bu2 |= 1u << (4 * r);
                }
              }
            }
          }
          const uint32_t bxy0 = bk0 | bk1 | (bk0 >> 4) | (bk1 >> 4);
          const uint32_t bxy1 = bk1 | bk2 | (bk1 >> 4) | (bk2 >> 4);
          const uint32_t byz0 = bk0 | (bk0 >> 4) | bu0 | (bu0 >> 4);
          const uint32_t byz1 = bk1 | (bk1 >> 4) | bu1 | (bu1 >> 4);
          const uint32_t bzx0 = bk0 | bk1 | bu0 | bu1;
          const uint32_t bzx1 = bk1 | bk2 | bu1 | bu2;
          const uint32_t bb[6] = {bxy0, byz0, bzx0, bxy1, byz1, bzx1};
#pragma unroll
          for (int s = 0; s < 6; ++s) keep[s] &= ~((bb[s] & kOnes) * 0xFu);
        }
        uint32_t cnt = 0;
#pragma unroll
        for (int s = 0; s < 6; ++s) {
          pc.d[s] = (Wv[s] ^ kFours) & keep[s];
          cnt += nz_fields(pc.d[s]);
        }
        // per-row counts (<= 6) -> bytes, warp inclusive scan
        uint32_t ce = cnt & 0x0F0F0F0Fu, co = (cnt >> 4) & 0x0F0F0F0Fu;
        uint32_t ie = ce, io = co;
#pragma unroll
        for (int s = 1; s < 32; s <<= 1) {
          uint32_t ue = __shfl_up_sync(0xffffffffu, ie, s), uo = __shfl_up_sync(0xffffffffu, io, s);
          if (lane >= s) { ie += ue; io += uo; }
        }
        pc.ex_e = ie - ce;
        pc.ex_o = io - co;
        if (lane == 31) sm.tot[tb][w] = make_uint2(ie, io);

        // rotate plane k+1 -> k
#pragma unroll
        for (int r = 0; r < RH; ++r) cur[r] = nxt[r];
        RX0 = RX0n;
        RX1 = RX1n;
        RY0 = RY0n;
        RY1 = RY1n;
        RYN = RYNn;
        bad_k = bad_k1;
      }
      p2 = p1;
      p1 = pc;
    }
    __syncthreads();
  }
}

// Exclusive scan of segment counts in (plane, band) order = ascending face id.
__global__ void __launch_bounds__(1024) seg_scan_kernel(const uint2* __restrict__ seg, long long nseg,
                                                        unsigned long long* __restrict__ seg_off,
                                                        uint64_t* __restrict__ count,
                                                        qtv_stats* stats, unsigned long long scanned,
                                                        const unsigned long long* status) {
  __shared__ unsigned long long warp_tot[32];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const long long per = (nseg + blockDim.x - 1) / blockDim.x;
  const long long s0 = tid * per, s1 = min(nseg, s0 + per);
  unsigned long long local = 0;
  for (long long s = s0; s < s1; ++s) local += seg[s].x;
  unsigned long long incl = local;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    unsigned long long u = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += u;
  }
  if (lane == 31) warp_tot[w] = incl;
  __syncthreads();
  if (w == 0) {
    unsigned long long v = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0ull;
    unsigned long long iv = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      unsigned long long u = __shfl_up_sync(0xffffffffu, iv, d);
      if (lane >= d) iv += u;
    }
    warp_tot[lane] = iv - v;
    if (lane == 31) {
      // a bounded wait that gave up in the sweep makes the result unusable
      *count = (*status & 0xffffffffull) ? QTV_COUNT_TIMEOUT : iv;
      if (stats) {
        stats->pierced = iv;
        stats->faces_scanned = scanned;
      }
    }
  }
  __syncthreads();
  unsigned long long run = warp_tot[w] + incl - local;
  for (long long s = s0; s < s1; ++s) {
    seg_off[s] = run;
    run += seg[s].x;
  }
}

// One warp per segment: staged records -> (face id, W) at the final offset.
__global__ void scatter_kernel(const uint2* __restrict__ seg, const unsigned long long* __restrict__ seg_off,
                               long long nseg, int nbands, int nx, int ny,
                               const uint32_t* __restrict__ staging, unsigned long long staging_cap,
                               uint64_t* __restrict__ face_ids, int8_t* __restrict__ winding,
                               unsigned long long capacity) {
  const int lane = threadIdx.x & 31;
  const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long s = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < nseg; s += warps) {
    const uint2 sg = seg[s];
    const unsigned long long off = seg_off[s];
    const long long k = s / nbands;
    const int band = (int)(s % nbands);
    const long long jrow0 = (long long)band * R;
    for (uint32_t q = lane; q < sg.x; q += 32) {
      const unsigned long long src = (unsigned long long)sg.y + q;
      const unsigned long long dst = off + q;
      if (src >= staging_cap || dst >= capacity) continue;
      const uint32_t rec = staging[src];
      const int wv = (int)(rec & 7u) - 4;
      const uint32_t o = (rec >> 3) & 3u;
      const uint32_t pos = rec >> 5;
      const uint32_t r = pos / (uint32_t)nx, x = pos % (uint32_t)nx;
      const unsigned long long lin = ((unsigned long long)k * ny + jrow0 + r) * nx + x;
      face_ids[dst] = (lin << 2) | o;
      winding[dst] = (int8_t)wv;
    }
  }
}

// Statistics pass (only when requested): one thread per node, FP32.
__global__ void stats_kernel(const float2* __restrict__ psi, int nx, int ny, int nz,
                             qtv_stats* stats) {
  unsigned long long amb = 0, zer = 0, bad = 0;
  const long long nn = (long long)nx * ny * nz;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < nn;
       q += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(q % nx);
    const int j = (int)((q / nx) % ny);
    const int k = (int)(q / ((long long)nx * ny));
#pragma unroll
    for (int o = 0; o < 3; ++o) {
      int di[4], dj[4], dk[4];
      if (o == 0) {
        if (i + 1 >= nx || j + 1 >= ny) continue;
        const int a0[4] = {0, 1, 1, 0}, b0[4] = {0, 0, 1, 1};
        for (int c = 0; c < 4; ++c) { di[c] = a0[c]; dj[c] = b0[c]; dk[c] = 0; }
      } else if (o == 1) {
        if (j + 1 >= ny || k + 1 >= nz) continue;
        const int a0[4] = {0, 1, 1, 0}, b0[4] = {0, 0, 1, 1};
        for (int c = 0; c < 4; ++c) { di[c] = 0; dj[c] = a0[c]; dk[c] = b0[c]; }
      } else {
        if (k + 1 >= nz || i + 1 >= nx) continue;
        const int a0[4] = {0, 1, 1, 0}, b0[4] = {0, 0, 1, 1};
        for (int c = 0; c < 4; ++c) { dk[c] = a0[c]; di[c] = b0[c]; dj[c] = 0; }
      }
      float2 v[4];
      bool z = false, nf = false;
      for (int c = 0; c < 4; ++c) {
        v[c] = psi[((long long)(k + dk[c]) * ny + (j + dj[c])) * nx + (i + di[c])];
        z |= (v[c].x == 0.f && v[c].y == 0.f);
        nf |= !(finite_f(v[c].x) && finite_f(v[c].y));
      }
      if (nf) { ++bad; continue; }
      if (z) ++zer;
      bool am = false;
      for (int c = 0; c < 4; ++c) {
        float2 p = v[c], n = v[(c + 1) & 3];
        if (p.x == 0.f && p.y == 0.f) p = make_float2(1.f, 0.f);
        if (n.x == 0.f && n.y == 0.f) n = make_float2(1.f, 0.f);
        const float zr = fmaf(n.x, p.x, n.y * p.y);
        const float zi = fmaf(n.y, p.x, -n.x * p.y);
        am |= (zr < 0.f) && (fabsf(zi) < 1.0e-4f * -zr);
      }
      if (am) ++amb;
    }
  }
  for (int d = 16; d; d >>= 1) {
    amb += __shfl_down_sync(0xffffffffu, amb, d);
    zer += __shfl_down_sync(0xffffffffu, zer, d);
    bad += __shfl_down_sync(0xffffffffu, bad, d);
  }
  if ((threadIdx.x & 31) == 0) {
    if (amb) atomicAdd((unsigned long long*)&stats->ambiguous, amb);
    if (zer) atomicAdd((unsigned long long*)&stats->zero_node_faces, zer);
    if (bad) atomicAdd((unsigned long long*)&stats->nonfinite_faces, bad);
  }
}

struct LaunchShape {
  int threads = 0;
  int blocks_per_sm = 0;
};

using SweepFn = void (*)(SweepArgs);

SweepFn sweep_fn(int nw, bool vec) {
  if (nw <= 8) return vec ? sweep_kernel<true, 256> : sweep_kernel<false, 256>;
  if (nw <= 16) return vec ? sweep_kernel<true, 512> : sweep_kernel<false, 512>;
  return vec ? sweep_kernel<true, 1024> : sweep_kernel<false, 1024>;
}

LaunchShape sweep_shape(int nw, bool vec) {
  static LaunchShape cache[2][kMaxWarpsX + 1];
  LaunchShape& s = cache[vec ? 1 : 0][nw];
  if (s.threads == 0) {
    int bps = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, sweep_fn(nw, vec), nw * 32, 0);
    s.threads = nw * 32;
    s.blocks_per_sm = bps > 0 ? bps : 1;
  }
  return s;
}

}  // namespace

int identify_needs(qtv_handle h, int num_sms, const qtv_grid& g, uint64_t capacity,
                   const void* psi, uint64_t max_warps, IdentNeeds* n) {
  *n = IdentNeeds();
  const uint64_t nbands = (uint64_t)(g.ny + R - 1) / R;
  const uint64_t nseg = nbands * (uint64_t)g.nz;
  if (staged_variant(h, g.nx, g.ny, g.nz, psi) >= 0) {
    BulkNeeds b;
    const int rc = bulk_needs(h, num_sms, g, capacity, max_warps, &b);
    if (rc) return rc;
    n->staging = b.recs;
    n->seg = b.segf;
    n->table = b.table;
    n->seg_off = b.seg_off;
    n->tiles = b.tiles;
  } else {
    n->staging = capacity > 0 ? capacity : 1;
    n->seg = nseg;
    n->seg_off = nseg;
  }
  return QTV_OK;
}

int identify_launch(qtv_handle h, const qtv_grid& g, const float2* psi, uint64_t* face_ids,
                    int8_t* winding, uint64_t capacity, uint64_t* count, qtv_stats* stats,
                    cudaStream_t st, const IdentScratch& sc, uint64_t max_warps, float* xyz,
                    float* resid, uint8_t* flags) {
  if (staged_variant(h, g.nx, g.ny, g.nz, psi) >= 0) {
    const int rc = bulk_identify(h, g, psi, face_ids, winding, capacity, count, stats, st, sc,
                                 max_warps, xyz, resid, flags);
    if (rc) return rc;
    if (stats) {
      TraceScope ts(h, K_STATS, st);
      stats_kernel<<<h->num_sms * 8, 256, 0, st>>>(psi, g.nx, g.ny, g.nz, stats);
      const cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return check_cuda(e, "stats_kernel launch");
    }
    return QTV_OK;
  }
  uint32_t* staging = sc.staging;
  const uint64_t staging_cap = capacity;
  uint2* seg = sc.seg;
  unsigned long long* seg_off = sc.seg_off;
  unsigned long long* counters = sc.counters;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int nw = (nx + 63) / 64;
  const int nbands = (ny + R - 1) / R;
  const bool vec = (nx % 2 == 0) && ((reinterpret_cast<uintptr_t>(psi) & 15u) == 0);
  const LaunchShape shp = sweep_shape(nw, vec);
  const long long resident = (long long)shp.blocks_per_sm * h->num_sms;
  // work items: (z-chunk, band); about 2 items per resident CTA
  long long want_chunks = (2 * resident + nbands - 1) / nbands;
  if (want_chunks < 1) want_chunks = 1;
  if (want_chunks > nz) want_chunks = nz;
  int kchunk = (int)((nz + want_chunks - 1) / want_chunks);
  if (kchunk < 4) kchunk = nz < 4 ? nz : 4;
  const int nzchunks = (nz + kchunk - 1) / kchunk;
  const long long nitems = (long long)nzchunks * nbands;
  const long long nseg = (long long)nz * nbands;
  if (nitems > 0x7fffffffLL) return set_error(QTV_ERR_ARG, "grid too large for one launch");

  cudaError_t e = cudaMemsetAsync(counters, 0, 4 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return check_cuda(e, "cudaMemsetAsync(counters)");
  if (stats) {
    e = cudaMemsetAsync(stats, 0, sizeof(qtv_stats), st);
    if (e != cudaSuccess) return check_cuda(e, "cudaMemsetAsync(stats)");
  }
  SweepArgs a;
  a.psi = psi;
  a.nx = nx;
  a.ny = ny;
  a.nz = nz;
  a.nbands = nbands;
  a.kchunk = kchunk;
  a.nitems = (int)nitems;
  a.staging = staging;
  a.staging_cap = staging_cap;
  a.staging_top = counters;
  a.seg = seg;
  a.stats = stats;
  {
    const int grid = (int)(nitems < resident ? nitems : resident);
    {
      TraceScope ts(h, K_SWEEP, st);
      sweep_fn(nw, vec)<<<grid, shp.threads, 0, st>>>(a);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return check_cuda(e, "sweep_kernel launch");
  }

  const unsigned long long scanned =
      (unsigned long long)(nx - 1) * (ny - 1) * nz + (unsigned long long)nx * (ny - 1) * (nz - 1) +
      (unsigned long long)(nx - 1) * ny * (nz - 1);
  {
    TraceScope ts(h, K_SEG_SCAN, st);
    seg_scan_kernel<<<1, 1024, 0, st>>>(seg, nseg, seg_off, count, stats, scanned, counters + 2);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return check_cuda(e, "seg_scan_kernel launch");
  {
    const long long warps_needed = nseg;
    long long blocks = (warps_needed + 7) / 8;
    const long long maxb = (long long)h->num_sms * 8;
    if (blocks > maxb) blocks = maxb;
    if (blocks < 1) blocks = 1;
    TraceScope ts(h, K_SCATTER, st);
    scatter_kernel<<<(int)blocks, 256, 0, st>>>(seg, seg_off, nseg, nbands, nx, ny, staging,
                                                staging_cap, face_ids, winding, capacity);
    e = cudaGetLastError();
    if (e != cudaSuccess) return check_cuda(e, "scatter_kernel launch");
  }
  if (xyz && capacity > 0) {
    const int rc = localize_launch(h, g, psi, face_ids, winding, capacity, count, xyz, resid, flags,
                                   st);
    if (rc) return rc;
  }
  if (stats) {
    TraceScope ts(h, K_STATS, st);
    stats_kernel<<<h->num_sms * 8, 256, 0, st>>>(psi, nx, ny, nz, stats);
    e = cudaGetLastError();
    if (e != cudaSuccess) return check_cuda(e, "stats_kernel launch");
  }
  return QTV_OK;
}

}  // namespace qtv
