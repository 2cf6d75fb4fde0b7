// node_form.cu -- the node form of the circulation (Sec. 2.2.2) and the
// density error of Eq. 7 (Sec. 5) on the GPU.
//
// Node form.  For every node and each of the three grid planes through it, the
// circulation of Eq. 5 around the ring of the node's eight in-plane neighbours
// (the 2h x 2h square centred on the node, counter-clockwise about the plane
// normal; (u, v) = (x, y), (y, z), (z, x) for the planes xy, yz, zx), as the
// integer S = C / (2 pi).  A node is a vortex node when the largest |C| of its
// three planes exceeds pi, i.e. when some S != 0.  S = 0 where the ring leaves
// the grid or passes through a NaN/Inf node (the node itself is not on its
// ring).
//
// Arithmetic.  Every directed edge a -> b contributes the integer branch
// crossing r (its wrapped phase difference minus theta_b - theta_a, over
// 2 pi), decided from the sign bits of Im a, Im b and the sign of the
// determinant Re a Im b - Im a Re b; the theta terms telescope around the
// ring, so S is the sum of the ring's eight r.  Each grid edge is
// evaluated once, in its forward direction, and a ring that runs it backwards
// adds -r (the argument of the conjugate is the exact negation).  Two
// consecutive edges along a grid line make one side of a ring:
//   X_k(i,j) = r_x(i-1,j,k) + r_x(i,j,k)    (x-edges through (i,j,k))
//   Y_k(i,j) = r_y(i,j-1,k) + r_y(i,j,k)
//   Z(i,j,k) = r_z(i,j,k-1) + r_z(i,j,k)
// and the three rings of node (i,j,k) are
//   S_xy = X_k(i,j-1) + Y_k(i+1,j) - X_k(i,j+1) - Y_k(i-1,j)
//   S_yz = Y_{k-1}(i,j) + Z(i,j+1,k) - Y_{k+1}(i,j) - Z(i,j-1,k)
//   S_zx = Z(i-1,j,k) + X_{k+1}(i,j) - Z(i+1,j,k) - X_{k-1}(i,j).
//
// Layout (bit-sliced).  A warp owns 30 columns (lanes 1..30; lanes 0 and 31
// hold the neighbour columns) of a band of NB = 14 rows, and each lane keeps
// one bit per row (rows j0 - 1 .. j0 + NB, halo rows included) in words:
// the sign bit of Im psi and the sign bits of the FP32 cross products of its
// x, y and z edges, as the identification sweep does.  An edge term is +1 when
// s_a = 0, s_b = 1 and the cross sign is 0, -1 when s_a = 1, s_b = 0 and the
// sign is 1; edges that touch a zero node count 0.  The eight terms of a ring
// are word shifts (rows) and shuffles (columns) of these edge words, and
// their sum mod 8 comes from a carry-save adder tree over the words: S mod 8
// = #nonzero - 2 #negative, exact in [-3, 4] because only a ring whose eight
// differences are all exact +-pi ties reaches |S| = 4.  The warp marches z
// over a chunk of planes, streaming each lane's column through a 3-slot ring
// in shared memory with cp.async one plane ahead.
//
// Output.  Vortex nodes in ascending linear node index with their three S:
// each warp step stages its records contiguously in a chunk of the staging
// buffer that the warp reserved (one atomic per chunk) and writes a table
// entry {staging base, count, per-row counts}; an exclusive scan over the
// (plane, band) totals and a scatter that interleaves the column segments of
// every row put them in order.  Optionally the dense S field [3][nz][ny][nx].
//
// Density error.  e = sum_q |rho(p_q)| / (n rho_bar), rho the density |psi|^2
// of the trilinearly interpolated field at the sample points, rho_bar the mean
// density over all nodes.  Sums run in FP32 over short runs and in FP64 across
// runs, over a partition fixed by the launch shape, so a call is reproducible.
#include <cstdio>

#include "qtv_internal.cuh"

namespace qtv {

struct NodeWork {
  unsigned long long* recs = nullptr;  // staged vortex-node records
  uint64_t recs_cap = 0;
  uint4* table = nullptr;              // per (plane, band, column segment)
  uint64_t table_cap = 0;
  unsigned int* segtot = nullptr;      // vortex nodes per (plane, band)
  uint64_t segtot_cap = 0;
  unsigned long long* seg_off = nullptr;
  uint64_t seg_off_cap = 0;
  unsigned long long* top = nullptr;   // staging bump counter
  double* partial = nullptr;           // density sums per block
  uint64_t partial_cap = 0;
  int resident_warps = 0;
};

void node_work_free(NodeWork* w) {
  if (!w) return;
  cudaFree(w->recs);
  cudaFree(w->table);
  cudaFree(w->segtot);
  cudaFree(w->seg_off);
  cudaFree(w->top);
  cudaFree(w->partial);
  delete w;
}

namespace {

constexpr int NT = 16;          // rows held: bit t = row j0 - 1 + t
constexpr int NB = NT - 2;      // owned rows per band: bits 1..NB
constexpr uint32_t kOwnedRows = (1u << (NB + 1)) - 2u;
constexpr uint32_t kRowsHeld = NT == 32 ? 0xFFFFFFFFu : (1u << NT) - 1u;
constexpr int NCOL = 30;        // owned columns per warp (lanes 1..30)
constexpr int NODE_WARPS = 8;   // warps per CTA
constexpr int kSlots = 3;       // plane slots of a warp's ring: p - 1, p, p + 1
constexpr uint32_t kChunk = 4096;  // staging records a warp reserves at a time
// table entry: base, count, then one row-count byte per row (NT bytes)
constexpr int kTabVec = (2 + NT / 4 + 3) / 4;
constexpr size_t kRingFloats2 = (size_t)NODE_WARPS * kSlots * NT * 32;
// the rings, then NT bytes of per-row counts per warp, then per warp and row
// the lane mask and the prefix of the step's records
constexpr size_t kNodeSmem =
    kRingFloats2 * sizeof(float2) + NODE_WARPS * NT + NODE_WARPS * 2 * NT * sizeof(uint32_t);
static_assert(NT == 16 || NT == 32, "rows per band");
constexpr int DENS_THREADS = 256;
constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ bool fin(float v) { return fabsf(v) <= 3.402823466e38f; }

// acc' = (acc << 1) | sign bit of x
__device__ __forceinline__ uint32_t push1(uint32_t acc, float x) {
  return __funnelshift_l(__float_as_uint(x), acc, 1);
}

// FP32 value of Re a Im b - Im a Re b with one rounding of the second product
// absorbed by the FMA; its sign bit decides the edge term
__device__ __forceinline__ float cross_f(float2 a, float2 b) { return fmaf(a.x, b.y, -(a.y * b.x)); }

// packed product of the (Re, Im) values: zero if a component of a node is
// zero, non-finite if a node is (or on FP32 under- or overflow, which merely
// selects the masking path)
__device__ __forceinline__ unsigned long long prod_step(unsigned long long acc, float2 v) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;"
      : "=l"(d)
      : "l"(acc), "l"((unsigned long long)__float_as_uint(v.x) |
                      ((unsigned long long)__float_as_uint(v.y) << 32)));
  return d;
}
__device__ __forceinline__ bool prod_special(unsigned long long acc) {
  const float px = fabsf(__uint_as_float((uint32_t)acc));
  const float py = fabsf(__uint_as_float((uint32_t)(acc >> 32)));
  return !(px > 0.f && px <= 3.402823466e38f && py > 0.f && py <= 3.402823466e38f);
}
constexpr unsigned long long kProdOne = 0x3f8000003f800000ull;  // (1.f, 1.f)

// edge words of a -> b from sign words, the cross-sign word n and the edges E
// that touch a zero node (which count 0): P = crossing +1, N = crossing -1
struct EW {
  uint32_t P, N;
};
__device__ __forceinline__ EW edge_w(uint32_t sa, uint32_t sb, uint32_t n, uint32_t E) {
  EW e;
  e.P = ~sa & sb & ~n & ~E;
  e.N = sa & ~sb & n & ~E;
  return e;
}
__device__ __forceinline__ EW shl(EW e) { return EW{e.P << 1, e.N << 1}; }
__device__ __forceinline__ EW shr(EW e) { return EW{e.P >> 1, e.N >> 1}; }
__device__ __forceinline__ EW sh_up(EW e) {
  return EW{__shfl_up_sync(FULL, e.P, 1), __shfl_up_sync(FULL, e.N, 1)};
}
__device__ __forceinline__ EW sh_dn(EW e) {
  return EW{__shfl_down_sync(FULL, e.P, 1), __shfl_down_sync(FULL, e.N, 1)};
}

// full adder on bit-sliced words
__device__ __forceinline__ void fa(uint32_t a, uint32_t b, uint32_t c, uint32_t& s, uint32_t& cy) {
  s = a ^ b ^ c;
  cy = (a & b) | (c & (a ^ b));
}

// Sum mod 8 of eight terms in {-1, 0, 1} given as (nonzero, negative) words:
// S = #nonzero - 2 #negative.  A ring of finite nodes has |S| <= 3 unless all
// eight of its edge differences are exact +-pi ties (S = +-4, read as 4), so
// the residue in [-3, 4] is S.
struct Mod8 {
  uint32_t b0, b1, b2;
};
__device__ __forceinline__ Mod8 ring_sum(const uint32_t z[8], const uint32_t g[8]) {
  uint32_t s1, c1, s2, c2, c4, t1, c5;
  fa(z[0], z[1], z[2], s1, c1);
  fa(z[3], z[4], z[5], s2, c2);
  const uint32_t s3 = z[6] ^ z[7], c3 = z[6] & z[7];
  uint32_t a0, a1;
  fa(s1, s2, s3, a0, c4);
  fa(c1, c2, c3, t1, c5);
  a1 = t1 ^ c4;
  const uint32_t a2 = c5 ^ (t1 & c4);
  // negatives mod 4
  uint32_t u1, d1c, u2, d2c, d4, v1, d5;
  fa(g[0], g[1], g[2], u1, d1c);
  fa(g[3], g[4], g[5], u2, d2c);
  const uint32_t u3 = g[6] ^ g[7], d3c = g[6] & g[7];
  uint32_t e0;
  fa(u1, u2, u3, e0, d4);
  fa(d1c, d2c, d3c, v1, d5);
  const uint32_t e1 = v1 ^ d4;
  (void)d5;
  // S = a - 2 e (mod 8)
  Mod8 r;
  r.b0 = a0;
  r.b1 = a1 ^ e0;
  r.b2 = a2 ^ e1 ^ (~a1 & e0);
  return r;
}

// value in [-3, 4] of row t of a residue
__device__ __forceinline__ int mod8_at(const Mod8& m, int t) {
  const int v = (int)((m.b0 >> t) & 1u) | (int)(((m.b1 >> t) & 1u) << 1) |
                (int)(((m.b2 >> t) & 1u) << 2);
  return v >= 5 ? v - 8 : v;
}

struct NodeArgs {
  const float2* psi;
  int nx, ny, nz;
  int nbands, nxseg, kchunk;
  long long nitems;               // z chunks * bands * column segments
  unsigned long long* recs;
  unsigned long long recs_cap;
  unsigned long long* top;        // staging chunk counter
  uint4* table;                   // [nz][nbands][nxseg][3]
  unsigned int* segtot;           // [nz][nbands], zeroed before the launch
  int8_t* dense;                  // [3][nz][ny][nx] or null
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(src)
               : "memory");
}

__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Each lane streams its column of the band (32 rows) through the warp's ring
// with cp.async; a lane also reads its right neighbour's column, so every
// slot is fenced by __syncwarp after its copies complete and before it is
// refilled.  Rows, columns and planes outside the grid hold (1, 1): finite
// and nonzero, and only ever on rings that the validity masks reject.
__global__ void __launch_bounds__(NODE_WARPS * 32) node_form_kernel(NodeArgs a) {
  extern __shared__ float2 node_ring[];
  const int lane = threadIdx.x & 31;
  float2* ring = node_ring + (size_t)(threadIdx.x >> 5) * kSlots * NT * 32;
  uint8_t* rcnt = reinterpret_cast<uint8_t*>(node_ring + kRingFloats2) + (threadIdx.x >> 5) * NT;
  // per row: lane mask of the vortex nodes and records of the rows before it
  uint32_t* rbal = reinterpret_cast<uint32_t*>(reinterpret_cast<uint8_t*>(node_ring + kRingFloats2) +
                                               NODE_WARPS * NT) + (threadIdx.x >> 5) * 2 * NT;
  uint32_t* rpre = rbal + NT;
  const long long nwarps = (long long)gridDim.x * NODE_WARPS;
  const long long nxyz = (long long)a.nx * a.ny * a.nz;
  const unsigned lt = (1u << lane) - 1u;
  unsigned long long chunk_at = 0;  // next free staging record of the warp's chunk
  uint32_t chunk_left = 0;
  for (long long it = (long long)blockIdx.x * NODE_WARPS + (threadIdx.x >> 5); it < a.nitems;
       it += nwarps) {
    const int xs = (int)(it % a.nxseg);
    const long long rest = it / a.nxseg;
    const int band = (int)(rest % a.nbands);
    const int zc = (int)(rest / a.nbands);
    const int x = xs * NCOL + lane - 1;
    const int j0 = band * NB;  // row t of the band is j0 - 1 + t
    const int kz0 = zc * a.kchunk;
    const int kz1 = min(a.nz, kz0 + a.kchunk);
    const bool xin = x >= 0 && x < a.nx;
    const bool own = lane >= 1 && lane <= NCOL && x < a.nx;
    const bool colring = x >= 1 && x <= a.nx - 2;
    uint32_t rload = 0, rring = 0;  // rows in the grid / rows whose y-ring fits
    for (int t = 0; t < NT; ++t) {
      const int j = j0 - 1 + t;
      if (j >= 0 && j < a.ny) rload |= 1u << t;
      if (j >= 1 && j <= a.ny - 2) rring |= 1u << t;
    }
    const uint32_t rin = rload & kOwnedRows;
    rring &= kOwnedRows;

    // plane q (kz0 - 1 <= q <= kz1) lives in slot (q - kz0 + 1) mod kSlots
    auto issue = [&](int q, int slot) {
      float2* d = ring + slot * NT * 32 + lane;
      const bool qin = q >= 0 && q < a.nz && xin;
      const float2* src = a.psi + ((long long)(qin ? q : 0) * a.ny + (j0 - 1)) * a.nx + x;
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        if (qin && ((rload >> t) & 1u)) cp_async8(d + t * 32, src);
        else d[t * 32] = make_float2(1.f, 1.f);
        src += a.nx;
      }
      cp_commit();
    };
    __syncwarp();
    issue(kz0 - 1, 0);
    int sp = 0;  // slot of plane p

    EW RXm{0, 0}, RXc{0, 0}, RYm{0, 0}, RYc{0, 0}, RZlo{0, 0};
    uint32_t Sprev = 0, ZBc = 0, Bm = 0, Bc = 0;

    for (int p = kz0 - 1; p <= kz1; ++p) {
      __syncwarp();  // every lane is done with the slot of plane p - 2
      const int s1 = sp + 1 == kSlots ? 0 : sp + 1;
      if (p + 1 <= kz1) issue(p + 1, s1);
      else cp_commit();
      cp_wait<1>();  // plane p has landed (this lane's copies)
      __syncwarp();  // ... and every lane's
      const float2* cur = ring + sp * NT * 32;
      const float2* prv = (p == kz0 - 1) ? cur : ring + (sp == 0 ? kSlots - 1 : sp - 1) * NT * 32;
      const int ln = lane < 31 ? lane + 1 : 31;
      uint32_t Sp = 0, NX = 0, NY = 0, NZ = 0;
      unsigned long long prod = kProdOne;
      float2 vup = make_float2(1.f, 1.f);
#pragma unroll (NT == 16 ? 16 : 4)
      for (int t = NT - 1; t >= 0; --t) {
        const float2 v = cur[t * 32 + lane];
        const float2 nb = cur[t * 32 + ln];
        const float2 pv = prv[t * 32 + lane];
        Sp = push1(Sp, v.y);
        NX = push1(NX, cross_f(v, nb));
        NZ = push1(NZ, cross_f(pv, v));
        NY = push1(NY, cross_f(v, vup));
        prod = prod_step(prod, v);
        vup = v;
      }
      NY &= kRowsHeld >> 1;  // the top row has no y-edge in the band
      uint32_t ZBp = 0, Bn = 0;
      if (__any_sync(FULL, prod_special(prod))) {
        for (int t = 0; t < NT; ++t) {
          const float2 v = cur[t * 32 + lane];
          if (((__float_as_uint(v.x) | __float_as_uint(v.y)) << 1) == 0u) ZBp |= 1u << t;
          if (!(fin(v.x) && fin(v.y))) Bn |= 1u << t;
        }
        Bn &= xin ? rload : 0u;
      }
      const uint32_t Spn = __shfl_down_sync(FULL, Sp, 1);
      const uint32_t ZBpn = __shfl_down_sync(FULL, ZBp, 1);
      const EW RXn = edge_w(Sp, Spn, NX, ZBp | ZBpn);
      const EW RYn = edge_w(Sp, Sp >> 1, NY, ZBp | (ZBp >> 1));
      const EW RZhi = edge_w(Sprev, Sp, NZ, ZBc | ZBp);  // edges p - 1 -> p
      if (p > kz0) {
        // finalize node plane k = p - 1: planes k - 1, k, k + 1 are m, c, n
        const int k = p - 1;
        const bool kring = k >= 1 && k <= a.nz - 2;
        const uint32_t Bl = __shfl_up_sync(FULL, Bc, 1), Br = __shfl_down_sync(FULL, Bc, 1);
        const uint32_t H = Bl | Bc | Br;
        const uint32_t bad0 = (H << 1) | (H >> 1) | Bl | Br;
        const uint32_t V = Bm | Bc | Bn;
        const uint32_t bad1 = (V << 1) | (V >> 1) | Bm | Bn;
        const uint32_t bad2 =
            __shfl_up_sync(FULL, V, 1) | __shfl_down_sync(FULL, V, 1) | Bm | Bn;
        const uint32_t ok0 = (own && colring) ? (rring & ~bad0) : 0u;
        const uint32_t ok1 = (own && kring) ? (rring & ~bad1) : 0u;
        const uint32_t ok2 = (own && colring && kring) ? (rin & ~bad2) : 0u;
        Mod8 S0, S1, S2;
        {  // xy ring
          const EW xl = sh_up(RXc), yr = sh_dn(RYc), yl = sh_up(RYc);
          const EW t1 = shl(xl), t2 = shl(RXc), t3 = shl(yr), t4 = yr;  // + terms
          const EW t5 = shr(RXc), t6 = shr(xl), t7 = yl, t8 = shl(yl);  // - terms
          const uint32_t z[8] = {t1.P | t1.N, t2.P | t2.N, t3.P | t3.N, t4.P | t4.N,
                                 t5.P | t5.N, t6.P | t6.N, t7.P | t7.N, t8.P | t8.N};
          const uint32_t g[8] = {t1.N, t2.N, t3.N, t4.N, t5.P, t6.P, t7.P, t8.P};
          S0 = ring_sum(z, g);
        }
        {  // yz ring (u = y, v = z)
          const EW t1 = shl(RYm), t2 = RYm, t3 = shr(RZlo), t4 = shr(RZhi);  // + terms
          const EW t5 = shl(RYn), t6 = RYn, t7 = shl(RZlo), t8 = shl(RZhi);  // - terms
          const uint32_t z[8] = {t1.P | t1.N, t2.P | t2.N, t3.P | t3.N, t4.P | t4.N,
                                 t5.P | t5.N, t6.P | t6.N, t7.P | t7.N, t8.P | t8.N};
          const uint32_t g[8] = {t1.N, t2.N, t3.N, t4.N, t5.P, t6.P, t7.P, t8.P};
          S1 = ring_sum(z, g);
        }
        {  // zx ring (u = z, v = x), all terms at the node's row
          const EW t1 = sh_up(RZlo), t2 = sh_up(RZhi), t3 = sh_up(RXn), t4 = RXn;  // + terms
          const EW t5 = sh_dn(RZlo), t6 = sh_dn(RZhi), t7 = sh_up(RXm), t8 = RXm;  // - terms
          const uint32_t z[8] = {t1.P | t1.N, t2.P | t2.N, t3.P | t3.N, t4.P | t4.N,
                                 t5.P | t5.N, t6.P | t6.N, t7.P | t7.N, t8.P | t8.N};
          const uint32_t g[8] = {t1.N, t2.N, t3.N, t4.N, t5.P, t6.P, t7.P, t8.P};
          S2 = ring_sum(z, g);
        }
        const uint32_t nz0 = (S0.b0 | S0.b1 | S0.b2) & ok0;
        const uint32_t nz1 = (S1.b0 | S1.b1 | S1.b2) & ok1;
        const uint32_t nz2 = (S2.b0 | S2.b1 | S2.b2) & ok2;
        const uint32_t F = nz0 | nz1 | nz2;  // vortex nodes of this lane's owned rows
        if (a.dense && own) {
#pragma unroll 1
          for (int t = 1; t <= NB; ++t) {
            if (!((rin >> t) & 1u)) continue;
            const long long q = ((long long)k * a.ny + (j0 - 1 + t)) * a.nx + x;
            a.dense[q] = (int8_t)(((ok0 >> t) & 1u) ? mod8_at(S0, t) : 0);
            a.dense[nxyz + q] = (int8_t)(((ok1 >> t) & 1u) ? mod8_at(S1, t) : 0);
            a.dense[2 * nxyz + q] = (int8_t)(((ok2 >> t) & 1u) ? mod8_at(S2, t) : 0);
          }
        }
        const uint32_t cnt = __reduce_add_sync(FULL, (uint32_t)__popc(F));
        const uint32_t rows_any = __reduce_or_sync(FULL, F);
        // records of this step: contiguous in the warp's staging chunk, row-major
        if (cnt > chunk_left) {
          unsigned long long b = 0;
          if (lane == 0) b = atomicAdd(a.top, (unsigned long long)kChunk);
          chunk_at = __shfl_sync(FULL, b, 0);
          chunk_left = kChunk;
        }
        const unsigned long long base = chunk_at;
        chunk_at += cnt;
        chunk_left -= cnt;
        // uniform pass over the rows with vortex nodes: each row's lane mask
        // and the records before it (warp-private shared memory); then every
        // lane writes its own records
        if (lane < NT / 4) reinterpret_cast<uint32_t*>(rcnt)[lane] = 0u;  // bytes of rows 1..NB
        __syncwarp();
        uint32_t run = 0;
#pragma unroll 1
        for (uint32_t rem = rows_any; rem; rem &= rem - 1u) {
          const int t = __ffs(rem) - 1;
          const unsigned bal = __ballot_sync(FULL, (F >> t) & 1u);
          if (lane == 0) {
            rbal[t] = bal;
            rpre[t] = run;
            rcnt[t - 1] = (uint8_t)__popc(bal);
          }
          run += (uint32_t)__popc(bal);
        }
        __syncwarp();
#pragma unroll 1
        for (uint32_t mine = F; mine; mine &= mine - 1u) {
          const int t = __ffs(mine) - 1;
          const unsigned long long q =
              base + rpre[t] + (unsigned long long)__popc(rbal[t] & lt);
          if (q < a.recs_cap) {
            const int v0 = ((ok0 >> t) & 1u) ? mod8_at(S0, t) : 0;
            const int v1 = ((ok1 >> t) & 1u) ? mod8_at(S1, t) : 0;
            const int v2 = ((ok2 >> t) & 1u) ? mod8_at(S2, t) : 0;
            const unsigned long long lin =
                ((unsigned long long)k * a.ny + (unsigned long long)(j0 - 1 + t)) * a.nx + x;
            a.recs[q] = (lin << 12) | (uint32_t)(v0 + 4) | ((uint32_t)(v1 + 4) << 4) |
                        ((uint32_t)(v2 + 4) << 8);
          }
        }
        __syncwarp();
        if (lane == 0) {
          if (cnt) atomicAdd(a.segtot + (long long)k * a.nbands + band, cnt);
          const uint32_t* rc = reinterpret_cast<const uint32_t*>(rcnt);
          uint32_t wv[4 * kTabVec] = {};
          wv[0] = (uint32_t)base;
          wv[1] = cnt;
#pragma unroll
          for (int q = 0; q < NT / 4; ++q) wv[2 + q] = rc[q];
          uint4* te = a.table + (((long long)k * a.nbands + band) * a.nxseg + xs) * kTabVec;
#pragma unroll
          for (int q = 0; q < kTabVec; ++q)
            te[q] = make_uint4(wv[4 * q], wv[4 * q + 1], wv[4 * q + 2], wv[4 * q + 3]);
        }
      }
      RXm = RXc;
      RXc = RXn;
      RYm = RYc;
      RYc = RYn;
      RZlo = RZhi;
      Sprev = Sp;
      ZBc = ZBp;
      Bm = Bc;
      Bc = Bn;
      sp = s1;
    }
  }
}

// Exclusive scan of the per-(plane, band) totals, (plane, band) order being
// ascending node order.  One block.
__global__ void __launch_bounds__(1024) node_scan_kernel(const unsigned int* __restrict__ segtot,
                                                         long long nseg,
                                                         unsigned long long* __restrict__ seg_off,
                                                         uint64_t* __restrict__ count) {
  __shared__ unsigned long long warp_tot[32];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const long long per = (nseg + blockDim.x - 1) / blockDim.x;
  const long long s0 = tid * per, s1 = min(nseg, s0 + per);
  unsigned long long local = 0;
  for (long long s = s0; s < s1; ++s) local += segtot[s];
  unsigned long long incl = local;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const unsigned long long u = __shfl_up_sync(FULL, incl, d);
    if (lane >= d) incl += u;
  }
  if (lane == 31) warp_tot[w] = incl;
  __syncthreads();
  if (w == 0) {
    const unsigned long long v = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0ull;
    unsigned long long iv = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned long long u = __shfl_up_sync(FULL, iv, d);
      if (lane >= d) iv += u;
    }
    warp_tot[lane] = iv - v;
    if (lane == 31) *count = iv;
  }
  __syncthreads();
  unsigned long long run = warp_tot[w] + incl - local;
  for (long long s = s0; s < s1; ++s) {
    seg_off[s] = run;
    run += segtot[s];
  }
}

// One warp per (plane, band): for each row in turn, the column segments in
// ascending x (lane = segment), each copying its staged records of that row.
__global__ void node_scatter_kernel(const uint4* __restrict__ table,
                                    const unsigned long long* __restrict__ seg_off, long long nseg,
                                    int nxseg, const unsigned long long* __restrict__ recs,
                                    unsigned long long recs_cap, uint64_t* __restrict__ node_ids,
                                    int8_t* __restrict__ circ, unsigned long long capacity) {
  const int lane = threadIdx.x & 31;
  const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long s = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < nseg;
       s += warps) {
    unsigned long long off = seg_off[s];
    const uint4* te = table + s * nxseg * kTabVec;
    for (int t = 1; t <= NB; ++t) {
      for (int xb = 0; xb < nxseg; xb += 32) {
        const int xsi = xb + lane;
        uint32_t wv[4 * kTabVec] = {};
        if (xsi < nxseg) {
#pragma unroll
          for (int q = 0; q < kTabVec; ++q) {
            const uint4 e = te[xsi * kTabVec + q];
            wv[4 * q] = e.x;
            wv[4 * q + 1] = e.y;
            wv[4 * q + 2] = e.z;
            wv[4 * q + 3] = e.w;
          }
        }
        const uint32_t base = wv[0];
        const uint32_t* rcw = wv + 2;
        uint32_t c = 0, pre = 0;
#pragma unroll
        for (int r = 1; r <= NB; ++r) {
          const uint32_t cr = (rcw[(r - 1) >> 2] >> (8 * ((r - 1) & 3))) & 0xFFu;
          if (r < t) pre += cr;
          if (r == t) c = cr;
        }
        // exclusive scan of c over the lanes
        uint32_t incl = c;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const uint32_t u = __shfl_up_sync(FULL, incl, d);
          if (lane >= d) incl += u;
        }
        const uint32_t tot = __shfl_sync(FULL, incl, 31);
        const unsigned long long dst0 = off + (incl - c);
        const unsigned long long src0 = (unsigned long long)base + pre;
        for (uint32_t q = 0; q < c; ++q) {
          const unsigned long long src = src0 + q, dst = dst0 + q;
          if (src >= recs_cap || dst >= capacity) continue;
          const unsigned long long rec = recs[src];
          node_ids[dst] = rec >> 12;
          circ[3 * dst] = (int8_t)((int)(rec & 15u) - 4);
          circ[3 * dst + 1] = (int8_t)((int)((rec >> 4) & 15u) - 4);
          circ[3 * dst + 2] = (int8_t)((int)((rec >> 8) & 15u) - 4);
        }
        off += tot;
      }
    }
  }
}

// FP64 sum of the block's per-thread values; thread 0 gets it.
__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int d = 16; d; d >>= 1) v += __shfl_down_sync(FULL, v, d);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sh[i];
  return r;
}

// Sum of |psi|^2 over all nodes: FP32 runs of up to 4 nodes (8 squares),
// FP64 across runs.
__global__ void __launch_bounds__(DENS_THREADS) density_mean_kernel(const float2* __restrict__ psi,
                                                                    long long n,
                                                                    double* __restrict__ partial) {
  __shared__ double sh[DENS_THREADS / 32];
  const long long stride = (long long)gridDim.x * DENS_THREADS;
  double acc = 0.0;
  long long q = (long long)blockIdx.x * DENS_THREADS + threadIdx.x;
  for (; q + 3 * stride < n; q += 4 * stride) {
    const float2 a = __ldg(psi + q), b = __ldg(psi + q + stride), c = __ldg(psi + q + 2 * stride),
                 d = __ldg(psi + q + 3 * stride);
    float run = a.x * a.x;
    run = fmaf(a.y, a.y, run);
    run = fmaf(b.x, b.x, run);
    run = fmaf(b.y, b.y, run);
    run = fmaf(c.x, c.x, run);
    run = fmaf(c.y, c.y, run);
    run = fmaf(d.x, d.x, run);
    run = fmaf(d.y, d.y, run);
    acc += (double)run;
  }
  for (; q < n; q += stride) {
    const float2 a = __ldg(psi + q);
    acc += (double)fmaf(a.y, a.y, a.x * a.x);
  }
  const double s = block_sum(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

struct DensArgs {
  const float2* psi;
  int nx, ny, nz;
  float h, ox, oy, oz;
  const float* xyz;
  unsigned long long n;
  const uint64_t* n_dev;
  float* rho;
  double* partial;
};

// Trilinear density at the points (grid coordinates (p - origin) / h; NaN
// outside [0, n - 1] per axis) and the FP64 sum of |rho| per block.
__global__ void __launch_bounds__(DENS_THREADS) density_points_kernel(DensArgs a) {
  __shared__ double sh[DENS_THREADS / 32];
  unsigned long long nn = a.n;
  if (a.n_dev) {
    const unsigned long long d = *a.n_dev;
    if (d < nn) nn = d;
  }
  double acc = 0.0;
  for (unsigned long long q = (unsigned long long)blockIdx.x * DENS_THREADS + threadIdx.x; q < nn;
       q += (unsigned long long)gridDim.x * DENS_THREADS) {
    const float x = (__ldg(a.xyz + 3 * q) - a.ox) / a.h;
    const float y = (__ldg(a.xyz + 3 * q + 1) - a.oy) / a.h;
    const float z = (__ldg(a.xyz + 3 * q + 2) - a.oz) / a.h;
    float r;
    if (!(x >= 0.f && y >= 0.f && z >= 0.f && x <= (float)(a.nx - 1) && y <= (float)(a.ny - 1) &&
          z <= (float)(a.nz - 1))) {
      r = __int_as_float(0x7fc00000);
    } else {
      const int i = min((int)floorf(x), max(a.nx - 2, 0));
      const int j = min((int)floorf(y), max(a.ny - 2, 0));
      const int k = min((int)floorf(z), max(a.nz - 2, 0));
      const float fx = x - (float)i, fy = y - (float)j, fz = z - (float)k;
      const int i1 = i + 1 < a.nx ? i + 1 : i, j1 = j + 1 < a.ny ? j + 1 : j,
                k1 = k + 1 < a.nz ? k + 1 : k;
      float re = 0.f, im = 0.f;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int ii = (c & 1) ? i1 : i, jj = (c & 2) ? j1 : j, kk = (c & 4) ? k1 : k;
        const float w = ((c & 1) ? fx : 1.f - fx) * ((c & 2) ? fy : 1.f - fy) *
                        ((c & 4) ? fz : 1.f - fz);
        const float2 v = __ldg(a.psi + ((long long)kk * a.ny + jj) * a.nx + ii);
        re = fmaf(w, v.x, re);
        im = fmaf(w, v.y, im);
      }
      r = fmaf(re, re, im * im);
    }
    if (a.rho) a.rho[q] = r;
    acc += (double)fabsf(r);
  }
  const double s = block_sum(acc, sh);
  if (threadIdx.x == 0) a.partial[blockIdx.x] = s;
}

// out = {e, mean |rho| over the points, rho_bar}; the partial sums are added
// in a fixed order by one warp.
__global__ void density_final_kernel(const double* __restrict__ pm, int nbm,
                                     const double* __restrict__ pp, int nbp, long long nodes,
                                     unsigned long long n, const uint64_t* n_dev,
                                     double* __restrict__ out) {
  const int lane = threadIdx.x;
  double sm = 0.0, sp = 0.0;
  for (int b = lane; b < nbm; b += 32) sm += pm[b];
  for (int b = lane; b < nbp; b += 32) sp += pp[b];
#pragma unroll
  for (int d = 16; d; d >>= 1) {
    sm += __shfl_down_sync(FULL, sm, d);
    sp += __shfl_down_sync(FULL, sp, d);
  }
  if (lane == 0) {
    unsigned long long nn = n;
    if (n_dev && *n_dev < nn) nn = *n_dev;
    const double rho_bar = nodes > 0 ? sm / (double)nodes : 0.0;
    out[0] = nn ? sp / (rho_bar * (double)nn) : 0.0;
    out[1] = nn ? sp / (double)nn : 0.0;
    out[2] = rho_bar;
  }
}

bool capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return false;
  return cs != cudaStreamCaptureStatusNone;
}

template <typename T>
int grow(T*& p, uint64_t& cap, uint64_t want, cudaStream_t st, const char* what) {
  if (want <= cap && p) return QTV_OK;
  if (capturing(st))
    return set_error(QTV_ERR_STATE, "%s: workspace must grow during stream capture", what);
  cudaFree(p);
  p = nullptr;
  cap = 0;
  const cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&p), want * sizeof(T));
  if (e != cudaSuccess) {
    p = nullptr;
    return check_cuda(e, what);
  }
  cap = want;
  return QTV_OK;
}

NodeWork* work_of(qtv_handle h, cudaStream_t st, int* rc) {
  *rc = QTV_OK;
  if (h->node) return h->node;
  if (capturing(st)) {
    *rc = set_error(QTV_ERR_STATE, "node-form workspace must be created outside stream capture");
    return nullptr;
  }
  NodeWork* w = new NodeWork();
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&w->top), 2 * sizeof(unsigned long long));
  if (e != cudaSuccess) {
    delete w;
    *rc = check_cuda(e, "cudaMalloc(node-form counter)");
    return nullptr;
  }
  int bps = 0;
  e = cudaFuncSetAttribute(node_form_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kNodeSmem);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, node_form_kernel, NODE_WARPS * 32,
                                                      kNodeSmem);
  if (e != cudaSuccess) {
    node_work_free(w);
    *rc = check_cuda(e, "occupancy(node_form_kernel)");
    return nullptr;
  }
  w->resident_warps = (bps > 0 ? bps : 1) * NODE_WARPS * h->num_sms;
  h->node = w;
  return w;
}

int launch_blocks(const NodeWork* w, long long nitems) {
  long long blocks = (nitems + NODE_WARPS - 1) / NODE_WARPS;
  const long long maxb = w->resident_warps / NODE_WARPS;
  if (blocks > maxb) blocks = maxb;
  if (blocks < 1) blocks = 1;
  return (int)blocks;
}

}  // namespace

int node_circulation_launch(qtv_handle h, const qtv_grid& g, const float2* psi,
                            uint64_t* node_ids, int8_t* circ, uint64_t capacity, uint64_t* count,
                            int8_t* dense, cudaStream_t st) {
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const long long nodes = (long long)nx * ny * nz;
  if (nodes == 0) {
    const cudaError_t e = cudaMemsetAsync(count, 0, sizeof(uint64_t), st);
    return check_cuda(e, "cudaMemsetAsync(count)");
  }
  int rc = QTV_OK;
  NodeWork* w = work_of(h, st, &rc);
  if (!w) return rc;
  const int nbands = (ny + NB - 1) / NB;
  const int nxseg = (nx + NCOL - 1) / NCOL;
  const long long per_chunk = (long long)nbands * nxseg;
  // about four work items per resident warp, chunks of at least 8 planes
  long long want = (4LL * w->resident_warps + per_chunk - 1) / per_chunk;
  if (want < 1) want = 1;
  int kchunk = (int)((nz + want - 1) / want);
  if (kchunk < 8) kchunk = nz < 8 ? nz : 8;
  const int nzchunks = (nz + kchunk - 1) / kchunk;
  const long long nitems = (long long)nzchunks * per_chunk;
  const long long nseg = (long long)nz * nbands;
  const uint64_t ntab = (uint64_t)nseg * nxseg * kTabVec;
  // staging: the records, plus what chunk switches leave unused (under one
  // step of at most NB * NCOL <= kChunk / 8 records per chunk, i.e. at most
  // 1/7 of the records) and the open chunk of every warp
  const long long launch_warps = (long long)launch_blocks(w, nitems) * NODE_WARPS;
  const uint64_t recs_need = capacity + capacity / 7 + 1 + (uint64_t)launch_warps * kChunk;
  static_assert(NB * NCOL * 8 <= (int)kChunk, "chunk slack bound");
  // table entries keep 32-bit staging offsets
  if (recs_need > 0xFFFFFFFFull)
    return set_error(QTV_ERR_ARG, "node form: %llu staging records (capacity %llu) exceed 2^32",
                     (unsigned long long)recs_need, (unsigned long long)capacity);
  rc = grow(w->recs, w->recs_cap, recs_need, st, "cudaMalloc(node records)");
  if (!rc) rc = grow(w->table, w->table_cap, ntab, st, "cudaMalloc(node table)");
  if (!rc) rc = grow(w->segtot, w->segtot_cap, (uint64_t)nseg, st, "cudaMalloc(node totals)");
  if (!rc) rc = grow(w->seg_off, w->seg_off_cap, (uint64_t)nseg, st, "cudaMalloc(node offsets)");
  if (rc) return rc;

  cudaError_t e = cudaMemsetAsync(w->top, 0, sizeof(unsigned long long), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(w->segtot, 0, nseg * sizeof(unsigned int), st);
  if (e != cudaSuccess) return check_cuda(e, "cudaMemsetAsync(node-form state)");
  NodeArgs a;
  a.psi = psi;
  a.nx = nx;
  a.ny = ny;
  a.nz = nz;
  a.nbands = nbands;
  a.nxseg = nxseg;
  a.kchunk = kchunk;
  a.nitems = nitems;
  a.recs = w->recs;
  a.recs_cap = w->recs_cap;
  a.top = w->top;
  a.table = w->table;
  a.segtot = w->segtot;
  a.dense = dense;
  {
    TraceScope ts(h, K_NODE_FORM, st);
    node_form_kernel<<<launch_blocks(w, nitems), NODE_WARPS * 32, kNodeSmem, st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return check_cuda(e, "node_form_kernel launch");
  }
  {
    TraceScope ts(h, K_NODE_SCAN, st);
    node_scan_kernel<<<1, 1024, 0, st>>>(w->segtot, nseg, w->seg_off, count);
    e = cudaGetLastError();
    if (e != cudaSuccess) return check_cuda(e, "node_scan_kernel launch");
  }
  if (capacity > 0 && node_ids && circ) {
    long long blocks = (nseg + 7) / 8;
    const long long maxb = (long long)h->num_sms * 16;
    if (blocks > maxb) blocks = maxb;
    TraceScope ts(h, K_NODE_SCATTER, st);
    node_scatter_kernel<<<(int)blocks, 256, 0, st>>>(w->table, w->seg_off, nseg, nxseg, w->recs,
                                                     w->recs_cap, node_ids, circ, capacity);
    e = cudaGetLastError();
    if (e != cudaSuccess) return check_cuda(e, "node_scatter_kernel launch");
  }
  return QTV_OK;
}

int density_error_launch(qtv_handle h, const qtv_grid& g, const float2* psi, const float* xyz,
                         uint64_t n, const uint64_t* n_dev, float* rho, double* out,
                         cudaStream_t st) {
  int rc = QTV_OK;
  NodeWork* w = work_of(h, st, &rc);
  if (!w) return rc;
  const long long nodes = (long long)g.nx * g.ny * g.nz;
  const int nbm = h->num_sms * 4;
  long long nbp_l = ((long long)n + DENS_THREADS - 1) / DENS_THREADS;
  if (nbp_l > h->num_sms * 4) nbp_l = h->num_sms * 4;
  if (nbp_l < 1) nbp_l = 1;
  const int nbp = (int)nbp_l;
  rc = grow(w->partial, w->partial_cap, (uint64_t)(nbm + nbp), st, "cudaMalloc(density sums)");
  if (rc) return rc;
  TraceScope ts(h, K_DENSITY, st);
  density_mean_kernel<<<nbm, DENS_THREADS, 0, st>>>(psi, nodes, w->partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return check_cuda(e, "density_mean_kernel launch");
  DensArgs a;
  a.psi = psi;
  a.nx = g.nx;
  a.ny = g.ny;
  a.nz = g.nz;
  a.h = g.h;
  a.ox = g.origin[0];
  a.oy = g.origin[1];
  a.oz = g.origin[2];
  a.xyz = xyz;
  a.n = n;
  a.n_dev = n_dev;
  a.rho = rho;
  a.partial = w->partial + nbm;
  density_points_kernel<<<nbp, DENS_THREADS, 0, st>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return check_cuda(e, "density_points_kernel launch");
  density_final_kernel<<<1, 32, 0, st>>>(w->partial, nbm, w->partial + nbm, nbp, nodes, n, n_dev,
                                         out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return check_cuda(e, "density_final_kernel launch");
  return QTV_OK;
}

}  // namespace qtv
