// lines.cu -- classification, ordering, orientation and Catmull-Rom curves of
// the vortex-core lines of a sample graph (Sec. 3.4) on the GPU, parallel
// over samples: no thread walks a line.
//
// Input: the pierced-face graph of qtv_face_graph (neighbour table, degrees,
// component labels = lowest face index), the sample positions, and the face
// ids and windings (a sample's circulation direction is W times its face
// normal).
//
// Classification (per component, from the degrees of its samples): Type III
// when some degree exceeds 2 (branch points, e.g. at reconnections), Type II
// (closed loop) when every degree is 2 and the component has more than one
// sample, else Type I (an open line, or a single sample).
//
// Pieces (the simple lines, as in a walk that always takes the lowest
// unused neighbour): a Type I component is one piece from its lower end; a
// Type II component is one closed piece from its lowest sample towards the
// lower of that sample's two neighbours; a Type III component splits at its
// branch points: every chain between branch points and ends is a piece,
// started at a branch point b through neighbour v, and it is found from the
// branch side that comes first in (b, v) order (from the lower branch point;
// from the lower first neighbour for a chain that returns to b, which is then
// closed; dead ends are never starts).
//
// Ordering without walking.  "Special" samples end the chains: samples of
// degree other than 2, and the lowest sample of each Type II component.  On
// the directed edges (u -> w) of the graph (numbered compactly: sample u owns
// the edges from the exclusive scan of the degrees), the successor of (u -> w) is
// (w -> x), x the neighbour of w other than u, unless w is special.  Pointer
// jumping over this successor (double-buffered rounds, log2 of the sample
// count of them) gives every directed edge its distance to the end of its
// chain, the end sample and the sample before it.  A sample inside a chain
// then knows both ends, which end starts its piece, its position from that
// start (the distance back to it) and the piece's place in the output.
//
// Output order: pieces in ascending order of (start sample, first
// neighbour); each piece's samples in order, oriented (Sec. 3.4, right-hand
// rule) to run along their circulation direction: reversed when the sum over
// segments of (p[i+1] - p[i]) . dir[i] (with the closing segment for closed
// pieces) is negative, a closed piece keeping its first sample.  Curves:
// uniform Catmull-Rom, 'per_segment' points per segment, end points repeated
// for open pieces and wrapped for closed ones, plus the last sample of an open
// piece; lengths are the polyline lengths of the curves.  Curve points are
// one thread each; orientation sums use one warp and lengths one block per
// piece, FP64 in a fixed order, so results do not depend on timing.
#include <cstdio>

#include "qtv_internal.cuh"

namespace qtv {

struct LineWork {
  void* buf = nullptr;
  size_t cap = 0;
};

void line_work_free(LineWork* w) {
  if (!w) return;
  cudaFree(w->buf);
  delete w;
}

namespace {

constexpr int LT = 256;
constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr int kMaxRounds = 64;  // jump rounds: log2 of 2^32 samples plus slack
constexpr int kSlots = 10;

__device__ __forceinline__ unsigned long long limit_n(unsigned long long n, const uint64_t* n_dev) {
  if (n_dev) {
    const unsigned long long d = *n_dev;
    if (d < n) n = d;
  }
  return n;
}

struct LineArgs {
  unsigned long long n;
  const uint64_t* n_dev;
  const uint32_t* nbr;
  const uint8_t* deg;
  const uint32_t* comp;
  const float* xyz;
  const uint64_t* face_ids;
  const int8_t* winding;
  // workspace
  uint32_t* cflags;  // per component label: 1 = a sample of degree > 2,
                     // 2 = a sample of degree < 2
  uint8_t* special;  // per sample
  uint32_t* deg32;   // degrees as 32-bit values (scan input)
  unsigned long long* aoff;   // per sample: first directed edge (exclusive scan of degrees)
  const unsigned long long* narcs;  // device: number of directed edges
  uint32_t* atail;   // per directed edge: tail sample
  uint32_t* ahead;   // per directed edge: head sample
  // per directed edge, double-buffered: x = successor edge, y = distance
  // (edges) to the end of the chain, z = last edge of the chain (one 16-byte
  // gather per jump)
  uint4* jmp[2];
  uint32_t* live;    // per round: 1 if an edge's chain has not ended yet
  uint32_t* fbuf;    // buffer of the final jump results
  uint32_t* pcount;  // per sample: pieces started there
  uint32_t* plen;    // per sample: nodes of the pieces started there
  unsigned long long* pfirst;  // exclusive scan of pcount
  unsigned long long* noff;    // exclusive scan of plen
  unsigned long long* edge_node_off;  // per starting edge slot: node offset of its piece
  uint32_t* tmp_nodes;   // unoriented node list
  double* dots;          // per piece: orientation sum
  // outputs
  qtv_piece* pieces;
  unsigned long long piece_cap;
  uint32_t* nodes;
  unsigned long long node_cap;
};

__device__ __forceinline__ int comp_type(const LineArgs& a, uint32_t L) {
  // every degree 2 (a loop; a lone sample has degree 0) -> II; a branch -> III
  const uint32_t f = a.cflags[L];
  if (f & 1u) return 3;
  if (f == 0u) return 2;
  return 1;
}

__global__ void stats_init_kernel(LineArgs a) {
  const unsigned long long nn = limit_n(a.n, a.n_dev);
  for (unsigned long long u = (unsigned long long)blockIdx.x * LT + threadIdx.x; u < nn;
       u += (unsigned long long)gridDim.x * LT) {
    a.cflags[u] = 0;
  }
}

__global__ void stats_kernel(LineArgs a) {
  const unsigned long long nn = limit_n(a.n, a.n_dev);
  for (unsigned long long u = (unsigned long long)blockIdx.x * LT + threadIdx.x; u < nn;
       u += (unsigned long long)gridDim.x * LT) {
    const uint32_t L = a.comp[u], d = a.deg[u];
    a.deg32[u] = d;
    // only line ends and branch points mark their component (interior samples
    // of degree 2 mark nothing), and a mark already set is not set again
    if (d != 2u) {
      const uint32_t bit = d > 2u ? 1u : 2u;
      if ((a.cflags[L] & bit) == 0u) atomicOr(a.cflags + L, bit);
    }
  }
}

__global__ void special_kernel(LineArgs a) {
  const unsigned long long nn = limit_n(a.n, a.n_dev);
  for (unsigned long long u = (unsigned long long)blockIdx.x * LT + threadIdx.x; u < nn;
       u += (unsigned long long)gridDim.x * LT) {
    const uint32_t L = a.comp[u];
    const int t = comp_type(a, L);
    const int d = a.deg[u];
    a.special[u] = (t == 2) ? (uint8_t)(u == L) : (uint8_t)(d != 2);
  }
}

// slot of neighbour x in the row of w (rows are ascending, at most 10)
__device__ __forceinline__ int slot_of(const LineArgs& a, uint32_t w, uint32_t x) {
  const uint32_t* r = a.nbr + (unsigned long long)w * kSlots;
  for (int s = 0; s < kSlots; ++s)
    if (r[s] == x) return s;
  return -1;
}

// directed edges in compact order: sample u owns edges aoff[u] .. + deg[u] - 1
__global__ void arcs_kernel(LineArgs a) {
  const unsigned long long nn = limit_n(a.n, a.n_dev);
  for (unsigned long long u = (unsigned long long)blockIdx.x * LT + threadIdx.x; u < nn;
       u += (unsigned long long)gridDim.x * LT) {
    const int d = a.deg[u];
    const unsigned long long e0 = a.aoff[u];
    for (int s = 0; s < d; ++s) {
      a.atail[e0 + s] = (uint32_t)u;
      a.ahead[e0 + s] = a.nbr[u * kSlots + s];
    }
  }
}

__global__ void edges_init_kernel(LineArgs a) {
  const unsigned long long ne = *a.narcs;
  for (unsigned long long e = (unsigned long long)blockIdx.x * LT + threadIdx.x; e < ne;
       e += (unsigned long long)gridDim.x * LT) {
    const uint32_t u = a.atail[e], w = a.ahead[e];
    if (a.special[w]) {
      a.jmp[0][e] = make_uint4(kNone, 1u, (uint32_t)e, 0u);
    } else {
      // w has degree 2: continue to its other neighbour
      const int sx = (a.nbr[(unsigned long long)w * kSlots] == u) ? 1 : 0;
      a.jmp[0][e] = make_uint4((uint32_t)(a.aoff[w] + sx), 1u, kNone, 0u);
    }
  }
}

// Round r of pointer jumping (src = r & 1).  It is skipped once the previous
// round left no edge with a successor (every chain has ended), so the rounds
// beyond the longest chain cost a launch each; fbuf names the buffer that the
// last round run wrote.
__global__ void jump_kernel(LineArgs a, int src, int r) {
  if (r > 0 && a.live[r - 1] == 0u) return;
  const unsigned long long ne = *a.narcs;
  const int d = src ^ 1;
  if (blockIdx.x == 0 && threadIdx.x == 0) *a.fbuf = (uint32_t)d;
  bool flagged = false;  // this block has seen the round's flag set
  for (unsigned long long e0 = (unsigned long long)blockIdx.x * LT; e0 < ne;
       e0 += (unsigned long long)gridDim.x * LT) {
    const unsigned long long e = e0 + threadIdx.x;
    bool more = false;
    if (e < ne) {
      const uint4 J = a.jmp[src][e];
      if (J.x == kNone) {
        // an edge whose chain ended two rounds ago already holds its final
        // values in both buffers
        if (r < 2 || a.jmp[d][e].x != kNone) a.jmp[d][e] = J;
      } else {
        const uint4 N = a.jmp[src][J.x];
        a.jmp[d][e] = make_uint4(N.x, J.y + N.y, N.z, 0u);
        more = N.x != kNone;
      }
    }
    // one flag per round, set by the first block that finds a live edge (a
    // block reads it at most once, so the flag's line sees few requests)
    if (__syncthreads_or(more) && !flagged) {
      flagged = true;
      if (threadIdx.x == 0 && *reinterpret_cast<volatile uint32_t*>(a.live + r) == 0u)
        a.live[r] = 1u;
    }
  }
}

// end sample and the sample before it, of the chain that edge e starts
__device__ __forceinline__ void chain_end(const LineArgs& a, int buf, uint32_t e, uint32_t& end,
                                          uint32_t& before) {
  const uint32_t l = a.jmp[buf][e].z;
  before = a.atail[l];
  end = a.ahead[l];
}

// is the chain that starts at special sample s through neighbour y (edge e) a
// piece start?
__device__ __forceinline__ bool discovering(const LineArgs& a, int buf, uint32_t s, uint32_t y,
                                            uint32_t e) {
  uint32_t end, before;
  chain_end(a, buf, e, end, before);
  const int t = comp_type(a, a.comp[s]);
  if (t == 1) return s < end;
  if (t == 2) return y < before;
  if (a.deg[s] <= 2) return false;  // dead end
  if (end == s) return y < before;
  if (a.deg[end] > 2) return s < end;
  return true;
}

__global__ void count_kernel(LineArgs a) {
  const int buf = (int)*a.fbuf;
  const unsigned long long nn = limit_n(a.n, a.n_dev);
  for (unsigned long long u = (unsigned long long)blockIdx.x * LT + threadIdx.x; u < nn;
       u += (unsigned long long)gridDim.x * LT) {
    uint32_t pc = 0, nl = 0;
    const int d = a.deg[u];
    if (d == 0) {
      pc = 1;
      nl = 1;
    } else if (a.special[u]) {
      for (int s = 0; s < d; ++s) {
        const unsigned long long e = a.aoff[u] + s;
        const uint32_t y = a.nbr[u * kSlots + s];
        if (!discovering(a, buf, (uint32_t)u, y, (uint32_t)e)) continue;
        uint32_t end, before;
        chain_end(a, buf, (uint32_t)e, end, before);
        ++pc;
        nl += (end == (uint32_t)u) ? a.jmp[buf][e].y : a.jmp[buf][e].y + 1;
      }
    }
    a.pcount[u] = pc;
    a.plen[u] = nl;
  }
}

// piece records, and the start and end samples of every piece
__global__ void pieces_kernel(LineArgs a) {
  const int buf = (int)*a.fbuf;
  const unsigned long long nn = limit_n(a.n, a.n_dev);
  for (unsigned long long u = (unsigned long long)blockIdx.x * LT + threadIdx.x; u < nn;
       u += (unsigned long long)gridDim.x * LT) {
    if (a.pcount[u] == 0) continue;
    unsigned long long p = a.pfirst[u], off = a.noff[u];
    const uint32_t L = a.comp[u];
    const uint8_t ct = (uint8_t)comp_type(a, L);
    const int d = a.deg[u];
    if (d == 0) {
      if (p < a.piece_cap) {
        qtv_piece r = {};
        r.first = off;
        r.count = 1;
        r.component = L;
        r.comp_type = ct;
        a.pieces[p] = r;
      }
      a.tmp_nodes[off] = (uint32_t)u;
      continue;
    }
    for (int s = 0; s < d; ++s) {
      const unsigned long long e = a.aoff[u] + s;
      const uint32_t y = a.nbr[u * kSlots + s];
      if (!discovering(a, buf, (uint32_t)u, y, (uint32_t)e)) continue;
      uint32_t end, before;
      chain_end(a, buf, (uint32_t)e, end, before);
      const bool closed = end == (uint32_t)u;
      const uint32_t cnt = closed ? a.jmp[buf][e].y : a.jmp[buf][e].y + 1;
      if (p < a.piece_cap) {
        qtv_piece r = {};
        r.first = off;
        r.count = cnt;
        r.component = L;
        r.closed = closed ? 1 : 0;
        r.comp_type = ct;
        a.pieces[p] = r;
      }
      a.edge_node_off[e] = off;
      a.tmp_nodes[off] = (uint32_t)u;
      if (!closed) a.tmp_nodes[off + cnt - 1] = end;
      ++p;
      off += cnt;
    }
  }
}

// samples inside chains: their piece and position from its start
__global__ void interior_kernel(LineArgs a) {
  const int buf = (int)*a.fbuf;
  const unsigned long long nn = limit_n(a.n, a.n_dev);
  for (unsigned long long u = (unsigned long long)blockIdx.x * LT + threadIdx.x; u < nn;
       u += (unsigned long long)gridDim.x * LT) {
    if (a.special[u] || a.deg[u] != 2) continue;
    const unsigned long long e0 = a.aoff[u], e1 = e0 + 1;
    uint32_t end0, bef0, end1, bef1;
    chain_end(a, buf, (uint32_t)e0, end0, bef0);
    chain_end(a, buf, (uint32_t)e1, end1, bef1);
    // the chain's end edges, seen from the ends: (end0 -> bef0), (end1 -> bef1)
    const int s0 = slot_of(a, end0, bef0), s1 = slot_of(a, end1, bef1);
    if (s0 < 0 || s1 < 0) continue;
    const unsigned long long f0 = a.aoff[end0] + s0;
    const unsigned long long f1 = a.aoff[end1] + s1;
    unsigned long long off;
    uint32_t pos;
    if (discovering(a, buf, end0, bef0, (uint32_t)f0)) {
      off = a.edge_node_off[f0];
      pos = a.jmp[buf][e0].y;
    } else if (discovering(a, buf, end1, bef1, (uint32_t)f1)) {
      off = a.edge_node_off[f1];
      pos = a.jmp[buf][e1].y;
    } else {
      continue;
    }
    a.tmp_nodes[off + pos] = (uint32_t)u;
  }
}

__device__ __forceinline__ void face_dir(const LineArgs& a, uint32_t u, double d[3]) {
  const int o = (int)(a.face_ids[u] & 3u);
  const double w = (double)a.winding[u];
  d[0] = (o == 1) ? w : 0.0;  // yz face: normal +x
  d[1] = (o == 2) ? w : 0.0;  // zx face: normal +y
  d[2] = (o == 0) ? w : 0.0;  // xy face: normal +z
}

// one warp per piece: orientation sum in a fixed order
__global__ void orient_kernel(LineArgs a, const unsigned long long* counts) {
  const unsigned long long np = min((unsigned long long)counts[0], a.piece_cap);
  const int lane = threadIdx.x & 31;
  const unsigned long long warps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
  for (unsigned long long p = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
       p < np; p += warps) {
    const qtv_piece r = a.pieces[p];
    double sum = 0.0;
    if (a.face_ids && a.winding && r.count >= 2 && r.first + r.count <= a.node_cap) {
      const unsigned long long nseg = r.closed ? r.count : r.count - 1;
      for (unsigned long long i = lane; i < nseg; i += 32) {
        const uint32_t u = a.tmp_nodes[r.first + i];
        const uint32_t v = a.tmp_nodes[r.first + (i + 1 == r.count ? 0 : i + 1)];
        double d[3];
        face_dir(a, u, d);
#pragma unroll
        for (int c = 0; c < 3; ++c)
          sum += ((double)a.xyz[3ull * v + c] - (double)a.xyz[3ull * u + c]) * d[c];
      }
    }
#pragma unroll
    for (int dd = 16; dd; dd >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, dd);
    if (lane == 0) {
      a.dots[p] = sum;
      if (sum < 0.0) a.pieces[p].reversed = 1;
    }
  }
}

// final node list: each piece in order, or reversed (closed: first kept)
__global__ void place_kernel(LineArgs a, const unsigned long long* counts) {
  const unsigned long long np = min((unsigned long long)counts[0], a.piece_cap);
  const int lane = threadIdx.x & 31;
  const unsigned long long warps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
  for (unsigned long long p = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
       p < np; p += warps) {
    const qtv_piece r = a.pieces[p];
    for (unsigned long long k = lane; k < r.count; k += 32) {
      unsigned long long src = k;
      if (r.reversed) src = r.closed ? (k == 0 ? 0 : r.count - k) : r.count - 1 - k;
      const unsigned long long dst = r.first + k;
      if (dst < a.node_cap) a.nodes[dst] = a.tmp_nodes[r.first + src];
    }
  }
}

// ---------------------------------------------------------------------------
// exclusive scan of u32 values into u64 (three passes, deterministic)
// ---------------------------------------------------------------------------
constexpr int SB = 1024;        // threads per scan block
constexpr int SPER = 4;         // values per thread
constexpr int SCHUNK = SB * SPER;

template <typename T>
__global__ void __launch_bounds__(SB) scan_blocks_kernel(const T* in, const uint64_t* n_dev,
                                                         unsigned long long n,
                                                         unsigned long long* out,
                                                         unsigned long long* bsum) {
  __shared__ unsigned long long wt[32];
  const unsigned long long nn = limit_n(n, n_dev);
  const unsigned long long base = (unsigned long long)blockIdx.x * SCHUNK + threadIdx.x * SPER;
  unsigned long long v[SPER], loc = 0;
#pragma unroll
  for (int i = 0; i < SPER; ++i) {
    v[i] = base + i < nn ? in[base + i] : 0;
    loc += v[i];
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned long long inc = loc;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const unsigned long long t = __shfl_up_sync(0xffffffffu, inc, d);
    if (lane >= d) inc += t;
  }
  if (lane == 31) wt[w] = inc;
  __syncthreads();
  if (w == 0) {
    const unsigned long long x = wt[lane];
    unsigned long long y = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned long long t = __shfl_up_sync(0xffffffffu, y, d);
      if (lane >= d) y += t;
    }
    wt[lane] = y - x;
    if (lane == 31) bsum[blockIdx.x] = y;
  }
  __syncthreads();
  unsigned long long run = wt[w] + inc - loc;
#pragma unroll
  for (int i = 0; i < SPER; ++i) {
    if (base + i < nn) out[base + i] = run;
    run += v[i];
  }
}

__global__ void scan_sums_kernel(unsigned long long* bsum, int nb, unsigned long long* total) {
  if (threadIdx.x == 0) {
    unsigned long long run = 0;
    for (int b = 0; b < nb; ++b) {
      const unsigned long long x = bsum[b];
      bsum[b] = run;
      run += x;
    }
    *total = run;
  }
}

__global__ void scan_add_kernel(const uint64_t* n_dev, unsigned long long n,
                                unsigned long long* out, const unsigned long long* bsum) {
  const unsigned long long nn = limit_n(n, n_dev);
  for (unsigned long long i = (unsigned long long)blockIdx.x * LT + threadIdx.x; i < nn;
       i += (unsigned long long)gridDim.x * LT)
    out[i] += bsum[i / SCHUNK];
}

template <typename T>
void scan_u32(const T* in, const uint64_t* n_dev, unsigned long long n,
              unsigned long long* out, unsigned long long* bsum, unsigned long long* total,
              int num_sms, cudaStream_t st) {
  const int nb = (int)((n + SCHUNK - 1) / SCHUNK);
  scan_blocks_kernel<T><<<nb > 0 ? nb : 1, SB, 0, st>>>(in, n_dev, n, out, bsum);
  scan_sums_kernel<<<1, 32, 0, st>>>(bsum, nb > 0 ? nb : 1, total);
  long long g = ((long long)n + LT - 1) / LT;
  if (g > (long long)num_sms * 16) g = (long long)num_sms * 16;
  scan_add_kernel<<<(int)(g > 0 ? g : 1), LT, 0, st>>>(n_dev, n, out, bsum);
}

// ---------------------------------------------------------------------------
// curves
// ---------------------------------------------------------------------------
struct CurveArgs {
  const float* xyz;
  const uint32_t* nodes;
  const qtv_piece* pieces;
  unsigned long long np;
  const uint64_t* np_dev;
  int per;
  uint32_t* npts;                 // per piece: curve points
  unsigned long long* cfirst;     // exclusive scan of npts
  float* curve;
  unsigned long long curve_cap;
  float* length;
};

__device__ __forceinline__ uint32_t curve_points(const qtv_piece& r, int per) {
  if (r.count < 2) return r.count;
  return r.closed ? r.count * (uint32_t)per : (r.count - 1) * (uint32_t)per + 1;
}

__global__ void curve_count_kernel(CurveArgs a) {
  const unsigned long long np = limit_n(a.np, a.np_dev);
  for (unsigned long long p = (unsigned long long)blockIdx.x * LT + threadIdx.x; p < np;
       p += (unsigned long long)gridDim.x * LT)
    a.npts[p] = curve_points(a.pieces[p], a.per);
}

__device__ __forceinline__ void sample_pos(const CurveArgs& a, const qtv_piece& r, long long i,
                                           float p[3]) {
  const uint32_t u = a.nodes[r.first + (unsigned long long)i];
  p[0] = a.xyz[3ull * u];
  p[1] = a.xyz[3ull * u + 1];
  p[2] = a.xyz[3ull * u + 2];
}

// one thread per curve point: its piece by binary search over the first points
__global__ void curve_kernel(CurveArgs a, const unsigned long long* total) {
  const unsigned long long np = limit_n(a.np, a.np_dev);
  const unsigned long long nt = min((unsigned long long)*total, a.curve_cap);
  for (unsigned long long g = (unsigned long long)blockIdx.x * LT + threadIdx.x; g < nt;
       g += (unsigned long long)gridDim.x * LT) {
    unsigned long long lo = 0, hi = np;  // last piece with cfirst <= g
    while (hi - lo > 1) {
      const unsigned long long mid = (lo + hi) >> 1;
      if (a.cfirst[mid] <= g) lo = mid;
      else hi = mid;
    }
    const qtv_piece r = a.pieces[lo];
    const long long k = (long long)(g - a.cfirst[lo]);
    const long long m = r.count;
    float out[3];
    const long long nseg = r.closed ? m : m - 1;
    if (m < 2 || k >= nseg * a.per) {
      // a one-sample piece, or the last sample of an open piece
      sample_pos(a, r, m < 2 ? 0 : m - 1, out);
    } else {
      // segment s and step ti of point k (k < count * per < 2^32 * per)
      long long s;
      int ti;
      if ((k >> 32) == 0) {
        const uint32_t k32 = (uint32_t)k, q = k32 / (uint32_t)a.per;
        s = q;
        ti = (int)(k32 - q * (uint32_t)a.per);
      } else {
        s = k / a.per;
        ti = (int)(k - s * a.per);
      }
      // ext = closed: [P[m-1], P[0..m-1], P[0], P[1]]; open: [P[0], P[0..m-1], P[m-1]]
      // (s + c - 1 lies in [-1, m + 1] and m >= 2, so one wrap suffices)
      long long id[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        long long x = s + c - 1;
        if (r.closed) x = x < 0 ? x + m : (x >= m ? x - m : x);
        else x = x < 0 ? 0 : (x > m - 1 ? m - 1 : x);
        id[c] = x;
      }
      float p0[3], p1[3], p2[3], p3[3];
      sample_pos(a, r, id[0], p0);
      sample_pos(a, r, id[1], p1);
      sample_pos(a, r, id[2], p2);
      sample_pos(a, r, id[3], p3);
      const float t = (float)ti / (float)a.per, t2 = t * t, t3 = t2 * t;
#pragma unroll
      for (int c = 0; c < 3; ++c)
        out[c] = 0.5f * (2.f * p1[c] + t * (p2[c] - p0[c]) +
                         t2 * (2.f * p0[c] - 5.f * p1[c] + 4.f * p2[c] - p3[c]) +
                         t3 * (-p0[c] + 3.f * p1[c] - 3.f * p2[c] + p3[c]));
    }
    a.curve[3 * g] = out[0];
    a.curve[3 * g + 1] = out[1];
    a.curve[3 * g + 2] = out[2];
  }
}

// one block per piece: polyline length of its curve (each segment's length in
// FP32 from exact coordinate differences, summed in FP64: each thread sums a
// fixed stride, then a fixed reduction tree)
__global__ void __launch_bounds__(LT) length_kernel(CurveArgs a) {
  __shared__ double part[LT / 32];
  const unsigned long long np = limit_n(a.np, a.np_dev);
  for (unsigned long long p = blockIdx.x; p < np; p += gridDim.x) {
    const qtv_piece r = a.pieces[p];
    const unsigned long long c0 = a.cfirst[p];
    const unsigned long long n = a.npts[p];
    double sum = 0.0;
    if (n >= 2 && c0 + n <= a.curve_cap) {
      const unsigned long long nseg = r.closed ? n : n - 1;
      for (unsigned long long i = threadIdx.x; i < nseg; i += LT) {
        const unsigned long long j = (i + 1 == n) ? 0 : i + 1;
        float s2 = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float d = a.curve[3 * (c0 + j) + c] - a.curve[3 * (c0 + i) + c];
          s2 = fmaf(d, d, s2);
        }
        sum += (double)sqrtf(s2);
      }
    }
#pragma unroll
    for (int d = 16; d; d >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, d);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < LT / 32; ++w) t += part[w];
      a.length[p] = (float)t;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// arc-length thinning of ordered pieces
// ---------------------------------------------------------------------------
constexpr double kThinUnit = 4294967296.0;  // arc-length units per length unit (2^32)

struct ThinArgs {
  const float* xyz;
  const uint32_t* nodes;
  const qtv_piece* pieces;
  unsigned long long np, ne;
  unsigned long long D;            // box length in arc-length units
  unsigned long long* v;           // per entry: rounded length of the segment ending there
  unsigned long long* X;           // exclusive scan of v
  uint32_t* flag;                  // per entry: starts a group
  unsigned long long* G;           // exclusive scan of flag
  float* out;
  unsigned long long out_cap;
  qtv_piece* out_pieces;
  const unsigned long long* total;  // groups (device)
};

// piece of node-list entry g (pieces are contiguous and in order)
__device__ __forceinline__ unsigned long long piece_of(const ThinArgs& a, unsigned long long g) {
  unsigned long long lo = 0, hi = a.np;
  while (hi - lo > 1) {
    const unsigned long long mid = (lo + hi) >> 1;
    if (a.pieces[mid].first <= g) lo = mid;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ double coord(const ThinArgs& a, unsigned long long g, int c) {
  return (double)a.xyz[3ull * a.nodes[g] + c];
}

__global__ void thin_len_kernel(ThinArgs a) {
  for (unsigned long long g = (unsigned long long)blockIdx.x * LT + threadIdx.x; g < a.ne;
       g += (unsigned long long)gridDim.x * LT) {
    const qtv_piece r = a.pieces[piece_of(a, g)];
    unsigned long long v = 0;
    if (g > r.first) {
      // FP64 length of the segment from the previous sample, summed in the
      // order ((dx^2 + dy^2) + dz^2) without contraction, then rounded
      const double dx = coord(a, g, 0) - coord(a, g - 1, 0);
      const double dy = coord(a, g, 1) - coord(a, g - 1, 1);
      const double dz = coord(a, g, 2) - coord(a, g - 1, 2);
      const double q = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
      v = (unsigned long long)__double2ll_rn(sqrt(q) * kThinUnit);
    }
    a.v[g] = v;
  }
}

__global__ void thin_flag_kernel(ThinArgs a) {
  for (unsigned long long g = (unsigned long long)blockIdx.x * LT + threadIdx.x; g < a.ne;
       g += (unsigned long long)gridDim.x * LT) {
    const qtv_piece r = a.pieces[piece_of(a, g)];
    uint32_t f = 1;
    if (g > r.first) {
      const unsigned long long s = a.X[g] + a.v[g] - a.X[r.first];
      const unsigned long long sp = a.X[g - 1] + a.v[g - 1] - a.X[r.first];
      f = (s / a.D) != (sp / a.D) ? 1u : 0u;
    }
    a.flag[g] = f;
  }
}

__global__ void thin_mean_kernel(ThinArgs a) {
  for (unsigned long long g = (unsigned long long)blockIdx.x * LT + threadIdx.x; g < a.ne;
       g += (unsigned long long)gridDim.x * LT) {
    if (!a.flag[g]) continue;
    const qtv_piece r = a.pieces[piece_of(a, g)];
    const unsigned long long end = r.first + r.count;
    double sx = 0.0, sy = 0.0, sz = 0.0;
    unsigned long long m = 0, e = g;
    do {
      sx = __dadd_rn(sx, coord(a, e, 0));
      sy = __dadd_rn(sy, coord(a, e, 1));
      sz = __dadd_rn(sz, coord(a, e, 2));
      ++m;
      ++e;
    } while (e < end && !a.flag[e]);
    const unsigned long long q = a.G[g];
    if (q < a.out_cap) {
      a.out[3 * q] = (float)(sx / (double)m);
      a.out[3 * q + 1] = (float)(sy / (double)m);
      a.out[3 * q + 2] = (float)(sz / (double)m);
    }
  }
}

__global__ void thin_pieces_kernel(ThinArgs a) {
  for (unsigned long long p = (unsigned long long)blockIdx.x * LT + threadIdx.x; p < a.np;
       p += (unsigned long long)gridDim.x * LT) {
    qtv_piece r = a.pieces[p];
    const unsigned long long g0 = a.G[r.first];
    const unsigned long long g1 = p + 1 < a.np ? a.G[a.pieces[p + 1].first] : *a.total;
    r.first = g0;
    r.count = (uint32_t)(g1 - g0);
    a.out_pieces[p] = r;
  }
}

bool capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return false;
  return cs != cudaStreamCaptureStatusNone;
}

int ensure(qtv_handle h, size_t bytes, cudaStream_t st, void** out) {
  if (!h->lines) h->lines = new LineWork();
  LineWork* w = h->lines;
  if (bytes > w->cap) {
    if (capturing(st))
      return set_error(QTV_ERR_STATE, "line workspace must grow outside stream capture");
    cudaFree(w->buf);
    w->buf = nullptr;
    w->cap = 0;
    const cudaError_t e = cudaMalloc(&w->buf, bytes);
    if (e != cudaSuccess) return check_cuda(e, "cudaMalloc(line workspace)");
    w->cap = bytes;
  }
  *out = w->buf;
  return QTV_OK;
}

template <typename T>
T* carve(char*& p, unsigned long long count) {
  T* r = reinterpret_cast<T*>(p);
  p += ((count * sizeof(T) + 255) / 256) * 256;
  return r;
}

}  // namespace

int line_pieces_launch(qtv_handle h, uint64_t n, const uint64_t* n_dev, const uint32_t* nbr,
                       const uint8_t* deg, const uint32_t* comp, const float* xyz,
                       const uint64_t* face_ids, const int8_t* winding, qtv_piece* pieces,
                       uint64_t piece_cap, uint32_t* nodes, uint64_t node_cap, uint64_t* counts,
                       cudaStream_t st) {
  const unsigned long long ne = (unsigned long long)n * kSlots;
  // each piece holds at least one edge and adds at most two end samples to
  // its interior ones; edges <= 5 n (degree <= 10)
  const unsigned long long nodes_max = 11ull * n + 1;
  const unsigned long long nb = (n + SCHUNK - 1) / SCHUNK + 1;
  size_t bytes = 0;
  {
    // sizes must match the carve sequence below
    const unsigned long long sz[] = {n * 4, n, ne * 16, ne * 16, n * 4, n * 4, n * 8, n * 8, ne * 8,
                                     nodes_max * 4, n * 8, nb * 8, nb * 8, 16,
                                     n * 4, n * 8, ne * 4, ne * 4, nb * 8, 8, kMaxRounds * 4 + 4};
    for (unsigned long long s : sz) bytes += ((s + 255) / 256) * 256;
  }
  void* buf = nullptr;
  int rc = ensure(h, bytes, st, &buf);
  if (rc) return rc;
  char* p = static_cast<char*>(buf);
  LineArgs a;
  a.n = n;
  a.n_dev = n_dev;
  a.nbr = nbr;
  a.deg = deg;
  a.comp = comp;
  a.xyz = xyz;
  a.face_ids = face_ids;
  a.winding = winding;
  a.cflags = carve<uint32_t>(p, n);
  a.special = carve<uint8_t>(p, n);
  a.jmp[0] = carve<uint4>(p, ne);
  a.jmp[1] = carve<uint4>(p, ne);
  a.pcount = carve<uint32_t>(p, n);
  a.plen = carve<uint32_t>(p, n);
  a.pfirst = carve<unsigned long long>(p, n);
  a.noff = carve<unsigned long long>(p, n);
  a.edge_node_off = carve<unsigned long long>(p, ne);
  a.tmp_nodes = carve<uint32_t>(p, nodes_max);
  a.dots = carve<double>(p, n);
  unsigned long long* bs1 = carve<unsigned long long>(p, nb);
  unsigned long long* bs2 = carve<unsigned long long>(p, nb);
  unsigned long long* tot = carve<unsigned long long>(p, 2);
  a.deg32 = carve<uint32_t>(p, n);
  a.aoff = carve<unsigned long long>(p, n);
  a.atail = carve<uint32_t>(p, ne);
  a.ahead = carve<uint32_t>(p, ne);
  unsigned long long* bs3 = carve<unsigned long long>(p, nb);
  unsigned long long* narcs = carve<unsigned long long>(p, 1);
  a.narcs = narcs;
  a.live = carve<uint32_t>(p, kMaxRounds + 1);
  a.fbuf = a.live + kMaxRounds;
  a.pieces = pieces;
  a.piece_cap = piece_cap;
  a.nodes = nodes;
  a.node_cap = node_cap;

  long long g = ((long long)n + LT - 1) / LT;
  if (g > (long long)h->num_sms * 16) g = (long long)h->num_sms * 16;
  if (g < 1) g = 1;
  long long ge = ((long long)ne + LT - 1) / LT;
  if (ge > (long long)h->num_sms * 32) ge = (long long)h->num_sms * 32;
  if (ge < 1) ge = 1;
  TraceScope ts(h, K_LINES, st);
  stats_init_kernel<<<(int)g, LT, 0, st>>>(a);
  stats_kernel<<<(int)g, LT, 0, st>>>(a);
  special_kernel<<<(int)g, LT, 0, st>>>(a);
  // compact directed edges: offsets by an exclusive scan of the degrees
  scan_u32(a.deg32, n_dev, n, a.aoff, bs3, narcs, h->num_sms, st);
  arcs_kernel<<<(int)g, LT, 0, st>>>(a);
  edges_init_kernel<<<(int)ge, LT, 0, st>>>(a);
  int rounds = 1;
  while ((1ull << rounds) < (unsigned long long)n + 1) ++rounds;
  cudaError_t e = cudaMemsetAsync(a.live, 0, (kMaxRounds + 1) * sizeof(uint32_t), st);
  if (e != cudaSuccess) return check_cuda(e, "cudaMemsetAsync(line rounds)");
  for (int r = 0; r < rounds; ++r) jump_kernel<<<(int)ge, LT, 0, st>>>(a, r & 1, r);
  count_kernel<<<(int)g, LT, 0, st>>>(a);
  scan_u32(a.pcount, n_dev, n, a.pfirst, bs1, tot, h->num_sms, st);
  scan_u32(a.plen, n_dev, n, a.noff, bs2, tot + 1, h->num_sms, st);
  e = cudaMemcpyAsync(counts, tot, 2 * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return check_cuda(e, "cudaMemcpyAsync(line counts)");
  pieces_kernel<<<(int)g, LT, 0, st>>>(a);
  interior_kernel<<<(int)g, LT, 0, st>>>(a);
  orient_kernel<<<h->num_sms * 8, LT, 0, st>>>(a, tot);
  place_kernel<<<h->num_sms * 8, LT, 0, st>>>(a, tot);
  e = cudaGetLastError();
  return check_cuda(e, "line pieces launch");
}

int piece_curves_launch(qtv_handle h, const float* xyz, const uint32_t* nodes,
                        const qtv_piece* pieces, uint64_t np, const uint64_t* np_dev, int per,
                        float* curve, uint64_t curve_cap, uint64_t* curve_first, float* length,
                        uint64_t* total, cudaStream_t st) {
  const unsigned long long nb = (np + SCHUNK - 1) / SCHUNK + 1;
  size_t bytes = ((np * 4 + 255) / 256) * 256 + ((nb * 8 + 255) / 256) * 256 + 256;
  void* buf = nullptr;
  int rc = ensure(h, bytes, st, &buf);
  if (rc) return rc;
  char* p = static_cast<char*>(buf);
  CurveArgs a;
  a.xyz = xyz;
  a.nodes = nodes;
  a.pieces = pieces;
  a.np = np;
  a.np_dev = np_dev;
  a.per = per;
  a.npts = carve<uint32_t>(p, np);
  unsigned long long* bs = carve<unsigned long long>(p, nb);
  a.cfirst = reinterpret_cast<unsigned long long*>(curve_first);
  a.curve = curve;
  a.curve_cap = curve_cap;
  a.length = length;
  long long g = ((long long)np + LT - 1) / LT;
  if (g > (long long)h->num_sms * 16) g = (long long)h->num_sms * 16;
  if (g < 1) g = 1;
  TraceScope ts(h, K_CURVES, st);
  curve_count_kernel<<<(int)g, LT, 0, st>>>(a);
  scan_u32(a.npts, np_dev, np, a.cfirst, bs, reinterpret_cast<unsigned long long*>(total),
           h->num_sms, st);
  curve_kernel<<<h->num_sms * 16, LT, 0, st>>>(a, reinterpret_cast<unsigned long long*>(total));
  long long gp = (long long)np;
  if (gp > (long long)h->num_sms * 16) gp = (long long)h->num_sms * 16;
  length_kernel<<<(int)(gp > 0 ? gp : 1), LT, 0, st>>>(a);
  const cudaError_t e = cudaGetLastError();
  return check_cuda(e, "piece curves launch");
}

int thin_pieces_launch(qtv_handle h, const float* xyz, const uint32_t* nodes,
                       const qtv_piece* pieces, uint64_t np, uint64_t nnodes, float box,
                       float* out_xyz, uint64_t out_cap, qtv_piece* out_pieces, uint64_t* total,
                       cudaStream_t st) {
  const unsigned long long ne = nnodes;
  const unsigned long long nb = (ne + SCHUNK - 1) / SCHUNK + 1;
  const unsigned long long sz[] = {ne * 8, ne * 8, ne * 4, ne * 8, nb * 8, nb * 8, 16};
  size_t bytes = 0;
  for (unsigned long long x : sz) bytes += ((x + 255) / 256) * 256;
  void* buf = nullptr;
  int rc = ensure(h, bytes, st, &buf);
  if (rc) return rc;
  char* p = static_cast<char*>(buf);
  ThinArgs a;
  a.xyz = xyz;
  a.nodes = nodes;
  a.pieces = pieces;
  a.np = np;
  a.ne = ne;
  const double Dd = (double)box * kThinUnit;
  a.D = Dd >= 1.0 ? (unsigned long long)llrint(Dd) : 1ull;
  a.v = carve<unsigned long long>(p, ne);
  a.X = carve<unsigned long long>(p, ne);
  a.flag = carve<uint32_t>(p, ne);
  a.G = carve<unsigned long long>(p, ne);
  unsigned long long* bs1 = carve<unsigned long long>(p, nb);
  unsigned long long* bs2 = carve<unsigned long long>(p, nb);
  unsigned long long* tots = carve<unsigned long long>(p, 2);
  a.out = out_xyz;
  a.out_cap = out_cap;
  a.out_pieces = out_pieces;
  a.total = tots + 1;
  long long g = ((long long)ne + LT - 1) / LT;
  if (g > (long long)h->num_sms * 16) g = (long long)h->num_sms * 16;
  if (g < 1) g = 1;
  long long gp = ((long long)np + LT - 1) / LT;
  if (gp > (long long)h->num_sms * 16) gp = (long long)h->num_sms * 16;
  if (gp < 1) gp = 1;
  TraceScope ts(h, K_THIN, st);
  thin_len_kernel<<<(int)g, LT, 0, st>>>(a);
  scan_u32(a.v, nullptr, ne, a.X, bs1, tots, h->num_sms, st);
  thin_flag_kernel<<<(int)g, LT, 0, st>>>(a);
  scan_u32(a.flag, nullptr, ne, a.G, bs2, tots + 1, h->num_sms, st);
  thin_mean_kernel<<<(int)g, LT, 0, st>>>(a);
  thin_pieces_kernel<<<(int)gp, LT, 0, st>>>(a);
  cudaError_t e = cudaMemcpyAsync(total, tots + 1, sizeof(uint64_t), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaGetLastError();
  return check_cuda(e, "thin pieces launch");
}

}  // namespace qtv
