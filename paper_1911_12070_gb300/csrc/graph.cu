// graph.cu -- the sample graph of Sec. 3.1 over pierced faces (or over the
// vortex nodes of the node form, 6-connected along grid lines as in the
// paper), and its connected components (the independent lines of Sec. 3.2),
// on the GPU.
//
// Adjacency.  Two pierced faces are adjacent when they bound the same unit
// cell (a cell with all corners in the grid); a line through a cell enters
// through one pierced face and leaves through another, so this links
// consecutive samples of a line, and a cell with 4 or 6 pierced faces links
// all of them (a branch, as at a reconnection).  A face bounds at most two
// cells and a cell has five other faces, so a face has at most 10
// neighbours; the output is a fixed-stride table nbr[a][10] (ascending
// indices into the face list, unused entries 0xFFFFFFFF) and deg[a].
// Neighbours are found by binary search in the ascending face list, within
// the slice of the face's grid row (plane k, row j), whose bounds come from a
// row table built by one lower-bound search per row.
//
// Components.  Union-find over the adjacency: every edge (a, b), a < b, links
// the root of the larger index under the root of the smaller one with a
// compare-and-swap, and finds shorten paths by halving.  Parents only ever
// decrease, so every root is the lowest face index of its component, and the
// final labels comp[a] = root are independent of the order in which threads
// ran.  Once all links are made, a separate pass writes every label with a
// read-only walk to its root (a halving store there could overwrite a label
// its owner had already set).  The CAS loop is lock-free (a failed CAS means
// another link succeeded); it is nonetheless bounded, and a call whose loop
// ran out reports QTV_COUNT_TIMEOUT as the component count.
#include <cstdio>

#include "qtv_internal.cuh"

namespace qtv {

struct GraphWork {
  uint32_t* rows = nullptr;  // row table: first face index of each (k, j) row
  uint64_t rows_cap = 0;
  unsigned long long* status = nullptr;
};

void graph_work_free(GraphWork* w) {
  if (!w) return;
  cudaFree(w->rows);
  cudaFree(w->status);
  delete w;
}

namespace {

constexpr int GT = 256;
constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr int kMaxTries = 1 << 20;  // CAS retries of one link before giving up

__device__ __forceinline__ unsigned long long limit_n(unsigned long long n, const uint64_t* n_dev) {
  if (n_dev) {
    const unsigned long long d = *n_dev;
    if (d < n) n = d;
  }
  return n;
}

// rows[r] = first index a with face_ids[a] in row r or later (r = k*ny + j),
// for r in [0, R]; rows[R] = n
__global__ void row_table_kernel(const uint64_t* __restrict__ ids, unsigned long long n,
                                 const uint64_t* n_dev, int nx, long long R, int shift,
                                 uint32_t* __restrict__ rows) {
  const unsigned long long nn = limit_n(n, n_dev);
  for (long long r = (long long)blockIdx.x * GT + threadIdx.x; r <= R;
       r += (long long)gridDim.x * GT) {
    const unsigned long long key = ((unsigned long long)r * (unsigned long long)nx) << shift;
    unsigned long long lo = 0, hi = nn;
    while (lo < hi) {
      const unsigned long long mid = (lo + hi) >> 1;
      if (__ldg(ids + mid) < key) lo = mid + 1;
      else hi = mid;
    }
    rows[r] = (uint32_t)lo;
  }
}

}  // namespace

cudaError_t row_table_launch(const uint64_t* ids, unsigned long long n, const uint64_t* n_dev,
                             int nx, long long R, int shift, uint32_t* rows, int num_sms,
                             cudaStream_t st) {
  long long blocks = (R + 1 + GT - 1) / GT;
  if (blocks > (long long)num_sms * 16) blocks = (long long)num_sms * 16;
  if (blocks < 1) blocks = 1;
  row_table_kernel<<<(int)blocks, GT, 0, st>>>(ids, n, n_dev, nx, R, shift, rows);
  return cudaGetLastError();
}

namespace {

struct GraphArgs {
  const uint64_t* ids;
  unsigned long long n;
  const uint64_t* n_dev;
  int nx, ny, nz;
  const uint32_t* rows;
  int shift;       // id = linear node index << shift (2 for faces, 0 for nodes)
  int stride;      // neighbour slots per entry (10 for faces, 6 for nodes)
  uint32_t* nbr;   // [n][stride]
  uint8_t* deg;
  uint32_t* comp;  // parents during the union-find
  unsigned long long* status;  // [0] components, [1] gave-up flag
};

// index of face id f in the list, or kNone
__device__ __forceinline__ uint32_t find_face(const GraphArgs& a, unsigned long long f) {
  const unsigned long long row = (f >> a.shift) / (unsigned long long)a.nx;
  unsigned long long lo = __ldg(a.rows + row), hi = __ldg(a.rows + row + 1);
  while (lo < hi) {
    const unsigned long long mid = (lo + hi) >> 1;
    const unsigned long long v = __ldg(a.ids + mid);
    if (v < f) lo = mid + 1;
    else hi = mid;
  }
  if (lo < (unsigned long long)__ldg(a.rows + row + 1) && __ldg(a.ids + lo) == f)
    return (uint32_t)lo;
  return kNone;
}

__global__ void __launch_bounds__(GT) adjacency_kernel(GraphArgs a) {
  const unsigned long long nn = limit_n(a.n, a.n_dev);
  const long long nx = a.nx, ny = a.ny, nz = a.nz;
  for (unsigned long long q = (unsigned long long)blockIdx.x * GT + threadIdx.x; q < nn;
       q += (unsigned long long)gridDim.x * GT) {
    const unsigned long long f = __ldg(a.ids + q);
    const int o = (int)(f & 3u);
    const long long lin = (long long)(f >> 2);
    long long i, j, k;
    split_lin((unsigned long long)lin, nx, ny, i, j, k);
    uint32_t nb[10];
    int m = 0;
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      // the cell below / above the face along its normal
      long long ci = i, cj = j, ck = k;
      if (side == 0) {
        if (o == 0) ck -= 1;
        else if (o == 1) ci -= 1;
        else cj -= 1;
      }
      if (ci < 0 || cj < 0 || ck < 0 || ci >= nx - 1 || cj >= ny - 1 || ck >= nz - 1) continue;
      const unsigned long long base = (unsigned long long)((ck * ny + cj) * nx + ci);
      const unsigned long long cand[6] = {
          (base << 2) | 0ull, ((base + (unsigned long long)(nx * ny)) << 2) | 0ull,
          (base << 2) | 1ull, ((base + 1ull) << 2) | 1ull,
          (base << 2) | 2ull, ((base + (unsigned long long)nx) << 2) | 2ull};
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        if (cand[c] == f) continue;
        const uint32_t idx = find_face(a, cand[c]);
        if (idx != kNone) nb[m++] = idx;
      }
    }
    // ascending order (at most 10 entries)
    for (int x = 1; x < m; ++x) {
      const uint32_t v = nb[x];
      int y = x - 1;
      while (y >= 0 && nb[y] > v) {
        nb[y + 1] = nb[y];
        --y;
      }
      nb[y + 1] = v;
    }
    uint32_t* row = a.nbr + q * 10;
    for (int x = 0; x < 10; ++x) row[x] = x < m ? nb[x] : kNone;
    a.deg[q] = (uint8_t)m;
    // union-find start: the smaller of the face and its lowest neighbour
    a.comp[q] = (m > 0 && nb[0] < (uint32_t)q) ? nb[0] : (uint32_t)q;
  }
}

// vortex-node graph: 6-connectivity along grid lines; candidates in the
// order -z, -y, -x, +x, +y, +z are ascending linear indices
__global__ void __launch_bounds__(GT) node_adjacency_kernel(GraphArgs a) {
  const unsigned long long nn = limit_n(a.n, a.n_dev);
  const long long nx = a.nx, ny = a.ny, nz = a.nz;
  for (unsigned long long q = (unsigned long long)blockIdx.x * GT + threadIdx.x; q < nn;
       q += (unsigned long long)gridDim.x * GT) {
    const unsigned long long u = __ldg(a.ids + q);
    long long i, j, k;
    split_lin(u, nx, ny, i, j, k);
    const unsigned long long sxy = (unsigned long long)(nx * ny);
    uint32_t nb[6];
    int m = 0;
    unsigned long long cand[6];
    bool ok[6];
    cand[0] = u - sxy;  ok[0] = k > 0;
    cand[1] = u - nx;   ok[1] = j > 0;
    cand[2] = u - 1;    ok[2] = i > 0;
    cand[3] = u + 1;    ok[3] = i + 1 < nx;
    cand[4] = u + nx;   ok[4] = j + 1 < ny;
    cand[5] = u + sxy;  ok[5] = k + 1 < nz;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      if (!ok[c]) continue;
      const uint32_t idx = find_face(a, cand[c]);
      if (idx != kNone) nb[m++] = idx;
    }
    uint32_t* row = a.nbr + q * 6;
#pragma unroll
    for (int x = 0; x < 6; ++x) row[x] = x < m ? nb[x] : kNone;
    a.deg[q] = (uint8_t)m;
    a.comp[q] = (m > 0 && nb[0] < (uint32_t)q) ? nb[0] : (uint32_t)q;
  }
}

__device__ __forceinline__ uint32_t find_root(uint32_t* parent, uint32_t x) {
  uint32_t p = *((volatile uint32_t*)parent + x);
  while (p != x) {
    const uint32_t g = *((volatile uint32_t*)parent + p);
    if (g != p) *((volatile uint32_t*)parent + x) = g;  // halving: parents only decrease
    x = p;
    p = g;
  }
  return x;
}

// root without path writes: the flatten pass may not halve, since a halving
// store could overwrite a label that its owner has already set to the root
__device__ __forceinline__ uint32_t find_root_ro(const uint32_t* parent, uint32_t x) {
  uint32_t p = *((const volatile uint32_t*)parent + x);
  while (p != x) {
    x = p;
    p = *((const volatile uint32_t*)parent + x);
  }
  return x;
}

__global__ void __launch_bounds__(GT) link_kernel(GraphArgs a) {
  const unsigned long long nn = limit_n(a.n, a.n_dev);
  for (unsigned long long q = (unsigned long long)blockIdx.x * GT + threadIdx.x; q < nn;
       q += (unsigned long long)gridDim.x * GT) {
    const int m = a.deg[q];
    for (int x = 0; x < m; ++x) {
      const uint32_t b = a.nbr[q * a.stride + x];
      if (b <= (uint32_t)q) continue;
      int tries = 0;
      while (true) {
        uint32_t ra = find_root(a.comp, (uint32_t)q), rb = find_root(a.comp, b);
        if (ra == rb) break;
        if (ra > rb) {
          const uint32_t t = ra;
          ra = rb;
          rb = t;
        }
        if (atomicCAS(a.comp + rb, rb, ra) == rb) break;
        if (++tries >= kMaxTries) {
          atomicOr(a.status + 1, 1ull);
          break;
        }
      }
    }
  }
}

__global__ void __launch_bounds__(GT) flatten_kernel(GraphArgs a) {
  const unsigned long long nn = limit_n(a.n, a.n_dev);
  unsigned long long roots = 0;
  for (unsigned long long q = (unsigned long long)blockIdx.x * GT + threadIdx.x; q < nn;
       q += (unsigned long long)gridDim.x * GT) {
    const uint32_t r = find_root_ro(a.comp, (uint32_t)q);
    *((volatile uint32_t*)a.comp + q) = r;
    roots += (r == (uint32_t)q) ? 1ull : 0ull;
  }
#pragma unroll
  for (int d = 16; d; d >>= 1) roots += __shfl_down_sync(0xffffffffu, roots, d);
  if ((threadIdx.x & 31) == 0 && roots) atomicAdd(a.status, roots);
}

__global__ void graph_status_kernel(const unsigned long long* status, uint64_t* ncomp) {
  *ncomp = status[1] ? QTV_COUNT_TIMEOUT : status[0];
}

bool capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return false;
  return cs != cudaStreamCaptureStatusNone;
}

}  // namespace

int face_graph_launch(qtv_handle h, const qtv_grid& g, const uint64_t* face_ids, uint64_t n,
                      const uint64_t* n_dev, uint32_t* nbr, uint8_t* deg, uint32_t* comp,
                      uint64_t* ncomp, cudaStream_t st, bool nodes) {
  if (!h->graph) {
    if (capturing(st))
      return set_error(QTV_ERR_STATE, "graph workspace must be created outside stream capture");
    GraphWork* w = new GraphWork();
    const cudaError_t e =
        cudaMalloc(reinterpret_cast<void**>(&w->status), 2 * sizeof(unsigned long long));
    if (e != cudaSuccess) {
      delete w;
      return check_cuda(e, "cudaMalloc(graph status)");
    }
    h->graph = w;
  }
  GraphWork* w = h->graph;
  const long long R = (long long)g.ny * g.nz;
  if ((uint64_t)(R + 1) > w->rows_cap) {
    if (capturing(st))
      return set_error(QTV_ERR_STATE, "graph workspace must grow outside stream capture");
    cudaFree(w->rows);
    w->rows = nullptr;
    w->rows_cap = 0;
    const cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&w->rows), (R + 1) * sizeof(uint32_t));
    if (e != cudaSuccess) return check_cuda(e, "cudaMalloc(graph rows)");
    w->rows_cap = (uint64_t)(R + 1);
  }
  cudaError_t e = cudaMemsetAsync(w->status, 0, 2 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return check_cuda(e, "cudaMemsetAsync(graph status)");
  TraceScope ts(h, K_GRAPH, st);
  {
    long long blocks = (R + 1 + GT - 1) / GT;
    if (blocks > (long long)h->num_sms * 16) blocks = (long long)h->num_sms * 16;
    row_table_kernel<<<(int)blocks, GT, 0, st>>>(face_ids, n, n_dev, g.nx, R, nodes ? 0 : 2,
                                                 w->rows);
  }
  GraphArgs a;
  a.ids = face_ids;
  a.n = n;
  a.n_dev = n_dev;
  a.nx = g.nx;
  a.ny = g.ny;
  a.nz = g.nz;
  a.rows = w->rows;
  a.shift = nodes ? 0 : 2;
  a.stride = nodes ? 6 : 10;
  a.nbr = nbr;
  a.deg = deg;
  a.comp = comp;
  a.status = w->status;
  long long blocks = ((long long)n + GT - 1) / GT;
  if (blocks > (long long)h->num_sms * 16) blocks = (long long)h->num_sms * 16;
  if (blocks < 1) blocks = 1;
  if (nodes) node_adjacency_kernel<<<(int)blocks, GT, 0, st>>>(a);
  else adjacency_kernel<<<(int)blocks, GT, 0, st>>>(a);
  link_kernel<<<(int)blocks, GT, 0, st>>>(a);
  flatten_kernel<<<(int)blocks, GT, 0, st>>>(a);
  graph_status_kernel<<<1, 1, 0, st>>>(w->status, ncomp);
  e = cudaGetLastError();
  return check_cuda(e, "face graph launch");
}

}  // namespace qtv
