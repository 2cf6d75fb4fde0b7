// reduce.cu -- box-mean reduction of a sample graph (Sec. 3.3.1-3.3.2) on the
// GPU, in an order-independent lattice form.
//
// The paper walks the graph: a box of side d centred on the current node takes
// the unprocessed nodes it reaches inside the box, they collapse to their mean
// with their external edges inherited, the walk moves on to an unprocessed
// neighbour, and whole passes repeat until positions settle (2 to 5 passes).
// That walk is sequential.  Here every pass is data-parallel instead: a
// lattice of boxes of side D covers space (shifted by D/2 in every axis on
// odd passes, so that no lattice boundary stays fixed), the nodes of one box
// that are connected through edges inside the box form one cluster, and each
// cluster collapses to one node at the mean of its members, keeping every
// edge that leaves it.  Passes repeat until one pass of each lattice merges
// nothing; then no further pass can change anything.
//
// Exactness.  Positions are held as 64-bit integers in units of 2^-32 of the
// input's length unit (x 2^32, exact in FP64 for an FP32 x, rounded to the
// nearest integer with ties to even; negative positions too);
// box keys are floor divisions of integers and a mean is the rounded integer
// quotient floor((sum + floor(c/2)) / c), so sums and means do not depend on the order in
// which threads add, and the result is the same on every run.
//
// Representation.  The graph is never rebuilt.  Each input node keeps the
// label of its current cluster (the lowest input index in it), and a cluster
// is represented by that node, which holds the cluster's position.  A pass
// keys the representatives, links (union-find, as in graph.cu: the larger
// root goes under the smaller with a CAS, so roots are cluster minima) every
// input edge whose ends lie in different clusters with equal keys, then
// relabels and averages.  A cluster's adjacency is the set of input edges
// that leave it, exactly the inherited connectivity of the paper's collapse.
//
// Launches: one set-up kernel, then for each of max_passes passes a fixed
// sequence of four kernels and a one-thread control kernel; once the control
// kernel has seen two quiet passes every later kernel returns at once, so the
// call synchronises nothing and can be captured into a CUDA graph.
#include "qtv_internal.cuh"

namespace qtv {

struct ReduceWork {
  long long* sum = nullptr;        // [cap][3] cluster sums of one pass (two's complement)
  unsigned int* cnt = nullptr;     // [cap] members of a new cluster
  unsigned long long* key = nullptr;  // [cap] packed box key of a representative
  unsigned int* par = nullptr;     // [cap] union-find parents of one pass
  unsigned int* nl = nullptr;      // [cap] new label of a representative
  unsigned long long* status = nullptr;  // [0] merges, [1] quiet, [2] passes, [3] done, [4] retry overflow
  uint64_t cap = 0;
};

void reduce_work_free(ReduceWork* w) {
  if (!w) return;
  cudaFree(w->sum);
  cudaFree(w->cnt);
  cudaFree(w->key);
  cudaFree(w->par);
  cudaFree(w->nl);
  cudaFree(w->status);
  delete w;
}

namespace {

constexpr int RT = 256;
constexpr int kMaxTries = 1 << 20;     // CAS retries of one link before giving up
constexpr double kFix = 4294967296.0;  // fixed-point units per length unit

struct ReduceArgs {
  unsigned long long n;
  const uint64_t* n_dev;
  const uint32_t* nbr;
  const uint8_t* deg;
  int stride;
  long long D;          // box side in fixed point
  int max_passes;
  uint32_t* lab;        // [n] cluster label of every node
  long long* q;         // [n][3] positions (valid at representatives)
  long long* sum;
  unsigned int* cnt;
  unsigned long long* key;
  unsigned int* par;
  unsigned int* nl;
  unsigned long long* status;
};

__device__ __forceinline__ unsigned long long limit_n(unsigned long long n, const uint64_t* n_dev) {
  if (n_dev) {
    const unsigned long long d = *n_dev;
    if (d < n) n = d;
  }
  return n;
}

__device__ __forceinline__ bool done(const ReduceArgs& a) {
  return *((const volatile unsigned long long*)a.status + 3) != 0ull;
}

// floor(x / d) for d > 0
__device__ __forceinline__ long long floor_div(long long x, long long d) {
  const long long qt = x / d;
  return (x % d != 0 && x < 0) ? qt - 1 : qt;
}

// 21 bits per axis (two's complement), enough for any grid below 2^20 boxes
__device__ __forceinline__ unsigned long long pack_key(long long kx, long long ky, long long kz) {
  const unsigned long long m = (1ull << 21) - 1ull;
  return ((unsigned long long)kx & m) | (((unsigned long long)ky & m) << 21) |
         (((unsigned long long)kz & m) << 42);
}

__global__ void __launch_bounds__(RT) reduce_init_kernel(ReduceArgs a, const float* __restrict__ xyz) {
  const unsigned long long nn = limit_n(a.n, a.n_dev);
  if (blockIdx.x == 0 && threadIdx.x < 5) a.status[threadIdx.x] = 0ull;
  for (unsigned long long u = (unsigned long long)blockIdx.x * RT + threadIdx.x; u < nn;
       u += (unsigned long long)gridDim.x * RT) {
    a.lab[u] = (uint32_t)u;
#pragma unroll
    for (int c = 0; c < 3; ++c) a.q[3 * u + c] = __double2ll_rn((double)xyz[3 * u + c] * kFix);
  }
}

// representatives: box key of this pass, fresh union-find parent, zero sums
__global__ void __launch_bounds__(RT) reduce_key_kernel(ReduceArgs a) {
  if (done(a)) return;
  const unsigned long long nn = limit_n(a.n, a.n_dev);
  const long long off = (a.status[2] & 1ull) ? a.D / 2 : 0;
  for (unsigned long long u = (unsigned long long)blockIdx.x * RT + threadIdx.x; u < nn;
       u += (unsigned long long)gridDim.x * RT) {
    if (a.lab[u] != (uint32_t)u) continue;
    a.key[u] = pack_key(floor_div(a.q[3 * u] - off, a.D), floor_div(a.q[3 * u + 1] - off, a.D),
                        floor_div(a.q[3 * u + 2] - off, a.D));
    a.par[u] = (uint32_t)u;
    a.sum[3 * u] = a.sum[3 * u + 1] = a.sum[3 * u + 2] = 0;
    a.cnt[u] = 0u;
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

__device__ __forceinline__ uint32_t find_root_ro(const uint32_t* parent, uint32_t x) {
  uint32_t p = *((const volatile uint32_t*)parent + x);
  while (p != x) {
    x = p;
    p = *((const volatile uint32_t*)parent + x);
  }
  return x;
}

// every input edge (u, v), u < v, between two clusters of equal key
__global__ void __launch_bounds__(RT) reduce_link_kernel(ReduceArgs a) {
  if (done(a)) return;
  const unsigned long long nn = limit_n(a.n, a.n_dev);
  for (unsigned long long u = (unsigned long long)blockIdx.x * RT + threadIdx.x; u < nn;
       u += (unsigned long long)gridDim.x * RT) {
    const int m = a.deg[u];
    const uint32_t lu = a.lab[u];
    const unsigned long long ku = a.key[lu];
    for (int x = 0; x < m; ++x) {
      const uint32_t v = a.nbr[u * (unsigned long long)a.stride + x];
      if (v <= (uint32_t)u || v >= nn) continue;
      const uint32_t lv = a.lab[v];
      if (lv == lu || a.key[lv] != ku) continue;
      int tries = 0;
      while (true) {
        uint32_t ra = find_root(a.par, lu), rb = find_root(a.par, lv);
        if (ra == rb) break;
        if (ra > rb) {
          const uint32_t t = ra;
          ra = rb;
          rb = t;
        }
        if (atomicCAS(a.par + rb, rb, ra) == rb) break;
        if (++tries >= kMaxTries) {
          atomicOr(a.status + 4, 1ull);
          break;
        }
      }
    }
  }
}

// representatives: new label (the root: lowest index of the merged cluster),
// position added to the new cluster's sum
__global__ void __launch_bounds__(RT) reduce_merge_kernel(ReduceArgs a) {
  if (done(a)) return;
  const unsigned long long nn = limit_n(a.n, a.n_dev);
  unsigned long long merges = 0;
  for (unsigned long long u = (unsigned long long)blockIdx.x * RT + threadIdx.x; u < nn;
       u += (unsigned long long)gridDim.x * RT) {
    if (a.lab[u] != (uint32_t)u) continue;
    const uint32_t r = find_root_ro(a.par, (uint32_t)u);
    a.nl[u] = r;
    merges += (r != (uint32_t)u) ? 1ull : 0ull;
#pragma unroll
    for (int c = 0; c < 3; ++c)
      atomicAdd(reinterpret_cast<unsigned long long*>(a.sum + 3 * r + c),
                (unsigned long long)a.q[3 * u + c]);
    atomicAdd(a.cnt + r, 1u);
  }
#pragma unroll
  for (int d = 16; d; d >>= 1) merges += __shfl_down_sync(0xffffffffu, merges, d);
  if ((threadIdx.x & 31) == 0 && merges) atomicAdd(a.status, merges);
}

// every node: its cluster's new label; new representatives: the rounded mean
__global__ void __launch_bounds__(RT) reduce_relabel_kernel(ReduceArgs a) {
  if (done(a)) return;
  const unsigned long long nn = limit_n(a.n, a.n_dev);
  for (unsigned long long u = (unsigned long long)blockIdx.x * RT + threadIdx.x; u < nn;
       u += (unsigned long long)gridDim.x * RT) {
    const uint32_t l = a.lab[u];
    const uint32_t r = a.nl[l];
    a.lab[u] = r;
    if (l == (uint32_t)u && r == (uint32_t)u) {
      const long long c = (long long)a.cnt[u];
#pragma unroll
      for (int k = 0; k < 3; ++k) a.q[3 * u + k] = floor_div(a.sum[3 * u + k] + c / 2, c);
    }
  }
}

// one thread: count the pass, stop after two quiet passes or max_passes
__global__ void reduce_control_kernel(ReduceArgs a) {
  if (done(a)) return;
  const unsigned long long merges = a.status[0];
  a.status[0] = 0ull;
  const unsigned long long passes = a.status[2] + 1ull;
  const unsigned long long quiet = merges ? 0ull : a.status[1] + 1ull;
  a.status[1] = quiet;
  a.status[2] = passes;
  if (quiet >= 2ull || passes >= (unsigned long long)a.max_passes) a.status[3] = 1ull;
}

// representatives: positions back to the length unit (exact in FP64);
// counts = (clusters, passes)
__global__ void __launch_bounds__(RT) reduce_out_kernel(ReduceArgs a, double* __restrict__ out,
                                                        uint64_t* counts) {
  const unsigned long long nn = limit_n(a.n, a.n_dev);
  unsigned long long reps = 0;
  for (unsigned long long u = (unsigned long long)blockIdx.x * RT + threadIdx.x; u < nn;
       u += (unsigned long long)gridDim.x * RT) {
    if (a.lab[u] != (uint32_t)u) continue;
    ++reps;
#pragma unroll
    for (int c = 0; c < 3; ++c) out[3 * u + c] = (double)a.q[3 * u + c] / kFix;
  }
#pragma unroll
  for (int d = 16; d; d >>= 1) reps += __shfl_down_sync(0xffffffffu, reps, d);
  if ((threadIdx.x & 31) == 0 && reps) atomicAdd(reinterpret_cast<unsigned long long*>(counts), reps);
}

__global__ void reduce_counts_kernel(const ReduceArgs a, uint64_t* counts) {
  counts[1] = a.status[2];
  if (a.status[4]) counts[0] = QTV_COUNT_TIMEOUT;
}

bool capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return false;
  return cs != cudaStreamCaptureStatusNone;
}

}  // namespace

int box_reduce_launch(qtv_handle h, uint64_t n, const uint64_t* n_dev, const uint32_t* nbr,
                      const uint8_t* deg, int stride, const float* xyz, float box, int max_passes,
                      uint32_t* label, double* out_xyz, uint64_t* counts, cudaStream_t st) {
  if (!h->reduce || h->reduce->cap < n) {
    if (capturing(st))
      return set_error(QTV_ERR_STATE, "reduction workspace must grow outside stream capture");
    reduce_work_free(h->reduce);
    h->reduce = nullptr;
    ReduceWork* w = new ReduceWork();
    const uint64_t c = n > 0 ? n : 1;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&w->sum), c * 3 * sizeof(long long));
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&w->cnt), c * sizeof(unsigned int));
    if (e == cudaSuccess)
      e = cudaMalloc(reinterpret_cast<void**>(&w->key), c * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&w->par), c * sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&w->nl), c * sizeof(unsigned int));
    if (e == cudaSuccess)
      e = cudaMalloc(reinterpret_cast<void**>(&w->status), 8 * sizeof(unsigned long long));
    if (e != cudaSuccess) {
      reduce_work_free(w);
      return check_cuda(e, "cudaMalloc(reduction workspace)");
    }
    w->cap = c;
    h->reduce = w;
  }
  ReduceWork* w = h->reduce;
  cudaError_t e = cudaMemsetAsync(counts, 0, 2 * sizeof(uint64_t), st);
  if (e != cudaSuccess) return check_cuda(e, "cudaMemsetAsync(reduction counts)");
  if (n == 0) return QTV_OK;
  ReduceArgs a;
  a.n = n;
  a.n_dev = n_dev;
  a.nbr = nbr;
  a.deg = deg;
  a.stride = stride;
  a.D = (long long)((double)box * kFix);
  a.max_passes = max_passes;
  a.lab = label;
  // positions live in the output array as fixed-point integers until the end
  a.q = reinterpret_cast<long long*>(out_xyz);
  a.sum = w->sum;
  a.cnt = w->cnt;
  a.key = w->key;
  a.par = w->par;
  a.nl = w->nl;
  a.status = w->status;
  long long blocks = ((long long)n + RT - 1) / RT;
  if (blocks > (long long)h->num_sms * 8) blocks = (long long)h->num_sms * 8;
  TraceScope ts(h, K_REDUCE, st);
  reduce_init_kernel<<<(int)blocks, RT, 0, st>>>(a, xyz);
  for (int p = 0; p < max_passes; ++p) {
    reduce_key_kernel<<<(int)blocks, RT, 0, st>>>(a);
    reduce_link_kernel<<<(int)blocks, RT, 0, st>>>(a);
    reduce_merge_kernel<<<(int)blocks, RT, 0, st>>>(a);
    reduce_relabel_kernel<<<(int)blocks, RT, 0, st>>>(a);
    reduce_control_kernel<<<1, 1, 0, st>>>(a);
  }
  reduce_out_kernel<<<(int)blocks, RT, 0, st>>>(a, out_xyz, counts);
  reduce_counts_kernel<<<1, 1, 0, st>>>(a, counts);
  e = cudaGetLastError();
  return check_cuda(e, "box reduction launch");
}

}  // namespace qtv
