// refine.cu -- sample refinement of Sec. 3.3.3 ("Locating more accurate
// sample points") on the GPU: an estimate x0 of a core sample is moved to a
// minimizer of the density rho = |psi|^2 (Eq. 6) within the plane through x0
// perpendicular to the local core direction t, which the paper takes from the
// pseudo-vorticity t = grad Re psi x grad Im psi.
//
// Arithmetic, per sample (one thread; FP32):
//   - psi between nodes is the trilinear interpolant; rho and grad rho are
//     those of the interpolant within the cell floor(x) (cell index clamped
//     to [0, n - 2]);
//   - grad Re psi and grad Im psi at x0 are the central-difference node
//     gradients (one-sided on the boundary, 0 along an axis of one node),
//     interpolated trilinearly; t is their cross product, normalized;
//   - descent on g = grad rho - (grad rho . t) t: each step starts at
//     alpha = 2 rho / |g|^2 (the exact step for a round bowl whose minimum is
//     0) and halves alpha until rho(x - alpha g) <= rho(x) - 1e-4 alpha |g|^2
//     with the new point in the grid and in the box |x - x0|_inf <= 1 (a step
//     leaving either is rejected, not projected); it stops, converged, when
//     no step of length >= tol decreases rho that way, or after max_iter
//     accepted steps.
// Positions are carried as an integer base (the cell of x0) plus an FP32
// offset, so steps far below the FP32 spacing of absolute coordinates still
// move the point.  Warps are persistent and each lane takes a new sample when
// its search ends (the number of steps varies from 0 to max_iter).
#include <cstdio>

#include "qtv_internal.cuh"

namespace qtv {
namespace {

constexpr int REF_THREADS = 128;

struct RefArgs {
  const float2* psi;
  int nx, ny, nz;
  float h, ox, oy, oz;
  const float* xyz0;          // world positions [n][3], or null
  const uint64_t* face_ids;   // faces whose centres are x0, or null
  unsigned long long n;
  const uint64_t* n_dev;
  int max_iter;
  float tol;
  float* xyz;
  float* rho;
  float* tangent;
  float* detj;
  int32_t* iters;
  uint8_t* flags;
};

struct Field {
  const float2* psi;
  int n[3];
  __device__ __forceinline__ float2 at(int i, int j, int k) const {
    return __ldg(psi + ((long long)k * n[1] + j) * n[0] + i);
  }
};

// cell and fraction of base + off along an axis of m nodes
__device__ __forceinline__ void cell_frac(int base, float off, int m, int& c, float& f) {
  const float fl = floorf(off);
  c = base + (int)fl;
  f = off - fl;
  const int hi = max(m - 2, 0);
  if (c > hi) {
    f += (float)(c - hi);
    c = hi;
  }
  if (c < 0) {
    f += (float)c;
    c = 0;
  }
}

// trilinear psi at the point (cells c, fractions f) and its partial derivatives
__device__ __forceinline__ float2 tri_eval(const Field& F, const int c[3], const float f[3],
                                           float2 d[3]) {
  float2 acc = make_float2(0.f, 0.f);
  d[0] = d[1] = d[2] = make_float2(0.f, 0.f);
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    int idx[3];
    float w[3], s[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int bit = (q >> a) & 1;
      idx[a] = c[a] + bit < F.n[a] ? c[a] + bit : c[a];
      w[a] = bit ? f[a] : 1.f - f[a];
      s[a] = bit ? 1.f : -1.f;
    }
    const float2 v = F.at(idx[0], idx[1], idx[2]);
    const float wt = w[0] * w[1] * w[2];
    acc.x = fmaf(wt, v.x, acc.x);
    acc.y = fmaf(wt, v.y, acc.y);
    const float dd[3] = {s[0] * w[1] * w[2], w[0] * s[1] * w[2], w[0] * w[1] * s[2]};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      d[a].x = fmaf(dd[a], v.x, d[a].x);
      d[a].y = fmaf(dd[a], v.y, d[a].y);
    }
  }
  return acc;
}

// central-difference gradient of psi at node (i,j,k) along axis a
__device__ __forceinline__ float2 node_grad(const Field& F, int i, int j, int k, int a) {
  int p[3] = {i, j, k}, q[3] = {i, j, k};
  const int m = F.n[a];
  if (m < 2) return make_float2(0.f, 0.f);
  float s = 0.5f;
  if (p[a] == 0) {
    q[a] = 1;
    s = 1.f;
  } else if (p[a] == m - 1) {
    p[a] = m - 2;
    s = 1.f;
  } else {
    p[a] -= 1;
    q[a] += 1;
  }
  const float2 lo = F.at(p[0], p[1], p[2]), hi = F.at(q[0], q[1], q[2]);
  return make_float2(s * (hi.x - lo.x), s * (hi.y - lo.y));
}

struct Pos {
  int base[3];    // integer base (cell of x0)
  float off[3];   // offset from the base
};

__device__ __forceinline__ bool pos_inside(const Pos& P, const int n[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float v = (float)P.base[a] + P.off[a];
    if (!(P.off[a] >= -(float)P.base[a] && v <= (float)(n[a] - 1))) return false;
  }
  return true;
}

// The eight corner values of the cell last evaluated: a search rarely
// leaves its cell, so most evaluations read no memory.
struct CellCache {
  int c[3];
  float2 v[8];
};

// rho and grad rho at P: trilinear psi and its derivatives from the corners
// in the same order and arithmetic as tri_eval
__device__ __forceinline__ float rho_at(const Field& F, const Pos& P, float g[3], CellCache& C) {
  int c[3];
  float f[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) cell_frac(P.base[a], P.off[a], F.n[a], c[a], f[a]);
  if (c[0] != C.c[0] || c[1] != C.c[1] || c[2] != C.c[2]) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      int idx[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int bit = (q >> a) & 1;
        idx[a] = c[a] + bit < F.n[a] ? c[a] + bit : c[a];
      }
      C.v[q] = F.at(idx[0], idx[1], idx[2]);
    }
    C.c[0] = c[0];
    C.c[1] = c[1];
    C.c[2] = c[2];
  }
  float2 v = make_float2(0.f, 0.f);
  float2 d[3];
  d[0] = d[1] = d[2] = make_float2(0.f, 0.f);
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    float w[3], s[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int bit = (q >> a) & 1;
      w[a] = bit ? f[a] : 1.f - f[a];
      s[a] = bit ? 1.f : -1.f;
    }
    const float2 u = C.v[q];
    const float wt = w[0] * w[1] * w[2];
    v.x = fmaf(wt, u.x, v.x);
    v.y = fmaf(wt, u.y, v.y);
    const float dd[3] = {s[0] * w[1] * w[2], w[0] * s[1] * w[2], w[0] * w[1] * s[2]};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      d[a].x = fmaf(dd[a], u.x, d[a].x);
      d[a].y = fmaf(dd[a], u.y, d[a].y);
    }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) g[a] = 2.f * fmaf(v.x, d[a].x, v.y * d[a].y);
  return fmaf(v.x, v.x, v.y * v.y);
}

// state of one sample's search
struct RState {
  Pos P0, P;
  float t[3];
  float rho;
  float grad[3];
  int it;
  uint8_t fl;
  unsigned long long qi;
  CellCache cache;
};

// x0, tangent, rho and grad rho at x0; true when the descent is to run
__device__ __forceinline__ bool ref_init(const RefArgs& A, const Field& F, unsigned long long qi,
                                         RState& S) {
  const float org[3] = {A.ox, A.oy, A.oz};
  S.qi = qi;
  S.it = 0;
  S.cache.c[0] = -1;  // no cell loaded
  S.t[0] = S.t[1] = S.t[2] = 0.f;
  S.rho = __int_as_float(0x7fc00000);
  bool in0 = true;
  if (A.face_ids) {
    const uint64_t id = A.face_ids[qi];
    const int o = (int)(id & 3u);
    const unsigned long long lin = id >> 2;
    long long i, j, k;
    split_lin(lin, A.nx, A.ny, i, j, k);
    S.P0.base[0] = (int)i;
    S.P0.base[1] = (int)j;
    S.P0.base[2] = (int)k;
    // face centre: half a cell along the two in-plane axes
    S.P0.off[0] = (o == 0 || o == 2) ? 0.5f : 0.f;
    S.P0.off[1] = (o == 0 || o == 1) ? 0.5f : 0.f;
    S.P0.off[2] = (o == 1 || o == 2) ? 0.5f : 0.f;
    in0 = pos_inside(S.P0, F.n);
  } else {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float g = (__ldg(A.xyz0 + 3 * qi + a) - org[a]) / A.h;
      const float fl = floorf(g);
      in0 = in0 && g >= 0.f && g <= (float)(F.n[a] - 1);
      S.P0.base[a] = in0 ? (int)fl : 0;
      S.P0.off[a] = in0 ? g - fl : g;
    }
  }
  S.P = S.P0;
  if (!in0) {
    S.fl = QTV_REFINE_NO_TANGENT;
    return false;
  }
  // pseudo-vorticity at x0
  int c[3];
  float f[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) cell_frac(S.P0.base[a], S.P0.off[a], F.n[a], c[a], f[a]);
  float gr[3] = {0.f, 0.f, 0.f}, gi[3] = {0.f, 0.f, 0.f};
  for (int q = 0; q < 8; ++q) {
    int idx[3];
    float wt = 1.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int bit = (q >> a) & 1;
      idx[a] = c[a] + bit < F.n[a] ? c[a] + bit : c[a];
      wt *= bit ? f[a] : 1.f - f[a];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float2 g = node_grad(F, idx[0], idx[1], idx[2], a);
      gr[a] = fmaf(wt, g.x, gr[a]);
      gi[a] = fmaf(wt, g.y, gi[a]);
    }
  }
  float t[3];
  t[0] = gr[1] * gi[2] - gr[2] * gi[1];
  t[1] = gr[2] * gi[0] - gr[0] * gi[2];
  t[2] = gr[0] * gi[1] - gr[1] * gi[0];
  const float tn = sqrtf(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
  S.rho = rho_at(F, S.P, S.grad, S.cache);
  if (!(tn > 0.f) || !(tn <= 3.402823466e38f)) {
    S.fl = QTV_REFINE_NO_TANGENT;
    return false;
  }
  S.t[0] = t[0] / tn;
  S.t[1] = t[1] / tn;
  S.t[2] = t[2] / tn;
  S.fl = QTV_REFINE_MAX_ITER;
  return true;
}

// one accepted step, or the decision to stop; true when the sample is done
__device__ __forceinline__ bool ref_step(const RefArgs& A, const Field& F, RState& S) {
  if (S.it >= A.max_iter) return true;  // flag stays QTV_REFINE_MAX_ITER
  const float gt = S.grad[0] * S.t[0] + S.grad[1] * S.t[1] + S.grad[2] * S.t[2];
  float g[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) g[a] = S.grad[a] - gt * S.t[a];
  const float gg = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
  if (!(gg > 0.f)) {
    S.fl = QTV_REFINE_CONVERGED;
    return true;
  }
  const float gn = sqrtf(gg);
  float alpha = 2.f * S.rho / gg;
  Pos Pn;
  float rn = 0.f, gnext[3];
  bool accepted = false;
  while (alpha * gn >= A.tol) {
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      Pn.base[a] = S.P.base[a];
      Pn.off[a] = S.P.off[a] - alpha * g[a];
      // box around x0 (same base as x0)
      ok = ok && fabsf(Pn.off[a] - S.P0.off[a]) <= 1.f;
    }
    if (ok && pos_inside(Pn, F.n)) {
      rn = rho_at(F, Pn, gnext, S.cache);
      if (rn <= S.rho - 1e-4f * alpha * gg) {
        accepted = true;
        break;
      }
    }
    alpha *= 0.5f;
  }
  if (!accepted) {
    S.fl = QTV_REFINE_CONVERGED;
    return true;
  }
  ++S.it;
  S.P = Pn;
  S.rho = rn;
  S.grad[0] = gnext[0];
  S.grad[1] = gnext[1];
  S.grad[2] = gnext[2];
  return false;
}

// conditioning at the result and the outputs of the sample
__device__ __forceinline__ void ref_finish(const RefArgs& A, const Field& F, const RState& S) {
  float dj = 0.f;
  if (!(S.fl & QTV_REFINE_NO_TANGENT)) {
    // in-plane Jacobian of psi at the result: basis e1 = normalize(t x a), a
    // the axis least aligned with t; e2 = t x e1
    const float t[3] = {S.t[0], S.t[1], S.t[2]};
    int m = 0;
    float am = fabsf(t[0]);
    if (fabsf(t[1]) < am) {
      m = 1;
      am = fabsf(t[1]);
    }
    if (fabsf(t[2]) < am) m = 2;
    const float ax[3] = {m == 0 ? 1.f : 0.f, m == 1 ? 1.f : 0.f, m == 2 ? 1.f : 0.f};
    float e1[3] = {t[1] * ax[2] - t[2] * ax[1], t[2] * ax[0] - t[0] * ax[2],
                   t[0] * ax[1] - t[1] * ax[0]};
    const float en = sqrtf(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
    e1[0] /= en;
    e1[1] /= en;
    e1[2] /= en;
    const float e2[3] = {t[1] * e1[2] - t[2] * e1[1], t[2] * e1[0] - t[0] * e1[2],
                         t[0] * e1[1] - t[1] * e1[0]};
    int cc[3];
    float ff[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) cell_frac(S.P.base[a], S.P.off[a], F.n[a], cc[a], ff[a]);
    float2 d[3];
    (void)tri_eval(F, cc, ff, d);
    float a1r = 0.f, a1i = 0.f, a2r = 0.f, a2i = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      a1r = fmaf(d[a].x, e1[a], a1r);
      a1i = fmaf(d[a].y, e1[a], a1i);
      a2r = fmaf(d[a].x, e2[a], a2r);
      a2i = fmaf(d[a].y, e2[a], a2i);
    }
    dj = a1r * a2i - a2r * a1i;
  }
  const float org[3] = {A.ox, A.oy, A.oz};
  const unsigned long long qi = S.qi;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    A.xyz[3 * qi + a] = org[a] + A.h * ((float)S.P.base[a] + S.P.off[a]);
    if (A.tangent) A.tangent[3 * qi + a] = S.t[a];
  }
  if (A.rho) A.rho[qi] = S.rho;
  if (A.detj) A.detj[qi] = dj;
  if (A.iters) A.iters[qi] = S.it;
  A.flags[qi] = S.fl;
}

// Persistent warps; each lane keeps one sample.  A lane whose search ends
// waits until kRefill lanes of its warp have (or none is searching); then
// those lanes write their results and take the next samples from the counter
// together (one atomic per warp and refill), so the long set-up and result
// code runs with many lanes at once while searches of very different lengths
// keep the warp busy.  Each sample is computed exactly as alone.
constexpr int kRefill = 12;

__global__ void __launch_bounds__(REF_THREADS, 6) refine_kernel(RefArgs A,
                                                             unsigned long long* counter) {
  unsigned long long nn = A.n;
  if (A.n_dev) {
    const unsigned long long d = *A.n_dev;
    if (d < nn) nn = d;
  }
  Field F;
  F.psi = A.psi;
  F.n[0] = A.nx;
  F.n[1] = A.ny;
  F.n[2] = A.nz;
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  RState S;
  // active: searching; done: search ended, result not yet written;
  // drained: no sample left for this lane
  bool active = false, done = false, drained = false;
  while (true) {
    const unsigned idle = __ballot_sync(0xffffffffu, !active && !drained);
    const unsigned busy = __ballot_sync(0xffffffffu, active);
    if (idle && (__popc(idle) >= kRefill || busy == 0u)) {
      if (done) {
        ref_finish(A, F, S);
        done = false;
      }
      const int leader = __ffs(idle) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(counter, (unsigned long long)__popc(idle));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (!active && !drained) {
        const unsigned long long qi = base + (unsigned long long)__popc(idle & lt);
        if (qi < nn) {
          if (ref_init(A, F, qi, S)) active = true;
          else ref_finish(A, F, S);
        } else {
          drained = true;
        }
      }
    }
    if (!__any_sync(0xffffffffu, active || done || !drained)) break;
    if (active && ref_step(A, F, S)) {
      active = false;
      done = true;
    }
  }
}

}  // namespace

int refine_launch(qtv_handle h, const qtv_grid& g, const float2* psi, const float* xyz0,
                  const uint64_t* face_ids, uint64_t n, const uint64_t* n_dev, int max_iter,
                  float tol, float* xyz, float* rho, float* tangent, float* detj, int32_t* iters,
                  uint8_t* flags, cudaStream_t st) {
  if (n == 0) return QTV_OK;
  RefArgs a;
  a.psi = psi;
  a.nx = g.nx;
  a.ny = g.ny;
  a.nz = g.nz;
  a.h = g.h;
  a.ox = g.origin[0];
  a.oy = g.origin[1];
  a.oz = g.origin[2];
  a.xyz0 = xyz0;
  a.face_ids = face_ids;
  a.n = n;
  a.n_dev = n_dev;
  a.max_iter = max_iter;
  a.tol = tol;
  a.xyz = xyz;
  a.rho = rho;
  a.tangent = tangent;
  a.detj = detj;
  a.iters = iters;
  a.flags = flags;
  if (!h->refine_counter) {
    const cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&h->refine_counter),
                                     sizeof(unsigned long long));
    if (e != cudaSuccess) {
      h->refine_counter = nullptr;
      return check_cuda(e, "cudaMalloc(refine counter)");
    }
  }
  // persistent: as many blocks as fit at once, fewer for short lists
  static int per_sm = 0;
  if (per_sm == 0) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, refine_kernel, REF_THREADS, 0) !=
            cudaSuccess ||
        b < 1)
      b = 1;
    per_sm = b;
  }
  long long blocks = ((long long)n + REF_THREADS - 1) / REF_THREADS;
  const long long maxb = (long long)h->num_sms * per_sm;
  if (blocks > maxb) blocks = maxb;
  TraceScope ts(h, K_REFINE, st);
  cudaError_t e = cudaMemsetAsync(h->refine_counter, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return check_cuda(e, "cudaMemsetAsync(refine counter)");
  refine_kernel<<<(int)blocks, REF_THREADS, 0, st>>>(a, h->refine_counter);
  e = cudaGetLastError();
  return check_cuda(e, "refine_kernel launch");
}

}  // namespace qtv
